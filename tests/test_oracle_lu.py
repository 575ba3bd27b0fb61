"""Pins of the oracle's LU with a symmetric pattern (pivots looked for only
within diagonal blocks) and its solve, independent of its C code.

* No pivoting on strictly column diagonally dominant inputs: scipy's
  partially pivoted LU (LAPACK getrf) then swaps nothing, and its unit-lower
  L_s / upper U_s relate to the Crout form by L = L_s diag(U_s) and
  U = diag(U_s)^{-1} U_s.
* One window holding every row: the oracle is plain partial pivoting and
  equals scipy's P, L, U (the row order exactly).
* Block-diagonal inputs whose blocks are the windows: each block equals
  scipy's partial pivoting of that block.
* Windows cut from a partition: Pi C = L U to rounding, Pi moves rows only
  inside their windows, and every multiplier of a window is at most 1 in
  magnitude (|L_ij| <= |L_jj|).
* SPD inputs without pivoting: L = G diag(G), U = diag(G)^{-1} G^T for
  numpy's Cholesky C = G G^T.
* The nonsymmetric tridiagonal tridiag(a, 2, c): the Thomas recurrence
  d_1 = 2, d_{k+1} = 2 - a c / d_k gives L_kk = d_k, L_{k+1,k} = a and
  U_{k,k+1} = c / d_k.
* A matrix with zero diagonal entries (gen.pivot_nodes_3d): no pivoting
  stops at column 0; pivoting within the nodes recovers the planted row
  order exactly; manufactured solutions."""
import numpy as np
import pytest
import scipy.linalg

import gen


def dense(rp, ci, v):
    n = len(rp) - 1
    A = np.zeros((n, n))
    np.add.at(A, (np.repeat(np.arange(n), np.diff(rp)), ci), v)
    return A


def crout(L_s, U_s):
    d = np.diag(U_s)
    return L_s * d[None, :], U_s / d[:, None]


@pytest.mark.parametrize("seed", range(3))
def test_no_pivoting_matches_scipy_on_column_dominant(orc, seed):
    n = [40, 75, 120][seed]
    rp, ci, v = gen.random_nonsym(n, 0.08, seed + 10, dominance=2.0)
    perm = gen.random_perm(n, seed)
    F = orc.lu_dense(rp, ci, v, perm)
    assert F.bad_col == -1
    C = dense(rp, ci, v)[np.ix_(perm, perm)]
    P, L_s, U_s = scipy.linalg.lu(C)
    assert np.array_equal(P, np.eye(n))  # dominance: getrf swaps nothing
    L, U = crout(L_s, U_s)
    assert np.array_equal(F.rho, np.arange(n))
    assert np.allclose(F.L, L, rtol=1e-12, atol=1e-13)
    assert np.allclose(F.U, U, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("seed", range(3))
def test_one_window_is_partial_pivoting(orc, seed):
    n = [30, 55, 80][seed]
    rp, ci, v = gen.random_nonsym(n, 0.3, seed + 20, dominance=0.0)
    F = orc.lu_dense(rp, ci, v, None, wend=np.full(n, n))
    assert F.bad_col == -1
    P, L_s, U_s = scipy.linalg.lu(dense(rp, ci, v))
    L, U = crout(L_s, U_s)
    assert np.array_equal(F.rho, np.argmax(P, axis=0))  # C = P L U: row i of P^T C
    assert np.allclose(F.L, L, rtol=1e-10, atol=1e-12)
    assert np.allclose(F.U, U, rtol=1e-10, atol=1e-12)


def test_block_diagonal_windows_are_per_block_partial_pivoting(orc):
    sizes = [7, 12, 5, 9]
    blocks = [dense(*gen.random_nonsym(m, 0.5, 30 + i, dominance=0.0)) for i, m in
              enumerate(sizes)]
    A = scipy.linalg.block_diag(*blocks)
    n = len(A)
    rows, cols = np.nonzero(A)
    rp = np.zeros(n + 1, dtype=np.int64)
    rp[1:] = np.cumsum(np.bincount(rows, minlength=n))
    starts = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    F = orc.lu_dense(rp, cols.astype(np.int32), A[rows, cols], None,
                     wend=orc.pivot_windows(starts, n, nb=64))
    assert F.bad_col == -1
    for b0, B in zip(starts, blocks):
        m = len(B)
        P, L_s, U_s = scipy.linalg.lu(B)
        L, U = crout(L_s, U_s)
        sl = slice(b0, b0 + m)
        assert np.array_equal(F.rho[sl] - b0, np.argmax(P, axis=0))
        assert np.allclose(F.L[sl, sl], L, rtol=1e-10, atol=1e-12)
        assert np.allclose(F.U[sl, sl], U, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("nb,seed", [(3, 0), (4, 1), (8, 2), (64, 3)])
def test_windowed_pivoting_invariants(orc, nb, seed):
    rp, ci, v = gen.nonsym_3d(5, 4, 4, wind=3.0, small_diag=0.4, seed=seed)
    n = len(rp) - 1
    perm = gen.nd_perm((5, 4, 4))
    so = orc.symbolic(rp, ci, perm)
    wend = orc.pivot_windows(so["sup_ptr"][:-1], n, nb=nb)
    F = orc.lu_dense(rp, ci, v, perm, wend=wend)
    assert F.bad_col == -1
    C = dense(rp, ci, v)[np.ix_(perm, perm)]
    R = C[F.rho] - F.L @ F.U
    assert np.max(np.abs(R)) <= 1e-12 * np.max(np.abs(C)) * max(1.0, np.max(np.abs(F.L)))
    assert sorted(F.rho) == list(range(n))
    for i in range(n):  # rows stay inside their window
        w0 = i
        while w0 > 0 and wend[w0 - 1] == wend[i]:
            w0 -= 1
        assert w0 <= F.rho[i] < wend[i]
    for j in range(n):  # multipliers of the window are <= 1
        for i in range(j + 1, wend[j]):
            assert abs(F.L[i, j]) <= abs(F.L[j, j]) * (1 + 1e-15)
    assert not np.array_equal(F.rho, np.arange(n))  # pivoting really happened


@pytest.mark.parametrize("seed", range(3))
def test_spd_without_pivoting_relates_to_cholesky(orc, seed):
    n = [25, 50, 70][seed]
    rp, ci, v = gen.random_spd(n, 0.15, seed + 40)
    perm = gen.random_perm(n, seed + 3)
    F = orc.lu_dense(rp, ci, v, perm)
    assert F.bad_col == -1
    G = np.linalg.cholesky(dense(rp, ci, v)[np.ix_(perm, perm)])
    g = np.diag(G)
    assert np.allclose(F.L, G * g[None, :], rtol=1e-12, atol=1e-12)
    assert np.allclose(F.U, G.T / g[:, None], rtol=1e-12, atol=1e-12)


def test_tridiagonal_closed_form(orc):
    n, a, c = 40, -1.3, -0.6
    rows = np.concatenate([np.arange(n), np.arange(1, n), np.arange(n - 1)])
    cols = np.concatenate([np.arange(n), np.arange(n - 1), np.arange(1, n)])
    vals = np.concatenate([np.full(n, 2.0), np.full(n - 1, a), np.full(n - 1, c)])
    rp, ci, v = gen._coo_to_csr(n, rows, cols, vals)
    F = orc.lu_dense(rp, ci, v, None)
    d = np.empty(n)
    d[0] = 2.0
    for k in range(n - 1):
        d[k + 1] = 2.0 - a * c / d[k]
    assert np.allclose(np.diag(F.L), d, rtol=1e-14)
    assert np.allclose(np.diag(F.L, -1), a, rtol=1e-14)
    assert np.allclose(np.diag(F.U, 1), c / d[:-1], rtol=1e-14)
    assert np.allclose(np.diag(F.U), 1.0)
    assert np.count_nonzero(np.tril(F.L, -2)) == 0 and np.count_nonzero(np.triu(F.U, 2)) == 0


def test_zero_diagonal_needs_pivoting(orc):
    shape, dofs = (4, 3, 3), 2
    rp, ci, v = gen.pivot_nodes_3d(*shape, dofs=dofs, seed=5)
    n = len(rp) - 1
    perm = gen.nd_perm(shape, dofs=dofs)
    assert orc.lu_dense(rp, ci, v, perm).bad_col == 0
    wend = orc.pivot_windows(np.arange(0, n, dofs), n)  # one window per node
    F = orc.lu_dense(rp, ci, v, perm, wend=wend)
    assert F.bad_col == -1
    # the planted order: inside every node, position t holds dof dofs-1-t
    want = (np.arange(n) // dofs) * dofs + (dofs - 1 - np.arange(n) % dofs)
    assert np.array_equal(F.rho, want)
    # and the factors are those of B = Pi_0 C without pivoting
    C = dense(rp, ci, v)[np.ix_(perm, perm)]
    P, L_s, U_s = scipy.linalg.lu(C[want])
    assert np.array_equal(P, np.eye(n))
    L, U = crout(L_s, U_s)
    assert np.allclose(F.L, L, rtol=1e-12, atol=1e-13)
    assert np.allclose(F.U, U, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("case", ["nonsym", "pivot"])
def test_manufactured_solution(orc, case):
    if case == "nonsym":
        shape = (6, 5, 4)
        rp, ci, v = gen.nonsym_3d(*shape, wind=3.0, small_diag=0.3, seed=7)
        perm = gen.nd_perm(shape)
    else:
        shape = (5, 4, 3)
        rp, ci, v = gen.pivot_nodes_3d(*shape, dofs=2, seed=8)
        perm = gen.nd_perm(shape, dofs=2)
    n = len(rp) - 1
    so = orc.symbolic(rp, ci, perm)
    F = orc.lu_dense(rp, ci, v, perm, wend=orc.pivot_windows(so["sup_ptr"][:-1], n))
    assert F.bad_col == -1
    xs = np.random.default_rng(2).uniform(-1, 1, (n, 3))
    b = np.stack([gen.csr_matvec(rp, ci, v, xs[:, r]) for r in range(3)], axis=1)
    x = orc.solve_lu(F, b, perm)
    assert orc.berr(rp, ci, v, x, b) <= 1e-14
    assert np.allclose(x, xs, rtol=1e-9, atol=1e-9)


def test_ties_go_to_the_smallest_original_row(orc):
    """Worked by hand, one window over all rows of
        C = [[0, 1, 0], [2, 0, 1], [-2, 1, 0]]:
    column 0 ties |2| = |-2| and takes row 1 (rho = 1, 0, 2), pivot 2,
    U_01 = 0, U_02 = 1/2, and row 2 becomes [-2, 1, 1]; column 1 ties
    between C's rows 0 and 2 (both 1) and keeps row 0, pivot 1, U_12 = 0;
    column 2 has pivot 1."""
    rows = [0, 1, 1, 2, 2]
    cols = [1, 0, 2, 0, 1]
    vals = [1.0, 2.0, 1.0, -2.0, 1.0]
    rp, ci, v = gen._coo_to_csr(3, rows + [0, 2], cols + [2, 2], vals + [0.0, 0.0])
    F = orc.lu_dense(rp, ci, v, None, wend=np.full(3, 3))
    assert F.bad_col == -1
    assert list(F.rho) == [1, 0, 2]
    assert np.array_equal(F.L, [[2, 0, 0], [0, 1, 0], [-2, 1, 1]])
    assert np.array_equal(F.U, [[1, 0, 0.5], [0, 1, 0], [0, 0, 1]])
