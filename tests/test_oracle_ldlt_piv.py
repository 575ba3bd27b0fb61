"""Pins of the oracle's LDL^T with symmetric (1x1) pivoting within diagonal
blocks and its solve, independent of its C code.

* No pivoting: equal to the oracle's unpivoted left-looking LDL^T (itself
  pinned in tests/test_oracle_ldlt.py) on indefinite quasi-definite inputs.
* One window over all rows of an SPD input: the largest remaining diagonal
  is LAPACK's pivoted Cholesky (dpstrf): the same order, L = G diag(G)^-1
  and D = diag(G)^2.
* Windows of whole nodes on indefinite inputs: Pi C Pi^T = L D L^T to rounding, rows stay in
  their windows, and each pivot is the largest remaining diagonal of its
  window: |d_j| >= |sum_{q >= j} L_iq^2 d_q| for the window's later rows i
  (the Schur complement's diagonal at step j, from the final factors).
* Saddle-point inputs with a zero (2,2) block and the multiplier ordered
  first in every node: no pivoting stops at column 0; pivoting within the
  nodes succeeds; manufactured solutions.
* A 3 x 3 worked by hand, with a tie."""
import numpy as np
import pytest
import scipy.linalg.lapack as lapack

import gen


def dense(rp, ci, v):
    n = len(rp) - 1
    A = np.zeros((n, n))
    np.add.at(A, (np.repeat(np.arange(n), np.diff(rp)), ci), v)
    return A


def p_first(perm):
    """The node pairs (u_i, p_i) of gen.nd_perm(..., dofs=2) with p_i first."""
    return np.ascontiguousarray(np.asarray(perm).reshape(-1, 2)[:, ::-1].ravel()).astype(np.int32)


@pytest.mark.parametrize("shape,seed", [((3, 3, 2), 0), ((4, 3, 3), 1)])
def test_no_pivoting_equals_left_looking_ldlt(orc, shape, seed):
    rp, ci, v = gen.kkt_3d(*shape, seed=seed)
    perm = gen.nd_perm(shape, dofs=2)
    F = orc.ldlt_dense(rp, ci, v, perm)
    G = orc.factor_ldlt(rp, ci, v, perm)
    assert F.bad_col == -1 and G.bad_col == -1
    assert np.array_equal(F.rho, np.arange(len(F.rho)))
    assert np.allclose(F.L, G.dense(), rtol=1e-12, atol=1e-12)
    assert np.allclose(F.D, G.D, rtol=1e-12)


@pytest.mark.parametrize("seed", range(3))
def test_one_window_spd_is_pivoted_cholesky(orc, seed):
    n = [20, 40, 60][seed]
    rp, ci, v = gen.random_spd(n, 0.2, seed + 90)
    F = orc.ldlt_dense(rp, ci, v, None, wend=np.full(n, n))
    assert F.bad_col == -1
    c, piv, rank, info = lapack.dpstrf(dense(rp, ci, v), lower=1)
    assert info == 0 and rank == n
    G = np.tril(c)
    g = np.diag(G)
    assert np.array_equal(F.rho, piv - 1)
    assert np.allclose(F.L, G / g[None, :], rtol=1e-11, atol=1e-12)
    assert np.allclose(F.D, g ** 2, rtol=1e-11)


@pytest.mark.parametrize("nodes,seed", [(1, 0), (2, 1), (4, 2), (32, 3)])
def test_windowed_symmetric_pivoting_invariants(orc, nodes, seed):
    shape = (4, 4, 3)
    rp, ci, v = gen.kkt_3d(*shape, delta=0.0, seed=seed)
    perm = p_first(gen.nd_perm(shape, dofs=2))
    n = len(rp) - 1
    # windows of whole nodes (a window holding a multiplier without its
    # velocity would have a zero pivot)
    wend = orc.pivot_windows(np.arange(0, n, 2 * nodes), n)
    F = orc.ldlt_dense(rp, ci, v, perm, wend=wend)
    assert F.bad_col == -1
    C = dense(rp, ci, v)[np.ix_(perm, perm)]
    Cp = C[np.ix_(F.rho, F.rho)]
    R = Cp - F.L @ np.diag(F.D) @ F.L.T
    scale = np.max(np.abs(C)) * max(1.0, np.max(np.abs(F.L)) ** 2 * np.max(np.abs(F.D)))
    assert np.max(np.abs(R)) <= 1e-12 * scale
    for i in range(n):
        w0 = i
        while w0 > 0 and wend[w0 - 1] == wend[i]:
            w0 -= 1
        assert w0 <= F.rho[i] < wend[i]
    for j in range(n):
        for i in range(j + 1, wend[j]):
            s = np.sum(F.L[i, j:] ** 2 * F.D[j:])
            assert abs(F.D[j]) >= abs(s) * (1 - 1e-12)
    assert not np.array_equal(F.rho, np.arange(n))
    assert np.any(F.D < 0) and np.any(F.D > 0)


def test_zero_block_needs_pivoting(orc):
    shape = (4, 3, 3)
    rp, ci, v = gen.kkt_3d(*shape, delta=0.0, seed=4)
    perm = p_first(gen.nd_perm(shape, dofs=2))
    n = len(rp) - 1
    assert orc.ldlt_dense(rp, ci, v, perm).bad_col == 0
    F = orc.ldlt_dense(rp, ci, v, perm, wend=orc.pivot_windows(np.arange(0, n, 2), n))
    assert F.bad_col == -1
    xs = np.random.default_rng(3).uniform(-1, 1, (n, 2))
    b = np.stack([gen.csr_matvec(rp, ci, v, xs[:, r]) for r in range(2)], axis=1)
    x = orc.solve_ldlt_piv(F, b, perm)
    assert orc.berr(rp, ci, v, x, b) <= 1e-14
    assert np.allclose(x, xs, rtol=1e-8, atol=1e-8)


def test_hand_worked_with_tie(orc):
    """C = [[1, 2, 0], [2, -3, 1], [0, 1, 3]], one window over all rows.
    Step 0: diagonals 1, -3, 3 tie at |3| between positions 1 and 2; the
    smaller starting row, 1, is taken: rho = 1, 0, 2, d_0 = -3, and the
    remaining block [[1, 0], [0, 3]] - [2, 1]^T [2, 1] / (-3) =
    [[7/3, 2/3], [2/3, 10/3]].  Step 1: |7/3| < |10/3|: swap, rho = 1, 2, 0,
    d_1 = 10/3, L_21 = (2/3)/(10/3) = 1/5, and d_2 = 7/3 - (2/3)^2/(10/3) = 11/5.
    Column 0 of L in the final order: (1, 1/(-3), 2/(-3)) for C's rows 1, 2, 0."""
    rows = [0, 0, 1, 1, 1, 2, 2]
    cols = [0, 1, 0, 1, 2, 1, 2]
    vals = [1.0, 2.0, 2.0, -3.0, 1.0, 1.0, 3.0]
    rp, ci, v = gen._coo_to_csr(3, rows, cols, vals)
    F = orc.ldlt_dense(rp, ci, v, None, wend=np.full(3, 3))
    assert F.bad_col == -1
    assert list(F.rho) == [1, 2, 0]
    assert np.allclose(F.D, [-3.0, 10.0 / 3, 11.0 / 5], rtol=1e-15)
    want = np.array([[1, 0, 0], [-1.0 / 3, 1, 0], [-2.0 / 3, 0.2, 1]])
    assert np.allclose(F.L, want, rtol=1e-15, atol=1e-15)
