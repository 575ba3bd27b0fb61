"""Pins for the FP64 oracle (CPU only).

Each pin ties the oracle to something other than itself: a library routine
(numpy/LAPACK dense Cholesky), a closed form (1D Laplacian factor, Dirichlet
Laplacian log-determinant), brute-force dense boolean elimination, or a
structural invariant of the elimination tree and supernode partition.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import gen


def dense(rp, ci, v):
    n = len(rp) - 1
    return sp.csr_matrix((v, ci, rp), shape=(n, n)).toarray()


def dense_pattern_L(C):
    """Structural pattern of L by dense boolean elimination (no values)."""
    n = C.shape[0]
    B = np.tril(C != 0)
    np.fill_diagonal(B, True)
    for j in range(n):
        below = np.nonzero(B[j + 1:, j])[0] + j + 1
        for a in below:
            B[a, below[below <= a]] = True
    return B


CASES = [(n, d, s) for n, d in [(1, 0.5), (2, 0.9), (17, 0.2), (60, 0.08), (150, 0.03)]
         for s in range(3)]


@pytest.mark.parametrize("n,density,seed", CASES)
def test_symbolic_vs_brute_force(orc, n, density, seed):
    rp, ci, v = gen.random_spd(n, density, seed)
    perm = gen.random_perm(n, seed + 11)
    s = orc.symbolic(rp, ci, perm)
    bp, bc = orc.brute_symbolic(rp, ci, perm)
    assert np.array_equal(s["parent"], bp)
    assert np.array_equal(s["colcount"], bc)
    assert s["nnzL"] == int(bc.sum())
    # invariants: parent(j) > j; struct(L_j) \ {j} subset of struct(L_parent)
    par = s["parent"]
    nz = par >= 0
    assert np.all(par[nz] > np.nonzero(nz)[0])
    assert np.all(s["colcount"][nz] - 1 <= s["colcount"][par[nz]])


@pytest.mark.parametrize("n,density,seed", CASES)
def test_numeric_vs_numpy_cholesky(orc, n, density, seed):
    rp, ci, v = gen.random_spd(n, density, seed, dense_rows=1 if seed == 2 else 0)
    perm = gen.random_perm(n, seed + 5)
    F = orc.factor(rp, ci, v, perm)
    assert F.bad_col == -1
    C = dense(rp, ci, v)[np.ix_(perm, perm)]
    Lref = np.linalg.cholesky(C)
    L = F.dense()
    assert np.max(np.abs(L - Lref)) <= 1e-13 * max(1.0, np.max(np.abs(Lref)))
    # residual of the oracle itself: ||C - L L^T||_F <= c n u ||C||_F
    res = np.linalg.norm(C - L @ L.T) / np.linalg.norm(C)
    assert res <= 10 * n * np.finfo(float).eps
    # structural pattern equals dense boolean elimination
    B = dense_pattern_L(C)
    P = np.zeros_like(B)
    for j in range(n):
        r, _ = F.column(j)
        P[r, j] = True
    assert np.array_equal(P, B)


@pytest.mark.parametrize("n,density,seed", CASES)
def test_supernodes_pattern_definition(orc, n, density, seed):
    """Fundamental supernodes, checked on the dense boolean pattern: inside a
    supernode column j+1 is j's only child and struct(L_j) = {j} u struct(L_j+1);
    at every boundary one of these fails (maximality)."""
    rp, ci, v = gen.random_spd(n, density, seed)
    perm = gen.random_perm(n, seed + 3)
    s = orc.symbolic(rp, ci, perm)
    sup = s["sup_ptr"]
    assert sup[0] == 0 and sup[-1] == n and np.all(np.diff(sup) > 0)
    C = dense(rp, ci, v)[np.ix_(perm, perm)]
    B = dense_pattern_L(C)
    par = np.full(n, -1)
    for j in range(n):
        nzr = np.nonzero(B[j + 1:, j])[0]
        if len(nzr):
            par[j] = j + 1 + nzr[0]
    nchild = np.bincount(par[par >= 0], minlength=n)

    def mergeable(j):
        same = np.array_equal(B[j + 1:, j], B[j + 1:, j + 1] | (np.arange(j + 1, n) == j + 1))
        return par[j] == j + 1 and nchild[j + 1] == 1 and same and B[j + 1, j]

    starts = set(sup[:-1].tolist())
    for j in range(n - 1):
        if (j + 1) in starts:
            assert not mergeable(j)
        else:
            assert mergeable(j)


def test_1d_laplacian_closed_form(orc):
    n = 200
    rp, ci, v = gen.laplacian_1d(n)
    s = orc.symbolic(rp, ci, None)
    assert np.array_equal(s["parent"][:-1], np.arange(1, n))
    assert s["parent"][-1] == -1
    assert np.all(s["colcount"][:-1] == 2) and s["colcount"][-1] == 1
    assert s["nnzL"] == 2 * n - 1
    assert s["flops"] == 4 * n - 3
    sup = s["sup_ptr"]
    assert len(sup) - 1 == n - 1
    assert sup[-2] == n - 2  # only the final pair {n-2, n-1} merges
    F = orc.factor(rp, ci, v, None)
    k = np.arange(1, n + 1, dtype=np.float64)  # 1-based
    diag = F.Lx[F.Lp[:-1]]
    assert np.allclose(diag, np.sqrt((k + 1) / k), rtol=1e-15, atol=0)
    off = F.Lx[F.Lp[:-2] + 1]
    assert np.allclose(off, -np.sqrt(k[:-1] / (k[:-1] + 1)), rtol=1e-14, atol=0)
    assert abs(F.logdet() - np.log(n + 1)) < 1e-12


def test_dense_and_diagonal_partitions(orc):
    n = 40
    rng = np.random.default_rng(0)
    M = rng.standard_normal((n, n))
    A = M @ M.T + n * np.eye(n)
    S = sp.csr_matrix(A)
    s = orc.symbolic(S.indptr.astype(np.int64), S.indices.astype(np.int32), None)
    assert list(s["sup_ptr"]) == [0, n]
    F = orc.factor(S.indptr.astype(np.int64), S.indices.astype(np.int32), S.data, None)
    assert np.allclose(F.dense(), np.linalg.cholesky(A), atol=1e-12)
    D = sp.csr_matrix(np.diag(np.arange(1.0, n + 1)))
    s = orc.symbolic(D.indptr.astype(np.int64), D.indices.astype(np.int32), None)
    assert np.all(s["parent"] == -1)
    assert list(s["sup_ptr"]) == list(range(n + 1))


def laplacian_logdet(shape):
    lams = [2.0 - 2.0 * np.cos(np.pi * np.arange(1, N + 1) / (N + 1)) for N in shape]
    grid = np.zeros([len(l) for l in lams])
    for ax, l in enumerate(lams):
        sh = [1] * len(lams)
        sh[ax] = len(l)
        grid = grid + l.reshape(sh)
    return float(np.sum(np.log(grid)))


@pytest.mark.parametrize("shape", [(64, 64), (37, 23), (12, 12, 12), (9, 14, 6)])
def test_laplacian_logdet_closed_form(orc, shape):
    if len(shape) == 2:
        rp, ci, v = gen.laplacian_2d(*shape)
    else:
        rp, ci, v = gen.laplacian_3d(*shape)
    perm = gen.nd_perm(shape)
    F = orc.factor(rp, ci, v, perm)
    ref = laplacian_logdet(shape)
    assert abs(F.logdet() - ref) <= 1e-11 * abs(ref)


def test_solve_manufactured(orc):
    rp, ci, v, perm, b = gen.config1()
    n = len(rp) - 1
    F = orc.factor(rp, ci, v, perm)
    xs = gen.rhs(n, 4, seed=9)
    B = gen.csr_matvec(rp, ci, v, xs)
    X = orc.solve(F, B, perm)
    assert orc.berr(rp, ci, v, X, B) <= 1e-15
    # kappa of the 64x64 Laplacian is ~1.7e3: forward error well below 1e-11
    assert np.max(np.abs(X - xs)) <= 1e-11
    x1 = orc.solve(F, b, perm)
    assert orc.berr(rp, ci, v, x1, b) <= 1e-15


def test_not_spd_column(orc):
    rp, ci, v = gen.laplacian_2d(20)
    perm = gen.nd_perm((20, 20))
    v = v.copy()
    old = int(perm[137])  # make C_137,137 negative
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    v[(rows == old) & (ci == old)] = -1.0
    F = orc.factor(rp, ci, v, perm)
    assert F.bad_col == 137


def test_subset_columns_exact(orc):
    rp, ci, v, perm, _ = gen.config1()
    s = orc.symbolic(rp, ci, perm)
    full = orc.factor(rp, ci, v, perm, sym=s)
    par = s["parent"]
    roots = [j for j in range(len(par)) if par[j] >= 0 and s["colcount"][j] > 20][:5]
    in_s = orc.descendant_closed(par, roots)
    sub = orc.factor(rp, ci, v, perm, in_s=in_s, sym=s)
    for j in np.nonzero(in_s)[0]:
        r1, x1 = full.column(j)
        r2, x2 = sub.column(j)
        assert np.array_equal(r1, r2)
        assert np.array_equal(x1, x2)
    first = np.zeros(len(par), dtype=np.uint8)
    first[:1000] = 1
    sub = orc.factor(rp, ci, v, perm, in_s=first, sym=s)
    assert np.array_equal(sub.Lx, full.Lx[: full.Lp[1000]])


def test_q1_symmetry_and_constant_modes():
    rp, ci, v = gen.q1_extruded(5, 4, 3, seed=7)
    A = dense(rp, ci, v)
    assert np.abs(A - A.T).max() <= 1e-12 * np.abs(A).max()
    n = A.shape[0]
    nx, ny, nz = 6, 5, 4
    assert n == 2 * nx * ny * nz
    # constant horizontal velocity has zero strain: only basal friction acts
    for comp in (0, 1):
        u = np.zeros(n)
        u[comp::2] = 1.0
        r = A @ u
        z = np.arange(n // 2) // (nx * ny)
        assert np.abs(r[comp::2][z > 0]).max() <= 1e-9 * np.abs(A).max()
        assert np.all(r[comp::2][z == 0] > 0)
        assert np.abs(r[1 - comp::2]).max() <= 1e-9 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 0


def test_laplacian_stencils():
    rp, ci, v = gen.laplacian_3d(7, 6, 5)
    A = dense(rp, ci, v)
    assert np.allclose(np.diag(A), 6.0) and set(np.unique(A)) <= {-1.0, 0.0, 6.0}
    assert rp[-1] == 7 * 6 * 5 + 2 * (6 * 6 * 5 + 7 * 5 * 5 + 7 * 6 * 4)
    rp, ci, v = gen.laplacian_3d(16, jump_block=8, seed=2)
    A = dense(rp, ci, v)
    assert np.abs(A - A.T).max() == 0
    # diagonal dominance with strict excess exactly at Dirichlet boundaries
    excess = np.diag(A) - (np.abs(A).sum(axis=1) - np.abs(np.diag(A)))
    assert excess.min() >= -1e-9 and excess.max() > 0


@pytest.mark.parametrize("shape,axes,dofs", [((13, 9), None, 1), ((9, 8, 7), None, 1),
                                             ((17, 11, 4), (0, 1), 2)])
def test_nd_perm_separates(shape, axes, dofs):
    perm = gen.nd_perm(shape, split_axes=axes, dofs=dofs)
    n = int(np.prod(shape)) * dofs
    assert np.array_equal(np.sort(perm), np.arange(n))
    if len(shape) == 2:
        rp, ci, v = gen.laplacian_2d(*shape)
    elif dofs == 1:
        rp, ci, v = gen.laplacian_3d(*shape)
    else:
        rp, ci, v = gen.q1_extruded(shape[0] - 1, shape[1] - 1, shape[2] - 1)
    A = dense(rp, ci, v) != 0
    C = A[np.ix_(perm, perm)]
    # top-level dissection: with the top separator removed, no edge joins the
    # part ordered first with the part ordered second
    nn = int(np.prod(shape))
    sizes = list(shape)
    cand = [a for a in (axes or range(len(shape))) if sizes[a] >= 3]
    ax = max(cand, key=lambda a: (sizes[a], -a))
    sep = int(np.prod(shape)) // shape[ax] * dofs
    left = (shape[ax] // 2) * (nn // shape[ax]) * dofs
    right_end = n - sep
    assert not C[:left, left:right_end].any()


@pytest.mark.parametrize("seed", range(6))
def test_expand_node_blocks_definition(orc, seed):
    """Block expansion against its dense definition: (i, j) is present iff
    node(i) == node(j) or some entry of A joins node(i) to node(j); A's
    values are kept and the added entries are zero; the expanded pattern
    contains A's and nodes of one DoF change nothing."""
    n = [6, 25, 60][seed % 3]
    rp, ci, v = gen.random_spd(n, 0.15, seed + 40)
    node_of, _ = gen.random_nodes(n, max_size=1 + seed % 3, seed=seed)
    erp, eci, ev = orc.expand_node_blocks(rp, ci, v, node_of)
    A = dense(rp, ci, v)
    E = dense(erp, eci, ev)
    want = np.zeros((n, n), dtype=bool)
    for i in range(n):
        for j in range(n):
            same = node_of[i] == node_of[j]
            link = any(A[a, b] != 0 for a in range(n) if node_of[a] == node_of[i]
                       for b in range(n) if node_of[b] == node_of[j])
            want[i, j] = same or link
    got = np.zeros((n, n), dtype=bool)
    got[np.repeat(np.arange(n), np.diff(erp)), eci] = True
    assert np.array_equal(got, want)
    assert np.array_equal(E, A)
    if seed % 3 == 0:
        one = orc.expand_node_blocks(rp, ci, v, np.arange(n))
        assert np.array_equal(one[0], rp) and np.array_equal(one[1], ci)


def test_berr_hand_computed(orc):
    """oracle.berr against the worked 3x3 example in tests/_berr_pins.py
    (residuals, norms and the maximum over right-hand sides by hand)."""
    import _berr_pins
    assert _berr_pins.failures(orc.berr) == set()
