"""LU of general matrices with a symmetric pattern on the GPU against the
oracle's dense windowed LU (paper Sec. 5: Tacho's LU of a general matrix
with a symmetric sparsity structure, pivots looked for only within the
diagonal blocks).

Workloads (pattern symmetric, values not):
* 7-point convection-diffusion with a weak wind (an M-matrix: LU without
  pivoting exists and is stable);
* the same with a strong wind and a share of tiny diagonal entries, where
  partial pivoting within the diagonal blocks swaps rows (analysis without
  relaxation, so the diagonal blocks -- 64-column pieces of the fronts --
  are cut from the fundamental supernodes, which the oracle computes by
  itself);
* node-block matrices with zero diagonal entries whose pivot sequence is
  unique within any block holding a node (gen.pivot_nodes_3d): LU without
  pivoting fails at column 0, with pivoting the row order must come out
  exactly.

Comparison: the row order rho bit-exactly; L and U element by element,
dense, in FP64 to relF <= max(1e-11, 1e-12 g) with the growth
g = ||(|L| |U|)||_F / ||C||_F of the oracle's factors: each computed entry
carries rounding errors of order (front size) x eps x (|L| |U|)_ij, so
two correct computations in different orders differ by about that much,
and pivoting restricted to diagonal blocks lets g reach the thousands on
the strong-wind case; backward error <= 1e-13 of the FP64 solve and of the
FP32 factor refined in FP64."""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu
BERR = 1e-13


@pytest.fixture(scope="module")
def mf():
    import torch
    assert torch.cuda.is_available()
    import paper_2506_05793_gb300 as m
    m.build()
    return m


def lu_factor(mf, rp, ci, v, perm, prec=0, pivot=0, relax=1, variant=2, queue=1, graphs=1):
    opt = mf.mf_options_default()
    opt.sptrsv = variant
    opt.relax = relax
    opt.small_queue = queue
    opt.use_graphs = graphs
    h = mf.mf_create(opt)
    s = mf.mf_symbolic_analyze(h, rp, ci, perm)
    f = mf.mf_factor_create_lu(h, s, prec, pivot)
    return h, s, f


def free(mf, h, s, f):
    mf.mf_factor_free(f)
    mf.mf_symbolic_free(s)
    mf.mf_destroy(h)


def dense_factors(mf, s, f, n):
    """The GPU factors as dense L (pivot order) and U, and rho."""
    info = mf.mf_symbolic_get_info(s)
    Lp, Li = mf.mf_symbolic_pattern(s)
    Lx = mf.mf_factor_export_L(f, info["nnz_L"])
    Ux = mf.mf_factor_export_U(f, info["nnz_L"])
    rho = mf.mf_factor_export_pivots(f, n)
    fronts = mf.mf_symbolic_fronts(s)
    col_front = np.repeat(np.arange(len(fronts) - 1), np.diff(fronts))
    fend = fronts[col_front + 1]
    pos = np.empty(n, dtype=np.int64)
    pos[rho] = np.arange(n)  # position of each row label
    cols = np.repeat(np.arange(n), np.diff(Lp))
    rows = Li.astype(np.int64)
    own = rows < fend[cols]  # labels of the column's own front are positions
    L = np.zeros((n, n))
    L[np.where(own, rows, pos[rows]), cols] = Lx
    U = np.zeros((n, n))
    U[cols, rows] = Ux
    return L, U, rho


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def factor_tol(F, rp, ci, v, perm):
    """max(1e-11, 1e-12 g), g = ||(|L| |U|)||_F / ||C||_F (module docstring)."""
    n = len(rp) - 1
    A = np.zeros((n, n))
    np.add.at(A, (np.repeat(np.arange(n), np.diff(rp)), ci), v)
    C = A[np.ix_(perm, perm)]
    g = np.linalg.norm(np.abs(F.L) @ np.abs(F.U)) / np.linalg.norm(C)
    return max(1e-11, 1e-12 * g)


def weak_wind(shape, seed=0):
    return gen.nonsym_3d(*shape, wind=0.5, seed=seed), gen.nd_perm(shape)


@pytest.mark.parametrize("shape", [(6, 5, 4), (15, 14, 16)])
def test_lu_without_pivoting_matches_oracle(mf, orc, shape):
    (rp, ci, v), perm = weak_wind(shape)
    n = len(rp) - 1
    h, s, f = lu_factor(mf, rp, ci, v, perm)
    try:
        mf.mf_factor_numeric(f, v)
        info = mf.mf_symbolic_get_info(s)
        if shape[0] >= 15:
            assert info["max_front"] > 128  # the blocked large-front kernels ran
        F = orc.lu_dense(rp, ci, v, perm)
        assert F.bad_col == -1
        L, U, rho = dense_factors(mf, s, f, n)
        assert np.array_equal(rho, np.arange(n))
        tol = factor_tol(F, rp, ci, v, perm)
        assert rel(L, F.L) <= tol
        assert rel(U, F.U) <= tol
        B = gen.rhs(n, 3, seed=2)
        X = mf.mf_solve(f, B)
        assert orc.berr(rp, ci, v, X, B) <= BERR
        Xo = orc.solve_lu(F, B, perm)
        assert np.max(np.abs(X - Xo)) <= 1e-10 * np.max(np.abs(Xo))
    finally:
        free(mf, h, s, f)


@pytest.mark.parametrize("shape,seed", [((7, 6, 5), 0), ((15, 14, 16), 1)])
def test_lu_pivoting_within_diagonal_blocks_matches_oracle(mf, orc, shape, seed):
    rp, ci, v = gen.nonsym_3d(*shape, wind=3.0, small_diag=0.3, seed=seed)
    perm = gen.nd_perm(shape)
    n = len(rp) - 1
    h, s, f = lu_factor(mf, rp, ci, v, perm, pivot=1, relax=0)
    try:
        mf.mf_factor_numeric(f, v)
        so = orc.symbolic(rp, ci, perm)
        # without relaxation the fronts are the fundamental supernodes
        assert np.array_equal(mf.mf_symbolic_fronts(s), so["sup_ptr"])
        F = orc.lu_dense(rp, ci, v, perm, wend=orc.pivot_windows(so["sup_ptr"][:-1], n))
        assert F.bad_col == -1
        L, U, rho = dense_factors(mf, s, f, n)
        assert np.array_equal(rho, F.rho)
        assert not np.array_equal(rho, np.arange(n))  # rows were really swapped
        tol = factor_tol(F, rp, ci, v, perm)
        assert rel(L, F.L) <= tol
        assert rel(U, F.U) <= tol
        B = gen.rhs(n, 2, seed=3)
        X = mf.mf_solve(f, B)
        assert orc.berr(rp, ci, v, X, B) <= BERR
    finally:
        free(mf, h, s, f)


@pytest.mark.parametrize("shape", [(5, 4, 3), (12, 11, 10)])
def test_zero_diagonal_needs_pivoting(mf, orc, shape):
    dofs = 2
    rp, ci, v = gen.pivot_nodes_3d(*shape, dofs=dofs, seed=4)
    perm = gen.nd_perm(shape, dofs=dofs)
    n = len(rp) - 1
    h, s, f = lu_factor(mf, rp, ci, v, perm, pivot=0)
    try:
        with pytest.raises(mf.MFError) as e:
            mf.mf_factor_numeric(f, v)
        assert e.value.code == mf.MF_ERR_NOT_SPD and e.value.column == 0
        assert "zero pivot" in str(e.value)
    finally:
        free(mf, h, s, f)
    h, s, f = lu_factor(mf, rp, ci, v, perm, pivot=1)
    try:
        mf.mf_factor_numeric(f, v)
        F = orc.lu_dense(rp, ci, v, perm, wend=orc.pivot_windows(np.arange(0, n, dofs), n))
        assert F.bad_col == -1
        L, U, rho = dense_factors(mf, s, f, n)
        want = (np.arange(n) // dofs) * dofs + (dofs - 1 - np.arange(n) % dofs)
        assert np.array_equal(rho, want)
        assert np.array_equal(F.rho, want)
        tol = factor_tol(F, rp, ci, v, perm)
        assert rel(L, F.L) <= tol
        assert rel(U, F.U) <= tol
        B = gen.rhs(n, 1, seed=5)
        X = mf.mf_solve(f, B)
        assert orc.berr(rp, ci, v, X, B) <= BERR
    finally:
        free(mf, h, s, f)


@pytest.mark.parametrize("pivot", [0, 1])
def test_lu_fp32_refined(mf, orc, pivot):
    shape = (15, 14, 16)
    if pivot:
        rp, ci, v = gen.pivot_nodes_3d(10, 9, 8, dofs=2, seed=6)
        perm = gen.nd_perm((10, 9, 8), dofs=2)
    else:
        (rp, ci, v), perm = weak_wind(shape, seed=3)
    n = len(rp) - 1
    h, s, f = lu_factor(mf, rp, ci, v, perm, prec=1, pivot=pivot)
    try:
        mf.mf_factor_numeric(f, v)
        if not pivot:
            F = orc.lu_dense(rp, ci, v, perm)
            L, U, _ = dense_factors(mf, s, f, n)
            assert rel(L, F.L) <= 1e-5 and rel(U, F.U) <= 1e-5
        B = gen.rhs(n, 2, seed=7)
        X, rep = mf.mf_solve_refined(f, B, tol=BERR, max_iter=10)
        assert orc.berr(rp, ci, v, X, B) <= BERR
        assert not rep["fell_back"]
    finally:
        free(mf, h, s, f)


@pytest.mark.parametrize("variant,queue,graphs", [(1, 1, 1), (2, 0, 1), (2, 1, 0)])
def test_lu_schedules_agree(mf, orc, variant, queue, graphs):
    rp, ci, v = gen.nonsym_3d(12, 11, 10, wind=3.0, small_diag=0.2, seed=8)
    perm = gen.nd_perm((12, 11, 10))
    n = len(rp) - 1
    B = gen.rhs(n, 4, seed=9)
    out = []
    for cfg in [(2, 1, 1), (variant, queue, graphs)]:
        h, s, f = lu_factor(mf, rp, ci, v, perm, pivot=1, variant=cfg[0], queue=cfg[1],
                            graphs=cfg[2])
        try:
            mf.mf_factor_numeric(f, v)
            info = mf.mf_symbolic_get_info(s)
            L = mf.mf_factor_export_L(f, info["nnz_L"])
            U = mf.mf_factor_export_U(f, info["nnz_L"])
            X = mf.mf_solve(f, B)
            assert orc.berr(rp, ci, v, X, B) <= BERR
            out.append((L, U, X))
        finally:
            free(mf, h, s, f)
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert np.max(np.abs(out[0][2] - out[1][2])) <= 1e-12 * np.max(np.abs(out[0][2]))


def test_lu_refactor_is_bitwise_deterministic(mf):
    rp, ci, v = gen.nonsym_3d(12, 12, 12, wind=3.0, small_diag=0.2, seed=10)
    perm = gen.nd_perm((12, 12, 12))
    h, s, f = lu_factor(mf, rp, ci, v, perm, pivot=1)
    try:
        info = mf.mf_symbolic_get_info(s)
        mf.mf_factor_numeric(f, v)
        a = mf.mf_factor_export_L(f, info["nnz_L"]), mf.mf_factor_export_U(f, info["nnz_L"])
        mf.mf_factor_numeric(f, v * 1.5)
        mf.mf_factor_numeric(f, v)
        b = mf.mf_factor_export_L(f, info["nnz_L"]), mf.mf_factor_export_U(f, info["nnz_L"])
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    finally:
        free(mf, h, s, f)


def test_lu_refuses_variant_3_and_unsymmetric_patterns(mf):
    (rp, ci, v), perm = weak_wind((6, 5, 4))
    opt = mf.mf_options_default()
    opt.sptrsv = 3
    h = mf.mf_create(opt)
    s = mf.mf_symbolic_analyze(h, rp, ci, perm)
    try:
        with pytest.raises(mf.MFError) as e:
            mf.mf_factor_create_lu(h, s, 0, 0)
        assert e.value.code == mf.MF_ERR_INVALID
    finally:
        mf.mf_symbolic_free(s)
        mf.mf_destroy(h)
    # a tridiagonal lower part plus one upper entry C(0, n-1): its transpose
    # is not in the analysed structure of column 0
    n = 40
    rows = np.concatenate([np.arange(n), np.arange(1, n), np.arange(n - 1), [0]])
    cols = np.concatenate([np.arange(n), np.arange(n - 1), np.arange(1, n), [n - 1]])
    vals = np.concatenate([np.full(n, 4.0), np.full(n - 1, -1.0), np.full(n - 1, -0.5), [0.3]])
    rp, ci, v = gen._coo_to_csr(n, rows, cols, vals)
    h = mf.mf_create(mf.mf_options_default())
    s = mf.mf_symbolic_analyze(h, rp, ci, None)
    try:
        with pytest.raises(mf.MFError) as e:
            mf.mf_factor_create_lu(h, s, 0, 1)
        assert e.value.code == mf.MF_ERR_INVALID
    finally:
        mf.mf_symbolic_free(s)
        mf.mf_destroy(h)


def test_lu_many_rhs_and_device_values(mf, orc):
    """40 right-hand sides (two solve chunks), values and right-hand sides
    given on the device."""
    import torch
    rp, ci, v = gen.nonsym_3d(12, 11, 10, wind=3.0, small_diag=0.2, seed=11)
    perm = gen.nd_perm((12, 11, 10))
    n = len(rp) - 1
    h, s, f = lu_factor(mf, rp, ci, v, perm, pivot=1)
    try:
        mf.mf_factor_numeric(f, torch.from_numpy(v).cuda())
        B = gen.rhs(n, 40, seed=12)
        X = mf.mf_solve(f, B)
        assert orc.berr(rp, ci, v, X, B) <= BERR
        Bd = torch.from_numpy(np.ascontiguousarray(B.T)).cuda().t()
        Xd = mf.mf_solve(f, Bd)
        torch.cuda.synchronize()
        assert np.array_equal(Xd.cpu().numpy(), X)
    finally:
        free(mf, h, s, f)


def test_lu_refinement_falls_back_to_fp64_lu(mf, orc):
    """max_iter = 0 forces the stagnation branch: the FP64 LU of the same
    kind (pivoting within the diagonal blocks) must deliver the FP64
    backward error."""
    rp, ci, v = gen.nonsym_3d(12, 11, 10, wind=3.0, small_diag=0.2, seed=13)
    perm = gen.nd_perm((12, 11, 10))
    n = len(rp) - 1
    h, s, f = lu_factor(mf, rp, ci, v, perm, prec=1, pivot=1)
    try:
        mf.mf_factor_numeric(f, v)
        B = gen.rhs(n, 1, seed=14)
        X, rep = mf.mf_solve_refined(f, B, tol=1e-15, max_iter=0)
        assert rep["fell_back"] == 1
        assert orc.berr(rp, ci, v, X, B) <= BERR
    finally:
        free(mf, h, s, f)


def test_lu_on_a_loaded_analysis(mf, orc, tmp_path):
    """An analysis saved and loaded again factors bit-identically."""
    rp, ci, v = gen.nonsym_3d(10, 9, 8, wind=3.0, small_diag=0.2, seed=15)
    perm = gen.nd_perm((10, 9, 8))
    h, s, f = lu_factor(mf, rp, ci, v, perm, pivot=1)
    path = str(tmp_path / "lu.mfs")
    try:
        mf.mf_factor_numeric(f, v)
        info = mf.mf_symbolic_get_info(s)
        a = mf.mf_factor_export_L(f, info["nnz_L"]), mf.mf_factor_export_U(f, info["nnz_L"])
        mf.mf_symbolic_save(s, path)
        t = mf.mf_symbolic_load(h, path)
        g = mf.mf_factor_create_lu(h, t, 0, 1)
        try:
            mf.mf_factor_numeric(g, v)
            b = mf.mf_factor_export_L(g, info["nnz_L"]), mf.mf_factor_export_U(g, info["nnz_L"])
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        finally:
            mf.mf_factor_free(g)
            mf.mf_symbolic_free(t)
    finally:
        free(mf, h, s, f)


@pytest.mark.parametrize("case", ["one", "diagonal", "dense"])
def test_lu_degenerate_shapes(mf, orc, case):
    """A 1 x 1 matrix, a diagonal matrix (fronts of one column, no update
    rows) and a dense nonsymmetric 150 x 150 block (one front, three 64-row
    pivot blocks with a ragged last one), with pivoting."""
    rng = np.random.default_rng(16)
    if case == "one":
        A = np.array([[-3.0]])
    elif case == "diagonal":
        A = np.diag(rng.uniform(-2, 2, 50) + np.where(rng.random(50) < 0.5, 3.0, -3.0))
    else:
        A = rng.uniform(-1, 1, (150, 150))
    n = len(A)
    rows, cols = np.nonzero(np.ones_like(A) if case == "dense" else A)
    rp = np.zeros(n + 1, dtype=np.int64)
    rp[1:] = np.cumsum(np.bincount(rows, minlength=n))
    ci = cols.astype(np.int32)
    v = A[rows, cols]
    h, s, f = lu_factor(mf, rp, ci, v, None, pivot=1)
    try:
        mf.mf_factor_numeric(f, v)
        B = gen.rhs(n, 2, seed=17)
        X = mf.mf_solve(f, B)
        assert orc.berr(rp, ci, v, X, B) <= BERR
        if case == "dense":
            so = orc.symbolic(rp, ci, None)  # one supernode: windows of 64 columns
            assert np.array_equal(mf.mf_symbolic_fronts(s), so["sup_ptr"])
            F = orc.lu_dense(rp, ci, v, None, wend=orc.pivot_windows(so["sup_ptr"][:-1], n))
            L, U, rho = dense_factors(mf, s, f, n)
            assert np.array_equal(rho, F.rho)
            tol = factor_tol(F, rp, ci, v, np.arange(n))
            assert rel(L, F.L) <= tol and rel(U, F.U) <= tol
    finally:
        free(mf, h, s, f)
