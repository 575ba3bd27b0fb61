"""LDL^T with symmetric pivoting within the diagonal blocks on the GPU against
the oracle's dense windowed LDL^T (paper Sec. 5: Tacho's LDL^T of symmetric
indefinite matrices, pivots looked for only inside each diagonal block).

Workload: saddle-point matrices [K B^T; B 0] (no regularisation, so LDL^T in
the analysed order breaks down) with the multiplier ordered before the
velocity in every node: the first column has a zero pivot.  The analysis is
the condensed one (2 dofs per node), so every front holds whole nodes, and
without relaxation, so the diagonal blocks -- 64-column pieces of the
fronts -- are cut from the supernodes of the block-expanded matrix, which
the oracle computes by itself.

Comparison: the pivot order bit-exactly; L and D element by element in FP64
to relF <= max(1e-11, 1e-12 g), g = ||(|L| |D| |L|^T)||_F / ||C||_F the
growth of the oracle's factors (each entry carries rounding of order front
size x eps x (|L| |D| |L|^T)_ij); backward error <= 1e-13 of the FP64 solve
and of the FP32 factor refined in FP64."""
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


def saddle(shape, seed=0):
    rp, ci, v = gen.kkt_3d(*shape, delta=0.0, seed=seed)
    perm = gen.nd_perm(shape, dofs=2)
    perm = np.ascontiguousarray(perm.reshape(-1, 2)[:, ::-1].ravel()).astype(np.int32)
    node_of = (np.arange(len(rp) - 1) // 2).astype(np.int32)
    return rp, ci, v, perm, node_of


def analyse(mf, rp, ci, perm, node_of, relax=0, variant=2, queue=1):
    opt = mf.mf_options_default()
    opt.relax = relax
    opt.sptrsv = variant
    opt.small_queue = queue
    h = mf.mf_create(opt)
    s = mf.mf_symbolic_analyze_condensed(h, rp, ci, perm, node_of=node_of)
    return h, s


def free(mf, h, s, f):
    mf.mf_factor_free(f)
    mf.mf_symbolic_free(s)
    mf.mf_destroy(h)


def dense_L(mf, s, f, n):
    info = mf.mf_symbolic_get_info(s)
    Lp, Li = mf.mf_symbolic_pattern(s)
    Lx = mf.mf_factor_export_L(f, info["nnz_L"])
    rho = mf.mf_factor_export_pivots(f, n)
    fronts = mf.mf_symbolic_fronts(s)
    fend = fronts[np.repeat(np.arange(len(fronts) - 1), np.diff(fronts)) + 1]
    pos = np.empty(n, dtype=np.int64)
    pos[rho] = np.arange(n)
    cols = np.repeat(np.arange(n), np.diff(Lp))
    rows = Li.astype(np.int64)
    L = np.zeros((n, n))
    L[np.where(rows < fend[cols], rows, pos[rows]), cols] = Lx
    return L, rho


def oracle_factor(orc, rp, ci, v, perm, node_of):
    erp, eci, ev = orc.expand_node_blocks(rp, ci, v, node_of)
    n = len(rp) - 1
    so = orc.symbolic(erp, eci, perm)
    F = orc.ldlt_dense(erp, eci, ev, perm, wend=orc.pivot_windows(so["sup_ptr"][:-1], n))
    A = np.zeros((n, n))
    np.add.at(A, (np.repeat(np.arange(n), np.diff(rp)), ci), v)
    C = A[np.ix_(perm, perm)]
    g = np.linalg.norm(np.abs(F.L) @ np.diag(np.abs(F.D)) @ np.abs(F.L).T) / np.linalg.norm(C)
    return F, so, max(1e-11, 1e-12 * g)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("shape", [(4, 3, 3), (12, 11, 10)])
def test_pivoted_ldlt_matches_oracle(mf, orc, shape):
    rp, ci, v, perm, node_of = saddle(shape)
    n = len(rp) - 1
    h, s = analyse(mf, rp, ci, perm, node_of)
    f = mf.mf_factor_create_ldlt(h, s, 0)
    try:
        with pytest.raises(mf.MFError) as e:
            mf.mf_factor_numeric(f, v)
        assert e.value.code == mf.MF_ERR_NOT_SPD and e.value.column == 0
    finally:
        mf.mf_factor_free(f)
    f = mf.mf_factor_create_ldlt_piv(h, s, 0)
    try:
        mf.mf_factor_numeric(f, v)
        F, so, tol = oracle_factor(orc, rp, ci, v, perm, node_of)
        assert F.bad_col == -1
        assert np.array_equal(mf.mf_symbolic_fronts(s), so["sup_ptr"])
        if shape[0] >= 12:
            assert mf.mf_symbolic_get_info(s)["max_front"] > 128
        L, rho = dense_L(mf, s, f, n)
        D = mf.mf_factor_export_D(f, n)
        assert np.array_equal(rho, F.rho)
        assert not np.array_equal(rho, np.arange(n))
        assert rel(L, F.L) <= tol
        assert rel(D, F.D) <= tol
        B = gen.rhs(n, 3, seed=2)
        X = mf.mf_solve(f, B)
        assert orc.berr(rp, ci, v, X, B) <= BERR
        Xo = orc.solve_ldlt_piv(F, B, perm)
        assert np.max(np.abs(X - Xo)) <= 1e-8 * np.max(np.abs(Xo))
    finally:
        free(mf, h, s, f)


def test_pivoted_ldlt_fp32_refined(mf, orc):
    rp, ci, v, perm, node_of = saddle((12, 11, 10), seed=1)
    n = len(rp) - 1
    h, s = analyse(mf, rp, ci, perm, node_of, relax=1)
    f = mf.mf_factor_create_ldlt_piv(h, s, 1)
    try:
        mf.mf_factor_numeric(f, v)
        B = gen.rhs(n, 2, seed=4)
        X, rep = mf.mf_solve_refined(f, B, tol=BERR, max_iter=30)
        assert orc.berr(rp, ci, v, X, B) <= BERR
        assert not rep["fell_back"]
    finally:
        free(mf, h, s, f)


@pytest.mark.parametrize("variant,queue", [(1, 1), (2, 0)])
def test_pivoted_ldlt_schedules_agree(mf, orc, variant, queue):
    rp, ci, v, perm, node_of = saddle((10, 9, 8), seed=2)
    n = len(rp) - 1
    B = gen.rhs(n, 2, seed=5)
    out = []
    for cfg in [(2, 1), (variant, queue)]:
        h, s = analyse(mf, rp, ci, perm, node_of, relax=1, variant=cfg[0], queue=cfg[1])
        f = mf.mf_factor_create_ldlt_piv(h, s, 0)
        try:
            mf.mf_factor_numeric(f, v)
            info = mf.mf_symbolic_get_info(s)
            L = mf.mf_factor_export_L(f, info["nnz_L"])
            X = mf.mf_solve(f, B)
            assert orc.berr(rp, ci, v, X, B) <= BERR
            out.append((L, X))
        finally:
            free(mf, h, s, f)
    assert np.array_equal(out[0][0], out[1][0])
    assert np.max(np.abs(out[0][1] - out[1][1])) <= 1e-12 * np.max(np.abs(out[0][1]))


def test_pivoted_ldlt_on_spd_and_variant_3_refused(mf, orc):
    shape = (14, 13, 12)
    rp, ci, v = gen.laplacian_3d(*shape)
    perm = gen.nd_perm(shape)
    n = len(rp) - 1
    h = mf.mf_create(mf.mf_options_default())
    s = mf.mf_symbolic_analyze(h, rp, ci, perm)
    f = mf.mf_factor_create_ldlt_piv(h, s, 0)
    try:
        mf.mf_factor_numeric(f, v)
        D = mf.mf_factor_export_D(f, n)
        assert np.all(D > 0)
        B = gen.rhs(n, 1, seed=6)
        X = mf.mf_solve(f, B)
        assert orc.berr(rp, ci, v, X, B) <= BERR
    finally:
        free(mf, h, s, f)
    opt = mf.mf_options_default()
    opt.sptrsv = 3
    h = mf.mf_create(opt)
    s = mf.mf_symbolic_analyze(h, rp, ci, perm)
    try:
        with pytest.raises(mf.MFError) as e:
            mf.mf_factor_create_ldlt_piv(h, s, 0)
        assert e.value.code == mf.MF_ERR_INVALID
    finally:
        mf.mf_symbolic_free(s)
        mf.mf_destroy(h)


def test_pivoted_ldlt_refinement_falls_back(mf, orc):
    """max_iter = 0: the FP64 pivoted LDL^T fallback delivers the FP64
    backward error."""
    rp, ci, v, perm, node_of = saddle((10, 9, 8), seed=3)
    n = len(rp) - 1
    h, s = analyse(mf, rp, ci, perm, node_of, relax=1)
    f = mf.mf_factor_create_ldlt_piv(h, s, 1)
    try:
        mf.mf_factor_numeric(f, v)
        B = gen.rhs(n, 1, seed=7)
        X, rep = mf.mf_solve_refined(f, B, tol=1e-15, max_iter=0)
        assert rep["fell_back"] == 1
        assert orc.berr(rp, ci, v, X, B) <= BERR
    finally:
        free(mf, h, s, f)


@pytest.mark.parametrize("case", ["diagonal", "dense"])
def test_pivoted_ldlt_degenerate_shapes(mf, orc, case):
    """A diagonal matrix with negative entries (one-column fronts) and a dense
    symmetric indefinite 150 x 150 block (one front, three pivot blocks with a
    ragged last one) against the oracle."""
    rng = np.random.default_rng(18)
    if case == "diagonal":
        A = np.diag(np.where(rng.random(40) < 0.5, -1.0, 1.0) * rng.uniform(1, 3, 40))
    else:
        M = rng.uniform(-1, 1, (150, 150))
        A = M + M.T
    n = len(A)
    rows, cols = np.nonzero(np.ones_like(A) if case == "dense" else A)
    rp = np.zeros(n + 1, dtype=np.int64)
    rp[1:] = np.cumsum(np.bincount(rows, minlength=n))
    ci = cols.astype(np.int32)
    v = A[rows, cols]
    h = mf.mf_create(mf.mf_options_default())
    s = mf.mf_symbolic_analyze(h, rp, ci, None)
    f = mf.mf_factor_create_ldlt_piv(h, s, 0)
    try:
        mf.mf_factor_numeric(f, v)
        B = gen.rhs(n, 2, seed=19)
        X = mf.mf_solve(f, B)
        assert orc.berr(rp, ci, v, X, B) <= BERR
        so = orc.symbolic(rp, ci, None)
        assert np.array_equal(mf.mf_symbolic_fronts(s), so["sup_ptr"])
        F = orc.ldlt_dense(rp, ci, v, None, wend=orc.pivot_windows(so["sup_ptr"][:-1], n))
        L, rho = dense_L(mf, s, f, n)
        assert np.array_equal(rho, F.rho)
        g = np.linalg.norm(np.abs(F.L) @ np.diag(np.abs(F.D)) @ np.abs(F.L).T) / np.linalg.norm(A)
        tol = max(1e-11, 1e-12 * g)
        assert rel(L, F.L) <= tol
        assert rel(mf.mf_factor_export_D(f, n), F.D) <= tol
    finally:
        free(mf, h, s, f)
