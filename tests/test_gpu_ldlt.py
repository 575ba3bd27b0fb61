"""LDL^T (no pivoting) of symmetric indefinite matrices on the GPU against the
oracle's LDL^T (paper Sec. 5: Tacho's symmetric factorizations besides
Cholesky).  Workload: quasi-definite saddle-point matrices [K B^T; B -dI]
(K the 7-point Laplacian, B a node-local coupling), 2 unknowns per node,
nested dissection on the grid: every ordering of them has an LDL^T.

Bars as for Cholesky: FP64 relF(L), relF(D) <= 1e-11 and berr <= 1e-13
(every SpTRSV variant); FP32 + FP64 refinement berr <= 1e-13; SPD inputs
give L sqrt(D) = the Cholesky factor; a zero pivot is reported with its
column."""
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


def kkt(shape, seed=0):
    rp, ci, v = gen.kkt_3d(*shape, seed=seed)
    return rp, ci, v, gen.nd_perm(shape, dofs=2)


def ldlt_factor(mf, rp, ci, v, perm, prec=0, variant=2):
    opt = mf.mf_options_default()
    opt.sptrsv = variant
    h = mf.mf_create(opt)
    s = mf.mf_symbolic_analyze(h, rp, ci, perm)
    f = mf.mf_factor_create_ldlt(h, s, prec)
    mf.mf_factor_numeric(f, v)
    return h, s, f


def free(mf, h, s, f):
    mf.mf_factor_free(f)
    mf.mf_symbolic_free(s)
    mf.mf_destroy(h)


@pytest.mark.parametrize("shape", [(6, 5, 4), (14, 12, 10), (24, 24, 20)])
def test_ldlt_matches_oracle(mf, orc, shape):
    rp, ci, v, perm = kkt(shape)
    n = len(rp) - 1
    h, s, f = ldlt_factor(mf, rp, ci, v, perm)
    try:
        info = mf.mf_symbolic_get_info(s)
        F = orc.factor_ldlt(rp, ci, v, perm)
        assert F.bad_col == -1
        L = mf.mf_factor_export_L(f, info["nnz_L"])
        D = mf.mf_factor_export_D(f, n)
        assert orc.rel_fro(L, F.Lx) <= 1e-11
        assert orc.rel_fro(D, F.D) <= 1e-11
        assert np.any(D < 0) and np.any(D > 0)
        if shape[0] >= 14:
            assert info["max_front"] > 128  # the tiled large-front kernels ran
        B = gen.rhs(n, 3, seed=4)
        X = mf.mf_solve(f, B)
        assert orc.berr(rp, ci, v, X, B) <= BERR
        Xo = orc.solve_ldlt(F, B, perm)
        assert np.max(np.abs(X - Xo)) <= 1e-9 * np.max(np.abs(Xo))
    finally:
        free(mf, h, s, f)


@pytest.mark.parametrize("variant", [1, 3, 4])
def test_ldlt_every_solve_variant(mf, orc, variant):
    rp, ci, v, perm = kkt((14, 12, 10), seed=1)
    n = len(rp) - 1
    h, s, f = ldlt_factor(mf, rp, ci, v, perm, variant=variant)
    try:
        B = gen.rhs(n, 2, seed=6)
        X = mf.mf_solve(f, B)
        assert orc.berr(rp, ci, v, X, B) <= BERR
    finally:
        free(mf, h, s, f)


def test_ldlt_fp32_refined(mf, orc):
    rp, ci, v, perm = kkt((14, 12, 10), seed=2)
    n = len(rp) - 1
    h, s, f = ldlt_factor(mf, rp, ci, v, perm, prec=1)
    try:
        B = gen.rhs(n, 2, seed=7)
        X, rep = mf.mf_solve_refined(f, B, tol=BERR, max_iter=30)
        assert orc.berr(rp, ci, v, X, B) <= BERR
    finally:
        free(mf, h, s, f)


def test_ldlt_of_spd_is_scaled_cholesky(mf, orc):
    rp, ci, v, perm, _ = gen.config3(16)
    n = len(rp) - 1
    h = mf.mf_create()
    s = mf.mf_symbolic_analyze(h, rp, ci, perm)
    info = mf.mf_symbolic_get_info(s)
    fl = mf.mf_factor_create_ldlt(h, s, 0)
    fc = mf.mf_factor_create(h, s, 0)
    try:
        mf.mf_factor_numeric(fl, v)
        mf.mf_factor_numeric(fc, v)
        L = mf.mf_factor_export_L(fl, info["nnz_L"])
        D = mf.mf_factor_export_D(fl, n)
        G = mf.mf_factor_export_L(fc, info["nnz_L"])
        Lp, Li = mf.mf_symbolic_pattern(s)
        col = np.repeat(np.arange(n), np.diff(Lp))
        assert np.all(D > 0)
        assert orc.rel_fro(L * np.sqrt(D)[col], G) <= 1e-12
    finally:
        mf.mf_factor_free(fl)
        mf.mf_factor_free(fc)
        mf.mf_symbolic_free(s)
        mf.mf_destroy(h)


def test_ldlt_zero_pivot_reported(mf):
    # [[0, 1], [1, 0]] in its natural order: the first pivot is zero
    rp = np.array([0, 1, 2], dtype=np.int64)
    ci = np.array([1, 0], dtype=np.int32)
    v = np.array([1.0, 1.0])
    h = mf.mf_create()
    s = mf.mf_symbolic_analyze(h, rp, ci)
    f = mf.mf_factor_create_ldlt(h, s, 0)
    try:
        with pytest.raises(mf.MFError) as e:
            mf.mf_factor_numeric(f, v)
        assert e.value.code == mf.MF_ERR_NOT_SPD and e.value.column == 0
        assert "zero pivot" in str(e.value)
    finally:
        free(mf, h, s, f)
