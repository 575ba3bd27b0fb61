"""SpTRSV variant 2 (Sec. 5): the solve of the large fronts' pivot blocks as a
product with the inverses of the diagonal blocks, kept from the
factorization, against the oracle and against the substitution variant."""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu

BERR = 1e-13


@pytest.fixture(scope="module")
def mf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2506_05793_gb300 as m
    m.build()
    return m


def case_matrix(case):
    if case.startswith("dense"):
        import scipy.sparse as sp
        n = int(case.split("_")[1])
        rng = np.random.default_rng(n)
        M = rng.standard_normal((n, n))
        A = sp.csr_matrix(M @ M.T + n * np.eye(n))
        return A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data, None
    if case == "lap3d_jump_20":
        rp, ci, v, perm, _ = gen.config3(20)
        return rp, ci, v, perm
    if case == "q1_14x12x4":
        rp, ci, v = gen.q1_extruded(14, 12, 4, seed=3)
        return rp, ci, v, gen.nd_perm((15, 13, 5), split_axes=(0, 1), dofs=2)
    rp, ci, v = gen.laplacian_2d(301, 157)
    return rp, ci, v, gen.nd_perm((301, 157))


def solve_with(mf, variant, rp, ci, v, perm, B, prec=0):
    opt = mf.mf_options_default()
    opt.sptrsv = variant
    h = mf.mf_create(opt)
    s = mf.mf_symbolic_analyze(h, rp, ci, perm)
    f = mf.mf_factor_create(h, s, prec)
    try:
        mf.mf_factor_numeric(f, v)
        X = mf.mf_solve(f, B)
        return X, mf.mf_symbolic_get_info(s)
    finally:
        mf.mf_factor_free(f)
        mf.mf_symbolic_free(s)
        mf.mf_destroy(h)


@pytest.mark.parametrize("case", ["dense_333", "lap3d_jump_20", "q1_14x12x4", "lap2d_301x157"])
@pytest.mark.parametrize("nrhs", [1, 9])
def test_inverse_variant_matches_oracle_and_substitution(mf, orc, case, nrhs):
    rp, ci, v, perm = case_matrix(case)
    n = len(rp) - 1
    B = gen.rhs(n, nrhs, seed=11 + nrhs)
    X2, info2 = solve_with(mf, 2, rp, ci, v, perm, B)
    X1, info1 = solve_with(mf, 1, rp, ci, v, perm, B)
    # the kept inverses take memory: the variant really ran
    assert info2["factor_bytes_fp64"] > info1["factor_bytes_fp64"]
    assert orc.berr(rp, ci, v, X2, B) <= BERR
    F = orc.factor(rp, ci, v, perm)
    Xo = orc.solve(F, B, perm)
    scale = np.max(np.abs(Xo))
    assert np.max(np.abs(X2 - Xo)) <= 1e-9 * scale
    assert np.max(np.abs(X2 - X1)) <= 1e-9 * scale


def test_inverse_variant_fp32_refinement(mf, orc):
    rp, ci, v, perm = case_matrix("lap3d_jump_20")
    n = len(rp) - 1
    B = gen.rhs(n, 3, seed=5)
    opt = mf.mf_options_default()
    opt.sptrsv = 2
    h = mf.mf_create(opt)
    s = mf.mf_symbolic_analyze(h, rp, ci, perm)
    f = mf.mf_factor_create(h, s, mf.MF_FP32)
    try:
        mf.mf_factor_numeric(f, v)
        X, rep = mf.mf_solve_refined(f, B, tol=BERR, max_iter=30)
        assert rep["berr"] <= BERR and rep["fell_back"] == 0
        assert orc.berr(rp, ci, v, X, B) <= BERR
    finally:
        mf.mf_factor_free(f)
        mf.mf_symbolic_free(s)
        mf.mf_destroy(h)
