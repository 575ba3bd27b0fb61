"""SpTRSV variants (Sec. 5) against the oracle and against each other:
variant 2 solves the large fronts' pivot blocks as a product with the kept
inverses of their diagonal blocks; variant 3 (partitioned inverse) makes each
level one product with [L11^{-1}; -L21 L11^{-1}], computed after the
factorization; variant 4 stores that inverse for every front as one sparse
matrix per level and sweep and solves on the global vector (one launch per
level and sweep, no front work vectors, no waits)."""
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


@pytest.mark.parametrize("case", ["dense_333", "dense_150", "lap3d_jump_20", "q1_14x12x4",
                                  "lap2d_301x157"])
@pytest.mark.parametrize("nrhs", [1, 5, 9])
def test_partitioned_inverse_matches_oracle_and_substitution(mf, orc, case, nrhs):
    rp, ci, v, perm = case_matrix(case)
    n = len(rp) - 1
    B = gen.rhs(n, nrhs, seed=21 + nrhs)
    X3, info3 = solve_with(mf, 3, rp, ci, v, perm, B)
    X1, info1 = solve_with(mf, 1, rp, ci, v, perm, B)
    # the partitioned inverse takes memory: the variant really ran
    assert info3["factor_bytes_fp64"] > info1["factor_bytes_fp64"]
    assert orc.berr(rp, ci, v, X3, B) <= BERR
    F = orc.factor(rp, ci, v, perm)
    Xo = orc.solve(F, B, perm)
    scale = np.max(np.abs(Xo))
    assert np.max(np.abs(X3 - Xo)) <= 1e-9 * scale
    assert np.max(np.abs(X3 - X1)) <= 1e-9 * scale


def test_partitioned_inverse_repeated_factorizations(mf, orc):
    """The inverse pass runs inside the factorization's CUDA graph: a second
    numeric factorization with other values must refresh it."""
    rp, ci, v, perm = case_matrix("lap3d_jump_20")
    n = len(rp) - 1
    B = gen.rhs(n, 2, seed=8)
    opt = mf.mf_options_default()
    opt.sptrsv = 3
    h = mf.mf_create(opt)
    s = mf.mf_symbolic_analyze(h, rp, ci, perm)
    f = mf.mf_factor_create(h, s, mf.MF_FP64)
    try:
        for scale in (1.0, 3.0):
            v2 = v * scale
            mf.mf_factor_numeric(f, v2)
            X = mf.mf_solve(f, B)
            assert orc.berr(rp, ci, v2, X, B) <= BERR
    finally:
        mf.mf_factor_free(f)
        mf.mf_symbolic_free(s)
        mf.mf_destroy(h)


@pytest.mark.parametrize("case", ["dense_333", "dense_150", "lap3d_jump_20", "q1_14x12x4",
                                  "lap2d_301x157"])
@pytest.mark.parametrize("nrhs", [1, 3, 9, 33])
def test_level_matrix_variant_matches_oracle_and_substitution(mf, orc, case, nrhs):
    rp, ci, v, perm = case_matrix(case)
    n = len(rp) - 1
    B = gen.rhs(n, nrhs, seed=31 + nrhs)
    X4, info4 = solve_with(mf, 4, rp, ci, v, perm, B)
    X1, info1 = solve_with(mf, 1, rp, ci, v, perm, B)
    X3, info3 = solve_with(mf, 3, rp, ci, v, perm, B)
    # P and its transpose for every front: more memory than variant 3
    assert info4["factor_bytes_fp64"] > info3["factor_bytes_fp64"]
    assert orc.berr(rp, ci, v, X4, B) <= BERR
    F = orc.factor(rp, ci, v, perm)
    Xo = orc.solve(F, B, perm)
    scale = np.max(np.abs(Xo))
    assert np.max(np.abs(X4 - Xo)) <= 1e-9 * scale
    assert np.max(np.abs(X4 - X1)) <= 1e-9 * scale


def test_level_matrix_variant_refactor_and_noalloc(mf, orc):
    """The inverses and their transposes are part of the factorization's
    graph: a second numeric factorization with other values refreshes them;
    the no-allocation entry point runs the same per-level products."""
    import torch
    rp, ci, v, perm = case_matrix("q1_14x12x4")
    n = len(rp) - 1
    B = gen.rhs(n, 2, seed=8)
    opt = mf.mf_options_default()
    opt.sptrsv = 4
    h = mf.mf_create(opt)
    s = mf.mf_symbolic_analyze(h, rp, ci, perm)
    mf.mf_symbolic_check(s)
    f = mf.mf_factor_create(h, s, mf.MF_FP64)
    try:
        for scale in (1.0, 3.0):
            v2 = v * scale
            mf.mf_factor_numeric(f, v2)
            X = mf.mf_solve(f, B)
            assert orc.berr(rp, ci, v2, X, B) <= BERR
            Bd = torch.from_numpy(np.ascontiguousarray(B.T)).cuda().t()
            Xd = torch.from_numpy(np.zeros((2, n))).cuda().t()
            mf.mf_solve_noalloc(f, Bd, Xd)
            mf.mf_solve_check(f)
            assert np.array_equal(Xd.cpu().numpy(), X)
    finally:
        mf.mf_factor_free(f)
        mf.mf_symbolic_free(s)
        mf.mf_destroy(h)


@pytest.mark.parametrize("variant", [2, 3, 4])
def test_inverse_variant_fp32_refinement(mf, orc, variant):
    rp, ci, v, perm = case_matrix("lap3d_jump_20")
    n = len(rp) - 1
    B = gen.rhs(n, 3, seed=5)
    opt = mf.mf_options_default()
    opt.sptrsv = variant
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
