"""Parity at the benchmark's full sizes, with the options bench.py times
(CUDA graph, tensor cores for FP32, kept diagonal-block inverses, lookahead).

The oracle cannot factor these matrices whole in test time, so the checks
are: (i) the leading columns of L (a descendant-closed set the oracle
factors exactly) element by element, (ii) properties that hold at any size:
the closed-form log-determinant of the 7-point Laplacian and the normwise
backward error of the solves (FP64 and FP32 + refinement) against 1e-13."""
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


def berr(rp, ci, v, X, B):
    """max over columns of ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf)."""
    n = len(rp) - 1
    X = X.reshape(n, -1)
    B = B.reshape(n, -1)
    rows = np.repeat(np.arange(n), np.diff(rp))
    anorm = np.max(np.bincount(rows, weights=np.abs(v), minlength=n))
    worst = 0.0
    for r in range(X.shape[1]):
        res = B[:, r] - np.bincount(rows, weights=v * X[ci, r], minlength=n)
        den = anorm * np.max(np.abs(X[:, r])) + np.max(np.abs(B[:, r]))
        worst = max(worst, float(np.max(np.abs(res)) / den))
    return worst


def laplacian_logdet(N):
    """log det of the 7-point Dirichlet Laplacian on N^3 (eigenvalues are
    sums over the axes of 2 - 2 cos(pi i / (N + 1)))."""
    lam = 2.0 - 2.0 * np.cos(np.pi * np.arange(1, N + 1) / (N + 1))
    grid = lam[:, None, None] + lam[None, :, None] + lam[None, None, :]
    return float(np.sum(np.log(grid)))


def test_laplacian_64_leading_columns_logdet_and_solve(mf, orc):
    N = 64
    rp, ci, v = gen.laplacian_3d(N)
    perm = gen.nd_perm((N, N, N))
    n = len(rp) - 1
    h = mf.mf_create()
    s = mf.mf_symbolic_analyze(h, rp, ci, perm)
    info = mf.mf_symbolic_get_info(s)
    f = mf.mf_factor_create(h, s, mf.MF_FP64)
    try:
        mf.mf_factor_numeric(f, v)
        Lx = mf.mf_factor_export_L(f, info["nnz_L"])
        Lp, Li = mf.mf_symbolic_pattern(s)
        # (i) the first J columns of the elimination order are descendant
        # closed: the oracle factors them exactly
        J = 20000
        in_s = np.zeros(n, dtype=np.uint8)
        in_s[:J] = 1
        F = orc.factor(rp, ci, v, perm, in_s=in_s)
        assert F.bad_col == -1
        assert np.array_equal(F.Lp[:J + 1], Lp[:J + 1])
        assert np.array_equal(F.Li[:F.Lp[J]], Li[:Lp[J]])
        ref = F.Lx[:F.Lp[J]]
        got = Lx[:Lp[J]]
        assert np.linalg.norm(got - ref) <= 1e-11 * np.linalg.norm(ref)
        # (ii) log det A = 2 sum log L_jj (rows sorted: the diagonal leads)
        diag = Lx[Lp[:-1]]
        assert np.all(Li[Lp[:-1]] == np.arange(n))
        ld = 2.0 * float(np.sum(np.log(diag)))
        ref_ld = laplacian_logdet(N)
        assert abs(ld - ref_ld) <= 1e-11 * abs(ref_ld)
        B = gen.rhs(n, 1, seed=1)
        X = mf.mf_solve(f, B)
        assert berr(rp, ci, v, X, B) <= BERR
    finally:
        mf.mf_factor_free(f)
        mf.mf_symbolic_free(s)
        mf.mf_destroy(h)


def test_q1_256x256x10_fp64_and_fp32_refinement(mf):
    rp, ci, v, perm, b = gen.config2()
    h = mf.mf_create()
    s = mf.mf_symbolic_analyze(h, rp, ci, perm)
    f64 = mf.mf_factor_create(h, s, mf.MF_FP64)
    f32 = mf.mf_factor_create(h, s, mf.MF_FP32)
    try:
        mf.mf_factor_numeric(f64, v)
        x = mf.mf_solve(f64, b)
        assert berr(rp, ci, v, x, b) <= BERR
        mf.mf_factor_numeric(f32, v)
        x2, rep = mf.mf_solve_refined(f32, b, tol=BERR, max_iter=30)
        assert rep["fell_back"] == 0 and rep["berr"] <= BERR
        assert berr(rp, ci, v, x2, b) <= BERR
        # FP32 + refinement reaches the FP64 solution to the conditioning
        assert np.max(np.abs(x2 - x)) <= 1e-8 * np.max(np.abs(x))
    finally:
        mf.mf_factor_free(f64)
        mf.mf_factor_free(f32)
        mf.mf_symbolic_free(s)
        mf.mf_destroy(h)


def test_jump_96_fp32_refinement_8_rhs(mf):
    rp, ci, v, perm, B = gen.config3(96, nrhs=8)
    h = mf.mf_create()
    s = mf.mf_symbolic_analyze(h, rp, ci, perm)
    f = mf.mf_factor_create(h, s, mf.MF_FP32)
    try:
        mf.mf_factor_numeric(f, v)
        X, rep = mf.mf_solve_refined(f, B, tol=BERR, max_iter=30)
        assert rep["fell_back"] == 0 and rep["berr"] <= BERR
        assert berr(rp, ci, v, X, B) <= BERR
    finally:
        mf.mf_factor_free(f)
        mf.mf_symbolic_free(s)
        mf.mf_destroy(h)


def test_batch_512_boxes_fp32_refinement(mf):
    mats, _ = gen.box_batch(512, 8, 48, seed=4)
    rp, ci, v = gen.block_diag_csr([(a, b, c) for a, b, c, _ in mats])
    n = len(rp) - 1
    h = mf.mf_create()
    s = mf.mf_symbolic_analyze_batch(h, [(a, b, p) for a, b, c, p in mats])
    f = mf.mf_factor_create(h, s, mf.MF_FP32)
    try:
        mf.mf_factor_numeric(f, v)
        B = gen.rhs(n, 1, seed=3)
        X, rep = mf.mf_solve_refined(f, B, tol=BERR, max_iter=30)
        assert rep["fell_back"] == 0 and rep["berr"] <= BERR
        assert berr(rp, ci, v, X, B) <= BERR
    finally:
        mf.mf_factor_free(f)
        mf.mf_symbolic_free(s)
        mf.mf_destroy(h)
