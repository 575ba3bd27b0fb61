"""FastILU and FastSpTRSV on the GPU against the oracle (paper Sec. 6).

Out-of-place sweeps are deterministic: the GPU factors and solutions must
equal the oracle's sweeps element by element, up to the rounding of the
sums (the same products in the same order; fused multiply-adds on the GPU),
bar 1e-12 relative to the largest entry.  In-place (asynchronous) sweeps
vary from run to run, so they are checked by what the definition fixes: the
sweeps converge to the exact incomplete factors (the fixed point), bar 1e-9.
Workload: the 3D Q1 elasticity matrix (27-point stencil, 3 dofs per node)
of the paper's FastILU experiments, on 8^3 and 16^3 nodes."""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def mf():
    import torch
    assert torch.cuda.is_available()
    import paper_2506_05793_gb300 as m
    m.build()
    return m


def run(mf, rp, ci, v, K, **kw):
    h = mf.mf_create()
    ilu = mf.mf_ilu_symbolic(h, rp, ci, K)
    mf.mf_ilu_numeric(ilu, v, **kw)
    return h, ilu, mf.mf_ilu_export(ilu)


@pytest.mark.parametrize("N,K", [(8, 0), (8, 1), (8, 2), (8, 3), (16, 0), (16, 1)])
@pytest.mark.parametrize("sweeps,omega,shift,warmup", [(1, 1.0, 0.0, False), (2, 1.0, 0.0, False),
                                                        (3, 0.7, 0.1, False), (2, 1.0, 0.0, True)])
def test_sweeps_match_oracle(mf, orc, N, K, sweeps, omega, shift, warmup):
    rp, ci, v = gen.elasticity_3d(N)
    h, ilu, lu = run(mf, rp, ci, v, K, sweeps=sweeps, omega=omega, shift=shift, warmup=warmup)
    try:
        pat = orc.iluk_pattern(rp, ci, K)
        a = pat.values_of(rp, ci, v, shift=shift)
        want = orc.fastilu(pat, a, sweeps, omega=omega, warmup=warmup)
        scale = np.max(np.abs(want))
        assert np.max(np.abs(lu - want)) <= TOL * scale
        # FastSpTRSV with these factors, both triangles, and the
        # preconditioner application U^-1 L^-1 b
        n = len(rp) - 1
        b = gen.rhs(n, 1, seed=K)
        for upper in (0, 1):
            x = mf.mf_ilu_trsv(ilu, b, upper, 4, omega=0.9)
            xo = orc.fast_trsv(pat, want, b, upper, 4, omega=0.9)
            assert np.max(np.abs(x - xo)) <= 1e-11 * np.max(np.abs(xo))
        z = orc.fast_trsv(pat, want, b, 0, 5)
        xo = orc.fast_trsv(pat, want, z, 1, 5)
        x = mf.mf_ilu_apply(ilu, b, 5)
        assert np.max(np.abs(x - xo)) <= 1e-11 * np.max(np.abs(xo))
    finally:
        mf.mf_ilu_free(ilu)
        mf.mf_destroy(h)


@pytest.mark.parametrize("K", [0, 2])
def test_in_place_sweeps_reach_the_incomplete_factors(mf, orc, K):
    rp, ci, v = gen.elasticity_3d(8)
    h, ilu, lu = run(mf, rp, ci, v, K, sweeps=100, in_place=True)
    try:
        pat = orc.iluk_pattern(rp, ci, K)
        ex = orc.ilu_exact(pat, pat.values_of(rp, ci, v))
        assert np.max(np.abs(lu - ex)) <= 1e-9 * np.max(np.abs(ex))
    finally:
        mf.mf_ilu_free(ilu)
        mf.mf_destroy(h)


def test_device_vectors_and_edge_cases(mf, orc):
    import torch
    # n = 1 and a diagonal matrix: L = I, U = D, one sweep is exact
    for n in (1, 7):
        rp = np.arange(n + 1, dtype=np.int64)
        ci = np.arange(n, dtype=np.int32)
        v = np.arange(1, n + 1, dtype=np.float64) + 1.0
        h, ilu, lu = run(mf, rp, ci, v, 2, sweeps=1)
        assert np.array_equal(lu, v)
        b = np.ones(n)
        assert np.allclose(mf.mf_ilu_apply(ilu, b, 1), b / v, rtol=1e-15)
        mf.mf_ilu_free(ilu)
        mf.mf_destroy(h)
    rp, ci, v = gen.elasticity_3d(6)
    h, ilu, lu = run(mf, rp, ci, torch.from_numpy(v).cuda(), 1, sweeps=2)
    try:
        b = gen.rhs(len(rp) - 1, 1, seed=1)
        xh = mf.mf_ilu_apply(ilu, b, 3)
        xd = mf.mf_ilu_apply(ilu, torch.from_numpy(b).cuda(), 3)
        assert np.array_equal(xd.cpu().numpy(), xh)
    finally:
        mf.mf_ilu_free(ilu)
        mf.mf_destroy(h)
