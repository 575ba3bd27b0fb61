"""mf_solve_noalloc: the solve for callers that must not allocate device
memory on their solve path.

On a fresh factor (no solve has run, so no solve work memory exists) two
calls in a row -- the second spanning several chunks of right-hand sides --
must leave the factor's solve work memory at zero bytes (nothing was
allocated behind the caller's back), meet the backward-error bar against the
oracle's definition, and give bit for bit the values of mf_solve, which runs
the same kernels on memory it allocates itself.  Problems whose work does not
fit the library's fixed array are refused.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mf():
    import torch
    assert torch.cuda.is_available()
    import paper_2506_05793_gb300 as m
    m.build()
    return m


def device_rhs(B):
    import torch
    return torch.from_numpy(np.ascontiguousarray(B.T)).cuda().t()


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_matches_oracle_and_solve_twice(mf, orc, prec):
    import torch
    rp, ci, v, perm, _ = gen.config3(20)
    n = len(rp) - 1
    h = mf.mf_create()
    s = mf.mf_symbolic_analyze(h, rp, ci, perm)
    f = mf.mf_factor_create(h, s, prec)
    mf.mf_factor_numeric(f, v)
    bar = 1e-13 if prec == 0 else 1e-5  # FP32 factor: about n * u_32 backward error
    out = []
    for call, nrhs in enumerate((3, 40)):  # two calls in a row; 40 spans chunks
        B = gen.rhs(n, nrhs, seed=11 + call)
        Bd = device_rhs(B)
        X = device_rhs(np.zeros((n, nrhs)))
        mf.mf_solve_noalloc(f, Bd, X)
        mf.mf_solve_check(f)
        assert mf.mf_factor_solve_work_bytes(f) == 0
        x = X.cpu().numpy()
        assert orc.berr(rp, ci, v, x, B) <= bar
        out.append((Bd, x))
    torch.cuda.synchronize()
    for Bd, x in out:
        ref = mf.mf_solve(f, Bd).cpu().numpy()
        assert np.array_equal(x, ref)
    assert mf.mf_factor_solve_work_bytes(f) > 0  # mf_solve allocated its own
    mf.mf_factor_free(f)
    mf.mf_symbolic_free(s)
    mf.mf_destroy(h)


def test_noalloc_rejects_oversize(mf):
    n = 6_000_000  # (n + front work) * 8 bytes > 32 MiB for one RHS
    rp, ci, v = gen.laplacian_1d(n)
    h = mf.mf_create()
    s = mf.mf_symbolic_analyze(h, rp, ci)
    f = mf.mf_factor_create(h, s, 0)
    mf.mf_factor_numeric(f, v)
    Bd = device_rhs(np.ones((n, 1)))
    X = device_rhs(np.zeros((n, 1)))
    with pytest.raises(mf.MFError) as e:
        mf.mf_solve_noalloc(f, Bd, X)
    assert e.value.code == mf.MF_ERR_INVALID
    assert "scratch" in str(e.value)
    mf.mf_factor_free(f)
    mf.mf_symbolic_free(s)
    mf.mf_destroy(h)
