"""mf_solve_noalloc: the solve for callers that must not allocate device
memory on their solve path.  It must agree with mf_solve (same kernels, work
memory from the library's fixed device array) on consecutive calls, and it
must refuse problems whose work does not fit that array.

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
def test_noalloc_matches_solve_twice(mf, prec):
    import torch
    rp, ci, v, perm, _ = gen.config3(20)
    n = len(rp) - 1
    h = mf.mf_create()
    s = mf.mf_symbolic_analyze(h, rp, ci, perm)
    f = mf.mf_factor_create(h, s, prec)
    mf.mf_factor_numeric(f, v)
    tol = 1e-13 if prec == 0 else 1e-6
    for call, nrhs in enumerate((3, 40)):  # two calls in a row; 40 spans chunks
        B = gen.rhs(n, nrhs, seed=11 + call)
        Bd = device_rhs(B)
        Xref = mf.mf_solve(f, Bd)
        X = device_rhs(np.zeros((n, nrhs)))
        mf.mf_solve_noalloc(f, Bd, X)
        torch.cuda.synchronize()
        a, r = X.cpu().numpy(), Xref.cpu().numpy()
        assert np.max(np.abs(a - r)) <= tol * np.max(np.abs(r))
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
