"""Failure detection of the solve's device waits, without a GPU fault.

(i) A bounded wait on a flag that nothing sets gives up, records
MF_ERR_TIMEOUT, and the context stays usable for a factor and a solve.
(ii) With a very short bound (one poll) the flag waits of a real solve run
out: the solve reports MF_ERR_TIMEOUT (host path: the call itself; device
and no-allocation paths: mf_solve_check), and once the default bound is
back the next solve on the same factor is clean and correct -- the record
belongs to one call and does not stick to the factor.  Nothing here faults
or hangs the GPU: a wait that runs out lets its kernel finish with wrong
values, which the status reports."""
import numpy as np
import pytest

import gen


@pytest.mark.gpu
def test_bounded_wait_reports_timeout_and_device_stays_usable(orc):
    import paper_2506_05793_gb300 as mf
    mf.build()
    assert mf.mf_diag_wait_timeout(1 << 14) == mf.MF_ERR_TIMEOUT
    assert "gave up" in mf.lib().mf_last_error_string().decode()
    rp, ci, v, perm, b = gen.config1()
    h = mf.mf_create()
    s = mf.mf_symbolic_analyze(h, rp, ci, perm)
    f = mf.mf_factor_create(h, s, mf.MF_FP64)
    mf.mf_factor_numeric(f, v)
    x = mf.mf_solve(f, b)
    assert orc.berr(rp, ci, v, x, b) <= 1e-13
    mf.mf_factor_free(f)
    mf.mf_symbolic_free(s)
    mf.mf_destroy(h)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [0, 1])
def test_solve_timeout_is_reported_and_cleared(orc, prec):
    import torch
    import paper_2506_05793_gb300 as mf
    mf.build()
    # top separator of 32^2 columns: large fronts whose 64-row pivot blocks
    # are chained by flags in both sweeps (SpTRSV variant 2, the default)
    N = 32
    rp, ci, v = gen.laplacian_3d(N)
    perm = gen.nd_perm((N, N, N))
    n = len(rp) - 1
    b = gen.rhs(n, 1, seed=5)
    h = mf.mf_create()
    s = mf.mf_symbolic_analyze(h, rp, ci, perm)
    f = mf.mf_factor_create(h, s, prec)
    mf.mf_factor_numeric(f, v)
    bar = 1e-13 if prec == 0 else 1e-5
    try:
        mf.mf_factor_set_wait_limit(f, 1)
        # host pointers: the call reports the timeout
        with pytest.raises(mf.MFError) as e:
            mf.mf_solve(f, b)
        assert e.value.code == mf.MF_ERR_TIMEOUT and "solve" in str(e.value)
        # device pointers and the no-allocation entry point: mf_solve_check
        bd = torch.from_numpy(b).cuda()
        xd = torch.empty_like(bd)
        mf.mf_solve(f, bd, xd)
        with pytest.raises(mf.MFError) as e:
            mf.mf_solve_check(f)
        assert e.value.code == mf.MF_ERR_TIMEOUT
        mf.mf_solve_noalloc(f, bd, xd)
        with pytest.raises(mf.MFError) as e:
            mf.mf_solve_check(f)
        assert e.value.code == mf.MF_ERR_TIMEOUT
        # the factorization itself is unaffected
        mf.mf_factor_check(f)
        # default bound again: every path is clean and the solution correct
        mf.mf_factor_set_wait_limit(f, 0)
        x = mf.mf_solve(f, b)
        assert orc.berr(rp, ci, v, x, b) <= bar
        mf.mf_solve(f, bd, xd)
        mf.mf_solve_check(f)
        assert orc.berr(rp, ci, v, xd.cpu().numpy(), b) <= bar
        mf.mf_solve_noalloc(f, bd, xd)
        mf.mf_solve_check(f)
        assert orc.berr(rp, ci, v, xd.cpu().numpy(), b) <= bar
    finally:
        mf.mf_factor_free(f)
        mf.mf_symbolic_free(s)
        mf.mf_destroy(h)


def test_wait_probe_rejects_bad_argument():
    import paper_2506_05793_gb300 as mf
    mf.build()
    assert mf.mf_diag_wait_timeout(0) == mf.MF_ERR_INVALID


def test_wait_limit_rejects_bad_argument():
    import paper_2506_05793_gb300 as mf
    mf.build()
    with pytest.raises(mf.MFError) as e:
        mf.mf_factor_set_wait_limit(None, 1)
    assert e.value.code == mf.MF_ERR_INVALID
