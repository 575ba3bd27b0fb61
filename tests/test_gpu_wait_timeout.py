"""Failure detection of the solve's device waits, without a GPU fault: a
bounded wait on a flag that nothing sets gives up, records MF_ERR_TIMEOUT in
the status word, and the context stays usable for a factor and a solve."""
import numpy as np
import pytest

import gen


@pytest.mark.gpu
def test_bounded_wait_reports_timeout_and_device_stays_usable():
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
    n = len(rp) - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    anorm = np.max(np.bincount(rows, weights=np.abs(v), minlength=n))
    r = b - gen.csr_matvec(rp, ci, v, x)
    assert np.max(np.abs(r)) / (anorm * np.max(np.abs(x)) + np.max(np.abs(b))) <= 1e-13
    mf.mf_factor_free(f)
    mf.mf_symbolic_free(s)
    mf.mf_destroy(h)


def test_wait_probe_rejects_bad_argument():
    import paper_2506_05793_gb300 as mf
    mf.build()
    assert mf.mf_diag_wait_timeout(0) == mf.MF_ERR_INVALID
