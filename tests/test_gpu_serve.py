"""Serving loop: continuous batching of factor and solve requests with
resident factors, admission under a device budget, p50/p99 latency.  Every
result must be the same alone and in the mix (bitwise: the kernels use no
atomics in sums and the schedule of a front does not depend on the mix)."""
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


def problems():
    out = []
    rng = np.random.default_rng(21)
    for i in range(6):
        a, b, c = (int(x) for x in rng.integers(6, 16, size=3))
        rp, ci, v = gen.laplacian_3d(a, b, c, jump_block=4 if i % 2 else None, seed=i)
        out.append((rp, ci, v, gen.nd_perm((a, b, c))))
    return out


def test_mix_equals_alone_and_meets_berr(mf, orc):
    probs = problems()
    h = mf.mf_create()
    syms = [mf.mf_symbolic_analyze(h, rp, ci, pm) for rp, ci, v, pm in probs]
    precs = [0, 1, 0, 1, 0, 1]
    rhs = [gen.rhs(len(p[0]) - 1, 2, seed=40 + i) for i, p in enumerate(probs)]
    rhs2 = [gen.rhs(len(p[0]) - 1, 3, seed=60 + i) for i, p in enumerate(probs)]
    # alone: one worker, one request at a time
    sv = mf.mf_server_create(h, workers=1)
    alone, alone2 = [], []
    for i, (rp, ci, v, pm) in enumerate(probs):
        req, fid, X = mf.mf_server_submit_factor(sv, syms[i], v, precs[i], rhs[i])
        assert mf.mf_server_wait(sv, req)[0] == 0
        req2, X2 = mf.mf_server_submit_solve(sv, fid, rhs2[i])
        assert mf.mf_server_wait(sv, req2)[0] == 0
        alone.append(X.copy())
        alone2.append(X2.copy())
        mf.mf_server_release_factor(sv, fid)
    mf.mf_server_free(sv)
    # mix: four workers, everything queued at once, solve-only requests queued
    # right behind their factor requests
    sv = mf.mf_server_create(h, workers=4)
    reqs = []
    for i, (rp, ci, v, pm) in enumerate(probs):
        req, fid, X = mf.mf_server_submit_factor(sv, syms[i], v, precs[i], rhs[i])
        req2, X2 = mf.mf_server_submit_solve(sv, fid, rhs2[i])
        reqs.append((req, X, req2, X2, fid))
    for i, (req, X, req2, X2, fid) in enumerate(reqs):
        assert mf.mf_server_wait(sv, req)[0] == 0
        assert mf.mf_server_wait(sv, req2)[0] == 0
        assert np.array_equal(X, alone[i])
        assert np.array_equal(X2, alone2[i])
        rp, ci, v, pm = probs[i]
        assert orc.berr(rp, ci, v, X, rhs[i]) <= 1e-13
        assert orc.berr(rp, ci, v, X2, rhs2[i]) <= 1e-13
    st = mf.mf_server_get_stats(sv)
    assert st["completed"] == 12 and st["failed"] == 0
    assert 0 < st["p50_ms"] <= st["p99_ms"]
    mf.mf_server_free(sv)
    for s in syms:
        mf.mf_symbolic_free(s)
    mf.mf_destroy(h)


def test_budget_admission_and_release(mf):
    """With a budget for about one factor, requests are admitted one at a time
    as factors are released; all complete."""
    probs = problems()[:3]
    h = mf.mf_create()
    syms = [mf.mf_symbolic_analyze(h, rp, ci, pm) for rp, ci, v, pm in probs]
    biggest = max(mf.mf_symbolic_get_info(s)["factor_bytes_fp64"] for s in syms)
    sv = mf.mf_server_create(h, workers=3, budget_bytes=int(biggest * 1.5))
    subs = []
    for i, (rp, ci, v, pm) in enumerate(probs):
        req, fid, X = mf.mf_server_submit_factor(sv, syms[i], v, 0, gen.rhs(len(rp) - 1, 1))
        subs.append((req, fid))
    for req, fid in subs:
        assert mf.mf_server_wait(sv, req)[0] == 0
        mf.mf_server_release_factor(sv, fid)
    st = mf.mf_server_get_stats(sv)
    assert st["peak_resident_bytes"] <= int(biggest * 1.5)
    assert st["resident_bytes"] == 0
    with pytest.raises(mf.MFError):
        tiny = mf.mf_server_create(h, workers=1, budget_bytes=16)
        try:
            mf.mf_server_submit_factor(tiny, syms[0], probs[0][2], 0)
        finally:
            mf.mf_server_free(tiny)
    mf.mf_server_free(sv)
    for s in syms:
        mf.mf_symbolic_free(s)
    mf.mf_destroy(h)
