"""Batched subdomains (many uneven matrices in one factorization) and the
autotuner.  The batch is the block-diagonal union analysed as one forest; a
subdomain's factor must be bitwise the same alone and inside the batch, and
every subdomain's solution must meet the backward-error bar."""
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


def small_batch(count=10, seed=11):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        a, b, c = (int(x) for x in rng.integers(5, 15, size=3))
        rp, ci, v = gen.laplacian_3d(a, b, c)
        out.append((rp, ci, v, gen.nd_perm((a, b, c))))
    return out


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_factor_equals_individual(mf, orc, prec):
    mats = small_batch()
    h = mf.mf_create()
    sb = mf.mf_symbolic_analyze_batch(h, [(rp, ci, pm) for rp, ci, v, pm in mats])
    fb = mf.mf_factor_create(h, sb, prec)
    vals = np.concatenate([v for _, _, v, _ in mats])
    mf.mf_factor_numeric(fb, vals)
    Lb = mf.mf_factor_export_L(fb, mf.mf_symbolic_get_info(sb)["nnz_L"])
    pos = 0
    for rp, ci, v, pm in mats:
        s = mf.mf_symbolic_analyze(h, rp, ci, pm)
        f = mf.mf_factor_create(h, s, prec)
        mf.mf_factor_numeric(f, v)
        L = mf.mf_factor_export_L(f, mf.mf_symbolic_get_info(s)["nnz_L"])
        assert np.array_equal(Lb[pos:pos + len(L)], L)  # bitwise, alone vs in the batch
        pos += len(L)
        mf.mf_factor_free(f)
        mf.mf_symbolic_free(s)
    assert pos == len(Lb)
    # solve of the whole batch, backward error per subdomain
    rpb, cib, vb = gen.block_diag_csr([(rp, ci, v) for rp, ci, v, _ in mats])
    n = len(rpb) - 1
    B = gen.rhs(n, 2, seed=5)
    if prec == 0:
        X = mf.mf_solve(fb, B)
    else:
        X, rep = mf.mf_solve_refined(fb, B, tol=1e-13)
        assert rep["fell_back"] == 0
    off = 0
    for rp, ci, v, pm in mats:
        m = len(rp) - 1
        assert orc.berr(rp, ci, v, X[off:off + m], B[off:off + m]) <= 1e-13
        off += m
    mf.mf_factor_free(fb)
    mf.mf_symbolic_free(sb)
    mf.mf_destroy(h)


@pytest.mark.parametrize("prec", [0, 1])
def test_autotune_returns_working_options_and_caches(mf, orc, prec):
    """The tuned options (relaxation, small-front limit, queue and the
    per-bucket trailing-update tiles) factor the matrix within the parity
    bars; a second call on the same pattern is served from the cache (no
    factorization: far faster); the analysis records the tuned tiles."""
    import time
    rp, ci, v, perm, _ = gen.config3(24)
    h = mf.mf_create()
    t0 = time.perf_counter()
    best, ms = mf.mf_autotune(h, rp, ci, perm, v, prec=prec, reps=1)
    t1 = time.perf_counter()
    best2, ms2 = mf.mf_autotune(h, rp, ci, perm, v, prec=prec, reps=1)
    t2 = time.perf_counter()
    assert ms > 0 and ms2 == ms and list(best2.update_tile) == list(best.update_tile)
    assert (t2 - t1) < 0.2 * (t1 - t0)
    assert best.small_front_max in (32, 64, 128) and best.relax in (0, 1)
    assert all(c in (0, 1, 2, 3, 4) for c in best.update_tile)
    assert any(c != 0 for c in best.update_tile)  # buckets with large fronts were tuned
    h2 = mf.mf_create(best)
    s = mf.mf_symbolic_analyze(h2, rp, ci, perm)
    assert list(mf.mf_symbolic_options(s).update_tile) == list(best.update_tile)
    f = mf.mf_factor_create(h2, s, prec)
    mf.mf_factor_numeric(f, v)
    B = gen.rhs(len(rp) - 1, 1, seed=2)
    if prec == 1:
        X, rep = mf.mf_solve_refined(f, B, tol=1e-13)
    else:
        X = mf.mf_solve(f, B)
    assert orc.berr(rp, ci, v, X, B) <= 1e-13
    mf.mf_factor_free(f)
    mf.mf_symbolic_free(s)
    mf.mf_destroy(h2)
    mf.mf_destroy(h)


@pytest.mark.parametrize("tiles", [(4, 4, 4, 4), (2, 2, 2, 2), (1, 1, 1, 1), (4, 2, 3, 1)])
@pytest.mark.parametrize("prec", [0, 1])
def test_every_update_tile_matches_oracle(mf, orc, tiles, prec):
    """FMA 32 / 64 / 128 and tensor-core trailing updates, alone and mixed
    per front-size bucket, against the oracle's factor."""
    # fronts of up to about 600 rows: buckets 0 and 1
    rp, ci, v = gen.q1_extruded(60, 40, 4, seed=2)
    perm = gen.nd_perm((61, 41, 5), split_axes=(0, 1), dofs=2)
    opt = mf.mf_options_default()
    for b in range(4):
        opt.update_tile[b] = tiles[b]
    h = mf.mf_create(opt)
    s = mf.mf_symbolic_analyze(h, rp, ci, perm)
    info = mf.mf_symbolic_get_info(s)
    f = mf.mf_factor_create(h, s, prec)
    try:
        mf.mf_factor_numeric(f, v)
        L = mf.mf_factor_export_L(f, info["nnz_L"])
        F = orc.factor(rp, ci, v, perm)
        assert orc.rel_fro(L, F.Lx) <= (1e-11 if prec == 0 else 5e-4)
    finally:
        mf.mf_factor_free(f)
        mf.mf_symbolic_free(s)
        mf.mf_destroy(h)


@pytest.mark.parametrize("small_max", [32, 64])
def test_small_front_limits_agree(mf, orc, small_max):
    """Different one-CTA/tiled splits give the same factor to rounding."""
    rp, ci, v, perm, _ = gen.config3(14)
    F = orc.factor(rp, ci, v, perm)
    opt = mf.mf_options_default()
    opt.small_front_max = small_max
    h = mf.mf_create(opt)
    s = mf.mf_symbolic_analyze(h, rp, ci, perm)
    f = mf.mf_factor_create(h, s, 0)
    mf.mf_factor_numeric(f, v)
    L = mf.mf_factor_export_L(f, mf.mf_symbolic_get_info(s)["nnz_L"])
    assert orc.rel_fro(L, F.Lx) <= 1e-11
    mf.mf_factor_free(f)
    mf.mf_symbolic_free(s)
    mf.mf_destroy(h)
