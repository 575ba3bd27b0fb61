"""The persistent small-front queue: every small front whose subtree holds
only small fronts is factored in one launch, each front waiting (bounded)
for its children's completion flags instead of a level barrier.

* The factor is bit for bit the one the per-level launches give (each
  front's arithmetic is the same; only the order of independent fronts
  changes), and matches the oracle.
* The small-front work of a batch of boxes collapses into one launch.
* Failure detection without a fault: with the first tickets skipped, the
  waits on flags that nothing raises give up after the factor's bound,
  MF_ERR_TIMEOUT is reported, and the next factorization is clean."""
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


def batch_case():
    mats, _ = gen.box_batch(12, 8, 24, seed=4)
    rp, ci, v = gen.block_diag_csr([(a, b, c) for a, b, c, _ in mats])
    offs = np.cumsum([0] + [len(m[0]) - 1 for m in mats])
    perm = np.concatenate([m[3] + o for m, o in zip(mats, offs[:-1])]).astype(np.int32)
    return rp, ci, v, perm


def factor_L(mf, rp, ci, v, perm, prec, queue):
    opt = mf.mf_options_default()
    opt.small_queue = queue
    h = mf.mf_create(opt)
    s = mf.mf_symbolic_analyze(h, rp, ci, perm)
    info = mf.mf_symbolic_get_info(s)
    f = mf.mf_factor_create(h, s, prec)
    mf.mf_factor_numeric(f, v)
    mf.mf_factor_numeric(f, v)  # graph replay of the same schedule
    L = mf.mf_factor_export_L(f, info["nnz_L"])
    launches = mf.mf_factor_launch_counts(f)[0]
    mf.mf_factor_free(f)
    mf.mf_symbolic_free(s)
    mf.mf_destroy(h)
    return L, info, launches


@pytest.mark.parametrize("case", ["jump20", "batch12"])
@pytest.mark.parametrize("prec", [0, 1])
def test_queue_matches_level_launches_bitwise(mf, orc, case, prec):
    if case == "jump20":
        rp, ci, v, perm, _ = gen.config3(20)
    else:
        rp, ci, v, perm = batch_case()
    Lq, info_q, nq = factor_L(mf, rp, ci, v, perm, prec, 1)
    Ll, info_l, nl = factor_L(mf, rp, ci, v, perm, prec, 0)
    assert info_q["queued_fronts"] > 0 and info_l["queued_fronts"] == 0
    assert nq < nl  # the small fronts of every level collapse into one launch
    assert np.array_equal(Lq, Ll)
    F = orc.factor(rp, ci, v, perm)
    assert orc.rel_fro(Lq, F.Lx) <= (1e-11 if prec == 0 else 5e-4)


def test_queue_wait_runs_out_and_factor_recovers(mf, orc):
    rp, ci, v, perm = batch_case()
    h = mf.mf_create()
    s = mf.mf_symbolic_analyze(h, rp, ci, perm)
    info = mf.mf_symbolic_get_info(s)
    f = mf.mf_factor_create(h, s, mf.MF_FP64)
    try:
        mf.mf_factor_numeric(f, v)
        mf.mf_factor_set_wait_limit(f, 1000)  # about 0.13 ms per wait
        rc = mf.mf_diag_small_queue(f, info["queued_fronts"] // 2)
        assert rc == mf.MF_ERR_TIMEOUT
        assert "queue" in mf.lib().mf_last_error_string().decode()
        mf.mf_factor_set_wait_limit(f, 0)
        mf.mf_factor_numeric(f, v)  # clean again, same values as the oracle
        L = mf.mf_factor_export_L(f, info["nnz_L"])
        F = orc.factor(rp, ci, v, perm)
        assert orc.rel_fro(L, F.Lx) <= 1e-11
        b = gen.rhs(len(rp) - 1, 1, seed=2)
        assert orc.berr(rp, ci, v, mf.mf_solve(f, b), b) <= 1e-13
    finally:
        mf.mf_factor_free(f)
        mf.mf_symbolic_free(s)
        mf.mf_destroy(h)


def test_queue_diag_rejects_bad_arguments(mf):
    rp, ci, v, perm, _ = gen.config3(12)
    h = mf.mf_create()
    s = mf.mf_symbolic_analyze(h, rp, ci, perm)
    f = mf.mf_factor_create(h, s, mf.MF_FP64)
    try:
        assert mf.mf_diag_small_queue(f, 1) == mf.MF_ERR_INVALID  # no numeric values yet
        mf.mf_factor_numeric(f, v)
        assert mf.mf_diag_small_queue(f, 0) == mf.MF_ERR_INVALID
    finally:
        mf.mf_factor_free(f)
        mf.mf_symbolic_free(s)
        mf.mf_destroy(h)
