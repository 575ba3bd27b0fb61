"""FastILU host side (no GPU): the library's ILU(k) pattern and the level of
every entry equal the oracle's bit for bit; bad arguments are refused."""
import numpy as np
import pytest

import gen


@pytest.fixture(scope="module")
def mf():
    import paper_2506_05793_gb300 as m
    m.build()
    return m


@pytest.mark.parametrize("case", ["random", "elasticity4", "lap3d_6", "messy"])
@pytest.mark.parametrize("K", [0, 1, 2, 3])
def test_pattern_matches_oracle(mf, orc, case, K):
    if case == "random":
        rp, ci, _ = gen.random_spd(120, 0.03, 9)
    elif case == "elasticity4":
        rp, ci, _ = gen.elasticity_3d(4)
    elif case == "lap3d_6":
        rp, ci, _ = gen.laplacian_3d(6)
    else:  # columns shuffled within rows, duplicates
        rp0, ci0, _ = gen.laplacian_3d(5)
        rng = np.random.default_rng(3)
        rows = []
        for i in range(len(rp0) - 1):
            r = list(ci0[rp0[i]:rp0[i + 1]])
            r += r[:2]
            rng.shuffle(r)
            rows.append(r)
        rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int64)
        ci = np.concatenate(rows).astype(np.int32)
    h = mf.mf_create()
    ilu = mf.mf_ilu_symbolic(h, rp, ci, K)
    try:
        Sp, Sj, Sl = mf.mf_ilu_pattern(ilu)
        pat = orc.iluk_pattern(rp, ci, K)
        assert np.array_equal(Sp, pat.Sp)
        assert np.array_equal(Sj, pat.Sj)
        assert np.array_equal(Sl, pat.Slev)
    finally:
        mf.mf_ilu_free(ilu)
        mf.mf_destroy(h)


def test_bad_arguments(mf):
    h = mf.mf_create()
    rp, ci, _ = gen.laplacian_2d(4)
    with pytest.raises(mf.MFError) as e:
        mf.mf_ilu_symbolic(h, rp, ci, -1)
    assert e.value.code == mf.MF_ERR_INVALID
    bad = ci.copy()
    bad[0] = 99
    with pytest.raises(mf.MFError):
        mf.mf_ilu_symbolic(h, rp, bad, 1)
    ilu = mf.mf_ilu_symbolic(h, rp, ci, 1)
    with pytest.raises(mf.MFError) as e:  # no numeric factors yet
        mf.mf_ilu_export(ilu)
    assert e.value.code == mf.MF_ERR_INVALID
    mf.mf_ilu_free(ilu)
    mf.mf_destroy(h)
