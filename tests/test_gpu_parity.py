"""GPU parity: the CUDA path through the C-ABI against the FP64 oracle.

Bars (FP64): integer outputs bit-exact, ||L - L_oracle||_F / ||L_oracle||_F
<= 1e-11, normwise backward error <= 1e-13.  FP32 factors: relF within a few
thousand FP32 ulps of the oracle and, after FP64 refinement, backward error
<= 1e-13.
"""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu

RELF64 = 1e-11
BERR = 1e-13


@pytest.fixture(scope="module")
def mf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2506_05793_gb300 as m
    m.build()
    torch.cuda.init()
    return m


@pytest.fixture(scope="module")
def handle(mf):
    h = mf.mf_create()
    yield h
    mf.mf_destroy(h)


def factor_and_compare(mf, handle, orc, rp, ci, v, perm, prec=0, nrhs=1, seed=0, sym=None):
    s = mf.mf_symbolic_analyze(handle, rp, ci, perm)
    f = mf.mf_factor_create(handle, s, prec)
    try:
        mf.mf_factor_numeric(f, v)
        info = mf.mf_symbolic_get_info(s)
        Lx = mf.mf_factor_export_L(f, info["nnz_L"])
        so = sym or orc.symbolic(rp, ci, perm)
        F = orc.factor(rp, ci, v, perm, sym=so)
        relF = orc.rel_fro(Lx, F.Lx)
        n = len(rp) - 1
        B = gen.rhs(n, nrhs, seed)
        X = mf.mf_solve(f, B)
        berr = orc.berr(rp, ci, v, X, B)
        Xo = orc.solve(F, B, perm)
        return dict(relF=relF, berr=berr, X=X, Xo=Xo, Lx=Lx, F=F, info=info)
    finally:
        mf.mf_factor_free(f)
        mf.mf_symbolic_free(s)


def test_config1_fp64(mf, handle, orc):
    rp, ci, v, perm, b = gen.config1()
    r = factor_and_compare(mf, handle, orc, rp, ci, v, perm)
    assert r["relF"] <= RELF64
    assert r["berr"] <= BERR
    assert np.max(np.abs(r["X"] - r["Xo"])) <= 1e-10 * np.max(np.abs(r["Xo"]))


@pytest.mark.parametrize("seed", range(12))
def test_random_fp64(mf, handle, orc, seed):
    n = [1, 2, 17, 60, 150, 300][seed % 6]
    rp, ci, v = gen.random_spd(n, 0.3 if n < 50 else 0.04, seed, dense_rows=2 if seed % 2 else 0)
    perm = gen.random_perm(n, seed + 1)
    r = factor_and_compare(mf, handle, orc, rp, ci, v, perm, nrhs=1 + seed % 3, seed=seed)
    assert r["relF"] <= RELF64
    assert r["berr"] <= BERR


@pytest.mark.parametrize("n", [64, 65, 129, 200, 333])
def test_dense_fronts_fp64(mf, handle, orc, n):
    """One dense supernode: exercises the blocked large-front path with
    ragged panel blocks and tiles (k not a multiple of 64)."""
    import scipy.sparse as sp
    rng = np.random.default_rng(n)
    M = rng.standard_normal((n, n))
    A = sp.csr_matrix(M @ M.T + n * np.eye(n))
    rp, ci, v = A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data
    r = factor_and_compare(mf, handle, orc, rp, ci, v, None, nrhs=3)
    assert r["info"]["nsuper"] == 1
    assert r["relF"] <= RELF64
    assert r["berr"] <= BERR


@pytest.mark.parametrize("case", ["lap3d_jump_20", "lap3d_17x23x11", "q1_14x12x4", "lap2d_301x157"])
def test_structured_fp64(mf, handle, orc, case):
    if case == "lap3d_jump_20":
        rp, ci, v, perm, _ = gen.config3(20)
    elif case == "lap3d_17x23x11":
        rp, ci, v = gen.laplacian_3d(17, 23, 11)
        perm = gen.nd_perm((17, 23, 11))
    elif case == "q1_14x12x4":
        rp, ci, v = gen.q1_extruded(14, 12, 4, seed=3)
        perm = gen.nd_perm((15, 13, 5), split_axes=(0, 1), dofs=2)
    else:
        rp, ci, v = gen.laplacian_2d(301, 157)
        perm = gen.nd_perm((301, 157))
    r = factor_and_compare(mf, handle, orc, rp, ci, v, perm, nrhs=2)
    assert r["info"]["max_front"] > 128  # the large-front path ran
    assert r["relF"] <= RELF64
    assert r["berr"] <= BERR


@pytest.mark.parametrize("nrhs", [1, 8, 33, 64])
def test_multi_rhs(mf, handle, orc, nrhs):
    rp, ci, v, perm, _ = gen.config3(14, nrhs=1)
    r = factor_and_compare(mf, handle, orc, rp, ci, v, perm, nrhs=nrhs, seed=nrhs)
    assert r["berr"] <= BERR
    assert np.max(np.abs(r["X"] - r["Xo"])) <= 1e-8 * np.max(np.abs(r["Xo"]))


def test_not_spd_reports_column(mf, handle, orc):
    rp, ci, v = gen.laplacian_2d(30)
    perm = gen.nd_perm((30, 30))
    v = v.copy()
    j = 517
    old = int(perm[j])
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    v[(rows == old) & (ci == old)] = -1.0
    assert orc.factor(rp, ci, v, perm).bad_col == j
    s = mf.mf_symbolic_analyze(handle, rp, ci, perm)
    f = mf.mf_factor_create(handle, s, 0)
    with pytest.raises(mf.MFError) as e:
        mf.mf_factor_numeric(f, v)
    assert e.value.code == mf.MF_ERR_NOT_SPD
    assert e.value.column == j
    # the factor object stays usable: refactor with the original values
    mf.mf_factor_numeric(f, gen.laplacian_2d(30)[2])
    mf.mf_factor_free(f)
    mf.mf_symbolic_free(s)


def test_refactor_and_determinism(mf, handle, orc):
    rp, ci, v, perm, _ = gen.config3(18)
    s = mf.mf_symbolic_analyze(handle, rp, ci, perm)
    info = mf.mf_symbolic_get_info(s)
    f = mf.mf_factor_create(handle, s, 0)
    mf.mf_factor_numeric(f, v)
    L1 = mf.mf_factor_export_L(f, info["nnz_L"])
    mf.mf_factor_numeric(f, v)
    L2 = mf.mf_factor_export_L(f, info["nnz_L"])
    assert np.array_equal(L1, L2)  # deterministic, no atomics in the sums
    mf.mf_factor_numeric(f, 4.0 * v)
    L3 = mf.mf_factor_export_L(f, info["nnz_L"])
    assert np.max(np.abs(L3 - 2.0 * L1)) <= 1e-13 * np.max(np.abs(L1))
    mf.mf_factor_free(f)
    mf.mf_symbolic_free(s)


def test_graph_and_direct_launch_agree(mf, orc):
    rp, ci, v, perm, _ = gen.config3(16)
    out = []
    for graphs in (0, 1):
        opt = mf.mf_options_default()
        opt.use_graphs = graphs
        h = mf.mf_create(opt)
        s = mf.mf_symbolic_analyze(h, rp, ci, perm)
        f = mf.mf_factor_create(h, s, 0)
        mf.mf_factor_numeric(f, v)
        mf.mf_factor_numeric(f, v)
        out.append(mf.mf_factor_export_L(f, mf.mf_symbolic_get_info(s)["nnz_L"]))
        mf.mf_factor_free(f)
        mf.mf_symbolic_free(s)
        mf.mf_destroy(h)
    assert np.array_equal(out[0], out[1])


def test_profile_counts_flops(mf, orc):
    rp, ci, v, perm, _ = gen.config3(20)
    opt = mf.mf_options_default()
    opt.profile = 1
    h = mf.mf_create(opt)
    s = mf.mf_symbolic_analyze(h, rp, ci, perm)
    f = mf.mf_factor_create(h, s, 0)
    mf.mf_factor_numeric(f, v)
    prof = mf.mf_factor_profile(f)
    total = sum(p["flops"] for p in prof.values())
    info = mf.mf_symbolic_get_info(s)
    # kernel flops = the fronts' work (explicit zeros of merged fronts included)
    assert abs(total - info["front_flops"]) <= 0.02 * info["front_flops"]
    assert info["front_flops"] >= info["flops"]
    assert all(p["ms"] >= 0 for p in prof.values())
    nf, ns = mf.mf_factor_launch_counts(f)
    assert nf == sum(p["launches"] for p in prof.values()) + 1  # + the value gather
    mf.mf_factor_free(f)
    mf.mf_symbolic_free(s)
    mf.mf_destroy(h)


def test_device_tensors_and_stream(mf, handle, orc):
    import torch
    rp, ci, v, perm, _ = gen.config3(12)
    n = len(rp) - 1
    s = mf.mf_symbolic_analyze(handle, rp, ci, perm)
    f = mf.mf_factor_create(handle, s, 0)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        vd = torch.from_numpy(v).cuda()
        mf.mf_factor_numeric(f, vd, stream=st)
        B = gen.rhs(n, 5, seed=4)
        Bd = torch.from_numpy(np.ascontiguousarray(B.T)).cuda().t()
        Xd = mf.mf_solve(f, Bd, stream=st)
        st.synchronize()
    X = Xd.cpu().numpy()
    assert orc.berr(rp, ci, v, X, B) <= BERR
    mf.mf_factor_free(f)
    mf.mf_symbolic_free(s)


def test_fp32_factor_and_refinement(mf, handle, orc):
    rp, ci, v, perm, _ = gen.config3(20)
    n = len(rp) - 1
    s = mf.mf_symbolic_analyze(handle, rp, ci, perm)
    info = mf.mf_symbolic_get_info(s)
    f = mf.mf_factor_create(handle, s, 1)
    mf.mf_factor_numeric(f, v)
    Lx = mf.mf_factor_export_L(f, info["nnz_L"])
    F = orc.factor(rp, ci, v, perm)
    relF = orc.rel_fro(Lx, F.Lx)
    assert relF <= 5e-4  # FP32 factor against the FP64 oracle
    B = gen.rhs(n, 3, seed=7)
    X, rep = mf.mf_solve_refined(f, B, tol=BERR, max_iter=30)
    assert rep["berr"] <= BERR
    assert orc.berr(rp, ci, v, X, B) <= BERR
    assert rep["fell_back"] == 0
    assert rep["berr_first"] > BERR  # the plain FP32 solve alone is not enough
    Xo = orc.solve(F, B, perm)
    assert np.max(np.abs(X - Xo)) <= 1e-6 * np.max(np.abs(Xo))
    mf.mf_factor_free(f)
    mf.mf_symbolic_free(s)


def test_refinement_falls_back_on_stagnation(mf, handle, orc):
    """max_iter = 0 forces the stagnation branch: the FP64 factorization of the
    same values must deliver the FP64 backward error."""
    rp, ci, v, perm, _ = gen.config3(12)
    n = len(rp) - 1
    s = mf.mf_symbolic_analyze(handle, rp, ci, perm)
    f = mf.mf_factor_create(handle, s, 1)
    mf.mf_factor_numeric(f, v)
    B = gen.rhs(n, 1, seed=8)
    X, rep = mf.mf_solve_refined(f, B, tol=1e-15, max_iter=0)
    assert rep["fell_back"] == 1
    assert orc.berr(rp, ci, v, X, B) <= BERR
    with pytest.raises(mf.MFError) as e:
        mf.mf_solve_refined(f, B, tol=1e-15, max_iter=0, allow_fallback=False)
    assert e.value.code == mf.MF_ERR_STAGNATION
    mf.mf_factor_free(f)
    mf.mf_symbolic_free(s)


def test_tiny_and_diagonal(mf, handle, orc):
    import scipy.sparse as sp
    for A in [sp.csr_matrix(np.array([[4.0]])), sp.csr_matrix(np.diag(np.arange(1.0, 40.0)))]:
        rp, ci, v = A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data
        r = factor_and_compare(mf, handle, orc, rp, ci, v, None)
        assert r["relF"] <= RELF64 and r["berr"] <= BERR


def test_relaxed_and_fundamental_fronts_agree(mf, orc):
    """Amalgamated fronts carry explicit zeros; the exported factor equals the
    one computed on fundamental supernodes (to rounding) and the oracle's."""
    rp, ci, v, perm, _ = gen.config3(18)
    F = orc.factor(rp, ci, v, perm)
    Ls = []
    for relax in (0, 1):
        opt = mf.mf_options_default()
        opt.relax = relax
        h = mf.mf_create(opt)
        s = mf.mf_symbolic_analyze(h, rp, ci, perm)
        f = mf.mf_factor_create(h, s, 0)
        mf.mf_factor_numeric(f, v)
        Ls.append(mf.mf_factor_export_L(f, mf.mf_symbolic_get_info(s)["nnz_L"]))
        mf.mf_factor_free(f)
        mf.mf_symbolic_free(s)
        mf.mf_destroy(h)
    for L in Ls:
        assert orc.rel_fro(L, F.Lx) <= RELF64
    assert orc.rel_fro(Ls[0], Ls[1]) <= RELF64


@pytest.mark.parametrize("case", ["dense_150", "dense_200", "dense_333", "lap3d_jump_20", "q1_14x12x4"])
def test_fp32_tensor_core_update(mf, orc, case):
    """FP32 factor with the tcgen05 split-TF32 trailing update agrees with the
    FP32 FMA path and with the FP64 oracle to FP32 accuracy."""
    import scipy.sparse as sp
    if case.startswith("dense"):
        n = int(case.split("_")[1])
        rng = np.random.default_rng(n)
        M = rng.standard_normal((n, n))
        A = sp.csr_matrix(M @ M.T + n * np.eye(n))
        rp, ci, v, perm = A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data, None
    elif case == "lap3d_jump_20":
        rp, ci, v, perm, _ = gen.config3(20)
    else:
        rp, ci, v = gen.q1_extruded(14, 12, 4, seed=3)
        perm = gen.nd_perm((15, 13, 5), split_axes=(0, 1), dofs=2)
    F = orc.factor(rp, ci, v, perm)
    out = {}
    for tc in (0, 1):
        opt = mf.mf_options_default()
        opt.tc = tc
        opt.profile = 1
        h = mf.mf_create(opt)
        s = mf.mf_symbolic_analyze(h, rp, ci, perm)
        f = mf.mf_factor_create(h, s, 1)
        mf.mf_factor_numeric(f, v)
        out[tc] = mf.mf_factor_export_L(f, mf.mf_symbolic_get_info(s)["nnz_L"])
        prof = mf.mf_factor_profile(f)
        if tc:
            assert prof["syrk_tc"]["launches"] > 0 and prof["syrk"]["launches"] == 0
        mf.mf_factor_free(f)
        mf.mf_symbolic_free(s)
        mf.mf_destroy(h)
    r_fma = orc.rel_fro(out[0], F.Lx)
    r_tc = orc.rel_fro(out[1], F.Lx)
    assert r_fma <= 5e-4 and r_tc <= 5e-4
    # split-TF32 keeps FP32 accuracy: within a small factor of the FMA path
    assert r_tc <= 4.0 * r_fma + 1e-6


def messy_csr(rp, ci, v, seed):
    """The same matrix as a messier CSR: columns shuffled inside each row,
    some entries split into two duplicates (summed back by the library), and
    a few explicit zeros added symmetrically (structural entries)."""
    rng = np.random.default_rng(seed)
    n = len(rp) - 1
    rows = [list(zip(ci[rp[i]:rp[i + 1]].tolist(), v[rp[i]:rp[i + 1]].tolist())) for i in range(n)]
    for i in range(n):
        out = []
        for c, x in rows[i]:
            if rng.random() < 0.2:
                a = float(rng.uniform(-1.0, 1.0))
                out += [(c, a), (c, x - a)]
            else:
                out.append((c, x))
        rows[i] = out
    for _ in range(n // 10):
        i, j = (int(t) for t in rng.integers(0, n, 2))
        if i != j:
            rows[i].append((j, 0.0))
            rows[j].append((i, 0.0))
    for i in range(n):
        rng.shuffle(rows[i])
    nrp = np.zeros(n + 1, dtype=np.int64)
    nrp[1:] = np.cumsum([len(r) for r in rows])
    nci = np.array([c for r in rows for c, _ in r], dtype=np.int32)
    nv = np.array([x for r in rows for _, x in r], dtype=np.float64)
    return nrp, nci, nv


@pytest.mark.parametrize("prec", [0, 1])
def test_unsorted_duplicate_and_zero_entries(mf, handle, orc, prec):
    rp, ci, v, perm, _ = gen.config3(12)
    mrp, mci, mv = messy_csr(rp, ci, v, seed=3)
    if prec == 0:
        r = factor_and_compare(mf, handle, orc, mrp, mci, mv, perm, nrhs=2)
        assert r["relF"] <= RELF64 and r["berr"] <= BERR
        # the solution is that of the clean matrix
        r0 = factor_and_compare(mf, handle, orc, rp, ci, v, perm, nrhs=2)
        assert np.max(np.abs(r["X"] - r0["X"])) <= 1e-10 * np.max(np.abs(r0["X"]))
    else:
        s = mf.mf_symbolic_analyze(handle, mrp, mci, perm)
        f = mf.mf_factor_create(handle, s, mf.MF_FP32)
        try:
            mf.mf_factor_numeric(f, mv)
            B = gen.rhs(len(rp) - 1, 2, 4)
            X, rep = mf.mf_solve_refined(f, B, tol=BERR, max_iter=30)
            assert rep["fell_back"] == 0 and orc.berr(rp, ci, v, X, B) <= BERR
        finally:
            mf.mf_factor_free(f)
            mf.mf_symbolic_free(s)


def test_empty_matrix(mf, handle):
    """n = 0: analysis, factorization and a solve of nothing succeed."""
    rp = np.zeros(1, dtype=np.int64)
    ci = np.zeros(0, dtype=np.int32)
    s = mf.mf_symbolic_analyze(handle, rp, ci)
    f = mf.mf_factor_create(handle, s, mf.MF_FP64)
    try:
        mf.mf_factor_numeric(f, np.zeros(0))
        assert mf.mf_factor_export_L(f, 0).size == 0
    finally:
        mf.mf_factor_free(f)
        mf.mf_symbolic_free(s)


def test_loaded_analysis_factors_identically(mf, orc, tmp_path):
    """An analysis saved and loaded back drives the same kernels: the factor
    and the solution are bit for bit those of the original analysis."""
    rp, ci, v, perm, _ = gen.config3(16)
    opt = mf.mf_options_default()
    opt.sptrsv = 3
    h = mf.mf_create(opt)
    s = mf.mf_symbolic_analyze(h, rp, ci, perm)
    path = str(tmp_path / "a.sym")
    mf.mf_symbolic_save(s, path)
    t = mf.mf_symbolic_load(h, path)
    out = []
    try:
        B = gen.rhs(len(rp) - 1, 3, 9)
        for sym in (s, t):
            f = mf.mf_factor_create(h, sym, mf.MF_FP64)
            try:
                mf.mf_factor_numeric(f, v)
                Lx = mf.mf_factor_export_L(f, mf.mf_symbolic_get_info(sym)["nnz_L"])
                out.append((Lx, mf.mf_solve(f, B)))
            finally:
                mf.mf_factor_free(f)
        assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
        assert orc.berr(rp, ci, v, out[1][1], B) <= BERR
    finally:
        mf.mf_symbolic_free(s)
        mf.mf_symbolic_free(t)
        mf.mf_destroy(h)
