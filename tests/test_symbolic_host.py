"""Host symbolic analysis of the library (C-ABI, no GPU) against the oracle.

Integer outputs must match bit for bit: elimination tree, column counts,
nnz(L), fundamental supernode partition and the CSC pattern of L.
"""
import numpy as np
import pytest

import gen


@pytest.fixture(scope="module")
def mf():
    import paper_2506_05793_gb300 as m
    m.build()
    return m


@pytest.fixture(scope="module")
def handle(mf):
    h = mf.mf_create()
    yield h
    mf.mf_destroy(h)


def check_integers(mf, handle, orc, rp, ci, perm):
    s = mf.mf_symbolic_analyze(handle, rp, ci, perm)
    try:
        so = orc.symbolic(rp, ci, perm)
        assert np.array_equal(mf.mf_symbolic_etree(s), so["parent"])
        assert np.array_equal(mf.mf_symbolic_colcounts(s), so["colcount"])
        assert np.array_equal(mf.mf_symbolic_supernodes(s), so["sup_ptr"])
        info = mf.mf_symbolic_get_info(s)
        assert info["nnz_L"] == so["nnzL"]
        assert info["flops"] == so["flops"]
        F = orc.factor(rp, ci, np.ones(len(ci)), perm, sym=so) if len(rp) < 400 else None
        if F is not None:
            Lp, Li = mf.mf_symbolic_pattern(s)
            assert np.array_equal(Lp, F.Lp) and np.array_equal(Li, F.Li)
        par, lev = mf.mf_symbolic_supernode_tree(s)
        # supernodal tree: parent index larger; the level of the front holding
        # a supernode never decreases towards the root (merged supernodes share it)
        nz = par >= 0
        assert np.all(par[nz] > np.nonzero(nz)[0])
        assert np.all(lev[par[nz]] >= lev[nz])
        return info
    finally:
        mf.mf_symbolic_free(s)


@pytest.mark.parametrize("seed", range(24))
def test_random_patterns(mf, handle, orc, seed):
    n = [1, 2, 5, 17, 60, 150, 300, 33][seed % 8]
    rp, ci, _ = gen.random_spd(n, 0.3 if n < 50 else 0.04, seed, dense_rows=seed % 3 == 0)
    perm = gen.random_perm(n, seed)
    check_integers(mf, handle, orc, rp, ci, perm if seed % 4 else None)


@pytest.mark.parametrize("case", ["cfg1", "lap3d_jump_16", "q1_12x10x3", "lap3d_20x9x13"])
def test_structured(mf, handle, orc, case):
    if case == "cfg1":
        rp, ci, v, perm, _ = gen.config1()
    elif case == "lap3d_jump_16":
        rp, ci, v, perm, _ = gen.config3(16)
    elif case == "q1_12x10x3":
        rp, ci, v = gen.q1_extruded(12, 10, 3)
        perm = gen.nd_perm((13, 11, 4), split_axes=(0, 1), dofs=2)
    else:
        rp, ci, v = gen.laplacian_3d(20, 9, 13)
        perm = gen.nd_perm((20, 9, 13))
    check_integers(mf, handle, orc, rp, ci, perm)


def test_invalid_inputs(mf, handle):
    rp, ci, _ = gen.laplacian_2d(4)
    bad = ci.copy()
    bad[3] = 99
    with pytest.raises(mf.MFError) as e:
        mf.mf_symbolic_analyze(handle, rp, bad)
    assert e.value.code == mf.MF_ERR_INVALID
    perm = np.arange(16, dtype=np.int32)
    perm[0] = 1
    with pytest.raises(mf.MFError) as e:
        mf.mf_symbolic_analyze(handle, rp, ci, perm)
    assert e.value.code == mf.MF_ERR_INVALID
    rp2 = rp.copy()
    rp2[5] = rp2[7]
    with pytest.raises(mf.MFError):
        mf.mf_symbolic_analyze(handle, rp2, ci)


def test_empty_matrix(mf, handle):
    s = mf.mf_symbolic_analyze(handle, np.zeros(1, dtype=np.int64), np.zeros(0, dtype=np.int32))
    info = mf.mf_symbolic_get_info(s)
    assert info["n"] == 0 and info["nsuper"] == 0 and info["nnz_L"] == 0
    mf.mf_symbolic_free(s)


def test_batch_is_block_diagonal_union(mf, handle, orc):
    mats = []
    for a, b, c in [(5, 6, 7), (8, 4, 3), (3, 3, 9)]:
        rp, ci, v = gen.laplacian_3d(a, b, c)
        mats.append((rp, ci, gen.nd_perm((a, b, c))))
    s = mf.mf_symbolic_analyze_batch(handle, mats)
    info = mf.mf_symbolic_get_info(s)
    tot_nnzL = 0
    tot_flops = 0.0
    for rp, ci, pm in mats:
        so = orc.symbolic(rp, ci, pm)
        tot_nnzL += so["nnzL"]
        tot_flops += so["flops"]
    assert info["nnz_L"] == tot_nnzL and info["flops"] == tot_flops
    par = mf.mf_symbolic_etree(s)
    assert np.sum(par == -1) >= 3
    mf.mf_symbolic_free(s)


@pytest.mark.parametrize("relax", [0, 1])
def test_relaxed_fronts_keep_exported_integers(mf, orc, relax):
    """Amalgamation changes internal fronts only: exported etree, counts,
    supernodes and pattern equal the oracle's with and without it."""
    opt = mf.mf_options_default()
    opt.relax = relax
    h = mf.mf_create(opt)
    rp, ci, v, perm, _ = gen.config3(12)
    info = check_integers(mf, h, orc, rp, ci, perm)
    if relax:
        assert info["nfronts"] < info["nsuper"]
        assert info["front_flops"] >= info["flops"]
    else:
        assert info["nfronts"] == info["nsuper"] and info["front_flops"] == info["flops"]
    mf.mf_destroy(h)


def test_update_memory_plan_reuses_chains(mf, handle):
    """Update matrices of finished chains are recycled: the plan stays far
    below holding every update matrix at once."""
    rp, ci, v, perm, _ = gen.config3(24)
    s = mf.mf_symbolic_analyze(handle, rp, ci, perm)
    info = mf.mf_symbolic_get_info(s)
    cc = mf.mf_symbolic_colcounts(s)
    sup = mf.mf_symbolic_supernodes(s)
    k = np.diff(sup)
    m = cc[sup[:-1]] - k
    all_u = float(np.sum(m.astype(np.float64) ** 2)) * 8
    assert info["factor_bytes_fp64"] < 0.5 * all_u
    mf.mf_symbolic_free(s)


# ---- condensed graph (paper Sec. 5: DoFs of one node compressed) ----------
def check_condensed(mf, handle, orc, rp, ci, perm, node_of=None, block=1):
    """Condensed analysis = the plain analysis of the block-expanded pattern
    (oracle), and no node is split between two supernodes."""
    n = len(rp) - 1
    nodes = node_of if node_of is not None else np.arange(n) // block
    erp, eci, _ = orc.expand_node_blocks(rp, ci, np.ones(len(ci)), nodes)
    s = mf.mf_symbolic_analyze_condensed(handle, rp, ci, perm, node_of=node_of, block=block)
    try:
        so = orc.symbolic(erp, eci, perm)
        assert np.array_equal(mf.mf_symbolic_etree(s), so["parent"])
        assert np.array_equal(mf.mf_symbolic_colcounts(s), so["colcount"])
        assert np.array_equal(mf.mf_symbolic_supernodes(s), so["sup_ptr"])
        info = mf.mf_symbolic_get_info(s)
        assert info["nnz_L"] == so["nnzL"] and info["flops"] == so["flops"]
        if n < 400:
            F = orc.factor(erp, eci, np.ones(len(eci)), perm, sym=so)
            Lp, Li = mf.mf_symbolic_pattern(s)
            assert np.array_equal(Lp, F.Lp) and np.array_equal(Li, F.Li)
        sup = mf.mf_symbolic_supernodes(s)
        pm = np.arange(n) if perm is None else np.asarray(perm)
        sn_of_col = np.repeat(np.arange(len(sup) - 1), np.diff(sup))
        node_new = np.asarray(nodes)[pm]
        for u in np.unique(node_new):
            assert len(np.unique(sn_of_col[node_new == u])) == 1
        return info
    finally:
        mf.mf_symbolic_free(s)


@pytest.mark.parametrize("seed", range(12))
def test_condensed_random_nodes(mf, handle, orc, seed):
    n = [7, 40, 150, 300][seed % 4]
    rp, ci, _ = gen.random_spd(n, 0.2 if n < 50 else 0.03, seed + 100)
    node_of, perm = gen.random_nodes(n, max_size=1 + seed % 4, seed=seed, scatter=seed % 2 == 0)
    check_condensed(mf, handle, orc, rp, ci, perm, node_of=node_of)


def test_condensed_fixed_blocks_and_identity(mf, handle, orc):
    rp, ci, _ = gen.random_spd(90, 0.05, 7)
    check_condensed(mf, handle, orc, rp, ci, None, block=3)
    # block 1: the condensed graph is the graph itself
    a = check_condensed(mf, handle, orc, rp, ci, None, block=1)
    b = check_integers(mf, handle, orc, rp, ci, None)
    assert a["nnz_L"] == b["nnz_L"]


def test_condensed_q1_two_dofs_equals_plain(mf, handle, orc):
    """The Q1 mesh couples both velocity DoFs of every node pair, so its node
    blocks are full and condensing them changes nothing."""
    rp, ci, v = gen.q1_extruded(12, 10, 3)
    perm = gen.nd_perm((13, 11, 4), split_axes=(0, 1), dofs=2)
    s0 = mf.mf_symbolic_analyze(handle, rp, ci, perm)
    s1 = mf.mf_symbolic_analyze_condensed(handle, rp, ci, perm, block=2)
    try:
        for get in (mf.mf_symbolic_etree, mf.mf_symbolic_colcounts, mf.mf_symbolic_supernodes):
            assert np.array_equal(get(s0), get(s1))
        assert np.array_equal(mf.mf_symbolic_pattern(s0)[1], mf.mf_symbolic_pattern(s1)[1])
    finally:
        mf.mf_symbolic_free(s0)
        mf.mf_symbolic_free(s1)
    check_condensed(mf, handle, orc, rp, ci, perm, block=2)


def test_condensed_invalid(mf, handle):
    rp, ci, _ = gen.laplacian_2d(4)
    with pytest.raises(mf.MFError) as e:
        mf.mf_symbolic_analyze_condensed(handle, rp, ci, None, block=0)
    assert e.value.code == mf.MF_ERR_INVALID
    # node {0, 1} split by the ordering
    perm = np.array([0, 2, 1] + list(range(3, 16)), dtype=np.int32)
    with pytest.raises(mf.MFError) as e:
        mf.mf_symbolic_analyze_condensed(handle, rp, ci, perm, block=2)
    assert e.value.code == mf.MF_ERR_INVALID
    bad = np.zeros(16, dtype=np.int32)
    bad[3] = 16
    with pytest.raises(mf.MFError) as e:
        mf.mf_symbolic_analyze_condensed(handle, rp, ci, None, node_of=bad)
    assert e.value.code == mf.MF_ERR_INVALID


def test_sptrsv_option_values(mf, orc):
    """Variants 1-4 are accepted (0 means 1); variant 3 adds the partitioned
    inverse, the size of the large fronts' L, to the factor's memory, and
    variant 4 its transpose as well; 5 is refused."""
    rp, ci, v, perm, _ = gen.config3(16)
    sizes = {}
    for variant in (0, 1, 2, 3, 4):
        opt = mf.mf_options_default()
        opt.sptrsv = variant
        h = mf.mf_create(opt)
        s = mf.mf_symbolic_analyze(h, rp, ci, perm)
        sizes[variant] = mf.mf_symbolic_get_info(s)["factor_bytes_fp64"]
        mf.mf_symbolic_free(s)
        mf.mf_destroy(h)
    assert sizes[0] == sizes[1] < sizes[2] < sizes[3] < sizes[4]
    opt = mf.mf_options_default()
    opt.sptrsv = 5
    with pytest.raises(mf.MFError) as e:
        mf.mf_create(opt)
    assert e.value.code == mf.MF_ERR_INVALID


def test_messy_csr_same_integers(mf, handle, orc):
    """Shuffled columns and duplicate entries leave every integer output
    unchanged (explicit zeros are structural and are left out here)."""
    rp, ci, v, perm, _ = gen.config3(10)
    rng = np.random.default_rng(5)
    n = len(rp) - 1
    rows = []
    for i in range(n):
        r = ci[rp[i]:rp[i + 1]].tolist()
        r += [c for c in r if rng.random() < 0.3]
        rng.shuffle(r)
        rows.append(r)
    mrp = np.zeros(n + 1, dtype=np.int64)
    mrp[1:] = np.cumsum([len(r) for r in rows])
    mci = np.array([c for r in rows for c in r], dtype=np.int32)
    a = mf.mf_symbolic_analyze(handle, rp, ci, perm)
    b = mf.mf_symbolic_analyze(handle, mrp, mci, perm)
    try:
        for get in (mf.mf_symbolic_etree, mf.mf_symbolic_colcounts, mf.mf_symbolic_supernodes):
            assert np.array_equal(get(a), get(b))
        assert np.array_equal(mf.mf_symbolic_pattern(a)[1], mf.mf_symbolic_pattern(b)[1])
    finally:
        mf.mf_symbolic_free(a)
        mf.mf_symbolic_free(b)


def test_save_and_load_round_trip(mf, handle, orc, tmp_path):
    """A saved analysis loads back identical: every integer output, the info
    record, and a byte-identical second save."""
    rp, ci, v, perm, _ = gen.config3(12)
    opt = mf.mf_options_default()
    opt.sptrsv = 3
    h3 = mf.mf_create(opt)
    s = mf.mf_symbolic_analyze(h3, rp, ci, perm)
    mf.mf_symbolic_pattern(s)  # builds the lazily kept supernode rows first
    p1, p2 = tmp_path / "a.sym", tmp_path / "b.sym"
    mf.mf_symbolic_save(s, str(p1))
    t = mf.mf_symbolic_load(handle, str(p1))
    try:
        for get in (mf.mf_symbolic_etree, mf.mf_symbolic_colcounts, mf.mf_symbolic_supernodes):
            assert np.array_equal(get(s), get(t))
        assert np.array_equal(mf.mf_symbolic_pattern(s)[1], mf.mf_symbolic_pattern(t)[1])
        assert mf.mf_symbolic_get_info(s) == mf.mf_symbolic_get_info(t)
        mf.mf_symbolic_save(t, str(p2))
        assert p1.read_bytes() == p2.read_bytes()
    finally:
        mf.mf_symbolic_free(s)
        mf.mf_symbolic_free(t)
        mf.mf_destroy(h3)


def test_load_rejects_bad_files(mf, handle, tmp_path):
    rp, ci, _ = gen.laplacian_2d(9)
    s = mf.mf_symbolic_analyze(handle, rp, ci)
    good = tmp_path / "g.sym"
    mf.mf_symbolic_save(s, str(good))
    mf.mf_symbolic_free(s)
    data = good.read_bytes()
    cases = {"missing": None, "empty": b"", "truncated": data[:len(data) // 2],
             "magic": b"X" + data[1:], "trailing": data + b"\\0" * 8}
    # a vector count far beyond the file: the count of rowptr follows the
    # header (32 bytes) and the two int64 scalars n, nnzA
    bad = bytearray(data)
    bad[48:56] = (1 << 60).to_bytes(8, "little")
    cases["count"] = bytes(bad)
    # one flipped bit deep in the payload, sizes intact: the hash rejects it
    flip = bytearray(data)
    flip[len(data) // 2] ^= 0x10
    cases["bitflip"] = bytes(flip)
    for name, content in cases.items():
        p = tmp_path / (name + ".sym")
        if content is not None:
            p.write_bytes(content)
        with pytest.raises(mf.MFError) as e:
            mf.mf_symbolic_load(handle, str(p))
        assert e.value.code == mf.MF_ERR_INVALID, name


def test_factor_over_budget_is_oom(mf):
    """A device budget smaller than the factor's bytes refuses the factor
    before any device allocation (host-side check, no GPU needed)."""
    opt = mf.mf_options_default()
    opt.budget_bytes = 1024
    h = mf.mf_create(opt)
    rp, ci, _ = gen.laplacian_2d(20)
    s = mf.mf_symbolic_analyze(h, rp, ci)
    try:
        with pytest.raises(mf.MFError) as e:
            mf.mf_factor_create(h, s, mf.MF_FP64)
        assert e.value.code == mf.MF_ERR_OOM
    finally:
        mf.mf_symbolic_free(s)
        mf.mf_destroy(h)


# ---- schedule consistency (host) ------------------------------------------
@pytest.mark.parametrize("variant", [1, 2, 3, 4])
@pytest.mark.parametrize("relax,small,queue", [(0, 128, 1), (1, 128, 1), (1, 32, 1), (1, 128, 0)])
def test_schedules_cover_every_front_once(mf, variant, relax, small, queue):
    opt = mf.mf_options_default()
    opt.sptrsv, opt.relax, opt.small_front_max = variant, relax, small
    opt.small_queue = queue
    h = mf.mf_create(opt)
    try:
        cases = [gen.config3(16)[:2] + (gen.config3(16)[3],)]
        rp, ci, _ = gen.q1_extruded(12, 10, 3)
        cases.append((rp, ci, gen.nd_perm((13, 11, 4), split_axes=(0, 1), dofs=2)))
        rp, ci, _ = gen.random_spd(300, 0.04, 3)
        cases.append((rp, ci, gen.random_perm(300, 4)))
        import scipy.sparse as sp
        M = np.random.default_rng(1).standard_normal((333, 333))
        A = sp.csr_matrix(M @ M.T + 333 * np.eye(333))
        cases.append((A.indptr.astype(np.int64), A.indices.astype(np.int32), None))
        for rp, ci, perm in cases:
            s = mf.mf_symbolic_analyze(h, rp, ci, perm)
            try:
                mf.mf_symbolic_check(s)
            finally:
                mf.mf_symbolic_free(s)
        mats, _ = gen.box_batch(12, 8, 20, seed=4)
        s = mf.mf_symbolic_analyze_batch(h, [(a, b, p) for a, b, c, p in mats])
        mf.mf_symbolic_check(s)
        mf.mf_symbolic_free(s)
    finally:
        mf.mf_destroy(h)


def test_schedules_of_tall_and_wide_fronts(mf):
    """Fronts with more than 512 pivot columns and more than 2,048 update
    rows: the one-right-hand-side update-row products then take every width
    of the forward product (tile 2: at most 128 pivot columns, 1: at most
    512, 0: wider) and every row split of the backward one (1, 2, 4 and 8
    CTAs per 64-column block).  The host check verifies for every launch
    that its width and split are ones its fronts allow, besides the
    coverage of every front."""
    h = mf.mf_create()
    try:
        cases = [(gen.laplacian_3d(48)[:2], gen.nd_perm((48, 48, 48)))]
        rp, ci, _ = gen.q1_extruded(96, 48, 10, seed=1)
        cases.append(((rp, ci), gen.nd_perm((97, 49, 11), split_axes=(0, 1), dofs=2)))
        for (rp, ci), perm in cases:
            s = mf.mf_symbolic_analyze(h, rp, ci, perm)
            try:
                info = mf.mf_symbolic_get_info(s)
                assert info["max_k"] > 512 and info["max_front"] > 2048
                mf.mf_symbolic_check(s)
            finally:
                mf.mf_symbolic_free(s)
    finally:
        mf.mf_destroy(h)


def _fnv1a(data):
    h = 1469598103934665603
    for byte in data:
        h = ((h ^ byte) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


# members of a saved analysis in file order, up to the work items
_MEMBERS = ["i8", "i8", ("v", 8), ("v", 4), ("v", 4), ("v", 4), ("v", 4), ("v", 8), ("v", 4),
            ("v", 4), ("v", 4), ("v", 8), ("v", 8), ("v", 4), ("v", 4), "i4", ("v", 4),
            ("v", 4), "i8", "i8", "i8", "i8", "i8", "i4", "i8", "i8", ("v", 64), ("v", 4),
            ("v", 4), ("v", 4), ("v", 4), ("v", 8), ("v", 4), ("v", 8), ("v", 8), "i8", "i8",
            "i8"]
_ROWIDX, _RELMAP, _ASRC, _ITEMS = 28, 29, 34, len(_MEMBERS)


def _member_pos(data, index, members=None):
    """Byte offset of member `index` (its element count for a vector)."""
    pos = 32
    for m in (members or _MEMBERS)[:index]:
        if isinstance(m, tuple):
            cnt = int.from_bytes(data[pos:pos + 8], "little")
            pos += 8 + cnt * m[1]
        else:
            pos += int(m[1])
    return pos


def _saved(mf, handle, tmp_path):
    rp, ci, v, perm, _ = gen.config3(8)
    s = mf.mf_symbolic_analyze(handle, rp, ci, perm)
    path = tmp_path / "a.sym"
    mf.mf_symbolic_save(s, str(path))
    mf.mf_symbolic_free(s)
    return path, bytearray(path.read_bytes()), len(rp) - 1


def _load_fails(mf, handle, path, data, what):
    data[-8:] = _fnv1a(data[32:-8]).to_bytes(8, "little")  # a matching hash
    path.write_bytes(bytes(data))
    with pytest.raises(mf.MFError) as e:
        mf.mf_symbolic_load(handle, str(path))
    assert e.value.code == mf.MF_ERR_INVALID
    assert what in str(e.value)


def test_load_rejects_a_repeated_item(mf, handle, tmp_path):
    """A saved analysis whose work list repeats one item, with its hash
    recomputed, fails the schedule check that the loader runs."""
    path, data, _ = _saved(mf, handle, tmp_path)
    pos = _member_pos(data, _ITEMS)
    nitems = int.from_bytes(data[pos:pos + 8], "little")
    assert nitems >= 2
    first = pos + 8
    data[first + 16:first + 32] = data[first:first + 16]  # item 1 := item 0
    _load_fails(mf, handle, path, data, "invalid schedule")


@pytest.mark.parametrize("member,width,value", [
    ("rowidx", 4, "n"), ("relmap", 4, 1 << 20), ("asrc", 8, 1 << 40), ("rowidx", 4, -1)])
def test_load_rejects_an_index_out_of_range(mf, handle, tmp_path, member, width, value):
    """Indices that device kernels dereference (front rows, relative maps,
    CSR source positions) are range-checked on load: a file planted with one
    out-of-range entry and a matching hash is refused before any device code
    could see it."""
    path, data, n = _saved(mf, handle, tmp_path)
    idx = {"rowidx": _ROWIDX, "relmap": _RELMAP, "asrc": _ASRC}[member]
    pos = _member_pos(data, idx)
    cnt = int.from_bytes(data[pos:pos + 8], "little")
    assert cnt > 0
    val = n if value == "n" else value
    at = pos + 8 + (cnt // 2) * width
    data[at:at + width] = int(val).to_bytes(width, "little", signed=True)
    _load_fails(mf, handle, path, data, "index out of range")


# the serialized members after Wsize, up to the forward gather sources:
# items, fsched, fsched_tc, soff, split_rows, split_rows_b, max_large,
# keep_inv, ioff, ninv, pinv, pinv_flops, arange, fwsched, bwsched, blkoff,
# ginv_ptr, ginv_src (Launch records are 40 bytes, Item records 16)
_TAIL = [("v", 16), ("v", 40), ("v", 40), ("v", 8), "i8", "i8", "i8", "i1", ("v", 8), "i8",
         "i1", "i8", ("v", 16), ("v", 40), ("v", 40), ("v", 4), ("v", 8), ("v", 8)]
_GINV_SRC = len(_MEMBERS) + len(_TAIL) - 1


def test_load_rejects_a_gather_source_on_a_pivot_row(mf, handle, tmp_path):
    """The chained pivot blocks of the solve pass their values through the
    pivot rows of their fronts' work vectors, which the forward gather must
    never read.  A saved analysis with one gather source moved onto a pivot
    row (row 0 of the first front's work vector; still inside the vector,
    so the range check passes) and a matching hash is refused by the
    schedule check."""
    path, data, _ = _saved(mf, handle, tmp_path)
    pos = _member_pos(data, _GINV_SRC, _MEMBERS + _TAIL)
    cnt = int.from_bytes(data[pos:pos + 8], "little")
    assert cnt > 0
    at = pos + 8 + (cnt // 2) * 8
    assert int.from_bytes(data[at:at + 8], "little", signed=True) > 0
    data[at:at + 8] = (0).to_bytes(8, "little", signed=True)
    _load_fails(mf, handle, path, data, "value slot")


def test_condensed_edge_cases(mf, handle, orc):
    """One node holding every DoF gives one dense supernode; node ids with
    gaps and single-DoF nodes mixed with larger ones match the expanded
    pattern; the empty matrix analyses."""
    rp, ci, _ = gen.random_spd(40, 0.1, 11)
    info = check_condensed(mf, handle, orc, rp, ci, None, node_of=np.zeros(40, dtype=np.int32))
    assert info["nsuper"] == 1 and info["nnz_L"] == 40 * 41 // 2
    node_of, perm = gen.random_nodes(60, max_size=3, seed=12)
    gappy = (node_of.astype(np.int64) * 7 % 59).astype(np.int32)  # ids spread out, still < n
    assert len(np.unique(gappy)) == len(np.unique(node_of))
    check_condensed(mf, handle, orc, *gen.random_spd(60, 0.08, 13)[:2], perm, node_of=gappy)
    s = mf.mf_symbolic_analyze_condensed(handle, np.zeros(1, dtype=np.int64),
                                         np.zeros(0, dtype=np.int32), None, block=2)
    assert mf.mf_symbolic_get_info(s)["n"] == 0
    mf.mf_symbolic_free(s)


def test_small_queue_holds_the_small_subforests(mf, orc):
    """The persistent queue holds exactly the small fronts whose subtree is
    all small (checked here against the supernodal tree), and turning it
    off leaves no queue."""
    rp, ci, v, perm, _ = gen.config3(16)
    for queue in (1, 0):
        opt = mf.mf_options_default()
        opt.small_queue = queue
        h = mf.mf_create(opt)
        s = mf.mf_symbolic_analyze(h, rp, ci, perm)
        info = mf.mf_symbolic_get_info(s)
        if queue:
            assert 0 < info["queued_fronts"] <= info["nfronts"]
        else:
            assert info["queued_fronts"] == 0
        mf.mf_symbolic_check(s)
        mf.mf_symbolic_free(s)
        mf.mf_destroy(h)


@pytest.mark.parametrize("tiles", [(0, 0, 0, 0), (4, 1, 2, 2), (2, 2, 2, 2), (1, 3, 4, 3),
                                   (4, 4, 4, 4)])
@pytest.mark.parametrize("variant", [2, 4])
def test_schedules_with_update_tiles(mf, tiles, variant):
    """Every per-bucket trailing-update choice gives schedules that cover
    each front's tiles exactly once (FMA 32 / 64 / 128 and tensor cores,
    mixed within a level), with and without the lookahead levels."""
    opt = mf.mf_options_default()
    opt.sptrsv = variant
    for b in range(4):
        opt.update_tile[b] = tiles[b]
    h = mf.mf_create(opt)
    try:
        rp, ci, v, perm, _ = gen.config3(24)
        s = mf.mf_symbolic_analyze(h, rp, ci, perm)
        mf.mf_symbolic_check(s)
        assert list(mf.mf_symbolic_options(s).update_tile) == list(tiles)
        mf.mf_symbolic_free(s)
        mats, _ = gen.box_batch(16, 8, 30, seed=4)
        s = mf.mf_symbolic_analyze_batch(h, [(a, b, p) for a, b, c, p in mats])
        mf.mf_symbolic_check(s)
        mf.mf_symbolic_free(s)
    finally:
        mf.mf_destroy(h)


def test_saved_analysis_keeps_its_options(mf, tmp_path):
    opt = mf.mf_options_default()
    opt.update_tile[2] = 2
    opt.small_queue = 32
    opt.relax = 0
    h = mf.mf_create(opt)
    rp, ci, v, perm, _ = gen.config3(10)
    s = mf.mf_symbolic_analyze(h, rp, ci, perm)
    path = str(tmp_path / "o.sym")
    mf.mf_symbolic_save(s, path)
    t = mf.mf_symbolic_load(h, path)
    a, b = mf.mf_symbolic_options(s), mf.mf_symbolic_options(t)
    for name, _ in mf.mf_options._fields_:
        assert list(getattr(a, name)) == list(getattr(b, name)) if name == "update_tile" \
            else getattr(a, name) == getattr(b, name)
    assert b.update_tile[2] == 2 and b.small_queue == 32 and b.relax == 0
    mf.mf_symbolic_free(s)
    mf.mf_symbolic_free(t)
    mf.mf_destroy(h)
