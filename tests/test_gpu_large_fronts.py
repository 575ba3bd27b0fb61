"""Element-by-element parity on fronts of thousands of columns, with the
options the benchmark times (CUDA graph, lookahead on the two prioritised
streams, tensor-core trailing updates for FP32, kept diagonal-block
inverses).  The fronts at the top of these trees take the paths that only
large fronts take -- multi-wave trailing-update grids, lookahead strips,
the four-slot staging area of the tensor-core update -- and the whole factor
is compared with the oracle's, entry by entry, including the largest front
alone.

Cases (each with a front of more than 2,000 pivot columns):
  * the extruded Q1 mesh generator of the benchmark on 96 x 48 x 10
    hexahedra (2 DoFs per node, horizontal nested dissection);
  * the 7-point coefficient-jump cube (1 / 1e3 on 8^3 blocks) on 48^3.

Bars: FP64 relF <= 1e-11 (the largest fronts have about 3,400 columns, so an
entry of L sums at most a few thousand FP64 products: about 3e3 x 1.1e-16 =
4e-13 relative to the magnitude of the terms, times the modest condition of
these matrices) and berr <= 1e-13.  FP32: relF against the FP64 oracle
<= 1e-4, below the worst-case n u_32 = 3,400 x 6e-8 = 2e-4 of a sum over the
largest front (measured on a GB300: 3e-7 to 7e-7 overall, at most 2.3e-6 on
the widest supernode), and the FP32 factor refined in FP64 must reach
berr <= 1e-13."""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu

CASES = {
    "q1_96x48x10": lambda: (gen.q1_extruded(96, 48, 10, seed=1),
                            gen.nd_perm((97, 49, 11), split_axes=(0, 1), dofs=2)),
    "jump_48": lambda: (gen.laplacian_3d(48, jump_block=8, jump_value=1e3, seed=2),
                        gen.nd_perm((48, 48, 48))),
}
_cache = {}


@pytest.fixture(scope="module")
def mf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2506_05793_gb300 as m
    m.build()
    return m


def case(orc, name):
    """(rp, ci, v, perm, oracle factor, b, oracle x), cached per case."""
    if name not in _cache:
        (rp, ci, v), perm = CASES[name]()
        F = orc.factor(rp, ci, v, perm, threads=0)
        assert F.bad_col == -1
        b = gen.rhs(len(rp) - 1, 1, seed=9)
        _cache[name] = (rp, ci, v, perm, F, b, orc.solve(F, b, perm))
    return _cache[name]


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", [0, 1])
def test_large_front_factor_elementwise(mf, orc, name, prec):
    rp, ci, v, perm, F, b, xo = case(orc, name)
    h = mf.mf_create()
    s = mf.mf_symbolic_analyze(h, rp, ci, perm)
    f = mf.mf_factor_create(h, s, prec)
    try:
        info = mf.mf_symbolic_get_info(s)
        assert info["max_k"] >= 2000, "case lost its large front"
        mf.mf_factor_numeric(f, v)
        Lx = mf.mf_factor_export_L(f, info["nnz_L"])
        Lp, _ = mf.mf_symbolic_pattern(s)
        assert np.array_equal(Lp, F.Lp)
        rel = orc.rel_fro(Lx, F.Lx)
        # the widest fundamental supernode alone, entry by entry
        sup = mf.mf_symbolic_supernodes(s)
        w = int(np.argmax(np.diff(sup)))
        a, z = F.Lp[sup[w]], F.Lp[sup[w + 1]]
        rel_top = orc.rel_fro(Lx[a:z], F.Lx[a:z])
        print("%s prec=%d relF=%.3e relF(widest supernode, %d columns)=%.3e"
              % (name, prec, rel, sup[w + 1] - sup[w], rel_top))
        assert sup[w + 1] - sup[w] >= 1000
        if prec == 0:
            assert rel <= 1e-11 and rel_top <= 1e-11
            x = mf.mf_solve(f, b)
            assert orc.berr(rp, ci, v, x, b) <= 1e-13
            assert np.max(np.abs(x - xo)) <= 1e-9 * np.max(np.abs(xo))
        else:
            assert rel <= 1e-4 and rel_top <= 1e-4
            x, rep = mf.mf_solve_refined(f, b, tol=1e-13, max_iter=30)
            assert rep["fell_back"] == 0
            assert orc.berr(rp, ci, v, x, b) <= 1e-13
    finally:
        mf.mf_factor_free(f)
        mf.mf_symbolic_free(s)
        mf.mf_destroy(h)


@pytest.mark.parametrize("name", list(CASES))
def test_large_front_column_export(mf, orc, name):
    """mf_factor_export_columns returns exactly the slice of the full export
    (a range that starts and ends inside fronts)."""
    rp, ci, v, perm, F, b, xo = case(orc, name)
    h = mf.mf_create()
    s = mf.mf_symbolic_analyze(h, rp, ci, perm)
    f = mf.mf_factor_create(h, s, 0)
    try:
        info = mf.mf_symbolic_get_info(s)
        mf.mf_factor_numeric(f, v)
        Lx = mf.mf_factor_export_L(f, info["nnz_L"])
        n = len(rp) - 1
        for j0, j1 in [(0, n), (n // 3 + 7, n - 1013), (n - 1, n), (5, 5)]:
            part = mf.mf_factor_export_columns(f, j0, j1, int(F.Lp[j1] - F.Lp[j0]))
            assert np.array_equal(part, Lx[F.Lp[j0]:F.Lp[j1]])
    finally:
        mf.mf_factor_free(f)
        mf.mf_symbolic_free(s)
        mf.mf_destroy(h)
