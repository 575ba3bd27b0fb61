"""GPU parity of factorizations built on a condensed-graph symbolic analysis
(paper Sec. 5): the factor is the Cholesky factor of the block-expanded
matrix (added positions are explicit zeros), compared element by element with
the oracle's factor of that matrix; the solves are checked against A."""
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
    return m


def run(mf, orc, rp, ci, v, perm, node_of, prec, nrhs=2):
    h = mf.mf_create()
    s = mf.mf_symbolic_analyze_condensed(h, rp, ci, perm, node_of=node_of)
    f = mf.mf_factor_create(h, s, prec)
    try:
        mf.mf_factor_numeric(f, v)
        info = mf.mf_symbolic_get_info(s)
        Lx = mf.mf_factor_export_L(f, info["nnz_L"])
        erp, eci, ev = orc.expand_node_blocks(rp, ci, v, node_of)
        F = orc.factor(erp, eci, ev, perm)
        n = len(rp) - 1
        B = gen.rhs(n, nrhs, 5)
        if prec == mf.MF_FP64:
            X = mf.mf_solve(f, B)
        else:
            X, rep = mf.mf_solve_refined(f, B, tol=BERR, max_iter=30)
            assert rep["fell_back"] == 0
        return orc.rel_fro(Lx, F.Lx), orc.berr(rp, ci, v, X, B)
    finally:
        mf.mf_factor_free(f)
        mf.mf_symbolic_free(s)
        mf.mf_destroy(h)


@pytest.mark.parametrize("seed", range(4))
def test_random_nodes_fp64(mf, orc, seed):
    n = [60, 150, 300, 300][seed]
    rp, ci, v = gen.random_spd(n, 0.05, seed + 200)
    node_of, perm = gen.random_nodes(n, max_size=2 + seed % 3, seed=seed)
    relF, berr = run(mf, orc, rp, ci, v, perm, node_of, mf.MF_FP64)
    assert relF <= RELF64 and berr <= BERR


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_laplacian_node_pairs(mf, orc, prec):
    """7-point 16^3 Laplacian with consecutive DoFs of the ND order paired
    into nodes: wider fronts with explicit zeros, large-front path."""
    rp, ci, v, perm, _ = gen.config3(16)
    n = len(rp) - 1
    node_of = np.empty(n, dtype=np.int32)
    node_of[perm] = np.arange(n) // 2
    p = mf.MF_FP64 if prec == "fp64" else mf.MF_FP32
    relF, berr = run(mf, orc, rp, ci, v, perm, node_of, p)
    assert berr <= BERR
    assert relF <= (RELF64 if prec == "fp64" else 5e-4)
