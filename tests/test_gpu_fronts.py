"""One front at a time over a grid of shapes (the edge sizes of the kernels):
a matrix whose analysis has a front with exactly k pivots and m update rows
(pivot block dense and fully coupled to the update rows, which a one-column
leaf keeps in a front of their own), factored in FP64 and in FP32 and
compared with the oracle.  k and m run over 1, 31-33, 63-65, 127-129 and a
few update sizes, so the one-CTA small-front kernel (k + m <= 128), the
blocked large-front path with ragged 64-column panels and tiles, and the
128 x 128 tensor-core tiles (FP32) all see their boundaries."""
import numpy as np
import pytest
import scipy.sparse as sp

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


@pytest.fixture(scope="module")
def handle(mf):
    opt = mf.mf_options_default()
    opt.relax = 0  # keep the fronts exactly as built
    h = mf.mf_create(opt)
    yield h
    mf.mf_destroy(h)


def front_matrix(k, m, seed):
    """Columns: k pivots, one leaf, m trailing rows (natural order).  Pivots
    couple to each other and to every trailing row; the leaf couples to the
    first trailing row only, giving it a second child so the trailing rows
    start a front of their own."""
    n = k + 1 + m
    rng = np.random.default_rng(seed)
    mask = np.zeros((n, n), dtype=bool)
    P, leaf, T = np.arange(k), k, np.arange(k + 1, n)
    mask[np.ix_(P, P)] = True
    mask[np.ix_(P, T)] = True
    mask[np.ix_(T, P)] = True
    mask[np.ix_(T, T)] = True
    if m:
        mask[leaf, T[0]] = mask[T[0], leaf] = True
    mask[leaf, leaf] = True
    M = np.where(mask, rng.uniform(-1.0, 1.0, (n, n)), 0.0)
    M = np.triu(M) + np.triu(M, 1).T
    np.fill_diagonal(M, np.abs(M).sum(axis=1) + 1.0)
    A = sp.csr_matrix(M)
    return A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data


KS = [1, 31, 32, 33, 63, 64, 65, 127, 128, 129]
MS = [0, 1, 31, 33, 64, 65, 200]


@pytest.mark.parametrize("k", KS)
def test_front_grid(mf, handle, orc, k):
    for m in MS:
        rp, ci, v = front_matrix(k, m, seed=1000 * k + m)
        n = len(rp) - 1
        s = mf.mf_symbolic_analyze(handle, rp, ci)
        try:
            sup = mf.mf_symbolic_supernodes(s)
            assert sup[0] == 0 and sup[1] == k  # the front of the k pivots
            cc = mf.mf_symbolic_colcounts(s)
            assert cc[0] == k + m  # with its m update rows
            F = orc.factor(rp, ci, v, None)
            B = gen.rhs(n, 2, seed=k + m)
            for prec in (mf.MF_FP64, mf.MF_FP32):
                f = mf.mf_factor_create(handle, s, prec)
                try:
                    mf.mf_factor_numeric(f, v)
                    Lx = mf.mf_factor_export_L(f, len(F.Lx))
                    relF = orc.rel_fro(Lx, F.Lx)
                    if prec == mf.MF_FP64:
                        X = mf.mf_solve(f, B)
                        assert relF <= RELF64, (k, m, relF)
                    else:
                        X, rep = mf.mf_solve_refined(f, B, tol=BERR, max_iter=30)
                        assert rep["fell_back"] == 0, (k, m)
                        assert relF <= 5e-4, (k, m, relF)
                    assert orc.berr(rp, ci, v, X, B) <= BERR, (k, m, prec)
                finally:
                    mf.mf_factor_free(f)
        finally:
            mf.mf_symbolic_free(s)
