"""Pins of the oracle's LDL^T (no pivoting) and its solve, independent of
its C code.

* SPD inputs: L D L^T relates to numpy's Cholesky C = G G^T by
  L = G diag(G)^-1 and D = diag(G)^2.
* Indefinite inputs (the quasi-definite saddle-point matrices): the pivots
  are ratios of leading principal minors, d_k = det(C_1:k) / det(C_1:k-1)
  (numpy determinants), and L D L^T reproduces C to rounding.
* The 1D Laplacian tridiag(-1, 2, -1): d_k = (k + 1) / k and
  l_{k+1,k} = -k / (k + 1) (1-based).
* Manufactured solutions of indefinite systems."""
import numpy as np
import pytest

import gen


def dense(rp, ci, v):
    n = len(rp) - 1
    A = np.zeros((n, n))
    A[np.repeat(np.arange(n), np.diff(rp)), ci] = v
    return A


@pytest.mark.parametrize("seed", range(4))
def test_spd_relates_to_cholesky(orc, seed):
    n = [20, 45, 60, 33][seed]
    rp, ci, v = gen.random_spd(n, 0.15, seed + 70)
    perm = gen.random_perm(n, seed)
    F = orc.factor_ldlt(rp, ci, v, perm)
    assert F.bad_col == -1
    C = dense(rp, ci, v)[np.ix_(perm, perm)]
    G = np.linalg.cholesky(C)
    g = np.diag(G)
    assert np.allclose(F.dense(), G / g[None, :], rtol=1e-12, atol=1e-12)
    assert np.allclose(F.D, g ** 2, rtol=1e-12)


@pytest.mark.parametrize("shape,seed", [((3, 3, 2), 0), ((4, 3, 2), 1), ((2, 2, 5), 2)])
def test_indefinite_pivots_are_minor_ratios(orc, shape, seed):
    rp, ci, v = gen.kkt_3d(*shape, seed=seed)
    perm = gen.nd_perm(shape, dofs=2)
    F = orc.factor_ldlt(rp, ci, v, perm)
    assert F.bad_col == -1
    C = dense(rp, ci, v)[np.ix_(perm, perm)]
    n = len(C)
    sign, logdet = zip(*[np.linalg.slogdet(C[:k, :k]) for k in range(1, n + 1)])
    dets = np.array(sign) * np.exp(np.array(logdet))
    want = dets / np.concatenate([[1.0], dets[:-1]])
    assert np.allclose(F.D, want, rtol=1e-8)
    assert np.any(F.D < 0) and np.any(F.D > 0)  # really indefinite
    L = F.dense()
    R = L @ np.diag(F.D) @ L.T - C
    assert np.max(np.abs(R)) <= 100 * n * 2.2e-16 * np.max(np.abs(C)) * np.max(np.abs(L)) ** 2


def test_1d_closed_form(orc):
    n = 30
    rp, ci, v = gen.laplacian_1d(n)
    F = orc.factor_ldlt(rp, ci, v, None)
    k = np.arange(1, n + 1, dtype=np.float64)
    assert np.allclose(F.D, (k + 1) / k, rtol=1e-14)
    L = F.dense()
    assert np.allclose(np.diag(L, -1), -k[:-1] / (k[:-1] + 1), rtol=1e-14)
    assert np.allclose(np.diag(L), 1.0)


def test_indefinite_manufactured_solution(orc):
    rp, ci, v = gen.kkt_3d(5, 4, 3, seed=3)
    perm = gen.nd_perm((5, 4, 3), dofs=2)
    n = len(rp) - 1
    F = orc.factor_ldlt(rp, ci, v, perm)
    xs = np.random.default_rng(1).uniform(-1, 1, (n, 2))
    b = np.stack([gen.csr_matvec(rp, ci, v, xs[:, r]) for r in range(2)], axis=1)
    x = orc.solve_ldlt(F, b, perm)
    assert orc.berr(rp, ci, v, x, b) <= 1e-15
    assert np.allclose(x, xs, rtol=1e-9, atol=1e-9)
