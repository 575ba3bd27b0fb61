"""Pins of the FastILU / FastSpTRSV oracle (paper Sec. 6), independent of its
C code.

* The ILU(k) pattern against a dense level-of-fill elimination written here
  (levels 0 for the entries of A and the diagonal, lev(i,k) + lev(k,j) + 1
  through each eliminated k, keep level <= k).
* The incomplete LU with k >= n is the exact LU, taken from numpy's
  Cholesky (A = C C^T gives L = C diag(C)^-1, U = diag(C) C^T).
* The exact incomplete factors are a fixed point of the sweep, the sweeps
  converge to them, and the first sweeps of a 3 x 3 tridiagonal system are
  worked out by hand below.
* FastSpTRSV after n sweeps equals the exact triangular solve (numpy), and
  its first sweep from x = 0 is b (unit lower) or b / u_ii (upper)."""
import numpy as np
import pytest
import scipy.sparse as sp

import gen


def dense(rp, ci, v, n):
    A = np.zeros((n, n))
    A[np.repeat(np.arange(n), np.diff(rp)), ci] = v
    return A


def brute_levels(rp, ci, n, K):
    INF = 10 ** 9
    lev = np.full((n, n), INF, dtype=np.int64)
    lev[np.repeat(np.arange(n), np.diff(rp)), ci] = 0
    np.fill_diagonal(lev, 0)
    for i in range(n):
        for k in range(i):
            if lev[i, k] > K:
                continue
            for j in range(k + 1, n):
                if lev[k, j] <= K:
                    lev[i, j] = min(lev[i, j], lev[i, k] + lev[k, j] + 1)
    return lev


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("K", [0, 1, 2, 5])
def test_iluk_pattern_brute_force(orc, seed, K):
    n = [9, 17, 25, 33, 40, 12][seed]
    rp, ci, _ = gen.random_spd(n, 0.12, seed + 40)
    pat = orc.iluk_pattern(rp, ci, K)
    lev = brute_levels(rp, ci, n, K)
    rows = np.repeat(np.arange(n), np.diff(pat.Sp))
    assert len(pat.Sj) == int(np.sum(lev <= K))
    assert np.all(lev[rows, pat.Sj] <= K)
    assert np.array_equal(pat.Slev, lev[rows, pat.Sj])
    for i in range(n):
        assert np.all(np.diff(pat.Sj[pat.Sp[i]:pat.Sp[i + 1]]) > 0)


def lu_from_cholesky(A):
    C = np.linalg.cholesky(A)
    d = np.diag(C)
    return C / d[None, :], d[:, None] * C.T


@pytest.mark.parametrize("case", ["random", "elasticity", "tridiagonal"])
def test_complete_fill_is_exact_lu(orc, case):
    if case == "random":
        rp, ci, v = gen.random_spd(30, 0.15, 3)
    elif case == "elasticity":
        rp, ci, v = gen.elasticity_3d(3)
    else:
        rp, ci, v = gen.laplacian_1d(25)
    n = len(rp) - 1
    K = 0 if case == "tridiagonal" else n  # a tridiagonal matrix has no fill
    pat = orc.iluk_pattern(rp, ci, K)
    lu = orc.ilu_exact(pat, pat.values_of(rp, ci, v))
    L, U = lu_from_cholesky(dense(rp, ci, v, n))
    want = np.where(pat.rows > pat.Sj, L[pat.rows, pat.Sj], U[pat.rows, pat.Sj])
    assert np.allclose(lu, want, rtol=1e-11, atol=1e-11 * np.max(np.abs(U)))
    # and S holds every nonzero of the exact factors
    assert np.count_nonzero(np.abs(np.tril(L, -1)) + np.abs(U) > 1e-14) <= len(pat.Sj)


def test_first_sweeps_by_hand(orc):
    """A = tridiag(1, 4, 1) of order 3, ILU(0) = its LU.  Entries in row
    order: u11, u12, l21, u22, u23, l32, u33.  Initial guess l_ij = a_ij/a_jj,
    u_ij = a_ij.  Sweep 1: u22 = 4 - l21 u12 = 3.75, l32 = a32 / u22(old) =
    1/4, u33 = 4 - l32(old) u23 = 3.75.  Sweep 2: l32 = 1 / 3.75.  Sweep 3:
    u33 = 4 - 1/3.75 (the exact LU).  With omega = 1/2 the first sweep gives
    u22 = u33 = (4 + 3.75) / 2."""
    rp, ci, v = gen.laplacian_1d(3)
    v = np.where(v > 0, 4.0, 1.0)
    pat = orc.iluk_pattern(rp, ci, 0)
    a = pat.values_of(rp, ci, v)
    got = [orc.fastilu(pat, a, s) for s in (1, 2, 3)]
    want1 = [4, 1, 0.25, 3.75, 1, 0.25, 3.75]
    want2 = [4, 1, 0.25, 3.75, 1, 1 / 3.75, 3.75]
    want3 = [4, 1, 0.25, 3.75, 1, 1 / 3.75, 4 - 1 / 3.75]
    for g, w in zip(got, (want1, want2, want3)):
        assert np.allclose(g, w, rtol=0, atol=1e-15)
    half = orc.fastilu(pat, a, 1, omega=0.5)
    assert np.allclose(half, [4, 1, 0.25, 3.875, 1, 0.25, 3.875], rtol=0, atol=1e-15)


@pytest.mark.parametrize("K", [0, 1, 2])
def test_exact_factors_are_the_fixed_point(orc, K):
    rp, ci, v = gen.elasticity_3d(4)
    pat = orc.iluk_pattern(rp, ci, K)
    a = pat.values_of(rp, ci, v)
    ex = orc.ilu_exact(pat, a)
    once = orc.fastilu(pat, a, 1, start=ex)
    assert np.max(np.abs(once - ex)) <= 1e-12 * np.max(np.abs(ex))
    many = orc.fastilu(pat, a, 60)
    assert np.max(np.abs(many - ex)) <= 1e-9 * np.max(np.abs(ex))


def test_warmup_starts_from_the_lower_level(orc):
    """Warm-up: FastILU(k-1) gives the initial values of the level < k
    entries, the level-k entries start at zero."""
    rp, ci, v = gen.laplacian_3d(5)
    pat = orc.iluk_pattern(rp, ci, 2)
    a = pat.values_of(rp, ci, v)
    w = orc.fastilu(pat, a, 2, warmup=True)
    l1 = orc.fastilu(pat, a, 2, warmup=True, K=1)
    start = np.where(pat.Slev < 2, l1, 0.0)
    assert np.array_equal(w, orc.fastilu(pat, a, 2, start=start))
    # and warm-up changes the result (it is not the plain initial guess)
    assert not np.allclose(w, orc.fastilu(pat, a, 2))


@pytest.mark.parametrize("upper", [0, 1])
def test_fast_trsv_exact_after_n_sweeps(orc, upper):
    rp, ci, v = gen.elasticity_3d(3)
    n = len(rp) - 1
    pat = orc.iluk_pattern(rp, ci, 1)
    lu = orc.ilu_exact(pat, pat.values_of(rp, ci, v))
    T = np.zeros((n, n))
    T[pat.rows, pat.Sj] = lu
    T = np.triu(T) if upper else np.tril(T, -1) + np.eye(n)
    b = gen.rhs(n, 1, seed=4)
    x = orc.fast_trsv(pat, lu, b, upper, n)
    assert np.allclose(x, np.linalg.solve(T, b), rtol=1e-12, atol=1e-12)
    one = orc.fast_trsv(pat, lu, b, upper, 1)
    assert np.allclose(one, b / np.diag(T), rtol=1e-15, atol=0)
