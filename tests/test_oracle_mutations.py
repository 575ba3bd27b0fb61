"""The oracle's pins must catch plausible mistakes.  Each case plants one
mistake in a copy of oracle/oracle.c (a wrong sign, a dropped term, a
transposed operand, a wrong index, a wrong operation), compiles it with gcc,
runs the pins against it on the CPU and requires at least one to fail.  Only
mistakes that keep every array size consistent are planted, so a mutated
oracle computes wrong numbers but never writes outside its buffers.  The
backward error (plain numpy in oracle/__init__.py) gets the same treatment:
a mistake planted in a copy of its source must fail the hand-computed pins
of tests/_berr_pins.py."""
import inspect
import os
import subprocess

import numpy as np
import pytest

import gen

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                   "oracle.c")

MUTATIONS = [
    ("factor: update sign flipped", "x[Li[t]] -= Lx[t] * ljk;", "x[Li[t]] += Lx[t] * ljk;"),
    ("factor: diagonal term of the update dropped",
     "for (int64_t t = q; t < Lp[k + 1]; ++t) x[Li[t]]",
     "for (int64_t t = q + 1; t < Lp[k + 1]; ++t) x[Li[t]]"),
    ("factor: L_kk used for L_jk (transposed operand)", "double ljk = Lx[q];",
     "double ljk = Lx[Lp[k]];"),
    ("factor: square root dropped", "double ljj = sqrt(d);", "double ljj = d;"),
    ("factor: column scaled by multiplying", "Lx[t] = x[i] / ljj;", "Lx[t] = x[i] * ljj;"),
    ("etree: parent taken as the next column", "if (next == -1) parent[r] = (int32_t)i;",
     "if (next == -1) parent[r] = (int32_t)(r + 1);"),
    ("supernodes: count condition off by one", "colcnt[j] == colcnt[j + 1] + 1",
     "colcnt[j] == colcnt[j + 1]"),
    ("supernodes: only-child condition dropped", "&&\n                nchild[j + 1] == 1;", ";"),
    ("solve: forward update sign flipped", "b[Li[t]] -= Lx[t] * zj;", "b[Li[t]] += Lx[t] * zj;"),
    ("solve: backward uses L instead of L^T", "s -= Lx[t] * b[Li[t]];", "s -= Lx[t] * b[j];"),
]


def pins(orc):
    """Pins of the oracle (independent of its C code: brute-force boolean
    elimination, numpy dense Cholesky, the 1D closed form, the supernode
    definition, manufactured solutions).  Returns the names of those that
    fail."""
    failed = set()

    def check(name, fn):
        try:
            if not fn():
                failed.add(name)
        except Exception:
            failed.add(name)

    for seed in range(4):
        n = [12, 30, 45, 60][seed]
        rp, ci, v = gen.random_spd(n, 0.15, seed + 500)
        perm = gen.random_perm(n, seed + 7)
        so = orc.symbolic(rp, ci, perm)
        bp, bc = orc.brute_symbolic(rp, ci, perm)
        check("brute etree", lambda: np.array_equal(so["parent"], bp))
        check("brute counts", lambda: np.array_equal(so["colcount"], bc))

        def supernode_definition():
            want = [0] + [j + 1 for j in range(n - 1)
                          if not (bp[j] == j + 1 and bc[j] == bc[j + 1] + 1
                                  and np.sum(bp == j + 1) == 1)] + [n]
            return np.array_equal(so["sup_ptr"], want)
        check("supernode definition", supernode_definition)

        A = np.zeros((n, n))
        A[np.repeat(np.arange(n), np.diff(rp)), ci] = v
        C = A[np.ix_(perm, perm)]
        F = orc.factor(rp, ci, v, perm)
        check("numpy cholesky", lambda: F.bad_col == -1 and np.allclose(
            F.dense(), np.linalg.cholesky(C), rtol=1e-12, atol=1e-12))
        xs = np.random.default_rng(seed).uniform(-1, 1, n)
        b = A @ xs
        check("manufactured solve", lambda: np.allclose(orc.solve(F, b, perm), xs, rtol=1e-9,
                                                       atol=1e-9))
    n = 20
    rp, ci, v = gen.laplacian_1d(n)
    F = orc.factor(rp, ci, v, None)
    k = np.arange(1, n + 1, dtype=np.float64)
    check("1D closed form", lambda: F.bad_col == -1 and np.allclose(
        F.Lx[F.Lp[:-1]], np.sqrt((k + 1) / k), rtol=1e-14))
    return failed


def test_pins_pass_on_the_oracle(orc):
    assert pins(orc) == set()


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(orc, tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation site not unique: " + name
    mutated = tmp_path / "oracle_mut.c"
    mutated.write_text(src.replace(old, new))
    lib_path = tmp_path / "liboracle_mut.so"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", str(lib_path), str(mutated),
                           "-lm"])
    saved = orc._load()
    orc._lib = orc.load_library(str(lib_path))
    try:
        failed = pins(orc)
    finally:
        orc._lib = saved
    assert failed, "no pin caught: " + name


BERR_MUTATIONS = [
    ("berr: ||b|| term dropped", " + np.max(np.abs(Bm[:, r]))", ""),
    ("berr: first right-hand side only", "for r in range(X.shape[1]):", "for r in range(1):"),
    ("berr: ||A|| taken as the largest entry",
     "np.max(np.bincount(rows, weights=np.abs(values), minlength=n))", "np.max(np.abs(values))"),
    ("berr: residual sign flipped", "np.abs(Bm[:, r] - ax)", "np.abs(Bm[:, r] + ax)"),
    ("berr: transposed operand in A x", "values * X[colind, r]", "values * X[rows, r]"),
    ("berr: ||x|| as a 1-norm", "np.max(np.abs(X[:, r]))", "np.sum(np.abs(X[:, r]))"),
]


@pytest.mark.parametrize("name,old,new", BERR_MUTATIONS, ids=[m[0] for m in BERR_MUTATIONS])
def test_berr_pins_catch_planted_mistake(orc, name, old, new):
    import _berr_pins
    src = inspect.getsource(orc.berr)
    assert src.count(old) == 1, "mutation site not unique: " + name
    ns = {"np": np}
    exec(src.replace(old, new), ns)
    assert _berr_pins.failures(ns["berr"]), "no pin caught: " + name


ILU_MUTATIONS = [
    ("iluk: level rule without the + 1", "int32_t nl = lk + Slev[q] + 1;", "int32_t nl = lk + Slev[q];"),
    ("ilu: multiplier not divided by the pivot", "double lik = vals[q] / vals[diag[k]];",
     "double lik = vals[q];"),
    ("fastilu: sum includes k = min(i, j)",
     "t < cp[j + 1] && cr[t] < m;", "t < cp[j + 1] && cr[t] <= m;"),
    ("fastilu: divided by u_ij instead of u_jj",
     "omega * s / old[diag[j]];", "omega * s / old[q];"),
    ("fastilu: damping applied to the wrong term",
     "out[q] = (1.0 - omega) * old[q] + omega * s;", "out[q] = omega * old[q] + (1.0 - omega) * s;"),
    ("fast_trsv: upper diagonal not divided", "if (upper) s /= lu[diag[i]];", ""),
]


def ilu_pins(orc):
    """The hand-worked first sweeps, the fixed point, the complete-fill LU,
    brute-force levels and exact triangular solves; names of the failures."""
    import _ilu_pin_cases as c
    return c.failures(orc)


@pytest.mark.parametrize("name,old,new", ILU_MUTATIONS, ids=[m[0] for m in ILU_MUTATIONS])
def test_ilu_pins_catch_planted_mistake(orc, tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation site not unique: " + name
    mutated = tmp_path / "oracle_mut.c"
    mutated.write_text(src.replace(old, new))
    lib_path = tmp_path / "liboracle_mut.so"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", str(lib_path), str(mutated),
                           "-lm"])
    saved = orc._load()
    orc._lib = orc.load_library(str(lib_path))
    try:
        failed = ilu_pins(orc)
    finally:
        orc._lib = saved
    assert failed, "no pin caught: " + name


def test_ilu_pins_pass_on_the_oracle(orc):
    assert ilu_pins(orc) == set()


LDLT_MUTATIONS = [
    ("ldlt: pivot weight d_k dropped from the update", "double w = Lx[q] * D[k];",
     "double w = Lx[q];"),
    ("ldlt: diagonal of L set to the pivot", "Lx[Lp[j]] = 1.0;", "Lx[Lp[j]] = d;"),
    ("ldlt: column not divided by the pivot", "Lx[t] = x[i] / d;", "Lx[t] = x[i];"),
    ("ldlt solve: D^{-1} step dropped", "for (int64_t j = 0; j < n; ++j) b[j] /= D[j];", ""),
    ("ldlt solve: backward uses L instead of L^T", "acc -= Lx[t] * b[Li[t]];",
     "acc -= Lx[t] * b[j];"),
]


def ldlt_pins(orc):
    import test_oracle_ldlt as t
    bad = set()
    for name, fn in [("cholesky", lambda: t.test_spd_relates_to_cholesky(orc, 1)),
                     ("minors", lambda: t.test_indefinite_pivots_are_minor_ratios(orc, (3, 3, 2), 0)),
                     ("1d", lambda: t.test_1d_closed_form(orc)),
                     ("manufactured", lambda: t.test_indefinite_manufactured_solution(orc))]:
        try:
            fn()
        except Exception:
            bad.add(name)
    return bad


@pytest.mark.parametrize("name,old,new", LDLT_MUTATIONS, ids=[m[0] for m in LDLT_MUTATIONS])
def test_ldlt_pins_catch_planted_mistake(orc, tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation site not unique: " + name
    mutated = tmp_path / "oracle_mut.c"
    mutated.write_text(src.replace(old, new))
    lib_path = tmp_path / "liboracle_mut.so"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", str(lib_path), str(mutated),
                           "-lm"])
    saved = orc._load()
    orc._lib = orc.load_library(str(lib_path))
    try:
        failed = ldlt_pins(orc)
    finally:
        orc._lib = saved
    assert failed, "no pin caught: " + name


def test_ldlt_pins_pass_on_the_oracle(orc):
    assert ldlt_pins(orc) == set()


LU_MUTATIONS = [
    ("lu: pivot of smallest magnitude",
     "fabs(colj[i]), b = fabs(colj[p]);\n      if (a > b || (a == b && rho[i] < rho[p])) p = i;",
     "fabs(colj[i]), b = fabs(colj[p]);\n      if (a < b || (a == b && rho[i] < rho[p])) p = i;"),
    ("lu: ties to the largest original row",
     "fabs(colj[i]), b = fabs(colj[p]);\n      if (a > b || (a == b && rho[i] < rho[p])) p = i;",
     "fabs(colj[i]), b = fabs(colj[p]);\n      if (a > b || (a == b && rho[i] > rho[p])) p = i;"),
    ("lu: window ignored",
     "for (int64_t i = j + 1; i < wend[j]; ++i) {\n      double a = fabs(colj[i])",
     "for (int64_t i = j + 1; i < n; ++i) {\n      double a = fabs(colj[i])"),
    ("lu: factored columns not swapped", "for (int64_t c = 0; c < n; ++c) {\n        double tmp",
     "for (int64_t c = j; c < n; ++c) {\n        double tmp"),
    ("lu: row order not recorded", "rho[p] = tr;\n    }\n    double piv = colj[j];",
     "rho[p] = rho[j];\n    }\n    double piv = colj[j];"),
    ("lu: U row multiplied by the pivot", "*ujc /= piv;", "*ujc *= piv;"),
    ("lu: update sign flipped", "colc[nzr[q]] -= colj[nzr[q]] * u;",
     "colc[nzr[q]] += colj[nzr[q]] * u;"),
    ("lu: L_cj used for U_jc (transposed operand)", "double u = colc[j];",
     "double u = colj[nzc[t]];"),
]


def lu_pins(orc):
    import test_oracle_lu as t
    bad = set()
    for name, fn in [("dominant", lambda: t.test_no_pivoting_matches_scipy_on_column_dominant(orc, 1)),
                     ("one window", lambda: t.test_one_window_is_partial_pivoting(orc, 0)),
                     ("blocks", lambda: t.test_block_diagonal_windows_are_per_block_partial_pivoting(orc)),
                     ("invariants", lambda: t.test_windowed_pivoting_invariants(orc, 4, 1)),
                     ("cholesky", lambda: t.test_spd_without_pivoting_relates_to_cholesky(orc, 0)),
                     ("tridiagonal", lambda: t.test_tridiagonal_closed_form(orc)),
                     ("zero diagonal", lambda: t.test_zero_diagonal_needs_pivoting(orc)),
                     ("ties", lambda: t.test_ties_go_to_the_smallest_original_row(orc))]:
        try:
            fn()
        except Exception:
            bad.add(name)
    return bad


@pytest.mark.parametrize("name,old,new", LU_MUTATIONS, ids=[m[0] for m in LU_MUTATIONS])
def test_lu_pins_catch_planted_mistake(orc, tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation site not unique: " + name
    mutated = tmp_path / "oracle_mut.c"
    mutated.write_text(src.replace(old, new))
    lib_path = tmp_path / "liboracle_mut.so"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", str(lib_path), str(mutated),
                           "-lm"])
    saved = orc._load()
    orc._lib = orc.load_library(str(lib_path))
    try:
        failed = lu_pins(orc)
    finally:
        orc._lib = saved
    assert failed, "no pin caught: " + name


def test_lu_pins_pass_on_the_oracle(orc):
    assert lu_pins(orc) == set()


LDLT_PIV_MUTATIONS = [
    ("ldlt piv: smallest diagonal as pivot",
     "double a = fabs(M[i * n + i]), b = fabs(M[p * n + p]);\n      if (a > b ||",
     "double a = fabs(M[i * n + i]), b = fabs(M[p * n + p]);\n      if (a < b ||"),
    ("ldlt piv: window ignored",
     "for (int64_t i = j + 1; i < wend[j]; ++i) {\n      double a = fabs(M[i * n + i])",
     "for (int64_t i = j + 1; i < n; ++i) {\n      double a = fabs(M[i * n + i])"),
    ("ldlt piv: columns not swapped", "for (int64_t r = 0; r < n; ++r) { /* columns j and p */",
     "for (int64_t r = 0; r < 0; ++r) { /* columns j and p */"),
    ("ldlt piv: rows not swapped", "for (int64_t c = 0; c < n; ++c) { /* rows j and p */",
     "for (int64_t c = 0; c < 0; ++c) { /* rows j and p */"),
    ("ldlt piv: row order not recorded", "rho[p] = tr;\n    }\n    double* colj",
     "rho[p] = rho[j];\n    }\n    double* colj"),
    ("ldlt piv: update sign flipped", "colc[nzr[q]] -= colj[nzr[q]] * w;",
     "colc[nzr[q]] += colj[nzr[q]] * w;"),
    ("ldlt piv: column not divided by the pivot", "for (int64_t q = 0; q < nr; ++q) colj[nzr[q]] /= dj;",
     "for (int64_t q = 0; q < nr; ++q) colj[nzr[q]] *= 1.0;"),
    ("ldlt piv: update without the pivot", "double w = colj[nzr[t]] / dj;",
     "double w = colj[nzr[t]];"),
]


def ldlt_piv_pins(orc):
    import test_oracle_ldlt_piv as t
    bad = set()
    for name, fn in [("no pivoting", lambda: t.test_no_pivoting_equals_left_looking_ldlt(orc, (3, 3, 2), 0)),
                     ("pstrf", lambda: t.test_one_window_spd_is_pivoted_cholesky(orc, 1)),
                     ("invariants", lambda: t.test_windowed_symmetric_pivoting_invariants(orc, 2, 1)),
                     ("zero block", lambda: t.test_zero_block_needs_pivoting(orc)),
                     ("hand", lambda: t.test_hand_worked_with_tie(orc))]:
        try:
            fn()
        except Exception:
            bad.add(name)
    return bad


@pytest.mark.parametrize("name,old,new", LDLT_PIV_MUTATIONS, ids=[m[0] for m in LDLT_PIV_MUTATIONS])
def test_ldlt_piv_pins_catch_planted_mistake(orc, tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation site not unique: " + name
    mutated = tmp_path / "oracle_mut.c"
    mutated.write_text(src.replace(old, new))
    lib_path = tmp_path / "liboracle_mut.so"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", str(lib_path), str(mutated),
                           "-lm"])
    saved = orc._load()
    orc._lib = orc.load_library(str(lib_path))
    try:
        failed = ldlt_piv_pins(orc)
    finally:
        orc._lib = saved
    assert failed, "no pin caught: " + name


def test_ldlt_piv_pins_pass_on_the_oracle(orc):
    assert ldlt_piv_pins(orc) == set()
