"""FP64 CPU oracle for the multifrontal Cholesky path -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library never does, and this
package imports nothing from the library.

What it computes (paper Sec. 5, Tacho: symbolic analysis, numerical
factorization ``P A P^T = L L^T`` of an SPD matrix, forward/backward solve;
the three phases of the paper's Ax=b statement in Sec. 3):

* ``lower_rows`` / ``lower_cols`` -- the lower triangle of ``C = A(perm, perm)``
  (``perm[new] = old``), duplicates summed.  Plain numpy.
* ``etree``      -- ``parent(j) = min{i > j : L_ij != 0}`` (Liu's algorithm, C).
* ``colcounts``  -- ``c_j = |struct(L_{*,j})|`` by row-subtree walks (C).
* ``supernodes`` -- fundamental supernode partition (C).
* ``factor``     -- left-looking column Cholesky, FP64 (C); optionally only the
  columns of a descendant-closed set (exact for those columns).
* ``solve``      -- ``x = P^T L^{-T} L^{-1} P b`` (C).
* ``factor_ldlt`` / ``solve_ldlt`` -- LDL^T without pivoting of a symmetric
  (possibly indefinite) C, and its solve (C).
* ``lu_dense`` / ``solve_lu`` / ``pivot_windows`` -- LU of a general matrix
  with a symmetric pattern (Crout: L lower, U unit upper), pivots looked for
  only within diagonal blocks, and its solve (dense, C).
* ``ldlt_dense`` / ``solve_ldlt_piv`` -- LDL^T with symmetric (1x1) pivoting
  within diagonal blocks and its solve (dense, C).
* ``expand_node_blocks`` -- the block-expanded pattern a condensed-graph
  analysis stands for (plain Python sets).
* ``brute_symbolic`` -- dense boolean elimination on tiny inputs (pure Python),
  an independent pin for etree / counts / nnz(L).
* ``berr``, ``rel_fro`` -- the error measures used by the parity tests.
* ``iluk_pattern``, ``ilu_exact``, ``fastilu``, ``fast_trsv`` -- FastILU and
  FastSpTRSV (paper Sec. 6): the ILU(k) pattern by levels of fill, the
  incomplete LU on it (the sweeps' fixed point), the sweeps of the factor
  (out of place) and of the triangular solves (C).

Pins (tests/test_oracle.py; LU: tests/test_oracle_lu.py, scipy's partially
pivoted LU, the Thomas recurrence, the Cholesky relation): dense numpy Cholesky, the closed-form 1D
Laplacian factor, the Dirichlet-Laplacian log-determinant, brute-force symbolic
elimination and the etree/count invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force=False):
    """Compile the C oracle with the host compiler (portable flags only;
    OpenMP for the multi-threaded factorization where the compiler has it)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    try:
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC,
                               "-lm"], stderr=subprocess.DEVNULL)
    except subprocess.CalledProcessError:
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def load_library(path):
    """Open a compiled oracle.c with its argument types declared.  The tests
    that plant a mistake in a copy of oracle.c load that copy with this and
    put it in place of the real library while the pins run."""
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    I = ctypes.c_int64
    lib.orc_etree.argtypes = [I, P, P, P, P]
    lib.orc_counts.argtypes = [I, P, P, P, P, P, P, P]
    lib.orc_pattern.argtypes = [I, P, P, P, P, P, P, P, P, P, P, P]
    lib.orc_factor.argtypes = [I, P, P, P, P, P, P, P, P, P, P, P, P]
    lib.orc_factor.restype = ctypes.c_int64
    lib.orc_par_threads.argtypes = [ctypes.c_int]
    lib.orc_par_threads.restype = ctypes.c_int
    lib.orc_factor_par.argtypes = [I, P, P, P, P, P, P, P, P, P, P, P, ctypes.c_int, P, P, P,
                                   P, P, P]
    lib.orc_factor_par.restype = ctypes.c_int64
    lib.orc_supernodes.argtypes = [I, P, P, P, P]
    lib.orc_supernodes.restype = ctypes.c_int64
    lib.orc_solve.argtypes = [I, P, P, P, P, I, I]
    lib.orc_factor_ldlt.argtypes = [I, P, P, P, P, P, P, P, P, P, P, P, P]
    lib.orc_factor_ldlt.restype = ctypes.c_int64
    lib.orc_solve_ldlt.argtypes = [I, P, P, P, P, P, I, I]
    lib.orc_iluk_pattern.argtypes = [I, P, P, ctypes.c_int32, I, P, P, P, P, P, P]
    lib.orc_iluk_pattern.restype = ctypes.c_int64
    lib.orc_ilu_exact.argtypes = [I, P, P, P, ctypes.c_int32, P, P, P]
    lib.orc_fastilu_sweep.argtypes = [I, P, P, P, ctypes.c_int32, P, P, P, P, P, P, P,
                                      ctypes.c_double, P, P]
    lib.orc_fast_trsv_sweep.argtypes = [I, P, P, P, ctypes.c_int32, P, P, ctypes.c_int, P, P, P,
                                        ctypes.c_double]
    lib.orc_lu_dense.argtypes = [I, P, P, P, P, P]
    lib.orc_lu_dense.restype = ctypes.c_int64
    lib.orc_ldlt_dense.argtypes = [I, P, P, P, P, P]
    lib.orc_ldlt_dense.restype = ctypes.c_int64
    return lib


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = load_library(_LIB)
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------------------
# Lower triangle of C = A(perm, perm)
# ---------------------------------------------------------------------------
def _lower_coo(rowptr, colind, values, perm):
    n = len(rowptr) - 1
    rowptr = np.asarray(rowptr, dtype=np.int64)
    if perm is None:
        iperm = np.arange(n, dtype=np.int64)
    else:
        perm = np.asarray(perm, dtype=np.int64)
        iperm = np.empty(n, dtype=np.int64)
        iperm[perm] = np.arange(n)
    rows_old = np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr))
    i = iperm[rows_old]
    j = iperm[np.asarray(colind, dtype=np.int64)]
    keep = i >= j
    v = None if values is None else np.asarray(values, dtype=np.float64)[keep]
    return n, i[keep], j[keep], v


def lower_rows(rowptr, colind, perm):
    """Strict lower triangle of C by rows: (rp int64[n+1], ci int32), sorted, unique."""
    n, i, j, _ = _lower_coo(rowptr, colind, None, perm)
    strict = i > j
    key = np.sort(i[strict] * n + j[strict])
    if len(key):
        key = key[np.concatenate(([True], key[1:] != key[:-1]))]
    r = key // n
    c = (key % n).astype(np.int32)
    rp = np.zeros(n + 1, dtype=np.int64)
    rp[1:] = np.cumsum(np.bincount(r, minlength=n))
    return rp, c


def lower_cols(rowptr, colind, values, perm):
    """Lower triangle of C (incl. diagonal) by columns, duplicates summed:
    (Cp int64[n+1], Cr int32, Cx float64), rows ascending within a column."""
    n, i, j, v = _lower_coo(rowptr, colind, values, perm)
    key = j * n + i
    order = np.argsort(key, kind="stable")
    key = key[order]
    v = v[order]
    uniq, start = np.unique(key, return_index=True)
    cx = np.add.reduceat(v, start) if len(v) else v
    c = uniq // n
    r = (uniq % n).astype(np.int32)
    cp = np.zeros(n + 1, dtype=np.int64)
    cp[1:] = np.cumsum(np.bincount(c, minlength=n))
    return cp, r, cx


# ---------------------------------------------------------------------------
# Symbolic
# ---------------------------------------------------------------------------
def etree(n, rp, ci):
    lib = _load()
    parent = np.empty(n, dtype=np.int32)
    anc = np.empty(n, dtype=np.int32)
    lib.orc_etree(n, _p(rp), _p(ci), _p(parent), _p(anc))
    return parent


def counts(n, rp, ci, parent, in_s=None):
    """(colcnt, rowcnt) restricted to columns in S (default: all)."""
    lib = _load()
    if in_s is None:
        in_s = np.ones(n, dtype=np.uint8)
    colcnt = np.empty(n, dtype=np.int64)
    rowcnt = np.empty(n, dtype=np.int64)
    mark = np.empty(n, dtype=np.int32)
    lib.orc_counts(n, _p(rp), _p(ci), _p(parent), _p(in_s), _p(colcnt), _p(rowcnt), _p(mark))
    return colcnt, rowcnt


def colcounts(n, rp, ci, parent):
    return counts(n, rp, ci, parent)[0]


def supernodes(n, parent, colcnt):
    lib = _load()
    sup = np.empty(n + 1, dtype=np.int32)
    nchild = np.empty(max(n, 1), dtype=np.int32)
    ns = lib.orc_supernodes(n, _p(parent), _p(colcnt), _p(sup), _p(nchild))
    return sup[: ns + 1].copy()


def symbolic(rowptr, colind, perm):
    """Dict with etree, colcounts, nnz(L), supernode partition and flops."""
    n = len(rowptr) - 1
    rp, ci = lower_rows(rowptr, colind, perm)
    parent = etree(n, rp, ci)
    cc = colcounts(n, rp, ci, parent)
    sup = supernodes(n, parent, cc)
    return {
        "n": n, "parent": parent, "colcount": cc, "nnzL": int(cc.sum()),
        "sup_ptr": sup, "flops": float(np.sum(cc.astype(np.float64) ** 2)),
        "rows": (rp, ci),
    }


def brute_symbolic(rowptr, colind, perm):
    """Dense boolean elimination on tiny inputs (n <= a few hundred).

    Returns (parent, colcount).  Independent of the C routines above."""
    n = len(rowptr) - 1
    A = np.zeros((n, n), dtype=bool)
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    A[rows, colind] = True
    if perm is not None:
        A = A[np.ix_(perm, perm)]
    A = A | A.T
    np.fill_diagonal(A, True)
    B = np.tril(A)
    for j in range(n):
        below = np.nonzero(B[j + 1:, j])[0] + j + 1
        for a in below:
            B[a, below[below <= a]] = True
    parent = np.full(n, -1, dtype=np.int32)
    for j in range(n):
        nz = np.nonzero(B[j + 1:, j])[0]
        if len(nz):
            parent[j] = j + 1 + nz[0]
    return parent, B.sum(axis=0).astype(np.int64)


# ---------------------------------------------------------------------------
# Numeric
# ---------------------------------------------------------------------------
class Factor:
    """L[:, S] in CSC form (Lp over all n columns; empty outside S)."""

    def __init__(self, n, Lp, Li, Lx, bad_col, flops):
        self.n, self.Lp, self.Li, self.Lx = n, Lp, Li, Lx
        self.bad_col = bad_col
        self.flops = flops

    def column(self, j):
        a, b = self.Lp[j], self.Lp[j + 1]
        return self.Li[a:b], self.Lx[a:b]

    def dense(self):
        L = np.zeros((self.n, self.n))
        for j in range(self.n):
            r, v = self.column(j)
            L[r, j] = v
        return L

    def logdet(self):
        """log det C = 2 sum log L_jj (full factor)."""
        return 2.0 * float(np.sum(np.log(self.Lx[self.Lp[:-1]])))


def threads_available():
    """Host threads the multi-threaded oracle uses by default (the CPUs this
    process may run on); 1 if the library was built without OpenMP."""
    lib = _load()
    try:
        cpus = len(os.sched_getaffinity(0))
    except AttributeError:
        cpus = os.cpu_count() or 1
    return min(cpus, lib.orc_par_threads(cpus))


def factor(rowptr, colind, values, perm, in_s=None, sym=None, threads=1):
    """Left-looking FP64 Cholesky of C = A(perm, perm); columns in S only.

    threads > 1 computes the columns of equal etree height in parallel
    (columns read only their own etree subtree), bitwise identical to the
    one-thread result; threads = 0 takes ``threads_available()``."""
    lib = _load()
    n = len(rowptr) - 1
    if sym is None:
        rp, ci = lower_rows(rowptr, colind, perm)
        parent = etree(n, rp, ci)
    else:
        rp, ci = sym["rows"]
        parent = sym["parent"]
    if in_s is None:
        in_s = np.ones(n, dtype=np.uint8)
    in_s = np.ascontiguousarray(in_s, dtype=np.uint8)
    colcnt, rowcnt = counts(n, rp, ci, parent, in_s)
    Lp = np.zeros(n + 1, dtype=np.int64)
    Lp[1:] = np.cumsum(colcnt)
    Rp = np.zeros(n + 1, dtype=np.int64)
    Rp[1:] = np.cumsum(rowcnt)
    Li = np.empty(int(Lp[-1]), dtype=np.int32)
    Rk = np.empty(int(Rp[-1]), dtype=np.int32)
    Rq = np.empty(int(Rp[-1]), dtype=np.int64)
    mark = np.empty(n, dtype=np.int32)
    fill = np.empty(n, dtype=np.int64)
    lib.orc_pattern(n, _p(rp), _p(ci), _p(parent), _p(in_s), _p(Lp), _p(Li), _p(Rp),
                    _p(Rk), _p(Rq), _p(mark), _p(fill))
    Cp, Cr, Cx = lower_cols(rowptr, colind, values, perm)
    Lx = np.zeros(int(Lp[-1]), dtype=np.float64)
    fl = ctypes.c_double(0.0)
    if threads == 0:
        threads = threads_available()
    nt = lib.orc_par_threads(int(threads)) if threads > 1 else 1
    if nt > 1:
        xs = np.zeros(nt * n, dtype=np.float64)
        height = np.empty(n, dtype=np.int32)
        order = np.empty(n, dtype=np.int32)
        hptr = np.empty(n + 2, dtype=np.int64)
        badm = np.empty(n, dtype=np.uint8)
        parent = np.ascontiguousarray(parent, dtype=np.int32)
        bad = lib.orc_factor_par(n, _p(Cp), _p(Cr), _p(Cx), _p(in_s), _p(Lp), _p(Li), _p(Lx),
                                 _p(Rp), _p(Rk), _p(Rq), _p(parent), nt, _p(xs), _p(height),
                                 _p(order), _p(hptr), _p(badm), ctypes.byref(fl))
    else:
        x = np.zeros(n, dtype=np.float64)
        bad = lib.orc_factor(n, _p(Cp), _p(Cr), _p(Cx), _p(in_s), _p(Lp), _p(Li), _p(Lx),
                             _p(Rp), _p(Rk), _p(Rq), _p(x), ctypes.byref(fl))
    F = Factor(n, Lp, Li, Lx, int(bad), fl.value)
    F.threads = nt
    return F


def factor_ldlt(rowptr, colind, values, perm, in_s=None, sym=None):
    """Left-looking FP64 LDL^T (no pivoting) of C = A(perm, perm); columns in
    S only.  Returns a Factor with L (unit diagonal stored) and F.D."""
    lib = _load()
    n = len(rowptr) - 1
    if sym is None:
        rp, ci = lower_rows(rowptr, colind, perm)
        parent = etree(n, rp, ci)
    else:
        rp, ci = sym["rows"]
        parent = sym["parent"]
    if in_s is None:
        in_s = np.ones(n, dtype=np.uint8)
    in_s = np.ascontiguousarray(in_s, dtype=np.uint8)
    colcnt, rowcnt = counts(n, rp, ci, parent, in_s)
    Lp = np.zeros(n + 1, dtype=np.int64)
    Lp[1:] = np.cumsum(colcnt)
    Rp = np.zeros(n + 1, dtype=np.int64)
    Rp[1:] = np.cumsum(rowcnt)
    Li = np.empty(int(Lp[-1]), dtype=np.int32)
    Rk = np.empty(int(Rp[-1]), dtype=np.int32)
    Rq = np.empty(int(Rp[-1]), dtype=np.int64)
    mark = np.empty(n, dtype=np.int32)
    fill = np.empty(n, dtype=np.int64)
    lib.orc_pattern(n, _p(rp), _p(ci), _p(parent), _p(in_s), _p(Lp), _p(Li), _p(Rp),
                    _p(Rk), _p(Rq), _p(mark), _p(fill))
    Cp, Cr, Cx = lower_cols(rowptr, colind, values, perm)
    Lx = np.zeros(int(Lp[-1]), dtype=np.float64)
    D = np.zeros(n, dtype=np.float64)
    x = np.zeros(n, dtype=np.float64)
    bad = lib.orc_factor_ldlt(n, _p(Cp), _p(Cr), _p(Cx), _p(in_s), _p(Lp), _p(Li), _p(Lx),
                              _p(D), _p(Rp), _p(Rk), _p(Rq), _p(x))
    F = Factor(n, Lp, Li, Lx, int(bad), float(np.sum(colcnt.astype(np.float64) ** 2)))
    F.D = D
    return F


def solve_ldlt(F, b, perm):
    """x = P^T L^{-T} D^{-1} L^{-1} P b."""
    lib = _load()
    n = F.n
    b = np.asarray(b, dtype=np.float64)
    one = b.ndim == 1
    B = b.reshape(n, -1)
    y = np.asfortranarray(B[perm] if perm is not None else B.copy())
    lib.orc_solve_ldlt(n, _p(F.Lp), _p(F.Li), _p(F.Lx), _p(F.D), _p(y), y.shape[1], n)
    x = np.empty_like(y)
    if perm is not None:
        x[perm] = y
    else:
        x[:] = y
    return x[:, 0] if one else x


def solve(F, b, perm):
    """x = P^T L^{-T} L^{-1} P b for b of shape (n,) or (n, nrhs)."""
    lib = _load()
    n = F.n
    b = np.asarray(b, dtype=np.float64)
    one = b.ndim == 1
    B = b.reshape(n, -1)
    y = np.asfortranarray(B[perm] if perm is not None else B.copy())
    lib.orc_solve(n, _p(F.Lp), _p(F.Li), _p(F.Lx), _p(y), y.shape[1], n)
    x = np.empty_like(y)
    if perm is not None:
        x[perm] = y
    else:
        x[:] = y
    return x[:, 0] if one else x


def descendant_closed(parent, roots):
    """Mask of the union of the etree subtrees rooted at ``roots``."""
    n = len(parent)
    in_s = np.zeros(n, dtype=np.uint8)
    roots = set(int(r) for r in roots)
    # a column belongs to S iff some ancestor-or-self is a chosen root;
    # ancestors have larger indices, so scan downwards
    memo = np.zeros(n, dtype=np.int8)  # 0 unknown, 1 in, 2 out
    for j in range(n - 1, -1, -1):
        if j in roots:
            memo[j] = 1
        else:
            p = parent[j]
            memo[j] = memo[p] if p >= 0 else 2
    in_s[memo == 1] = 1
    return in_s


def factor_sample(rowptr, colind, values, perm, seconds=15.0, sym=None):
    """Time the oracle on the first J columns of the elimination order
    (descendant-closed), growing J until the run takes about ``seconds``.

    Returns (flops, elapsed_s, J)."""
    n = len(rowptr) - 1
    if sym is None:
        rp, ci = lower_rows(rowptr, colind, perm)
        sym = {"rows": (rp, ci), "parent": etree(n, rp, ci)}
    J = max(1, n // 64)
    while True:
        in_s = np.zeros(n, dtype=np.uint8)
        in_s[:J] = 1
        t0 = time.perf_counter()
        F = factor(rowptr, colind, values, perm, in_s=in_s, sym=sym)
        dt = time.perf_counter() - t0
        if dt >= seconds * 0.5 or J >= n:
            return F.flops, dt, J
        J = min(n, int(J * max(2.0, min(8.0, seconds / max(dt, 1e-3)))))


# ---------------------------------------------------------------------------
# Condensed graph (paper Sec. 5: the DoFs of one node compressed into one
# vertex of the graph the symbolic analysis runs on)
# ---------------------------------------------------------------------------
def expand_node_blocks(rowptr, colind, values, node_of):
    """The block-expanded matrix the condensed-graph analysis describes:
    every node block (u, v) of A holding at least one entry, and every
    diagonal block (u, u), becomes dense; the entries of A keep their values
    (duplicates summed) and the added positions hold zeros.  Its symbolic
    analysis and Cholesky factor are what the condensed analysis must
    reproduce.  Returns (rowptr, colind, values) with columns sorted."""
    n = len(rowptr) - 1
    node_of = np.asarray(node_of, dtype=np.int64)
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    cols = np.asarray(colind, dtype=np.int64)
    nn = int(node_of.max()) + 1 if n else 0
    pairs = set(zip(node_of[rows].tolist(), node_of[cols].tolist()))
    pairs |= {(u, u) for u in set(node_of.tolist())}
    dofs = [[] for _ in range(nn)]
    for i in range(n):
        dofs[node_of[i]].append(i)
    entries = {}
    for (u, v) in pairs:
        for i in dofs[u]:
            for j in dofs[v]:
                entries[(i, j)] = 0.0
    for r, c, x in zip(rows.tolist(), cols.tolist(), np.asarray(values, dtype=np.float64).tolist()):
        entries[(r, c)] += x
    keys = sorted(entries)
    rp = np.zeros(n + 1, dtype=np.int64)
    for (r, _) in keys:
        rp[r + 1] += 1
    rp = np.cumsum(rp)
    ci = np.array([c for (_, c) in keys], dtype=np.int32)
    vx = np.array([entries[k] for k in keys], dtype=np.float64)
    return rp, ci, vx


# ---------------------------------------------------------------------------
# LU with a symmetric pattern, pivoting within diagonal blocks (Sec. 5)
# ---------------------------------------------------------------------------
class LU:
    """Pi C = L U of C = A(perm, perm): ``L`` dense lower triangular, ``U``
    dense unit upper triangular, ``rho[i]`` the row of C in position i,
    ``bad_col`` -1 or the first zero pivot."""

    def __init__(self, L, U, rho, bad_col):
        self.L, self.U, self.rho, self.bad_col = L, U, rho, bad_col
        self.n = len(rho)


def pivot_windows(starts, n, nb=64):
    """wend[j] for pivot windows cut out of a partition of 0..n-1: the blocks
    start at ``starts`` (ascending, starts[0] = 0), each block is cut into
    pieces of nb columns from its first one, and column j may take its pivot
    from the rows j .. wend[j]-1 of its piece."""
    bounds = list(np.asarray(starts, dtype=np.int64)) + [n]
    wend = np.empty(n, dtype=np.int64)
    for b0, b1 in zip(bounds[:-1], bounds[1:]):
        for c0 in range(int(b0), int(b1), nb):
            wend[c0:min(c0 + nb, b1)] = min(c0 + nb, b1)
    return wend


def lu_dense(rowptr, colind, values, perm, wend=None):
    """Dense right-looking Crout LU of C = A(perm, perm) (n up to a few
    thousand), pivots only from rows j .. wend[j]-1 (default: no pivoting)."""
    lib = _load()
    n = len(rowptr) - 1
    A = np.zeros((n, n))
    np.add.at(A, (np.repeat(np.arange(n), np.diff(rowptr)), colind), values)
    C = A if perm is None else A[np.ix_(perm, perm)]
    M = np.asfortranarray(C)
    if wend is None:
        wend = np.arange(1, n + 1, dtype=np.int64)
    wend = np.ascontiguousarray(wend, dtype=np.int64)
    rho = np.empty(n, dtype=np.int64)
    nzr = np.empty(n, dtype=np.int64)
    nzc = np.empty(n, dtype=np.int64)
    bad = lib.orc_lu_dense(n, _p(M), _p(wend), _p(rho), _p(nzr), _p(nzc))
    L = np.tril(M)
    U = np.triu(M, 1) + np.eye(n)
    return LU(L, U, rho, int(bad))


def solve_lu(F, b, perm):
    """x = P^T U^{-1} L^{-1} Pi P b (triangular solves by scipy)."""
    from scipy.linalg import solve_triangular
    b = np.asarray(b, dtype=np.float64)
    one = b.ndim == 1
    B = b.reshape(F.n, -1)
    y = B[perm] if perm is not None else B.copy()
    z = solve_triangular(F.L, y[F.rho], lower=True)
    w = solve_triangular(F.U, z, lower=False, unit_diagonal=True)
    x = np.empty_like(w)
    if perm is not None:
        x[perm] = w
    else:
        x[:] = w
    return x[:, 0] if one else x


class LDLT:
    """Pi C Pi^T = L D L^T of C = A(perm, perm): ``L`` dense unit lower
    triangular, ``D`` the pivots, ``rho[i]`` the row (and column) of C in
    position i, ``bad_col`` -1 or the first zero pivot."""

    def __init__(self, L, D, rho, bad_col):
        self.L, self.D, self.rho, self.bad_col = L, D, rho, bad_col
        self.n = len(rho)


def ldlt_dense(rowptr, colind, values, perm, wend=None):
    """Dense LDL^T of the symmetric C = A(perm, perm) with symmetric
    pivoting: column j takes the largest-magnitude diagonal entry among
    positions j .. wend[j]-1 of the current Schur complement (default: no
    pivoting)."""
    lib = _load()
    n = len(rowptr) - 1
    A = np.zeros((n, n))
    np.add.at(A, (np.repeat(np.arange(n), np.diff(rowptr)), colind), values)
    C = A if perm is None else A[np.ix_(perm, perm)]
    M = np.asfortranarray(C)
    if wend is None:
        wend = np.arange(1, n + 1, dtype=np.int64)
    wend = np.ascontiguousarray(wend, dtype=np.int64)
    rho = np.empty(n, dtype=np.int64)
    D = np.zeros(n)
    nzr = np.empty(n, dtype=np.int64)
    bad = lib.orc_ldlt_dense(n, _p(M), _p(wend), _p(rho), _p(D), _p(nzr))
    L = np.tril(M, -1) + np.eye(n)
    return LDLT(L, D, rho, int(bad))


def solve_ldlt_piv(F, b, perm):
    """x = P^T Pi^T L^{-T} D^{-1} L^{-1} Pi P b (triangular solves by scipy)."""
    from scipy.linalg import solve_triangular
    b = np.asarray(b, dtype=np.float64)
    one = b.ndim == 1
    B = b.reshape(F.n, -1)
    y = B[perm] if perm is not None else B.copy()
    z = solve_triangular(F.L, y[F.rho], lower=True, unit_diagonal=True)
    z = z / F.D[:, None]
    w = solve_triangular(F.L.T, z, lower=False, unit_diagonal=True)
    u = np.empty_like(w)
    u[F.rho] = w
    x = np.empty_like(u)
    if perm is not None:
        x[perm] = u
    else:
        x[:] = u
    return x[:, 0] if one else x


# ---------------------------------------------------------------------------
# Error measures
# ---------------------------------------------------------------------------
def berr(rowptr, colind, values, x, b):
    """max over RHS columns of ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf)."""
    n = len(rowptr) - 1
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    anorm = np.max(np.bincount(rows, weights=np.abs(values), minlength=n))
    X = np.asarray(x).reshape(n, -1)
    Bm = np.asarray(b).reshape(n, -1)
    worst = 0.0
    for r in range(X.shape[1]):
        ax = np.bincount(rows, weights=values * X[colind, r], minlength=n)
        res = np.max(np.abs(Bm[:, r] - ax))
        den = anorm * np.max(np.abs(X[:, r])) + np.max(np.abs(Bm[:, r]))
        worst = max(worst, res / den)
    return worst


def rel_fro(Lx_test, Lx_ref):
    """||L - L_ref||_F / ||L_ref||_F over a common pattern."""
    d = np.asarray(Lx_test, dtype=np.float64) - np.asarray(Lx_ref, dtype=np.float64)
    return float(np.linalg.norm(d) / np.linalg.norm(Lx_ref))


# ---------------------------------------------------------------------------
# FastILU / FastSpTRSV (paper Sec. 6; the algorithms of Chow and Patel)
# ---------------------------------------------------------------------------
class IluPattern:
    """ILU(k) pattern S with the level of fill of every entry; the CSC of S
    (cp, cr, cq) and the diagonal positions, for the sweeps."""

    def __init__(self, n, Sp, Sj, Slev, K):
        self.n, self.Sp, self.Sj, self.Slev, self.K = n, Sp, Sj, Slev, K
        rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(Sp))
        self.diag = np.empty(n, dtype=np.int64)
        on = np.nonzero(rows == Sj)[0]
        self.diag[rows[on]] = on
        order = np.lexsort((rows, Sj))  # by column, then row
        self.cr = rows[order].astype(np.int32)
        self.cq = order.astype(np.int64)
        self.cp = np.zeros(n + 1, dtype=np.int64)
        self.cp[1:] = np.cumsum(np.bincount(Sj, minlength=n))
        self.rows = rows

    def values_of(self, rowptr, colind, values, shift=0.0):
        """A on S (zeros at the fill; the diagonal times 1 + shift)."""
        n = self.n
        a = np.zeros(len(self.Sj))
        key = self.rows * n + self.Sj
        rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr))
        k2 = rows * n + np.asarray(colind, dtype=np.int64)
        at = np.searchsorted(key, k2)
        np.add.at(a, at, np.asarray(values, dtype=np.float64))
        a[self.diag] *= 1.0 + shift
        return a


def iluk_pattern(rowptr, colind, K):
    """ILU(K) pattern by levels of fill (C), with its levels."""
    lib = _load()
    n = len(rowptr) - 1
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    ci = np.ascontiguousarray(colind, dtype=np.int32)
    cap = max(16, 4 * len(ci) + n)
    work = [np.empty(max(n, 1), dtype=np.int32) for _ in range(3)]
    while True:
        Sp = np.empty(n + 1, dtype=np.int64)
        Sj = np.empty(cap, dtype=np.int32)
        Sl = np.empty(cap, dtype=np.int32)
        nnz = lib.orc_iluk_pattern(n, _p(rp), _p(ci), int(K), cap, _p(Sp), _p(Sj), _p(Sl),
                                   *[_p(w) for w in work])
        if nnz >= 0:
            return IluPattern(n, Sp, Sj[:nnz].copy(), Sl[:nnz].copy(), int(K))
        cap *= 2


def ilu_exact(pat, a, K=None):
    """Incomplete LU on the entries of level <= K (default: the pattern's)."""
    lib = _load()
    vals = np.array(a, dtype=np.float64)
    pos = np.empty(pat.n, dtype=np.int64)
    lib.orc_ilu_exact(pat.n, _p(pat.Sp), _p(pat.Sj), _p(pat.Slev),
                      pat.K if K is None else int(K), _p(pat.diag), _p(vals), _p(pos))
    return vals


def fastilu_initial(pat, a, K=None):
    """Initial guess of the sweeps: l_ij = a_ij / a_jj, u_ij = a_ij (zero at
    the fill)."""
    v = np.array(a, dtype=np.float64)
    low = pat.rows > pat.Sj
    v[low] = v[low] / a[pat.diag[pat.Sj[low]]]
    return v


def fastilu(pat, a, sweeps, omega=1.0, warmup=False, start=None, K=None):
    """FastILU(K) on the pattern (K defaults to the pattern's level):
    `sweeps` out-of-place sweeps from the initial guess (or `start`); with
    warmup, FastILU(K-1) first (recursively, same sweeps) gives the initial
    values of the entries of level < K, those of level K starting at zero.
    Returns the factors on S (entries of level > K hold the initial guess
    and are not part of the result)."""
    lib = _load()
    K = pat.K if K is None else int(K)
    if start is None:
        if warmup and K > 0:
            prev = fastilu(pat, a, sweeps, omega, warmup=True, K=K - 1)
            start = np.where(pat.Slev < K, prev, 0.0)
        else:
            start = fastilu_initial(pat, a)
    return _sweeps(lib, pat, a, start, sweeps, omega, K)


def _sweeps(lib, pat, a, start, sweeps, omega, K):
    cur = np.array(start, dtype=np.float64)
    nxt = np.empty_like(cur)
    w = np.zeros(pat.n)
    mark = np.zeros(pat.n, dtype=np.int8)
    a = np.ascontiguousarray(a, dtype=np.float64)
    for _ in range(sweeps):
        lib.orc_fastilu_sweep(pat.n, _p(pat.Sp), _p(pat.Sj), _p(pat.Slev), int(K), _p(pat.diag),
                              _p(pat.cp), _p(pat.cr), _p(pat.cq), _p(a), _p(cur), _p(nxt),
                              float(omega), _p(w), _p(mark))
        cur, nxt = nxt, cur
    return cur


def fast_trsv(pat, lu, b, upper, sweeps, omega=1.0, K=None):
    """FastSpTRSV: `sweeps` Jacobi sweeps on L (unit diagonal) or U from x = 0."""
    lib = _load()
    b = np.ascontiguousarray(b, dtype=np.float64)
    lu = np.ascontiguousarray(lu, dtype=np.float64)
    x = np.zeros(pat.n)
    y = np.empty(pat.n)
    for _ in range(sweeps):
        lib.orc_fast_trsv_sweep(pat.n, _p(pat.Sp), _p(pat.Sj), _p(pat.Slev),
                                pat.K if K is None else int(K), _p(pat.diag), _p(lu),
                                1 if upper else 0, _p(b), _p(x), _p(y), float(omega))
        x, y = y, x
    return x
