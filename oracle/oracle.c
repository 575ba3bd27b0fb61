/*
 * oracle.c -- plain, slow, obviously-correct CPU reference for the
 * supernodal multifrontal Cholesky path.  TEST INFRASTRUCTURE ONLY: it is
 * used by tests/, the smoke check and the CPU-baseline leg of the benchmark,
 * never by the library.  It shares no code with the GPU library.
 *
 * Everything works on C = P A P^T (new numbering), whose lower triangle is
 * given by the caller:
 *   - "rows" form: strict lower part by rows (row i lists columns j < i),
 *   - "cols" form: lower part incl. diagonal by columns (column j lists rows
 *     i >= j, values summed over duplicates).
 *
 * The method (paper Sec. 5, Tacho: multifrontal Cholesky of an SPD matrix,
 * three phases: symbolic analysis, numerical factorization, solve) reaches the
 * unique Cholesky factor of C, so the oracle computes that definition with
 * the textbook column-by-column (left-looking) algorithm:
 *   etree        parent(j) = min{ i > j : L_ij != 0 }       (Liu's algorithm)
 *   col counts   c_j = |struct(L_{*,j})| incl. diagonal     (row subtrees)
 *   supernodes   fundamental: j+1 joins j iff parent(j) = j+1,
 *                c_j = c_{j+1} + 1 and j is the only child of j+1
 *   numeric      x = C[j:,j] - sum_{k: L_jk != 0} L[j:,k] L_jk;
 *                L_jj = sqrt(x_j), L[j+1:,j] = x[j+1:] / L_jj
 *   solve        L z = P b, L^T w = z, x = P^T w
 *
 * All routines can be restricted to a set S of columns closed under etree
 * descendants (mask in_s); column j of L only depends on columns in the
 * subtree of j, so L[:, S] is exact.  S = {0..J-1} is always closed because
 * parent(j) > j.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Elimination tree by Liu's algorithm with path compression over the rows of
 * the strict lower triangle.  anc: workspace of n ints. */
void orc_etree(int64_t n, const int64_t* rp, const int32_t* ci, int32_t* parent,
               int32_t* anc) {
  for (int64_t i = 0; i < n; ++i) {
    parent[i] = -1;
    anc[i] = -1;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      int32_t r = ci[p];
      /* climb the compressed ancestor forest from r towards i */
      while (r != -1 && r < i) {
        int32_t next = anc[r];
        anc[r] = (int32_t)i;
        if (next == -1) parent[r] = (int32_t)i;
        r = next;
      }
    }
  }
}

/* Row-subtree walk: row i of L touches exactly the etree nodes on the paths
 * from each k (C_ik != 0, k < i) up to i.  Counts per column (incl. the
 * diagonal) and per row (off-diagonal), restricted to columns in S. */
void orc_counts(int64_t n, const int64_t* rp, const int32_t* ci,
                const int32_t* parent, const uint8_t* in_s, int64_t* colcnt,
                int64_t* rowcnt, int32_t* mark) {
  for (int64_t i = 0; i < n; ++i) {
    colcnt[i] = 0;
    rowcnt[i] = 0;
    mark[i] = -1;
  }
  for (int64_t i = 0; i < n; ++i) {
    mark[i] = (int32_t)i;
    if (in_s[i]) colcnt[i] += 1;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      int32_t k = ci[p];
      while (k != -1 && in_s[k] && mark[k] != i) {
        mark[k] = (int32_t)i;
        colcnt[k] += 1;
        rowcnt[i] += 1;
        k = parent[k];
      }
    }
  }
}

/* Fill the pattern of L[:, S] (Li, rows sorted ascending, diagonal first) and
 * the row lists (for row i: columns k < i with L_ik != 0 and the position of
 * L_ik inside column k).  Lp/Rp are prefix sums of colcnt/rowcnt. */
void orc_pattern(int64_t n, const int64_t* rp, const int32_t* ci,
                 const int32_t* parent, const uint8_t* in_s, const int64_t* Lp,
                 int32_t* Li, const int64_t* Rp, int32_t* Rk, int64_t* Rq,
                 int32_t* mark, int64_t* fill) {
  for (int64_t i = 0; i < n; ++i) {
    mark[i] = -1;
    fill[i] = Lp[i];
  }
  for (int64_t i = 0; i < n; ++i) {
    int64_t rpos = Rp[i];
    mark[i] = (int32_t)i;
    if (in_s[i]) Li[fill[i]++] = (int32_t)i;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      int32_t k = ci[p];
      while (k != -1 && in_s[k] && mark[k] != i) {
        mark[k] = (int32_t)i;
        Rk[rpos] = k;
        Rq[rpos] = fill[k];
        ++rpos;
        Li[fill[k]++] = (int32_t)i;
        k = parent[k];
      }
    }
  }
}

/* Column j of the left-looking factorization: x = C[j:, j] minus the
 * contributions L[j:, k] L_jk of every column k < j with L_jk != 0 (in the
 * order of j's row list), then L_jj = sqrt(x_j) and L[j+1:, j] = x / L_jj.
 * x: dense workspace of n doubles, zero on entry and exit.  Reads only
 * columns of j's etree subtree.  Returns 0, or 1 if the pivot is not
 * positive (column j is then left unwritten). */
static int factor_column(int64_t j, const int64_t* Cp, const int32_t* Cr,
                         const double* Cx, const int64_t* Lp, const int32_t* Li,
                         double* Lx, const int64_t* Rp, const int32_t* Rk,
                         const int64_t* Rq, double* x) {
  for (int64_t p = Cp[j]; p < Cp[j + 1]; ++p) x[Cr[p]] += Cx[p];
  for (int64_t r = Rp[j]; r < Rp[j + 1]; ++r) {
    int32_t k = Rk[r];
    int64_t q = Rq[r]; /* position of L_jk in column k */
    double ljk = Lx[q];
    for (int64_t t = q; t < Lp[k + 1]; ++t) x[Li[t]] -= Lx[t] * ljk;
  }
  double d = x[j];
  if (!(d > 0.0)) {
    for (int64_t t = Lp[j]; t < Lp[j + 1]; ++t) x[Li[t]] = 0.0;
    return 1;
  }
  double ljj = sqrt(d);
  Lx[Lp[j]] = ljj;
  x[j] = 0.0;
  for (int64_t t = Lp[j] + 1; t < Lp[j + 1]; ++t) {
    int32_t i = Li[t];
    Lx[t] = x[i] / ljj;
    x[i] = 0.0;
  }
  return 0;
}

/* Left-looking numeric factorization of the columns in S, in increasing
 * order.  Cp/Cr/Cx: lower triangle of C by columns.  x: dense workspace of n
 * doubles, zero on entry and exit.  Returns -1 on success or the first column
 * whose pivot is not positive (NOT SPD).  flops_done receives sum c_j^2 over
 * the columns completed. */
int64_t orc_factor(int64_t n, const int64_t* Cp, const int32_t* Cr,
                   const double* Cx, const uint8_t* in_s, const int64_t* Lp,
                   const int32_t* Li, double* Lx, const int64_t* Rp,
                   const int32_t* Rk, const int64_t* Rq, double* x,
                   double* flops_done) {
  double fl = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    if (!in_s[j]) continue;
    if (factor_column(j, Cp, Cr, Cx, Lp, Li, Lx, Rp, Rk, Rq, x)) {
      *flops_done = fl;
      return j;
    }
    double c = (double)(Lp[j + 1] - Lp[j]);
    fl += c * c;
  }
  *flops_done = fl;
  return -1;
}

/* The same factorization on several host threads (OpenMP), exact and
 * deterministic: column j reads only columns of its own etree subtree, so
 * columns of equal height in the etree (height = 1 + the largest height of a
 * child, leaves 0) never read one another and are computed in parallel, one
 * height after the other.  Each column is computed by factor_column exactly
 * as in orc_factor, so L is bitwise the same.  A column whose subtree holds a
 * failed pivot is skipped; the smallest failing column is returned, which is
 * the column orc_factor reports.  parent: the etree; threads <= 0 means the
 * OpenMP default; xs: threads * n doubles of zeroed workspace (threads as
 * orc_par_threads returns); height, order: n ints of workspace; hptr: n + 2
 * int64 of workspace.  flops_done: sum c_j^2 over the completed columns. */
int orc_par_threads(int threads) {
#ifdef _OPENMP
  return threads > 0 ? threads : omp_get_max_threads();
#else
  (void)threads;
  return 1;
#endif
}

int64_t orc_factor_par(int64_t n, const int64_t* Cp, const int32_t* Cr,
                       const double* Cx, const uint8_t* in_s, const int64_t* Lp,
                       const int32_t* Li, double* Lx, const int64_t* Rp,
                       const int32_t* Rk, const int64_t* Rq, const int32_t* parent,
                       int threads, double* xs, int32_t* height, int32_t* order,
                       int64_t* hptr, uint8_t* bad, double* flops_done) {
  int nt = orc_par_threads(threads);
  int32_t hmax = 0;
  for (int64_t j = 0; j < n; ++j) height[j] = 0;
  for (int64_t j = 0; j < n; ++j) {
    bad[j] = 0;
    if (height[j] > hmax) hmax = height[j];
    if (parent[j] >= 0 && height[parent[j]] < height[j] + 1) height[parent[j]] = height[j] + 1;
  }
  for (int64_t h = 0; h <= (int64_t)hmax + 1; ++h) hptr[h] = 0;
  for (int64_t j = 0; j < n; ++j) hptr[height[j] + 1] += 1;
  for (int64_t h = 0; h <= hmax; ++h) hptr[h + 1] += hptr[h];
  for (int64_t j = 0; j < n; ++j) order[hptr[height[j]]++] = (int32_t)j;
  for (int64_t h = hmax; h > 0; --h) hptr[h] = hptr[h - 1];
  hptr[0] = 0;
  double fl = 0.0;
  int64_t first_bad = -1;
  for (int64_t h = 0; h <= hmax; ++h) {
    const int64_t lo = hptr[h], hi = hptr[h + 1];
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt) reduction(+ : fl)
#endif
    for (int64_t q = lo; q < hi; ++q) {
      const int64_t j = order[q];
      if (!in_s[j]) continue;
      int tid = 0;
#ifdef _OPENMP
      tid = omp_get_thread_num();
#endif
      if (bad[j]) continue; /* a descendant failed */
      if (factor_column(j, Cp, Cr, Cx, Lp, Li, Lx, Rp, Rk, Rq, xs + (int64_t)tid * n)) {
        bad[j] = 2;
      } else {
        double c = (double)(Lp[j + 1] - Lp[j]);
        fl += c * c;
      }
    }
    /* serial: propagate failures to the parents (next heights) */
    for (int64_t q = lo; q < hi; ++q) {
      const int64_t j = order[q];
      if (bad[j] == 2 && (first_bad < 0 || j < first_bad)) first_bad = j;
      if (bad[j] && parent[j] >= 0) bad[parent[j]] = bad[parent[j]] ? bad[parent[j]] : 1;
    }
  }
  (void)nt;
  *flops_done = fl;
  return first_bad;
}

/* Fundamental supernodes.  sup_ptr receives the first column of every
 * supernode followed by n; returns the number of supernodes.  nchild: n ints
 * of workspace. */
int64_t orc_supernodes(int64_t n, const int32_t* parent, const int64_t* colcnt,
                       int32_t* sup_ptr, int32_t* nchild) {
  for (int64_t j = 0; j < n; ++j) nchild[j] = 0;
  for (int64_t j = 0; j < n; ++j)
    if (parent[j] >= 0) nchild[parent[j]] += 1;
  int64_t ns = 0;
  if (n == 0) {
    sup_ptr[0] = 0;
    return 0;
  }
  sup_ptr[ns++] = 0;
  for (int64_t j = 0; j + 1 < n; ++j) {
    int joins = parent[j] == j + 1 && colcnt[j] == colcnt[j + 1] + 1 &&
                nchild[j + 1] == 1;
    if (!joins) sup_ptr[ns++] = (int32_t)(j + 1);
  }
  sup_ptr[ns] = (int32_t)n;
  return ns;
}

/* Solve L L^T w = y in place (y overwritten by w), nrhs columns with leading
 * dimension ld.  Full factor only. */
void orc_solve(int64_t n, const int64_t* Lp, const int32_t* Li,
               const double* Lx, double* y, int64_t nrhs, int64_t ld) {
  for (int64_t r = 0; r < nrhs; ++r) {
    double* b = y + r * ld;
    for (int64_t j = 0; j < n; ++j) { /* forward: L z = b */
      double zj = b[j] / Lx[Lp[j]];
      b[j] = zj;
      for (int64_t t = Lp[j] + 1; t < Lp[j + 1]; ++t) b[Li[t]] -= Lx[t] * zj;
    }
    for (int64_t j = n - 1; j >= 0; --j) { /* backward: L^T w = z */
      double s = b[j];
      for (int64_t t = Lp[j] + 1; t < Lp[j + 1]; ++t) s -= Lx[t] * b[Li[t]];
      b[j] = s / Lx[Lp[j]];
    }
  }
}

/* ------------------------------------------------------------------------
 * FastILU and FastSpTRSV (paper Sec. 6, the algorithms of Chow and Patel).
 *
 * Pattern S of ILU(k) by levels of fill: entries of A (and the diagonal) have
 * level 0; eliminating with row k gives entry (i, j) the level
 * lev(i, k) + lev(k, j) + 1, the smallest over all k < min(i, j); S keeps the
 * entries of level <= K.  The rows are built in order, row i from the finished
 * upper parts of the rows k < i it meets, taking those k in increasing order
 * (a min-heap of column indices).  Output: Sp (n + 1), Sj (columns sorted),
 * Slev (levels).  Returns nnz(S), or -1 if cap entries are not enough.
 * Work: lev, heap, list (n ints each).
 * ------------------------------------------------------------------------ */
static void heap_push(int32_t* h, int64_t* hn, int32_t v) {
  int64_t c = (*hn)++;
  h[c] = v;
  while (c > 0) {
    int64_t p = (c - 1) / 2;
    if (h[p] <= h[c]) break;
    int32_t t = h[p];
    h[p] = h[c];
    h[c] = t;
    c = p;
  }
}

static int32_t heap_pop(int32_t* h, int64_t* hn) {
  int32_t top = h[0];
  h[0] = h[--(*hn)];
  int64_t c = 0;
  for (;;) {
    int64_t l = 2 * c + 1, r = l + 1, m = c;
    if (l < *hn && h[l] < h[m]) m = l;
    if (r < *hn && h[r] < h[m]) m = r;
    if (m == c) break;
    int32_t t = h[m];
    h[m] = h[c];
    h[c] = t;
    c = m;
  }
  return top;
}

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

int64_t orc_iluk_pattern(int64_t n, const int64_t* rp, const int32_t* ci, int32_t K,
                         int64_t cap, int64_t* Sp, int32_t* Sj, int32_t* Slev,
                         int32_t* lev, int32_t* heap, int32_t* list) {
  const int32_t INF = 0x7fffffff;
  for (int64_t i = 0; i < n; ++i) lev[i] = INF;
  int64_t nnz = 0;
  Sp[0] = 0;
  for (int64_t i = 0; i < n; ++i) {
    int64_t cnt = 0, hn = 0;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      int32_t c = ci[p];
      if (lev[c] == INF) {
        lev[c] = 0;
        list[cnt++] = c;
        if (c < i) heap_push(heap, &hn, c);
      }
    }
    if (lev[i] == INF) {
      lev[i] = 0;
      list[cnt++] = (int32_t)i;
    }
    while (hn > 0) {
      int32_t k = heap_pop(heap, &hn);
      int32_t lk = lev[k];
      for (int64_t q = Sp[k]; q < Sp[k + 1]; ++q) {
        int32_t j = Sj[q];
        if (j <= k) continue;
        int32_t nl = lk + Slev[q] + 1;
        if (nl > K) continue;
        if (lev[j] == INF) {
          lev[j] = nl;
          list[cnt++] = j;
          if (j < i) heap_push(heap, &hn, j);
        } else if (nl < lev[j]) {
          lev[j] = nl;
        }
      }
    }
    qsort(list, (size_t)cnt, sizeof(int32_t), cmp_i32);
    if (nnz + cnt > cap) return -1;
    for (int64_t q = 0; q < cnt; ++q) {
      Sj[nnz + q] = list[q];
      Slev[nnz + q] = lev[list[q]];
      lev[list[q]] = INF;
    }
    nnz += cnt;
    Sp[i + 1] = nnz;
  }
  return nnz;
}

/* Incomplete LU on the entries of S with level <= K (the fixed point that the
 * FastILU sweeps approach): row by row, for each k < i of row i in increasing
 * order, l_ik = a_ik / u_kk and a_ij -= l_ik u_kj for the entries (i, j) of
 * S.  vals: A on S (zeros at fill) in, L (strictly lower, unit diagonal
 * implied) and U (upper with the diagonal) on S out.  diag: position of
 * (i, i) in row i.  pos: n int64 of work. */
void orc_ilu_exact(int64_t n, const int64_t* Sp, const int32_t* Sj, const int32_t* Slev,
                   int32_t K, const int64_t* diag, double* vals, int64_t* pos) {
  for (int64_t i = 0; i < n; ++i) pos[i] = -1;
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t q = Sp[i]; q < Sp[i + 1]; ++q)
      if (Slev[q] <= K) pos[Sj[q]] = q;
    for (int64_t q = Sp[i]; q < diag[i]; ++q) {
      if (Slev[q] > K) continue;
      int32_t k = Sj[q];
      double lik = vals[q] / vals[diag[k]];
      vals[q] = lik;
      for (int64_t r = diag[k] + 1; r < Sp[k + 1]; ++r) {
        if (Slev[r] > K) continue;
        int64_t at = pos[Sj[r]];
        if (at >= 0) vals[at] -= lik * vals[r];
      }
    }
    for (int64_t q = Sp[i]; q < Sp[i + 1]; ++q) pos[Sj[q]] = -1;
  }
}

/* One FastILU sweep, out of place (every entry from the previous sweep's
 * factors, so the result does not depend on the order of the updates): for
 * each (i, j) in S of level <= K,
 *   s = a_ij - sum_{k < min(i, j)} l_ik u_kj,
 *   l_ij = (1 - omega) l_ij + omega s / u_jj   (i > j),
 *   u_ij = (1 - omega) u_ij + omega s          (i <= j),
 * with l and u read from `old`.  The sum runs over k in increasing order,
 * through row i of L (scattered into w) and column j of S (cp, cr, cq: the
 * CSC of S, rows increasing, cq the CSR position).  w: n doubles, zero on
 * entry and exit; mark: n chars, zero on entry and exit. */
void orc_fastilu_sweep(int64_t n, const int64_t* Sp, const int32_t* Sj, const int32_t* Slev,
                       int32_t K, const int64_t* diag, const int64_t* cp, const int32_t* cr,
                       const int64_t* cq, const double* a, const double* old, double* out,
                       double omega, double* w, char* mark) {
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t q = Sp[i]; q < diag[i]; ++q)
      if (Slev[q] <= K) {
        w[Sj[q]] = old[q];
        mark[Sj[q]] = 1;
      }
    for (int64_t q = Sp[i]; q < Sp[i + 1]; ++q) {
      if (Slev[q] > K) {
        out[q] = old[q];
        continue;
      }
      int32_t j = Sj[q];
      int64_t m = i < j ? i : j;
      double s = a[q];
      for (int64_t t = cp[j]; t < cp[j + 1] && cr[t] < m; ++t)
        if (Slev[cq[t]] <= K && mark[cr[t]]) s -= w[cr[t]] * old[cq[t]];
      if (i > j) out[q] = (1.0 - omega) * old[q] + omega * s / old[diag[j]];
      else out[q] = (1.0 - omega) * old[q] + omega * s;
    }
    for (int64_t q = Sp[i]; q < diag[i]; ++q) {
      w[Sj[q]] = 0.0;
      mark[Sj[q]] = 0;
    }
  }
}

/* One FastSpTRSV sweep (Jacobi, out of place) with the factors on S of level
 * <= K: lower (unit diagonal) x_i = (1 - omega) x_i + omega (b_i -
 * sum_{j < i} l_ij x_j), or upper x_i = (1 - omega) x_i + omega (b_i -
 * sum_{j > i} u_ij x_j) / u_ii, every x_j from the previous sweep (xo). */
void orc_fast_trsv_sweep(int64_t n, const int64_t* Sp, const int32_t* Sj, const int32_t* Slev,
                         int32_t K, const int64_t* diag, const double* lu, int upper,
                         const double* b, const double* xo, double* x, double omega) {
  for (int64_t i = 0; i < n; ++i) {
    double s = b[i];
    int64_t q0 = upper ? diag[i] + 1 : Sp[i];
    int64_t q1 = upper ? Sp[i + 1] : diag[i];
    for (int64_t q = q0; q < q1; ++q)
      if (Slev[q] <= K) s -= lu[q] * xo[Sj[q]];
    if (upper) s /= lu[diag[i]];
    x[i] = (1.0 - omega) * xo[i] + omega * s;
  }
}

/* ------------------------------------------------------------------------
 * LDL^T of a symmetric (possibly indefinite) C = P A P^T without pivoting
 * (paper Sec. 5: the symmetric factorizations Tacho offers besides
 * Cholesky): C = L D L^T, L unit lower triangular, D diagonal.  It exists
 * when every leading principal minor is nonzero, e.g. for any symmetric
 * permutation of a quasi-definite matrix.  Left-looking, column j:
 *   x = C[j:, j] - sum_{k < j, L_jk != 0} L[j:, k] d_k L_jk,
 *   d_j = x_j,  L[j+1:, j] = x[j+1:] / d_j,  L_jj = 1.
 * Same pattern and row lists as orc_factor (struct(L) does not depend on
 * the values).  Lx receives L (diagonal entries 1), D the pivots.  Returns
 * -1, or the first column whose pivot is zero. */
int64_t orc_factor_ldlt(int64_t n, const int64_t* Cp, const int32_t* Cr, const double* Cx,
                        const uint8_t* in_s, const int64_t* Lp, const int32_t* Li, double* Lx,
                        double* D, const int64_t* Rp, const int32_t* Rk, const int64_t* Rq,
                        double* x) {
  for (int64_t j = 0; j < n; ++j) {
    if (!in_s[j]) continue;
    for (int64_t p = Cp[j]; p < Cp[j + 1]; ++p) x[Cr[p]] += Cx[p];
    for (int64_t r = Rp[j]; r < Rp[j + 1]; ++r) {
      int32_t k = Rk[r];
      int64_t q = Rq[r]; /* position of L_jk in column k */
      double w = Lx[q] * D[k];
      for (int64_t u = q; u < Lp[k + 1]; ++u) x[Li[u]] -= Lx[u] * w;
    }
    double d = x[j];
    if (d == 0.0) {
      for (int64_t t = Lp[j]; t < Lp[j + 1]; ++t) x[Li[t]] = 0.0;
      return j;
    }
    D[j] = d;
    Lx[Lp[j]] = 1.0;
    x[j] = 0.0;
    for (int64_t t = Lp[j] + 1; t < Lp[j + 1]; ++t) {
      int32_t i = Li[t];
      Lx[t] = x[i] / d;
      x[i] = 0.0;
    }
  }
  return -1;
}

/* Solve L D L^T w = y in place (nrhs columns, leading dimension ld). */
void orc_solve_ldlt(int64_t n, const int64_t* Lp, const int32_t* Li, const double* Lx,
                    const double* D, double* y, int64_t nrhs, int64_t ld) {
  for (int64_t r = 0; r < nrhs; ++r) {
    double* b = y + r * ld;
    for (int64_t j = 0; j < n; ++j) /* forward: L z = b (unit diagonal) */
      for (int64_t t = Lp[j] + 1; t < Lp[j + 1]; ++t) b[Li[t]] -= Lx[t] * b[j];
    for (int64_t j = 0; j < n; ++j) b[j] /= D[j];
    for (int64_t j = n - 1; j >= 0; --j) { /* backward: L^T w = z */
      double acc = b[j];
      for (int64_t t = Lp[j] + 1; t < Lp[j + 1]; ++t) acc -= Lx[t] * b[Li[t]];
      b[j] = acc;
    }
  }
}

/*
 * LU of a general matrix with a symmetric sparsity pattern (paper Sec. 5:
 * besides Cholesky and LDL^T, Tacho factors general matrices whose
 * structure is symmetric), pivots looked for only within diagonal blocks
 * (paper Sec. 5, the comparison with SuperLU: Tacho searches each diagonal
 * block for its pivots instead of pivoting across whole columns).
 *
 * Dense right-looking Gaussian elimination in Crout form on the n x n
 * column-major M = C = P A P^T:  Pi C = L U, L lower triangular, U unit
 * upper triangular, Pi a row permutation.  Column j takes its pivot from
 * the rows j .. wend[j]-1 of its diagonal block (wend[j] = j + 1: no
 * pivoting): the row of largest magnitude, ties going to the row that
 * started in the smallest position of C.  That row is swapped with row j
 * across all n columns; then U(j, c) = M(j, c) / M(j, j) for c > j and
 * M(i, c) -= M(i, j) U(j, c) for i, c > j.  On return M holds L on and
 * below the diagonal and U above it, and rho[i] is the row of C now in
 * position i.  Returns -1, or the first column whose pivot is zero.  Zero
 * entries of column j and of row j are skipped in the update (the result is
 * the same; sparse C just goes faster).  nzr, nzc: workspace of n each.
 */
int64_t orc_lu_dense(int64_t n, double* M, const int64_t* wend, int64_t* rho, int64_t* nzr,
                     int64_t* nzc) {
  for (int64_t i = 0; i < n; ++i) rho[i] = i;
  for (int64_t j = 0; j < n; ++j) {
    double* colj = M + j * n;
    int64_t p = j;
    for (int64_t i = j + 1; i < wend[j]; ++i) {
      double a = fabs(colj[i]), b = fabs(colj[p]);
      if (a > b || (a == b && rho[i] < rho[p])) p = i;
    }
    if (p != j) {
      for (int64_t c = 0; c < n; ++c) {
        double tmp = M[c * n + j];
        M[c * n + j] = M[c * n + p];
        M[c * n + p] = tmp;
      }
      int64_t tr = rho[j];
      rho[j] = rho[p];
      rho[p] = tr;
    }
    double piv = colj[j];
    if (piv == 0.0) return j;
    int64_t nr = 0, nc = 0;
    for (int64_t i = j + 1; i < n; ++i)
      if (colj[i] != 0.0) nzr[nr++] = i;
    for (int64_t c = j + 1; c < n; ++c) {
      double* ujc = M + c * n + j;
      if (*ujc != 0.0) {
        *ujc /= piv;
        nzc[nc++] = c;
      }
    }
    for (int64_t t = 0; t < nc; ++t) {
      double* colc = M + nzc[t] * n;
      double u = colc[j];
      for (int64_t q = 0; q < nr; ++q) colc[nzr[q]] -= colj[nzr[q]] * u;
    }
  }
  return -1;
}

/*
 * LDL^T of a symmetric C = P A P^T with symmetric pivoting within diagonal
 * blocks (paper Sec. 5: Tacho's LDL^T of symmetric indefinite matrices,
 * with pivots looked for only inside each diagonal block): Pi C Pi^T =
 * L D L^T, L unit lower triangular, D diagonal (1x1 pivots).  Dense, on the
 * full symmetric n x n column-major M = C.  Column j takes as pivot the
 * diagonal entry of largest magnitude among positions j .. wend[j]-1 of the
 * current Schur complement (wend[j] = j + 1: no pivoting), ties going to the
 * row that started in the smallest position; rows j and p and columns j and
 * p are swapped; then d_j = M(j, j) and, for i, c > j,
 * M(i, c) -= M(i, j) M(c, j) / d_j, which keeps M symmetric; finally
 * L(i, j) = M(i, j) / d_j.  On return the strict lower part of M holds L,
 * D the pivots and rho[i] the row of C now in position i.  Returns -1, or
 * the first column whose pivot is zero.  nzr: workspace of n.
 */
int64_t orc_ldlt_dense(int64_t n, double* M, const int64_t* wend, int64_t* rho, double* D,
                       int64_t* nzr) {
  for (int64_t i = 0; i < n; ++i) rho[i] = i;
  for (int64_t j = 0; j < n; ++j) {
    int64_t p = j;
    for (int64_t i = j + 1; i < wend[j]; ++i) {
      double a = fabs(M[i * n + i]), b = fabs(M[p * n + p]);
      if (a > b || (a == b && rho[i] < rho[p])) p = i;
    }
    if (p != j) {
      for (int64_t c = 0; c < n; ++c) { /* rows j and p */
        double tmp = M[c * n + j];
        M[c * n + j] = M[c * n + p];
        M[c * n + p] = tmp;
      }
      for (int64_t r = 0; r < n; ++r) { /* columns j and p */
        double tmp = M[j * n + r];
        M[j * n + r] = M[p * n + r];
        M[p * n + r] = tmp;
      }
      int64_t tr = rho[j];
      rho[j] = rho[p];
      rho[p] = tr;
    }
    double* colj = M + j * n;
    double dj = colj[j];
    if (dj == 0.0) return j;
    D[j] = dj;
    int64_t nr = 0;
    for (int64_t i = j + 1; i < n; ++i)
      if (colj[i] != 0.0) nzr[nr++] = i;
    for (int64_t t = 0; t < nr; ++t) {
      double* colc = M + nzr[t] * n;
      double w = colj[nzr[t]] / dj;
      for (int64_t q = 0; q < nr; ++q) colc[nzr[q]] -= colj[nzr[q]] * w;
    }
    for (int64_t q = 0; q < nr; ++q) colj[nzr[q]] /= dj;
  }
  return -1;
}
