// factor_kernels.cu -- numeric multifrontal Cholesky kernels for sm_103a.
//
// Paper Sec. 5 (Tacho): multifrontal Cholesky of an SPD matrix with
// level-set scheduling; many small dense blocks at the bottom of the tree,
// fewer larger ones near the root.  Per front s (k pivot columns, m update
// rows, nf = k + m):
//   assemble   F = A(rows_s, cols_s) + sum_children extend(U_c)
//   POTRF      L11 = chol(F11)
//   TRSM       L21 = F21 L11^{-T}
//   SYRK       U_s = F22 - L21 L21^T   (lower triangle)
// Front storage: the L panel (nf x k, column-major, ld = nf) and the update
// matrix U_s (m x m, column-major) are separate arrays; element (r, c) of
// the front lives in the panel for c < k and in U_s for c >= k.
//
// Extend-add is parent-pull: the parent's kernel reads its children's U_c
// through the child-to-parent relative maps in a fixed order, so the result
// is deterministic and needs no atomics.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "kernels.h"

namespace mf {
namespace {

// Default bound of a queue wait: about kQueueSpin x 128 ns (0.5 s).
constexpr int kQueueSpin = 1 << 22;
// threads of a queue CTA: queued fronts are small (k + m <= 64 by default),
// so more, smaller CTAs per SM overlap the latency of the per-column steps
constexpr int kQueueThreads = 128;

template <typename T>
struct FD {
  const SnInfo* sn;
  const int32_t* children;
  const int32_t* relmap;
  const int64_t* acol_ptr;
  const int32_t* arow;
  const int64_t* asrc_ptr;
  const int64_t* asrc;
  const Item* items;
  const double* vals;
  const T* av;
  const Item* arange;
  T* L;
  T* U;
  unsigned long long* status;
  const int64_t* soff;
  float* split;    // staging area 0: rows of 256 floats (two panel slots)
  float* split_b;  // staging area 1: rows of 512 floats (four slots, lookahead levels)
  T* dinv;
  const int64_t* ioff;  // per front: first kept diagonal-inverse slot (or -1)
  T* P;                 // partitioned inverse (SpTRSV variants 3, 4) or nullptr
  T* PT;                // variant 4: P transposed per front (k x nf, ld k) or nullptr
  int* qstate;          // small-front queue: ticket counter, then one flag per front
  int wait_polls;       // polls before a queue wait gives up
  T* D;                 // LDL^T: the pivots by permuted column; nullptr for Cholesky
  // LU (lu != 0): Lu holds U^T in the layout of L and Uu the transposed
  // update matrices; Lb is the trailing update's second operand and dinv_t
  // the inverse the panel solve multiplies by (Cholesky: L and dinv)
  const T* Lb;
  const T* dinv_t;
  int lu;
  T* Lu;
  T* Uu;
  T* dinvu;
  const int64_t* uacol_ptr;
  const int32_t* uarow;
  const T* avu;
  uint8_t* piv;  // pivoting: row taken by each pivot position of a 64-row block
  int32_t* ipos;  // LDL^T with symmetric pivoting: position each row ended in
};

template <typename T>
FD<T> make_fd(const FactorArgs& a) {
  FD<T> d;
  d.sn = a.sym.sn;
  d.children = a.sym.children;
  d.relmap = a.sym.relmap;
  d.acol_ptr = a.sym.acol_ptr;
  d.arow = a.sym.arow;
  d.asrc_ptr = a.sym.asrc_ptr;
  d.asrc = a.sym.asrc;
  d.items = a.sym.items;
  d.vals = a.vals;
  d.av = static_cast<const T*>(a.av);
  d.arange = a.sym.arange;
  d.L = static_cast<T*>(a.L);
  d.U = static_cast<T*>(a.U);
  d.status = a.status;
  d.soff = a.sym.soff;
  d.split = a.split;
  d.split_b = a.split_b;
  d.dinv = static_cast<T*>(a.dinv);
  d.ioff = a.sym.ioff;
  d.P = static_cast<T*>(a.P);
  d.PT = static_cast<T*>(a.PT);
  d.qstate = a.qstate;
  d.wait_polls = a.wait_polls > 0 ? a.wait_polls : kQueueSpin;
  d.D = static_cast<T*>(a.D);
  d.lu = a.lu;
  d.Lu = static_cast<T*>(a.Lu);
  d.Uu = static_cast<T*>(a.Uu);
  d.dinvu = static_cast<T*>(a.dinvu);
  d.uacol_ptr = a.uacol_ptr;
  d.uarow = a.uarow;
  d.avu = static_cast<const T*>(a.avu);
  d.piv = a.piv;
  d.ipos = a.ipos;
  // LU, lower half: L21 = F21 U11^{-1} (the inverse of the U^T block), the
  // update's second operand is U^T
  d.Lb = a.lu ? d.Lu : d.L;
  d.dinv_t = a.lu ? d.dinvu : d.dinv;
  return d;
}

// LU with a symmetric pattern (paper Sec. 5): the upper half of a front is
// kept transposed, U^T in the layout of L, so the same assembly, panel solve
// and trailing-update kernels serve it with the two halves exchanged:
// U12^T = (Pi F12)^T L11^{-T} and (F22 - L21 U12)^T = F22^T - U12^T L21^T.
// These kernels run twice as many CTAs for an LU factor; the second half
// takes the upper view.
template <typename T>
__device__ __forceinline__ FD<T> upper_view(const FD<T>& d) {
  FD<T> e = d;
  e.L = d.Lu;
  e.Lb = d.L;
  e.U = d.Uu;
  e.acol_ptr = d.uacol_ptr;
  e.arow = d.uarow;
  e.av = d.avu;
  e.dinv_t = d.dinv;
  return e;
}

// Block index within the launch's items, and whether this CTA works on the
// upper half of an LU factor.
template <typename T>
__device__ __forceinline__ int lu_block(const FD<T>& d, bool& upper) {
  const int half = (int)(gridDim.x >> 1);
  upper = d.lu != 0 && (int)blockIdx.x >= half;
  return upper ? (int)blockIdx.x - half : (int)blockIdx.x;
}

// Column c of front f: element (r, c) is col[r] (r >= k when c >= k).
template <typename T>
__device__ __forceinline__ T* front_col(const FD<T>& d, const SnInfo& f, int c) {
  const int64_t nf = (int64_t)f.k + f.m;
  if (c < f.k) return d.L + f.Loff + (int64_t)c * nf;
  return d.U + (f.Uoff + (int64_t)(c - f.k) * f.m - f.k);
}

__device__ __forceinline__ double dsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float dsqrt(float x) { return sqrtf(x); }

// IEEE round-to-nearest reciprocal (the CUDA intrinsics)
__device__ __forceinline__ double recip_rn(double x) { return __drcp_rn(x); }
__device__ __forceinline__ float recip_rn(float x) { return __frcp_rn(x); }

// Partial Cholesky of the first `k` columns of an n x n lower-triangular
// block held column-major in shared memory (ld), n <= kSmallMax.  Records
// the first non-positive pivot (global column col0 + j).  With D (LDL^T,
// paper Sec. 5) the partial factorization is F = L D L^T instead: d_j =
// F_jj (recorded in D[col0 + j]; a zero pivot is the failure), L(:, j) =
// F(:, j) / d_j with L_jj = 1.
//   1. the k pivot columns, right-looking inside them, one barrier per
//      column: F(i, c) -= F(i, j) F(c, j) / d_j for j < c < k, i >= c, the
//      columns left unscaled (one reciprocal per step, no square root);
//   2. column j scaled by 1 / sqrt(d_j) (L_jj = sqrt(d_j)) or 1 / d_j;
//   3. the trailing m x m block (m = n - k) in one pass, F22 -= L21 L21^T
//      (LDL^T: L21 D L21^T), each thread accumulating 4 x 4 tiles over the k
//      columns in registers (about half a shared load per FMA).
template <typename T>
__device__ void smem_partial_chol(T* F, int ld, int n, int k, int col0,
                                  unsigned long long* status, T* D) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int j = 0; j < k; ++j) {
    const T dj = F[j * ld + j];
    if (tid == 0 && !(D ? dj != T(0) : dj > T(0)))
      atomicMin(status, (unsigned long long)(col0 + j));
    const T rd = recip_rn(dj);
    for (int c = j + 1 + warp; c < k; c += nw) {
      const T fc = F[j * ld + c] * rd;
      for (int i = c + lane; i < n; i += 32) F[c * ld + i] -= F[j * ld + i] * fc;
    }
    __syncthreads();
  }
  for (int j = warp; j < k; j += nw) {
    const T dj = F[j * ld + j];
    const T sj = D ? recip_rn(dj) : recip_rn(dsqrt(dj));
    for (int i = j + 1 + lane; i < n; i += 32) F[j * ld + i] *= sj;
    if (lane == 0) {
      F[j * ld + j] = D ? T(1) : dj * sj;
      if (D) D[col0 + j] = dj;
    }
  }
  __syncthreads();
  const int m = n - k;
  if (m <= 0 || k == 0) return;
  const int nt = (m + 3) >> 2;
  for (int e = tid; e < nt * nt; e += blockDim.x) {
    const int I = e / nt, J = e - I * nt;
    if (I < J) continue;
    const int r0 = k + 4 * I, q0 = k + 4 * J;
    T acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
    for (int j = 0; j < k; ++j) {
      const T* colj = F + j * ld;
      const T w = D ? D[col0 + j] : T(1);
      T a[4], bq[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = r0 + u < n ? colj[r0 + u] : T(0);
        bq[u] = q0 + u < n ? colj[q0 + u] * w : T(0);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], bq[v], acc[u][v]);
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int c = q0 + v;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = r0 + u;
        if (r < n && c < n && r >= c) F[c * ld + r] -= acc[u][v];
      }
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Small fronts: one CTA assembles and factors the whole front in shared
// memory and writes the L panel and the update matrix.  The children's
// update matrices are read through L2 (ld.global.cg): in the persistent
// queue a child may have been written by another CTA of the same launch,
// into memory that the plan reuses, so a line left in this SM's L1 from an
// earlier use must not be seen.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void small_front_body(const FD<T>& d, int s, T* F) {
  const SnInfo f = d.sn[s];
  const int k = f.k, m = f.m, nf = k + m;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int i = tid; i < nf * nf; i += blockDim.x) F[i] = T(0);
  __syncthreads();
  for (int c = warp; c < k; c += nw) {
    const int g = f.first + c;
    for (int64_t e = d.acol_ptr[g] + lane; e < d.acol_ptr[g + 1]; e += 32)
      F[c * nf + d.arow[e]] = d.av[e];
  }
  __syncthreads();
  for (int ci = 0; ci < f.nchild; ++ci) {
    const SnInfo ch = d.sn[d.children[f.child_begin + ci]];
    const int mc = ch.m;
    const int32_t* map = d.relmap + ch.map_off;
    const T* Uc = d.U + ch.Uoff;
    // a child of a small front has mc < kSmallMax rows: its column in at
    // most four lanes' steps, loads issued together
    for (int jc = warp; jc < mc; jc += nw) {
      const int dc = map[jc];
      const T* u = Uc + (int64_t)jc * mc;
      int pi[kSmallMax / 32];
      T uv[kSmallMax / 32];
#pragma unroll
      for (int q = 0; q < kSmallMax / 32; ++q) {
        const int ic = jc + lane + 32 * q;
        pi[q] = ic < mc ? map[ic] : 0;
        uv[q] = ic < mc ? __ldcg(u + ic) : T(0);
      }
#pragma unroll
      for (int q = 0; q < kSmallMax / 32; ++q)
        if (jc + lane + 32 * q < mc) F[dc * nf + pi[q]] += uv[q];
    }
    __syncthreads();
  }
  smem_partial_chol(F, nf, nf, k, f.first, d.status, d.D);
  T* Lp = d.L + f.Loff;
  for (int c = warp; c < k; c += nw)
    for (int r = lane; r < nf; r += 32) Lp[(int64_t)c * nf + r] = F[c * nf + r];
  T* Up = d.U + f.Uoff;
  for (int c = warp; c < m; c += nw)
    for (int r = lane; r < m; r += 32) Up[(int64_t)c * m + r] = F[(k + c) * nf + k + r];
}

// Pivot search of LU with pivoting within diagonal blocks (paper Sec. 5:
// Tacho looks for pivots only inside each diagonal block): warp 0 returns
// the row of largest |col[i]| over i in [j, we), ties going to the row
// that started in the smallest position (orig[i]).
template <typename T>
__device__ __forceinline__ int block_pivot(const T* col, const int* orig, int j, int we) {
  const int lane = threadIdx.x & 31;
  T bv = T(-1);
  int bo = 1 << 30, bi = j;
  for (int i = j + lane; i < we; i += 32) {
    const T a = fabs(col[i]);
    const int o = orig[i];
    if (a > bv || (a == bv && o < bo)) {
      bv = a;
      bo = o;
      bi = i;
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const T ov = __shfl_down_sync(0xffffffffu, bv, off);
    const int oo = __shfl_down_sync(0xffffffffu, bo, off);
    const int oi = __shfl_down_sync(0xffffffffu, bi, off);
    if (ov > bv || (ov == bv && oo < bo)) {
      bv = ov;
      bo = oo;
      bi = oi;
    }
  }
  return __shfl_sync(0xffffffffu, bi, 0);
}

// The same search over the diagonal entries F(i, i) of a column-major block
// (leading dimension ld): symmetric pivoting of LDL^T.
template <typename T>
__device__ __forceinline__ int block_pivot_diag(const T* F, int ld, const int* orig, int j, int we) {
  const int lane = threadIdx.x & 31;
  T bv = T(-1);
  int bo = 1 << 30, bi = j;
  for (int i = j + lane; i < we; i += 32) {
    const T a = fabs(F[i * ld + i]);
    const int o = orig[i];
    if (a > bv || (a == bv && o < bo)) {
      bv = a;
      bo = o;
      bi = i;
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const T ov = __shfl_down_sync(0xffffffffu, bv, off);
    const int oo = __shfl_down_sync(0xffffffffu, bo, off);
    const int oi = __shfl_down_sync(0xffffffffu, bi, off);
    if (ov > bv || (ov == bv && oo < bo)) {
      bv = ov;
      bo = oo;
      bi = oi;
    }
  }
  return __shfl_sync(0xffffffffu, bi, 0);
}

// Unblocked right-looking LDL^T with symmetric pivoting (paper Sec. 5: LDL^T
// of symmetric indefinite matrices, pivots looked for only inside each
// diagonal block) of the first k columns of an n x n symmetric block held in
// full, column-major, in shared memory (ld): column j takes the diagonal
// entry of largest magnitude among positions j .. end of its 64-row block
// (ties to the row that started first, orig), swaps rows and columns j and p,
// then F(i, c) -= F(i, j) F(c, j) / d_j for i, c > j (both triangles, so F
// stays symmetric) and L(i, j) = F(i, j) / d_j, L_jj = 1.  Records the
// pivots in D[col0 + j] and the first zero pivot.
template <typename T>
__device__ __forceinline__ void smem_ldlt_piv(T* F, int ld, int n, int k, int col0,
                                              unsigned long long* status, T* D, int* orig) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  __shared__ int s_p;
  for (int j = 0; j < k; ++j) {
    if (warp == 0) {
      const int p = block_pivot_diag(F, ld, orig, j, min(k, (j & ~(kNB - 1)) + kNB));
      if (lane == 0) s_p = p;
    }
    __syncthreads();
    const int p = s_p;
    if (p != j) {
      for (int c = tid; c < n; c += blockDim.x) {  // rows j and p
        const T t = F[c * ld + j];
        F[c * ld + j] = F[c * ld + p];
        F[c * ld + p] = t;
      }
      __syncthreads();
      for (int r = tid; r < n; r += blockDim.x) {  // columns j and p
        const T t = F[j * ld + r];
        F[j * ld + r] = F[p * ld + r];
        F[p * ld + r] = t;
      }
      if (tid == 0) {
        const int t = orig[j];
        orig[j] = orig[p];
        orig[p] = t;
      }
    }
    __syncthreads();
    const T dj = F[j * ld + j];
    if (tid == 0 && !(dj != T(0))) atomicMin(status, (unsigned long long)(col0 + j));
    const T rinv = T(1) / dj;
    for (int c = j + 1 + warp; c < n; c += nw) {
      const T w = F[j * ld + c] * rinv;
      for (int i = j + 1 + lane; i < n; i += 32) F[c * ld + i] -= F[j * ld + i] * w;
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < n; i += blockDim.x) F[j * ld + i] *= rinv;
    if (tid == 0) {
      F[j * ld + j] = T(1);
      D[col0 + j] = dj;
    }
    __syncthreads();
  }
}

// Unblocked right-looking LU in Crout form (L lower, U unit upper) of the
// first k columns of an n x n block held column-major in shared memory
// (ld): for j < k, U(j, c) = F(j, c) / F(j, j) for c > j, then
// F(i, c) -= F(i, j) U(j, c) for i, c > j.  With `orig` (pivoting) column
// j first takes the largest-magnitude row among the rows j .. end of its
// 64-row block (rows < k only) and swaps it with row j across all n
// columns; orig tracks where each row started.  Records the first zero
// pivot (global column col0 + j).
template <typename T>
__device__ __forceinline__ void smem_partial_lu(T* F, int ld, int n, int k, int col0,
                                unsigned long long* status, int* orig) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  __shared__ int s_p;
  for (int j = 0; j < k; ++j) {
    if (orig) {
      if (warp == 0) {
        const int p = block_pivot(F + j * ld, orig, j, min(k, (j & ~(kNB - 1)) + kNB));
        if (lane == 0) s_p = p;
      }
      __syncthreads();
      const int p = s_p;
      if (p != j) {
        for (int c = tid; c < n; c += blockDim.x) {
          const T t = F[c * ld + j];
          F[c * ld + j] = F[c * ld + p];
          F[c * ld + p] = t;
        }
        if (tid == 0) {
          const int t = orig[j];
          orig[j] = orig[p];
          orig[p] = t;
        }
      }
      __syncthreads();
    }
    const T piv = F[j * ld + j];
    if (tid == 0 && !(piv != T(0))) atomicMin(status, (unsigned long long)(col0 + j));
    const T rinv = T(1) / piv;
    for (int c = j + 1 + tid; c < n; c += blockDim.x) F[c * ld + j] *= rinv;
    __syncthreads();
    for (int c = j + 1 + warp; c < n; c += nw) {
      const T u = F[c * ld + j];
      for (int i = j + 1 + lane; i < n; i += 32) F[c * ld + i] -= F[j * ld + i] * u;
    }
    __syncthreads();
  }
}

// Small front of an LU factor: the whole front F (lower entries of C into
// their columns, upper entries into their rows, the children's lower and
// transposed-upper update matrices) in shared memory with leading dimension
// nf + 1, partial LU, then L, U^T (unit diagonal) and the two halves of the
// update matrix written out.
template <typename T>
__device__ __forceinline__ void small_front_lu(const FD<T>& d, int s, T* F) {
  __shared__ int orig[kSmallMax];
  const SnInfo f = d.sn[s];
  const int k = f.k, m = f.m, nf = k + m, ld = nf + 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int i = tid; i < nf * ld; i += blockDim.x) F[i] = T(0);
  for (int i = tid; i < k; i += blockDim.x) orig[i] = i;
  __syncthreads();
  for (int c = warp; c < k; c += nw) {
    const int g = f.first + c;
    for (int64_t e = d.acol_ptr[g] + lane; e < d.acol_ptr[g + 1]; e += 32)
      F[c * ld + d.arow[e]] = d.av[e];
    for (int64_t e = d.uacol_ptr[g] + lane; e < d.uacol_ptr[g + 1]; e += 32)
      F[d.uarow[e] * ld + c] = d.avu[e];
  }
  __syncthreads();
  for (int ci = 0; ci < f.nchild; ++ci) {
    const SnInfo ch = d.sn[d.children[f.child_begin + ci]];
    const int mc = ch.m;
    const int32_t* map = d.relmap + ch.map_off;
    const T* Ul = d.U + ch.Uoff;
    const T* Uh = d.Uu + ch.Uoff;
    for (int jc = warp; jc < mc; jc += nw) {
      const int dc = map[jc];
      const T* ul = Ul + (int64_t)jc * mc;
      const T* uh = Uh + (int64_t)jc * mc;
      for (int ic = jc + lane; ic < mc; ic += 32) {
        const int di = map[ic];
        F[dc * ld + di] += __ldcg(ul + ic);
        if (ic > jc) F[di * ld + dc] += __ldcg(uh + ic);
      }
    }
    __syncthreads();
  }
  smem_partial_lu(F, ld, nf, k, f.first, d.status, d.piv ? orig : nullptr);
  T* Lp = d.L + f.Loff;
  T* Up = d.Lu + f.Loff;
  for (int c = warp; c < k; c += nw)
    for (int r = lane; r < nf; r += 32) {
      Lp[(int64_t)c * nf + r] = r >= c ? F[c * ld + r] : T(0);
      Up[(int64_t)c * nf + r] = r > c ? F[r * ld + c] : (r == c ? T(1) : T(0));
    }
  if (d.piv)
    for (int i = tid; i < k; i += blockDim.x) d.piv[f.first + i] = (uint8_t)(orig[i] - (i & ~(kNB - 1)));
  T* Ul = d.U + f.Uoff;
  T* Uh = d.Uu + f.Uoff;
  for (int c = warp; c < m; c += nw)
    for (int r = lane; r < m; r += 32) {
      Ul[(int64_t)c * m + r] = F[(k + c) * ld + k + r];
      Uh[(int64_t)c * m + r] = F[(k + r) * ld + k + c];
    }
}

// Small front of an LDL^T factor with symmetric pivoting: the front as for
// Cholesky (lower entries, children's update matrices), mirrored into the
// upper triangle, leading dimension nf + 1; then the pivoted partial LDL^T,
// L, the pivots and the update matrix written out, and each row's final
// position recorded.
template <typename T>
__device__ __forceinline__ void small_front_ldlt_piv(const FD<T>& d, int s, T* F) {
  __shared__ int orig[kSmallMax];
  const SnInfo f = d.sn[s];
  const int k = f.k, m = f.m, nf = k + m, ld = nf + 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int i = tid; i < nf * ld; i += blockDim.x) F[i] = T(0);
  for (int i = tid; i < k; i += blockDim.x) orig[i] = i;
  __syncthreads();
  for (int c = warp; c < k; c += nw) {
    const int g = f.first + c;
    for (int64_t e = d.acol_ptr[g] + lane; e < d.acol_ptr[g + 1]; e += 32)
      F[c * ld + d.arow[e]] = d.av[e];
  }
  __syncthreads();
  for (int ci = 0; ci < f.nchild; ++ci) {
    const SnInfo ch = d.sn[d.children[f.child_begin + ci]];
    const int mc = ch.m;
    const int32_t* map = d.relmap + ch.map_off;
    const T* Uc = d.U + ch.Uoff;
    for (int jc = warp; jc < mc; jc += nw) {
      const int dc = map[jc];
      const T* u = Uc + (int64_t)jc * mc;
      for (int ic = jc + lane; ic < mc; ic += 32) F[dc * ld + map[ic]] += __ldcg(u + ic);
    }
    __syncthreads();
  }
  for (int idx = tid; idx < nf * nf; idx += blockDim.x) {
    const int c = idx / nf, r = idx % nf;
    if (r < c) F[c * ld + r] = F[r * ld + c];
  }
  __syncthreads();
  smem_ldlt_piv(F, ld, nf, k, f.first, d.status, d.D, orig);
  T* Lp = d.L + f.Loff;
  for (int c = warp; c < k; c += nw)
    for (int r = lane; r < nf; r += 32) Lp[(int64_t)c * nf + r] = r >= c ? F[c * ld + r] : T(0);
  for (int i = tid; i < k; i += blockDim.x) {
    d.piv[f.first + i] = (uint8_t)(orig[i] - (i & ~(kNB - 1)));
    d.ipos[f.first + orig[i]] = f.first + i;
  }
  T* Up = d.U + f.Uoff;
  for (int c = warp; c < m; c += nw)
    for (int r = lane; r < m; r += 32) Up[(int64_t)c * m + r] = F[(k + c) * ld + k + r];
}

// Small-front kinds: 0 Cholesky / LDL^T without pivoting, 1 LU, 2 LDL^T
// with symmetric pivoting (1 and 2 pad the shared leading dimension).
template <typename T, int MODE>
__device__ __forceinline__ void small_front(const FD<T>& d, int s, T* F) {
  if (MODE == 1) small_front_lu(d, s, F);
  else if (MODE == 2) small_front_ldlt_piv(d, s, F);
  else small_front_body(d, s, F);
}

template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_small_front(FD<T> d, int64_t item_off) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  small_front<T, MODE>(d, d.items[item_off + blockIdx.x].s, reinterpret_cast<T*>(smem_raw));
}

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// ---------------------------------------------------------------------------
// Persistent small-front queue (paper Sec. 5: level-set scheduling, with the
// many small blocks at the bottom of the tree taken in one launch).  The
// `count` queued fronts are in level order; every CTA repeatedly takes the
// next ticket, waits until each child of that front has raised its
// completion flag, factors the front as k_small_front does and raises its
// own flag.  A CTA only waits for fronts with smaller tickets, which CTAs
// already running have taken, so the queue always drains.  Each wait is
// bounded (wait_polls polls 128 ns apart): when it runs out the CTA records
// MF_ERR_TIMEOUT in status[1] and goes on, so the launch always ends.
// ---------------------------------------------------------------------------
template <typename T, int MODE>
__global__ void __launch_bounds__(kQueueThreads) k_small_queue(FD<T> d, int64_t item_off, int count) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_ticket;
  int* ticket = d.qstate;
  int* done = d.qstate + 1;
  for (;;) {
    if (threadIdx.x == 0) s_ticket = atomicAdd(ticket, 1);
    __syncthreads();
    const int t = s_ticket;
    if (t >= count) break;
    const int s = d.items[item_off + t].s;
    const SnInfo f = d.sn[s];
    if (threadIdx.x < 32) {
      for (int ci = threadIdx.x; ci < f.nchild; ci += 32) {
        const int* flag = done + d.children[f.child_begin + ci];
        int spins = 0;
        while (ld_acquire_gpu(flag) == 0) {
          if (++spins > d.wait_polls) {
            atomicExch(d.status + 1, (unsigned long long)MF_ERR_TIMEOUT);
            break;
          }
          __nanosleep(128);
        }
      }
    }
    __syncthreads();
    small_front<T, MODE>(d, s, reinterpret_cast<T*>(smem_raw));
    // every thread's stores are ordered before thread 0's release by the
    // CTA barrier; the GPU-scope release store is cumulative
    __syncthreads();
    if (threadIdx.x == 0)
      asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(done + s), "r"(1) : "memory");
  }
}

// ---------------------------------------------------------------------------
// Large fronts, assembly of a chunk of front columns [a, b).  Warp w owns the
// columns a + w, a + w + 8, ...: it zeroes each one, scatters the entries of
// A into it, then adds every child's update column that lands on it,
// children in their fixed order.  A parent column has a single owner, so the
// CTA needs no barrier and the sums are deterministic.  The child columns
// landing in [a, b) are the range [lo, hi) of the child's (increasing)
// relative map; the one landing on column c is found by bisection.
// ---------------------------------------------------------------------------
template <typename T, bool LU>
__global__ void __launch_bounds__(256) k_assemble(FD<T> d0, int64_t item_off) {
  bool upper = false;
  const int bid = LU ? lu_block(d0, upper) : (int)blockIdx.x;
  const FD<T> d = (LU && upper) ? upper_view(d0) : d0;
  const Item it = d.items[item_off + bid];
  const SnInfo f = d.sn[it.s];
  const int k = f.k, nf = k + f.m, c0 = it.a, c1 = it.b;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = c0 + warp; c < c1; c += nw) {
    T* __restrict__ col = front_col(d, f, c);
    for (int r = (c < k ? 0 : c) + lane; r < nf; r += 32) col[r] = T(0);
    __syncwarp();
    if (c < k) {
      const int g = f.first + c;
      for (int64_t e = d.acol_ptr[g] + lane; e < d.acol_ptr[g + 1]; e += 32)
        col[d.arow[e]] = d.av[e];
      __syncwarp();
    }
    for (const Item* rg = d.arange + it.t; rg->s >= 0; ++rg) {
      const SnInfo ch = d.sn[rg->s];
      const int32_t* __restrict__ map = d.relmap + ch.map_off;
      // at most kAsmCols child columns land in the chunk: one lane each
      // reads its map entry and a ballot finds the one landing on c
      const int lo = rg->t, hi = rg->a;
      const unsigned hit = __ballot_sync(0xffffffffu, lo + lane < hi && map[lo + lane] == c);
      if (!hit) continue;
      const int jc = lo + __ffs(hit) - 1, mc = ch.m;
      const T* __restrict__ u = d.U + ch.Uoff + (int64_t)jc * mc;
      int ic = jc + lane;
      for (; ic + 32 < mc; ic += 64) {
        const int p0 = map[ic], p1 = map[ic + 32];
        const T v0 = u[ic], v1 = u[ic + 32];
        const T a0 = col[p0], a1 = col[p1];
        col[p0] = a0 + v0;
        col[p1] = a1 + v1;
      }
      if (ic < mc) col[map[ic]] += u[ic];
      __syncwarp();
    }
  }
}

// Diagonal block of panel step c0 (b x b, padded with the identity to 64 x 64)
// into shared memory D (column-major, leading dimension ld).  Every thread
// issues all its global loads before the first shared store, so the DRAM
// latency is paid once, not once per element.
template <typename T, int NT>
__device__ __forceinline__ void load_diag_block(const FD<T>& d, const SnInfo& f, int c0, int b,
                                                T* D, int ld) {
  constexpr int PER = kNB * kNB / NT;
  const int64_t nf = (int64_t)f.k + f.m;
  const T* base = d.L + f.Loff + (int64_t)c0 * nf + c0;
  T v[PER];
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int idx = threadIdx.x + u * NT, c = idx / kNB, i = idx % kNB;
    v[u] = (i < b && c < b) ? (i >= c ? base[(int64_t)c * nf + i] : T(0)) : (i == c ? T(1) : T(0));
  }
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int idx = threadIdx.x + u * NT;
    D[(idx / kNB) * ld + (idx % kNB)] = v[u];
  }
}

// ---------------------------------------------------------------------------
// Large fronts, panel step t: Cholesky factor and inverse of the b x b
// diagonal block (b <= 64, padded with the identity to 64 x 64), one CTA of
// 256 threads per front.  The kernel sits on the critical path of every
// panel step, so it is blocked for few barriers, keeps every warp's work
// uniform (an FP64 warp instruction costs the same with 1 or 32 lanes
// active) and is written as compact loops.
//
// Factor, by 16-column blocks B (rows/columns j0 .. j0 + 15):
//   (a) one warp: L_BB = chol(A_BB) and its inverse Y_BB (column
//       substitution, lane c solves L_BB y = e_c);
//   (b) rows below: L_iB = A_iB Y_BB^T;
//   (c) trailing lower part: A_ic -= L_iB L_cB^T (triangle enumerated evenly
//       over the threads).
// Inverse: the off-diagonal blocks by distance d = i - j = 1, 2, 3:
//   Y_ij = -Y_ii (sum_{k=j}^{i-1} L_ik Y_kj).
// ---------------------------------------------------------------------------
constexpr int kPB = 16;  // block size inside the diagonal-block kernel


template <typename T>
constexpr size_t potrf_smem() {
  return ((size_t)2 * kNB * (kNB + 1) + (size_t)3 * kPB * (kPB + 1)) * sizeof(T);
}

template <typename T>
__global__ void __launch_bounds__(256) k_potrf(FD<T> d, int64_t item_off) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int ld = kNB + 1, tld = kPB + 1;
  T* D = reinterpret_cast<T*>(smem_raw);  // D[c * ld + r] = A(r, c), then L(r, c)
  T* Y = D + kNB * ld;                    // Y[c * ld + r] = L^{-1}(r, c)
  T* Tm = Y + kNB * ld;                   // Tm[(m * kPB + c) * tld + r]: block products
  // LDL^T (d.D set): the block's pivots; L_BB has a unit diagonal, so its
  // inverse is computed the same way
  __shared__ T piv_of[kNB];
  const bool ldlt = d.D != nullptr;
  const Item it = d.items[item_off + blockIdx.x];
  const SnInfo f = d.sn[it.s];
  const int c0 = it.t * kNB;
  const int b = min(kNB, f.k - c0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  load_diag_block<T, 256>(d, f, c0, b, D, ld);
  // only the 16-column blocks holding real pivots are factored and
  // inverted; beyond them the padded block is the identity, and so is its
  // inverse
  const int nbk = (b + kPB - 1) / kPB, bend = nbk * kPB;
  for (int idx = tid; idx < kNB * ld; idx += blockDim.x) {
    const int c = idx / ld, r = idx % ld;
    Y[idx] = (c >= bend && r == c) ? T(1) : T(0);
  }
  __syncthreads();
  for (int j0 = 0; j0 < bend; j0 += kPB) {
    // (a) diagonal block: lane r < 16 owns row j0 + r (lanes 16..31 repeat
    // rows 0..15 and write nothing).  The rows stay in registers and the
    // elimination takes no square root: A(r, c) -= A(r, t) A(c, t) / d_t,
    // one reciprocal per step, the values of column t by shuffles, so a
    // step's dependent chain is shuffle -> reciprocal -> FMA; the scaling
    // to L (by 1 / sqrt(d_t), or 1 / d_t for LDL^T) comes after all 16 steps.
    if (warp == 0) {
      const int r = lane & (kPB - 1);
      T a[kPB];
#pragma unroll
      for (int c = 0; c < kPB; ++c) a[c] = c <= r ? D[(j0 + c) * ld + j0 + r] : T(0);
      T myd = T(1);  // this lane's pivot d_r
#pragma unroll
      for (int t = 0; t < kPB; ++t) {
        const T dt = __shfl_sync(0xffffffffu, a[t], t);
        if (t == r) myd = dt;
        const T art = a[t] * recip_rn(dt);
        // (fixed trip count: the loop unrolls and a[] stays in registers)
#pragma unroll
        for (int c = 0; c < kPB; ++c) {
          if (c > t) {
            const T act = __shfl_sync(0xffffffffu, a[t], c);
            if (c <= r && r > t) a[c] = fma(-art, act, a[c]);
          }
        }
      }
      if (lane < kPB && j0 + r < b && !(ldlt ? myd != T(0) : myd > T(0)))
        atomicMin(d.status, (unsigned long long)(f.first + c0 + j0 + r));
      const T mys = ldlt ? recip_rn(myd) : recip_rn(dsqrt(myd));
      if (lane < kPB) {
#pragma unroll
        for (int c = 0; c < kPB; ++c) {
          const T sc = __shfl_sync(0x0000ffffu, mys, c);
          if (c < r) D[(j0 + c) * ld + j0 + r] = a[c] * sc;
        }
        D[(j0 + r) * ld + j0 + r] = ldlt ? T(1) : myd * mys;
        piv_of[j0 + r] = myd;
      }
      __syncwarp();
      // inverse of L_BB: lane c < 16 solves L_BB y = e_c, right-looking with
      // y in registers; the reciprocals of the diagonal are computed once
      const T rdl = T(1) / D[(j0 + (lane & (kPB - 1))) * ld + j0 + (lane & (kPB - 1))];
      const int c = lane & (kPB - 1);
      T acc[kPB], y[kPB];
#pragma unroll
      for (int q = 0; q < kPB; ++q) acc[q] = T(0);
#pragma unroll
      for (int q = 0; q < kPB; ++q) {
        const T rq = __shfl_sync(0xffffffffu, rdl, q);
        y[q] = q < c ? T(0) : ((q == c ? T(1) : T(0)) + acc[q]) * rq;
#pragma unroll
        for (int q2 = q + 1; q2 < kPB; ++q2) acc[q2] = fma(-D[(j0 + q) * ld + j0 + q2], y[q], acc[q2]);
      }
      if (lane < kPB) {
#pragma unroll
        for (int q = 0; q < kPB; ++q) Y[(j0 + c) * ld + j0 + q] = y[q];
      }
    }
    __syncthreads();
    const int base = j0 + kPB, n2 = bend - base;
    if (n2 == 0) break;
    // (b) L_iB = A_iB Y_BB^T for rows i >= base: element e -> (i, t)
    {
      T v[3];
      for (int q = 0; q < 3; ++q) {
        const int e = tid + q * 256;
        v[q] = T(0);
        if (e < n2 * kPB) {
          const int i = base + e / kPB, t = e % kPB;
          T av[kPB], yv[kPB];
#pragma unroll
          for (int k = 0; k < kPB; ++k) {
            av[k] = D[(j0 + k) * ld + i];
            yv[k] = Y[(j0 + k) * ld + j0 + t];  // zero for k > t
          }
          T s = T(0);
#pragma unroll
          for (int k = 0; k < kPB; ++k) s = fma(av[k], yv[k], s);
          v[q] = ldlt ? s / piv_of[j0 + t] : s;  // LDL^T: L_iB = A_iB L_BB^-T D_B^-1
        }
      }
      __syncthreads();
      for (int q = 0; q < 3; ++q) {
        const int e = tid + q * 256;
        if (e < n2 * kPB) D[(j0 + e % kPB) * ld + base + e / kPB] = v[q];
      }
      __syncthreads();
    }
    // (c) trailing lower part: element e of the n2 x n2 triangle -> (i, c)
    const int E = n2 * (n2 + 1) / 2;
    for (int e = tid; e < E; e += blockDim.x) {
      int i = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
      while (i * (i + 1) / 2 > e) --i;
      while ((i + 1) * (i + 2) / 2 <= e) ++i;
      const int c = e - i * (i + 1) / 2;
      T li[kPB], lc[kPB];
#pragma unroll
      for (int t = 0; t < kPB; ++t) {
        li[t] = D[(j0 + t) * ld + base + i];
        lc[t] = D[(j0 + t) * ld + base + c];
        if (ldlt) lc[t] *= piv_of[j0 + t];  // A_ic -= L_iB D_B L_cB^T
      }
      T s = D[(base + c) * ld + base + i];
#pragma unroll
      for (int t = 0; t < kPB; ++t) s = fma(-li[t], lc[t], s);
      D[(base + c) * ld + base + i] = s;
    }
    __syncthreads();
  }
  // off-diagonal blocks of the inverse, by block distance
  const int r = tid & (kPB - 1), c = tid >> 4;  // element (r, c) of a 16 x 16 block
  for (int dd = 1; dd < nbk; ++dd) {
    const int nb = nbk - dd;
    for (int m = 0; m < nb; ++m) {
      const int bi = m + dd, bj = m;
      T s = T(0);
      for (int kb = bj; kb < bi; ++kb) {
        T lv[kPB], yv[kPB];
#pragma unroll
        for (int t = 0; t < kPB; ++t) {
          lv[t] = D[(kb * kPB + t) * ld + bi * kPB + r];
          yv[t] = Y[(bj * kPB + c) * ld + kb * kPB + t];
        }
#pragma unroll
        for (int t = 0; t < kPB; ++t) s = fma(lv[t], yv[t], s);
      }
      Tm[(m * kPB + c) * tld + r] = s;
    }
    __syncthreads();
    for (int m = 0; m < nb; ++m) {
      const int bi = m + dd, bj = m;
      T yv[kPB], tv[kPB];
#pragma unroll
      for (int t = 0; t < kPB; ++t) {
        yv[t] = Y[(bi * kPB + t) * ld + bi * kPB + r];  // zero for t > r
        tv[t] = Tm[(m * kPB + c) * tld + t];
      }
      T s = T(0);
#pragma unroll
      for (int t = 0; t < kPB; ++t) s = fma(yv[t], tv[t], s);
      Y[(bj * kPB + c) * ld + bi * kPB + r] = -s;
    }
    __syncthreads();
  }
  for (int idx = tid; idx < b * b; idx += blockDim.x) {
    const int cc = idx / b, rr = idx % b;
    if (rr >= cc) front_col(d, f, c0 + cc)[c0 + rr] = D[cc * ld + rr];
  }
  if (ldlt)
    for (int i = tid; i < b; i += blockDim.x) d.D[f.first + c0 + i] = piv_of[i];
  T* Dv = d.dinv + (int64_t)it.b * kNB * kNB;
  for (int idx = tid; idx < kNB * kNB; idx += blockDim.x) {
    const int cc = idx / kNB, rr = idx % kNB;
    Dv[cc * kNB + rr] = Y[cc * ld + rr];
  }
}

// ---------------------------------------------------------------------------
// LU (paper Sec. 5), large fronts, panel step t: the b x b diagonal block
// F = [lower part from L, upper part from U^T] (padded with the identity to
// 64 x 64), one CTA per front: Crout LU Pi F = L U (U unit upper), with
// pivoting Pi chosen within the block (largest magnitude in the column among
// the block's remaining rows); L and U^T go back to the two halves of the
// front, their inverses to the slots of dinv and dinvu, and Pi to piv.
// Nothing outside the block moves here: the upper half's panel solve reads
// F12 in pivot order, and the rows' earlier columns of the front are
// reordered once the factorization is done (k_lu_swap).
// ---------------------------------------------------------------------------
template <typename T>
constexpr size_t getrf_smem() {
  return (size_t)3 * kNB * (kNB + 1) * sizeof(T);
}

template <typename T>
__global__ void __launch_bounds__(256) k_getrf(FD<T> d, int64_t item_off) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int ld = kNB + 1;
  T* A = reinterpret_cast<T*>(smem_raw);  // A[c * ld + r] = F(r, c), then L / U
  T* Yl = A + kNB * ld;                   // L^{-1}, column-major
  T* Yu = Yl + kNB * ld;                  // (U^T)^{-1}; first the U^T block as loaded
  __shared__ int orig[kNB];
  __shared__ int s_p;
  const Item it = d.items[item_off + blockIdx.x];
  const SnInfo f = d.sn[it.s];
  const int64_t nf = (int64_t)f.k + f.m;
  const int c0 = it.t * kNB;
  const int b = min(kNB, f.k - c0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  T* FL = d.L + f.Loff + (int64_t)c0 * nf + c0;  // element (r, c) at [c * nf + r]
  T* FU = d.Lu + f.Loff + (int64_t)c0 * nf + c0;
  for (int idx = tid; idx < kNB * kNB; idx += blockDim.x) {
    const int c = idx / kNB, r = idx % kNB;
    const bool in = r < b && c < b;
    A[c * ld + r] = in ? (r >= c ? FL[(int64_t)c * nf + r] : T(0)) : (r == c ? T(1) : T(0));
    Yu[c * ld + r] = (in && r > c) ? FU[(int64_t)c * nf + r] : T(0);
  }
  if (tid < kNB) orig[tid] = tid;
  __syncthreads();
  for (int idx = tid; idx < kNB * kNB; idx += blockDim.x) {
    const int c = idx / kNB, r = idx % kNB;
    if (r < c) A[c * ld + r] = Yu[r * ld + c];  // F(r, c) = U^T(c, r)
  }
  __syncthreads();
  for (int j = 0; j < b; ++j) {
    if (d.piv) {
      if (warp == 0) {
        const int p = block_pivot(A + j * ld, orig, j, b);
        if (lane == 0) s_p = p;
      }
      __syncthreads();
      const int p = s_p;
      if (p != j) {
        if (tid < kNB) {
          const T t = A[tid * ld + j];
          A[tid * ld + j] = A[tid * ld + p];
          A[tid * ld + p] = t;
        }
        if (tid == 0) {
          const int t = orig[j];
          orig[j] = orig[p];
          orig[p] = t;
        }
      }
      __syncthreads();
    }
    const T piv = A[j * ld + j];
    if (tid == 0 && !(piv != T(0))) atomicMin(d.status, (unsigned long long)(f.first + c0 + j));
    const T rinv = T(1) / piv;
    if (tid > j && tid < b) A[tid * ld + j] *= rinv;  // U(j, c), c = tid
    __syncthreads();
    const int nt = b - j - 1;
    for (int e = tid; e < nt * nt; e += blockDim.x) {
      const int c = j + 1 + e / nt, r = j + 1 + e % nt;
      A[c * ld + r] -= A[j * ld + r] * A[c * ld + j];
    }
    __syncthreads();
  }
  // inverses by column substitution: thread c < 64 solves L y = e_c,
  // thread 64 + c solves U^T y = e_c (unit diagonal, U^T(i, q) = A(q, i))
  if (tid < 2 * kNB) {
    const int c = tid & (kNB - 1);
    const bool up = tid >= kNB;
    T* Y = up ? Yu : Yl;
    for (int i = 0; i < kNB; ++i) {
      T y = T(0);
      if (i >= c) {
        T acc = i == c ? T(1) : T(0);
        for (int q = c; q < i; ++q) acc -= (up ? A[i * ld + q] : A[q * ld + i]) * Y[c * ld + q];
        y = up ? acc : acc / A[i * ld + i];
      }
      Y[c * ld + i] = y;
    }
  }
  __syncthreads();
  for (int idx = tid; idx < b * b; idx += blockDim.x) {
    const int cc = idx / b, rr = idx % b;
    if (rr >= cc) FL[(int64_t)cc * nf + rr] = A[cc * ld + rr];
    if (rr >= cc) FU[(int64_t)cc * nf + rr] = rr == cc ? T(1) : A[rr * ld + cc];
  }
  if (d.piv && tid < b) d.piv[f.first + c0 + tid] = (uint8_t)orig[tid];
  T* Dl = d.dinv + (int64_t)it.b * kNB * kNB;
  T* Du = d.dinvu + (int64_t)it.b * kNB * kNB;
  for (int idx = tid; idx < kNB * kNB; idx += blockDim.x) {
    const int cc = idx / kNB, rr = idx % kNB;
    Dl[idx] = Yl[cc * ld + rr];
    Du[idx] = Yu[cc * ld + rr];
  }
}

// ---------------------------------------------------------------------------
// LDL^T with symmetric pivoting (paper Sec. 5), large fronts, panel step t:
// the b x b diagonal block (lower part of L's half, mirrored, padded with
// the identity), one CTA per front: Pi F Pi^T = L D L^T with the pivots
// chosen inside the block (largest remaining diagonal, ties to the row that
// started first); L (unit diagonal), D, the inverse of L (dinv slot), the
// block's permutation (piv) and each row's final position (ipos) are
// written.  The panel solve reads F21 in the block's pivot order, and the
// rows' earlier columns are reordered after the factorization (k_lu_swap).
// ---------------------------------------------------------------------------
template <typename T>
constexpr size_t sytrf_smem() {
  return (size_t)2 * kNB * (kNB + 1) * sizeof(T);
}

template <typename T>
__global__ void __launch_bounds__(256) k_sytrf(FD<T> d, int64_t item_off) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int ld = kNB + 1;
  T* A = reinterpret_cast<T*>(smem_raw);  // A[c * ld + r] = F(r, c), both triangles
  T* Y = A + kNB * ld;                    // L^{-1}, column-major
  __shared__ int orig[kNB];
  __shared__ T piv_of[kNB];
  __shared__ int s_p;
  const Item it = d.items[item_off + blockIdx.x];
  const SnInfo f = d.sn[it.s];
  const int64_t nf = (int64_t)f.k + f.m;
  const int c0 = it.t * kNB;
  const int b = min(kNB, f.k - c0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  T* FL = d.L + f.Loff + (int64_t)c0 * nf + c0;
  for (int idx = tid; idx < kNB * kNB; idx += blockDim.x) {
    const int c = idx / kNB, r = idx % kNB;
    A[c * ld + r] = (r < b && c < b) ? (r >= c ? FL[(int64_t)c * nf + r] : T(0))
                                     : (r == c ? T(1) : T(0));
  }
  if (tid < kNB) orig[tid] = tid;
  __syncthreads();
  for (int idx = tid; idx < b * b; idx += blockDim.x) {
    const int c = idx / b, r = idx % b;
    if (r < c) A[c * ld + r] = A[r * ld + c];
  }
  __syncthreads();
  for (int j = 0; j < b; ++j) {
    if (warp == 0) {
      const int p = block_pivot_diag(A, ld, orig, j, b);
      if (lane == 0) s_p = p;
    }
    __syncthreads();
    const int p = s_p;
    if (p != j) {
      if (tid < kNB) {  // rows j and p
        const T t = A[tid * ld + j];
        A[tid * ld + j] = A[tid * ld + p];
        A[tid * ld + p] = t;
      }
      __syncthreads();
      if (tid < kNB) {  // columns j and p
        const T t = A[j * ld + tid];
        A[j * ld + tid] = A[p * ld + tid];
        A[p * ld + tid] = t;
      }
      if (tid == 0) {
        const int t = orig[j];
        orig[j] = orig[p];
        orig[p] = t;
      }
      __syncthreads();
    }
    const T dj = A[j * ld + j];
    if (tid == 0 && !(dj != T(0))) atomicMin(d.status, (unsigned long long)(f.first + c0 + j));
    const T rinv = T(1) / dj;
    const int nt = b - j - 1;
    for (int e = tid; e < nt * nt; e += blockDim.x) {
      const int c = j + 1 + e / nt, r = j + 1 + e % nt;
      A[c * ld + r] -= A[j * ld + r] * (A[j * ld + c] * rinv);
    }
    __syncthreads();
    if (tid > j && tid < b) A[j * ld + tid] *= rinv;
    if (tid == 0) {
      piv_of[j] = dj;
      A[j * ld + j] = T(1);
    }
    __syncthreads();
  }
  // inverse of the unit lower L: thread c < 64 solves L y = e_c
  if (tid < kNB) {
    const int c = tid;
    for (int i = 0; i < kNB; ++i) {
      T y = T(0);
      if (i >= c) {
        T acc = i == c ? T(1) : T(0);
        for (int q = c; q < i; ++q) acc -= A[q * ld + i] * Y[c * ld + q];
        y = acc;
      }
      Y[c * ld + i] = y;
    }
  }
  __syncthreads();
  for (int idx = tid; idx < b * b; idx += blockDim.x) {
    const int cc = idx / b, rr = idx % b;
    if (rr >= cc) FL[(int64_t)cc * nf + rr] = A[cc * ld + rr];
  }
  if (tid < b) {
    d.D[f.first + c0 + tid] = piv_of[tid];
    d.piv[f.first + c0 + tid] = (uint8_t)orig[tid];
    d.ipos[f.first + c0 + orig[tid]] = f.first + c0 + tid;
  }
  T* Dv = d.dinv + (int64_t)it.b * kNB * kNB;
  for (int idx = tid; idx < kNB * kNB; idx += blockDim.x) {
    const int cc = idx / kNB, rr = idx % kNB;
    Dv[idx] = Y[cc * ld + rr];
  }
}

// LU with pivoting, after the factorization: in a large front, the rows of
// each later 64-row pivot block t take the order of their pivots in the
// front's earlier columns too (k_getrf reordered them only from the block
// on), so that every pivot row of a front is stored in pivot order.  One
// CTA per (front, t >= 1); warp w moves columns w, w + 8, ...; lanes hold
// rows lane and lane + 32 and take their new values by shuffles.
template <typename T>
__global__ void __launch_bounds__(256) k_lu_swap(FD<T> d, const Item* items) {
  const Item it = items[blockIdx.x];
  const SnInfo f = d.sn[it.s];
  const int64_t nf = (int64_t)f.k + f.m;
  const int c0 = it.t * kNB, b = min(kNB, f.k - c0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint8_t* pv = d.piv + f.first + c0;
  const int s0 = lane < b ? (int)pv[lane] : lane;
  const int s1 = lane + 32 < b ? (int)pv[lane + 32] : lane + 32;
  for (int c = warp; c < c0; c += 8) {
    T* col = d.L + f.Loff + (int64_t)c * nf + c0;
    const T v0 = lane < b ? col[lane] : T(0);
    const T v1 = lane + 32 < b ? col[lane + 32] : T(0);
    const T a0 = __shfl_sync(0xffffffffu, v0, s0 & 31), a1 = __shfl_sync(0xffffffffu, v1, s0 & 31);
    const T b0 = __shfl_sync(0xffffffffu, v0, s1 & 31), b1 = __shfl_sync(0xffffffffu, v1, s1 & 31);
    if (lane < b) col[lane] = s0 < 32 ? a0 : a1;
    if (lane + 32 < b) col[lane + 32] = s1 < 32 ? b0 : b1;
  }
}

// ---------------------------------------------------------------------------
// Large fronts, panel step t: rows [r0, r0 + kTrsmRows) of the panel below
// the diagonal block, X = A L_tt^{-T} as a product with the inverse from
// k_potrf.  Thread (r, g) computes X(r, j) for j = 16 g .. 16 g + 15.
// ---------------------------------------------------------------------------
template <typename T>
__host__ __device__ constexpr int trsm_li_pitch() {
  return kNB + 16 / (int)sizeof(T);  // rows of Li 16-byte aligned
}

template <typename T>
constexpr size_t trsm_smem() {
  return (size_t)kNB * (kNB + 1) * sizeof(T) + (size_t)kNB * trsm_li_pitch<T>() * sizeof(T);
}

template <typename T, bool LU>
__global__ void __launch_bounds__(256) k_trsm(FD<T> d0, int64_t item_off) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  bool upper = false;
  const int bid = LU ? lu_block(d0, upper) : (int)blockIdx.x;
  const FD<T> d = (LU && upper) ? upper_view(d0) : d0;
  T(*As)[kNB + 1] = reinterpret_cast<T(*)[kNB + 1]>(smem_raw);  // As[c][r] = A(r0 + r, c0 + c)
  constexpr int LP = trsm_li_pitch<T>();
  T(*Li)[LP] = reinterpret_cast<T(*)[LP]>(
      smem_raw + (size_t)kNB * (kNB + 1) * sizeof(T));          // Li[c][j] = Linv(j, c)
  const Item it = d.items[item_off + bid];
  const SnInfo f = d.sn[it.s];
  const int nf = f.k + f.m;
  const int c0 = it.t * kNB;
  const int b = min(kNB, f.k - c0);
  const int r0 = it.a;
  const int rows = min(kTrsmRows, nf - r0);
  const int tid = threadIdx.x, r = tid & 63, g = tid >> 6;
  const T* Dv = (LU ? d.dinv_t : d.dinv) + (int64_t)it.b * kNB * kNB;
  // LU with pivoting, upper half: the columns of F12^T come in the pivot
  // order of the diagonal block (Pi F12), the rows' own permutation
  // (LDL^T with symmetric pivoting: F21's columns, likewise)
  const uint8_t* pv = (LU ? (upper && d.piv) : (d.D && d.piv)) ? d.piv + f.first + c0 : nullptr;
  {
    // all global loads of this thread in flight before the first shared store
    constexpr int PER = kNB * kNB / 256;
    const T* P = d.L + f.Loff + (int64_t)c0 * nf + r0;
    T va[PER], vl[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int idx = tid + u * 256, c = idx / kNB, rr = idx % kNB;
      const int cs = (pv && c < b) ? (int)pv[c] : c;
      va[u] = (c < b && rr < rows) ? P[(int64_t)cs * nf + rr] : T(0);
      vl[u] = Dv[idx];
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int idx = tid + u * 256, c = idx / kNB, rr = idx % kNB;
      As[c][rr] = va[u];
      Li[c][rr] = vl[u];
    }
  }
  __syncthreads();
  // thread (r, g): row r, the 16 contiguous columns j = 16 g + q; the product
  // is triangular (c <= j), so c stops at the thread's last column, and at
  // the panel width b (A is zero beyond it; columns j >= b stay zero)
  T x[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) x[q] = T(0);
  const int cend = 16 * g < b ? min(16 * g + 15, b - 1) : -1;
  for (int c = 0; c <= cend; ++c) {
    const T a = As[c][r];
    // the 16 inverse values as four (FP64: eight) 16-byte shared loads
    T lv[16];
    const uint4* lrow = reinterpret_cast<const uint4*>(&Li[c][16 * g]);
#pragma unroll
    for (int v = 0; v < 16 * (int)sizeof(T) / 16; ++v)
      reinterpret_cast<uint4*>(lv)[v] = lrow[v];
#pragma unroll
    for (int q = 0; q < 16; ++q) x[q] = fma(a, lv[q], x[q]);
  }
  if (d.D) {  // LDL^T: L21 = A L_tt^{-T} D_t^{-1}
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int j = 16 * g + q;
      if (j < b) x[q] /= d.D[f.first + c0 + j];
    }
  }
  if (r < rows) {
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int j = 16 * g + q;
      if (j < b) front_col(d, f, c0 + j)[r0 + r] = x[q];
    }
  }
  if (d.split != nullptr) {
    // FP32 tensor-core path: tf32 hi / lo split of the solved rows, row-major
    // staging rows holding four panel slots (area 0, slot = step mod 4) or
    // eight (area 1, lookahead levels, slot = step mod 8), each slot 64 hi
    // then 64 lo floats; zero beyond the panel width b
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) As[16 * g + q][r] = (16 * g + q) < b ? x[q] : T(0);
    __syncthreads();
    const int64_t so = d.soff[it.s];
    const bool area1 = (so >> kSoffAreaShift) != 0;
    const int64_t srow = so & (((int64_t)1 << kSoffAreaShift) - 1);
    const int sw = area1 ? 1024 : 512;
    float* out = (area1 ? d.split_b : d.split) + (srow + r0) * sw + (it.t & (area1 ? 7 : 3)) * 128;
    for (int idx = tid; idx < rows * kNB; idx += blockDim.x) {
      const int rw = idx / kNB, c = idx % kNB;
      const float xv = (float)As[c][rw];
      uint32_t hb;
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hb) : "f"(xv));
      const float hi = __uint_as_float(hb);
      out[(int64_t)rw * sw + c] = hi;
      out[(int64_t)rw * sw + kNB + c] = xv - hi;
    }
  }
}

// ---------------------------------------------------------------------------
// Large fronts, panel step t: trailing lower update of the TILE x TILE tile
// (I, J), I >= J:  C -= P_I P_J^T with P the b panel columns.  256 threads,
// thread (tr, tc) of a 16 x 16 grid holds the (TILE/16)^2 entries
// (tr + 16 i, tc + 16 j); the tile is a per-front-size choice of the
// schedule (32, 64 or 128).
// ---------------------------------------------------------------------------
template <typename T, int TILE>
constexpr size_t syrk_smem() {
  return (size_t)2 * kNB * TILE * sizeof(T);
}

template <typename T, int TILE, bool LU>
__device__ __forceinline__ void syrk_tile(const FD<T>& d, int bid, int64_t item_off) {
  constexpr int R = TILE / 16;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T(*As)[TILE] = reinterpret_cast<T(*)[TILE]>(smem_raw);
  T(*Bs)[TILE] = reinterpret_cast<T(*)[TILE]>(smem_raw + (size_t)kNB * TILE * sizeof(T));
  const Item it = d.items[item_off + bid];
  const SnInfo f = d.sn[it.s];
  const int nf = f.k + f.m;
  const int c0 = it.t * kNB;
  const int b = min(kNB, f.k - c0);
  const int p0 = c0 + b;
  const int rI = p0 + it.a * TILE, rJ = p0 + it.b * TILE;
  const int tid = threadIdx.x;
  const T* P = d.L + f.Loff + (int64_t)c0 * nf;
  const T* Pb = LU ? d.Lb + f.Loff + (int64_t)c0 * nf : P;  // LU: the other half
  for (int idx = tid; idx < b * TILE; idx += blockDim.x) {
    const int q = idx / TILE, r = idx % TILE;
    const T* col = P + (int64_t)q * nf;
    const T* colb = LU ? Pb + (int64_t)q * nf : col;
    As[q][r] = (rI + r < nf) ? col[rI + r] : T(0);
    // LDL^T: C -= P_I D P_J^T, the pivots folded into the B operand
    const T w = d.D ? d.D[f.first + c0 + q] : T(1);
    Bs[q][r] = (rJ + r < nf) ? colb[rJ + r] * w : T(0);
  }
  __syncthreads();
  const int tr = tid & 15, tc = tid >> 4;
  T acc[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) acc[i][j] = T(0);
  for (int q = 0; q < b; ++q) {
    T a[R], bb[R];
#pragma unroll
    for (int i = 0; i < R; ++i) a[i] = As[q][tr + 16 * i];
#pragma unroll
    for (int j = 0; j < R; ++j) bb[j] = Bs[q][tc + 16 * j];
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
      for (int j = 0; j < R; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
  }
  // two-phase read-modify-write: for tiles up to 64 all R^2 loads of the
  // thread are in flight before any store; for 128 (64 values per thread)
  // one column's R loads at a time, to stay within registers
  constexpr int G = R <= 4 ? R : 1;  // columns per load/store group
#pragma unroll
  for (int j0 = 0; j0 < R; j0 += G) {
    T* p[R][G];
    T cur[R][G];
#pragma unroll
    for (int jj = 0; jj < G; ++jj) {
      const int c = rJ + tc + 16 * (j0 + jj);
      T* col = c < nf ? front_col(d, f, c) : nullptr;
#pragma unroll
      for (int i = 0; i < R; ++i) {
        const int r = rI + tr + 16 * i;
        p[i][jj] = (col && r < nf && r >= c) ? col + r : nullptr;
      }
    }
#pragma unroll
    for (int jj = 0; jj < G; ++jj)
#pragma unroll
      for (int i = 0; i < R; ++i) cur[i][jj] = p[i][jj] ? *p[i][jj] : T(0);
#pragma unroll
    for (int jj = 0; jj < G; ++jj)
#pragma unroll
      for (int i = 0; i < R; ++i)
        if (p[i][jj]) *p[i][jj] = cur[i][jj] - acc[i][j0 + jj];
  }
}

template <typename T, int TILE, bool LU>
__global__ void __launch_bounds__(256) k_syrk(FD<T> d, int64_t item_off) {
  if (LU) {
    bool upper = false;
    const int bid = lu_block(d, upper);
    if (upper) syrk_tile<T, TILE, LU>(upper_view(d), bid, item_off);
    else syrk_tile<T, TILE, LU>(d, bid, item_off);
  } else {
    syrk_tile<T, TILE, LU>(d, (int)blockIdx.x, item_off);
  }
}

// ---------------------------------------------------------------------------
// Partitioned inverse (SpTRSV variant 3, Sec. 5).  For a large front with
// pivot columns [L11; L21], P = [L11^{-1}; -L21 L11^{-1}] in the layout of L:
// the front's columns of the level's L_l^{-1}.  L11 X = I is solved by block
// rows, right-looking, over all rows of the front at once (update rows start
// at zero, so they end at -L21 X).  Init writes P = 0 and the kept inverses
// L_jj^{-1} on the diagonal blocks; step t takes, for every tile (i, j) with
// i > t >= j, P(i, j) -= L(i, t) P(t, j) and finalises block row t + 1 with
// P(t+1, j) = L_{t+1,t+1}^{-1} P(t+1, j).
// ---------------------------------------------------------------------------
// Init, item (s, j): column block j of front s.
template <typename T>
__global__ void __launch_bounds__(256) k_pinv_init(FD<T> d, int64_t item_off) {
  const Item it = d.items[item_off + blockIdx.x];
  const SnInfo f = d.sn[it.s];
  const int nf = f.k + f.m, c0 = it.t * kNB, bj = min(kNB, f.k - c0);
  const T* Dv = d.dinv + (d.ioff[it.s] + it.t) * (int64_t)(kNB * kNB);
  T* Pc = d.P + f.Loff + (int64_t)c0 * nf;
  for (int c = 0; c < bj; ++c)
    for (int r = threadIdx.x; r < nf; r += blockDim.x) {
      const int rr = r - c0;
      Pc[(int64_t)c * nf + r] = (rr >= c && rr < bj) ? Dv[c * kNB + rr] : T(0);
    }
}

template <typename T>
constexpr size_t pinv_smem() {
  return (size_t)2 * kNB * (kNB + 1) * sizeof(T);
}

// Step t, item (s, t, i, j): one 64 x 64 tile.  Thread (tx, ty) owns rows
// tx + 16 a and columns ty + 16 b of the tile.
template <typename T>
__global__ void __launch_bounds__(256) k_pinv_step(FD<T> d, int64_t item_off) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T(*As)[kNB + 1] = reinterpret_cast<T(*)[kNB + 1]>(smem_raw);  // As[q][r]
  T(*Bs)[kNB + 1] = reinterpret_cast<T(*)[kNB + 1]>(
      smem_raw + (size_t)kNB * (kNB + 1) * sizeof(T));         // Bs[q][c]
  const Item it = d.items[item_off + blockIdx.x];
  const SnInfo f = d.sn[it.s];
  const int k = f.k, nf = k + f.m, nb = (k + kNB - 1) / kNB;
  const int t = it.t, i = it.a, j = it.b;
  const int r0 = i < nb ? i * kNB : k + (i - nb) * kNB;
  const int rows = min(kNB, (i < nb ? k : nf) - r0);
  const int t0 = t * kNB, bt = min(kNB, k - t0);
  const int c0 = j * kNB, bj = min(kNB, k - c0);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const T* Lp = d.L + f.Loff;
  T* Pp = d.P + f.Loff;
  // As[q][r] = L(r0 + r, t0 + q), Bs[q][c] = P(t0 + q, c0 + c) (final)
  for (int idx = tid; idx < kNB * kNB; idx += 256) {
    const int q = idx / kNB, r = idx % kNB;
    As[q][r] = (q < bt && r < rows) ? Lp[(int64_t)(t0 + q) * nf + r0 + r] : T(0);
  }
  for (int idx = tid; idx < kNB * kNB; idx += 256) {
    const int c = idx / kNB, q = idx % kNB;
    Bs[q][c] = (q < bt && c < bj) ? Pp[(int64_t)(c0 + c) * nf + t0 + q] : T(0);
  }
  __syncthreads();
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  for (int q = 0; q < bt; ++q) {
    T av[4], bv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) av[a] = As[q][tx + 16 * a];
#pragma unroll
    for (int b = 0; b < 4; ++b) bv[b] = Bs[q][ty + 16 * b];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
  }
  T cv[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int r = tx + 16 * a, c = ty + 16 * b;
      cv[a][b] = (r < rows && c < bj) ? Pp[(int64_t)(c0 + c) * nf + r0 + r] - acc[a][b] : T(0);
    }
  if (i == t + 1 && i < nb) {
    // block row i is complete: P(i, j) = L_ii^{-1} P(i, j) (lower triangular,
    // so rows r < rows only need q <= r < rows)
    const T* Dv = d.dinv + (d.ioff[it.s] + i) * (int64_t)(kNB * kNB);
    __syncthreads();
    for (int idx = tid; idx < kNB * kNB; idx += 256) As[idx / kNB][idx % kNB] = Dv[idx];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) Bs[tx + 16 * a][ty + 16 * b] = cv[a][b];
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
    for (int q = 0; q < rows; ++q) {
      T av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[q][tx + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[q][ty + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) cv[a][b] = acc[a][b];
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int r = tx + 16 * a, c = ty + 16 * b;
      if (r < rows && c < bj) Pp[(int64_t)(c0 + c) * nf + r0 + r] = cv[a][b];
    }
}

// ---------------------------------------------------------------------------
// SpTRSV variant 4 (Sec. 5): the partitioned inverse of every front, then
// its transpose.  k_pinv_small takes a front without kept diagonal-block
// inverses (k + m <= 128) in one CTA: with L11 and L21 in shared memory
// (L11 and Z packed by rows), thread c solves L11 z = e_c by substitution
// into column c of Z = L11^{-1}, then P = [Z; -L21 Z] is written in the
// layout of L (zero above the diagonal of Z).
// ---------------------------------------------------------------------------
template <typename T>
constexpr size_t pinv_small_smem() {
  return (size_t)kSmallMax * (kSmallMax + 1) * sizeof(T);
}

template <typename T>
__global__ void __launch_bounds__(256) k_pinv_small(FD<T> d, int64_t item_off) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SnInfo f = d.sn[d.items[item_off + blockIdx.x].s];
  const int k = f.k, m = f.m, nf = k + m;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int np = k * (k + 1) / 2;
  T* Ls = reinterpret_cast<T*>(smem_raw);  // L11 packed by rows: (i, c) at i(i+1)/2 + c
  T* Zs = Ls + np;                         // Z packed the same way
  T* Ws = Zs + np;                         // L21: (r, p) at p m + r
  const T* Lp = d.L + f.Loff;
  T* Pp = d.P + f.Loff;
  for (int c = warp; c < k; c += nw) {
    for (int i = c + lane; i < k; i += 32) Ls[i * (i + 1) / 2 + c] = Lp[(int64_t)c * nf + i];
    for (int r = lane; r < m; r += 32) Ws[c * m + r] = Lp[(int64_t)c * nf + k + r];
  }
  __syncthreads();
  for (int c = tid; c < k; c += blockDim.x)
    for (int i = c; i < k; ++i) {
      const T* li = Ls + i * (i + 1) / 2;
      T acc = i == c ? T(1) : T(0);
      for (int q = c; q < i; ++q) acc -= li[q] * Zs[q * (q + 1) / 2 + c];
      Zs[i * (i + 1) / 2 + c] = acc / li[i];
    }
  __syncthreads();
  for (int c = warp; c < k; c += nw) {
    T* pc = Pp + (int64_t)c * nf;
    for (int i = lane; i < k; i += 32) pc[i] = i >= c ? Zs[i * (i + 1) / 2 + c] : T(0);
    for (int r = lane; r < m; r += 32) {
      T acc = T(0);
      for (int q = c; q < k; ++q) acc += Ws[q * m + r] * Zs[q * (q + 1) / 2 + c];
      pc[k + r] = -acc;
    }
  }
}

// PT = P^T front by front (64 x 64 tiles through shared memory): row i of
// P_s becomes the k contiguous values PT[Loff + i k ...], so the forward
// products read each row of P with unit stride.  Item (s, 0, i0, j0).
template <typename T>
__global__ void __launch_bounds__(256) k_pt(FD<T> d, int64_t item_off) {
  __shared__ T tile[kNB][kNB + 1];
  const Item it = d.items[item_off + blockIdx.x];
  const SnInfo f = d.sn[it.s];
  const int k = f.k, nf = k + f.m, i0 = it.a, j0 = it.b;
  const T* Pp = d.P + f.Loff;
  T* Q = d.PT + f.Loff;
  for (int idx = threadIdx.x; idx < kNB * kNB; idx += blockDim.x) {
    const int c = idx / kNB, r = idx % kNB;
    if (i0 + r < nf && j0 + c < k) tile[c][r] = Pp[(int64_t)(j0 + c) * nf + i0 + r];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < kNB * kNB; idx += blockDim.x) {
    const int r = idx / kNB, c = idx % kNB;
    if (i0 + r < nf && j0 + c < k) Q[(int64_t)(i0 + r) * k + j0 + c] = tile[c][r];
  }
}

// av[e] = T(sum of the CSR values of lower entry e): one pass per numeric
// call, so the assembly kernels read values in their own order.
template <typename T>
__global__ void k_gather_values(const int64_t* asrc_ptr, const int64_t* asrc, const double* vals,
                                T* av, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int64_t p = asrc_ptr[e]; p < asrc_ptr[e + 1]; ++p) v += vals[asrc[p]];
    av[e] = T(v);
  }
}

// Shared memory of a small front of size class `param` (LU pads the leading
// dimension by one).
template <typename T>
size_t small_smem(int param, bool lu) {
  return (size_t)param * (param + (lu ? 1 : 0)) * sizeof(T);
}

template <typename T, int MODE>
cudaError_t small_attributes(int bytes) {
  cudaError_t e = cudaFuncSetAttribute(k_small_front<T, MODE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_small_queue<T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              bytes);
}

// Small-front launches of one kind (one CTA per front, or the queue).
template <typename T, int MODE>
cudaError_t launch_small(const Launch& L, const FD<T>& d, cudaStream_t st) {
  const size_t smem = small_smem<T>(L.param, MODE != 0);
  if (L.kind == K_SMALL) {
    k_small_front<T, MODE><<<L.count, 256, smem, st>>>(d, L.item_off);
    return cudaGetLastError();
  }
  // the queue: one resident wave, SMs x the blocks per SM the front size allows
  int dev = 0, sms = 0, per = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_small_queue<T, MODE>, kQueueThreads,
                                                      smem);
  if (e != cudaSuccess) return e;
  const int blocks = std::max(1, std::min(L.count, sms * std::max(per, 1)));
  k_small_queue<T, MODE><<<blocks, kQueueThreads, smem, st>>>(d, L.item_off, L.count);
  return cudaGetLastError();
}

template <typename T, bool LU>
cudaError_t syrk_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_syrk<T, 32, LU>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)syrk_smem<T, 32>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_syrk<T, 128, LU>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)syrk_smem<T, 128>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_syrk<T, 64, LU>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)syrk_smem<T, 64>());
}

// Trailing-update launch with the schedule's tile; LU runs both halves.
template <typename T, bool LU>
void launch_syrk(const Launch& L, const FD<T>& d, dim3 grid, cudaStream_t st) {
  if (L.tile == 32) k_syrk<T, 32, LU><<<grid, 256, syrk_smem<T, 32>(), st>>>(d, L.item_off);
  else if (L.tile == 128) k_syrk<T, 128, LU><<<grid, 256, syrk_smem<T, 128>(), st>>>(d, L.item_off);
  else k_syrk<T, 64, LU><<<grid, 256, syrk_smem<T, 64>(), st>>>(d, L.item_off);
}

template <typename T>
cudaError_t init_t() {
  const int small_max = (int)small_smem<T>(kSmallMax, false);
  const int small_max_pad = (int)small_smem<T>(kSmallMax, true);
  cudaError_t e = small_attributes<T, 0>(small_max);
  if (e != cudaSuccess) return e;
  e = small_attributes<T, 1>(small_max_pad);
  if (e != cudaSuccess) return e;
  e = small_attributes<T, 2>(small_max_pad);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_getrf<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)getrf_smem<T>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_sytrf<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sytrf_smem<T>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_trsm<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)trsm_smem<T>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_trsm<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)trsm_smem<T>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_potrf<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)potrf_smem<T>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_pinv_step<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)pinv_smem<T>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_pinv_small<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)pinv_small_smem<T>());
  if (e != cudaSuccess) return e;
  e = syrk_attributes<T, false>();
  if (e != cudaSuccess) return e;
  return syrk_attributes<T, true>();
}

template <typename T>
cudaError_t launch_t(const Launch& L, const FactorArgs& a, cudaStream_t st) {
  const FD<T> d = make_fd<T>(a);
  const dim3 grid(L.count);
  // LU: assembly, panel solve and trailing update run both halves
  const dim3 grid2(a.lu ? 2 * L.count : L.count);
  switch (L.kind) {
    case K_SMALL:
    case K_SMALL_Q:
      if (a.lu) return launch_small<T, 1>(L, d, st);
      if (a.D && a.piv) return launch_small<T, 2>(L, d, st);
      return launch_small<T, 0>(L, d, st);
    case K_ASSEMBLE:
      if (a.lu) k_assemble<T, true><<<grid2, 256, 0, st>>>(d, L.item_off);
      else k_assemble<T, false><<<grid, 256, 0, st>>>(d, L.item_off);
      break;
    case K_POTRF:
      if (a.lu) k_getrf<T><<<grid, 256, getrf_smem<T>(), st>>>(d, L.item_off);
      else if (a.D && a.piv) k_sytrf<T><<<grid, 256, sytrf_smem<T>(), st>>>(d, L.item_off);
      else k_potrf<T><<<grid, 256, potrf_smem<T>(), st>>>(d, L.item_off);
      break;
    case K_TRSM:
      if (a.lu) k_trsm<T, true><<<grid2, 256, trsm_smem<T>(), st>>>(d, L.item_off);
      else k_trsm<T, false><<<grid, 256, trsm_smem<T>(), st>>>(d, L.item_off);
      break;
    case K_SYRK:
      if (a.lu) launch_syrk<T, true>(L, d, grid2, st);
      else launch_syrk<T, false>(L, d, grid, st);
      break;
    case K_SYRK_TC:
      return launch_syrk_tc(L, a, st);
    case K_PINV_INIT:
      k_pinv_init<T><<<grid, 256, 0, st>>>(d, L.item_off);
      break;
    case K_PINV:
      k_pinv_step<T><<<grid, 256, pinv_smem<T>(), st>>>(d, L.item_off);
      break;
    case K_PINV_SMALL:
      k_pinv_small<T><<<grid, 256, pinv_small_smem<T>(), st>>>(d, L.item_off);
      break;
    case K_PT:
      k_pt<T><<<grid, 256, 0, st>>>(d, L.item_off);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t factor_kernels_init(int prec) {
  return prec == MF_FP32 ? init_t<float>() : init_t<double>();
}

cudaError_t launch_gather_values(int prec, const FactorArgs& a, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int64_t g = (n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  if (prec == MF_FP32)
    k_gather_values<float><<<(int)g, 256, 0, st>>>(a.sym.asrc_ptr, a.sym.asrc, a.vals,
                                                   static_cast<float*>(a.av), n);
  else
    k_gather_values<double><<<(int)g, 256, 0, st>>>(a.sym.asrc_ptr, a.sym.asrc, a.vals,
                                                    static_cast<double*>(a.av), n);
  return cudaGetLastError();
}

cudaError_t launch_gather_upper(int prec, const int64_t* src_ptr, const int64_t* src,
                                const double* vals, void* avu, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int64_t g = (n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  if (prec == MF_FP32)
    k_gather_values<float><<<(int)g, 256, 0, st>>>(src_ptr, src, vals, static_cast<float*>(avu), n);
  else
    k_gather_values<double><<<(int)g, 256, 0, st>>>(src_ptr, src, vals, static_cast<double*>(avu), n);
  return cudaGetLastError();
}

cudaError_t launch_lu_swap(int prec, const FactorArgs& a, cudaStream_t st) {
  if (a.lu_swap_count <= 0 || a.piv == nullptr) return cudaSuccess;
  if (prec == MF_FP32)
    k_lu_swap<float><<<a.lu_swap_count, 256, 0, st>>>(make_fd<float>(a), a.lu_swap);
  else
    k_lu_swap<double><<<a.lu_swap_count, 256, 0, st>>>(make_fd<double>(a), a.lu_swap);
  return cudaGetLastError();
}

cudaError_t launch_factor(int prec, const Launch& L, const FactorArgs& a, cudaStream_t st) {
  if (L.count <= 0) return cudaSuccess;
  return prec == MF_FP32 ? launch_t<float>(L, a, st) : launch_t<double>(L, a, st);
}

}  // namespace mf
