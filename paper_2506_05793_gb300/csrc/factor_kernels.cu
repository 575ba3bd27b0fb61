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

#include <cstdint>

#include "kernels.h"

namespace mf {
namespace {

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
  T* L;
  T* U;
  unsigned long long* status;
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
  d.L = static_cast<T*>(a.L);
  d.U = static_cast<T*>(a.U);
  d.status = a.status;
  return d;
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

// Sum of the (possibly duplicated) CSR entries of one front entry.
template <typename T>
__device__ __forceinline__ T a_entry(const FD<T>& d, int64_t e) {
  double v = 0.0;
  for (int64_t p = d.asrc_ptr[e]; p < d.asrc_ptr[e + 1]; ++p) v += d.vals[d.asrc[p]];
  return T(v);
}

__device__ __forceinline__ int lower_bound_i32(const int32_t* a, int n, int key) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Unblocked right-looking partial Cholesky of the first `k` columns of an
// n x n lower-triangular block held column-major in shared memory (ld).
// Records the first non-positive pivot (global column col0 + j).
template <typename T>
__device__ void smem_partial_chol(T* F, int ld, int n, int k, int col0,
                                  unsigned long long* status) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int j = 0; j < k; ++j) {
    const T dj = F[j * ld + j];
    if (tid == 0 && !(dj > T(0))) atomicMin(status, (unsigned long long)(col0 + j));
    const T ljj = dsqrt(dj);
    const T rinv = T(1) / ljj;
    __syncthreads();
    for (int i = j + 1 + tid; i < n; i += blockDim.x) F[j * ld + i] *= rinv;
    if (tid == 0) F[j * ld + j] = ljj;
    __syncthreads();
    for (int c = j + 1 + warp; c < n; c += nw) {
      const T lc = F[j * ld + c];
      for (int i = c + lane; i < n; i += 32) F[c * ld + i] -= F[j * ld + i] * lc;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Small fronts: one CTA assembles and factors the whole front in shared
// memory and writes the L panel and the update matrix.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_small_front(FD<T> d, int64_t item_off) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* F = reinterpret_cast<T*>(smem_raw);
  const Item it = d.items[item_off + blockIdx.x];
  const SnInfo f = d.sn[it.s];
  const int k = f.k, m = f.m, nf = k + m;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int i = tid; i < nf * nf; i += blockDim.x) F[i] = T(0);
  __syncthreads();
  for (int c = warp; c < k; c += nw) {
    const int g = f.first + c;
    for (int64_t e = d.acol_ptr[g] + lane; e < d.acol_ptr[g + 1]; e += 32)
      F[c * nf + d.arow[e]] = a_entry(d, e);
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
      for (int ic = jc + lane; ic < mc; ic += 32) F[dc * nf + map[ic]] += u[ic];
    }
    __syncthreads();
  }
  smem_partial_chol(F, nf, nf, k, f.first, d.status);
  T* Lp = d.L + f.Loff;
  for (int c = warp; c < k; c += nw)
    for (int r = lane; r < nf; r += 32) Lp[(int64_t)c * nf + r] = F[c * nf + r];
  T* Up = d.U + f.Uoff;
  for (int c = warp; c < m; c += nw)
    for (int r = lane; r < m; r += 32) Up[(int64_t)c * m + r] = F[(k + c) * nf + k + r];
}

// ---------------------------------------------------------------------------
// Large fronts, assembly of a chunk of front columns [a, b): zero, scatter
// the entries of A, then pull every child's update matrix in order.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_assemble(FD<T> d, int64_t item_off) {
  const Item it = d.items[item_off + blockIdx.x];
  const SnInfo f = d.sn[it.s];
  const int k = f.k, nf = k + f.m, c0 = it.a, c1 = it.b;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int c = c0 + warp; c < c1; c += nw) {
    T* col = front_col(d, f, c);
    const int r0 = c < k ? 0 : c;
    for (int r = r0 + lane; r < nf; r += 32) col[r] = T(0);
  }
  __syncthreads();
  const int ce = c1 < k ? c1 : k;
  for (int c = c0 + warp; c < ce; c += nw) {
    T* col = front_col(d, f, c);
    const int g = f.first + c;
    for (int64_t e = d.acol_ptr[g] + lane; e < d.acol_ptr[g + 1]; e += 32)
      col[d.arow[e]] = a_entry(d, e);
  }
  __syncthreads();
  for (int ci = 0; ci < f.nchild; ++ci) {
    const SnInfo ch = d.sn[d.children[f.child_begin + ci]];
    const int mc = ch.m;
    const int32_t* map = d.relmap + ch.map_off;
    const int lo = lower_bound_i32(map, mc, c0);
    const int hi = lower_bound_i32(map, mc, c1);
    const T* Uc = d.U + ch.Uoff;
    for (int jc = lo + warp; jc < hi; jc += nw) {
      T* col = front_col(d, f, map[jc]);
      const T* u = Uc + (int64_t)jc * mc;
      for (int ic = jc + lane; ic < mc; ic += 32) col[map[ic]] += u[ic];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Large fronts, panel step t: Cholesky of the b x b diagonal block.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_potrf(FD<T> d, int64_t item_off) {
  __shared__ T D[kNB * (kNB + 1)];
  const Item it = d.items[item_off + blockIdx.x];
  const SnInfo f = d.sn[it.s];
  const int c0 = it.t * kNB;
  const int b = min(kNB, f.k - c0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  constexpr int ld = kNB + 1;
  for (int c = warp; c < b; c += nw) {
    const T* col = front_col(d, f, c0 + c) + c0;
    for (int r = c + lane; r < b; r += 32) D[c * ld + r] = col[r];
  }
  __syncthreads();
  smem_partial_chol(D, ld, b, b, f.first + c0, d.status);
  for (int c = warp; c < b; c += nw) {
    T* col = front_col(d, f, c0 + c) + c0;
    for (int r = c + lane; r < b; r += 32) col[r] = D[c * ld + r];
  }
}

// ---------------------------------------------------------------------------
// Large fronts, panel step t: rows [r0, r0 + kTrsmRows) of the panel below
// the diagonal block, X = A L_tt^{-T}; one thread per row.
// ---------------------------------------------------------------------------
template <typename T>
constexpr size_t trsm_smem() {
  return (size_t)(kNB * (kNB + 1) + kNB * (kTrsmRows + 1) + kNB) * sizeof(T);
}

template <typename T>
__global__ void __launch_bounds__(kTrsmRows) k_trsm(FD<T> d, int64_t item_off) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T(*D)[kNB + 1] = reinterpret_cast<T(*)[kNB + 1]>(smem_raw);  // D[c][r] = L_tt(r, c)
  T(*X)[kTrsmRows + 1] = reinterpret_cast<T(*)[kTrsmRows + 1]>(
      smem_raw + (size_t)kNB * (kNB + 1) * sizeof(T));          // X[c][row]
  T* rinv = reinterpret_cast<T*>(smem_raw + (size_t)(kNB * (kNB + 1) + kNB * (kTrsmRows + 1)) *
                                                sizeof(T));
  const Item it = d.items[item_off + blockIdx.x];
  const SnInfo f = d.sn[it.s];
  const int nf = f.k + f.m;
  const int c0 = it.t * kNB;
  const int b = min(kNB, f.k - c0);
  const int r0 = it.a;
  const int rows = min(kTrsmRows, nf - r0);
  const int tid = threadIdx.x;
  for (int c = 0; c < b; ++c) {
    const T* col = front_col(d, f, c0 + c);
    if (tid < b && tid >= c) D[c][tid] = col[c0 + tid];
    if (tid < rows) X[c][tid] = col[r0 + tid];
  }
  __syncthreads();
  if (tid < b) rinv[tid] = T(1) / D[tid][tid];
  __syncthreads();
  if (tid < rows) {
    for (int j = 0; j < b; ++j) {
      T x = X[j][tid];
      for (int i = 0; i < j; ++i) x -= X[i][tid] * D[i][j];
      X[j][tid] = x * rinv[j];
    }
    for (int c = 0; c < b; ++c) front_col(d, f, c0 + c)[r0 + tid] = X[c][tid];
  }
}

// ---------------------------------------------------------------------------
// Large fronts, panel step t: trailing lower update of the kTile x kTile
// tile (I, J), I >= J:  C -= P_I P_J^T with P the b panel columns.
// ---------------------------------------------------------------------------
template <typename T>
constexpr size_t syrk_smem() {
  return (size_t)2 * kNB * kTile * sizeof(T);
}

template <typename T>
__global__ void __launch_bounds__(256) k_syrk(FD<T> d, int64_t item_off) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T(*As)[kTile] = reinterpret_cast<T(*)[kTile]>(smem_raw);
  T(*Bs)[kTile] = reinterpret_cast<T(*)[kTile]>(smem_raw + (size_t)kNB * kTile * sizeof(T));
  const Item it = d.items[item_off + blockIdx.x];
  const SnInfo f = d.sn[it.s];
  const int nf = f.k + f.m;
  const int c0 = it.t * kNB;
  const int b = min(kNB, f.k - c0);
  const int p0 = c0 + b;
  const int rI = p0 + it.a * kTile, rJ = p0 + it.b * kTile;
  const int tid = threadIdx.x;
  const T* P = d.L + f.Loff + (int64_t)c0 * nf;
  for (int idx = tid; idx < b * kTile; idx += blockDim.x) {
    const int q = idx / kTile, r = idx % kTile;
    const T* col = P + (int64_t)q * nf;
    As[q][r] = (rI + r < nf) ? col[rI + r] : T(0);
    Bs[q][r] = (rJ + r < nf) ? col[rJ + r] : T(0);
  }
  __syncthreads();
  const int tr = tid & 15, tc = tid >> 4;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  for (int q = 0; q < b; ++q) {
    T a[4], bb[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = As[q][tr + 16 * i];
#pragma unroll
    for (int j = 0; j < 4; ++j) bb[j] = Bs[q][tc + 16 * j];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int c = rJ + tc + 16 * j;
    if (c >= nf) continue;
    T* col = front_col(d, f, c);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = rI + tr + 16 * i;
      if (r < nf && r >= c) col[r] -= acc[i][j];
    }
  }
}

template <typename T>
cudaError_t init_t() {
  cudaError_t e = cudaFuncSetAttribute(k_small_front<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kSmallMax * kSmallMax * (int)sizeof(T));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_trsm<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)trsm_smem<T>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_syrk<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)syrk_smem<T>());
}

template <typename T>
cudaError_t launch_t(const Launch& L, const FactorArgs& a, cudaStream_t st) {
  const FD<T> d = make_fd<T>(a);
  const dim3 grid(L.count);
  switch (L.kind) {
    case K_SMALL:
      k_small_front<T><<<grid, 256, (size_t)L.param * L.param * sizeof(T), st>>>(d, L.item_off);
      break;
    case K_ASSEMBLE:
      k_assemble<T><<<grid, 256, 0, st>>>(d, L.item_off);
      break;
    case K_POTRF:
      k_potrf<T><<<grid, 256, 0, st>>>(d, L.item_off);
      break;
    case K_TRSM:
      k_trsm<T><<<grid, kTrsmRows, trsm_smem<T>(), st>>>(d, L.item_off);
      break;
    case K_SYRK:
      k_syrk<T><<<grid, 256, syrk_smem<T>(), st>>>(d, L.item_off);
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

cudaError_t launch_factor(int prec, const Launch& L, const FactorArgs& a, cudaStream_t st) {
  if (L.count <= 0) return cudaSuccess;
  return prec == MF_FP32 ? launch_t<float>(L, a, st) : launch_t<double>(L, a, st);
}

}  // namespace mf
