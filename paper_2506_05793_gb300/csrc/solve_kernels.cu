// solve_kernels.cu -- supernodal triangular solves and the FP64 residual.
//
// Paper Sec. 5, SpTRSV variant 1: level-set scheduling over the supernodal
// blocks; for each supernode i, x_i := L_ii^{-1} b_i (TRSV/TRSM) and then
// b_k := b_k - L_ki x_i (GEMV/GEMM) for the rows below; several right-hand
// sides use TRSM/GEMM instead of TRSV/GEMV.  Small supernodes are batched
// one CTA each; large ones are blocked by kNB columns with the diagonal solve
// and the row-block updates batched over the level.
//
// Forward sweep (leaves -> root) is multifrontal: supernode s owns a work
// front W_s (nf x nrhs).  W_s[0:k] starts as b(first..first+k) and W_s[k:]
// as 0; every child c adds its update vector W_c[k_c:] through the relative
// map (parent-pull, fixed order, deterministic).  After the diagonal solve
// and the update, W_s[k:] holds u_s = -L21 x_s + sum of the children's rows
// for the parent to pull.
// Backward sweep (root -> leaves): x_s = L11^{-T} (y_s - L21^T x(rows_s)),
// gathering x at the update rows from the already final ancestors.
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"

namespace mf {
namespace {

template <typename T>
struct SD {
  const SnInfo* sn;
  const int32_t* children;
  const int32_t* relmap;
  const int32_t* rowidx;
  const Item* items;
  const T* L;
  T* Y;
  T* W;
  int64_t n;
  int nrhs;
};

template <typename T>
SD<T> make_sd(const SolveArgs& a) {
  SD<T> d;
  d.sn = a.sym.sn;
  d.children = a.sym.children;
  d.relmap = a.sym.relmap;
  d.rowidx = a.sym.rowidx;
  d.items = a.sym.items;
  d.L = static_cast<const T*>(a.L);
  d.Y = static_cast<T*>(a.Y);
  d.W = static_cast<T*>(a.W);
  d.n = a.n;
  d.nrhs = a.nrhs;
  return d;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// W_s pointer for rhs r: element i of the front work vector is Ws(r)[i].
template <typename T>
__device__ __forceinline__ T* wfront(const SD<T>& d, const SnInfo& f, int r) {
  const int64_t nf = (int64_t)f.k + f.m;
  return d.W + f.woff * d.nrhs + (int64_t)r * nf;
}

// ---------------------------------------------------------------------------
// Forward, small supernode: gather, diagonal solve and update in shared memory.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_fw_small(SD<T> d, int64_t item_off) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* F = reinterpret_cast<T*>(smem_raw);  // F[r * nf + i]
  const SnInfo f = d.sn[d.items[item_off + blockIdx.x].s];
  const int k = f.k, nf = k + f.m, nrhs = d.nrhs;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < nf * nrhs; idx += blockDim.x) {
    const int r = idx / nf, i = idx % nf;
    F[idx] = i < k ? d.Y[(int64_t)r * d.n + f.first + i] : T(0);
  }
  __syncthreads();
  for (int ci = 0; ci < f.nchild; ++ci) {
    const SnInfo ch = d.sn[d.children[f.child_begin + ci]];
    const int mc = ch.m;
    const int32_t* map = d.relmap + ch.map_off;
    for (int idx = tid; idx < mc * nrhs; idx += blockDim.x) {
      const int r = idx / mc, ic = idx % mc;
      F[r * nf + map[ic]] += wfront(d, ch, r)[ch.k + ic];
    }
    __syncthreads();
  }
  const T* Lp = d.L + f.Loff;
  for (int j = 0; j < k; ++j) {
    const T* col = Lp + (int64_t)j * nf;
    if (tid < nrhs) F[tid * nf + j] = F[tid * nf + j] / col[j];
    __syncthreads();
    const int len = nf - j - 1;
    for (int idx = tid; idx < len * nrhs; idx += blockDim.x) {
      const int r = idx / len, i = j + 1 + idx % len;
      F[r * nf + i] -= col[i] * F[r * nf + j];
    }
    __syncthreads();
  }
  for (int idx = tid; idx < nf * nrhs; idx += blockDim.x) {
    const int r = idx / nf, i = idx % nf;
    if (i < k) d.Y[(int64_t)r * d.n + f.first + i] = F[idx];
    else wfront(d, f, r)[i] = F[idx];
  }
}

// Forward, large supernode: initialise W_s and pull the children.
template <typename T>
__global__ void __launch_bounds__(256) k_fw_gather(SD<T> d, int64_t item_off) {
  const SnInfo f = d.sn[d.items[item_off + blockIdx.x].s];
  const int k = f.k, nf = k + f.m, nrhs = d.nrhs;
  const int tid = threadIdx.x;
  for (int64_t idx = tid; idx < (int64_t)nf * nrhs; idx += blockDim.x) {
    const int r = (int)(idx / nf), i = (int)(idx % nf);
    wfront(d, f, r)[i] = i < k ? d.Y[(int64_t)r * d.n + f.first + i] : T(0);
  }
  __syncthreads();
  for (int ci = 0; ci < f.nchild; ++ci) {
    const SnInfo ch = d.sn[d.children[f.child_begin + ci]];
    const int mc = ch.m;
    const int32_t* map = d.relmap + ch.map_off;
    for (int64_t idx = tid; idx < (int64_t)mc * nrhs; idx += blockDim.x) {
      const int r = (int)(idx / mc), ic = (int)(idx % mc);
      wfront(d, f, r)[map[ic]] += wfront(d, ch, r)[ch.k + ic];
    }
    __syncthreads();
  }
}

// Forward, large supernode, block t: x_t = L_tt^{-1} W[c0:c0+b]; written to
// W and to Y.
template <typename T>
__global__ void __launch_bounds__(256) k_fw_diag(SD<T> d, int64_t item_off) {
  __shared__ T X[kSolveChunk][kNB + 1];
  const Item it = d.items[item_off + blockIdx.x];
  const SnInfo f = d.sn[it.s];
  const int nf = f.k + f.m, nrhs = d.nrhs;
  const int c0 = it.t * kNB, b = min(kNB, f.k - c0);
  const int tid = threadIdx.x;
  for (int idx = tid; idx < b * nrhs; idx += blockDim.x) {
    const int r = idx / b, i = idx % b;
    X[r][i] = wfront(d, f, r)[c0 + i];
  }
  __syncthreads();
  const T* Lp = d.L + f.Loff;
  for (int j = 0; j < b; ++j) {
    const T* col = Lp + (int64_t)(c0 + j) * nf + c0;
    if (tid < nrhs) X[tid][j] = X[tid][j] / col[j];
    __syncthreads();
    const int len = b - j - 1;
    for (int idx = tid; idx < len * nrhs; idx += blockDim.x) {
      const int r = idx / len, i = j + 1 + idx % len;
      X[r][i] -= col[i] * X[r][j];
    }
    __syncthreads();
  }
  for (int idx = tid; idx < b * nrhs; idx += blockDim.x) {
    const int r = idx / b, i = idx % b;
    wfront(d, f, r)[c0 + i] = X[r][i];
    d.Y[(int64_t)r * d.n + f.first + c0 + i] = X[r][i];
  }
}

// Forward, large supernode, block t: W[rows] -= L[rows, c0:c0+b] x_t for a
// block of kTrsmRows rows starting at it.a (one thread per row).
template <typename T>
__global__ void __launch_bounds__(kTrsmRows) k_fw_upd(SD<T> d, int64_t item_off) {
  __shared__ T X[kNB][kSolveChunk];
  const Item it = d.items[item_off + blockIdx.x];
  const SnInfo f = d.sn[it.s];
  const int nf = f.k + f.m, nrhs = d.nrhs;
  const int c0 = it.t * kNB, b = min(kNB, f.k - c0);
  const int r0 = it.a, rows = min(kTrsmRows, nf - r0);
  const int tid = threadIdx.x;
  for (int idx = tid; idx < b * nrhs; idx += blockDim.x) {
    const int r = idx / b, q = idx % b;
    X[q][r] = wfront(d, f, r)[c0 + q];
  }
  __syncthreads();
  if (tid >= rows) return;
  T acc[kSolveChunk];
#pragma unroll
  for (int r = 0; r < kSolveChunk; ++r) acc[r] = T(0);
  const T* Lp = d.L + f.Loff + (int64_t)c0 * nf + r0 + tid;
  for (int q = 0; q < b; ++q) {
    const T l = Lp[(int64_t)q * nf];
#pragma unroll
    for (int r = 0; r < kSolveChunk; ++r)
      if (r < nrhs) acc[r] = fma(l, X[q][r], acc[r]);
  }
#pragma unroll
  for (int r = 0; r < kSolveChunk; ++r)
    if (r < nrhs) wfront(d, f, r)[r0 + tid] -= acc[r];
}

// ---------------------------------------------------------------------------
// Backward, small supernode: one CTA; warps own right-hand sides.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_bw_small(SD<T> d, int64_t item_off) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SnInfo f = d.sn[d.items[item_off + blockIdx.x].s];
  const int k = f.k, m = f.m, nf = k + m, nrhs = d.nrhs;
  T* G = reinterpret_cast<T*>(smem_raw);  // G[r * k + j]
  T* Xr = G + k * nrhs;                   // Xr[r * m + i]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int32_t* urow = d.rowidx + f.rows_off + k;
  for (int idx = tid; idx < k * nrhs; idx += blockDim.x) {
    const int r = idx / k, j = idx % k;
    G[idx] = d.Y[(int64_t)r * d.n + f.first + j];
  }
  for (int idx = tid; idx < m * nrhs; idx += blockDim.x) {
    const int r = idx / m, i = idx % m;
    Xr[idx] = d.Y[(int64_t)r * d.n + urow[i]];
  }
  __syncthreads();
  const T* Lp = d.L + f.Loff;
  if (m > 0) {
    for (int p = warp; p < k * nrhs; p += nw) {
      const int r = p / k, j = p % k;
      const T* col = Lp + (int64_t)j * nf + k;
      T s = T(0);
      for (int i = lane; i < m; i += 32) s = fma(col[i], Xr[r * m + i], s);
      s = warp_sum(s);
      if (lane == 0) G[r * k + j] -= s;
    }
    __syncthreads();
  }
  for (int r = warp; r < nrhs; r += nw) {
    T* g = G + r * k;
    for (int j = k - 1; j >= 0; --j) {
      const T* col = Lp + (int64_t)j * nf;
      T s = T(0);
      for (int i = j + 1 + lane; i < k; i += 32) s = fma(col[i], g[i], s);
      s = warp_sum(s);
      if (lane == 0) g[j] = (g[j] - s) / col[j];
      __syncwarp();
    }
  }
  __syncthreads();
  for (int idx = tid; idx < k * nrhs; idx += blockDim.x) {
    const int r = idx / k, j = idx % k;
    d.Y[(int64_t)r * d.n + f.first + j] = G[idx];
  }
}

// Backward, large supernode: g[u-block] = y - L21[:, u-block]^T x(rows) into W.
template <typename T>
__global__ void __launch_bounds__(256) k_bw_offdiag(SD<T> d, int64_t item_off) {
  const Item it = d.items[item_off + blockIdx.x];
  const SnInfo f = d.sn[it.s];
  const int k = f.k, m = f.m, nf = k + m, nrhs = d.nrhs;
  const int u0 = it.a, ub = min(kNB, k - u0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int32_t* urow = d.rowidx + f.rows_off + k;
  const T* Lp = d.L + f.Loff;
  for (int p = warp; p < ub * nrhs; p += nw) {
    const int r = p / ub, j = u0 + p % ub;
    const T* col = Lp + (int64_t)j * nf + k;
    const T* y = d.Y + (int64_t)r * d.n;
    T s = T(0);
    for (int i = lane; i < m; i += 32) s = fma(col[i], y[urow[i]], s);
    s = warp_sum(s);
    if (lane == 0) wfront(d, f, r)[j] = y[f.first + j] - s;
  }
}

// Backward, large supernode, block t: x_t = L_tt^{-T} g_t (warp per RHS).
template <typename T>
__global__ void __launch_bounds__(256) k_bw_diag(SD<T> d, int64_t item_off) {
  const Item it = d.items[item_off + blockIdx.x];
  const SnInfo f = d.sn[it.s];
  const int nf = f.k + f.m, nrhs = d.nrhs;
  const int c0 = it.t * kNB, b = min(kNB, f.k - c0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const T* Lp = d.L + f.Loff;
  for (int r = warp; r < nrhs; r += nw) {
    T* g = wfront(d, f, r) + c0;
    for (int j = b - 1; j >= 0; --j) {
      const T* col = Lp + (int64_t)(c0 + j) * nf + c0;
      T s = T(0);
      for (int i = j + 1 + lane; i < b; i += 32) s = fma(col[i], g[i], s);
      s = warp_sum(s);
      if (lane == 0) g[j] = (g[j] - s) / col[j];
      __syncwarp();
    }
    for (int i = lane; i < b; i += 32) d.Y[(int64_t)r * d.n + f.first + c0 + i] = g[i];
  }
}

// Backward, large supernode, block t: g[u-block] -= L[t-block, u-block]^T x_t.
template <typename T>
__global__ void __launch_bounds__(256) k_bw_upd(SD<T> d, int64_t item_off) {
  const Item it = d.items[item_off + blockIdx.x];
  const SnInfo f = d.sn[it.s];
  const int nf = f.k + f.m, nrhs = d.nrhs;
  const int c0 = it.t * kNB, b = min(kNB, f.k - c0);
  const int u0 = it.a, ub = min(kNB, c0 - u0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const T* Lp = d.L + f.Loff;
  for (int p = warp; p < ub * nrhs; p += nw) {
    const int r = p / ub, j = u0 + p % ub;
    const T* col = Lp + (int64_t)j * nf + c0;
    T* g = wfront(d, f, r);
    T s = T(0);
    for (int i = lane; i < b; i += 32) s = fma(col[i], g[c0 + i], s);
    s = warp_sum(s);
    if (lane == 0) g[j] -= s;
  }
}

// ---------------------------------------------------------------------------
// Permutations and FP64 residual kernels.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_perm_in(const double* B, int64_t ldb, const int32_t* perm, T* Y, int64_t n,
                          int nrhs, const double* inv_scale) {
  const int64_t total = n * nrhs;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / n);
    const int64_t i = idx % n;
    const double s = inv_scale ? inv_scale[r] : 1.0;
    Y[idx] = T(B[r * ldb + perm[i]] * s);
  }
}

template <typename T>
__global__ void k_perm_out(const T* Y, const int32_t* perm, double* X, int64_t ldx, int64_t n,
                           int nrhs, const double* scale, int accumulate) {
  const int64_t total = n * nrhs;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / n);
    const int64_t i = idx % n;
    const double v = (double)Y[idx] * (scale ? scale[r] : 1.0);
    double* dst = X + r * ldx + perm[i];
    if (accumulate) *dst += v; else *dst = v;
  }
}

// atomic max for non-negative doubles through their IEEE bit patterns
__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

// one warp per row: r = b - A x, plus max |r| and max |x| per RHS
__global__ void k_residual(const int64_t* rowptr, const int32_t* colind, const double* vals,
                           int64_t n, const double* B, int64_t ldb, const double* X, int64_t ldx,
                           double* R, int nrhs, double* rnorm, double* xnorm) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = wid; row < n; row += nwarps) {
    for (int r = 0; r < nrhs; ++r) {
      const double* x = X + r * ldx;
      double s = 0.0;
      for (int64_t p = rowptr[row] + lane; p < rowptr[row + 1]; p += 32) s = fma(vals[p], x[colind[p]], s);
      s = warp_sum(s);
      if (lane == 0) {
        const double res = B[r * ldb + row] - s;
        R[r * n + row] = res;
        atomic_max_nonneg(&rnorm[r], fabs(res));
        atomic_max_nonneg(&xnorm[r], fabs(x[row]));
      }
    }
  }
}

__global__ void k_norms(const int64_t* rowptr, const double* vals, int64_t n, const double* B,
                        int64_t ldb, int nrhs, double* out) {
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < n;
       row += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int64_t p = rowptr[row]; p < rowptr[row + 1]; ++p) s += fabs(vals[p]);
    atomic_max_nonneg(&out[0], s);
    for (int r = 0; r < nrhs; ++r) atomic_max_nonneg(&out[1 + r], fabs(B[r * ldb + row]));
  }
}

template <typename T>
cudaError_t init_t() {
  return cudaFuncSetAttribute(k_fw_small<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kSmallMax * kSolveChunk * (int)sizeof(T));
}

template <typename T>
cudaError_t launch_t(const Launch& L, const SolveArgs& a, cudaStream_t st) {
  const SD<T> d = make_sd<T>(a);
  const dim3 grid(L.count);
  switch (L.kind) {
    case K_FW_SMALL:
      k_fw_small<T><<<grid, 256, (size_t)L.param * a.nrhs * sizeof(T), st>>>(d, L.item_off);
      break;
    case K_FW_GATHER:
      k_fw_gather<T><<<grid, 256, 0, st>>>(d, L.item_off);
      break;
    case K_FW_DIAG:
      k_fw_diag<T><<<grid, 256, 0, st>>>(d, L.item_off);
      break;
    case K_FW_UPD:
      k_fw_upd<T><<<grid, kTrsmRows, 0, st>>>(d, L.item_off);
      break;
    case K_BW_SMALL:
      k_bw_small<T><<<grid, 256, (size_t)L.param * a.nrhs * sizeof(T), st>>>(d, L.item_off);
      break;
    case K_BW_OFFDIAG:
      k_bw_offdiag<T><<<grid, 256, 0, st>>>(d, L.item_off);
      break;
    case K_BW_DIAG:
      k_bw_diag<T><<<grid, 256, 0, st>>>(d, L.item_off);
      break;
    case K_BW_UPD:
      k_bw_upd<T><<<grid, 256, 0, st>>>(d, L.item_off);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

int grid_for(int64_t total) {
  int64_t g = (total + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t solve_kernels_init(int prec) {
  return prec == MF_FP32 ? init_t<float>() : init_t<double>();
}

cudaError_t launch_solve(int prec, const Launch& L, const SolveArgs& a, cudaStream_t st) {
  if (L.count <= 0) return cudaSuccess;
  return prec == MF_FP32 ? launch_t<float>(L, a, st) : launch_t<double>(L, a, st);
}

cudaError_t launch_perm_in(int prec, const double* B, int64_t ldb, const int32_t* perm, void* Y,
                           int64_t n, int32_t nrhs, const double* inv_scale, cudaStream_t st) {
  const int g = grid_for(n * nrhs);
  if (prec == MF_FP32)
    k_perm_in<float><<<g, 256, 0, st>>>(B, ldb, perm, static_cast<float*>(Y), n, nrhs, inv_scale);
  else
    k_perm_in<double><<<g, 256, 0, st>>>(B, ldb, perm, static_cast<double*>(Y), n, nrhs, inv_scale);
  return cudaGetLastError();
}

cudaError_t launch_perm_out(int prec, const void* Y, const int32_t* perm, double* X, int64_t ldx,
                            int64_t n, int32_t nrhs, const double* scale, int32_t accumulate,
                            cudaStream_t st) {
  const int g = grid_for(n * nrhs);
  if (prec == MF_FP32)
    k_perm_out<float><<<g, 256, 0, st>>>(static_cast<const float*>(Y), perm, X, ldx, n, nrhs, scale,
                                         accumulate);
  else
    k_perm_out<double><<<g, 256, 0, st>>>(static_cast<const double*>(Y), perm, X, ldx, n, nrhs,
                                          scale, accumulate);
  return cudaGetLastError();
}

cudaError_t launch_residual(const int64_t* rowptr, const int32_t* colind, const double* vals,
                            int64_t n, const double* B, int64_t ldb, const double* X, int64_t ldx,
                            double* R, int32_t nrhs, double* rnorm, double* xnorm,
                            cudaStream_t st) {
  int64_t g = (n * 32 + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  if (g < 1) g = 1;
  k_residual<<<(int)g, 256, 0, st>>>(rowptr, colind, vals, n, B, ldb, X, ldx, R, nrhs, rnorm, xnorm);
  return cudaGetLastError();
}

cudaError_t launch_norms(const int64_t* rowptr, const double* vals, int64_t n, const double* B,
                         int64_t ldb, int32_t nrhs, double* out, cudaStream_t st) {
  k_norms<<<grid_for(n), 256, 0, st>>>(rowptr, vals, n, B, ldb, nrhs, out);
  return cudaGetLastError();
}

}  // namespace mf
