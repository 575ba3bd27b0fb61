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

// Default bound of a flag wait: about kSpinLimit x 128 ns (0.5 s).
constexpr int kSpinLimit = 1 << 22;

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
  const int32_t* blkoff;
  const int64_t* ginv_ptr;
  const int64_t* ginv_src;
  const T* dinv;         // diagonal-block inverses (SpTRSV variant 2) or nullptr
  const int64_t* ioff;   // per front: first inverse slot, -1 if none
  const T* P;            // partitioned inverse (SpTRSV variants 3, 4) or nullptr
  const T* PT;           // variant 4: P transposed per front or nullptr
  const Item* v4grp;     // variant 4: forward row groups (front, front row)
  unsigned long long* status;  // the solve's timeout record (one word)
  // LU with pivoting (forward sweep): pivot position i of a front takes the
  // values of row (i & ~63) + piv[first + i]; nullptr elsewhere
  const uint8_t* piv;
  // LDL^T with symmetric pivoting, backward sweep: the solution of row r
  // sits at position ipos[r] (update rows are read through it); nullptr
  // elsewhere
  const int32_t* ipos;
  int64_t n;
  int nrhs;
  int wait_polls;  // polls before a flag wait gives up
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
  d.blkoff = a.sym.blkoff;
  d.ginv_ptr = a.sym.ginv_ptr;
  d.ginv_src = a.sym.ginv_src;
  d.dinv = static_cast<const T*>(a.dinv);
  d.ioff = a.sym.ioff;
  d.P = static_cast<const T*>(a.P);
  d.PT = static_cast<const T*>(a.PT);
  d.v4grp = a.sym.v4grp;
  d.status = a.status;
  d.piv = a.piv;
  d.ipos = a.ipos;
  d.n = a.n;
  d.nrhs = a.nrhs;
  d.wait_polls = a.wait_polls > 0 ? a.wait_polls : kSpinLimit;
  return d;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// The whole CTA waits until *flag != 0 (thread 0 polls with acquire loads,
// 128 ns apart); after `limit` polls it gives up, records MF_ERR_TIMEOUT in
// *status and lets the block continue (no hang).  Used by the wait probe of
// the diagnostics; the solve's chains poll value slots instead.

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void cta_wait(const int* flag, unsigned long long* status, int limit) {
  if (threadIdx.x == 0) {
    int spins = 0;
    while (ld_acquire(flag) == 0) {
      if (++spins > limit) {
        atomicExch(status, (unsigned long long)MF_ERR_TIMEOUT);
        break;
      }
      // the first polls back to back (a chain's next block usually arrives
      // within a few microseconds), then 128 ns apart
      if (spins > 64) __nanosleep(128);
    }
  }
  __syncthreads();
}

// Solved values of a pivot block reach the later blocks of the same front
// through the pivot rows' slots of the front work vector W (unused
// otherwise by the chained fronts), which the host fills with the
// all-ones bit pattern before each sweep: a NaN that IEEE arithmetic never
// returns (its NaNs are canonical).  The producer stores each value with a
// relaxed GPU-scope store; a consumer thread polls its slot with relaxed
// loads until the pattern is gone, so a hand-off costs the store's trip to
// L2 and one poll, not a release, an acquire and a reload of the values.
// A poll gives up after `limit` tries, records MF_ERR_TIMEOUT in *status
// and returns the pattern (the CTA goes on; no hang).
__device__ __forceinline__ void st_slot(double* p, double v) {
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(__double_as_longlong(v))
               : "memory");
}
__device__ __forceinline__ void st_slot(float* p, float v) {
  asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(__float_as_uint(v)) : "memory");
}
__device__ __forceinline__ bool ld_slot(const double* p, double* v) {
  long long b;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(b) : "l"(p) : "memory");
  *v = __longlong_as_double(b);
  return b != -1ll;
}
__device__ __forceinline__ bool ld_slot(const float* p, float* v) {
  unsigned b;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(b) : "l"(p) : "memory");
  *v = __uint_as_float(b);
  return b != 0xffffffffu;
}
template <typename T>
__device__ __forceinline__ T poll_slot(const T* p, unsigned long long* status, int limit) {
  T v;
  int spins = 0;
  while (!ld_slot(p, &v)) {
    if (++spins > limit) {
      atomicExch(status, (unsigned long long)MF_ERR_TIMEOUT);
      break;
    }
    if (spins > 64) __nanosleep(128);
  }
  return v;
}

// Row pitches of the per-RHS shared arrays: padded so that lanes stepping
// through rows do not hit the same bank (xs rows stay 16-byte aligned).
template <int R>
constexpr int xs_pitch() { return R == 1 ? 1 : R + 4; }
template <int R>
constexpr int red_pitch() { return R == 1 ? 1 : R + 1; }

// acc[r] += l * xq[r] for the R right-hand sides of one staged row; for
// R >= 4 the row (16-byte aligned, pitch xs_pitch) is read 16 bytes at a
// time.  Lanes beyond the caller's nrhs accumulate values that are never
// written out.
template <typename T, int R>
__device__ __forceinline__ void axpy_row(T (&acc)[R], T l, const T* xq) {
  if constexpr (R < 4) {
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = fma(l, xq[r], acc[r]);
  } else if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int r = 0; r < R; r += 4) {
      const float4 v = *reinterpret_cast<const float4*>(xq + r);
      acc[r] = fma(l, v.x, acc[r]);
      acc[r + 1] = fma(l, v.y, acc[r + 1]);
      acc[r + 2] = fma(l, v.z, acc[r + 2]);
      acc[r + 3] = fma(l, v.w, acc[r + 3]);
    }
  } else {
#pragma unroll
    for (int r = 0; r < R; r += 2) {
      const double2 v = *reinterpret_cast<const double2*>(xq + r);
      acc[r] = fma(l, v.x, acc[r]);
      acc[r + 1] = fma(l, v.y, acc[r + 1]);
    }
  }
}

template <typename T, int R>
constexpr size_t fw_level_smem() {
  return ((size_t)kNB * xs_pitch<R>() + (size_t)kNB * R + (size_t)4 * kNB * red_pitch<R>() +
          (size_t)kNB * (kNB + 1) + kNB) * sizeof(T);
}
template <typename T, int R>
constexpr size_t bw_level_smem() {
  return ((size_t)kNB * xs_pitch<R>() + (size_t)4 * kNB * red_pitch<R>() +
          (size_t)kNB * (kNB + 1) + kNB) * sizeof(T);
}

// ---------------------------------------------------------------------------
// Forward, one 64-row pivot block p of a large front (the update rows of
// the level run afterwards in k_fw_gemv).  The block gathers its rows of the
// front work vector, w = b(first..) + the children's update entries (inverse
// relative maps, children in fixed order), then
//   x_p = L_pp^{-1} (w_p - sum_{a<p} L_pa x_a),
// written to Y and to block p's slots; the values of earlier blocks are
// polled from their slots (st_slot / poll_slot).  Thread (row, g): row of the block, g = quarter of the
// 64 columns of L_pa.  The L values of block a+1 are loaded into registers
// while the block waits for x_a, so the DRAM latency is off the critical path.
// ---------------------------------------------------------------------------
template <typename T, int R>
__global__ void __launch_bounds__(256, 2)
    k_fw_level(SD<T> d, int64_t item_off, int* counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int RX = xs_pitch<R>(), RP = red_pitch<R>();
  T* xs = reinterpret_cast<T*>(smem_raw);  // xs[q * RX + r]
  T* ws = xs + kNB * RX;                   // ws[row * R + r]  gathered w
  T* red = ws + kNB * R;                   // red[(g * kNB + row) * RP + r]
  T* D = red + 4 * kNB * RP;               // D[c * (kNB + 1) + i] = L(r0 + i, r0 + c)
  T* rinv = D + kNB * (kNB + 1);
  constexpr int ld = kNB + 1;
  __shared__ int s_item;
  if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
  __syncthreads();
  const int nrhs = d.nrhs;
  const Item it = d.items[item_off + s_item];
  const SnInfo f = d.sn[it.s];
  const int k = f.k, nf = k + f.m;
  const int r0 = it.a, rows = it.b;
  const int tid = threadIdx.x, row = tid & 63, g = tid >> 6, lane = tid & 31, warp = tid >> 5;
  const T* Lp = d.L + f.Loff;
  const int nblk = r0 / kNB;  // earlier pivot blocks of the front
  // L values of block 0 (thread: column 16 g + qq of the block, its row)
  T Lc[16];
  const bool live = row < rows;
  {
    const int bs0 = min(kNB, k);
#pragma unroll
    for (int qq = 0; qq < 16; ++qq) {
      const int q = g * 16 + qq;
      Lc[qq] = (nblk > 0 && live && q < bs0) ? Lp[(int64_t)q * nf + r0 + row] : T(0);
    }
  }
  // pivot blocks: the inverse of the diagonal block when it was kept
  // (SpTRSV variant 2), else the diagonal block and the reciprocals of its
  // diagonal for the substitution
  const int64_t islot = d.dinv != nullptr ? d.ioff[it.s] : -1;
  if (islot >= 0) {
    T v[kNB * kNB / 256];
    const T* Q = d.dinv + (islot + r0 / kNB) * (int64_t)(kNB * kNB);
#pragma unroll
    for (int u = 0; u < kNB * kNB / 256; ++u) {
      const int idx = tid + u * 256, c = idx / kNB, i = idx % kNB;
      v[u] = (c < rows && i < rows) ? Q[idx] : T(0);
    }
#pragma unroll
    for (int u = 0; u < kNB * kNB / 256; ++u) {
      const int idx = tid + u * 256;
      D[(idx / kNB) * ld + (idx % kNB)] = v[u];
    }
  } else {
    // all global loads of the diagonal block in flight before the stores
    T v[kNB * kNB / 256];
    const T* P = Lp + (int64_t)r0 * nf + r0;
#pragma unroll
    for (int u = 0; u < kNB * kNB / 256; ++u) {
      const int idx = tid + u * 256, c = idx / kNB, i = idx % kNB;
      v[u] = (c < rows && i < rows && i >= c) ? P[(int64_t)c * nf + i] : T(0);
    }
#pragma unroll
    for (int u = 0; u < kNB * kNB / 256; ++u) {
      const int idx = tid + u * 256;
      D[(idx / kNB) * ld + (idx % kNB)] = v[u];
    }
    if (tid < rows) rinv[tid] = T(1) / P[(int64_t)tid * nf + tid];
  }
  // gather w for the rows of this block
  for (int idx = tid; idx < rows * nrhs; idx += blockDim.x) {
    const int rw = idx / nrhs, r = idx % nrhs;
    const int i0 = r0 + rw;
    const int i = (d.piv && i0 < k) ? r0 + (int)d.piv[f.first + i0] : i0;
    T w = i < k ? d.Y[(int64_t)r * d.n + f.first + i] : T(0);
    const int64_t gi = f.woff + i;
    for (int64_t e = d.ginv_ptr[gi]; e < d.ginv_ptr[gi + 1]; ++e)
      w += d.W[d.ginv_src[e] * nrhs + r];
    ws[rw * R + r] = w;
  }
  T acc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = T(0);
  for (int a = 0; a < nblk; ++a) {
    T Ln[16];
    const bool more = a + 1 < nblk;
    const int bsn = more ? min(kNB, k - (a + 1) * kNB) : 0;
#pragma unroll
    for (int qq = 0; qq < 16; ++qq) {
      const int q = g * 16 + qq;
      Ln[qq] = (more && live && q < bsn) ? Lp[(int64_t)((a + 1) * kNB + q) * nf + r0 + row] : T(0);
    }
    const int bsa = min(kNB, k - a * kNB);
    const T* sl = d.W + (f.woff + (int64_t)a * kNB) * nrhs;  // block a's slots
    for (int idx = tid; idx < bsa * nrhs; idx += blockDim.x) {
      const int r = idx / bsa, q = idx % bsa;
      xs[q * RX + r] = poll_slot(sl + (int64_t)q * nrhs + r, d.status, d.wait_polls);
    }
    __syncthreads();
#pragma unroll
    for (int qq = 0; qq < 16; ++qq) {
      const int q = g * 16 + qq;
      if (q < bsa) axpy_row<T, R>(acc, Lc[qq], xs + q * RX);
    }
    __syncthreads();
#pragma unroll
    for (int qq = 0; qq < 16; ++qq) Lc[qq] = Ln[qq];
  }
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (r < nrhs) red[(g * kNB + row) * RP + r] = acc[r];
  __syncthreads();
  for (int idx = tid; idx < rows * nrhs; idx += blockDim.x) {
    const int rw = idx / nrhs, r = idx % nrhs;
    const T sum = red[(0 * kNB + rw) * RP + r] + red[(1 * kNB + rw) * RP + r] +
                  red[(2 * kNB + rw) * RP + r] + red[(3 * kNB + rw) * RP + r];
    xs[rw * RX + r] = ws[rw * R + r] - sum;
  }
  __syncthreads();
  if (islot >= 0) {
    // x = L_pp^{-1} u: thread (row, g) sums 16 columns, four partial sums
    T a2[R];
#pragma unroll
    for (int r = 0; r < R; ++r) a2[r] = T(0);
#pragma unroll
    for (int qq = 0; qq < 16; ++qq) {
      const int c = g * 16 + qq;
      if (c < rows) axpy_row<T, R>(a2, D[c * ld + row], xs + c * RX);
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (r < nrhs) red[(g * kNB + row) * RP + r] = a2[r];
    __syncthreads();
    for (int idx = tid; idx < rows * nrhs; idx += blockDim.x) {
      const int rw = idx / nrhs, r = idx % nrhs;
      const T x = red[(0 * kNB + rw) * RP + r] + red[(1 * kNB + rw) * RP + r] +
                  red[(2 * kNB + rw) * RP + r] + red[(3 * kNB + rw) * RP + r];
      d.Y[(int64_t)r * d.n + f.first + r0 + rw] = x;
      st_slot(d.W + (f.woff + r0 + rw) * nrhs + r, x);
    }
    return;
  }
  // column-oriented substitution, one warp per right-hand side; lane owns
  // rows lane and lane + 32 of the block
  for (int r = warp; r < nrhs; r += 8) {
    T v0 = lane < rows ? xs[lane * RX + r] : T(0);
    T v1 = lane + 32 < rows ? xs[(lane + 32) * RX + r] : T(0);
    for (int j = 0; j < rows; ++j) {
      const T xj = __shfl_sync(0xffffffffu, j < 32 ? v0 : v1, j & 31) * rinv[j];
      if (j < 32) {
        if (lane == j) v0 = xj;
        else if (lane > j && lane < rows) v0 = fma(-D[j * ld + lane], xj, v0);
        if (lane + 32 < rows) v1 = fma(-D[j * ld + lane + 32], xj, v1);
      } else {
        if (lane + 32 == j) v1 = xj;
        else if (lane + 32 > j && lane + 32 < rows) v1 = fma(-D[j * ld + lane + 32], xj, v1);
      }
    }
    if (lane < rows) {
      d.Y[(int64_t)r * d.n + f.first + r0 + lane] = v0;
      st_slot(d.W + (f.woff + r0 + lane) * nrhs + r, v0);
    }
    if (lane + 32 < rows) {
      d.Y[(int64_t)r * d.n + f.first + r0 + lane + 32] = v1;
      st_slot(d.W + (f.woff + r0 + lane + 32) * nrhs + r, v1);
    }
  }
}

// ---------------------------------------------------------------------------
// Backward, one 64-column pivot block c of a large front:
//   x_c = L_cc^{-T} (y'_c - sum_{a>c} L_ac^T x_a),
// y' = y - L21[:, c]^T x(update rows), already formed by k_bw_gemv1 /
// k_bw_gemm; the values of later blocks are polled from their slots.  Thread (col, g)
// holds rows 16 g .. 16 g + 15 of its column of the current 64-row tile in
// registers; the next tile is loaded while the block waits.
// ---------------------------------------------------------------------------
template <typename T, int R>
__global__ void __launch_bounds__(256, 2)
    k_bw_level(SD<T> d, int64_t item_off, int* counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int ld = kNB + 1;
  constexpr int RX = xs_pitch<R>(), RP = red_pitch<R>();
  T* xs = reinterpret_cast<T*>(smem_raw);  // xs[i * RX + r]
  T* red = xs + kNB * RX;                  // red[(g * kNB + c) * RP + r]
  T* Dt = red + 4 * kNB * RP;              // Dt[j * ld + c] = L(c0 + j, c0 + c)
  T* rinv = Dt + kNB * ld;
  __shared__ int s_item;
  if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
  __syncthreads();
  const int nrhs = d.nrhs;
  const Item it = d.items[item_off + s_item];
  const SnInfo f = d.sn[it.s];
  const int k = f.k, nf = k + f.m;
  const int c0 = it.a, bs = it.b;
  const int tid = threadIdx.x, col = tid & 63, g = tid >> 6, lane = tid & 31, warp = tid >> 5;
  const T* Lp = d.L + f.Loff;
  const bool live = col < bs;
  const T* Lcol = Lp + (int64_t)(c0 + (live ? col : 0)) * nf;
  const int PB = (k + kNB - 1) / kNB;
  // tiles: the later pivot blocks of the front, last first (the update rows
  // were subtracted from y by k_bw_gemv1 / k_bw_gemm)
  const int ntiles = PB - 1 - c0 / kNB;
  T Lc[16];
  {
    int i0 = 0, ti = 0;
    if (ntiles > 0) {
      i0 = (PB - 1) * kNB;
      ti = min(kNB, k - i0);
    }
#pragma unroll
    for (int ii = 0; ii < 16; ++ii) {
      const int i = g * 16 + ii;
      Lc[ii] = (live && i < ti) ? Lcol[i0 + i] : T(0);
    }
  }
  // Dt[j * ld + c] = (j, c) entry of the diagonal block, or of its inverse
  // when that was kept (SpTRSV variant 2)
  const int64_t islot = d.dinv != nullptr ? d.ioff[it.s] : -1;
  {
    // all global loads of the diagonal block in flight before the stores
    T v[kNB * kNB / 256];
    const T* P = Lp + (int64_t)c0 * nf + c0;
    const T* Q = islot >= 0 ? d.dinv + (islot + c0 / kNB) * (int64_t)(kNB * kNB) : nullptr;
#pragma unroll
    for (int u = 0; u < kNB * kNB / 256; ++u) {
      const int idx = tid + u * 256, c = idx / kNB, j = idx % kNB;
      const bool in = c < bs && j < bs && j >= c;
      v[u] = in ? (Q ? Q[idx] : P[(int64_t)c * nf + j]) : T(0);
    }
#pragma unroll
    for (int u = 0; u < kNB * kNB / 256; ++u) {
      const int idx = tid + u * 256;
      Dt[(idx % kNB) * ld + idx / kNB] = v[u];
    }
    if (islot < 0 && tid < bs) rinv[tid] = T(1) / P[(int64_t)tid * nf + tid];
  }
  // the block's own y' (final before this launch) is loaded up front, off the
  // critical path of the chain
  constexpr int YP = (kNB * R + 255) / 256;
  T ypre[YP];
#pragma unroll
  for (int u = 0; u < YP; ++u) {
    const int idx = tid + 256 * u;
    ypre[u] = idx < bs * nrhs ? d.Y[(int64_t)(idx / bs) * d.n + f.first + c0 + idx % bs] : T(0);
  }
  T acc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = T(0);
  for (int tI = 0; tI < ntiles; ++tI) {
    const int i0 = (PB - 1 - tI) * kNB;
    const int ti = min(kNB, k - i0);
    T Ln[16];
    {
      int n0 = 0, nt = 0;
      if (tI + 1 < ntiles) {
        n0 = (PB - 2 - tI) * kNB;
        nt = min(kNB, k - n0);
      }
#pragma unroll
      for (int ii = 0; ii < 16; ++ii) {
        const int i = g * 16 + ii;
        Ln[ii] = (live && i < nt) ? Lcol[n0 + i] : T(0);
      }
    }
    const T* sl = d.W + (f.woff + i0) * nrhs;  // the later block's slots
    for (int idx = tid; idx < ti * nrhs; idx += blockDim.x) {
      const int i = idx % ti, r = idx / ti;
      xs[i * RX + r] = poll_slot(sl + (int64_t)i * nrhs + r, d.status, d.wait_polls);
    }
    __syncthreads();
#pragma unroll
    for (int ii = 0; ii < 16; ++ii) {
      const int i = g * 16 + ii;
      if (i < ti) axpy_row<T, R>(acc, Lc[ii], xs + i * RX);
    }
    __syncthreads();
#pragma unroll
    for (int ii = 0; ii < 16; ++ii) Lc[ii] = Ln[ii];
  }
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (r < nrhs) red[(g * kNB + col) * RP + r] = acc[r];
  __syncthreads();
#pragma unroll
  for (int u = 0; u < YP; ++u) {
    const int idx = tid + 256 * u;
    if (idx >= bs * nrhs) break;
    const int c = idx % bs, r = idx / bs;
    const T sum = red[(0 * kNB + c) * RP + r] + red[(1 * kNB + c) * RP + r] +
                  red[(2 * kNB + c) * RP + r] + red[(3 * kNB + c) * RP + r];
    xs[c * RX + r] = ypre[u] - sum;
  }
  __syncthreads();
  if (islot >= 0) {
    // x = L_cc^{-T} v: thread (col, g) sums rows 16 g .. 16 g + 15 of
    // column col of the inverse, four partial sums
    T a2[R];
#pragma unroll
    for (int r = 0; r < R; ++r) a2[r] = T(0);
#pragma unroll
    for (int qq = 0; qq < 16; ++qq) {
      const int j = g * 16 + qq;
      if (j < bs) axpy_row<T, R>(a2, Dt[j * ld + col], xs + j * RX);
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (r < nrhs) red[(g * kNB + col) * RP + r] = a2[r];
    __syncthreads();
    for (int idx = tid; idx < bs * nrhs; idx += blockDim.x) {
      const int c = idx / nrhs, r = idx % nrhs;
      const T x = red[(0 * kNB + c) * RP + r] + red[(1 * kNB + c) * RP + r] +
                  red[(2 * kNB + c) * RP + r] + red[(3 * kNB + c) * RP + r];
      d.Y[(int64_t)r * d.n + f.first + c0 + c] = x;
      st_slot(d.W + (f.woff + c0 + c) * nrhs + r, x);
    }
    return;
  }
  // right-looking substitution with L_cc^T, one warp per right-hand side;
  // lane owns columns lane and lane + 32 of the block
  for (int r = warp; r < nrhs; r += 8) {
    T v0 = lane < bs ? xs[lane * RX + r] : T(0);
    T v1 = lane + 32 < bs ? xs[(lane + 32) * RX + r] : T(0);
    for (int j = bs - 1; j >= 0; --j) {
      const T xj = __shfl_sync(0xffffffffu, j < 32 ? v0 : v1, j & 31) * rinv[j];
      if (j < 32) {
        if (lane == j) v0 = xj;
        else if (lane < j) v0 = fma(-Dt[j * ld + lane], xj, v0);
      } else {
        if (lane + 32 == j) v1 = xj;
        else if (lane + 32 < j) v1 = fma(-Dt[j * ld + lane + 32], xj, v1);
        v0 = fma(-Dt[j * ld + lane], xj, v0);
      }
    }
    if (lane < bs) {
      d.Y[(int64_t)r * d.n + f.first + c0 + lane] = v0;
      st_slot(d.W + (f.woff + c0 + lane) * nrhs + r, v0);
    }
    if (lane + 32 < bs) {
      d.Y[(int64_t)r * d.n + f.first + c0 + lane + 32] = v1;
      st_slot(d.W + (f.woff + c0 + lane + 32) * nrhs + r, v1);
    }
  }
}

// ---------------------------------------------------------------------------
// Streaming products of the large fronts, run after every pivot of the level
// (forward) or before any (backward), so they never wait.  Shared memory
// holds kGemvStage staged values plus the per-block partial sums.
// ---------------------------------------------------------------------------
constexpr int kGemvStage = 4096;

template <typename T, int R>
constexpr size_t gemv_smem() {
  return ((size_t)kGemvStage + (size_t)4 * kNB * R) * sizeof(T);
}

// Forward, one 64-row block of update rows of a front:
//   W(rows) = w(rows) - L21(rows, :) x1,
// x1 = the front's solved pivots (in Y), staged in chunks of kGemvStage / R
// columns.  Thread (row, g) takes columns g, g + 4, ...; a warp reads 32
// consecutive rows of one column.
template <typename T, int R>
__global__ void __launch_bounds__(256) k_fw_gemv(SD<T> d, int64_t item_off) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sx = reinterpret_cast<T*>(smem_raw);  // sx[j * R + r]
  T* red = sx + kGemvStage;                // red[(g * kNB + row) * R + r]
  constexpr int CH = kGemvStage / R;
  const Item it = d.items[item_off + blockIdx.x];
  const SnInfo f = d.sn[it.s];
  const int k = f.k, nf = k + f.m, nrhs = d.nrhs;
  const int r0 = it.a, rows = it.b;
  const int tid = threadIdx.x, row = tid & 63, g = tid >> 6;
  const bool live = row < rows;
  const T* Lr = d.L + f.Loff + r0 + (live ? row : 0);
  T acc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = T(0);
  for (int j0 = 0; j0 < k; j0 += CH) {
    const int cl = min(CH, k - j0);
    __syncthreads();
    for (int idx = tid; idx < cl * nrhs; idx += blockDim.x) {
      const int j = idx % cl, r = idx / cl;
      sx[j * R + r] = d.Y[(int64_t)r * d.n + f.first + j0 + j];
    }
    __syncthreads();
#pragma unroll 8
    for (int j = g; j < cl; j += 4) axpy_row<T, R>(acc, Lr[(int64_t)(j0 + j) * nf], sx + j * R);
  }
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (r < nrhs) red[(g * kNB + row) * R + r] = acc[r];
  __syncthreads();
  for (int idx = tid; idx < rows * nrhs; idx += blockDim.x) {
    const int rw = idx / nrhs, r = idx % nrhs;
    const int i = r0 + rw;
    T w = T(0);
    const int64_t gi = f.woff + i;
    for (int64_t e = d.ginv_ptr[gi]; e < d.ginv_ptr[gi + 1]; ++e)
      w += d.W[d.ginv_src[e] * nrhs + r];
    const T sum = red[(0 * kNB + rw) * R + r] + red[(1 * kNB + rw) * R + r] +
                  red[(2 * kNB + rw) * R + r] + red[(3 * kNB + rw) * R + r];
    d.W[gi * nrhs + r] = w - sum;
  }
}

// One right-hand side.  Launches whose fronts have at most kFwNarrowK pivot
// columns: one CTA per 64 update rows, thread (row, g) summing the columns
// j = g mod 4 of its row (a warp reads 32 consecutive rows of one column),
// U loads of L per thread in flight, one barrier to add the four partial
// sums; U = 2 (32 registers, eight CTAs per SM) when every front of the
// launch has at most 128 pivot columns, else 8.  Wider launches: four CTAs
// per item, CTA (item, sub) taking rows r0 + 16 sub .. + 16 and thread
// (row, g) the columns j = g mod 16, the 16 partial sums of a row added in
// a fixed order.  The threads that finish a row load its children's entry
// range before the product, so one round trip of the gather is off the
// critical path.
template <typename T, int U>
__global__ void __launch_bounds__(256, U == 2 ? 8 : 5) k_fw_gemv1r(SD<T> d, int64_t item_off) {
  __shared__ T red[4][kNB];
  const Item it = d.items[item_off + blockIdx.x];
  const SnInfo f = d.sn[it.s];
  const int k = f.k, nf = k + f.m;
  const int tid = threadIdx.x, row = tid & (kNB - 1), g = tid >> 6;
  const int rows = it.b, r0 = it.a;
  const int64_t gi = f.woff + r0 + tid;
  int64_t e0 = 0, e1 = 0;
  if (tid < rows) {
    e0 = d.ginv_ptr[gi];
    e1 = d.ginv_ptr[gi + 1];
  }
  const T* Lr = d.L + f.Loff + r0 + (row < rows ? row : 0);
  const T* yx = d.Y + f.first;  // the front's solved pivots
  T a[U];
#pragma unroll
  for (int u = 0; u < U; ++u) a[u] = T(0);
  int j = g;
  for (; j + 4 * (U - 1) < k; j += 4 * U) {
    T l[U];
#pragma unroll
    for (int u = 0; u < U; ++u) l[u] = Lr[(int64_t)(j + 4 * u) * nf];
#pragma unroll
    for (int u = 0; u < U; ++u) a[u] = fma(l[u], yx[j + 4 * u], a[u]);
  }
  for (; j < k; j += 4) a[0] = fma(Lr[(int64_t)j * nf], yx[j], a[0]);
#pragma unroll
  for (int w = 1; w < U; w *= 2)
#pragma unroll
    for (int u = 0; u < U; u += 2 * w) a[u] += a[u + w];
  red[g][row] = a[0];
  __syncthreads();
  if (tid < rows) {
    const T sum = (red[0][tid] + red[1][tid]) + (red[2][tid] + red[3][tid]);
    T w = T(0);
    for (int64_t e = e0; e < e1; ++e) w += d.W[d.ginv_src[e]];
    d.W[gi] = w - sum;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_fw_gemv1(SD<T> d, int64_t item_off) {
  __shared__ T red[16][17];
  const int sub = blockIdx.x & 3;
  const Item it = d.items[item_off + (blockIdx.x >> 2)];
  const int rows = min(16, it.b - 16 * sub);
  if (rows <= 0) return;  // whole CTA
  const SnInfo f = d.sn[it.s];
  const int k = f.k, nf = k + f.m;
  const int r0 = it.a + 16 * sub;
  const int tid = threadIdx.x, row = tid & 15, g = tid >> 4;
  const int64_t gi = f.woff + r0 + tid;
  int64_t e0 = 0, e1 = 0;
  if (tid < rows) {
    e0 = d.ginv_ptr[gi];
    e1 = d.ginv_ptr[gi + 1];
  }
  const bool live = row < rows;
  const T* Lr = d.L + f.Loff + r0 + (live ? row : 0);
  const T* yx = d.Y + f.first;  // the front's solved pivots
  // eight independent loads of L per thread in flight
  T a[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) a[u] = T(0);
  int j = g;
  for (; j + 112 < k; j += 128) {
    T l[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) l[u] = Lr[(int64_t)(j + 16 * u) * nf];
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] = fma(l[u], yx[j + 16 * u], a[u]);
  }
  for (; j < k; j += 16) a[0] = fma(Lr[(int64_t)j * nf], yx[j], a[0]);
  red[g][row] = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
  __syncthreads();
  if (tid < rows) {
    T sum = T(0);
#pragma unroll
    for (int q = 0; q < 16; ++q) sum += red[q][tid];
    T w = T(0);
    for (int64_t e = e0; e < e1; ++e) w += d.W[d.ginv_src[e]];
    d.W[gi] = w - sum;
  }
}

// Backward, one right-hand side: the P CTAs of a 64-column item (P = 1, 2,
// 4 or 8, chosen per launch by the largest number of update rows of its
// fronts, so that one warp reads at most about 512 of them) take 64 / P
// columns each.  Warp w of a CTA takes 8 of those columns (column group
// w mod G) and one of 8 / G row groups (w div G), G the number of 8-column
// groups the CTA's columns fill (a power of two up to 8 / P, so all eight
// warps of an item of two columns read its rows); a lane reads NR =
// 16 bytes / sizeof(T) rows per step (rows t + 32 u, u < NR, coalesced per
// column), so every thread has 128 bytes of L in flight (16 FP64 or 32 FP32
// loads) without spills at 80 registers (three CTAs per SM).  Each lane
// keeps 8 column sums; the warps' sums of a column are added over the row
// groups in a fixed order.  Levels whose fronts have few update rows thus run one CTA
// per item and many rows per CTA, which amortises the CTA's start-up and
// gather latency; levels with many update rows split the rows for
// parallelism.
template <typename T>
__global__ void __launch_bounds__(256, 3) k_bw_gemv1(SD<T> d, int64_t item_off, int per) {
  constexpr int NC = 8;                    // columns per warp
  constexpr int NR = 16 / (int)sizeof(T);  // rows per lane and step
  __shared__ T red[8][NC];
  const int sub = blockIdx.x % per;
  const Item it = d.items[item_off + blockIdx.x / per];
  const int ncta = kNB / per;  // columns of this CTA: 64, 32, 16 or 8
  if (ncta * sub >= it.b) return;  // whole CTA
  const SnInfo f = d.sn[it.s];
  const int k = f.k, m = f.m, nf = k + f.m;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // column groups: as many 8-column groups as the CTA's columns need (a
  // power of two up to 8 / P), the other warps split the rows further
  const int wc = min(ncta, it.b - ncta * sub);
  int ngrp = 1;
  while (ngrp * NC < wc) ngrp *= 2;
  const int nrg = 8 / ngrp;  // row groups
  const int cg = warp % ngrp, rg = warp / ngrp;
  const int cb = it.a + ncta * sub;  // first column of the CTA
  const int c0 = cb + NC * cg;       // first column of the warp
  const int nc = min(NC, it.a + it.b - c0);
  const T* Lb = d.L + f.Loff + (int64_t)c0 * nf + k;
  const int32_t* frow = d.rowidx + f.rows_off + k;
  T acc[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) acc[q] = T(0);
  if (nc > 0) {
    // the rows' global indices are loaded one step ahead, so a step waits
    // for one round trip (L and the gathered x together), not two
    const int step = nrg * 32 * NR;
    int32_t gn[NR];
#pragma unroll
    for (int u = 0; u < NR; ++u) {
      const int i = rg * 32 * NR + lane + 32 * u;
      gn[u] = frow[i < m ? i : 0];
    }
#pragma unroll 1
    for (int t = rg * 32 * NR + lane; t < m; t += step) {
      T xv[NR];
      T lv[NR][NC];
      int32_t gc[NR];
#pragma unroll
      for (int u = 0; u < NR; ++u) {
        gc[u] = gn[u];
        const int i = t + step + 32 * u;
        gn[u] = frow[i < m ? i : 0];
      }
#pragma unroll
      for (int u = 0; u < NR; ++u) {
        const int i = t + 32 * u;
        const bool ok = i < m;
        const T* p = Lb + (ok ? i : 0);
#pragma unroll
        for (int q = 0; q < NC; ++q, p += nf) lv[u][q] = (ok && q < nc) ? *p : T(0);
        xv[u] = ok ? d.Y[d.ipos ? d.ipos[gc[u]] : gc[u]] : T(0);
      }
#pragma unroll
      for (int u = 0; u < NR; ++u)
#pragma unroll
        for (int q = 0; q < NC; ++q) acc[q] = fma(lv[u][q], xv[u], acc[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    const T v = warp_sum(acc[q]);
    if (lane == 0) red[warp][q] = v;
  }
  __syncthreads();
  if (tid < wc) {
    const int g = tid / NC, q = tid % NC;
    T sum = T(0);
    for (int r = 0; r < nrg; ++r) sum += red[r * ngrp + g][q];
    d.Y[f.first + cb + tid] -= sum;
  }
}

// Backward update-row sums for several right-hand sides (R >= 8): the block
// [c0, c0 + bs) of a front takes Y(c0 + c, r) -= (L21^T X2)(c, r) as a small
// GEMM over chunks of kBwRows update rows.  The chunk of L21 is staged
// transposed in shared memory (coalesced loads, padded rows), the chunk of
// X2 row-major; thread (c, g) accumulates column c for the R / 4 consecutive
// right-hand sides of group g (16-byte shared reads, warp broadcasts).  The
// next chunk's global loads are in registers while the current one is used.
constexpr int kBwRows = 64;

template <typename T, int R>
constexpr size_t bw_gemm_smem() {
  return ((size_t)kNB * (kBwRows + 1) + (size_t)kBwRows * R) * sizeof(T);
}

// One chunk of rows [i0, i0 + kBwRows) of a column block, as registers: PL
// values of the P / L block (transposed staging) and PX of the right-hand
// side rows, then stored to shared memory after the previous chunk is done.
template <typename T, int R>
struct BwChunk {
  static constexpr int PL = kNB * kBwRows / 256;
  static constexpr int PX = kBwRows * R / 256;
  T pl[PL], px[PX];
  __device__ __forceinline__ void store(T* Ls, T* xs) const {
    constexpr int lds = kBwRows + 1;
#pragma unroll
    for (int u = 0; u < PL; ++u) {
      const int idx = threadIdx.x + u * 256;
      Ls[(idx / kBwRows) * lds + idx % kBwRows] = pl[u];
    }
#pragma unroll
    for (int u = 0; u < PX; ++u) {
      const int idx = threadIdx.x + u * 256;
      xs[(idx % kBwRows) * R + idx / kBwRows] = px[u];
    }
  }
};

template <typename T, int R>
__global__ void __launch_bounds__(256) k_bw_gemm(SD<T> d, int64_t item_off) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int lds = kBwRows + 1;
  constexpr int RG = R / 4;                 // right-hand sides per thread
  T* Ls = reinterpret_cast<T*>(smem_raw);   // Ls[c * lds + i] = L21(i0 + i, c0 + c)
  T* xs = Ls + kNB * lds;                   // xs[i * R + r] = X2(i0 + i, r)
  const Item it = d.items[item_off + blockIdx.x];
  const SnInfo f = d.sn[it.s];
  const int k = f.k, m = f.m, nf = k + m, nrhs = d.nrhs;
  const int c0 = it.a, bs = it.b;
  const int tid = threadIdx.x, c = tid & (kNB - 1), g = tid >> 6;
  const T* Lp = d.L + f.Loff;
  const int32_t* frow = d.rowidx + f.rows_off + k;
  BwChunk<T, R> nx;
  auto fetch = [&](int i0) {
    const int ch = min(kBwRows, m - i0);
#pragma unroll
    for (int u = 0; u < BwChunk<T, R>::PL; ++u) {
      const int idx = tid + u * 256, cc = idx / kBwRows, i = idx % kBwRows;
      nx.pl[u] = (cc < bs && i < ch) ? Lp[(int64_t)(c0 + cc) * nf + k + i0 + i] : T(0);
    }
#pragma unroll
    for (int u = 0; u < BwChunk<T, R>::PX; ++u) {
      const int idx = tid + u * 256, i = idx % kBwRows, r = idx / kBwRows;
      nx.px[u] = (i < ch && r < nrhs)
                     ? d.Y[(int64_t)r * d.n + (d.ipos ? d.ipos[frow[i0 + i]] : frow[i0 + i])]
                     : T(0);
    }
  };
  T acc[RG];
#pragma unroll
  for (int q = 0; q < RG; ++q) acc[q] = T(0);
  if (m > 0) fetch(0);
  for (int i0 = 0; i0 < m; i0 += kBwRows) {
    __syncthreads();
    nx.store(Ls, xs);
    __syncthreads();
    if (i0 + kBwRows < m) fetch(i0 + kBwRows);
#pragma unroll 4
    for (int i = 0; i < kBwRows; ++i) axpy_row<T, RG>(acc, Ls[c * lds + i], xs + i * R + g * RG);
  }
  if (c < bs) {
#pragma unroll
    for (int q = 0; q < RG; ++q) {
      const int r = g * RG + q;
      if (r < nrhs) d.Y[(int64_t)r * d.n + f.first + c0 + c] -= acc[q];
    }
  }
}

// ---------------------------------------------------------------------------
// SpTRSV variant 3 (Sec. 5, partitioned inverse).  For a large front,
// P = [L11^{-1}; -L21 L11^{-1}] (layout of L) turns the pivot solve and the
// update-row product into one product whose row (column) blocks are
// independent: no flags, no chains.  Forward: the pivot rows' gathered w is
// staged in the front's work vector (rows woff .. woff + k of W); then
// x = L11^{-1} w goes to Y and the update rows take w_u + (-L21 L11^{-1}) w.
// Backward: the pivot rows' forward result y is staged in W; then
// x_c = sum_i P(i, c) v_i with v = [y; x of the update rows].
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_fw_pgather(SD<T> d, int64_t item_off) {
  const Item it = d.items[item_off + blockIdx.x];
  const SnInfo f = d.sn[it.s];
  const int nrhs = d.nrhs;
  for (int idx = threadIdx.x; idx < it.b * nrhs; idx += blockDim.x) {
    const int rw = idx / nrhs, r = idx % nrhs;
    const int i = it.a + rw;
    const int64_t gi = f.woff + i;
    T w = d.Y[(int64_t)r * d.n + f.first + i];
    for (int64_t e = d.ginv_ptr[gi]; e < d.ginv_ptr[gi + 1]; ++e)
      w += d.W[d.ginv_src[e] * nrhs + r];
    d.W[gi * nrhs + r] = w;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_bw_pcopy(SD<T> d, int64_t item_off) {
  const Item it = d.items[item_off + blockIdx.x];
  const SnInfo f = d.sn[it.s];
  const int nrhs = d.nrhs;
  for (int idx = threadIdx.x; idx < it.b * nrhs; idx += blockDim.x) {
    const int rw = idx / nrhs, r = idx % nrhs;
    const int i = it.a + rw;
    d.W[(f.woff + i) * nrhs + r] = d.Y[(int64_t)r * d.n + f.first + i];
  }
}

// Forward product, one right-hand side, four CTAs of 16 rows per 64-row item
// (item field t: 0 pivot rows, 1 update rows); thread (row, g) sums the
// columns j = g (mod 16), the 16 partial sums of a row in a fixed order.
template <typename T>
__global__ void __launch_bounds__(256) k_fw_pinv1(SD<T> d, int64_t item_off) {
  __shared__ T red[16][17];
  const int sub = blockIdx.x & 3;
  const Item it = d.items[item_off + (blockIdx.x >> 2)];
  const int rows = min(16, it.b - 16 * sub);
  if (rows <= 0) return;  // whole CTA
  const SnInfo f = d.sn[it.s];
  const int k = f.k, nf = k + f.m;
  const int r0 = it.a + 16 * sub;
  const bool piv = it.t == 0;
  const int kend = piv ? r0 + rows : k;  // L11^{-1} is lower triangular
  const int tid = threadIdx.x, row = tid & 15, g = tid >> 4;
  const bool live = row < rows;
  const T* Pr = d.P + f.Loff + r0 + (live ? row : 0);
  const T* wv = d.W + f.woff;  // the pivot rows' gathered w
  T a0 = T(0), a1 = T(0);
  int j = g;
  for (; j + 16 < kend; j += 32) {
    a0 = fma(Pr[(int64_t)j * nf], wv[j], a0);
    a1 = fma(Pr[(int64_t)(j + 16) * nf], wv[j + 16], a1);
  }
  if (j < kend) a0 = fma(Pr[(int64_t)j * nf], wv[j], a0);
  red[g][row] = a0 + a1;
  __syncthreads();
  if (tid < rows) {
    T sum = T(0);
#pragma unroll
    for (int q = 0; q < 16; ++q) sum += red[q][tid];
    const int i = r0 + tid;
    if (piv) {
      d.Y[f.first + i] = sum;
    } else {
      const int64_t gi = f.woff + i;
      T w = T(0);
      for (int64_t e = d.ginv_ptr[gi]; e < d.ginv_ptr[gi + 1]; ++e) w += d.W[d.ginv_src[e]];
      d.W[gi] = w + sum;
    }
  }
}

// Forward product, several right-hand sides: w staged in chunks of
// kGemvStage / R columns, thread (row, g) takes columns g, g + 4, ...
template <typename T, int R>
__global__ void __launch_bounds__(256) k_fw_pinv(SD<T> d, int64_t item_off) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sx = reinterpret_cast<T*>(smem_raw);  // sx[j * R + r]
  T* red = sx + kGemvStage;                // red[(g * kNB + row) * R + r]
  constexpr int CH = kGemvStage / R;
  const Item it = d.items[item_off + blockIdx.x];
  const SnInfo f = d.sn[it.s];
  const int k = f.k, nf = k + f.m, nrhs = d.nrhs;
  const int r0 = it.a, rows = it.b;
  const bool piv = it.t == 0;
  const int kend = piv ? r0 + rows : k;
  const int tid = threadIdx.x, row = tid & 63, g = tid >> 6;
  const bool live = row < rows;
  const T* Pr = d.P + f.Loff + r0 + (live ? row : 0);
  T acc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = T(0);
  for (int j0 = 0; j0 < kend; j0 += CH) {
    const int cl = min(CH, kend - j0);
    __syncthreads();
    for (int idx = tid; idx < cl * nrhs; idx += blockDim.x) {
      const int j = idx / nrhs, r = idx % nrhs;
      sx[j * R + r] = d.W[(f.woff + j0 + j) * nrhs + r];
    }
    __syncthreads();
#pragma unroll 8
    for (int j = g; j < cl; j += 4) axpy_row<T, R>(acc, Pr[(int64_t)(j0 + j) * nf], sx + j * R);
  }
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (r < nrhs) red[(g * kNB + row) * R + r] = acc[r];
  __syncthreads();
  for (int idx = tid; idx < rows * nrhs; idx += blockDim.x) {
    const int rw = idx / nrhs, r = idx % nrhs;
    const int i = r0 + rw;
    const T sum = red[(0 * kNB + rw) * R + r] + red[(1 * kNB + rw) * R + r] +
                  red[(2 * kNB + rw) * R + r] + red[(3 * kNB + rw) * R + r];
    if (piv) {
      d.Y[(int64_t)r * d.n + f.first + i] = sum;
    } else {
      const int64_t gi = f.woff + i;
      T w = T(0);
      for (int64_t e = d.ginv_ptr[gi]; e < d.ginv_ptr[gi + 1]; ++e)
        w += d.W[d.ginv_src[e] * nrhs + r];
      d.W[gi * nrhs + r] = w + sum;
    }
  }
}

// Backward product, one right-hand side: CTA (item, sub) takes columns
// c0 + 16 sub .. + 16; its warps split the rows i >= those columns
// (coalesced), each lane keeps 16 column sums, warps added in a fixed order.
template <typename T>
__global__ void __launch_bounds__(256) k_bw_pinv1(SD<T> d, int64_t item_off) {
  __shared__ T red[8][16];
  const int sub = blockIdx.x & 3;
  const Item it = d.items[item_off + (blockIdx.x >> 2)];
  const int nc = min(16, it.b - 16 * sub);
  if (nc <= 0) return;  // whole CTA
  const SnInfo f = d.sn[it.s];
  const int k = f.k, nf = k + f.m;
  const int cb = it.a + 16 * sub;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const T* Pb = d.P + f.Loff + (int64_t)cb * nf;
  const int32_t* frow = d.rowidx + f.rows_off;
  T acc[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q] = T(0);
  for (int i = cb + warp * 32 + lane; i < nf; i += 256) {
    const T vi = i < k ? d.W[f.woff + i] : d.Y[frow[i]];
    T lv[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) lv[q] = q < nc ? Pb[(int64_t)q * nf + i] : T(0);
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = fma(lv[q], vi, acc[q]);
  }
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const T v = warp_sum(acc[q]);
    if (lane == 0) red[warp][q] = v;
  }
  __syncthreads();
  if (tid < nc) {
    T sum = T(0);
#pragma unroll
    for (int w = 0; w < 8; ++w) sum += red[w][tid];
    d.Y[f.first + cb + tid] = sum;
  }
}

// Backward product, R >= 8 right-hand sides: chunks of kBwRows rows from the
// block's first column down, staged transposed (P) and row-major (v), the
// next chunk prefetched into registers as in k_bw_gemm.
template <typename T, int R>
__global__ void __launch_bounds__(256) k_bw_pinv(SD<T> d, int64_t item_off) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int lds = kBwRows + 1;
  constexpr int RG = R / 4;
  T* Ls = reinterpret_cast<T*>(smem_raw);   // Ls[c * lds + i] = P(i0 + i, c0 + c)
  T* xs = Ls + kNB * lds;                   // xs[i * R + r] = v(i0 + i, r)
  const Item it = d.items[item_off + blockIdx.x];
  const SnInfo f = d.sn[it.s];
  const int k = f.k, nf = k + f.m, nrhs = d.nrhs;
  const int c0 = it.a, bs = it.b;
  const int tid = threadIdx.x, c = tid & (kNB - 1), g = tid >> 6;
  const T* Pp = d.P + f.Loff;
  const int32_t* frow = d.rowidx + f.rows_off;
  BwChunk<T, R> nx;
  auto fetch = [&](int i0) {
    const int ch = min(kBwRows, nf - i0);
#pragma unroll
    for (int u = 0; u < BwChunk<T, R>::PL; ++u) {
      const int idx = tid + u * 256, cc = idx / kBwRows, i = idx % kBwRows;
      nx.pl[u] = (cc < bs && i < ch) ? Pp[(int64_t)(c0 + cc) * nf + i0 + i] : T(0);
    }
#pragma unroll
    for (int u = 0; u < BwChunk<T, R>::PX; ++u) {
      const int idx = tid + u * 256, i = idx % kBwRows, r = idx / kBwRows;
      const int gi = i0 + i;
      T v = T(0);
      if (i < ch && r < nrhs)
        v = gi < k ? d.W[(f.woff + gi) * nrhs + r] : d.Y[(int64_t)r * d.n + frow[gi]];
      nx.px[u] = v;
    }
  };
  T acc[RG];
#pragma unroll
  for (int q = 0; q < RG; ++q) acc[q] = T(0);
  fetch(c0);
  for (int i0 = c0; i0 < nf; i0 += kBwRows) {
    __syncthreads();
    nx.store(Ls, xs);
    __syncthreads();
    if (i0 + kBwRows < nf) fetch(i0 + kBwRows);
#pragma unroll 4
    for (int i = 0; i < kBwRows; ++i) axpy_row<T, RG>(acc, Ls[c * lds + i], xs + i * R + g * RG);
  }
  if (c < bs) {
#pragma unroll
    for (int q = 0; q < RG; ++q) {
      const int r = g * RG + q;
      if (r < nrhs) d.Y[(int64_t)r * d.n + f.first + c0 + c] = acc[q];
    }
  }
}

// ---------------------------------------------------------------------------
// Fronts with k + m <= 64: one warp per front (8 per CTA), few registers so
// that many fronts are in flight.  Lane l owns front rows l and l + 32.  The
// work vector of front s lives in W[(woff_s + i) * nrhs + r].  Right-hand
// sides go in blocks of RB, so every column of L loaded serves RB of them.
// Forward: gather w, then for each pivot j: x_j = w_j / L_jj and
// w_i -= L_ij x_j below it (the next column is loaded while this one is used).
// ---------------------------------------------------------------------------
template <typename T, int RB>
__global__ void __launch_bounds__(256) k_fw_tiny(SD<T> d, int64_t item_off, int64_t count) {
  const int lane = threadIdx.x & 31;
  const int64_t w_id = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (w_id >= count) return;
  const SnInfo f = d.sn[d.items[item_off + w_id].s];
  const int k = f.k, nf = k + f.m, nrhs = d.nrhs;
  const T* Lp = d.L + f.Loff;
  const int i0 = lane, i1 = lane + 32;
  const T rd0 = i0 < k ? T(1) / Lp[(int64_t)i0 * nf + i0] : T(0);
  const T rd1 = i1 < k ? T(1) / Lp[(int64_t)i1 * nf + i1] : T(0);
  // LU with pivoting: pivot position i takes the values of row piv (one
  // 64-row block here)
  const int s0 = (d.piv && i0 < k) ? (int)d.piv[f.first + i0] : i0;
  const int s1 = (d.piv && i1 < k) ? (int)d.piv[f.first + i1] : i1;
  const int64_t g0 = f.woff + s0, g1 = f.woff + s1;
  const int64_t e00 = i0 < nf ? d.ginv_ptr[g0] : 0, e01 = i0 < nf ? d.ginv_ptr[g0 + 1] : 0;
  const int64_t e10 = i1 < nf ? d.ginv_ptr[g1] : 0, e11 = i1 < nf ? d.ginv_ptr[g1 + 1] : 0;
  // the first child's entry of both rows loads together; rows with more
  // children add the rest afterwards, in the same order
  const int64_t src0 = e00 < e01 ? d.ginv_src[e00] : -1, src1 = e10 < e11 ? d.ginv_src[e10] : -1;
  for (int rb = 0; rb < nrhs; rb += RB) {
    T w0[RB], w1[RB];
#pragma unroll
    for (int q = 0; q < RB; ++q) {
      const int r = rb + q;
      T v0 = T(0), v1 = T(0);
      if (r < nrhs) {
        if (i0 < k) v0 = d.Y[(int64_t)r * d.n + f.first + s0];
        if (i1 < k) v1 = d.Y[(int64_t)r * d.n + f.first + s1];
        if (src0 >= 0) v0 += d.W[src0 * nrhs + r];
        if (src1 >= 0) v1 += d.W[src1 * nrhs + r];
        for (int64_t e = e00 + 1; e < e01; ++e) v0 += d.W[d.ginv_src[e] * nrhs + r];
        for (int64_t e = e10 + 1; e < e11; ++e) v1 += d.W[d.ginv_src[e] * nrhs + r];
      }
      w0[q] = v0;
      w1[q] = v1;
    }
    T c0 = i0 < nf ? Lp[i0] : T(0), c1 = i1 < nf ? Lp[i1] : T(0);
    for (int j = 0; j < k; ++j) {
      T n0 = T(0), n1 = T(0);
      if (j + 1 < k) {
        const T* nc = Lp + (int64_t)(j + 1) * nf;
        n0 = i0 < nf ? nc[i0] : T(0);
        n1 = i1 < nf ? nc[i1] : T(0);
      }
      const T rj = __shfl_sync(0xffffffffu, j < 32 ? rd0 : rd1, j & 31);
#pragma unroll
      for (int q = 0; q < RB; ++q) {
        const T xj = __shfl_sync(0xffffffffu, j < 32 ? w0[q] : w1[q], j & 31) * rj;
        if (i0 == j) w0[q] = xj;
        else if (i0 > j) w0[q] = fma(-c0, xj, w0[q]);
        if (i1 == j) w1[q] = xj;
        else if (i1 > j) w1[q] = fma(-c1, xj, w1[q]);
      }
      c0 = n0;
      c1 = n1;
    }
#pragma unroll
    for (int q = 0; q < RB; ++q) {
      const int r = rb + q;
      if (r >= nrhs) break;
      if (i0 < k) d.Y[(int64_t)r * d.n + f.first + i0] = w0[q];
      else if (i0 < nf) d.W[(f.woff + i0) * nrhs + r] = w0[q];
      if (i1 < k) d.Y[(int64_t)r * d.n + f.first + i1] = w1[q];
      else if (i1 < nf) d.W[(f.woff + i1) * nrhs + r] = w1[q];
    }
  }
}

// Backward, one warp per front with k + m <= 64: for j = k-1 .. 0,
//   x_j = (y_j - sum_{i > j} L_ij x_i) / L_jj,
// x_i being the ancestors' final values for the update rows and the values
// just solved for the pivot rows; one warp reduction per column and RHS.
template <typename T, int RB>
__global__ void __launch_bounds__(256) k_bw_tiny(SD<T> d, int64_t item_off, int64_t count) {
  const int lane = threadIdx.x & 31;
  const int64_t w_id = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (w_id >= count) return;
  const SnInfo f = d.sn[d.items[item_off + w_id].s];
  const int k = f.k, nf = k + f.m, nrhs = d.nrhs;
  const T* Lp = d.L + f.Loff;
  const int32_t* frow = d.rowidx + f.rows_off;
  const int i0 = lane, i1 = lane + 32;
  const T rd0 = i0 < k ? T(1) / Lp[(int64_t)i0 * nf + i0] : T(0);
  const T rd1 = i1 < k ? T(1) / Lp[(int64_t)i1 * nf + i1] : T(0);
  int32_t fr0 = (i0 >= k && i0 < nf) ? frow[i0] : 0;
  int32_t fr1 = (i1 >= k && i1 < nf) ? frow[i1] : 0;
  if (d.ipos) {  // LDL^T with symmetric pivoting: where those rows' solution sits
    fr0 = (i0 >= k && i0 < nf) ? d.ipos[fr0] : 0;
    fr1 = (i1 >= k && i1 < nf) ? d.ipos[fr1] : 0;
  }
  for (int rb = 0; rb < nrhs; rb += RB) {
    T x0[RB], x1[RB], y0[RB], y1[RB];
#pragma unroll
    for (int q = 0; q < RB; ++q) {
      const int r = rb + q;
      const T* yr = d.Y + (int64_t)(r < nrhs ? r : 0) * d.n;
      const bool live = r < nrhs;
      x0[q] = (live && i0 >= k && i0 < nf) ? yr[fr0] : T(0);
      x1[q] = (live && i1 >= k && i1 < nf) ? yr[fr1] : T(0);
      y0[q] = (live && i0 < k) ? yr[f.first + i0] : T(0);
      y1[q] = (live && i1 < k) ? yr[f.first + i1] : T(0);
    }
    T c0 = T(0), c1 = T(0);
    if (k > 0) {
      const T* col = Lp + (int64_t)(k - 1) * nf;
      c0 = i0 < nf ? col[i0] : T(0);
      c1 = i1 < nf ? col[i1] : T(0);
    }
    for (int j = k - 1; j >= 0; --j) {
      T n0 = T(0), n1 = T(0);
      if (j > 0) {
        const T* nc = Lp + (int64_t)(j - 1) * nf;
        n0 = i0 < nf ? nc[i0] : T(0);
        n1 = i1 < nf ? nc[i1] : T(0);
      }
      const T rj = __shfl_sync(0xffffffffu, j < 32 ? rd0 : rd1, j & 31);
#pragma unroll
      for (int q = 0; q < RB; ++q) {
        T p = (i0 > j ? c0 * x0[q] : T(0)) + (i1 > j ? c1 * x1[q] : T(0));
        p = warp_sum(p);
        const T yj = __shfl_sync(0xffffffffu, j < 32 ? y0[q] : y1[q], j & 31);
        const T xj = (yj - p) * rj;
        if (i0 == j) x0[q] = xj;
        if (i1 == j) x1[q] = xj;
      }
      c0 = n0;
      c1 = n1;
    }
#pragma unroll
    for (int q = 0; q < RB; ++q) {
      const int r = rb + q;
      if (r >= nrhs) break;
      if (i0 < k) d.Y[(int64_t)r * d.n + f.first + i0] = x0[q];
      if (i1 < k) d.Y[(int64_t)r * d.n + f.first + i1] = x1[q];
    }
  }
}

// ---------------------------------------------------------------------------
// Fronts with 64 < k + m <= 32 H: one warp per front (8 per CTA), no flags;
// the front's work vectors for RB right-hand sides are staged in shared
// memory (ws[i * RB + q]).  Forward, per block of 32 pivots [jb, jb + 32):
// the 32 x 32 triangle is solved in registers (lane l owns row jb + l, one
// shuffle per pivot and RHS, the RB solves interleaved), then the rows below
// take w_i -= sum_jj L(i, jb + jj) x_jj with all loads of a row issued
// together and each L value used for the RB right-hand sides.  Rows of
// earlier blocks are not read again.
// ---------------------------------------------------------------------------
template <typename T, int H, int RB>
__global__ void __launch_bounds__(256, 2) k_fw_warp(SD<T> d, int64_t item_off, int64_t count) {
  static_assert(H % 4 == 0, "rows per lane are gathered four at a time");
  constexpr int LB = sizeof(T) == 8 ? 16 : 32;  // L loads issued together
  __shared__ __align__(16) T ws_all[8 * 32 * H * RB];
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  const int64_t w_id = (int64_t)blockIdx.x * 8 + wq;
  if (w_id >= count) return;
  T* ws = ws_all + wq * 32 * H * RB;
  const SnInfo f = d.sn[d.items[item_off + w_id].s];
  const int k = f.k, nf = k + f.m, nrhs = d.nrhs;
  const T* Lp = d.L + f.Loff;
  for (int rb = 0; rb < nrhs; rb += RB) {
    __syncwarp();
    // four rows per lane at a time: their entry ranges, then their first
    // children's entries, then those values load together (rows with more
    // children add the rest afterwards, in the same order)
#pragma unroll 1
    for (int h0 = 0; h0 < H; h0 += 4) {
      int64_t e0[4], e1[4], src[4];
      int si[4];  // LU with pivoting: the row whose values pivot position i takes
#pragma unroll
      for (int hh = 0; hh < 4; ++hh) {
        const int i = lane + 32 * (h0 + hh);
        si[hh] = (d.piv && i < k) ? (i & ~(kNB - 1)) + (int)d.piv[f.first + i] : i;
        e0[hh] = i < nf ? d.ginv_ptr[f.woff + si[hh]] : 0;
        e1[hh] = i < nf ? d.ginv_ptr[f.woff + si[hh] + 1] : 0;
      }
#pragma unroll
      for (int hh = 0; hh < 4; ++hh) src[hh] = e0[hh] < e1[hh] ? d.ginv_src[e0[hh]] : -1;
#pragma unroll
      for (int q = 0; q < RB; ++q) {
        const int r = rb + q;
        T v[4];
#pragma unroll
        for (int hh = 0; hh < 4; ++hh) {
          const int i = lane + 32 * (h0 + hh);
          v[hh] = (r < nrhs && i < k) ? d.Y[(int64_t)r * d.n + f.first + si[hh]] : T(0);
        }
#pragma unroll
        for (int hh = 0; hh < 4; ++hh)
          if (r < nrhs && src[hh] >= 0) v[hh] += d.W[src[hh] * nrhs + r];
#pragma unroll
        for (int hh = 0; hh < 4; ++hh) {
          const int i = lane + 32 * (h0 + hh);
          if (r < nrhs)
            for (int64_t e = e0[hh] + 1; e < e1[hh]; ++e) v[hh] += d.W[d.ginv_src[e] * nrhs + r];
          ws[i * RB + q] = v[hh];
        }
      }
    }
    __syncwarp();
    for (int jb = 0; jb < k; jb += 32) {
      const int bc = min(32, k - jb);
      // rows jb + lane of columns jb .. jb + bc (indices clamped into the
      // front so every load is valid and all of them issue together)
      const int ir = min(jb + lane, nf - 1);
      T dl[32];
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) dl[jj] = Lp[(int64_t)(jb + min(jj, bc - 1)) * nf + ir];
      const int id = jb + min(lane, bc - 1);
      const T rdb = lane < bc ? T(1) / Lp[(int64_t)id * nf + id] : T(0);
      T v[RB];
#pragma unroll
      for (int q = 0; q < RB; ++q) v[q] = ws[(jb + lane) * RB + q];
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) {
        if (jj < bc) {
#pragma unroll
          for (int q = 0; q < RB; ++q) {
            const T xj = __shfl_sync(0xffffffffu, v[q] * rdb, jj);
            if (lane == jj) v[q] = xj;
            else if (lane > jj) v[q] = fma(-dl[jj], xj, v[q]);
          }
        }
      }
      if (jb + lane < nf) {
#pragma unroll
        for (int q = 0; q < RB; ++q) ws[(jb + lane) * RB + q] = v[q];
      }
      __syncwarp();
      // later rows: w_i -= sum_jj L(i, jb + jj) x_jj (x_jj = ws[jb + jj])
      for (int i = jb + 32 + lane; i < nf + lane; i += 32) {
        const int ic = min(i, nf - 1);
        T u[RB];
#pragma unroll
        for (int q = 0; q < RB; ++q) u[q] = ws[ic * RB + q];
#pragma unroll
        for (int q0 = 0; q0 < 32; q0 += LB) {
          T lv[LB];
#pragma unroll
          for (int q = 0; q < LB; ++q) lv[q] = Lp[(int64_t)(jb + min(q0 + q, bc - 1)) * nf + ic];
#pragma unroll
          for (int q = 0; q < LB; ++q)
            if (q0 + q < bc) axpy_row<T, RB>(u, -lv[q], ws + (jb + q0 + q) * RB);
        }
        if (i < nf) {
#pragma unroll
          for (int q = 0; q < RB; ++q) ws[i * RB + q] = u[q];
        }
      }
      __syncwarp();
    }
#pragma unroll
    for (int h = 0; h < H; ++h) {
      const int i = lane + 32 * h;
#pragma unroll
      for (int q = 0; q < RB; ++q) {
        const int r = rb + q;
        if (r >= nrhs) break;
        if (i < k) d.Y[(int64_t)r * d.n + f.first + i] = ws[i * RB + q];
        else if (i < nf) d.W[(f.woff + i) * nrhs + r] = ws[i * RB + q];
      }
    }
  }
}

// Sum over the warp of 32 per-lane vectors: lane l returns sum_lanes p[l].
// Five halving exchange steps (31 shuffles) instead of 32 reductions.
template <typename T>
__device__ __forceinline__ T transpose_sum32(T (&p)[32], int lane) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const bool hi = (lane & o) != 0;
#pragma unroll
    for (int jj = 0; jj < o; ++jj) {
      const T send = hi ? p[jj] : p[jj + o];
      const T keep = hi ? p[jj + o] : p[jj];
      p[jj] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return p[0];
}

// Sum over the warp of 32 per-lane vectors of 16 values: lane l returns
// sum_lanes p[l mod 16].  One exchange across the half-warps, then four
// halving steps within each half (31 shuffles).
template <typename T>
__device__ __forceinline__ T transpose_sum16(T (&p)[16], int lane) {
#pragma unroll
  for (int jj = 0; jj < 16; ++jj) p[jj] += __shfl_xor_sync(0xffffffffu, p[jj], 16);
#pragma unroll
  for (int o = 8; o >= 1; o >>= 1) {
    const bool hi = (lane & o) != 0;
#pragma unroll
    for (int jj = 0; jj < o; ++jj) {
      const T send = hi ? p[jj] : p[jj + o];
      const T keep = hi ? p[jj + o] : p[jj];
      p[jj] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return p[0];
}

// Backward, one warp per front, pivot columns in blocks of 32 from the last:
//   x_j = (y_j - sum_{i > j} L_ij x_i) / L_jj.
// x of the update rows (ancestors' final values) and of solved pivot rows
// sit in shared memory.  For block [j0, j0 + 32): lanes own rows to form the
// sums over rows i >= j0 + 32 (coalesced L reads), a transposed reduction
// hands column j0 + l's sum to lane l, and the triangle of the diagonal
// block is solved with lane l owning column j0 + l (one shuffle per pivot).
// ---------------------------------------------------------------------------
// Three CTAs per SM without spills.
template <typename T, int H>
__global__ void __launch_bounds__(256, 3) k_bw_warp(SD<T> d, int64_t item_off, int64_t count) {
  constexpr int LB = sizeof(T) == 8 ? 16 : 32;
  __shared__ T xs_all[8 * 32 * H];
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  const int64_t w_id = (int64_t)blockIdx.x * 8 + wq;
  if (w_id >= count) return;
  T* xs = xs_all + wq * 32 * H;
  const SnInfo f = d.sn[d.items[item_off + w_id].s];
  const int k = f.k, nf = k + f.m, nrhs = d.nrhs;
  const T* Lp = d.L + f.Loff;
  const int32_t* frow = d.rowidx + f.rows_off;
  for (int r = 0; r < nrhs; ++r) {
    const T* yr = d.Y + (int64_t)r * d.n;
    __syncwarp();
#pragma unroll
    for (int h = 0; h < H; ++h) {
      const int i = lane + 32 * h;
      if (i >= k && i < nf) xs[i] = yr[d.ipos ? d.ipos[frow[i]] : frow[i]];
    }
    __syncwarp();
    for (int b = (k - 1) >> 5; b >= 0; --b) {
      const int j0 = 32 * b, bc = min(32, k - j0);
      T acc;
      if constexpr (sizeof(T) == 8) {
        // FP64: two passes of 16 columns (16 sums and 16 loads per lane at
        // a time), so the kernel fits three CTAs per SM; the loads and round
        // trips per front are those of one pass over 32 columns
        T part[2];
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
          T p[16];
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) p[jj] = T(0);
          if (16 * hf < bc) {  // the same for the whole warp
            for (int i = j0 + bc + lane; i < nf; i += 32) {
              const T xi = xs[i];
              T lv[16];
#pragma unroll
              for (int q = 0; q < 16; ++q)
                lv[q] = Lp[(int64_t)(j0 + min(16 * hf + q, bc - 1)) * nf + i];
#pragma unroll
              for (int q = 0; q < 16; ++q) p[q] = fma(lv[q], xi, p[q]);
            }
          }
          part[hf] = transpose_sum16(p, lane);
        }
        acc = lane < 16 ? part[0] : part[1];
      } else {
        T p[32];
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) p[jj] = T(0);
        for (int i = j0 + bc + lane; i < nf; i += 32) {
          const T xi = xs[i];
#pragma unroll
          for (int q0 = 0; q0 < 32; q0 += LB) {
            T lv[LB];
#pragma unroll
            for (int q = 0; q < LB; ++q) lv[q] = Lp[(int64_t)(j0 + min(q0 + q, bc - 1)) * nf + i];
#pragma unroll
            for (int q = 0; q < LB; ++q) p[q0 + q] = fma(lv[q], xi, p[q0 + q]);
          }
        }
        acc = transpose_sum32(p, lane);
      }
      const bool own = lane < bc;
      const int j = j0 + min(lane, bc - 1);
      const T yv = own ? yr[f.first + j] : T(0);
      const T rinv = own ? T(1) / Lp[(int64_t)j * nf + j] : T(0);
      T xj = T(0);
      // the triangle of the diagonal block, rows from the last, in halves of
      // 16 (lane: its column j, rows j0 + ii with ii > lane)
#pragma unroll
      for (int h0 = 16; h0 >= 0; h0 -= 16) {
        T lc[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) lc[q] = Lp[(int64_t)j * nf + j0 + min(h0 + q, bc - 1)];
#pragma unroll
        for (int q = 0; q < 16; ++q)
          if (!(own && h0 + q > lane && h0 + q < bc)) lc[q] = T(0);
#pragma unroll
        for (int q = 15; q >= 0; --q) {
          const int ii = h0 + q;
          if (ii < bc) {
            const T xi = __shfl_sync(0xffffffffu, (yv - acc) * rinv, ii);
            if (lane == ii) xj = xi;
            acc = fma(lc[q], xi, acc);
          }
        }
      }
      if (own) {
        xs[j] = xj;
        d.Y[(int64_t)r * d.n + f.first + j] = xj;
      }
      __syncwarp();
    }
  }
}

// ---------------------------------------------------------------------------
// SpTRSV variant 4 (Sec. 5): one sparse product per level and sweep with the
// level's partitioned inverse, on the permuted global vectors: Y holds the
// right-hand side and receives the forward additions, then the solution;
// F (the first n x nrhs values of W) the forward results of the pivot rows.
// Nothing waits: a level reads only rows that earlier levels finished.
// Forward, one warp per row of the level's matrix (item: row, first group,
// end group, pivot?): sum over its groups (front s, front row i) of row i of
// P_s (contiguous in PT) times y at the front's pivot columns; a pivot row
// stores the sum in F, an update row adds it to Y.
// ---------------------------------------------------------------------------
template <typename T, int R>
__device__ __forceinline__ void warp_reduce_r(T (&acc)[R]) {
#pragma unroll
  for (int rr = 0; rr < R; ++rr) acc[rr] = warp_sum(acc[rr]);
}

template <typename T, int R>
__global__ void __launch_bounds__(256) k_v4_fw(SD<T> d, int64_t item_off, int count) {
  const int w = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (w >= count) return;
  const Item it = d.items[item_off + w];
  const int nr = d.nrhs;
  T acc[R];
#pragma unroll
  for (int rr = 0; rr < R; ++rr) acc[rr] = T(0);
  for (int g = it.t; g < it.a; ++g) {
    const Item gr = d.v4grp[g];
    const SnInfo f = d.sn[gr.s];
    const int len = gr.t < f.k ? gr.t + 1 : f.k;
    const T* pv = d.PT + f.Loff + (int64_t)gr.t * f.k;
    const T* y = d.Y + f.first;
    // four independent loads per lane in flight (rows of the top fronts
    // hold thousands of values)
    int c = lane;
    for (; c + 96 < len; c += 128) {
      const T v0 = pv[c], v1 = pv[c + 32], v2 = pv[c + 64], v3 = pv[c + 96];
#pragma unroll
      for (int rr = 0; rr < R; ++rr)
        if (rr < nr) {
          const T* yr = y + (int64_t)rr * d.n;
          acc[rr] = fma(v0, yr[c], acc[rr]);
          acc[rr] = fma(v1, yr[c + 32], acc[rr]);
          acc[rr] = fma(v2, yr[c + 64], acc[rr]);
          acc[rr] = fma(v3, yr[c + 96], acc[rr]);
        }
    }
    for (; c < len; c += 32) {
      const T v = pv[c];
#pragma unroll
      for (int rr = 0; rr < R; ++rr)
        if (rr < nr) acc[rr] = fma(v, y[c + (int64_t)rr * d.n], acc[rr]);
    }
  }
  warp_reduce_r<T, R>(acc);
  if (lane == 0) {
    const int64_t r = it.s;
#pragma unroll
    for (int rr = 0; rr < R; ++rr)
      if (rr < nr) {
        if (it.b) d.W[r + rr * d.n] = acc[rr];
        else d.Y[r + rr * d.n] += acc[rr];
      }
  }
}

// Backward, one warp per pivot column c of a front s of the level (item:
// s, c): x(first_s + c) = sum over the front rows i >= c of P_s(i, c) times
// F (pivot rows) or the final x (update rows, finished by earlier levels).
template <typename T, int R>
__global__ void __launch_bounds__(256) k_v4_bw(SD<T> d, int64_t item_off, int count) {
  const int w = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (w >= count) return;
  const Item it = d.items[item_off + w];
  const SnInfo f = d.sn[it.s];
  const int c = it.t, k = f.k, nf = k + f.m, nr = d.nrhs;
  const T* pc = d.P + f.Loff + (int64_t)c * nf;
  const int32_t* rows = d.rowidx + f.rows_off;
  T acc[R];
#pragma unroll
  for (int rr = 0; rr < R; ++rr) acc[rr] = T(0);
  int i = c + lane;
  for (; i + 96 < nf; i += 128) {  // four independent loads per lane in flight
    T v[4];
    const T* src[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int q = i + 32 * u;
      v[u] = pc[q];
      src[u] = q < k ? d.W + f.first + q : d.Y + rows[q];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int rr = 0; rr < R; ++rr)
        if (rr < nr) acc[rr] = fma(v[u], src[u][(int64_t)rr * d.n], acc[rr]);
  }
  for (; i < nf; i += 32) {
    const T v = pc[i];
    const T* src = i < k ? d.W + f.first + i : d.Y + rows[i];
#pragma unroll
    for (int rr = 0; rr < R; ++rr)
      if (rr < nr) acc[rr] = fma(v, src[(int64_t)rr * d.n], acc[rr]);
  }
  warp_reduce_r<T, R>(acc);
  if (lane == 0) {
#pragma unroll
    for (int rr = 0; rr < R; ++rr)
      if (rr < nr) d.Y[f.first + c + (int64_t)rr * d.n] = acc[rr];
  }
}

template <typename T, int R>
void launch_v4(const Launch& L, const SolveArgs& a, cudaStream_t st) {
  const SD<T> d = make_sd<T>(a);
  const int blocks = (int)((L.count + 7) / 8);
  if (L.kind == K_V4_FW) k_v4_fw<T, R><<<blocks, 256, 0, st>>>(d, L.item_off, L.count);
  else k_v4_bw<T, R><<<blocks, 256, 0, st>>>(d, L.item_off, L.count);
}

// Diagnostic: the solve's bounded wait on a flag that nothing sets.  Gives
// up after `limit` polls and records MF_ERR_TIMEOUT in *status.
__global__ void k_wait_probe(const int* flag, unsigned long long* status, int limit) {
  cta_wait(flag, status, limit);
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
__global__ void k_perm_out(const T* Y, const int32_t* perm, const int32_t* ipos, double* X,
                           int64_t ldx, int64_t n, int nrhs, const double* scale, int accumulate) {
  const int64_t total = n * nrhs;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / n);
    const int64_t i = idx % n;
    const int64_t src = ipos ? (int64_t)r * n + ipos[i] : idx;
    const double v = (double)Y[src] * (scale ? scale[r] : 1.0);
    double* dst = X + r * ldx + perm[i];
    if (accumulate) *dst += v; else *dst = v;
  }
}

// atomic max for non-negative doubles through their IEEE bit patterns (the
// order of non-negative doubles is that of their bits); shared or global
__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

// The max-norms are reduced per block in shared memory first, then one
// global atomic per block and value: a global atomic per row would serialize
// millions of updates on the same address.

// r = b - A x, plus max |r| and max |x| per RHS.  G lanes per row (G = 4 to
// 32 by the mean row length, so short rows do not leave most of a warp
// idle); a group's lanes take the row's entries G apart and add their sums
// by shuffles.  The rows of a warp advance together, so the shuffles see
// every lane; the max-norms are kept per thread and reduced once per warp.
template <int G>
__global__ void k_residual(const int64_t* rowptr, const int32_t* colind, const double* vals,
                           int64_t n, const double* B, int64_t ldb, const double* X, int64_t ldx,
                           double* R, int nrhs, double* rnorm, double* xnorm) {
  extern __shared__ double smax[];  // [0, nrhs): |r|, [nrhs, 2 nrhs): |x|
  for (int i = threadIdx.x; i < 2 * nrhs; i += blockDim.x) smax[i] = 0.0;
  __syncthreads();
  constexpr int RPW = 32 / G;  // rows per warp and step
  const int lane = threadIdx.x & 31, sub = lane & (G - 1);
  const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int r = 0; r < nrhs; ++r) {
    const double* x = X + r * ldx;
    double rmax = 0.0, xmax = 0.0;
    for (int64_t base = gwarp * RPW; base < n; base += nwarps * RPW) {
      const int64_t row = base + lane / G;
      double s = 0.0;
      if (row < n) {
        const int64_t p0 = rowptr[row], p1 = rowptr[row + 1];
        double s2 = 0.0;
        int64_t p = p0 + sub;
        for (; p + G < p1; p += 2 * G) {
          const double v0 = vals[p], v1 = vals[p + G];
          const int32_t j0 = colind[p], j1 = colind[p + G];
          s = fma(v0, x[j0], s);
          s2 = fma(v1, x[j1], s2);
        }
        if (p < p1) s = fma(vals[p], x[colind[p]], s);
        s += s2;
      }
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (sub == 0 && row < n) {
        const double res = B[r * ldb + row] - s;
        R[r * n + row] = res;
        rmax = fmax(rmax, fabs(res));
        xmax = fmax(xmax, fabs(x[row]));
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
      xmax = fmax(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
    }
    if (lane == 0) {
      atomic_max_nonneg(&smax[r], rmax);
      atomic_max_nonneg(&smax[nrhs + r], xmax);
    }
  }
  __syncthreads();
  for (int r = threadIdx.x; r < nrhs; r += blockDim.x) {
    atomic_max_nonneg(&rnorm[r], smax[r]);
    atomic_max_nonneg(&xnorm[r], smax[nrhs + r]);
  }
}

// max row sum of |A| into out[0], max |b_r| into out[1 + r]
// (dynamic shared memory: 1 + nrhs doubles)
__global__ void k_norms(const int64_t* rowptr, const double* vals, int64_t n, const double* B,
                        int64_t ldb, int nrhs, double* out) {
  extern __shared__ double smax[];
  for (int i = threadIdx.x; i < 1 + nrhs; i += blockDim.x) smax[i] = 0.0;
  __syncthreads();
  double amax = 0.0;
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < n;
       row += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int64_t p = rowptr[row]; p < rowptr[row + 1]; ++p) s += fabs(vals[p]);
    amax = fmax(amax, s);
    for (int r = 0; r < nrhs; ++r) atomic_max_nonneg(&smax[1 + r], fabs(B[r * ldb + row]));
  }
  atomic_max_nonneg(&smax[0], amax);
  __syncthreads();
  for (int i = threadIdx.x; i < 1 + nrhs; i += blockDim.x) atomic_max_nonneg(&out[i], smax[i]);
}

template <typename T, int R>
cudaError_t init_r() {
  cudaError_t e = cudaFuncSetAttribute(k_fw_level<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)fw_level_smem<T, R>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_bw_level<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bw_level_smem<T, R>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fw_gemv<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)gemv_smem<T, R>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fw_pinv<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)gemv_smem<T, R>());
  if constexpr (R >= 8) {
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_bw_gemm<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)bw_gemm_smem<T, R>());
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_bw_pinv<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)bw_gemm_smem<T, R>());
  }
  return e;
}

template <typename T>
cudaError_t init_t() {
  cudaError_t e = init_r<T, 1>();
  if (e == cudaSuccess) e = init_r<T, 8>();
  if (e == cudaSuccess) e = init_r<T, kSolveChunk>();
  return e;
}

template <typename T, int R>
cudaError_t launch_r(const Launch& L, const SolveArgs& a, cudaStream_t st) {
  const SD<T> d = make_sd<T>(a);
  if (L.kind == K_FW_LEVEL)
    k_fw_level<T, R><<<L.count, 256, fw_level_smem<T, R>(), st>>>(d, L.item_off,
                                                                   a.sync + 2 * L.level);
  else if (L.kind == K_BW_LEVEL)
    k_bw_level<T, R><<<L.count, 256, bw_level_smem<T, R>(), st>>>(d, L.item_off,
                                                                   a.sync + 2 * L.level + 1);
  else if (L.kind == K_FW_GEMV) {
    if constexpr (R == 1) {
      if (L.tile == 2) k_fw_gemv1r<T, 2><<<L.count, 256, 0, st>>>(d, L.item_off);
      else if (L.tile == 1) k_fw_gemv1r<T, 8><<<L.count, 256, 0, st>>>(d, L.item_off);
      else k_fw_gemv1<T><<<4 * L.count, 256, 0, st>>>(d, L.item_off);
    }
    else k_fw_gemv<T, R><<<L.count, 256, gemv_smem<T, R>(), st>>>(d, L.item_off);
  } else if (L.kind == K_FW_PINV) {
    if constexpr (R == 1) k_fw_pinv1<T><<<4 * L.count, 256, 0, st>>>(d, L.item_off);
    else k_fw_pinv<T, R><<<L.count, 256, gemv_smem<T, R>(), st>>>(d, L.item_off);
  } else if (L.kind == K_BW_PINV) {
    if constexpr (R >= 8) k_bw_pinv<T, R><<<L.count, 256, bw_gemm_smem<T, R>(), st>>>(d, L.item_off);
    else k_bw_pinv1<T><<<4 * L.count, 256, 0, st>>>(d, L.item_off);
  } else if constexpr (R >= 8) {
    k_bw_gemm<T, R><<<L.count, 256, bw_gemm_smem<T, R>(), st>>>(d, L.item_off);
  } else {
    // CTAs per item: the launch's row split P (1, 2, 4 or 8)
    const int per = (int)L.tile;
    // the builder writes 1, 2, 4 or 8 and a loaded analysis is checked for it
    if (per != 1 && per != 2 && per != 4 && per != 8) return cudaErrorInvalidValue;
    k_bw_gemv1<T><<<per * L.count, 256, 0, st>>>(d, L.item_off, per);
  }
  return cudaSuccess;
}

template <typename T, int H>
void launch_warp(bool fw, const Launch& L, const SolveArgs& a, cudaStream_t st) {
  const SD<T> d = make_sd<T>(a);
  const int blocks = (int)((L.count + 7) / 8);
  if constexpr (H == 2) {
    if (a.nrhs >= 2) {
      if (fw) k_fw_tiny<T, 8><<<blocks, 256, 0, st>>>(d, L.item_off, L.count);
      else k_bw_tiny<T, 8><<<blocks, 256, 0, st>>>(d, L.item_off, L.count);
    } else {
      if (fw) k_fw_tiny<T, 1><<<blocks, 256, 0, st>>>(d, L.item_off, L.count);
      else k_bw_tiny<T, 1><<<blocks, 256, 0, st>>>(d, L.item_off, L.count);
    }
  } else {
    // right-hand sides per pass of the forward kernel: as many as its static
    // shared memory (8 warps x 32 H rows x RB values) allows, up to 4
    constexpr int rb_max = (48 * 1024) / (8 * 32 * H * (int)sizeof(T));
    if (!fw) {
      k_bw_warp<T, H><<<blocks, 256, 0, st>>>(d, L.item_off, L.count);
    } else if (a.nrhs >= 4 && rb_max >= 4) {
      if constexpr (rb_max >= 4) k_fw_warp<T, H, 4><<<blocks, 256, 0, st>>>(d, L.item_off, L.count);
    } else if (a.nrhs >= 2 && rb_max >= 2) {
      if constexpr (rb_max >= 2) k_fw_warp<T, H, 2><<<blocks, 256, 0, st>>>(d, L.item_off, L.count);
    } else {
      k_fw_warp<T, H, 1><<<blocks, 256, 0, st>>>(d, L.item_off, L.count);
    }
  }
}

template <typename T>
cudaError_t launch_t(const Launch& L, const SolveArgs& a, cudaStream_t st) {
  if (L.kind == K_FW_WARP || L.kind == K_BW_WARP) {
    const bool fw = L.kind == K_FW_WARP;
    switch (L.param) {
      case 2: launch_warp<T, 2>(fw, L, a, st); break;
      case 4: launch_warp<T, 4>(fw, L, a, st); break;
      case 8: launch_warp<T, 8>(fw, L, a, st); break;
      case 16: launch_warp<T, 16>(fw, L, a, st); break;
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  if (L.kind == K_V4_FW || L.kind == K_V4_BW) {
    if (a.nrhs <= 1) launch_v4<T, 1>(L, a, st);
    else if (a.nrhs <= 4) launch_v4<T, 4>(L, a, st);
    else if (a.nrhs <= 8) launch_v4<T, 8>(L, a, st);
    else launch_v4<T, kSolveChunk>(L, a, st);
    return cudaGetLastError();
  }
  if (L.kind == K_FW_PGATHER || L.kind == K_BW_PCOPY) {
    const SD<T> d = make_sd<T>(a);
    if (L.kind == K_FW_PGATHER) k_fw_pgather<T><<<L.count, 256, 0, st>>>(d, L.item_off);
    else k_bw_pcopy<T><<<L.count, 256, 0, st>>>(d, L.item_off);
    return cudaGetLastError();
  }
  if (L.kind != K_FW_LEVEL && L.kind != K_BW_LEVEL && L.kind != K_FW_GEMV &&
      L.kind != K_BW_GEMV && L.kind != K_FW_PINV && L.kind != K_BW_PINV)
    return cudaErrorInvalidValue;
  cudaError_t e;
  if (a.nrhs <= 1) e = launch_r<T, 1>(L, a, st);
  else if (a.nrhs <= 8) e = launch_r<T, 8>(L, a, st);
  else e = launch_r<T, kSolveChunk>(L, a, st);
  if (e != cudaSuccess) return e;
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

cudaError_t launch_wait_probe(const int* flag, unsigned long long* status, int limit,
                              cudaStream_t st) {
  k_wait_probe<<<1, 64, 0, st>>>(flag, status, limit);
  return cudaGetLastError();
}

cudaError_t launch_solve(int prec, const Launch& L, const SolveArgs& a, cudaStream_t st) {
  if (L.count <= 0) return cudaSuccess;
  return prec == MF_FP32 ? launch_t<float>(L, a, st) : launch_t<double>(L, a, st);
}

namespace {
template <typename T>
__global__ void k_dscale(T* Y, const T* D, int64_t n, int32_t nrhs) {
  const int64_t total = n * nrhs;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x)
    Y[e] /= D[e % n];
}
}  // namespace

cudaError_t launch_dscale(int prec, void* Y, const void* D, int64_t n, int32_t nrhs,
                          cudaStream_t st) {
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  const int g = grid_for(n * nrhs);
  if (prec == MF_FP32)
    k_dscale<float><<<g, 256, 0, st>>>(static_cast<float*>(Y), static_cast<const float*>(D), n, nrhs);
  else
    k_dscale<double><<<g, 256, 0, st>>>(static_cast<double*>(Y), static_cast<const double*>(D), n,
                                        nrhs);
  return cudaGetLastError();
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

cudaError_t launch_perm_out(int prec, const void* Y, const int32_t* perm, const int32_t* ipos,
                            double* X, int64_t ldx, int64_t n, int32_t nrhs, const double* scale,
                            int32_t accumulate, cudaStream_t st) {
  const int g = grid_for(n * nrhs);
  if (prec == MF_FP32)
    k_perm_out<float><<<g, 256, 0, st>>>(static_cast<const float*>(Y), perm, ipos, X, ldx, n, nrhs,
                                         scale, accumulate);
  else
    k_perm_out<double><<<g, 256, 0, st>>>(static_cast<const double*>(Y), perm, ipos, X, ldx, n,
                                          nrhs, scale, accumulate);
  return cudaGetLastError();
}

cudaError_t launch_residual(const int64_t* rowptr, const int32_t* colind, const double* vals,
                            int64_t n, int64_t nnz_hint, const double* B, int64_t ldb,
                            const double* X, int64_t ldx, double* R, int32_t nrhs, double* rnorm,
                            double* xnorm, cudaStream_t st) {
  // lanes per row by the mean row length (the CSR's last row pointer is on
  // the device, so the length comes from the caller: nnz / n)
  const int64_t nnz = nnz_hint;
  const double mean = n > 0 ? (double)nnz / (double)n : 0.0;
  const int G = mean <= 8 ? 4 : mean <= 16 ? 8 : mean <= 32 ? 16 : 32;
  int64_t g = (n * G + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  if (g < 1) g = 1;
  const size_t sm = 2 * (size_t)nrhs * sizeof(double);
  if (G == 4)
    k_residual<4><<<(int)g, 256, sm, st>>>(rowptr, colind, vals, n, B, ldb, X, ldx, R, nrhs, rnorm, xnorm);
  else if (G == 8)
    k_residual<8><<<(int)g, 256, sm, st>>>(rowptr, colind, vals, n, B, ldb, X, ldx, R, nrhs, rnorm, xnorm);
  else if (G == 16)
    k_residual<16><<<(int)g, 256, sm, st>>>(rowptr, colind, vals, n, B, ldb, X, ldx, R, nrhs, rnorm, xnorm);
  else
    k_residual<32><<<(int)g, 256, sm, st>>>(rowptr, colind, vals, n, B, ldb, X, ldx, R, nrhs, rnorm, xnorm);
  return cudaGetLastError();
}

cudaError_t launch_norms(const int64_t* rowptr, const double* vals, int64_t n, const double* B,
                         int64_t ldb, int32_t nrhs, double* out, cudaStream_t st) {
  k_norms<<<grid_for(n), 256, (1 + (size_t)nrhs) * sizeof(double), st>>>(rowptr, vals, n, B, ldb,
                                                                         nrhs, out);
  return cudaGetLastError();
}

}  // namespace mf
