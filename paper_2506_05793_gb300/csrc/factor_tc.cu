// factor_tc.cu -- FP32 trailing update of large fronts on the 5th-generation
// tensor cores of sm_103a (tcgen05, kind::tf32) with split-TF32 operands.
//
// One panel step of a front factors b <= 64 pivot columns; the trailing lower
// triangle is then updated, C -= P P^T, with P the solved panel rows (paper
// Sec. 5: dense POTRF/TRSM/SYRK per front).  To keep FP32 accuracy on TF32
// tensor cores each panel value is split, p = hi + lo with hi = tf32(p) and
// lo = p - hi, and C -= hi hi^T + hi lo^T + lo hi^T (the lo lo^T term is
// below FP32 rounding).  The TRSM kernel writes hi and lo of every panel row
// into a row-major staging buffer (128 floats per row: 64 hi, 64 lo).
//
// One CTA (128 threads) computes one 128 x 128 tile (I, J), I >= J:
//   - the 64-wide K range is staged in two halves of 32 through one 64 KB
//     shared-memory buffer (so three CTAs fit on an SM and overlap); each half
//     is copied with cp.async in the canonical K-major 128-byte-swizzle layout
//     (8-row atoms of 8 x 16-byte units, unit u of row r stored at u ^ (r & 7));
//   - one elected thread issues 12 tcgen05.mma per half (3 products x 4
//     k-steps of 8) into a 128 x 128 FP32 accumulator in tensor memory and
//     commits them to an mbarrier (phase 0, then phase 1);
//   - after a bounded wait, each warp reads its 32 accumulator lanes with
//     tcgen05.ld and subtracts them from the lower part of the tile in HBM,
//     loading the next 32 columns' old values before storing the current.
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"

namespace mf {
namespace {

constexpr int kTcM = 128;
constexpr int kTcN = 128;
constexpr uint32_t kTmemCols = 128;
constexpr int kOpBytes = 128 * 128;  // one 128-row x 32-float swizzled K-chunk
constexpr size_t kTcSmem = 4 * (size_t)kOpBytes + 1024 + 64;
constexpr long long kMbarSpin = 1ll << 22;  // try_wait polls before giving up

// instruction descriptor: D = F32, A = B = TF32, both K-major, M = N = 128
constexpr uint32_t kIdescTf32 = (1u << 4) | (2u << 7) | (2u << 10) |
                                ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor, K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(src_bytes)
               : "memory");
}

// Copy K-half h (k in [32 h, 32 h + 32)) of 128 staging rows (row R0 + r) into
// the swizzled hi and lo chunks; rows at or beyond `valid` are zero-filled.
__device__ __forceinline__ void load_half(const float* split, int64_t R0, int valid, int h,
                                          uint32_t hi_base, uint32_t lo_base) {
  for (int idx = threadIdx.x; idx < 128 * 16; idx += blockDim.x) {
    const int r = idx >> 4, U = idx & 15;
    const int part = U >> 3, u = U & 7;
    const uint32_t dst = (part ? lo_base : hi_base) + r * 128 + ((u ^ (r & 7)) << 4);
    const bool ok = r < valid;
    const float* src = split + (ok ? (R0 + r) * 128 + part * 64 + h * 32 + u * 4 : 0);
    cp_async16(dst, src, ok ? 16 : 0);
  }
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (long long spin = 0; spin < kMbarSpin; ++spin) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accum) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(kIdescTf32), "r"(accum)
      : "memory");
}

template <typename T>
struct TcArgs {
  const SnInfo* sn;
  const Item* items;
  const int64_t* soff;
  const float* split;
  T* L;
  T* U;
  unsigned long long* status;
};

__global__ void __launch_bounds__(128, 3) k_syrk_tc(TcArgs<float> d, int64_t item_off) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned operand chunks: A hi, A lo, B hi, B lo (one K-half each)
  const uint32_t sbase = (smem_u32(smem_raw) + 1023u) & ~1023u;
  unsigned char* gbase = smem_raw + (sbase - smem_u32(smem_raw));
  const uint32_t a_hi = sbase, a_lo = sbase + kOpBytes;
  const uint32_t b_hi = sbase + 2 * kOpBytes, b_lo = sbase + 3 * kOpBytes;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(gbase + 4 * kOpBytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbase + 4 * kOpBytes + 8);

  const Item it = d.items[item_off + blockIdx.x];
  const SnInfo f = d.sn[it.s];
  const int nf = f.k + f.m;
  const int c0 = it.t * kNB;
  const int b = min(kNB, f.k - c0);
  const int p0 = c0 + b;
  const int rI = p0 + it.a * kTcM, rJ = p0 + it.b * kTcN;
  const bool diag = it.a == it.b;
  const int64_t R0 = d.soff[it.s];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t mb = smem_u32(mbar);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  const uint32_t bh = diag ? a_hi : b_hi, bl = diag ? a_lo : b_lo;
  bool ok = true;
  uint32_t tmem = 0;
  for (int h = 0; h < 2; ++h) {
    load_half(d.split, R0 + rI, nf - rI, h, a_hi, a_lo);
    if (!diag) load_half(d.split, R0 + rJ, nf - rJ, h, b_hi, b_lo);
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    tmem = *tmem_slot;
    if (tid == 0) {
      // small terms first: lo*hi, hi*lo, then hi*hi; 4 k-steps of 8 each
      const uint32_t as[3] = {a_lo, a_hi, a_hi};
      const uint32_t bs[3] = {bh, bl, bh};
      for (int term = 0; term < 3; ++term)
        for (int ks = 0; ks < 4; ++ks)
          mma_tf32(tmem, sdesc_sw128(as[term] + ks * 32), sdesc_sw128(bs[term] + ks * 32),
                   (h | term | ks) != 0);
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mb)
          : "memory");
    }
    // the MMAs of this half must finish reading shared memory (and, for the
    // second half, writing the accumulator) before anyone goes on
    ok = ok && mbar_wait(mb, (uint32_t)h);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (!ok) break;
  }
  if (!ok) {
    if (lane == 0) atomicExch(d.status + 1, (unsigned long long)MF_ERR_TIMEOUT);
  } else {
    const int i = warp * 32 + lane;  // accumulator lane = row of the tile
    const int r = rI + i;
    const bool rowok = r < nf;
    // element (r, c) of the front: L panel for c < k, update matrix beyond
    auto addr = [&](int c) -> float* {
      if (c < f.k) return d.L + f.Loff + (int64_t)c * nf + r;
      return d.U + (f.Uoff + (int64_t)(c - f.k) * f.m + (r - f.k));
    };
    float cur[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int c = rJ + j;
      cur[j] = (rowok && c < nf && r >= c) ? *addr(c) : 0.0f;
    }
    for (int cb = 0; cb < kTcN / 32; ++cb) {
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cb * 32);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
          "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
            "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
            "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
            "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
            "=r"(v[31])
          : "r"(taddr)
          : "memory");
      // the next chunk's old values are loaded before this chunk is stored
      float nxt[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int c = rJ + (cb + 1) * 32 + j;
        nxt[j] = (cb < 3 && rowok && c < nf && r >= c) ? *addr(c) : 0.0f;
      }
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int c = rJ + cb * 32 + j;
        if (rowok && c < nf && r >= c) *addr(c) = cur[j] - __uint_as_float(v[j]);
      }
#pragma unroll
      for (int j = 0; j < 32; ++j) cur[j] = nxt[j];
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
}

}  // namespace

size_t tc_smem_bytes() { return kTcSmem; }

cudaError_t factor_tc_init() {
  return cudaFuncSetAttribute(k_syrk_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
}

cudaError_t launch_syrk_tc(const Launch& L, const FactorArgs& a, cudaStream_t st) {
  if (L.count <= 0) return cudaSuccess;
  TcArgs<float> d;
  d.sn = a.sym.sn;
  d.items = a.sym.items;
  d.soff = a.sym.soff;
  d.split = a.split;
  d.L = static_cast<float*>(a.L);
  d.U = static_cast<float*>(a.U);
  d.status = a.status;
  k_syrk_tc<<<L.count, 128, kTcSmem, st>>>(d, L.item_off);
  return cudaGetLastError();
}

}  // namespace mf
