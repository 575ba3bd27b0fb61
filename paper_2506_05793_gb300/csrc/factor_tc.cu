// factor_tc.cu -- FP32 trailing update of large fronts on the 5th-generation
// tensor cores of sm_103a (tcgen05, kind::tf32) with split-TF32 operands.
//
// One panel step of a front factors b <= 64 pivot columns; the trailing lower
// triangle is then updated, C -= P P^T, with P the solved panel rows (paper
// Sec. 5: dense POTRF/TRSM/SYRK per front).  To keep FP32 accuracy on TF32
// tensor cores each panel value is split, p = hi + lo with hi = tf32(p) and
// lo = p - hi, and C -= hi hi^T + hi lo^T + lo hi^T (the lo lo^T term is
// below FP32 rounding).  The TRSM kernel writes hi and lo of every panel row
// into a row-major staging buffer (512 floats per row: four panel slots of
// 64 hi then 64 lo, slot = panel mod 4; 1024 floats and eight slots on the
// lookahead levels, where a group's bulk pass runs beside the next group's
// panels).
//
// Panels are grouped by four to quarter the traffic of the trailing matrix:
// inside a group g0 .. gl the next panel's 64 columns are updated
// left-looking after each panel t < gl (a strip with panels g0 .. t), and
// after gl one pass with K up to 256 updates everything beyond it.
//
// One CTA (128 threads) computes one 128 x 128 tile (I, J), I >= J:
//   - the K range (64 per panel, up to 256) is staged in quarters of 32
//     through one 64 KB shared-memory buffer (so three CTAs fit on an SM
//     and overlap); one thread
//     copies each half with TMA (a tensor map over the staging buffer, boxes
//     of 128 rows x 32 floats with 128-byte swizzle), which writes the
//     canonical K-major layout the MMA descriptors expect (8-row atoms of
//     8 x 16-byte units, unit u of row r stored at u ^ (r & 7));
//   - one elected thread issues 12 tcgen05.mma per half (3 products x 4
//     k-steps of 8) into a 128 x 128 FP32 accumulator in tensor memory and
//     commits them to an mbarrier (phase 0, then phase 1);
//   - after a bounded wait, each warp reads its 32 accumulator lanes with
//     tcgen05.ld and subtracts them from the lower part of the tile in HBM,
//     loading the next 32 columns' old values before storing the current.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "kernels.h"

namespace mf {
namespace {

constexpr int kTcM = 128;
constexpr int kTcN = 128;
constexpr uint32_t kTmemCols = 128;
constexpr int kOpBytes = 128 * 128;  // one 128-row x 32-float swizzled K-chunk
constexpr int kMaxQuarters = 8;  // K = 256: four panels of two 32-wide quarters
constexpr size_t kTcSmem = 4 * (size_t)kOpBytes + 1024 + 256;
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


// TMA copy of one 128-row x 32-float box of the staging buffer (element
// column x, row y) into shared memory at dst; completion is counted on mbar.
__device__ __forceinline__ void tma_box(uint32_t dst, const CUtensorMap* map, int x, int64_t y,
                                        uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"((int)y), "r"(mbar)
      : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes)
               : "memory");
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

__global__ void __launch_bounds__(128, 3)
    k_syrk_tc(TcArgs<float> d, const __grid_constant__ CUtensorMap smap0,
              const __grid_constant__ CUtensorMap smap1, int area, int64_t item_off) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned operand chunks: A hi, A lo, B hi, B lo (one K-half each)
  const uint32_t sbase = (smem_u32(smem_raw) + 1023u) & ~1023u;
  unsigned char* gbase = smem_raw + (sbase - smem_u32(smem_raw));
  const uint32_t a_hi = sbase, a_lo = sbase + kOpBytes;
  const uint32_t b_hi = sbase + 2 * kOpBytes, b_lo = sbase + 3 * kOpBytes;
  // one single-use barrier per event (MMAs of quarter q at + 8 q, TMA of
  // quarter q at + 64 + 8 q, q < 8), each waited once on phase 0: a thread
  // that reaches its wait late can never mistake a later phase for its own
  uint64_t* mbar = reinterpret_cast<uint64_t*>(gbase + 4 * kOpBytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbase + 4 * kOpBytes + 16 * 8);

  const Item it = d.items[item_off + blockIdx.x];
  const SnInfo f = d.sn[it.s];
  const int nf = f.k + f.m;
  // panels tt .. tt + nK - 1 (one group) applied to the columns beyond the
  // last of them: all of them (a group pass) or, for a strip, only the next
  // panel's 64 columns
  const int tt = it.t & 0xffff, nK = (it.t >> 16) & 0xff, strip = it.t >> 24;
  const int tl = tt + nK - 1;  // last panel applied
  const int c0 = tl * kNB;
  const int b = min(kNB, f.k - c0);
  const int p0 = c0 + b;
  const int rI = p0 + it.a * kTcM, rJ = p0 + it.b * kTcN;
  const int cmax = strip ? min(f.k, p0 + kNB) : nf;  // columns updated: [p0, cmax)
  const int nq = min(2 * nK, kMaxQuarters);          // K quarters of 32
  const bool diag = it.a == it.b;
  // staging rows: area 0 holds four panel slots per row, area 1 eight
  const int64_t R0 = d.soff[it.s] & (((int64_t)1 << kSoffAreaShift) - 1);
  const CUtensorMap* smap = area ? &smap1 : &smap0;
  const int smask = area ? 7 : 3;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t mb0 = smem_u32(mbar);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    for (int q = 0; q < 2 * kMaxQuarters; ++q)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb0 + 8 * q) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const int i = warp * 32 + lane;  // accumulator lane = row of the tile
  const int r = rI + i;
  const bool rowok = r < nf;
  // element (r, c) of the front: L panel for c < k, update matrix beyond.
  // Per 32-column chunk one base pointer and a column stride; a chunk that
  // straddles k takes the per-column path.
  auto col_ptr = [&](int c) -> float* {
    if (c < f.k) return d.L + f.Loff + (int64_t)c * nf + r;
    return d.U + f.Uoff + (int64_t)(c - f.k) * f.m + (r - f.k);
  };
  auto chunk_load = [&](int cbase, float (&out)[32]) {
    const int lim = rowok ? min(min(32, cmax - cbase), r - cbase + 1) : 0;  // valid j < lim
    if (cbase + 32 <= f.k || cbase >= f.k) {
      const bool inL = cbase < f.k;
      const int64_t ld = inL ? nf : f.m;
      const float* p = inL ? d.L + f.Loff + (int64_t)cbase * nf + r
                           : d.U + f.Uoff + (int64_t)(cbase - f.k) * f.m + (r - f.k);
#pragma unroll
      for (int j = 0; j < 32; ++j) out[j] = j < lim ? p[j * ld] : 0.0f;
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j) out[j] = j < lim ? *col_ptr(cbase + j) : 0.0f;
    }
  };
  auto chunk_store = [&](int cbase, const float (&cur)[32], const uint32_t (&v)[32]) {
    const int lim = rowok ? min(min(32, cmax - cbase), r - cbase + 1) : 0;
    if (cbase + 32 <= f.k || cbase >= f.k) {
      const bool inL = cbase < f.k;
      const int64_t ld = inL ? nf : f.m;
      float* p = inL ? d.L + f.Loff + (int64_t)cbase * nf + r
                     : d.U + f.Uoff + (int64_t)(cbase - f.k) * f.m + (r - f.k);
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (j < lim) p[j * ld] = cur[j] - __uint_as_float(v[j]);
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (j < lim) *col_ptr(cbase + j) = cur[j] - __uint_as_float(v[j]);
    }
  };
  // the tile of C goes to L2 while the operands load and multiply: thread t
  // prefetches the rows of column rJ + t that the epilogue will touch
  {
    const int c = rJ + tid;
    const int lo = max(rI, c), hi = min(rI + kTcM, nf);
    if (c < cmax && lo < hi) {
      const float* p = c < f.k ? d.L + f.Loff + (int64_t)c * nf + lo
                               : d.U + f.Uoff + (int64_t)(c - f.k) * f.m + (lo - f.k);
      for (int o = 0; o < hi - lo; o += 32) asm volatile("prefetch.global.L2 [%0];" ::"l"(p + o));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(p + (hi - lo - 1)));
    }
  }
  float cur[32];
  chunk_load(rJ, cur);
  const uint32_t bh = diag ? a_hi : b_hi, bl = diag ? a_lo : b_lo;
  bool ok = true;
  for (int q = 0; q < nq; ++q) {
    const uint32_t mb = mb0 + 8 * q, mbt = mb0 + 8 * kMaxQuarters + 8 * q;
    const int h = q & 1;                                           // half of a panel
    const int slot = (tt + (q >> 1)) & smask;                     // staging slot of the panel
    const int x0 = slot * 128 + h * 32;
    // rows of the staging buffer beyond the front belong to other fronts (or
    // are zero); they only reach accumulator rows / columns that the
    // epilogue discards
    if (tid == 0) {
      mbar_expect_tx(mbt, (diag ? 2u : 4u) * (uint32_t)kOpBytes);
      tma_box(a_hi, smap, x0, R0 + rI, mbt);
      tma_box(a_lo, smap, x0 + 64, R0 + rI, mbt);
      if (!diag) {
        tma_box(b_hi, smap, x0, R0 + rJ, mbt);
        tma_box(b_lo, smap, x0 + 64, R0 + rJ, mbt);
      }
    }
    ok = ok && mbar_wait(mbt, 0u);
    if (!ok) break;
    if (tid == 0) {
      // small terms first: lo*hi, hi*lo, then hi*hi; 4 k-steps of 8 each
      const uint32_t as[3] = {a_lo, a_hi, a_hi};
      const uint32_t bs[3] = {bh, bl, bh};
      for (int term = 0; term < 3; ++term)
        for (int ks = 0; ks < 4; ++ks)
          mma_tf32(tmem, sdesc_sw128(as[term] + ks * 32), sdesc_sw128(bs[term] + ks * 32),
                   (q | term | ks) != 0);
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mb)
          : "memory");
    }
    // the MMAs of this half must finish reading shared memory (and, for the
    // second half, writing the accumulator) before anyone goes on
    ok = ok && mbar_wait(mb, 0u);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (!ok) break;
  }
  if (!ok) {
    if (lane == 0) atomicExch(d.status + 1, (unsigned long long)MF_ERR_TIMEOUT);
  } else {
    for (int cb = 0; cb < kTcN / 32; ++cb) {
      const int cbase = rJ + cb * 32;
      if (cbase >= cmax) break;  // same for the whole CTA
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
      if (cb + 1 < kTcN / 32 && cbase + 32 < cmax) chunk_load(cbase + 32, nxt);
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      chunk_store(cbase, cur, v);
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

cudaError_t make_split_map(float* split, int64_t rows, int width, void* map_out) {
  typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                               const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                               const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                               CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static EncodeFn encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = reinterpret_cast<EncodeFn>(fn);
  }
  CUtensorMap m;
  const cuuint64_t dims[2] = {(cuuint64_t)width, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)width * sizeof(float)};
  const cuuint32_t box[2] = {32, 128};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, split, dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  std::memcpy(map_out, &m, sizeof(m));
  return cudaSuccess;
}

cudaError_t launch_syrk_tc(const Launch& L, const FactorArgs& a, cudaStream_t st) {
  if (L.count <= 0) return cudaSuccess;
  if (!a.split_map || !a.split_map_b) return cudaErrorInvalidValue;
  CUtensorMap m0, m1;
  std::memcpy(&m0, a.split_map, sizeof(m0));
  std::memcpy(&m1, a.split_map_b, sizeof(m1));
  TcArgs<float> d;
  d.sn = a.sym.sn;
  d.items = a.sym.items;
  d.soff = a.sym.soff;
  d.split = a.split;
  d.L = static_cast<float*>(a.L);
  d.U = static_cast<float*>(a.U);
  d.status = a.status;
  k_syrk_tc<<<L.count, 128, kTcSmem, st>>>(d, m0, m1, (int)L.area, L.item_off);
  return cudaGetLastError();
}

}  // namespace mf
