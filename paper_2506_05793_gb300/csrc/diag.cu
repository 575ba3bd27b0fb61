// diag.cu -- measured FP64 peak of this GPU, for the roofline of the FP64
// front kernels (no paper counterpart).
//
// Two register-resident loops, each long enough (about 10^11 flops) that
// launch costs vanish:
//   kind 0: DFMA -- every thread runs kChains independent FMA chains;
//   kind 1: DMMA -- every warp issues mma.sync m8n8k4 f64 into kChains/2
//           independent accumulator tiles.
// Both read their operands from registers only and store one value per
// thread at the end, so the compiler keeps every instruction.
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"

namespace mf {
namespace {

constexpr int kChains = 16;

__global__ void __launch_bounds__(256) k_peak_dfma(double* out, int64_t iters, double a, double b) {
  double acc[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c] = (double)(threadIdx.x + c);
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = fma(acc[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_peak_dmma(double* out, int64_t iters, double a, double b) {
  // per lane: A fragment 1 double, B fragment 1 double, C/D 2 doubles
  constexpr int kTiles = kChains / 2;
  double c[kTiles][2];
  const double av = a + threadIdx.x * 1e-3, bv = b - threadIdx.x * 1e-3;
#pragma unroll
  for (int t = 0; t < kTiles; ++t) c[t][0] = c[t][1] = 0.0;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int t = 0; t < kTiles; ++t)
      asm volatile(
          "mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
          : "+d"(c[t][0]), "+d"(c[t][1])
          : "d"(av), "d"(bv));
  }
  double s = 0.0;
#pragma unroll
  for (int t = 0; t < kTiles; ++t) s += c[t][0] + c[t][1];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

int peak_fp64_blocks_per_sm(int kind) {
  int nb = 0;
  if (kind == 0)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_peak_dfma, 256, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_peak_dmma, 256, 0);
  return nb > 0 ? nb : 1;
}

cudaError_t launch_peak_fp64(int kind, double* out, int blocks, int64_t iters, cudaStream_t st) {
  if (kind == 0)
    k_peak_dfma<<<blocks, 256, 0, st>>>(out, iters, 0.999999, 1e-9);
  else
    k_peak_dmma<<<blocks, 256, 0, st>>>(out, iters, 0.999999, 1e-9);
  return cudaGetLastError();
}

// flops of one launch
double peak_fp64_flops(int kind, int blocks, int64_t iters) {
  const double threads = (double)blocks * 256.0;
  if (kind == 0) return threads * (double)iters * kChains * 2.0;
  // one m8n8k4 per warp: 8 x 8 x 4 FMAs
  return threads / 32.0 * (double)iters * (kChains / 2) * 8.0 * 8.0 * 4.0 * 2.0;
}

}  // namespace mf
