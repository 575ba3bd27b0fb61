// ilu_kernels.cu -- FastILU and FastSpTRSV sweeps (paper Sec. 6, after Chow
// and Patel) on sm_103a.
//
// The factor sweep updates every entry (i, j) of the ILU(k) pattern S
// independently:
//   s = a_ij - sum_{k < min(i, j)} l_ik u_kj,
//   l_ij = (1 - w) l_ij + w s / u_jj (i > j),  u_ij = (1 - w) u_ij + w s (i <= j).
// One thread per entry walks row i of L (the entries left of the diagonal,
// columns increasing) and column j of S (rows increasing) together and sums
// the products of matching k in increasing k, the order the definition
// reads.  Out of place the sweep depends only on the previous sweep's
// factors; in place (old == out) it reads whatever its neighbours have
// written, as the paper's asynchronous sweep does.
#include <cuda_runtime.h>

#include "ilu.h"

namespace mf {
namespace {

constexpr int kThreads = 256;

int grid_of(int64_t items) {
  const int64_t g = (items + kThreads - 1) / kThreads;
  return (int)(g < 1 ? 1 : g);
}

__global__ void k_ilu_gather(IluDev d, const double* vals, double shift, double* aS) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= d.nnz) return;
  double s = 0.0;
  for (int64_t p = d.a_ptr[q]; p < d.a_ptr[q + 1]; ++p) s += vals[d.a_src[p]];
  if (d.Si[q] == d.Sj[q]) s *= 1.0 + shift;
  aS[q] = s;
}

__global__ void k_ilu_init(IluDev d, const double* aS, int K, int warm, double* F) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= d.nnz) return;
  const int lev = d.Slev[q];
  if (warm) {
    if (lev == K) F[q] = 0.0;
    return;
  }
  if (lev > K) return;
  const int i = d.Si[q], j = d.Sj[q];
  F[q] = i > j ? aS[q] / aS[d.diag[j]] : aS[q];
}

__global__ void k_ilu_sweep(IluDev d, const double* aS, int K, const double* old, double* out,
                            double omega) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= d.nnz) return;
  if (d.Slev[q] > K) {  // not part of this level's factors: carried over
    if (out != old) out[q] = old[q];
    return;
  }
  const int i = d.Si[q], j = d.Sj[q];
  const int m = i < j ? i : j;
  double s = aS[q];
  // row i of L: positions Sp[i] .. diag[i]-1, column k = Sj[a]
  int64_t a = d.Sp[i];
  const int64_t a_end = d.diag[i];
  // column j of S: positions cp[j] .. cp[j+1]-1, row k = cr[b]
  int64_t b = d.cp[j];
  const int64_t b_end = d.cp[j + 1];
  while (a < a_end && b < b_end) {
    const int ka = d.Sj[a], kb = d.cr[b];
    if (ka >= m || kb >= m) break;
    if (ka < kb) {
      ++a;
    } else if (kb < ka) {
      ++b;
    } else {
      const int64_t pb = d.cq[b];
      if (d.Slev[a] <= K && d.Slev[pb] <= K) s -= old[a] * old[pb];
      ++a;
      ++b;
    }
  }
  const double prev = old[q];
  out[q] = i > j ? (1.0 - omega) * prev + omega * s / old[d.diag[j]]
                 : (1.0 - omega) * prev + omega * s;
}

__global__ void k_ilu_trsv(IluDev d, const double* LU, int K, int upper, const double* b,
                           const double* xo, double* x, double omega) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= d.n) return;
  double s = b[i];
  const int64_t q0 = upper ? d.diag[i] + 1 : d.Sp[i];
  const int64_t q1 = upper ? d.Sp[i + 1] : d.diag[i];
  for (int64_t q = q0; q < q1; ++q)
    if (d.Slev[q] <= K) s -= LU[q] * xo[d.Sj[q]];
  if (upper) s /= LU[d.diag[i]];
  x[i] = (1.0 - omega) * xo[i] + omega * s;
}

}  // namespace

cudaError_t launch_ilu_gather(const IluDev& d, const double* vals, double shift, double* aS,
                              cudaStream_t st) {
  if (d.nnz == 0) return cudaSuccess;
  k_ilu_gather<<<grid_of(d.nnz), kThreads, 0, st>>>(d, vals, shift, aS);
  return cudaGetLastError();
}

cudaError_t launch_ilu_init(const IluDev& d, const double* aS, int32_t K, int32_t warm,
                            double* F, cudaStream_t st) {
  if (d.nnz == 0) return cudaSuccess;
  k_ilu_init<<<grid_of(d.nnz), kThreads, 0, st>>>(d, aS, K, warm, F);
  return cudaGetLastError();
}

cudaError_t launch_ilu_sweep(const IluDev& d, const double* aS, int32_t K, const double* old,
                             double* out, double omega, cudaStream_t st) {
  if (d.nnz == 0) return cudaSuccess;
  k_ilu_sweep<<<grid_of(d.nnz), kThreads, 0, st>>>(d, aS, K, old, out, omega);
  return cudaGetLastError();
}

cudaError_t launch_ilu_trsv(const IluDev& d, const double* LU, int32_t K, int32_t upper,
                            const double* b, const double* xo, double* x, double omega,
                            cudaStream_t st) {
  if (d.n == 0) return cudaSuccess;
  k_ilu_trsv<<<grid_of(d.n), kThreads, 0, st>>>(d, LU, K, upper, b, xo, x, omega);
  return cudaGetLastError();
}

}  // namespace mf
