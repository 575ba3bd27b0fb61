// ilu.h -- FastILU / FastSpTRSV (paper Sec. 6): device kernels' argument
// blocks and launchers (ilu_kernels.cu), used by ilu.cpp.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace mf {

// Device copy of an ILU(k) pattern S: rows Sp/Sj (columns increasing), the
// row of every entry (Si), its level of fill (Slev), the diagonal positions,
// the columns of S (cp, cr = rows increasing, cq = position in the rows) and
// the gather of A's values onto S (entries a_ptr[q] .. a_ptr[q+1] of a_src).
struct IluDev {
  int64_t n = 0, nnz = 0;
  const int64_t* Sp = nullptr;
  const int32_t* Sj = nullptr;
  const int32_t* Si = nullptr;
  const int32_t* Slev = nullptr;
  const int64_t* diag = nullptr;
  const int64_t* cp = nullptr;
  const int32_t* cr = nullptr;
  const int64_t* cq = nullptr;
  const int64_t* a_ptr = nullptr;
  const int64_t* a_src = nullptr;
};

// aS[q] = sum of A's values gathered onto entry q, the diagonal times 1 + shift
cudaError_t launch_ilu_gather(const IluDev& d, const double* vals, double shift, double* aS,
                              cudaStream_t st);
// F = the sweeps' initial guess on the entries of level <= K (l_ij = a_ij /
// a_jj, u_ij = a_ij); with warm = 1 only the entries of level exactly K are
// set to zero (the others keep the values of FastILU(K - 1))
cudaError_t launch_ilu_init(const IluDev& d, const double* aS, int32_t K, int32_t warm,
                            double* F, cudaStream_t st);
// one FastILU sweep on the entries of level <= K: out of place (old -> out)
// or, with old == out, in place (the asynchronous sweep)
cudaError_t launch_ilu_sweep(const IluDev& d, const double* aS, int32_t K, const double* old,
                             double* out, double omega, cudaStream_t st);
// one FastSpTRSV sweep (Jacobi) with L (unit diagonal) or U on level <= K
cudaError_t launch_ilu_trsv(const IluDev& d, const double* LU, int32_t K, int32_t upper,
                            const double* b, const double* xo, double* x, double omega,
                            cudaStream_t st);

}  // namespace mf
