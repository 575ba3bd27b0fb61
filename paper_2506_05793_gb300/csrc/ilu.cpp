// ilu.cpp -- FastILU and FastSpTRSV (paper Sec. 6): the ILU(k) pattern on the
// host, the sweeps on the device (ilu_kernels.cu), behind the C-ABI.
//
// Symbolic: the ILU(k) pattern by levels of fill.  Entries of A and the
// diagonal have level 0; row i meets the rows k < i of its pattern in
// increasing order (a priority queue of the columns still to eliminate),
// and every entry (k, j), j > k, of a finished row k gives (i, j) the level
// lev(i, k) + lev(k, j) + 1 if that is lower; entries of level <= k are kept.
// The pattern keeps every entry's level, so the warm-up (FastILU(k-1) first)
// runs on the same arrays restricted to the lower levels.
#include <cuda_runtime.h>

#include <algorithm>
#include <functional>
#include <new>
#include <queue>
#include <string>
#include <vector>

#include "ilu.h"
#include "mf_internal.h"

using mf::set_error;

#define ILU_CK(x)                                                                         \
  do {                                                                                    \
    cudaError_t e_ = (x);                                                                 \
    if (e_ != cudaSuccess)                                                                \
      return set_error(e_ == cudaErrorMemoryAllocation ? MF_ERR_OOM : MF_ERR_CUDA,       \
                       std::string(#x) + ": " + cudaGetErrorString(e_));                  \
  } while (0)

struct mf_ilu {
  int64_t n = 0, nnzA = 0;
  int32_t level = 0;
  std::vector<int64_t> Sp, diag, cp, cq, a_ptr, a_src;
  std::vector<int32_t> Sj, Si, Slev, cr;
  mf::IluDev d;
  std::vector<void*> dev;    // device arrays of the pattern
  double* vals = nullptr;    // A's values (CSR order)
  double* aS = nullptr;      // A on S
  double* F[2] = {nullptr, nullptr};
  int cur = 0;               // which of F holds the factors
  double* xw[3] = {nullptr, nullptr, nullptr};  // solve work: two iterates, z
  double* io[2] = {nullptr, nullptr};           // host-pointer staging of b, x
  bool numeric_done = false;
  ~mf_ilu() {
    for (void* p : dev) cudaFree(p);
    cudaFree(vals);
    cudaFree(aS);
    for (double* p : F) cudaFree(p);
    for (double* p : xw) cudaFree(p);
    for (double* p : io) cudaFree(p);
  }
};

namespace {

int iluk_symbolic(mf_ilu& I, int64_t n, const int64_t* rp, const int32_t* ci, int32_t K) {
  constexpr int32_t kNone = -1;
  std::vector<int32_t> lev(n, kNone), cols;
  std::priority_queue<int32_t, std::vector<int32_t>, std::greater<int32_t>> pending;
  I.Sp.assign(n + 1, 0);
  for (int64_t i = 0; i < n; ++i) {
    cols.clear();
    auto meet = [&](int32_t j, int32_t l) {
      if (lev[j] == kNone) {
        lev[j] = l;
        cols.push_back(j);
        if (j < i) pending.push(j);
      } else if (l < lev[j]) {
        lev[j] = l;
      }
    };
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) meet(ci[p], 0);
    meet((int32_t)i, 0);
    while (!pending.empty()) {
      const int32_t k = pending.top();
      pending.pop();
      const int32_t lk = lev[k];
      for (int64_t q = I.diag[k] + 1; q < I.Sp[k + 1]; ++q) {
        const int32_t l = lk + I.Slev[q] + 1;
        if (l <= K) meet(I.Sj[q], l);
      }
    }
    std::sort(cols.begin(), cols.end());
    for (int32_t j : cols) {
      if (j == i) I.diag.push_back((int64_t)I.Sj.size());
      I.Sj.push_back(j);
      I.Si.push_back((int32_t)i);
      I.Slev.push_back(lev[j]);
      lev[j] = kNone;
    }
    I.Sp[i + 1] = (int64_t)I.Sj.size();
  }
  const int64_t nnz = (int64_t)I.Sj.size();
  // columns of S, rows increasing
  I.cp.assign(n + 1, 0);
  for (int64_t q = 0; q < nnz; ++q) I.cp[I.Sj[q] + 1]++;
  for (int64_t j = 0; j < n; ++j) I.cp[j + 1] += I.cp[j];
  I.cr.resize(nnz);
  I.cq.resize(nnz);
  std::vector<int64_t> fill(I.cp.begin(), I.cp.end() - 1);
  for (int64_t q = 0; q < nnz; ++q) {
    const int64_t at = fill[I.Sj[q]]++;
    I.cr[at] = I.Si[q];
    I.cq[at] = q;
  }
  // gather of A's entries onto S (duplicates summed in CSR order)
  std::vector<int64_t> cnt(nnz + 1, 0), where(rp[n]);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      const int64_t lo = I.Sp[i];
      const int32_t* row = I.Sj.data() + lo;
      const int64_t len = I.Sp[i + 1] - lo;
      const int64_t at = lo + (std::lower_bound(row, row + len, ci[p]) - row);
      where[p] = at;
      cnt[at + 1]++;
    }
  for (int64_t q = 0; q < nnz; ++q) cnt[q + 1] += cnt[q];
  I.a_ptr = cnt;
  I.a_src.resize(rp[n]);
  for (int64_t p = 0; p < rp[n]; ++p) I.a_src[cnt[where[p]]++] = p;
  return MF_OK;
}

template <typename V>
cudaError_t upload(mf_ilu& I, const V** dst, const std::vector<V>& src) {
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, std::max<size_t>(src.size(), 1) * sizeof(V));
  if (e != cudaSuccess) return e;
  I.dev.push_back(p);
  *dst = static_cast<const V*>(p);
  if (src.empty()) return cudaSuccess;
  return cudaMemcpy(p, src.data(), src.size() * sizeof(V), cudaMemcpyHostToDevice);
}

}  // namespace

extern "C" {

int mf_ilu_symbolic(mf_handle* h, int64_t n, const int64_t* rowptr, const int32_t* colind,
                    int32_t level, mf_ilu** out) {
  if (!h || !out || !rowptr || n < 0 || n >= (int64_t)INT32_MAX || level < 0)
    return set_error(MF_ERR_INVALID, "invalid ILU(k) arguments");
  *out = nullptr;
  if (rowptr[0] != 0) return set_error(MF_ERR_INVALID, "rowptr[0] != 0");
  for (int64_t i = 0; i < n; ++i)
    if (rowptr[i + 1] < rowptr[i]) return set_error(MF_ERR_INVALID, "rowptr is decreasing");
  if (rowptr[n] > 0 && !colind) return set_error(MF_ERR_INVALID, "colind is NULL");
  for (int64_t p = 0; p < rowptr[n]; ++p)
    if (colind[p] < 0 || colind[p] >= n) return set_error(MF_ERR_INVALID, "colind out of range");
  mf_ilu* I = new (std::nothrow) mf_ilu();
  if (!I) return set_error(MF_ERR_OOM, "host allocation failed");
  I->n = n;
  I->nnzA = rowptr[n];
  I->level = level;
  try {
    iluk_symbolic(*I, n, rowptr, colind, level);
  } catch (const std::bad_alloc&) {
    delete I;
    return set_error(MF_ERR_OOM, "host allocation failed");
  }
  I->d.n = n;
  I->d.nnz = (int64_t)I->Sj.size();
  *out = I;
  return MF_OK;
}

}  // extern "C"

// Device copy of S and the sweeps' work memory, made by the first numeric
// call (the symbolic phase is host-only).
static int ensure_device(mf_ilu* I) {
  if (I->aS) return MF_OK;
  const int64_t n = I->n;
  cudaError_t e = upload(*I, &I->d.Sp, I->Sp);
  if (e == cudaSuccess) e = upload(*I, &I->d.Sj, I->Sj);
  if (e == cudaSuccess) e = upload(*I, &I->d.Si, I->Si);
  if (e == cudaSuccess) e = upload(*I, &I->d.Slev, I->Slev);
  if (e == cudaSuccess) e = upload(*I, &I->d.diag, I->diag);
  if (e == cudaSuccess) e = upload(*I, &I->d.cp, I->cp);
  if (e == cudaSuccess) e = upload(*I, &I->d.cr, I->cr);
  if (e == cudaSuccess) e = upload(*I, &I->d.cq, I->cq);
  if (e == cudaSuccess) e = upload(*I, &I->d.a_ptr, I->a_ptr);
  if (e == cudaSuccess) e = upload(*I, &I->d.a_src, I->a_src);
  const size_t nz = std::max<int64_t>(I->d.nnz, 1) * sizeof(double);
  if (e == cudaSuccess) e = cudaMalloc(&I->vals, std::max<int64_t>(I->nnzA, 1) * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&I->aS, nz);
  if (e == cudaSuccess) e = cudaMalloc(&I->F[0], nz);
  if (e == cudaSuccess) e = cudaMalloc(&I->F[1], nz);
  for (int k = 0; k < 3 && e == cudaSuccess; ++k)
    e = cudaMalloc(&I->xw[k], std::max<int64_t>(n, 1) * sizeof(double));
  for (int k = 0; k < 2 && e == cudaSuccess; ++k)
    e = cudaMalloc(&I->io[k], std::max<int64_t>(n, 1) * sizeof(double));
  if (e != cudaSuccess) {
    cudaFree(I->aS);
    I->aS = nullptr;
    return set_error(e == cudaErrorMemoryAllocation ? MF_ERR_OOM : MF_ERR_CUDA,
                     std::string("ILU(k) device setup: ") + cudaGetErrorString(e));
  }
  return MF_OK;
}

extern "C" {

int mf_ilu_info(const mf_ilu* I, int64_t* n, int64_t* nnz) {
  if (!I) return set_error(MF_ERR_INVALID, "NULL ILU");
  if (n) *n = I->n;
  if (nnz) *nnz = I->d.nnz;
  return MF_OK;
}

int mf_ilu_pattern(const mf_ilu* I, int64_t* Sp, int32_t* Sj, int32_t* Slev) {
  if (!I || !Sp) return set_error(MF_ERR_INVALID, "NULL argument");
  std::copy(I->Sp.begin(), I->Sp.end(), Sp);
  if (Sj) std::copy(I->Sj.begin(), I->Sj.end(), Sj);
  if (Slev) std::copy(I->Slev.begin(), I->Slev.end(), Slev);
  return MF_OK;
}

int mf_ilu_numeric(mf_ilu* I, const double* values, int32_t values_on_device, int32_t sweeps,
                   double omega, double shift, int32_t warmup, int32_t in_place, void* stream) {
  if (!I || (!values && I->nnzA) || sweeps < 0 || !(omega > 0.0) || omega > 1.0)
    return set_error(MF_ERR_INVALID, "invalid FastILU arguments");
  const int rc0 = ensure_device(I);
  if (rc0 != MF_OK) return rc0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (I->nnzA)
    ILU_CK(cudaMemcpyAsync(I->vals, values, I->nnzA * sizeof(double),
                           values_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  ILU_CK(mf::launch_ilu_gather(I->d, I->vals, shift, I->aS, st));
  // warm-up: FastILU(0), then each level from the one below it
  const int32_t first = warmup ? 0 : I->level;
  int cur = 0;
  for (int32_t K = first; K <= I->level; ++K) {
    if (K == first) {
      ILU_CK(mf::launch_ilu_init(I->d, I->aS, K, 0, I->F[cur], st));
    } else {
      ILU_CK(mf::launch_ilu_init(I->d, I->aS, K, 1, I->F[cur], st));
    }
    for (int32_t s = 0; s < sweeps; ++s) {
      if (in_place) {
        ILU_CK(mf::launch_ilu_sweep(I->d, I->aS, K, I->F[cur], I->F[cur], omega, st));
      } else {
        ILU_CK(mf::launch_ilu_sweep(I->d, I->aS, K, I->F[cur], I->F[1 - cur], omega, st));
        cur = 1 - cur;
      }
    }
  }
  I->cur = cur;
  I->numeric_done = true;
  return MF_OK;
}

int mf_ilu_export(const mf_ilu* I, double* LU) {
  if (!I || (!LU && I->d.nnz)) return set_error(MF_ERR_INVALID, "NULL argument");
  if (!I->numeric_done) return set_error(MF_ERR_INVALID, "no numeric FastILU yet");
  ILU_CK(cudaDeviceSynchronize());
  if (I->d.nnz)
    ILU_CK(cudaMemcpy(LU, I->F[I->cur], I->d.nnz * sizeof(double), cudaMemcpyDeviceToHost));
  return MF_OK;
}

static int trsv_dev(mf_ilu* I, int32_t upper, int32_t sweeps, double omega, const double* b,
                    double* x, cudaStream_t st) {
  // Jacobi from x = 0: iterates alternate between two work vectors; the last
  // one is copied to x
  const size_t bytes = I->n * sizeof(double);
  ILU_CK(cudaMemsetAsync(I->xw[0], 0, bytes, st));
  int c = 0;
  for (int32_t s = 0; s < sweeps; ++s) {
    ILU_CK(mf::launch_ilu_trsv(I->d, I->F[I->cur], I->level, upper, b, I->xw[c], I->xw[1 - c],
                               omega, st));
    c = 1 - c;
  }
  ILU_CK(cudaMemcpyAsync(x, I->xw[c], bytes, cudaMemcpyDeviceToDevice, st));
  return MF_OK;
}

static int with_io(mf_ilu* I, const double* b, double* x, int32_t on_device, cudaStream_t st,
                   const std::function<int(const double*, double*)>& body) {
  if (on_device) return body(b, x);
  const size_t bytes = I->n * sizeof(double);
  ILU_CK(cudaMemcpyAsync(I->io[0], b, bytes, cudaMemcpyHostToDevice, st));
  const int rc = body(I->io[0], I->io[1]);
  if (rc != MF_OK) return rc;
  ILU_CK(cudaMemcpyAsync(x, I->io[1], bytes, cudaMemcpyDeviceToHost, st));
  ILU_CK(cudaStreamSynchronize(st));
  return MF_OK;
}

int mf_ilu_trsv(mf_ilu* I, int32_t upper, int32_t sweeps, double omega, const double* b, double* x,
                int32_t on_device, void* stream) {
  if (!I || ((!b || !x) && I->n) || sweeps < 0 || !(omega > 0.0) || omega > 1.0)
    return set_error(MF_ERR_INVALID, "invalid FastSpTRSV arguments");
  if (!I->numeric_done) return set_error(MF_ERR_INVALID, "no numeric FastILU yet");
  if (I->n == 0) return MF_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return with_io(I, b, x, on_device, st, [&](const double* bd, double* xd) {
    return trsv_dev(I, upper ? 1 : 0, sweeps, omega, bd, xd, st);
  });
}

int mf_ilu_apply(mf_ilu* I, int32_t sweeps, double omega, const double* b, double* x,
                 int32_t on_device, void* stream) {
  if (!I || ((!b || !x) && I->n) || sweeps < 0 || !(omega > 0.0) || omega > 1.0)
    return set_error(MF_ERR_INVALID, "invalid FastILU apply arguments");
  if (!I->numeric_done) return set_error(MF_ERR_INVALID, "no numeric FastILU yet");
  if (I->n == 0) return MF_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return with_io(I, b, x, on_device, st, [&](const double* bd, double* xd) {
    const int rc = trsv_dev(I, 0, sweeps, omega, bd, I->xw[2], st);  // z = L^-1 b
    if (rc != MF_OK) return rc;
    return trsv_dev(I, 1, sweeps, omega, I->xw[2], xd, st);        // x = U^-1 z
  });
}

int mf_ilu_free(mf_ilu* I) {
  delete I;
  return MF_OK;
}

}  // extern "C"
