// noalloc.cu -- solve entry point that allocates no memory.
//
// mf_solve allocates its work buffers on first use and stages host
// pointers through device copies.  Some callers cannot allow that on their
// solve path; mf_solve_noalloc instead runs the same solve kernels with
// their work memory carved out of one fixed device array defined here.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "kernels.h"
#include "mf_internal.h"

namespace {

constexpr size_t kScratchBytes = (size_t)32 << 20;  // 32 MiB

// Work memory of mf_solve_noalloc.  Every GPU that loads this library holds
// it until the process exits.  Host code must not use the name as a device
// address: the address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_solve_scratch[kScratchBytes];

constexpr int kMaxDevices = 128;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of g_solve_scratch on the current device, looked up once
// per device (with that device current) and cached.
int scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess)
    return mf::set_error(MF_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return mf::set_error(MF_ERR_INVALID, "device index out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_solve_scratch);
    if (e != cudaSuccess || p == nullptr)
      return mf::set_error(MF_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return MF_OK;
}

}  // namespace

extern "C" int mf_solve_noalloc(mf_factor* f, int32_t nrhs, const double* B, int64_t ldb,
                                double* X, int64_t ldx, void* stream) {
  if (!f) return mf::set_error(MF_ERR_INVALID, "NULL factor");
  int64_t n = 0;
  const bool ready = mf::factor_ready(f, &n);
  if (nrhs < 0 || ldb < n || ldx < n || (nrhs > 0 && n > 0 && (!B || !X)))
    return mf::set_error(MF_ERR_INVALID, "invalid solve arguments");
  if (nrhs == 0 || n == 0) return MF_OK;
  void* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc != MF_OK) return rc;
  if (!ready) return mf::set_error(MF_ERR_INVALID, "factor has no numeric values");
  return mf::solve_in_scratch(f, nrhs, B, ldb, X, ldx, scratch, kScratchBytes,
                              static_cast<cudaStream_t>(stream));
}
