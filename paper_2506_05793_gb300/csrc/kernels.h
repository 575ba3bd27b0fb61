// kernels.h -- type-erased argument blocks and launchers of the device
// kernels (factor_kernels.cu, solve_kernels.cu).  Host code in capi.cpp
// fills these and calls the launchers; it never sees a template.
#pragma once

#include <cuda_runtime.h>

#include "mf_internal.h"

namespace mf {

// Device mirror of a symbolic object (read-only during numeric work).
struct DevSym {
  SnInfo* sn = nullptr;
  int32_t* children = nullptr;
  int32_t* relmap = nullptr;
  int32_t* rowidx = nullptr;
  int64_t* acol_ptr = nullptr;
  int32_t* arow = nullptr;
  int64_t* asrc_ptr = nullptr;
  int64_t* asrc = nullptr;
  Item* items = nullptr;
  int32_t* blkoff = nullptr;   // per front: first 64-column block (solve flags)
  int64_t* soff = nullptr;     // per front: first row in the split buffer
  int64_t* ioff = nullptr;     // per front: first diagonal-block inverse slot (or -1)
  Item* arange = nullptr;      // assembly chunks: (child, lo, hi) ranges, sentinel -1
  int64_t* ginv_ptr = nullptr; // forward gather (inverse relative maps)
  int64_t* ginv_src = nullptr;
  int32_t* perm = nullptr;     // perm[new] = old
  int64_t* rowptr = nullptr;   // A (original order) for the FP64 residual
  int32_t* colind = nullptr;
  Item* v4grp = nullptr;       // variant 4: forward row groups (front, front row)
};

struct FactorArgs {
  DevSym sym;
  const double* vals;          // A values, CSR order (device)
  void* av;                    // T[nnz_lower]: lower entries of C in assembly order
  void* L;                     // T[Lsize]
  void* U;                     // T[Usize]
  // [0] = first non-positive pivot column, [1] = MF_ERR_TIMEOUT when a bounded
  // wait of the factorization gave up (both all-ones when clear)
  unsigned long long* status;
  // FP32 tensor-core path: four panel slots per row, each 64 tf32 "hi" then 64 "lo" floats
  // (row soff[front] + front row); nullptr elsewhere
  float* split;
  float* split_b;           // eight-slot staging rows of lookahead levels
  const void* split_map;    // host copy of the TMA tensor map over split (128 bytes)
  const void* split_map_b;  // same over split_b
  // per large front of the level (slot in item field b): 64 x 64 inverse of
  // the current diagonal block of the factor, T
  void* dinv;
  // partitioned inverse P (T[Lsize], layout of L) or nullptr
  void* P = nullptr;
  void* PT = nullptr;  // variant 4: P transposed per front (k x nf, ld k) or nullptr
  // small-front queue: [0] ticket counter, then one completion flag per
  // front (zeroed before the queue launch)
  int* qstate = nullptr;
  int32_t wait_polls = 0;  // polls before a queue wait gives up (0: default)
  void* D = nullptr;       // LDL^T: T[n] pivots by permuted column; nullptr for Cholesky
  // LU with a symmetric pattern (lu != 0): U^T in the layout of L (Lu), the
  // transposed update matrices (Uu), the inverses of the U^T diagonal blocks
  // (dinvu, slots as dinv), the upper entries of C in their own assembly
  // lists (uacol_ptr / uarow, values avu), and with pivoting (lu == 2) the
  // row chosen for each pivot position inside its 64-row block (piv[n])
  int32_t lu = 0;
  void* Lu = nullptr;
  void* Uu = nullptr;
  void* dinvu = nullptr;
  const int64_t* uacol_ptr = nullptr;
  const int32_t* uarow = nullptr;
  void* avu = nullptr;
  uint8_t* piv = nullptr;
  // pivoting: the rows of each later 64-row block of a large front are
  // reordered in the front's earlier columns once the factorization is done
  // (items (front, step), count lu_swap_count)
  const Item* lu_swap = nullptr;
  int32_t lu_swap_count = 0;
  // LDL^T with symmetric pivoting (D and piv set, lu == 0): ipos[r] = the
  // pivot position that row r of P A P^T ended in (int32[n])
  int32_t* ipos = nullptr;
};

struct SolveArgs {
  DevSym sym;
  const void* L;  // T
  void* Y;        // T[n * nrhs]  permuted RHS / solution
  // T[Wsize * nrhs] front work vectors; the pivot rows' slots of the
  // flag-chained fronts carry their solved values, all ones before a sweep
  void* W;
  // int32[2 * nlevels + 1], zero before every solve: one ticket counter per
  // level and sweep
  int32_t* sync;
  unsigned long long* status;  // the solve's timeout record: MF_ERR_TIMEOUT when a wait gives up
  // diagonal-block inverses of the large fronts (slots sym.ioff), or nullptr
  // to solve the pivot blocks by substitution
  const void* dinv = nullptr;
  // partitioned inverse (SpTRSV variants 3, 4), T[Lsize], or nullptr
  const void* P = nullptr;
  const void* PT = nullptr;  // variant 4: P transposed per front
  int64_t n;
  int32_t nrhs;
  int32_t nlevels;
  int32_t wait_polls = 0;  // polls before a wait gives up (0: the default bound)
  // LU with pivoting, forward sweep: pivot position i of a 64-row block
  // takes row (i & ~63) + piv[i] of that block; nullptr elsewhere
  const uint8_t* piv = nullptr;
  // LDL^T with symmetric pivoting (backward sweep and output): the solution
  // of row r of P A P^T sits at position ipos[r]; nullptr elsewhere
  const int32_t* ipos = nullptr;
};

// prec: MF_FP64 or MF_FP32.  All launchers return cudaGetLastError().
cudaError_t factor_kernels_init(int prec);
cudaError_t launch_factor(int prec, const Launch& L, const FactorArgs& a, cudaStream_t st);
// av[e] = sum of the CSR values of lower entry e (duplicates summed), cast to
// T; for LU also avu from the upper entries' lists (src_ptr / src, nnz_upper)
cudaError_t launch_gather_values(int prec, const FactorArgs& a, int64_t nnz_lower, cudaStream_t st);
cudaError_t launch_gather_upper(int prec, const int64_t* src_ptr, const int64_t* src,
                                const double* vals, void* avu, int64_t nnz_upper, cudaStream_t st);
// LU with pivoting: reorder the later pivot blocks' rows in their fronts'
// earlier columns (after the factorization; no-op without pivoting)
cudaError_t launch_lu_swap(int prec, const FactorArgs& a, cudaStream_t st);
// tcgen05 FP32 trailing update (factor_tc.cu)
cudaError_t factor_tc_init();
cudaError_t launch_syrk_tc(const Launch& L, const FactorArgs& a, cudaStream_t st);
// tensor map (128 bytes, written to map_out) over a staging buffer of
// `rows` rows of `width` floats (512 or 1024)
cudaError_t make_split_map(float* split, int64_t rows, int width, void* map_out);
cudaError_t solve_kernels_init(int prec);
// LDL^T solve: Y[i + r n] /= D[i] for the n x nrhs values (between sweeps)
cudaError_t launch_dscale(int prec, void* Y, const void* D, int64_t n, int32_t nrhs,
                          cudaStream_t st);
cudaError_t launch_solve(int prec, const Launch& L, const SolveArgs& a, cudaStream_t st);
cudaError_t launch_wait_probe(const int* flag, unsigned long long* status, int limit,
                              cudaStream_t st);
// FP64 peak probes (diag.cu): kind 0 DFMA, 1 DMMA; out holds blocks x 256
// doubles; peak_fp64_flops gives the flops of one launch
cudaError_t launch_peak_fp64(int kind, double* out, int blocks, int64_t iters, cudaStream_t st);
double peak_fp64_flops(int kind, int blocks, int64_t iters);
int peak_fp64_blocks_per_sm(int kind);  // resident 256-thread blocks per SM

// Y[i, r] = T(scale_r * B[perm[i], r]) with scale_r = inv_scale ? inv_scale[r] : 1.
cudaError_t launch_perm_in(int prec, const double* B, int64_t ldb, const int32_t* perm,
                           void* Y, int64_t n, int32_t nrhs, const double* inv_scale,
                           cudaStream_t st);
// X[perm[i], r] (=|+=) scale_r * Y[i, r]; accumulate != 0 adds.
// X(perm[i], r) = Y(i, r) (ipos: Y(ipos[i], r), LDL^T with symmetric pivoting)
cudaError_t launch_perm_out(int prec, const void* Y, const int32_t* perm, const int32_t* ipos,
                            double* X, int64_t ldx, int64_t n, int32_t nrhs, const double* scale,
                            int32_t accumulate, cudaStream_t st);

// FP64 residual R = B - A X (A in original order), with per-RHS maxima of
// |R|, |X| accumulated into rnorm[r], xnorm[r] (must be zeroed before).
// nnz_hint: entries of A (the lanes per row follow the mean row length)
cudaError_t launch_residual(const int64_t* rowptr, const int32_t* colind, const double* vals,
                            int64_t n, int64_t nnz_hint, const double* B, int64_t ldb,
                            const double* X, int64_t ldx, double* R, int32_t nrhs, double* rnorm,
                            double* xnorm, cudaStream_t st);
// out[0] = max_i sum_j |A_ij|; out[1 + r] = max_i |B_ir|  (out zeroed before)
cudaError_t launch_norms(const int64_t* rowptr, const double* vals, int64_t n,
                         const double* B, int64_t ldb, int32_t nrhs, double* out,
                         cudaStream_t st);

}  // namespace mf
