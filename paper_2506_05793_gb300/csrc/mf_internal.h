// mf_internal.h -- shared host/device declarations of the GB300 multifrontal
// Cholesky library (not part of the public C-ABI).
#pragma once

#include <cstdint>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/mfchol.h"

typedef struct CUstream_st* cudaStream_t;

namespace mf {

// Panel width of the blocked large-front factorization and of the blocked
// solve, the square tile of the trailing update, rows per TRSM block, and the
// column chunk of the large-front assembly.
constexpr int kNB = 64;
constexpr int kTile = 64;
constexpr int kTcTile = 128;  // square tile of the tensor-core trailing update
constexpr int kTrsmRows = 64;
constexpr int kAsmCols = 32;
constexpr int kSmallMax = 128;   // largest front (k+m) of the one-CTA kernel
constexpr int kSolveChunk = 32;  // right-hand sides per solve pass
constexpr int kWarpSolve = 512;  // fronts this small are solved by one warp

// Per-supernode record, read by every kernel (64 bytes).
struct SnInfo {
  int32_t first;        // first (permuted) column
  int32_t k;            // width (pivot columns)
  int32_t m;            // update rows
  int32_t nchild;       // children in the supernodal tree
  int32_t child_begin;  // offset into the children list
  int32_t parent;       // parent supernode or -1
  int64_t Loff;         // L panel offset (elements), (k+m) x k column-major
  int64_t Uoff;         // update matrix offset (elements), m x m column-major
  int64_t rows_off;     // offset into rowidx (k+m global row indices)
  int64_t map_off;      // offset into relmap (m positions in the parent front)
  int64_t woff;         // offset (elements per RHS) of the solve work front
};
static_assert(sizeof(SnInfo) == 64, "SnInfo layout");

// One work item of a batched launch.
struct Item {
  int32_t s, t, a, b;
};

enum Kind : int32_t {
  K_SMALL = 0,     // fused assemble + partial Cholesky of a small front
  K_ASSEMBLE = 1,  // zero + scatter A + extend-add of children (large fronts)
  K_POTRF = 2,     // diagonal block Cholesky
  K_TRSM = 3,      // panel rows * L_tt^{-T}
  K_SYRK = 4,      // trailing lower update
  K_SYRK_TC = 5,   // FP32 trailing update on tcgen05 tensor cores (128 x 128)
  K_NKINDS_FACTOR = 6,
  K_SMALL_Q = 9,     // persistent queue: every small front whose subtree is all small
  K_PINV_INIT = 7,   // partitioned inverse: P = 0, diagonal blocks = their inverses
  K_PINV = 8,        // partitioned inverse, step t: P(i, j) -= L(i, t) P(t, j), i > t >= j
  K_FW_LEVEL = 11,   // per 64-row block: gather, GEMV with solved blocks, diagonal solve
  K_BW_LEVEL = 12,   // per 64-column block: transposed GEMV, diagonal solve
  K_FW_WARP = 13,    // one warp per front with k + m <= kWarpSolve (forward)
  K_BW_WARP = 14,    // one warp per front with k + m <= kWarpSolve (backward)
  K_FW_GEMV = 15,    // per 64 update rows: w -= L21 x1 (after the level's pivots)
  K_BW_GEMV = 16,    // per 64 pivot columns: y -= L21^T x2 (before the chains)
  K_FW_PGATHER = 17, // variant 3: gather the pivot rows' w into the front work vector
  K_FW_PINV = 18,    // variant 3: rows of P times w (x for pivot rows, w update below)
  K_BW_PCOPY = 19,   // variant 3: stage the forward result y of the pivot rows
  K_BW_PINV = 20,    // variant 3: x(cols) = P^T [y; x of the update rows]
  K_PINV_SMALL = 21, // variant 4: partitioned inverse of a front without kept inverses (one CTA)
  K_PT = 22,         // variant 4: PT = P^T per front (64 x 64 tiles)
  K_V4_FW = 23,      // variant 4, forward: one warp per row of the level's matrix
  K_V4_BW = 24,      // variant 4, backward: one warp per pivot column
};

struct Launch {
  int32_t kind;
  int32_t level;
  int32_t count;   // items (= CTAs)
  int32_t param;   // small-front size class (max k+m) or step
  int64_t item_off;
  double flops;    // algorithmic flops of this launch
  // lookahead on levels with few large fronts: `side` launches run on a
  // second stream, overlapping the next panels' factorization; `join` makes
  // the main stream wait for the side stream first.  `area` selects the
  // tensor-core staging area (0: two panel slots, 1: four).
  int8_t side = 0;
  int8_t join = 0;
  int8_t area = 0;
  // K_SYRK: square tile of the FMA trailing update (32, 64 or 128; 0 = 64);
  // K_FW_GEMV: 2 when every front of the launch has at most 128 pivot
  // columns, 1 when at most kFwNarrowK (one CTA per 64 update rows), else 0
  // (four); K_BW_GEMV: CTAs per item (1, 2, 4 or 8: bw_gemv_split of the
  // launch's largest number of update rows)
  uint8_t tile = 0;
};

// Forward update-row product of one right-hand side: launches whose fronts
// have at most this many pivot columns take one CTA per 64 update rows,
// wider ones four
constexpr int kFwNarrowK = 512;
inline int fw_gemv_tile(int maxk) { return maxk <= 2 * kNB ? 2 : maxk <= kFwNarrowK ? 1 : 0; }

// Backward update-row product of one right-hand side: CTAs per 64-column
// item for a launch whose fronts have at most m update rows, so that a warp
// reads at most about 512 rows (1, 2, 4 or 8)
inline int bw_gemv_split(int m) { return m <= 512 ? 1 : m <= 1024 ? 2 : m <= 2048 ? 4 : 8; }

// levels with at most this many large fronts factor with lookahead
constexpr int kLookaheadFronts = 64;
// split-buffer offsets carry the staging area in bit 48 and up
constexpr int kSoffAreaShift = 48;

}  // namespace mf

// Host-side symbolic object.
struct mf_symbolic {
  int64_t n = 0;
  int64_t nnzA = 0;
  std::vector<int64_t> rowptr;
  std::vector<int32_t> colind;
  std::vector<int32_t> perm, iperm;
  std::vector<int32_t> parent;    // column etree
  std::vector<int64_t> colcount;  // c_j
  std::vector<int32_t> sup_ptr;   // nsuper + 1 (fundamental supernodes, exported)
  std::vector<int32_t> col2sn;
  std::vector<int32_t> fs_rowidx;    // rows of each fundamental supernode (lazy)
  std::vector<int64_t> fs_rows_off;  // nsuper + 1 (empty until first needed)
  std::vector<int64_t> low_cp;       // strict lower triangle of C by columns
  std::vector<int32_t> low_cr;
  std::vector<int32_t> fs_parent;    // fundamental supernodal tree
  // fronts: contiguous column ranges after relaxed amalgamation; every
  // numeric structure below (sn, rowidx, relmap, schedules) is per front
  int32_t relax = 1;
  mf_options opt_used{};           // the options the analysis was made with
  std::vector<int32_t> front_ptr;  // nfronts + 1
  std::vector<int32_t> col2front;
  double front_flops = 0.0;        // sum over front columns of (rows)^2
  int64_t nsuper = 0, nnzL = 0, nnz_lower = 0;
  double flops = 0.0;
  int32_t nlevels = 0;
  int64_t max_front = 0, max_k = 0;
  std::vector<mf::SnInfo> sn;
  std::vector<int32_t> children;
  std::vector<int32_t> rowidx;
  std::vector<int32_t> relmap;
  std::vector<int32_t> slevel;
  // assembly of A into the fronts: per permuted column j, entries
  // acol_ptr[j]..acol_ptr[j+1] with front-relative row arow[e] and source
  // CSR positions asrc[asrc_ptr[e] .. asrc_ptr[e+1]) (duplicates summed)
  std::vector<int64_t> acol_ptr;
  std::vector<int32_t> arow;
  std::vector<int64_t> asrc_ptr;
  std::vector<int64_t> asrc;
  int64_t Lsize = 0, Usize = 0, Wsize = 0;
  // launch schedules
  std::vector<mf::Item> items;
  std::vector<mf::Launch> fsched;
  std::vector<mf::Launch> fsched_tc;  // FP32 with tensor-core trailing updates
  std::vector<int64_t> soff;          // per front: first row in the split buffer
  int64_t split_rows = 0;    // staging rows of area 0 (2 panel slots per row)
  int64_t split_rows_b = 0;  // staging rows of area 1 (4 slots, lookahead levels)
  int64_t max_large = 0;              // most large fronts in one level
  // diagonal-block inverses kept for the solve (SpTRSV variant 2): slot of
  // the first 64-column block of each large front (-1 elsewhere), slot count
  bool keep_inv = false;
  std::vector<int64_t> ioff;
  int64_t ninv = 0;
  // partitioned inverse (SpTRSV variant 3): per large front of the solve
  // P = [L11^{-1}; -L21 L11^{-1}] in the layout of L, computed after the
  // factorization (pinv_flops of extra work)
  bool pinv = false;
  double pinv_flops = 0.0;
  // SpTRSV variant 4: per-level sparse products (groups (front, front row)
  // of the forward rows, in the order of the forward items)
  bool v4 = false;
  std::vector<mf::Item> v4_grp;
  std::vector<mf::Item> arange;       // assembly: (child, lo, hi, 0) lists per chunk
  std::vector<mf::Launch> fwsched, bwsched;
  std::vector<int32_t> blkoff;     // per front: first 64-column block index
  // forward-solve gather: entries ginv_ptr[woff+i]..[woff+i+1] of front row
  // i are the global work-vector rows (child woff + child row) added into it
  std::vector<int64_t> ginv_ptr;
  std::vector<int64_t> ginv_src;
  // device mirror, created on first use by a factor on this device
  mutable std::mutex dev_mu;
  mutable std::shared_ptr<void> dev;
  mutable int dev_device = -1;
};

struct mf_handle {
  int device = 0;
  mf_options opt{};
};

namespace mf {
// symbolic.cpp
int analyze(mf_symbolic& S, int64_t n, const int64_t* rowptr, const int32_t* colind,
            const int32_t* perm, const int32_t* node_of, std::string& err);
// update_tile: the per-front-size-bucket trailing-update choice (4 codes,
// mf_options.update_tile) or nullptr for the defaults
void build_schedules(mf_symbolic& S, int small_max, int small_queue, const int32_t* update_tile);
int tile_bucket(int nf);
int check_schedules(const mf_symbolic& S, std::string& err);
void ensure_fundamental_rows(const mf_symbolic& S);
// LU with a symmetric pattern: assembly lists of the strictly upper entries
// of C = P A P^T (entry C(j, i), i > j, goes to row i of column j of the
// front's U^T half), in the format of acol_ptr / arow / asrc_ptr / asrc.
// MF_ERR_INVALID when an upper entry falls outside its front (the pattern
// is not structurally symmetric).
struct UpperAssembly {
  std::vector<int64_t> col_ptr;  // n + 1
  std::vector<int32_t> row;      // front-relative rows
  std::vector<int64_t> src_ptr;  // entries + 1
  std::vector<int64_t> src;      // CSR positions (duplicates summed)
};
int build_upper_assembly(const mf_symbolic& S, UpperAssembly& out, std::string& err);
// error reporting (capi.cpp)
int set_error(int code, const std::string& msg);
// solve with caller-provided work memory (capi.cpp)
int solve_in_scratch(mf_factor* f, int32_t nrhs, const double* B, int64_t ldb, double* X,
                     int64_t ldx, void* scratch, size_t scratch_bytes, cudaStream_t st);
bool factor_ready(const mf_factor* f, int64_t* n);
}  // namespace mf
