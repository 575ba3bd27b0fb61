// capi.cpp -- the extern "C" boundary (include/mfchol.h): handles, symbolic
// objects, device factors, solves and the mixed-precision refinement loop.
//
// Phases follow the paper's Ax=b statement (Sec. 3): symbolic analysis on
// the host, numerical setup (copy values, factor) and solve on the device.
// Every step of the numeric path runs in this library's kernels; there is no
// CPU fallback.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "kernels.h"
#include "mf_internal.h"

namespace {
thread_local std::string g_err;
thread_local int64_t g_errcol = -1;
}  // namespace

namespace mf {
int set_error(int code, const std::string& msg) {
  g_err = msg;
  if (code != MF_ERR_NOT_SPD) g_errcol = -1;
  return code;
}
}  // namespace mf

using mf::set_error;

#define MF_CK(x)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (x);                                                                 \
    if (e_ != cudaSuccess)                                                                \
      return set_error(e_ == cudaErrorMemoryAllocation ? MF_ERR_OOM : MF_ERR_CUDA,       \
                       std::string(#x) + ": " + cudaGetErrorString(e_));                  \
  } while (0)

namespace {

// Device copy of the symbolic structures; freed with the last user.
struct DevSymOwner {
  mf::DevSym d;
  std::vector<void*> allocs;
  ~DevSymOwner() {
    for (void* p : allocs) cudaFree(p);
  }
  template <typename V>
  cudaError_t up(V** dst, const std::vector<V>& src) {
    *dst = nullptr;
    if (src.empty()) return cudaSuccess;
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, src.size() * sizeof(V));
    if (e != cudaSuccess) return e;
    allocs.push_back(p);
    *dst = static_cast<V*>(p);
    return cudaMemcpy(p, src.data(), src.size() * sizeof(V), cudaMemcpyHostToDevice);
  }
};

int get_devsym(const mf_symbolic* S, std::shared_ptr<DevSymOwner>& out) {
  int dev = 0;
  MF_CK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(S->dev_mu);
  if (S->dev && S->dev_device == dev) {
    out = std::static_pointer_cast<DevSymOwner>(S->dev);
    return MF_OK;
  }
  auto o = std::make_shared<DevSymOwner>();
  MF_CK(o->up(&o->d.sn, S->sn));
  MF_CK(o->up(&o->d.children, S->children));
  MF_CK(o->up(&o->d.relmap, S->relmap));
  MF_CK(o->up(&o->d.rowidx, S->rowidx));
  MF_CK(o->up(&o->d.acol_ptr, S->acol_ptr));
  MF_CK(o->up(&o->d.arow, S->arow));
  MF_CK(o->up(&o->d.asrc_ptr, S->asrc_ptr));
  MF_CK(o->up(&o->d.asrc, S->asrc));
  MF_CK(o->up(&o->d.items, S->items));
  MF_CK(o->up(&o->d.blkoff, S->blkoff));
  MF_CK(o->up(&o->d.soff, S->soff));
  MF_CK(o->up(&o->d.ioff, S->ioff));
  MF_CK(o->up(&o->d.arange, S->arange));
  MF_CK(o->up(&o->d.ginv_ptr, S->ginv_ptr));
  MF_CK(o->up(&o->d.ginv_src, S->ginv_src));
  MF_CK(o->up(&o->d.perm, S->perm));
  MF_CK(o->up(&o->d.rowptr, S->rowptr));
  MF_CK(o->up(&o->d.colind, S->colind));
  MF_CK(o->up(&o->d.v4grp, S->v4_grp));
  S->dev = o;
  S->dev_device = dev;
  out = o;
  return MF_OK;
}

// NVTX range over one API phase (symbolic analysis, numeric factorization,
// solve, refined solve), visible in timeline profilers; a no-op unless a
// tool is attached.
struct PhaseRange {
  explicit PhaseRange(const char* name) { nvtxRangePushA(name); }
  ~PhaseRange() { nvtxRangePop(); }
  PhaseRange(const PhaseRange&) = delete;
  PhaseRange& operator=(const PhaseRange&) = delete;
};

size_t elem_size(int prec) { return prec == MF_FP32 ? sizeof(float) : sizeof(double); }

constexpr int kStatusWords = 4;
constexpr int kStatusSolve = 2;  // the solve's timeout record

// Device bytes of one factor: L, update matrices, diagonal-block inverses,
// values in assembly order and the CSR values (plus the partitioned inverse,
// the size of L, for SpTRSV variant 3); FP32 adds the tensor-core
// staging rows (two panels of 64 hi + 64 lo floats per row).
int64_t factor_bytes(const mf_symbolic* S, int prec) {
  const int64_t inv_slots = S->keep_inv ? S->ninv : S->max_large;
  return (S->Lsize * (S->v4 ? 3 : S->pinv ? 2 : 1) + S->Usize + inv_slots * mf::kNB * mf::kNB +
          S->nnz_lower) *
             (int64_t)elem_size(prec) +
         S->nnzA * (int64_t)sizeof(double) +
         (prec == MF_FP32 ? (std::max<int64_t>(S->split_rows, 1) * 512 +
                             std::max<int64_t>(S->split_rows_b, 1) * 1024) *
                                (int64_t)sizeof(float)
                          : 0);
}

}  // namespace

struct mf_factor {
  mf_handle* h = nullptr;
  const mf_symbolic* S = nullptr;
  int prec = MF_FP64;
  std::shared_ptr<DevSymOwner> ds;
  void* L = nullptr;
  void* U = nullptr;
  double* vals = nullptr;
  unsigned long long* status = nullptr;
  unsigned long long* status_host = nullptr;
  // solve work
  void* Y = nullptr;
  void* W = nullptr;
  double* Bd = nullptr;
  double* Xd = nullptr;
  double* Rd = nullptr;
  int64_t io_cap = 0;  // doubles in each of Bd/Xd/Rd
  int32_t* sync = nullptr;  // solve ticket counters and block flags
  bool tc = false;          // FP32 trailing updates on tcgen05 tensor cores
  float* split = nullptr;   // tf32 hi/lo staging rows of the panels
  float* split_b = nullptr; // four-slot staging rows of lookahead levels
  alignas(128) unsigned char split_map[128];    // TMA tensor map over split
  alignas(128) unsigned char split_map_b[128];  // TMA tensor map over split_b
  // enqueue_factor runs on two internal streams forked from the caller's:
  // the critical path (panels, first tile columns) at high priority and the
  // lookahead bulk updates at low priority, so that freed SM slots go to the
  // critical path first
  cudaStream_t crit = nullptr, side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_side = nullptr, ev_in = nullptr, ev_out = nullptr;
  void* dinv = nullptr;     // inverses of the current diagonal blocks (scratch)
  void* P = nullptr;        // partitioned inverse (SpTRSV variants 3, 4), layout of L
  void* PT = nullptr;       // variant 4: P transposed front by front
  void* av = nullptr;       // lower entries of C in assembly order (T)
  int* qstate = nullptr;    // small-front queue: ticket, then one flag per front
  bool ldlt = false;        // LDL^T (unit L, pivots in D) instead of Cholesky
  void* Dp = nullptr;       // LDL^T pivots by permuted column (T[n])
  // LU with a symmetric pattern: 1 without pivoting, 2 with pivots looked
  // for within the diagonal blocks
  int lu = 0;
  void* Lu = nullptr;         // U^T in the layout of L (T[Lsize])
  void* dinvu = nullptr;      // inverses of the U^T diagonal blocks (slots of dinv)
  void* avu = nullptr;        // strictly upper entries of C in assembly order (T)
  int64_t* uacol_ptr = nullptr;  // their assembly lists (n + 1 / entries / entries + 1 / sources)
  int32_t* uarow = nullptr;
  int64_t* uasrc_ptr = nullptr;
  int64_t* uasrc = nullptr;
  int64_t nnz_upper = 0;
  uint8_t* piv = nullptr;     // pivoting: row taken by each pivot position of its 64-row block
  mf::Item* lu_swap = nullptr;  // pivoting: (front, step) of the later pivot blocks of large fronts
  int32_t lu_swap_count = 0;
  bool sympiv = false;        // LDL^T with symmetric pivoting within the diagonal blocks
  int32_t* ipos = nullptr;    // symmetric pivoting: position each row of P A P^T ended in
  double* small = nullptr;  // per-RHS scalars for refinement
  // graph of the numeric factorization
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  // profiling
  std::vector<cudaEvent_t> ev;
  double prof_ms[mf::K_NKINDS_FACTOR] = {0};
  int64_t prof_n[mf::K_NKINDS_FACTOR] = {0};
  double prof_fl[mf::K_NKINDS_FACTOR] = {0};
  bool numeric_done = false;
  int32_t wait_polls = 0;     // bound of the solve's flag waits (0: the default)
  mf_factor* fb64 = nullptr;  // FP64 fallback of the refinement loop

  ~mf_factor() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    cudaFree(L);
    cudaFree(U);
    cudaFree(vals);
    cudaFree(status);
    if (status_host) cudaFreeHost(status_host);
    cudaFree(Y);
    cudaFree(W);
    cudaFree(Bd);
    cudaFree(Xd);
    cudaFree(Rd);
    cudaFree(small);
    cudaFree(sync);
    cudaFree(split);
    cudaFree(split_b);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_side) cudaEventDestroy(ev_side);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (side) cudaStreamDestroy(side);
    if (crit) cudaStreamDestroy(crit);
    cudaFree(dinv);
    cudaFree(P);
    cudaFree(PT);
    cudaFree(av);
    cudaFree(qstate);
    cudaFree(Dp);
    cudaFree(Lu);
    cudaFree(dinvu);
    cudaFree(avu);
    cudaFree(uacol_ptr);
    cudaFree(uarow);
    cudaFree(uasrc_ptr);
    cudaFree(uasrc);
    cudaFree(piv);
    cudaFree(lu_swap);
    cudaFree(ipos);
    delete fb64;
  }
};

extern "C" {

int mf_options_default(mf_options* opt) {
  if (!opt) return set_error(MF_ERR_INVALID, "opt is NULL");
  std::memset(opt, 0, sizeof(*opt));
  opt->small_front_max = mf::kSmallMax;
  opt->use_graphs = 1;
  opt->profile = 0;
  opt->relax = 1;
  opt->sptrsv = 2;
  opt->small_queue = 1;
  opt->tc = 1;
  opt->budget_bytes = 0;
  return MF_OK;
}

int mf_create(mf_handle** h, const mf_options* opt) {
  if (!h) return set_error(MF_ERR_INVALID, "h is NULL");
  *h = nullptr;
  mf_handle* H = new (std::nothrow) mf_handle();
  if (!H) return set_error(MF_ERR_OOM, "host allocation failed");
  if (opt) H->opt = *opt; else mf_options_default(&H->opt);
  if (H->opt.small_front_max <= 0 || H->opt.small_front_max > mf::kSmallMax)
    H->opt.small_front_max = mf::kSmallMax;
  if (H->opt.sptrsv == 0) H->opt.sptrsv = 1;  // zero-filled options: substitution
  if (H->opt.sptrsv < 1 || H->opt.sptrsv > 4) {
    delete H;
    return set_error(MF_ERR_INVALID, "sptrsv must be 1, 2, 3 or 4");
  }
  // The symbolic phase is host-only, so a handle is usable without a GPU;
  // device calls report MF_ERR_CUDA later if no device is present.
  if (cudaGetDevice(&H->device) != cudaSuccess) {
    H->device = -1;
    cudaGetLastError();
  }
  *h = H;
  return MF_OK;
}

int mf_destroy(mf_handle* h) {
  delete h;
  return MF_OK;
}

const char* mf_last_error_string(void) { return g_err.c_str(); }
int64_t mf_last_error_column(void) { return g_errcol; }

// ---------------------------------------------------------------------------
// Symbolic
// ---------------------------------------------------------------------------
static int analyze_common(mf_handle* h, int64_t n, const int64_t* rowptr,
                          const int32_t* colind, const int32_t* perm, const int32_t* node_of,
                          mf_symbolic** s) {
  PhaseRange range_("mf_symbolic_analyze");
  if (!h || !s) return set_error(MF_ERR_INVALID, "NULL handle or output");
  *s = nullptr;
  mf_symbolic* S = new (std::nothrow) mf_symbolic();
  if (!S) return set_error(MF_ERR_OOM, "host allocation failed");
  std::string err;
  int rc;
  S->relax = h->opt.relax ? 1 : 0;
  S->opt_used = h->opt;
  S->keep_inv = h->opt.sptrsv >= 2;
  S->pinv = h->opt.sptrsv >= 3;
  S->v4 = h->opt.sptrsv == 4;
  try {
    rc = mf::analyze(*S, n, rowptr, colind, perm, node_of, err);
    if (rc == MF_OK)
      mf::build_schedules(*S, h->opt.small_front_max, h->opt.small_queue, h->opt.update_tile);
  } catch (const std::bad_alloc&) {
    rc = MF_ERR_OOM;
    err = "host allocation failed";
  }
  if (rc != MF_OK) {
    delete S;
    return set_error(rc, err);
  }
  *s = S;
  return MF_OK;
}

int mf_symbolic_analyze(mf_handle* h, int64_t n, const int64_t* rowptr, const int32_t* colind,
                        const int32_t* perm, mf_symbolic** s) {
  return analyze_common(h, n, rowptr, colind, perm, nullptr, s);
}

int mf_symbolic_analyze_condensed(mf_handle* h, int64_t n, const int64_t* rowptr,
                                  const int32_t* colind, const int32_t* perm,
                                  const int32_t* node_of, int32_t block, mf_symbolic** s) {
  if (!h || !s) return set_error(MF_ERR_INVALID, "NULL handle or output");
  *s = nullptr;
  if (node_of) return analyze_common(h, n, rowptr, colind, perm, node_of, s);
  if (block < 1) return set_error(MF_ERR_INVALID, "block must be >= 1 without node_of");
  if (n < 0 || n >= (int64_t)INT32_MAX) return set_error(MF_ERR_INVALID, "n out of range");
  std::vector<int32_t> nodes;
  try {
    nodes.resize(n);
  } catch (const std::bad_alloc&) {
    return set_error(MF_ERR_OOM, "host allocation failed");
  }
  for (int64_t i = 0; i < n; ++i) nodes[i] = (int32_t)(i / block);
  return analyze_common(h, n, rowptr, colind, perm, nodes.data(), s);
}

int mf_symbolic_analyze_batch(mf_handle* h, int32_t count, const int64_t* ns,
                              const int64_t* const* rowptrs, const int32_t* const* colinds,
                              const int32_t* const* perms, mf_symbolic** s) {
  if (!h || !s || count < 0 || (count > 0 && (!ns || !rowptrs || !colinds)))
    return set_error(MF_ERR_INVALID, "invalid batch arguments");
  int64_t N = 0, NNZ = 0;
  for (int32_t b = 0; b < count; ++b) {
    if (ns[b] < 0 || !rowptrs[b]) return set_error(MF_ERR_INVALID, "invalid batch member");
    N += ns[b];
    NNZ += rowptrs[b][ns[b]];
  }
  if (N >= (int64_t)INT32_MAX) return set_error(MF_ERR_INVALID, "batch too large");
  std::vector<int64_t> rp;
  std::vector<int32_t> ci, pm;
  try {
    rp.reserve(N + 1);
    ci.reserve(NNZ);
    pm.reserve(N);
  } catch (const std::bad_alloc&) {
    return set_error(MF_ERR_OOM, "host allocation failed");
  }
  rp.push_back(0);
  int64_t off = 0;
  for (int32_t b = 0; b < count; ++b) {
    const int64_t n = ns[b];
    const int64_t* r = rowptrs[b];
    if (r[0] != 0) return set_error(MF_ERR_INVALID, "batch member rowptr[0] != 0");
    for (int64_t i = 0; i < n; ++i) {
      if (r[i + 1] < r[i]) return set_error(MF_ERR_INVALID, "batch member rowptr decreasing");
      for (int64_t p = r[i]; p < r[i + 1]; ++p) {
        const int32_t c = colinds[b][p];
        if (c < 0 || c >= n) return set_error(MF_ERR_INVALID, "batch member colind out of range");
        ci.push_back((int32_t)(c + off));
      }
      rp.push_back((int64_t)ci.size());
    }
    for (int64_t i = 0; i < n; ++i) {
      const int32_t o = (perms && perms[b]) ? perms[b][i] : (int32_t)i;
      if (o < 0 || o >= n) return set_error(MF_ERR_INVALID, "batch member perm out of range");
      pm.push_back((int32_t)(o + off));
    }
    off += n;
  }
  return mf_symbolic_analyze(h, N, rp.data(), ci.data(), pm.data(), s);
}

int mf_symbolic_check(const mf_symbolic* s) {
  if (!s) return set_error(MF_ERR_INVALID, "NULL argument");
  std::string err;
  const int rc = mf::check_schedules(*s, err);
  return rc == MF_OK ? MF_OK : set_error(rc, err);
}

int mf_symbolic_free(mf_symbolic* s) {
  delete s;
  return MF_OK;
}

int mf_symbolic_get_info(const mf_symbolic* s, mf_symbolic_info* info) {
  if (!s || !info) return set_error(MF_ERR_INVALID, "NULL argument");
  info->n = s->n;
  info->nnz_lower = s->nnz_lower;
  info->nsuper = s->nsuper;
  info->nnz_L = s->nnzL;
  info->flops = s->flops;
  info->nlevels = s->nlevels;
  info->max_front = s->max_front;
  info->max_k = s->max_k;
  info->factor_bytes_fp64 = factor_bytes(s, MF_FP64);
  info->factor_bytes_fp32 = factor_bytes(s, MF_FP32);
  info->nfronts = (int64_t)s->sn.size();
  info->front_flops = s->front_flops;
  info->queued_fronts = (!s->fsched.empty() && s->fsched[0].kind == mf::K_SMALL_Q)
                            ? s->fsched[0].count
                            : 0;
  return MF_OK;
}

int mf_symbolic_fronts(const mf_symbolic* s, int32_t* front_ptr) {
  if (!s || !front_ptr) return set_error(MF_ERR_INVALID, "NULL argument");
  for (size_t F = 0; F < s->sn.size(); ++F) front_ptr[F] = s->sn[F].first;
  front_ptr[s->sn.size()] = (int32_t)s->n;
  return MF_OK;
}

int mf_symbolic_etree(const mf_symbolic* s, int32_t* parent) {
  if (!s || (!parent && s->n)) return set_error(MF_ERR_INVALID, "NULL argument");
  std::copy(s->parent.begin(), s->parent.end(), parent);
  return MF_OK;
}

int mf_symbolic_colcounts(const mf_symbolic* s, int64_t* counts) {
  if (!s || (!counts && s->n)) return set_error(MF_ERR_INVALID, "NULL argument");
  std::copy(s->colcount.begin(), s->colcount.end(), counts);
  return MF_OK;
}

int mf_symbolic_supernodes(const mf_symbolic* s, int32_t* sup_ptr) {
  if (!s || !sup_ptr) return set_error(MF_ERR_INVALID, "NULL argument");
  if (s->n == 0) {
    sup_ptr[0] = 0;
    return MF_OK;
  }
  std::copy(s->sup_ptr.begin(), s->sup_ptr.end(), sup_ptr);
  return MF_OK;
}

int mf_symbolic_pattern(const mf_symbolic* s, int64_t* Lp, int32_t* Li) {
  if (!s || !Lp || (!Li && s->nnzL)) return set_error(MF_ERR_INVALID, "NULL argument");
  try {
    mf::ensure_fundamental_rows(*s);
  } catch (const std::bad_alloc&) {
    return set_error(MF_ERR_OOM, "host allocation failed");
  }
  Lp[0] = 0;
  int64_t pos = 0;
  for (int64_t sn = 0; sn < s->nsuper; ++sn) {
    const int32_t* rows = s->fs_rowidx.data() + s->fs_rows_off[sn];
    const int64_t nr = s->fs_rows_off[sn + 1] - s->fs_rows_off[sn];
    const int32_t f = s->sup_ptr[sn], k = s->sup_ptr[sn + 1] - f;
    for (int t = 0; t < k; ++t) {
      for (int64_t r = t; r < nr; ++r) Li[pos++] = rows[r];
      Lp[f + t + 1] = pos;
    }
  }
  return MF_OK;
}

int mf_symbolic_supernode_tree(const mf_symbolic* s, int32_t* sparent, int32_t* level) {
  if (!s) return set_error(MF_ERR_INVALID, "NULL argument");
  for (int64_t i = 0; i < s->nsuper; ++i) {
    if (sparent) sparent[i] = s->fs_parent[i];
    if (level) level[i] = s->slevel[s->col2front[s->sup_ptr[i]]];
  }
  return MF_OK;
}

// ---------------------------------------------------------------------------
// Factor
// ---------------------------------------------------------------------------
static int factor_create(mf_handle* h, const mf_symbolic* s, int32_t prec, bool ldlt, int lu,
                         bool sympiv, mf_factor** f);

int mf_factor_create(mf_handle* h, const mf_symbolic* s, int32_t prec, mf_factor** f) {
  return factor_create(h, s, prec, false, 0, false, f);
}

int mf_factor_create_ldlt(mf_handle* h, const mf_symbolic* s, int32_t prec, mf_factor** f) {
  return factor_create(h, s, prec, true, 0, false, f);
}

int mf_factor_create_ldlt_piv(mf_handle* h, const mf_symbolic* s, int32_t prec, mf_factor** f) {
  return factor_create(h, s, prec, true, 0, true, f);
}

int mf_factor_create_lu(mf_handle* h, const mf_symbolic* s, int32_t prec, int32_t pivot,
                        mf_factor** f) {
  if (pivot != 0 && pivot != 1) return set_error(MF_ERR_INVALID, "pivot must be 0 or 1");
  return factor_create(h, s, prec, false, pivot ? 2 : 1, false, f);
}

// Pivoting within the diagonal blocks (LU rows, LDL^T rows and columns): the
// per-column pivot bytes, the reordering items of the later pivot blocks of
// large fronts and, for symmetric pivoting, each row's final position.
static int pivot_extras(mf_factor* F) {
  const mf_symbolic* s = F->S;
  MF_CK(cudaMalloc(&F->piv, std::max<int64_t>(s->n, 1)));
  MF_CK(cudaMemset(F->piv, 0, std::max<int64_t>(s->n, 1)));
  if (F->sympiv) MF_CK(cudaMalloc(&F->ipos, std::max<int64_t>(s->n, 1) * sizeof(int32_t)));
  std::vector<mf::Item> sw;
  for (const mf::Launch& L : s->fsched)
    if (L.kind == mf::K_POTRF)
      for (int32_t i = 0; i < L.count; ++i) {
        const mf::Item& it = s->items[L.item_off + i];
        if (it.t >= 1) sw.push_back({it.s, it.t, 0, 0});
      }
  F->lu_swap_count = (int32_t)sw.size();
  MF_CK(cudaMalloc(&F->lu_swap, std::max<size_t>(sw.size() * sizeof(mf::Item), 8)));
  if (!sw.empty())
    MF_CK(cudaMemcpy(F->lu_swap, sw.data(), sw.size() * sizeof(mf::Item), cudaMemcpyHostToDevice));
  return MF_OK;
}

// Device copies of the LU extras: U^T half, second update pool (in U),
// inverses of the U^T blocks, upper assembly lists and values, pivots and
// the reordering items of the later pivot blocks.
static int lu_extras(mf_factor* F) {
  const mf_symbolic* s = F->S;
  const size_t es = elem_size(F->prec);
  mf::UpperAssembly ua;
  std::string err;
  try {
    const int rc = mf::build_upper_assembly(*s, ua, err);
    if (rc != MF_OK) return set_error(rc, err);
  } catch (const std::bad_alloc&) {
    return set_error(MF_ERR_OOM, "host allocation failed");
  }
  F->nnz_upper = (int64_t)ua.row.size();
  const int64_t inv_slots = s->keep_inv ? s->ninv : s->max_large;
  MF_CK(cudaMalloc(&F->Lu, std::max<int64_t>(s->Lsize, 1) * es));
  MF_CK(cudaMalloc(&F->dinvu, std::max<int64_t>(inv_slots, 1) * mf::kNB * mf::kNB * es));
  MF_CK(cudaMalloc(&F->avu, std::max<int64_t>(F->nnz_upper, 1) * es));
  auto up = [](void** d, const void* h, size_t bytes) -> cudaError_t {
    cudaError_t e = cudaMalloc(d, std::max<size_t>(bytes, 8));
    if (e == cudaSuccess && bytes) e = cudaMemcpy(*d, h, bytes, cudaMemcpyHostToDevice);
    return e;
  };
  MF_CK(up((void**)&F->uacol_ptr, ua.col_ptr.data(), ua.col_ptr.size() * sizeof(int64_t)));
  MF_CK(up((void**)&F->uarow, ua.row.data(), ua.row.size() * sizeof(int32_t)));
  MF_CK(up((void**)&F->uasrc_ptr, ua.src_ptr.data(), ua.src_ptr.size() * sizeof(int64_t)));
  MF_CK(up((void**)&F->uasrc, ua.src.data(), ua.src.size() * sizeof(int64_t)));
  return MF_OK;
}

static int factor_create(mf_handle* h, const mf_symbolic* s, int32_t prec, bool ldlt, int lu,
                         bool sympiv, mf_factor** f) {
  if (!h || !s || !f) return set_error(MF_ERR_INVALID, "NULL argument");
  if (prec != MF_FP64 && prec != MF_FP32) return set_error(MF_ERR_INVALID, "bad precision");
  *f = nullptr;
  if ((lu || sympiv) && (s->pinv || s->v4))
    return set_error(MF_ERR_INVALID,
                     "LU and pivoted LDL^T factors solve with SpTRSV variants 1 and 2 only");
  // LU keeps a second half of the same size as L and the update matrices
  const int64_t need = factor_bytes(s, prec) +
                       (lu ? (s->Lsize + s->Usize + s->nnz_lower) * (int64_t)elem_size(prec) : 0);
  if (h->opt.budget_bytes > 0 && need > h->opt.budget_bytes)
    return set_error(MF_ERR_OOM, "factor exceeds the device budget");
  std::unique_ptr<mf_factor> F(new (std::nothrow) mf_factor());
  if (!F) return set_error(MF_ERR_OOM, "host allocation failed");
  F->h = h;
  F->S = s;
  F->prec = prec;
  int rc = get_devsym(s, F->ds);
  if (rc != MF_OK) return rc;
  const size_t es = elem_size(prec);
  MF_CK(cudaMalloc(&F->L, std::max<int64_t>(s->Lsize, 1) * es));
  // LU: the transposed upper update matrices follow the lower ones
  MF_CK(cudaMalloc(&F->U, std::max<int64_t>(s->Usize, 1) * es * (lu ? 2 : 1)));
  MF_CK(cudaMalloc(&F->vals, std::max<int64_t>(s->nnzA, 1) * sizeof(double)));
  // status words (all-ones when clear): [0] first non-positive pivot column,
  // [1] a bounded wait of the factorization gave up, [2] one of the solve
  // gave up; [3] unused
  MF_CK(cudaMalloc(&F->status, kStatusWords * sizeof(unsigned long long)));
  MF_CK(cudaMallocHost(&F->status_host, kStatusWords * sizeof(unsigned long long)));
  MF_CK(cudaMemset(F->status, 0xff, kStatusWords * sizeof(unsigned long long)));
  // diagonal-block inverses: one slot per large front of a level, or one per
  // 64 pivot columns of every large front when the solve uses them
  const int64_t inv_slots = s->keep_inv ? s->ninv : s->max_large;
  MF_CK(cudaMalloc(&F->dinv, std::max<int64_t>(inv_slots, 1) * mf::kNB * mf::kNB * es));
  MF_CK(cudaMalloc(&F->av, std::max<int64_t>(s->nnz_lower, 1) * es));
  MF_CK(cudaMalloc(&F->qstate, (s->sn.size() + 1) * sizeof(int)));
  if (s->pinv) MF_CK(cudaMalloc(&F->P, std::max<int64_t>(s->Lsize, 1) * es));
  if (s->v4) MF_CK(cudaMalloc(&F->PT, std::max<int64_t>(s->Lsize, 1) * es));
  MF_CK(mf::factor_kernels_init(prec));
  MF_CK(mf::solve_kernels_init(prec));
  F->ldlt = ldlt;
  if (ldlt) MF_CK(cudaMalloc(&F->Dp, std::max<int64_t>(s->n, 1) * es));
  F->lu = lu;
  F->sympiv = sympiv;
  if (lu) {
    const int rc = lu_extras(F.get());
    if (rc != MF_OK) return rc;
  }
  if (lu == 2 || sympiv) {
    const int rc = pivot_extras(F.get());
    if (rc != MF_OK) return rc;
  }
  // LDL^T: the pivots enter the trailing update as a scaling of one operand,
  // and LU updates with two different operands, which the FMA tiles do; the
  // tensor-core path stays with Cholesky
  if (prec == MF_FP32 && h->opt.tc && !ldlt && !lu && !sympiv) {
    F->tc = true;
    MF_CK(mf::factor_tc_init());
    const int64_t srows = std::max<int64_t>(s->split_rows, 1);
    const int64_t srows_b = std::max<int64_t>(s->split_rows_b, 1);
    MF_CK(cudaMalloc(&F->split, srows * 512 * sizeof(float)));
    MF_CK(cudaMalloc(&F->split_b, srows_b * 1024 * sizeof(float)));
    // rows past a front are read (and discarded) by the tile kernel: keep
    // them finite
    MF_CK(cudaMemset(F->split, 0, srows * 512 * sizeof(float)));
    MF_CK(cudaMemset(F->split_b, 0, srows_b * 1024 * sizeof(float)));
    MF_CK(mf::make_split_map(F->split, srows, 512, F->split_map));
    MF_CK(mf::make_split_map(F->split_b, srows_b, 1024, F->split_map_b));
  }
  *f = F.release();
  return MF_OK;
}

// Enqueue the numeric factorization on st.  With `capturing` the calls are
// being recorded into a CUDA graph: profile events then become event-record
// nodes of the graph, so per-launch timing also works for graph replays.
static mf::FactorArgs factor_args(const mf_factor* F) {
  mf::FactorArgs a;
  a.sym = F->ds->d;
  a.vals = F->vals;
  a.L = F->L;
  a.U = F->U;
  a.status = F->status;
  a.split = F->tc ? F->split : nullptr;
  a.split_b = F->tc ? F->split_b : nullptr;
  a.split_map = F->tc ? F->split_map : nullptr;
  a.split_map_b = F->tc ? F->split_map_b : nullptr;
  a.dinv = F->dinv;
  a.P = F->P;
  a.PT = F->PT;
  a.av = F->av;
  a.qstate = F->qstate;
  a.wait_polls = F->wait_polls;
  a.D = F->Dp;
  if (F->lu) {
    a.lu = F->lu;
    a.Lu = F->Lu;
    a.Uu = static_cast<unsigned char*>(F->U) + F->S->Usize * elem_size(F->prec);
    a.dinvu = F->dinvu;
    a.uacol_ptr = F->uacol_ptr;
    a.uarow = F->uarow;
    a.avu = F->avu;
  }
  a.piv = F->piv;
  a.lu_swap = F->lu_swap;
  a.lu_swap_count = F->lu_swap_count;
  a.ipos = F->ipos;
  return a;
}

static int enqueue_factor(mf_factor* F, cudaStream_t st, bool profile, bool capturing) {
  const mf_symbolic* S = F->S;
  const mf::FactorArgs a = factor_args(F);
  const std::vector<mf::Launch>& sched = F->tc ? S->fsched_tc : S->fsched;
  MF_CK(cudaMemsetAsync(F->status, 0xff, 2 * sizeof(unsigned long long), st));
  MF_CK(mf::launch_gather_values(F->prec, a, S->nnz_lower, st));
  if (F->lu)
    MF_CK(mf::launch_gather_upper(F->prec, F->uasrc_ptr, F->uasrc, F->vals, F->avu, F->nnz_upper,
                                  st));
  if (profile && F->ev.size() < 2 * sched.size()) {
    const size_t old = F->ev.size();
    F->ev.resize(2 * sched.size());
    for (size_t i = old; i < F->ev.size(); ++i) MF_CK(cudaEventCreate(&F->ev[i]));
  }
  if (!F->side) {
    int lo = 0, hi = 0;
    MF_CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    MF_CK(cudaStreamCreateWithPriority(&F->crit, cudaStreamNonBlocking, hi));
    MF_CK(cudaStreamCreateWithPriority(&F->side, cudaStreamNonBlocking, lo));
    for (cudaEvent_t* e : {&F->ev_fork, &F->ev_side, &F->ev_in, &F->ev_out})
      MF_CK(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  }
  // the schedule runs on crit, lookahead launches on side (forked from
  // crit); crit joins side when a launch asks, at every change of level and
  // at the end, and st waits for crit, so the factorization as a whole stays
  // ordered on st
  MF_CK(cudaEventRecord(F->ev_in, st));
  MF_CK(cudaStreamWaitEvent(F->crit, F->ev_in, 0));
  if (!sched.empty() && sched[0].kind == mf::K_SMALL_Q)
    MF_CK(cudaMemsetAsync(F->qstate, 0, (S->sn.size() + 1) * sizeof(int), F->crit));
  bool pending = false;
  int32_t level = -1;
  for (size_t i = 0; i < sched.size(); ++i) {
    const mf::Launch& L = sched[i];
    if (pending && (L.join || L.level != level)) {
      MF_CK(cudaStreamWaitEvent(F->crit, F->ev_side, 0));
      pending = false;
    }
    level = L.level;
    cudaStream_t ls = F->crit;
    if (L.side) {
      MF_CK(cudaEventRecord(F->ev_fork, F->crit));
      MF_CK(cudaStreamWaitEvent(F->side, F->ev_fork, 0));
      ls = F->side;
    }
    const unsigned rec = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    if (profile) MF_CK(cudaEventRecordWithFlags(F->ev[2 * i], ls, rec));
    MF_CK(mf::launch_factor(F->prec, L, a, ls));
    if (profile) MF_CK(cudaEventRecordWithFlags(F->ev[2 * i + 1], ls, rec));
    if (L.side) {
      MF_CK(cudaEventRecord(F->ev_side, F->side));
      pending = true;
    }
  }
  if (pending) MF_CK(cudaStreamWaitEvent(F->crit, F->ev_side, 0));
  if (F->piv) MF_CK(mf::launch_lu_swap(F->prec, a, F->crit));
  MF_CK(cudaEventRecord(F->ev_out, F->crit));
  MF_CK(cudaStreamWaitEvent(st, F->ev_out, 0));
  return MF_OK;
}

int mf_factor_numeric(mf_factor* f, const double* values, int32_t values_on_device, void* stream,
                      int32_t async) {
  PhaseRange range_("mf_factor_numeric");
  if (!f || (!values && f->S->nnzA)) return set_error(MF_ERR_INVALID, "NULL argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const mf_symbolic* S = f->S;
  if (S->nnzA)
    MF_CK(cudaMemcpyAsync(f->vals, values, S->nnzA * sizeof(double),
                          values_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  const bool profile = f->h->opt.profile != 0;
  if (f->h->opt.use_graphs) {
    if (!f->gexec) {
      MF_CK(cudaStreamCreateWithFlags(&f->cap_stream, cudaStreamNonBlocking));
      MF_CK(cudaStreamBeginCapture(f->cap_stream, cudaStreamCaptureModeThreadLocal));
      int rc = enqueue_factor(f, f->cap_stream, profile, true);
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamEndCapture(f->cap_stream, &g);
      if (rc != MF_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
      }
      MF_CK(e);
      // per-node priorities keep the critical path ahead of the bulk updates
      e = cudaGraphInstantiate(&f->gexec, g, cudaGraphInstantiateFlagUseNodePriority);
      cudaGraphDestroy(g);
      MF_CK(e);
    }
    MF_CK(cudaGraphLaunch(f->gexec, st));
  } else {
    int rc = enqueue_factor(f, st, profile, false);
    if (rc != MF_OK) return rc;
  }
  f->numeric_done = true;
  if (async) return MF_OK;
  return mf_factor_check(f, stream);
}

int mf_factor_check(mf_factor* f, void* stream) {
  if (!f) return set_error(MF_ERR_INVALID, "NULL factor");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  MF_CK(cudaMemcpyAsync(f->status_host, f->status, 2 * sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost, st));
  MF_CK(cudaStreamSynchronize(st));
  if (f->h->opt.profile) {
    const std::vector<mf::Launch>& sched = f->tc ? f->S->fsched_tc : f->S->fsched;
    for (int k = 0; k < mf::K_NKINDS_FACTOR; ++k) {
      f->prof_ms[k] = 0;
      f->prof_n[k] = 0;
      f->prof_fl[k] = 0;
    }
    if (f->ev.size() >= 2 * sched.size()) {
      for (size_t i = 0; i < sched.size(); ++i) {
        float ms = 0.f;
        MF_CK(cudaEventElapsedTime(&ms, f->ev[2 * i], f->ev[2 * i + 1]));
        const int k = sched[i].kind == mf::K_SMALL_Q ? (int)mf::K_SMALL : sched[i].kind;
        if (k >= mf::K_NKINDS_FACTOR) continue;  // partitioned-inverse pass
        f->prof_ms[k] += ms;
        f->prof_n[k] += 1;
        f->prof_fl[k] += sched[i].flops;
      }
    }
  }
  const unsigned long long bad = f->status_host[0];
  if (f->status_host[1] != ~0ull)
    return set_error(MF_ERR_TIMEOUT, "a bounded device wait in the factorization gave up");
  if (bad != ~0ull) {
    set_error(MF_ERR_NOT_SPD, f->ldlt ? "zero pivot in the LDL^T factorization"
                              : f->lu ? "zero pivot in the LU factorization"
                                      : "matrix is not positive definite");
    g_errcol = (int64_t)bad;
    return MF_ERR_NOT_SPD;
  }
  return MF_OK;
}

int mf_factor_free(mf_factor* f) {
  delete f;
  return MF_OK;
}

int mf_factor_export_L(const mf_factor* f, double* Lx) {
  if (!f || (!Lx && f->S->nnzL)) return set_error(MF_ERR_INVALID, "NULL argument");
  const mf_symbolic* S = f->S;
  const size_t es = elem_size(f->prec);
  std::vector<unsigned char> buf;
  try {
    buf.resize(S->Lsize * es);
  } catch (const std::bad_alloc&) {
    return set_error(MF_ERR_OOM, "host allocation failed");
  }
  try {
    mf::ensure_fundamental_rows(*S);
  } catch (const std::bad_alloc&) {
    return set_error(MF_ERR_OOM, "host allocation failed");
  }
  MF_CK(cudaDeviceSynchronize());
  if (S->Lsize) MF_CK(cudaMemcpy(buf.data(), f->L, S->Lsize * es, cudaMemcpyDeviceToHost));
  // gather the fundamental pattern out of the front panels
  std::vector<int32_t> pos(S->n, -1);
  int64_t out = 0;
  const float* b32 = reinterpret_cast<const float*>(buf.data());
  const double* b64 = reinterpret_cast<const double*>(buf.data());
  for (size_t F = 0; F < S->sn.size(); ++F) {
    const mf::SnInfo& I = S->sn[F];
    const int64_t nf = I.k + I.m;
    const int32_t* frows = S->rowidx.data() + I.rows_off;
    for (int64_t r = 0; r < nf; ++r) pos[frows[r]] = (int32_t)r;
    for (int32_t j = I.first; j < I.first + I.k; ++j) {
      const int32_t sn = S->col2sn[j];
      const int32_t t = j - S->sup_ptr[sn];
      const int32_t* rows = S->fs_rowidx.data() + S->fs_rows_off[sn];
      const int64_t nr = S->fs_rows_off[sn + 1] - S->fs_rows_off[sn];
      const int64_t col = I.Loff + (int64_t)(j - I.first) * nf;
      for (int64_t r = t; r < nr; ++r) {
        const int64_t idx = col + pos[rows[r]];
        Lx[out++] = f->prec == MF_FP32 ? (double)b32[idx] : b64[idx];
      }
    }
  }
  return MF_OK;
}

int mf_factor_export_D(const mf_factor* f, double* D) {
  if (!f || (!D && f->S->n)) return set_error(MF_ERR_INVALID, "NULL argument");
  if (!f->ldlt) return set_error(MF_ERR_INVALID, "not an LDL^T factor");
  const int64_t n = f->S->n;
  MF_CK(cudaDeviceSynchronize());
  if (f->prec == MF_FP32) {
    std::vector<float> t(n);
    if (n) MF_CK(cudaMemcpy(t.data(), f->Dp, n * sizeof(float), cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < n; ++i) D[i] = t[i];
  } else if (n) {
    MF_CK(cudaMemcpy(D, f->Dp, n * sizeof(double), cudaMemcpyDeviceToHost));
  }
  return MF_OK;
}

static int export_columns(const mf_factor* f, const void* base, int64_t j0, int64_t j1,
                          double* Lx);

int mf_factor_export_columns(const mf_factor* f, int64_t j0, int64_t j1, double* Lx) {
  if (!f) return set_error(MF_ERR_INVALID, "NULL factor");
  return export_columns(f, f->L, j0, j1, Lx);
}

int mf_factor_export_U(const mf_factor* f, double* Ux) {
  if (!f) return set_error(MF_ERR_INVALID, "NULL factor");
  if (!f->lu) return set_error(MF_ERR_INVALID, "not an LU factor");
  return export_columns(f, f->Lu, 0, f->S->n, Ux);
}

int mf_factor_export_pivots(const mf_factor* f, int32_t* rho) {
  if (!f || (!rho && f->S->n)) return set_error(MF_ERR_INVALID, "NULL argument");
  if (!f->lu && !f->sympiv) return set_error(MF_ERR_INVALID, "not an LU or pivoted LDL^T factor");
  const int64_t n = f->S->n;
  std::vector<uint8_t> p(f->piv ? n : 0);
  MF_CK(cudaDeviceSynchronize());
  if (f->piv && n) MF_CK(cudaMemcpy(p.data(), f->piv, n, cudaMemcpyDeviceToHost));
  for (const mf::SnInfo& I : f->S->sn)
    for (int32_t c = 0; c < I.k; ++c)
      rho[I.first + c] = f->piv ? I.first + (c & ~(mf::kNB - 1)) + p[I.first + c] : I.first + c;
  return MF_OK;
}

static int export_columns(const mf_factor* f, const void* base, int64_t j0, int64_t j1,
                          double* Lx) {
  const mf_symbolic* S = f->S;
  if (j0 < 0 || j1 < j0 || j1 > S->n || (!Lx && j1 > j0))
    return set_error(MF_ERR_INVALID, "invalid column range");
  if (j1 == j0) return MF_OK;
  const size_t es = elem_size(f->prec);
  std::vector<unsigned char> buf;
  std::vector<int32_t> pos;
  try {
    mf::ensure_fundamental_rows(*S);
    pos.assign(S->n, -1);
  } catch (const std::bad_alloc&) {
    return set_error(MF_ERR_OOM, "host allocation failed");
  }
  MF_CK(cudaDeviceSynchronize());
  int64_t out = 0;
  for (int32_t F = S->col2front[j0]; F <= S->col2front[j1 - 1]; ++F) {
    const mf::SnInfo& I = S->sn[F];
    const int64_t nf = I.k + I.m;
    try {
      buf.resize((size_t)(nf * I.k) * es);
    } catch (const std::bad_alloc&) {
      return set_error(MF_ERR_OOM, "host allocation failed");
    }
    MF_CK(cudaMemcpy(buf.data(), static_cast<const unsigned char*>(base) + I.Loff * es,
                     buf.size(), cudaMemcpyDeviceToHost));
    const float* b32 = reinterpret_cast<const float*>(buf.data());
    const double* b64 = reinterpret_cast<const double*>(buf.data());
    const int32_t* frows = S->rowidx.data() + I.rows_off;
    for (int64_t r = 0; r < nf; ++r) pos[frows[r]] = (int32_t)r;
    const int64_t c0 = std::max<int64_t>(I.first, j0), c1 = std::min<int64_t>(I.first + I.k, j1);
    for (int64_t j = c0; j < c1; ++j) {
      const int32_t sn = S->col2sn[j];
      const int32_t t = (int32_t)(j - S->sup_ptr[sn]);
      const int32_t* rows = S->fs_rowidx.data() + S->fs_rows_off[sn];
      const int64_t nr = S->fs_rows_off[sn + 1] - S->fs_rows_off[sn];
      const int64_t col = (j - I.first) * nf;
      for (int64_t r = t; r < nr; ++r) {
        const int64_t idx = col + pos[rows[r]];
        Lx[out++] = f->prec == MF_FP32 ? (double)b32[idx] : b64[idx];
      }
    }
  }
  return MF_OK;
}

int mf_factor_launch_counts(const mf_factor* f, int64_t* factor_launches, int64_t* solve_launches) {
  if (!f) return set_error(MF_ERR_INVALID, "NULL factor");
  // + 1: the gather of the values into assembly order
  if (factor_launches)
    *factor_launches = (int64_t)(f->tc ? f->S->fsched_tc.size() : f->S->fsched.size()) + 1;
  if (solve_launches) *solve_launches = (int64_t)(f->S->fwsched.size() + f->S->bwsched.size() + 2);
  // (a solve pass also issues one memset of its ticket counters and flags)
  return MF_OK;
}

int mf_factor_profile(const mf_factor* f, double* ms, int64_t* launches, double* flops) {
  if (!f) return set_error(MF_ERR_INVALID, "NULL factor");
  for (int k = 0; k < mf::K_NKINDS_FACTOR; ++k) {
    if (ms) ms[k] = f->prof_ms[k];
    if (launches) launches[k] = f->prof_n[k];
    if (flops) flops[k] = f->prof_fl[k];
  }
  return MF_OK;
}

int mf_factor_kind_items(const mf_factor* f, int64_t* items, int64_t* launches) {
  if (!f || !items) return set_error(MF_ERR_INVALID, "NULL argument");
  for (int k = 0; k < mf::K_NKINDS_FACTOR; ++k) {
    items[k] = 0;
    if (launches) launches[k] = 0;
  }
  for (const mf::Launch& L : f->tc ? f->S->fsched_tc : f->S->fsched) {
    const int k = L.kind == mf::K_SMALL_Q ? (int)mf::K_SMALL : L.kind;
    if (k >= mf::K_NKINDS_FACTOR) continue;
    items[k] += L.count;
    if (launches) launches[k] += 1;
  }
  return MF_OK;
}

int mf_diag_wait_timeout(int32_t polls, void* stream) {
  if (polls < 1) return set_error(MF_ERR_INVALID, "polls must be positive");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  void* buf = nullptr;
  MF_CK(cudaMalloc(&buf, 256));
  int rc = MF_OK;
  unsigned long long host[1] = {0};
  int* flag = static_cast<int*>(buf);
  unsigned long long* status = reinterpret_cast<unsigned long long*>(static_cast<char*>(buf) + 128);
  cudaError_t e = cudaMemsetAsync(buf, 0, 256, st);
  if (e == cudaSuccess) e = mf::launch_wait_probe(flag, status, polls, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(host, status, sizeof(host), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(buf);
  if (e != cudaSuccess) return set_error(MF_ERR_CUDA, std::string("wait probe: ") + cudaGetErrorString(e));
  if (host[0] == (unsigned long long)MF_ERR_TIMEOUT)
    rc = set_error(MF_ERR_TIMEOUT, "device wait gave up after " + std::to_string(polls) + " polls");
  else
    rc = set_error(MF_ERR_INTERNAL, "wait probe returned without a timeout record");
  return rc;
}

int mf_diag_fp64_peak(int32_t kind, void* stream, double* tflops) {
  if ((kind != 0 && kind != 1) || !tflops) return set_error(MF_ERR_INVALID, "invalid peak probe");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  MF_CK(cudaGetDevice(&dev));
  MF_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * mf::peak_fp64_blocks_per_sm(kind);  // one full wave
  const int64_t iters = kind == 0 ? 20000 : 6000;
  double* out = nullptr;
  MF_CK(cudaMalloc(&out, (size_t)blocks * 256 * sizeof(double)));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 0.f;
  // one short warm-up launch, then the best of three timed launches
  if (e == cudaSuccess) e = mf::launch_peak_fp64(kind, out, blocks, iters / 16, st);
  for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
    e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) e = mf::launch_peak_fp64(kind, out, blocks, iters, st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && (best == 0.f || ms < best)) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return set_error(MF_ERR_CUDA, std::string("peak probe: ") + cudaGetErrorString(e));
  *tflops = best > 0.f ? mf::peak_fp64_flops(kind, blocks, iters) / (best * 1e-3) / 1e12 : 0.0;
  return MF_OK;
}

}  // extern "C"

namespace {

// Results of mf_autotune, keyed by a 64-bit FNV-1a hash of the pattern, the
// ordering, the precision, the repetitions, the options that shape the
// search and the device (SM count and compute capability), for the life of
// the process.  A repeated call on the same pattern returns at once.
struct TuneResult {
  mf_options opt;
  double ms;
};
std::mutex g_tune_mu;
std::map<uint64_t, TuneResult> g_tune_cache;

uint64_t fnv(uint64_t h, const void* p, size_t bytes) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < bytes; ++i) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}

}  // namespace

int mf_autotune(mf_handle* h, int64_t n, const int64_t* rowptr, const int32_t* colind,
                const int32_t* perm, const double* values, int32_t values_on_device, int32_t prec,
                int32_t reps, mf_options* best, double* best_ms) {
  if (!h || !best || !best_ms || reps < 1 || !rowptr || n < 0)
    return set_error(MF_ERR_INVALID, "invalid autotune arguments");
  if (prec != MF_FP64 && prec != MF_FP32) return set_error(MF_ERR_INVALID, "bad precision");
  *best = h->opt;
  *best_ms = -1.0;
  int dev = 0, sms = 0, ccmaj = 0, ccmin = 0;
  MF_CK(cudaGetDevice(&dev));
  MF_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  MF_CK(cudaDeviceGetAttribute(&ccmaj, cudaDevAttrComputeCapabilityMajor, dev));
  MF_CK(cudaDeviceGetAttribute(&ccmin, cudaDevAttrComputeCapabilityMinor, dev));
  uint64_t key = 1469598103934665603ull;
  key = fnv(key, &n, sizeof(n));
  key = fnv(key, rowptr, (n + 1) * sizeof(int64_t));
  if (rowptr[n] > 0) key = fnv(key, colind, rowptr[n] * sizeof(int32_t));
  if (perm) key = fnv(key, perm, n * sizeof(int32_t));
  const int32_t shape[8] = {prec, reps, h->opt.sptrsv, h->opt.tc, h->opt.use_graphs, sms, ccmaj, ccmin};
  key = fnv(key, shape, sizeof(shape));
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto hit = g_tune_cache.find(key);
    if (hit != g_tune_cache.end()) {
      *best = hit->second.opt;
      best->budget_bytes = h->opt.budget_bytes;
      best->profile = h->opt.profile;
      *best_ms = hit->second.ms;
      return MF_OK;
    }
  }
  cudaStream_t st = nullptr;
  MF_CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  MF_CK(cudaEventCreate(&e0));
  MF_CK(cudaEventCreate(&e1));
  int rc = MF_OK;
  const bool tc_on = prec == MF_FP32 && h->opt.tc;
  // one candidate: analysis with its options (reused while relax is the
  // same), then a warm-up factorization and `reps` timed ones
  mf_symbolic* S = nullptr;
  int S_relax = -1;
  auto measure = [&](const mf_options& o, double* ms) -> int {
    mf_handle tmp = *h;
    tmp.opt = o;
    tmp.opt.profile = 0;
    tmp.opt.use_graphs = 1;
    if (!S || S_relax != o.relax) {
      if (S) mf_symbolic_free(S);
      S = nullptr;
      int r = mf_symbolic_analyze(&tmp, n, rowptr, colind, perm, &S);
      if (r != MF_OK) return r;
      S_relax = o.relax;
    } else {
      try {
        mf::build_schedules(*S, o.small_front_max, o.small_queue, o.update_tile);
      } catch (const std::bad_alloc&) {
        return set_error(MF_ERR_OOM, "host allocation failed");
      }
      S->opt_used = tmp.opt;
      std::lock_guard<std::mutex> lk(S->dev_mu);  // schedules changed: new device copy
      S->dev.reset();
      S->dev_device = -1;
    }
    mf_factor* f = nullptr;
    int r = mf_factor_create(&tmp, S, prec, &f);
    if (r != MF_OK) return r;
    r = mf_factor_numeric(f, values, values_on_device, st, 0);
    float t = 0.f;
    if (r == MF_OK) {
      cudaEventRecord(e0, st);
      for (int i = 0; i < reps && r == MF_OK; ++i) r = mf_factor_numeric(f, values, values_on_device, st, 1);
      cudaEventRecord(e1, st);
      if (r == MF_OK) r = mf_factor_check(f, st);
      if (r == MF_OK && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
        r = set_error(MF_ERR_CUDA, "cudaEventElapsedTime failed");
    }
    mf_factor_free(f);
    *ms = (double)t / reps;
    return r;
  };
  mf_options cur = h->opt;
  for (int b = 0; b < 4; ++b) cur.update_tile[b] = 0;
  double cur_ms = -1.0;
  auto consider = [&](const mf_options& o) {
    double ms = 0.0;
    const int r = measure(o, &ms);
    if (r == MF_OK && (cur_ms < 0 || ms < cur_ms)) {
      cur = o;
      cur_ms = ms;
    }
    return r;
  };
  // 1) relaxation x small-front limit x queue, default tiles
  const int smalls[3] = {mf::kSmallMax, 64, 32};
  for (int relax = 1; relax >= 0 && rc == MF_OK; --relax)
    for (int si = 0; si < 3 && rc == MF_OK; ++si)
      for (int q = 1; q >= 0 && rc == MF_OK; --q) {
        mf_options o = cur;
        o.relax = relax;
        o.small_front_max = smalls[si];
        o.small_queue = q;
        rc = consider(o);
      }
  // 2) per front-size bucket, largest first: the trailing-update tile of
  // the buckets that hold large fronts (coordinate descent)
  if (rc == MF_OK) {
    mf_options o = cur;
    double ms = 0.0;
    rc = measure(o, &ms);  // the winner's analysis, for its buckets
    bool present[4] = {false, false, false, false};
    if (rc == MF_OK)
      for (const mf::SnInfo& f : S->sn)
        if (f.k + f.m > cur.small_front_max) present[mf::tile_bucket(f.k + f.m)] = true;
    const int cand_tc[3] = {3, 4, 1}, cand_fma[3] = {4, 1, 2};  // the default first
    const int* cand = tc_on ? cand_tc : cand_fma;
    for (int b = 3; b >= 0 && rc == MF_OK; --b) {
      if (!present[b]) continue;
      for (int c = 0; c < 3 && rc == MF_OK; ++c) {
        mf_options t = cur;
        t.update_tile[b] = cand[c];
        if (cand[c] == (cur.update_tile[b] ? cur.update_tile[b] : cand[0])) continue;
        rc = consider(t);
      }
      if (rc == MF_OK && cur.update_tile[b] == 0) cur.update_tile[b] = cand[0];
    }
  }
  if (S) mf_symbolic_free(S);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  if (rc != MF_OK) return rc;
  *best = cur;
  *best_ms = cur_ms;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = {cur, cur_ms};
  return MF_OK;
}

int mf_symbolic_options(const mf_symbolic* s, mf_options* opt) {
  if (!s || !opt) return set_error(MF_ERR_INVALID, "NULL argument");
  *opt = s->opt_used;
  return MF_OK;
}

// ---------------------------------------------------------------------------
// Solve
// ---------------------------------------------------------------------------
namespace {

int64_t sync_ints(const mf_symbolic* S) { return 2 * (int64_t)S->nlevels + 1; }

// Enqueue one solve pass (nrhs <= kSolveChunk) on Y/W/sync work memory.
int solve_pass(mf_factor* f, int32_t cn, const double* B, int64_t ldb, double* X, int64_t ldx,
               const double* inv_scale, const double* scale, int accumulate, void* Y, void* W,
               int32_t* sync, cudaStream_t st) {
  const mf_symbolic* S = f->S;
  MF_CK(cudaMemsetAsync(sync, 0, sync_ints(S) * sizeof(int32_t), st));
  MF_CK(mf::launch_perm_in(f->prec, B, ldb, f->ds->d.perm, Y, S->n, cn, inv_scale, st));
  mf::SolveArgs a;
  a.sym = f->ds->d;
  a.L = f->L;
  a.Y = Y;
  a.W = W;
  a.sync = sync;
  a.status = f->status + kStatusSolve;
  a.wait_polls = f->wait_polls;
  a.n = S->n;
  a.nrhs = cn;
  a.nlevels = S->nlevels;
  a.dinv = S->keep_inv ? f->dinv : nullptr;
  a.P = f->P;
  a.PT = f->PT;
  a.piv = f->piv;
  a.ipos = f->ipos;
  // the flag-chained pivot blocks hand their values over through slots of W
  // that must start as the all-ones pattern in each sweep (variant 4 keeps
  // its forward results in W and has no chains)
  const size_t wbytes = (size_t)S->Wsize * cn * elem_size(f->prec);
  if (!S->v4) MF_CK(cudaMemsetAsync(W, 0xff, wbytes, st));
  for (const mf::Launch& L : S->fwsched) MF_CK(mf::launch_solve(f->prec, L, a, st));
  // LDL^T: z = D^{-1} z between the sweeps (the forward results sit in Y,
  // or for SpTRSV variant 4 in the first n x nrhs values of W)
  if (f->ldlt) MF_CK(mf::launch_dscale(f->prec, S->v4 ? W : Y, f->Dp, S->n, cn, st));
  // LU: the backward sweep solves U x = y with U^T, stored like L
  if (f->lu) {
    a.L = f->Lu;
    a.dinv = S->keep_inv ? f->dinvu : nullptr;
    a.piv = nullptr;
  }
  if (!S->v4) MF_CK(cudaMemsetAsync(W, 0xff, wbytes, st));
  for (const mf::Launch& L : S->bwsched) MF_CK(mf::launch_solve(f->prec, L, a, st));
  MF_CK(mf::launch_perm_out(f->prec, Y, f->ds->d.perm, f->ipos, X, ldx, S->n, cn, scale,
                            accumulate, st));
  return MF_OK;
}

int ensure_solve_buffers(mf_factor* f) {
  const mf_symbolic* S = f->S;
  const size_t es = elem_size(f->prec);
  if (!f->Y) MF_CK(cudaMalloc(&f->Y, std::max<int64_t>(S->n * mf::kSolveChunk, 1) * es));
  if (!f->W) MF_CK(cudaMalloc(&f->W, std::max<int64_t>(S->Wsize * mf::kSolveChunk, 1) * es));
  if (!f->small) MF_CK(cudaMalloc(&f->small, 4096 * sizeof(double)));
  if (!f->sync) MF_CK(cudaMalloc(&f->sync, sync_ints(S) * sizeof(int32_t)));
  return MF_OK;
}

int ensure_io(mf_factor* f, int64_t doubles) {
  if (doubles <= f->io_cap) return MF_OK;
  cudaFree(f->Bd);
  cudaFree(f->Xd);
  cudaFree(f->Rd);
  f->Bd = f->Xd = f->Rd = nullptr;
  f->io_cap = 0;
  MF_CK(cudaMalloc(&f->Bd, doubles * sizeof(double)));
  MF_CK(cudaMalloc(&f->Xd, doubles * sizeof(double)));
  MF_CK(cudaMalloc(&f->Rd, doubles * sizeof(double)));
  f->io_cap = doubles;
  return MF_OK;
}

// Clear the solve's timeout record (stream-ordered).  Every public solve
// call does this once before its first pass, so a record always belongs to
// the last call.
int reset_solve_status(mf_factor* f, cudaStream_t st) {
  MF_CK(cudaMemsetAsync(f->status + kStatusSolve, 0xff, sizeof(unsigned long long), st));
  return MF_OK;
}

// Read the solve's timeout record after synchronizing st.
int read_solve_status(mf_factor* f, cudaStream_t st) {
  MF_CK(cudaMemcpyAsync(f->status_host + kStatusSolve, f->status + kStatusSolve,
                        sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  MF_CK(cudaStreamSynchronize(st));
  if (f->status_host[kStatusSolve] != ~0ull)
    return set_error(MF_ERR_TIMEOUT, "a bounded device wait in the solve gave up");
  return MF_OK;
}

// X (=|+=) scale * A^{-1} (inv_scale * B), device pointers, chunked RHS.
int solve_dev(mf_factor* f, int32_t nrhs, const double* B, int64_t ldb, double* X, int64_t ldx,
              const double* inv_scale, const double* scale, int accumulate, cudaStream_t st) {
  const mf_symbolic* S = f->S;
  int rc = ensure_solve_buffers(f);
  if (rc != MF_OK) return rc;
  for (int32_t c0 = 0; c0 < nrhs; c0 += mf::kSolveChunk) {
    const int32_t cn = std::min<int32_t>(mf::kSolveChunk, nrhs - c0);
    rc = solve_pass(f, cn, B + c0 * ldb, ldb, X + c0 * ldx, ldx, inv_scale ? inv_scale + c0 : nullptr,
                    scale ? scale + c0 : nullptr, accumulate, f->Y, f->W, f->sync, st);
    if (rc != MF_OK) return rc;
  }
  return MF_OK;
}

}  // namespace

namespace mf {

// Solve with caller-provided work memory (no allocation): Y and W of each
// chunk of right-hand sides are carved out of `scratch`.  Used by the
// no-allocation entry point; B and X are device pointers.
int solve_in_scratch(mf_factor* f, int32_t nrhs, const double* B, int64_t ldb, double* X,
                     int64_t ldx, void* scratch, size_t scratch_bytes, cudaStream_t st) {
  const mf_symbolic* S = f->S;
  const size_t es = elem_size(f->prec);
  const size_t per_rhs = (size_t)(S->n + S->Wsize) * es;
  const size_t slack = 512;  // alignment of the W carve-out
  const size_t sync_bytes = ((size_t)sync_ints(S) * sizeof(int32_t) + 255) / 256 * 256;
  if (per_rhs + slack + sync_bytes > scratch_bytes)
    return set_error(MF_ERR_INVALID,
                     "problem too large for the no-allocation solve: needs " +
                         std::to_string(per_rhs + slack + sync_bytes) +
                         " scratch bytes for one right-hand side, limit " +
                         std::to_string(scratch_bytes));
  const int32_t chunk =
      (int32_t)std::min<size_t>(kSolveChunk, (scratch_bytes - slack - sync_bytes) / per_rhs);
  unsigned char* base = static_cast<unsigned char*>(scratch);
  int32_t* sync = reinterpret_cast<int32_t*>(base);
  const int rs = reset_solve_status(f, st);
  if (rs != MF_OK) return rs;
  for (int32_t c0 = 0; c0 < nrhs; c0 += chunk) {
    const int32_t cn = std::min<int32_t>(chunk, nrhs - c0);
    void* Y = base + sync_bytes;
    const size_t woff = sync_bytes + ((size_t)S->n * cn * es + 255) / 256 * 256;
    void* W = base + woff;
    const int rc = solve_pass(f, cn, B + c0 * ldb, ldb, X + c0 * ldx, ldx, nullptr, nullptr, 0, Y,
                              W, sync, st);
    if (rc != MF_OK) return rc;
  }
  return MF_OK;
}

bool factor_ready(const mf_factor* f, int64_t* n) {
  *n = f->S->n;
  return f->numeric_done;
}

}  // namespace mf

extern "C" {

int mf_solve(mf_factor* f, int32_t nrhs, const double* B, int64_t ldb, double* X, int64_t ldx,
             int32_t on_device, void* stream) {
  PhaseRange range_("mf_solve");
  if (!f) return set_error(MF_ERR_INVALID, "NULL factor");
  const int64_t n = f->S->n;
  if (nrhs < 0 || ldb < n || ldx < n || (nrhs > 0 && n > 0 && (!B || !X)))
    return set_error(MF_ERR_INVALID, "invalid solve arguments");
  if (!f->numeric_done) return set_error(MF_ERR_INVALID, "factor has no numeric values");
  if (nrhs == 0 || n == 0) return MF_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = reset_solve_status(f, st);
  if (rc != MF_OK) return rc;
  if (on_device) return solve_dev(f, nrhs, B, ldb, X, ldx, nullptr, nullptr, 0, st);
  rc = ensure_io(f, n * (int64_t)nrhs);
  if (rc != MF_OK) return rc;
  MF_CK(cudaMemcpy2DAsync(f->Bd, n * sizeof(double), B, ldb * sizeof(double), n * sizeof(double),
                          nrhs, cudaMemcpyHostToDevice, st));
  rc = solve_dev(f, nrhs, f->Bd, n, f->Xd, n, nullptr, nullptr, 0, st);
  if (rc != MF_OK) return rc;
  MF_CK(cudaMemcpy2DAsync(X, ldx * sizeof(double), f->Xd, n * sizeof(double), n * sizeof(double),
                          nrhs, cudaMemcpyDeviceToHost, st));
  return read_solve_status(f, st);
}

int mf_solve_check(mf_factor* f, void* stream) {
  if (!f) return set_error(MF_ERR_INVALID, "NULL factor");
  return read_solve_status(f, static_cast<cudaStream_t>(stream));
}

int mf_factor_set_wait_limit(mf_factor* f, int32_t polls) {
  if (!f || polls < 0) return set_error(MF_ERR_INVALID, "invalid wait limit");
  if (polls != f->wait_polls && f->gexec) {
    // the bound is a parameter of the captured factorization: capture again
    MF_CK(cudaGraphExecDestroy(f->gexec));
    f->gexec = nullptr;
  }
  f->wait_polls = polls;
  return MF_OK;
}

int mf_diag_small_queue(mf_factor* f, int32_t skip, void* stream) {
  if (!f) return set_error(MF_ERR_INVALID, "NULL factor");
  const mf_symbolic* S = f->S;
  const std::vector<mf::Launch>& sched = f->tc ? S->fsched_tc : S->fsched;
  if (!f->numeric_done || sched.empty() || sched[0].kind != mf::K_SMALL_Q)
    return set_error(MF_ERR_INVALID, "factor has no small-front queue or no numeric values");
  if (skip < 1 || skip >= sched[0].count) return set_error(MF_ERR_INVALID, "skip out of range");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const mf::FactorArgs a = factor_args(f);
  const int first = skip;
  MF_CK(cudaMemsetAsync(f->qstate, 0, (S->sn.size() + 1) * sizeof(int), st));
  MF_CK(cudaMemcpyAsync(f->qstate, &first, sizeof(int), cudaMemcpyHostToDevice, st));
  MF_CK(cudaMemsetAsync(f->status, 0xff, 2 * sizeof(unsigned long long), st));
  MF_CK(mf::launch_factor(f->prec, sched[0], a, st));
  MF_CK(cudaMemcpyAsync(f->status_host, f->status, 2 * sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost, st));
  MF_CK(cudaStreamSynchronize(st));
  if (f->status_host[1] == (unsigned long long)MF_ERR_TIMEOUT)
    return set_error(MF_ERR_TIMEOUT, "a small-front queue wait gave up (tickets before " +
                                         std::to_string(skip) + " were skipped)");
  return set_error(MF_ERR_INTERNAL, "no small-front queue wait gave up");
}

int mf_factor_solve_work_bytes(const mf_factor* f, int64_t* bytes) {
  if (!f || !bytes) return set_error(MF_ERR_INVALID, "NULL argument");
  const mf_symbolic* S = f->S;
  const int64_t es = (int64_t)elem_size(f->prec);
  int64_t b = 0;
  if (f->Y) b += std::max<int64_t>(S->n * mf::kSolveChunk, 1) * es;
  if (f->W) b += std::max<int64_t>(S->Wsize * mf::kSolveChunk, 1) * es;
  if (f->small) b += 4096 * (int64_t)sizeof(double);
  if (f->sync) b += sync_ints(S) * (int64_t)sizeof(int32_t);
  b += 3 * f->io_cap * (int64_t)sizeof(double);
  *bytes = b;
  return MF_OK;
}

int mf_solve_refined(mf_factor* f, int32_t nrhs, const double* B, int64_t ldb, double* X,
                     int64_t ldx, int32_t on_device, double tol, int32_t max_iter,
                     int32_t allow_fallback, mf_ir_report* rep, void* stream) {
  PhaseRange range_("mf_solve_refined");
  if (!f) return set_error(MF_ERR_INVALID, "NULL factor");
  const mf_symbolic* S = f->S;
  const int64_t n = S->n;
  if (nrhs < 0 || nrhs > 512 || ldb < n || ldx < n || (nrhs > 0 && n > 0 && (!B || !X)))
    return set_error(MF_ERR_INVALID, "invalid refinement arguments");
  if (!f->numeric_done) return set_error(MF_ERR_INVALID, "factor has no numeric values");
  if (rep) std::memset(rep, 0, sizeof(*rep));
  if (nrhs == 0 || n == 0) return MF_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = ensure_io(f, n * (int64_t)nrhs);
  if (rc != MF_OK) return rc;
  rc = ensure_solve_buffers(f);
  if (rc != MF_OK) return rc;
  rc = reset_solve_status(f, st);
  if (rc != MF_OK) return rc;
  // device B (ld n) and X (ld n)
  if (on_device)
    MF_CK(cudaMemcpy2DAsync(f->Bd, n * sizeof(double), B, ldb * sizeof(double), n * sizeof(double),
                            nrhs, cudaMemcpyDeviceToDevice, st));
  else
    MF_CK(cudaMemcpy2DAsync(f->Bd, n * sizeof(double), B, ldb * sizeof(double), n * sizeof(double),
                            nrhs, cudaMemcpyHostToDevice, st));
  double* dsm = f->small;  // [0] |A|, [1..nrhs] |b|, then rnorm, xnorm, scale, inv
  double* d_an = dsm;
  double* d_bn = dsm + 1;
  double* d_rn = dsm + 1 + nrhs;
  double* d_xn = d_rn + nrhs;
  double* d_sc = d_xn + nrhs;
  double* d_isc = d_sc + nrhs;
  MF_CK(cudaMemsetAsync(dsm, 0, (1 + nrhs) * sizeof(double), st));
  MF_CK(mf::launch_norms(f->ds->d.rowptr, f->vals, n, f->Bd, n, nrhs, d_an, st));
  std::vector<double> hn(1 + 2 * nrhs), hs(2 * nrhs);
  MF_CK(cudaMemcpyAsync(hn.data(), dsm, (1 + nrhs) * sizeof(double), cudaMemcpyDeviceToHost, st));
  // x0 = solve(b)
  rc = solve_dev(f, nrhs, f->Bd, n, f->Xd, n, nullptr, nullptr, 0, st);
  if (rc != MF_OK) return rc;
  MF_CK(cudaStreamSynchronize(st));
  const double anorm = hn[0];
  std::vector<double> bnorm(hn.begin() + 1, hn.begin() + 1 + nrhs);
  std::vector<double> hist;
  double berr = 0.0;
  int it = 0;
  bool converged = false;
  for (;; ++it) {
    MF_CK(cudaMemsetAsync(d_rn, 0, 2 * nrhs * sizeof(double), st));
    MF_CK(mf::launch_residual(f->ds->d.rowptr, f->ds->d.colind, f->vals, n, S->nnzA, f->Bd, n, f->Xd, n,
                              f->Rd, nrhs, d_rn, d_xn, st));
    MF_CK(cudaMemcpyAsync(hn.data() + 1, d_rn, 2 * nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
    MF_CK(cudaStreamSynchronize(st));
    berr = 0.0;
    for (int r = 0; r < nrhs; ++r) {
      const double den = anorm * hn[1 + nrhs + r] + bnorm[r];
      const double br = den > 0 ? hn[1 + r] / den : 0.0;
      berr = std::max(berr, br);
    }
    if (it == 0 && rep) rep->berr_first = berr;
    hist.push_back(berr);
    if (berr <= tol) {
      converged = true;
      break;
    }
    const bool stagnated =
        it >= max_iter || (hist.size() >= 3 && berr > 0.5 * hist[hist.size() - 3]);
    if (stagnated) break;
    for (int r = 0; r < nrhs; ++r) {
      const double rn = hn[1 + r];
      hs[r] = rn;
      hs[nrhs + r] = rn > 0 ? 1.0 / rn : 0.0;
    }
    MF_CK(cudaMemcpyAsync(d_sc, hs.data(), 2 * nrhs * sizeof(double), cudaMemcpyHostToDevice, st));
    rc = solve_dev(f, nrhs, f->Rd, n, f->Xd, n, d_isc, d_sc, 1, st);
    if (rc != MF_OK) return rc;
  }
  bool fell_back = false;
  if (!converged) {
    if (!allow_fallback) {
      if (rep) {
        rep->iterations = it;
        rep->berr = berr;
      }
      return set_error(MF_ERR_STAGNATION, "iterative refinement stagnated");
    }
    if (!f->fb64) {
      rc = factor_create(f->h, S, MF_FP64, f->ldlt, f->lu, f->sympiv, &f->fb64);
      if (rc != MF_OK) return rc;
    }
    f->fb64->wait_polls = f->wait_polls;
    rc = mf_factor_numeric(f->fb64, f->vals, 1, stream, 0);
    if (rc != MF_OK) return rc;
    rc = reset_solve_status(f->fb64, st);
    if (rc != MF_OK) return rc;
    rc = solve_dev(f->fb64, nrhs, f->Bd, n, f->Xd, n, nullptr, nullptr, 0, st);
    if (rc != MF_OK) return rc;
    MF_CK(cudaMemsetAsync(d_rn, 0, 2 * nrhs * sizeof(double), st));
    MF_CK(mf::launch_residual(f->ds->d.rowptr, f->ds->d.colind, f->vals, n, S->nnzA, f->Bd, n, f->Xd, n,
                              f->Rd, nrhs, d_rn, d_xn, st));
    MF_CK(cudaMemcpyAsync(hn.data() + 1, d_rn, 2 * nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
    MF_CK(cudaStreamSynchronize(st));
    berr = 0.0;
    for (int r = 0; r < nrhs; ++r) {
      const double den = anorm * hn[1 + nrhs + r] + bnorm[r];
      berr = std::max(berr, den > 0 ? hn[1 + r] / den : 0.0);
    }
    fell_back = true;
  }
  if (on_device)
    MF_CK(cudaMemcpy2DAsync(X, ldx * sizeof(double), f->Xd, n * sizeof(double), n * sizeof(double),
                            nrhs, cudaMemcpyDeviceToDevice, st));
  else
    MF_CK(cudaMemcpy2DAsync(X, ldx * sizeof(double), f->Xd, n * sizeof(double), n * sizeof(double),
                            nrhs, cudaMemcpyDeviceToHost, st));
  MF_CK(cudaStreamSynchronize(st));
  if (rep) {
    rep->iterations = it;
    rep->fell_back = fell_back ? 1 : 0;
    rep->berr = berr;
  }
  // a solve whose wait gave up has produced wrong values: report it even
  // if the refinement recovered
  rc = read_solve_status(f, st);
  if (rc == MF_OK && fell_back) rc = read_solve_status(f->fb64, st);
  return rc;
}

}  // extern "C"
