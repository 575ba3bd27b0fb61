/*
 * mfchol.h -- C-ABI of the GB300 supernodal multifrontal sparse Cholesky.
 *
 * The calls follow the three phases of the paper's Ax=b statement (Sec. 3:
 * symbolic analysis on the pattern only, numerical setup that copies the
 * values and factors P A P^T = L L^T, solve by forward and backward
 * substitution) and the reuse contract stated there (one analysis per
 * pattern, repeated numerical factorizations as values change, many solves
 * per factorization).  The factorization is Tacho's multifrontal Cholesky of
 * an SPD matrix with level-set scheduling (paper Sec. 5); the solve is the
 * level-set supernodal SpTRSV of paper Sec. 5, in its variants 1 (diagonal
 * blocks by substitution), 2 (inverted diagonal blocks, the default) and 3
 * (partitioned inverse), chosen by mf_options.sptrsv.
 *
 * Conventions
 *   - A is given as FULL symmetric CSR: rowptr (int64, n+1 entries, rowptr[0]
 *     = 0), colind (int32, rowptr[n] entries, any order within a row,
 *     duplicates summed), values (double, same order as colind).
 *   - perm[new] = old, i.e. C = A(perm, perm).  NULL means identity.
 *     Only entries (r, c) whose permuted indices satisfy iperm[r] >= iperm[c]
 *     are read (the lower triangle of C).
 *   - Exported supernodes are fundamental (no relaxed amalgamation) and are
 *     numbered by their first column in the permuted order.  The numeric
 *     phase works on internal fronts (runs of supernodes merged by relaxed
 *     amalgamation); their explicit zeros never reach exported values.
 *   - Device pointers are plain CUDA device addresses of the current device;
 *     stream arguments are cudaStream_t values passed as void* (NULL = the
 *     legacy default stream).
 *
 * Ownership: the caller owns every array it passes; the library copies what
 * it keeps.  Objects returned through out-parameters belong to the caller
 * and are released with the matching *_free / mf_destroy.  Device buffers
 * passed in are borrowed for the call and must stay valid until the work
 * enqueued on the given stream has completed.
 *
 * Errors: every entry point returns an mf_status.  No entry point aborts,
 * exits or traps.  A per-thread message is available from
 * mf_last_error_string(); for MF_ERR_NOT_SPD the first failing column (in
 * the permuted order) is available from mf_last_error_column().
 */
#ifndef MFCHOL_H
#define MFCHOL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum mf_status {
  MF_OK = 0,
  MF_ERR_INVALID = 1,     /* malformed CSR / perm / argument */
  MF_ERR_NOT_SPD = 2,     /* non-positive pivot; see mf_last_error_column */
  MF_ERR_OOM = 3,         /* device allocation failed or budget exceeded */
  MF_ERR_CUDA = 4,        /* a CUDA runtime call failed */
  MF_ERR_TIMEOUT = 5,     /* a bounded device wait gave up */
  MF_ERR_STAGNATION = 6,  /* refinement stagnated and FP64 fallback is off */
  MF_ERR_INTERNAL = 7     /* internal consistency check failed */
} mf_status;

typedef enum mf_precision { MF_FP64 = 0, MF_FP32 = 1 } mf_precision;

typedef struct mf_handle mf_handle;
typedef struct mf_symbolic mf_symbolic;
typedef struct mf_factor mf_factor;

/* Tuning and behaviour switches.  mf_options_default fills sane values. */
typedef struct mf_options {
  int32_t small_front_max;  /* fronts with k+m <= this run in one CTA (<=128) */
  int32_t use_graphs;       /* 1: capture the factorization in a CUDA graph */
  int32_t profile;          /* 1: time every launch with CUDA events (recorded
                               inside the CUDA graph when graphs are on) */
  int32_t relax;            /* 1: relaxed amalgamation of the internal fronts */
  int64_t budget_bytes;     /* device bytes a factor may hold (0 = no limit) */
  int32_t tc;               /* 1: FP32 trailing updates on tcgen05 tensor cores
                               (split-TF32, FP32 accuracy); 0: FP32 FMA */
  int32_t sptrsv;           /* solve of the large fronts' pivot blocks (Sec. 5,
                               SpTRSV variants): 1 = substitution with the
                               64 x 64 diagonal blocks; 2 = product with their
                               inverses, kept from the factorization (default;
                               more memory: 64 x 64 values per 64 pivot columns
                               of every large front, about 5% of the factor);
                               3 = partitioned inverse: after the factorization
                               every large front also stores
                               [L11^{-1}; -L21 L11^{-1}] (the level's L_l^{-1},
                               as much memory again as those fronts' L and
                               about (k^3/3 + m k^2) more flops per front), and
                               each level of the solve is one product with it
                               instead of a chain of diagonal blocks;
                               4 = the level's partitioned inverse as one
                               sparse matrix per level and sweep: every front
                               (small ones too) stores P and its transpose
                               (about twice the memory of L), and the solve is
                               one product per level and sweep on the global
                               vector, with no front work vectors and no
                               waits.  0 is taken as 1.  Fixed at symbolic
                               analysis. */
  int32_t small_queue;      /* 1 (default): every front of k+m <= 64 whose
                               subtree holds only such fronts runs in one
                               persistent launch (a device queue in level
                               order, each front waiting, with a bounded
                               wait, for its children's completion flags);
                               a value q >= 2 takes fronts of k+m <= q (at
                               most small_front_max); 0: one launch per level
                               and size class.  Fixed at symbolic analysis. */
  int32_t update_tile[4];   /* trailing update of the large fronts per front
                               size bucket (k+m <= 512, <= 2048, <= 8192,
                               larger): 0 default (FP32 with tc: tcgen05
                               128 x 128 tiles; otherwise FMA 32 x 32), 1 FMA
                               64 x 64, 2 FMA 128 x 128, 3 tcgen05 128 x 128
                               (FP32 with tc; FMA 32 x 32 otherwise), 4 FMA
                               32 x 32.  mf_autotune picks them.  Fixed at
                               symbolic analysis. */
} mf_options;

/* Summary of a symbolic analysis. */
typedef struct mf_symbolic_info {
  int64_t n;
  int64_t nnz_lower;      /* entries of the lower triangle of C (unique) */
  int64_t nsuper;         /* fundamental supernodes */
  int64_t nnz_L;          /* sum_j c_j, structural, incl. the diagonal */
  double flops;           /* sum_j c_j^2 (paper-independent Cholesky count) */
  int64_t nlevels;        /* levels of the front tree (level-set schedule) */
  int64_t max_front;      /* max over fronts of k + m */
  int64_t max_k;          /* max front width */
  int64_t factor_bytes_fp64;  /* device bytes of an FP64 factor (L + update) */
  int64_t factor_bytes_fp32;  /* device bytes of an FP32 factor */
  int64_t nfronts;        /* internal fronts after relaxed amalgamation */
  double front_flops;     /* flops of the fronts incl. explicit zeros */
  int64_t queued_fronts;  /* small fronts in the persistent queue launch */
} mf_symbolic_info;

/* Refinement report of mf_solve_refined. */
typedef struct mf_ir_report {
  int32_t iterations;     /* refinement steps taken */
  int32_t fell_back;      /* 1 if the FP64 fallback factorization was used */
  double berr;            /* final max over RHS of the normwise backward error */
  double berr_first;      /* backward error of the unrefined FP32 solve */
} mf_ir_report;

/* ---- library, errors --------------------------------------------------- */

/* Fill *opt with defaults.  Returns MF_ERR_INVALID if opt is NULL. */
int mf_options_default(mf_options* opt);

/* Create a handle bound to the current CUDA device.  opt may be NULL
 * (defaults).  The handle owns nothing else; destroy it last. */
int mf_create(mf_handle** h, const mf_options* opt);
int mf_destroy(mf_handle* h);

/* Message of the last failing call on this thread ("" if none).  The
 * pointer stays valid until the next call on this thread. */
const char* mf_last_error_string(void);

/* Permuted column of the last MF_ERR_NOT_SPD on this thread, else -1. */
int64_t mf_last_error_column(void);

/* ---- phase 1: symbolic analysis (host; paper Sec. 3 step 1) ------------- */

/* Analyse the pattern of C = A(perm, perm): elimination tree (Liu),
 * column counts (Gilbert-Ng-Peyton row-subtree leaves), fundamental
 * supernodes, front row lists, child-to-parent relative maps, level sets and
 * the device memory plan.  Host arrays only.  Errors: MF_ERR_INVALID for a
 * malformed CSR (rowptr not non-decreasing, colind out of range) or a perm
 * that is not a permutation. */
int mf_symbolic_analyze(mf_handle* h, int64_t n, const int64_t* rowptr,
                        const int32_t* colind, const int32_t* perm,
                        mf_symbolic** s);

/* Symbolic analysis on a condensed graph (paper Sec. 5, graph condensation:
 * the DoFs of one mesh node are compressed into one vertex).  node_of[i]
 * (n entries, original numbering, values in [0, n)) names the node of DoF i;
 * with node_of NULL the nodes are fixed blocks of `block` consecutive DoFs
 * (node_of[i] = i / block, block >= 1).  perm (as in mf_symbolic_analyze,
 * NULL = identity) must place the DoFs of every node at consecutive
 * positions.  Every node block of C that holds an entry, and every diagonal
 * node block, is treated as dense: the result is the symbolic analysis of
 * that block-expanded pattern, computed from the node graph (etree and
 * DoF-weighted column counts on the nodes, expanded to DoFs).  The DoFs of a
 * node therefore always share one supernode.  Entries of the expanded
 * pattern that A lacks are explicit zeros of L.  When every node block of A
 * that holds an entry is already full, the result equals
 * mf_symbolic_analyze's.  Errors: as mf_symbolic_analyze, plus
 * MF_ERR_INVALID for node_of out of range, block < 1 without node_of, or a
 * node whose DoFs are not consecutive in the ordering. */
int mf_symbolic_analyze_condensed(mf_handle* h, int64_t n, const int64_t* rowptr,
                                  const int32_t* colind, const int32_t* perm,
                                  const int32_t* node_of, int32_t block,
                                  mf_symbolic** s);

/* Block-diagonal union of `count` independent matrices (a batch of
 * subdomains, paper Sec. 5: many subdomain solves per GPU).  Matrix b
 * occupies rows/cols [off_b, off_b + n_b) of the union, off_b = sum of the
 * previous n.  perms[b] may be NULL.  The union is one symbolic object: its
 * elimination forest has one tree per matrix and one level schedule, so a
 * single factorization covers the whole batch. */
int mf_symbolic_analyze_batch(mf_handle* h, int32_t count, const int64_t* ns,
                              const int64_t* const* rowptrs,
                              const int32_t* const* colinds,
                              const int32_t* const* perms, mf_symbolic** s);

/* Checkpoint / restart of the analysis (the paper has no counterpart; the
 * analysis depends on the pattern only, so a restarted program can load it
 * instead of repeating it).  mf_symbolic_save writes the complete analysis,
 * schedules included, to the file at path; mf_symbolic_load reads it back
 * into a new object owned by the caller (release with mf_symbolic_free).  The
 * loaded analysis keeps the options it was made with (relaxation,
 * small-front limit, SpTRSV variant), not h's.  The format is native-endian
 * and tied to this library version, and carries a 64-bit hash of its
 * contents: a file from another version or kind of machine, or a truncated
 * or damaged file, gives MF_ERR_INVALID, as does a path that cannot be
 * opened.  Host only. */
int mf_symbolic_save(const mf_symbolic* s, const char* path);
int mf_symbolic_load(mf_handle* h, const char* path, mf_symbolic** s);

/* Host-side consistency check of the analysis's launch schedules: every
 * front's work appears exactly once, in launches of its own level, in level
 * order (assembly chunks, panels, TRSM rows, trailing tiles, the
 * partitioned-inverse tiles, the solve blocks of both sweeps).  Returns MF_OK,
 * or MF_ERR_INTERNAL with the first violation in mf_last_error_string.  For
 * tests and diagnostics; the analysis calls do not run it.  The paper has no
 * counterpart. */
int mf_symbolic_check(const mf_symbolic* s);

/* The options the analysis was made with (from mf_create, or the tuned ones
 * mf_autotune returned); kept by mf_symbolic_save / mf_symbolic_load. */
int mf_symbolic_options(const mf_symbolic* s, mf_options* opt);

int mf_symbolic_free(mf_symbolic* s);
int mf_symbolic_get_info(const mf_symbolic* s, mf_symbolic_info* info);
/* parent[j] of the column elimination tree (-1 for roots), n entries. */
int mf_symbolic_etree(const mf_symbolic* s, int32_t* parent);
/* c_j = |struct(L_{*,j})| including the diagonal, n entries. */
int mf_symbolic_colcounts(const mf_symbolic* s, int64_t* counts);
/* First column of each supernode followed by n: nsuper + 1 entries. */
int mf_symbolic_supernodes(const mf_symbolic* s, int32_t* sup_ptr);
/* CSC pattern of L: Lp (n+1 entries), Li (nnz_L entries, rows ascending
 * within a column, diagonal first). */
int mf_symbolic_pattern(const mf_symbolic* s, int64_t* Lp, int32_t* Li);
/* Supernodal elimination tree parent (-1 for roots), nsuper entries, and
 * the level (0 = leaves) of the internal front holding each supernode,
 * nsuper entries.  Either may be NULL.  Internal fronts are contiguous runs
 * of supernodes merged by relaxed amalgamation (mf_options.relax); the
 * exported etree, supernodes, counts and pattern never change with it. */
int mf_symbolic_supernode_tree(const mf_symbolic* s, int32_t* sparent,
                               int32_t* level);
/* First column of each internal front followed by n: nfronts + 1 entries
 * (mf_symbolic_info.nfronts).  With relax = 0 the fronts are the
 * fundamental supernodes. */
int mf_symbolic_fronts(const mf_symbolic* s, int32_t* front_ptr);

/* Autotuner (no paper counterpart; the paper tunes by hand).  Times the
 * numeric factorization of the given matrix and values in precision prec,
 * each candidate factored once to warm up, then `reps` times (CUDA events,
 * the factor's own graph):
 *   1. relaxed amalgamation on/off x small-front limit 32/64/128 x the
 *      small-front queue on/off, with the default trailing updates;
 *   2. then, for each front-size bucket that holds large fronts (largest
 *      bucket first, the others fixed), the trailing-update tile
 *      (update_tile: FMA 32 / 64 / 128 for FP64 and FP32 without tensor
 *      cores; tcgen05 128 / FMA 32 / FMA 64 for FP32 with them).
 * *best receives h's options with the fastest choices and *best_ms its mean
 * time.  Results are cached for the life of the process under a hash of
 * the pattern, the ordering, prec, reps, h's solve variant / tensor-core /
 * graph options and the device: a second call on the same pattern returns
 * the cached choice without factoring.  An analysis made with the returned
 * options records them, and mf_symbolic_save / _load keep them
 * (mf_symbolic_options).  Values: host or device pointer as
 * values_on_device says.  Errors as mf_symbolic_analyze / mf_factor_*. */
int mf_autotune(mf_handle* h, int64_t n, const int64_t* rowptr,
                const int32_t* colind, const int32_t* perm,
                const double* values, int32_t values_on_device, int32_t prec,
                int32_t reps, mf_options* best, double* best_ms);

/* ---- phase 2: numerical factorization (device; paper Sec. 3 step 2) ----- */

/* Allocate device storage for the factor of s in the given precision
 * (MF_FP64 or MF_FP32): supernodal L panels, update matrices, the copy of
 * the values and the device schedule.  Errors: MF_ERR_OOM if the allocation
 * fails or exceeds the handle's budget. */
int mf_factor_create(mf_handle* h, const mf_symbolic* s, int32_t prec,
                     mf_factor** f);

/* As mf_factor_create, for the LDL^T factorization P A P^T = L D L^T of a
 * symmetric, possibly indefinite matrix (paper Sec. 5: besides Cholesky,
 * Tacho factors symmetric indefinite matrices as LDL^T): L unit lower
 * triangular (its unit diagonal is stored, so mf_factor_export_L returns
 * it), D diagonal with 1 x 1 pivots taken in the analysed order, without
 * pivoting.  It exists when every leading principal minor of P A P^T is
 * nonzero, for instance for every ordering of a symmetric quasi-definite
 * matrix ([K B^T; B -C] with K and C positive definite).  mf_factor_numeric
 * then returns MF_ERR_NOT_SPD for the first zero pivot (its column through
 * mf_last_error_column).  The same analysis, kernels and solves serve
 * (every SpTRSV variant; the solve applies D^{-1} between the sweeps);
 * FP32 factors use the FMA trailing update (no tensor cores) and refine in
 * FP64 as with Cholesky, their fallback being an FP64 LDL^T. */
int mf_factor_create_ldlt(mf_handle* h, const mf_symbolic* s, int32_t prec,
                          mf_factor** f);

/* As mf_factor_create_ldlt, with symmetric pivoting within the diagonal
 * blocks (paper Sec. 5: Tacho's LDL^T of symmetric indefinite matrices
 * looks for pivots only inside each diagonal block): Pi P A P^T Pi^T =
 * L D L^T with 1x1 pivots.  The diagonal blocks are those of
 * mf_factor_create_lu (64-column pieces of each internal front's pivot
 * columns); column j takes the diagonal entry of largest magnitude among the
 * block's remaining positions of the current Schur complement, ties going
 * to the row that started first.  Pi only reorders rows and columns inside
 * those blocks.  A block whose remaining diagonal is all zero (for instance
 * [[0, 1], [1, 0]]) is reported as a zero pivot (MF_ERR_NOT_SPD): 2x2
 * pivots are not used.  D is in pivot order (mf_factor_export_D), the row
 * order comes from mf_factor_export_pivots, and the rows of L are labelled
 * as for a pivoted LU.  Solves, refinement and fallback as for LDL^T, with
 * SpTRSV variants 1 and 2 only (an analysis for variant 3 or 4 is refused
 * with MF_ERR_INVALID). */
int mf_factor_create_ldlt_piv(mf_handle* h, const mf_symbolic* s, int32_t prec,
                              mf_factor** f);

/* LDL^T factor: the pivots D (n doubles, permuted order: D[j] belongs to
 * column j of P A P^T, or pivot position j with symmetric pivoting).
 * Synchronous.  MF_ERR_INVALID for a Cholesky factor. */
int mf_factor_export_D(const mf_factor* f, double* D);

/* As mf_factor_create, for the LU factorization of a general matrix with a
 * structurally symmetric pattern (paper Sec. 5: besides Cholesky and
 * LDL^T, Tacho factors general matrices whose sparsity structure is
 * symmetric): Pi P A P^T = L U, L lower triangular, U unit upper triangular
 * (Crout form), on the same analysis; the analysed pattern must be
 * structurally symmetric, the values need not be symmetric.
 *   pivot = 0: no pivoting (Pi = I); the factorization exists when every
 *     leading principal minor of P A P^T is nonzero (for instance for
 *     column diagonally dominant matrices).
 *   pivot = 1: pivots looked for only within diagonal blocks (paper Sec. 5,
 *     the comparison with SuperLU: Tacho searches each diagonal block for
 *     its pivots instead of whole columns).  The diagonal blocks are the
 *     64-column pieces into which each internal front's pivot columns are
 *     cut from its first column (mf_symbolic_fronts).  Column j takes the
 *     row of largest magnitude among the rows of its block not yet chosen,
 *     ties going to the row that started first, so Pi only reorders rows
 *     inside those blocks and L and U keep the analysed sparsity.
 * Values are given to mf_factor_numeric as for Cholesky (all entries of the
 * CSR pattern, both triangles); it returns MF_ERR_NOT_SPD for the first
 * zero pivot (its column through mf_last_error_column).  Solves, refinement
 * and serving take LU factors like Cholesky ones (SpTRSV variants 1 and 2;
 * an analysis made for variant 3 or 4 is refused); FP32 factors use the FMA
 * trailing update and refine in FP64 with an FP64 LU of the same kind as
 * fallback.  Device memory: about twice that of a Cholesky factor.
 * Errors: MF_ERR_INVALID for pivot not in {0, 1}, for an analysis of
 * SpTRSV variant 3 or 4, or when an upper entry of A falls outside the
 * analysed structure (pattern not structurally symmetric). */
int mf_factor_create_lu(mf_handle* h, const mf_symbolic* s, int32_t prec, int32_t pivot,
                        mf_factor** f);

/* LU factor: U transposed in the layout of mf_factor_export_L (entry (i, j)
 * of the pattern, i >= j, receives U(j, i); the diagonal is 1).
 * Synchronous.  MF_ERR_INVALID for a factor that is not LU. */
int mf_factor_export_U(const mf_factor* f, double* Ux);

/* LU or pivoted LDL^T factor: rho[i] = the row (LDL^T: row and column) of
 * P A P^T (permuted numbering) that ended in pivot position i; the
 * identity without pivoting.  Synchronous.  With
 * pivoting, the rows of L are labelled as follows by mf_factor_export_L and
 * mf_factor_export_columns: in a column j of internal front F, a pattern row
 * i that is a pivot column of F holds L(i, j) (pivot order), and a row i of
 * a later front keeps the label it had before that front pivoted, so it
 * holds L(rho^{-1}(i), j).  U is not affected (its rows are pivot
 * positions, its columns are never permuted).  MF_ERR_INVALID for a factor
 * that is neither. */
int mf_factor_export_pivots(const mf_factor* f, int32_t* rho);

/* Numerical factorization P A P^T = L L^T with the given values (CSR order
 * of the analysed pattern; nnz = rowptr[n] entries; host or device pointer
 * as values_on_device says).  Enqueued on `stream`.  Unless `async` is
 * non-zero the call waits for the stream and returns MF_ERR_NOT_SPD (with
 * the first failing permuted column) if a pivot was not positive.  With
 * async != 0 it returns after enqueueing; mf_factor_check reads the status.
 * May be called again with new values (refactorization reuses storage). */
int mf_factor_numeric(mf_factor* f, const double* values,
                      int32_t values_on_device, void* stream, int32_t async);

/* Wait for `stream` and return the status of the last numeric call:
 * MF_ERR_NOT_SPD (first failing column through mf_last_error_column) or
 * MF_ERR_TIMEOUT if a bounded device wait of the factorization (the
 * tensor-core trailing update's copy/MMA barriers) gave up.  Solve failures
 * are reported by the solve calls and mf_solve_check, never here. */
int mf_factor_check(mf_factor* f, void* stream);

/* Bound of the device waits on this factor -- the solve kernels' waits for
 * the values of earlier pivot blocks and the small-front queue's waits for
 * children -- in polls of about
 * 128 ns (0 restores the default, 2^22 polls, about half a second).  A wait
 * that runs out records MF_ERR_TIMEOUT for the call in progress and lets
 * its kernel finish (no hang); the values of that call are then wrong, and
 * the call (or mf_solve_check / mf_factor_check) reports it.  A very short
 * bound makes the waits of a real solve run out, which tests that
 * reporting.  Changing the bound re-captures the factorization's CUDA graph
 * at the next numeric call.  Errors: MF_ERR_INVALID for polls < 0. */
int mf_factor_set_wait_limit(mf_factor* f, int32_t polls);

/* Bytes of solve work memory (work vectors, right-hand-side staging, ticket
 * counters)
 * that the factor currently holds on the device; 0 until a solve that
 * allocates (mf_solve, mf_solve_refined) has run. */
int mf_factor_solve_work_bytes(const mf_factor* f, int64_t* bytes);

int mf_factor_free(mf_factor* f);

/* Copy L to the host in CSC order of mf_symbolic_pattern (nnz_L doubles;
 * FP32 factors are widened).  Synchronous. */
int mf_factor_export_L(const mf_factor* f, double* Lx);

/* Copy the columns j0 .. j1-1 (permuted numbering) of L to the host: the
 * sum of their column counts c_j doubles, column by column in the order of
 * mf_symbolic_pattern (entries Lp[j0] .. Lp[j1] of mf_factor_export_L's
 * output).  Copies only the fronts holding those columns, so a sample of a
 * very large factor can be checked without moving all of L.  Synchronous.
 * Errors: MF_ERR_INVALID for a range outside [0, n]. */
int mf_factor_export_columns(const mf_factor* f, int64_t j0, int64_t j1,
                             double* Lx);

/* Kernel launches issued by one numeric factorization / one 1-RHS solve. */
int mf_factor_launch_counts(const mf_factor* f, int64_t* factor_launches,
                            int64_t* solve_launches);

/* With profiling on (mf_options.profile), per-kernel-kind totals of the last
 * numeric call: kinds 0 small-front, 1 assemble, 2 potrf, 3 trsm, 4 syrk,
 * 5 syrk on tensor cores.  ms[kind], launches[kind] and flops[kind]
 * (algorithmic) for 6 kinds. */
int mf_factor_profile(const mf_factor* f, double* ms, int64_t* launches,
                      double* flops);

/* Work items (CTAs) and launches per kernel kind (the 6 kinds of
 * mf_factor_profile) of one numeric factorization, from its schedule; for
 * the trailing-update kinds an item is one tile.  launches may be NULL. */
int mf_factor_kind_items(const mf_factor* f, int64_t* items, int64_t* launches);

/* ---- phase 3: solve (device; paper Sec. 3 step 3, Sec. 5 SpTRSV) -------- */

/* X = A^{-1} B for nrhs right-hand sides, column-major, FP64 at the
 * boundary (an FP32 factor solves in FP32).  B and X are both host or both
 * device pointers as on_device says; B may equal X.  Enqueued on stream;
 * synchronous for host pointers.  Every solve call clears the factor's
 * solve timeout record first; with host pointers the call returns
 * MF_ERR_TIMEOUT if a bounded wait of its kernels gave up, with device
 * pointers mf_solve_check reads the record. */
int mf_solve(mf_factor* f, int32_t nrhs, const double* B, int64_t ldb,
             double* X, int64_t ldx, int32_t on_device, void* stream);

/* Wait for `stream` and return the status of the last solve call on f
 * (mf_solve with device pointers, mf_solve_noalloc): MF_ERR_TIMEOUT if a
 * bounded device wait of that solve gave up (its X is then wrong), else
 * MF_OK.  Reads one word of device memory into pinned host memory that the
 * factor already holds; allocates nothing. */
int mf_solve_check(mf_factor* f, void* stream);

/* Solve without allocating memory.  The paper has no counterpart: this
 * entry point exists for callers that must not allocate device memory on
 * their solve path, e.g. a latency-critical serving loop (cudaMalloc can
 * synchronize the device and takes unpredictable time) or a host program
 * whose device memory is all handed to a pool it does not control.
 * mf_solve allocates its work buffers on first use and stages host pointers
 * through device copies; this call runs the same solve kernels with their
 * work memory taken from one fixed 32 MiB device array inside the library
 * (every GPU that loads the library holds that array until exit).  B and X
 * are device pointers, column-major, as in mf_solve (B may equal X).  It
 * needs (n + front work) * 8 bytes per right-hand side for an FP64 factor
 * (4 for FP32); right-hand sides are processed in chunks that fit.  A factor
 * too large for even one right-hand side is rejected with MF_ERR_INVALID
 * and a message giving the bytes needed.  No cudaMalloc, cudaFree or other
 * allocating call is made, but the first call on each device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  Every call shares the
 * array, so calls whose work overlaps on the GPU (other streams, other
 * threads) race and corrupt each other's results; serialize them.  The
 * looked-up address is cached per device index for the life of the
 * process: it does not survive cudaDeviceReset (or any other teardown of
 * the device's primary context) -- do not call this entry point after one.
 * Enqueued on stream; returns without waiting; mf_solve_check reports a
 * solve whose bounded waits gave up. */
int mf_solve_noalloc(mf_factor* f, int32_t nrhs, const double* B, int64_t ldb,
                     double* X, int64_t ldx, void* stream);

/* Diagnostic for the failure detection of the solve kernels (no paper
 * counterpart): runs a bounded device wait of the kind the solve's chains
 * use, on one CTA, against a flag that nothing sets, giving up after
 * `polls` polls of about 128 ns each (the solve itself uses 2^22 unless
 * mf_factor_set_wait_limit says otherwise).  The kernel records MF_ERR_TIMEOUT in a status
 * word and returns; the device stays usable.  Allocates and frees 256 bytes
 * of device memory and synchronizes `stream`.  Returns MF_ERR_TIMEOUT (the
 * expected outcome), MF_ERR_INVALID for polls < 1, MF_ERR_CUDA on a CUDA
 * error. */
int mf_diag_wait_timeout(int32_t polls, void* stream);

/* Diagnostic (no paper counterpart): the measured FP64 peak of the current
 * GPU in TFLOP/s, the denominator of the FP64 front kernels' roofline.
 * kind 0 times a register-resident DFMA loop (16 independent FMA chains per
 * thread, one full wave of resident 256-thread blocks), kind 1 a DMMA loop (mma.sync m8n8k4 f64, 8
 * independent accumulator tiles per warp); best of three launches of about
 * 10^11 flops each, CUDA events on `stream` (synchronized).  Allocates and
 * frees a small device buffer.  Errors: MF_ERR_INVALID for another kind or
 * a NULL output, MF_ERR_CUDA. */
int mf_diag_fp64_peak(int32_t kind, void* stream, double* tflops);

/* Diagnostic for the failure detection of the small-front queue (no paper
 * counterpart): runs the factor's persistent small-front launch alone with
 * its first `skip` tickets already taken, so the queued fronts whose
 * children sit in the skipped part wait on completion flags that nothing
 * raises.  Each such wait gives up after the factor's wait bound
 * (mf_factor_set_wait_limit; set a short one first), records MF_ERR_TIMEOUT
 * and lets the kernel finish; the device stays usable, and the factor's
 * values are garbage until the next mf_factor_numeric.  Synchronizes
 * `stream`.  Returns MF_ERR_TIMEOUT (expected), MF_ERR_INTERNAL if no wait
 * gave up, MF_ERR_INVALID without a queue, before a numeric call or for
 * skip outside [1, queued fronts). */
int mf_diag_small_queue(mf_factor* f, int32_t skip, void* stream);

/* Mixed-precision solve: f is an FP32 factor; the residual r = B - A X, the
 * update X += D and the backward error
 *   berr = ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf)
 * are FP64 (A = the values of the last numeric call).  Each step solves the
 * residual scaled by 1/||r||_inf in FP32.  Stops when berr <= tol for every
 * RHS.  Stagnation (berr not halved over two steps, or max_iter reached)
 * triggers an FP64 factorization of the same values and an FP64 solve,
 * unless allow_fallback is 0 (then MF_ERR_STAGNATION).  rep may be NULL.
 * Returns MF_ERR_TIMEOUT if a bounded wait of any of its solves gave up,
 * even when the refinement then reached tol. */
int mf_solve_refined(mf_factor* f, int32_t nrhs, const double* B, int64_t ldb,
                     double* X, int64_t ldx, int32_t on_device, double tol,
                     int32_t max_iter, int32_t allow_fallback,
                     mf_ir_report* rep, void* stream);

/* ---- FastILU / FastSpTRSV (paper Sec. 6, after Chow and Patel) -----------
 * An incomplete LU factorization A ~ L U (L unit lower, U upper) on the
 * ILU(k) pattern S, computed by sweeps in which every entry of S is updated
 * independently, and triangular solves by Jacobi sweeps in which every
 * entry of the solution is updated independently.  FP64, one GPU. */

typedef struct mf_ilu mf_ilu;

/* Pattern S of ILU(level) by levels of fill (host): entries of A and the
 * diagonal have level 0; eliminating row k gives (i, j) the level
 * lev(i, k) + lev(k, j) + 1; S keeps the entries of level <= `level`.  A is
 * CSR (rowptr n + 1 int64, colind int32, any order, duplicates allowed);
 * the caller keeps ownership.  Host only: the first mf_ilu_numeric call
 * uploads S and allocates the device work of the sweeps.  Errors:
 * MF_ERR_INVALID for a bad CSR or level < 0, MF_ERR_OOM. */
int mf_ilu_symbolic(mf_handle* h, int64_t n, const int64_t* rowptr,
                    const int32_t* colind, int32_t level, mf_ilu** out);
/* n and |S|. */
int mf_ilu_info(const mf_ilu* ilu, int64_t* n, int64_t* nnz);
/* S as CSR (Sp n + 1, Sj |S| columns increasing per row) and the level of
 * every entry (Slev |S|); Sj and Slev may be NULL. */
int mf_ilu_pattern(const mf_ilu* ilu, int64_t* Sp, int32_t* Sj, int32_t* Slev);
/* FastILU: values (CSR order of the analysed pattern, host or device) with
 * the diagonal scaled by 1 + shift (the Manteuffel shift); initial guess
 * l_ij = a_ij / a_jj, u_ij = a_ij (zero at fill entries); then `sweeps`
 * sweeps over S, each entry (i, j):
 *   s = a_ij - sum_{k < min(i, j)} l_ik u_kj,
 *   l_ij = (1 - omega) l_ij + omega s / u_jj  (i > j),
 *   u_ij = (1 - omega) u_ij + omega s         (i <= j),
 * out of place (in_place = 0: every entry from the previous sweep; the
 * result does not depend on the order of the updates) or in place
 * (in_place = 1: entries read what other threads have already written, the
 * asynchronous sweep of the paper; results vary from run to run).  With
 * warmup, FastILU(level - 1) runs first, recursively, and initializes the
 * entries of lower level (those of level `level` start at zero).  0 < omega
 * <= 1.  Enqueued on stream. */
int mf_ilu_numeric(mf_ilu* ilu, const double* values, int32_t values_on_device,
                   int32_t sweeps, double omega, double shift, int32_t warmup,
                   int32_t in_place, void* stream);
/* The factors on S in the order of mf_ilu_pattern: l_ij for i > j, u_ij for
 * i <= j (|S| doubles, host).  Synchronous. */
int mf_ilu_export(const mf_ilu* ilu, double* LU);
/* FastSpTRSV: `sweeps` Jacobi sweeps from x = 0 with L (upper = 0, unit
 * diagonal) or U (upper = 1):
 *   x_i = (1 - omega) x_i + omega (b_i - sum_{j != i} t_ij x_j) / t_ii,
 * every x_j from the previous sweep.  b and x (n doubles) are both host or
 * both device pointers as on_device says; synchronous for host pointers. */
int mf_ilu_trsv(mf_ilu* ilu, int32_t upper, int32_t sweeps, double omega,
                const double* b, double* x, int32_t on_device, void* stream);
/* Preconditioner application x = U^-1 L^-1 b with FastSpTRSV (`sweeps`
 * each), as mf_ilu_trsv. */
int mf_ilu_apply(mf_ilu* ilu, int32_t sweeps, double omega, const double* b,
                 double* x, int32_t on_device, void* stream);
int mf_ilu_free(mf_ilu* ilu);

/* ---- serving loop (no paper counterpart beyond Sec. 5's many subdomain
 * solves per GPU; continuous batching of factor and solve requests) ----- */

typedef struct mf_server mf_server;

typedef struct mf_server_stats {
  int64_t completed;
  int64_t failed;
  double p50_ms;          /* request latency, submit to completion */
  double p99_ms;
  double mean_ms;
  double solves_per_s;    /* completed solves over the served span */
  int64_t resident_bytes; /* device bytes of resident or in-flight factors */
  int64_t peak_resident_bytes;
} mf_server_stats;

/* Start `workers` worker threads (each with its own CUDA stream on the
 * current device).  Factor requests are admitted while the device bytes of
 * resident and in-flight factors stay within budget_bytes (0 = no limit).
 * h must outlive the server. */
int mf_server_create(mf_handle* h, int32_t workers, int64_t budget_bytes,
                     mf_server** sv);

/* Queue a factor request: factor s with `values` (host, CSR order) in
 * precision prec, keep the factor resident, and solve nrhs host right-hand
 * sides B into X (nrhs may be 0).  FP32 factors solve with FP64 refinement to
 * berr 1e-13.  s, values, B and X must stay valid until the request is done.
 * *req identifies the request, *factor_id the resident factor.  Errors:
 * MF_ERR_OOM if the factor can never fit the budget. */
int mf_server_submit_factor(mf_server* sv, const mf_symbolic* s,
                            const double* values, int32_t prec, int32_t nrhs,
                            const double* B, int64_t ldb, double* X,
                            int64_t ldx, int64_t* req, int64_t* factor_id);

/* Queue a solve of nrhs host right-hand sides against a resident (or still
 * queued) factor.  Requests on one factor run one at a time; other requests
 * proceed meanwhile. */
int mf_server_submit_solve(mf_server* sv, int64_t factor_id, int32_t nrhs,
                           const double* B, int64_t ldb, double* X,
                           int64_t ldx, int64_t* req);

/* Completion state of a request (done flag, mf_status, latency in ms). */
int mf_server_poll(mf_server* sv, int64_t req, int32_t* done, int32_t* status,
                   double* latency_ms);
/* Block until the request is done. */
int mf_server_wait(mf_server* sv, int64_t req, int32_t* status,
                   double* latency_ms);
/* Free a resident factor; deferred until no running or queued request uses
 * it (solve requests submitted before the release still run). */
int mf_server_release_factor(mf_server* sv, int64_t factor_id);
int mf_server_get_stats(mf_server* sv, mf_server_stats* out);
/* Finish the queued requests, join the workers, free resident factors. */
int mf_server_free(mf_server* sv);

#ifdef __cplusplus
}
#endif
#endif /* MFCHOL_H */
