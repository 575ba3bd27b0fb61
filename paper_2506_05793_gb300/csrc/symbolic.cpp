// symbolic.cpp -- host symbolic analysis of the multifrontal Cholesky
// (paper Sec. 3, phase 1: "symbolic analysis uses only the sparsity
// structure"; run sequentially on one host core as the paper describes for
// Tacho, its cost amortised over many numeric factorizations).
//
// Steps, all on C = A(perm, perm):
//   1. validate the CSR and the permutation;
//   2. strict lower triangle of C by rows and by columns;
//   3. elimination tree (Liu's algorithm with path compression);
//   4. postorder and column counts with the row-subtree leaf/LCA method of
//      Gilbert, Ng and Peyton (O(nnz(A) alpha(n)), no fill-in enumeration);
//   5. fundamental supernodes;
//   6. front row lists by merging each supernode's A pattern with its
//      children's update rows; child-to-parent relative maps;
//   7. level sets of the supernodal tree (height: leaves = 0), memory plan,
//      per-column assembly map of A into the fronts.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <set>
#include <numeric>
#include <unordered_map>
#include <utility>

#include "mf_internal.h"

namespace mf {

namespace {

// Phase timings of the analysis on stderr when MF_SYMBOLIC_TIMING is set.
struct PhaseTimer {
  bool on = std::getenv("MF_SYMBOLIC_TIMING") != nullptr;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  void mark(const char* what) {
    if (!on) return;
    const auto t1 = std::chrono::steady_clock::now();
    std::fprintf(stderr, "[mf symbolic] %-28s %8.3f s\n", what,
                 std::chrono::duration<double>(t1 - t0).count());
    t0 = t1;
  }
};

int invalid(std::string& err, const std::string& msg) {
  err = msg;
  return MF_ERR_INVALID;
}

// Elimination tree and column counts of an n x n symmetric pattern given
// by its strict lower triangle, by rows (rp/ri) and by columns (cp/cr).
// Steps 3-4: Liu's etree with path compression, then the row-subtree
// leaf/LCA counts of Gilbert, Ng and Peyton.  With weights w (one per
// row/column), count[j] is the sum of w over the structure of column j of L
// (the diagonal included); without, the plain count c_j.
int etree_counts(int64_t n, const std::vector<int64_t>& rp, const std::vector<int32_t>& ri,
                 const std::vector<int64_t>& cp, const std::vector<int32_t>& cr,
                 const int64_t* w, std::vector<int32_t>& parent, std::vector<int64_t>& delta,
                 std::string& err) {
  auto W = [w](int32_t j) -> int64_t { return w ? w[j] : 1; };
  // ---- 3. elimination tree
  parent.assign(n, -1);
  {
    std::vector<int32_t> anc(n, -1);
    for (int32_t i = 0; i < n; ++i) {
      for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
        int32_t r = ri[p];
        while (r != -1 && r < i) {
          const int32_t nx = anc[r];
          anc[r] = i;
          if (nx == -1) parent[r] = i;
          r = nx;
        }
      }
    }
  }
  // ---- 4. postorder + column counts (row-subtree leaves and LCAs)
  std::vector<int32_t> post(n);
  {
    std::vector<int32_t> head(n, -1), next(n, -1), stack;
    for (int32_t j = (int32_t)n - 1; j >= 0; --j) {
      if (parent[j] != -1) {
        next[j] = head[parent[j]];
        head[parent[j]] = j;
      }
    }
    int32_t k = 0;
    stack.reserve(n);
    for (int32_t r = 0; r < n; ++r) {
      if (parent[r] != -1) continue;
      stack.push_back(r);
      while (!stack.empty()) {
        const int32_t p = stack.back();
        const int32_t c = head[p];
        if (c == -1) {
          stack.pop_back();
          post[k++] = p;
        } else {
          head[p] = next[c];
          stack.push_back(c);
        }
      }
    }
    if (k != n) {
      err = "postorder incomplete";
      return MF_ERR_INTERNAL;
    }
  }
  delta.assign(n, 0);
  {
    std::vector<int32_t> first(n, -1), maxfirst(n, -1), prevleaf(n, -1), ancestor(n);
    for (int32_t k = 0; k < n; ++k) {
      int32_t j = post[k];
      delta[j] = (first[j] == -1) ? W(j) : 0;  // etree leaf: row subtree {j}
      for (; j != -1 && first[j] == -1; j = parent[j]) first[j] = k;
    }
    std::iota(ancestor.begin(), ancestor.end(), 0);
    for (int32_t k = 0; k < n; ++k) {
      const int32_t j = post[k];
      if (parent[j] != -1) delta[parent[j]] -= W(j);  // row subtree j ends below parent(j)
      for (int64_t p = cp[j]; p < cp[j + 1]; ++p) {
        const int32_t i = cr[p];
        if (first[j] <= maxfirst[i]) continue;  // j is not a leaf of row subtree i
        maxfirst[i] = first[j];
        const int32_t jprev = prevleaf[i];
        prevleaf[i] = j;
        delta[j] += W(i);
        if (jprev != -1) {
          int32_t q = jprev;
          while (q != ancestor[q]) q = ancestor[q];
          for (int32_t s = jprev; s != q;) {
            const int32_t sp = ancestor[s];
            ancestor[s] = q;
            s = sp;
          }
          delta[q] -= W(i);  // lca of consecutive leaves counted twice
        }
      }
      if (parent[j] != -1) ancestor[j] = parent[j];
    }
    for (int32_t k = 0; k < n; ++k) {
      const int32_t j = post[k];
      if (parent[j] != -1) delta[parent[j]] += delta[j];
    }
  }
  return MF_OK;
}

// Condensed-graph analysis (paper Sec. 5, "condensed" graph option): the
// degrees of freedom of one node (node_of[dof], original numbering) take
// consecutive positions of the elimination order and are treated as one
// dense block.  The elimination tree and column counts are computed on the
// node graph (a node's weight is its DoF count) and expanded: within a node
// the DoFs form a chain, the last DoF's parent is the first DoF of the
// parent node, and DoF t of node q has count[q] - t entries.  cp/cr are
// replaced by the block-expanded strict lower pattern, from which the front
// rows follow; a node therefore never straddles two supernodes.
int condensed_structure(int64_t n, const int32_t* node_of, const std::vector<int32_t>& perm,
                        const std::vector<int64_t>& rp, const std::vector<int32_t>& ri,
                        std::vector<int64_t>& cp, std::vector<int32_t>& cr,
                        std::vector<int32_t>& parent, std::vector<int64_t>& delta,
                        std::string& err) {
  // nodes in elimination order; nq[i] = node of permuted DoF i
  std::vector<int32_t> nq(n), seen(n, 0);
  std::vector<int32_t> nstart;
  for (int64_t i = 0; i < n; ++i) {
    const int32_t u = node_of[perm[i]];
    if (u < 0 || u >= n) return invalid(err, "node_of out of range");
    if (i == 0 || u != node_of[perm[i - 1]]) {
      if (seen[u]) return invalid(err, "the DoFs of a node are not consecutive in the ordering");
      seen[u] = 1;
      nstart.push_back((int32_t)i);
    }
    nq[i] = (int32_t)nstart.size() - 1;
  }
  const int64_t nc = (int64_t)nstart.size();
  nstart.push_back((int32_t)n);
  std::vector<int64_t> size(nc);
  for (int64_t q = 0; q < nc; ++q) size[q] = nstart[q + 1] - nstart[q];
  // node graph: strict lower triangle by rows (deduplicated), then by columns
  std::vector<int64_t> nrp(nc + 1, 0);
  std::vector<int32_t> nri, mark(nc, -1);
  for (int64_t u = 0; u < nc; ++u) {
    for (int32_t i = nstart[u]; i < nstart[u + 1]; ++i)
      for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
        const int32_t v = nq[ri[p]];
        if (v < u && mark[v] != u) {
          mark[v] = (int32_t)u;
          nri.push_back(v);
        }
      }
    nrp[u + 1] = (int64_t)nri.size();
  }
  std::vector<int64_t> ncp(nc + 1, 0);
  for (int32_t v : nri) ncp[v + 1]++;
  for (int64_t q = 0; q < nc; ++q) ncp[q + 1] += ncp[q];
  std::vector<int32_t> ncr(nri.size());
  {
    std::vector<int64_t> fill(ncp.begin(), ncp.end() - 1);
    for (int64_t u = 0; u < nc; ++u)
      for (int64_t p = nrp[u]; p < nrp[u + 1]; ++p) ncr[fill[nri[p]]++] = (int32_t)u;
  }
  std::vector<int32_t> nparent;
  std::vector<int64_t> ncount;
  int rc = etree_counts(nc, nrp, nri, ncp, ncr, size.data(), nparent, ncount, err);
  if (rc != MF_OK) return rc;
  // expand to DoFs
  parent.assign(n, -1);
  delta.assign(n, 0);
  for (int64_t q = 0; q < nc; ++q)
    for (int32_t i = nstart[q]; i < nstart[q + 1]; ++i) {
      parent[i] = i + 1 < nstart[q + 1] ? i + 1 : (nparent[q] < 0 ? -1 : nstart[nparent[q]]);
      delta[i] = ncount[q] - (i - nstart[q]);
    }
  // block-expanded strict lower pattern by columns (rows sorted)
  int64_t total = 0;
  for (int64_t q = 0; q < nc; ++q) {
    int64_t below = 0;
    for (int64_t p = ncp[q]; p < ncp[q + 1]; ++p) below += size[ncr[p]];
    total += size[q] * below + size[q] * (size[q] - 1) / 2;
  }
  cp.assign(n + 1, 0);
  cr.clear();
  cr.reserve(total);
  for (int64_t q = 0; q < nc; ++q)
    for (int32_t j = nstart[q]; j < nstart[q + 1]; ++j) {
      for (int32_t i = j + 1; i < nstart[q + 1]; ++i) cr.push_back(i);
      for (int64_t p = ncp[q]; p < ncp[q + 1]; ++p)
        for (int32_t i = nstart[ncr[p]]; i < nstart[ncr[p] + 1]; ++i) cr.push_back(i);
      cp[j + 1] = (int64_t)cr.size();
    }
  return MF_OK;
}

}  // namespace

// Device memory of the update matrices.  U_s is written when front s is
// factored and read when its parent is assembled; after that it is dead.
//
// Fronts in the persistent small-front queue (inq) run first, in any order
// that respects the tree, several at once: a block may only be reused by a
// front that is certain to start after the block's reader finished, i.e. by
// the reader itself or one of its ancestors.  So the queued part is planned
// subtree by subtree: every queued front inherits, as its pool, the free
// ranges of its children's pools plus the children's update matrices (which
// it reads before it writes its own), takes its own block from the pool
// (best fit) or from new memory at the top, and passes the rest on.  After
// the queue, the pools of its top fronts are free.
//
// The other fronts run level by level (every launch of a level completes
// before the next level starts): blocks are placed best fit in a simulated
// heap, level by level (free blocks indexed by offset for coalescing and by
// size for the fit), and a block read at level l is free from level l + 1.
// Chains of thin fronts reuse the same memory instead of holding every
// update matrix at once.  Returns the peak size (elements) and sets Uoff for
// every front.
int64_t plan_update_memory(mf_symbolic& S, const std::vector<char>& inq) {
  const int64_t ns = (int64_t)S.sn.size();
  std::vector<std::vector<int32_t>> bylev(S.nlevels);
  for (int64_t s = 0; s < ns; ++s) bylev[S.slevel[s]].push_back((int32_t)s);
  std::map<int64_t, int64_t> by_off;              // offset -> size
  std::set<std::pair<int64_t, int64_t>> by_size;   // (size, offset)
  auto erase_size = [&](int64_t size, int64_t off) { by_size.erase({size, off}); };
  std::vector<std::vector<std::pair<int64_t, int64_t>>> release(S.nlevels + 1);
  // 32-element alignment keeps every update matrix 128/256-byte aligned
  auto usize = [&](int64_t s) -> int64_t {
    const SnInfo& I = S.sn[s];
    return I.parent < 0 ? 0 : (((int64_t)I.m * I.m) + 31) / 32 * 32;
  };
  auto free_block = [&](int64_t off, int64_t size) {
    auto nx = by_off.lower_bound(off);
    if (nx != by_off.end() && off + size == nx->first) {
      size += nx->second;
      erase_size(nx->second, nx->first);
      nx = by_off.erase(nx);
    }
    if (nx != by_off.begin()) {
      auto pv = std::prev(nx);
      if (pv->first + pv->second == off) {
        off = pv->first;
        size += pv->second;
        erase_size(pv->second, pv->first);
        by_off.erase(pv);
      }
    }
    by_off.emplace(off, size);
    by_size.insert({size, off});
  };
  int64_t top = 0;
  // ---- queued fronts: pools passed up the tree (children have smaller
  // indices than their parents)
  {
    std::vector<std::vector<std::pair<int64_t, int64_t>>> pool(ns);
    for (int64_t s = 0; s < ns; ++s) {
      if (!inq[s]) continue;
      SnInfo& I = S.sn[s];
      std::vector<std::pair<int64_t, int64_t>>& P = pool[s];
      for (int32_t ci = I.child_begin; ci < I.child_begin + I.nchild; ++ci) {
        const int32_t c = S.children[ci];
        std::vector<std::pair<int64_t, int64_t>>& Q = pool[c];
        P.insert(P.end(), Q.begin(), Q.end());
        std::vector<std::pair<int64_t, int64_t>>().swap(Q);
        const int64_t cs = usize(c);
        if (cs > 0) P.push_back({S.sn[c].Uoff, cs});
      }
      std::sort(P.begin(), P.end());
      size_t w = 0;
      for (size_t q = 0; q < P.size(); ++q) {
        if (w > 0 && P[w - 1].first + P[w - 1].second == P[q].first) P[w - 1].second += P[q].second;
        else P[w++] = P[q];
      }
      P.resize(w);
      const int64_t sz = usize(s);
      I.Uoff = 0;
      if (sz == 0) continue;
      size_t best = P.size();
      for (size_t q = 0; q < P.size(); ++q)
        if (P[q].second >= sz && (best == P.size() || P[q].second < P[best].second)) best = q;
      if (best < P.size()) {
        I.Uoff = P[best].first;
        P[best].first += sz;
        P[best].second -= sz;
        if (P[best].second == 0) P.erase(P.begin() + best);
      } else {
        I.Uoff = top;
        top += sz;
      }
    }
    // after the queue: the pools of its top fronts are free; the update
    // matrices of those tops stay live until their (level-scheduled) parent
    for (int64_t s = 0; s < ns; ++s) {
      if (!inq[s]) continue;
      const int32_t p = S.sn[s].parent;
      if (p >= 0 && inq[p]) continue;
      for (const auto& r : pool[s]) free_block(r.first, r.second);
      const int64_t sz = usize(s);
      if (sz > 0) release[S.slevel[p]].push_back({S.sn[s].Uoff, sz});
    }
  }
  // ---- the other fronts, level by level
  for (int32_t lev = 0; lev < S.nlevels; ++lev) {
    // blocks read at level lev-1 are dead now
    if (lev >= 1) {
      for (const auto& blk : release[lev - 1]) free_block(blk.first, blk.second);
      release[lev - 1].clear();
    }
    std::vector<int32_t> L;
    for (int32_t s : bylev[lev])
      if (!inq[s]) L.push_back(s);
    std::sort(L.begin(), L.end(), [&](int32_t a, int32_t b) {
      return (int64_t)S.sn[a].m * S.sn[a].m > (int64_t)S.sn[b].m * S.sn[b].m;
    });
    for (int32_t s : L) {
      SnInfo& I = S.sn[s];
      const int64_t sz = usize(s);
      if (sz == 0) {
        I.Uoff = 0;
        continue;
      }
      int64_t off = -1;
      auto fit = by_size.lower_bound({sz, (int64_t)-1});
      if (fit != by_size.end()) {
        const int64_t bsize = fit->first;
        off = fit->second;
        by_size.erase(fit);
        by_off.erase(off);
        if (bsize > sz) {
          by_off.emplace(off + sz, bsize - sz);
          by_size.insert({bsize - sz, off + sz});
        }
      } else {
        // grow the heap, absorbing a free block that ends at the top
        off = top;
        if (!by_off.empty()) {
          auto last = std::prev(by_off.end());
          if (last->first + last->second == top) {
            off = last->first;
            erase_size(last->second, last->first);
            by_off.erase(last);
          }
        }
        top = off + sz;
      }
      I.Uoff = off;
      release[S.slevel[I.parent]].push_back({off, sz});
    }
  }
  return top;
}

int analyze(mf_symbolic& S, int64_t n, const int64_t* rowptr, const int32_t* colind,
            const int32_t* perm, const int32_t* node_of, std::string& err) {
  if (n < 0 || n >= (int64_t)INT32_MAX) return invalid(err, "n out of range");
  if (!rowptr) return invalid(err, "rowptr is NULL");
  if (rowptr[0] != 0) return invalid(err, "rowptr[0] != 0");
  for (int64_t i = 0; i < n; ++i)
    if (rowptr[i + 1] < rowptr[i]) return invalid(err, "rowptr is decreasing");
  const int64_t nnz = rowptr[n];
  if (nnz > 0 && !colind) return invalid(err, "colind is NULL");
  for (int64_t p = 0; p < nnz; ++p)
    if (colind[p] < 0 || colind[p] >= n) return invalid(err, "colind out of range");

  PhaseTimer timer;
  S.n = n;
  S.nnzA = nnz;
  S.rowptr.assign(rowptr, rowptr + n + 1);
  S.colind.assign(colind, colind + nnz);
  S.perm.resize(n);
  S.iperm.assign(n, -1);
  for (int64_t i = 0; i < n; ++i) {
    int32_t o = perm ? perm[i] : (int32_t)i;
    if (o < 0 || o >= n || S.iperm[o] != -1) return invalid(err, "perm is not a permutation");
    S.perm[i] = o;
    S.iperm[o] = (int32_t)i;
  }
  const std::vector<int32_t>& ip = S.iperm;

  // ---- 2. strict lower triangle of C by rows (rp/ri) and columns (cp/cr)
  std::vector<int64_t> rp(n + 1, 0), cp(n + 1, 0);
  for (int64_t ro = 0; ro < n; ++ro) {
    const int32_t i = ip[ro];
    for (int64_t p = rowptr[ro]; p < rowptr[ro + 1]; ++p) {
      const int32_t j = ip[colind[p]];
      if (j < i) {
        rp[i + 1]++;
        cp[j + 1]++;
      }
    }
  }
  for (int64_t i = 0; i < n; ++i) {
    rp[i + 1] += rp[i];
    cp[i + 1] += cp[i];
  }
  std::vector<int32_t> ri(rp[n]), cr(cp[n]);
  {
    std::vector<int64_t> rf(rp.begin(), rp.end() - 1), cf(cp.begin(), cp.end() - 1);
    for (int64_t ro = 0; ro < n; ++ro) {
      const int32_t i = ip[ro];
      for (int64_t p = rowptr[ro]; p < rowptr[ro + 1]; ++p) {
        const int32_t j = ip[colind[p]];
        if (j < i) {
          ri[rf[i]++] = j;
          cr[cf[j]++] = i;
        }
      }
    }
  }

  timer.mark("lower triangle");
  std::vector<int32_t>& parent = S.parent;
  std::vector<int64_t> delta;
  if (!node_of) {
    int rc = etree_counts(n, rp, ri, cp, cr, nullptr, parent, delta, err);
    if (rc != MF_OK) return rc;
  } else {
    int rc = condensed_structure(n, node_of, S.perm, rp, ri, cp, cr, parent, delta, err);
    if (rc != MF_OK) return rc;
  }
  timer.mark("column counts");
  S.colcount = delta;
  S.nnzL = 0;
  S.flops = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    S.nnzL += S.colcount[j];
    S.flops += (double)S.colcount[j] * (double)S.colcount[j];
  }

  // ---- 5. fundamental supernodes
  std::vector<int32_t> nchild(n, 0);
  for (int64_t j = 0; j < n; ++j)
    if (parent[j] != -1) nchild[parent[j]]++;
  S.sup_ptr.clear();
  S.sup_ptr.push_back(0);
  for (int64_t j = 0; j + 1 < n; ++j) {
    const bool joins = parent[j] == j + 1 && S.colcount[j] == S.colcount[j + 1] + 1 &&
                       nchild[j + 1] == 1;
    if (!joins) S.sup_ptr.push_back((int32_t)(j + 1));
  }
  if (n > 0) S.sup_ptr.push_back((int32_t)n);
  const int64_t ns = n > 0 ? (int64_t)S.sup_ptr.size() - 1 : 0;
  S.nsuper = ns;
  S.col2sn.assign(n, 0);
  for (int64_t s = 0; s < ns; ++s)
    for (int32_t j = S.sup_ptr[s]; j < S.sup_ptr[s + 1]; ++j) S.col2sn[j] = (int32_t)s;

  // supernodal tree and children lists (children in increasing order)
  std::vector<int32_t> sparent(ns, -1);
  std::vector<int32_t> schild_cnt(ns + 1, 0);
  for (int64_t s = 0; s < ns; ++s) {
    const int32_t l = S.sup_ptr[s + 1] - 1;
    const int32_t p = parent[l];
    sparent[s] = p == -1 ? -1 : S.col2sn[p];
    if (p != -1) {
      if (p != S.sup_ptr[sparent[s]]) {
        err = "child supernode does not attach to the parent's first column";
        return MF_ERR_INTERNAL;
      }
      schild_cnt[sparent[s] + 1]++;
    }
  }
  for (int64_t s = 0; s < ns; ++s) schild_cnt[s + 1] += schild_cnt[s];
  S.fs_parent = sparent;
  S.children.assign(schild_cnt[ns], 0);
  {
    std::vector<int32_t> fillc(schild_cnt.begin(), schild_cnt.end() - 1);
    for (int64_t s = 0; s < ns; ++s)
      if (sparent[s] != -1) S.children[fillc[sparent[s]]++] = (int32_t)s;
  }

  timer.mark("supernodes");
  // update rows of each fundamental supernode: m_s = c_first - k_s
  std::vector<int32_t> fs_m(ns, 0);
  for (int64_t s = 0; s < ns; ++s)
    fs_m[s] = (int32_t)(S.colcount[S.sup_ptr[s]] - (S.sup_ptr[s + 1] - S.sup_ptr[s]));
  S.fs_rowidx.clear();
  S.fs_rows_off.clear();

  // ---- 7. relaxed amalgamation of fundamental supernodes into fronts.
  // A child whose columns end right before its parent's first column is
  // merged into the parent when the merged front stays small or gains few
  // explicit zeros (size thresholds 4 / 16 / 48 columns with zero fractions
  // 0.8 / 0.1 / 0.05).  Explicit zeros stay exactly zero in the numeric
  // phase, so the exported factor (fundamental pattern) is unchanged; the
  // merge turns chains of thin supernodes into wide dense fronts.
  std::vector<int32_t> fstart(ns), is_top(ns, 1);
  {
    std::vector<double> csum(n + 1, 0.0);
    for (int64_t j = 0; j < n; ++j) csum[j + 1] = csum[j] + (double)S.colcount[j];
    for (int64_t s = 0; s < ns; ++s) {
      fstart[s] = S.sup_ptr[s];
      if (!S.relax || fstart[s] == 0) continue;
      const int32_t c = S.col2sn[fstart[s] - 1];
      if (sparent[c] != s) continue;
      const int32_t l = S.sup_ptr[s + 1] - 1;
      const double k = (double)(l - fstart[c] + 1);
      const double nf = k + fs_m[s];
      const double total = k * nf - k * (k - 1) / 2.0;
      const double zfrac = (total - (csum[l + 1] - csum[fstart[c]])) / total;
      const bool merge = k <= 4 || (k <= 16 && zfrac < 0.8) || (k <= 48 && zfrac < 0.1) ||
                         zfrac < 0.05;
      if (merge) {
        fstart[s] = fstart[c];
        is_top[c] = 0;
      }
    }
  }
  std::vector<int32_t> tops;
  for (int64_t s = 0; s < ns; ++s)
    if (is_top[s]) tops.push_back((int32_t)s);
  const int64_t nfr = (int64_t)tops.size();
  S.front_ptr.assign(nfr + 1, 0);
  std::vector<int32_t> fs2front(ns, -1);
  for (int64_t F = 0; F < nfr; ++F) {
    S.front_ptr[F] = fstart[tops[F]];
    for (int32_t s = S.col2sn[fstart[tops[F]]]; s <= tops[F]; ++s) fs2front[s] = (int32_t)F;
  }
  S.front_ptr[nfr] = (int32_t)n;
  S.col2front.assign(n, 0);
  for (int64_t F = 0; F < nfr; ++F)
    for (int32_t j = S.front_ptr[F]; j < S.front_ptr[F + 1]; ++j) S.col2front[j] = (int32_t)F;

  // front tree and children lists (children in increasing order)
  std::vector<int32_t> fparent(nfr, -1), fchild_cnt(nfr + 1, 0);
  for (int64_t F = 0; F < nfr; ++F) {
    const int32_t sp = sparent[tops[F]];
    fparent[F] = sp < 0 ? -1 : fs2front[sp];
    if (fparent[F] >= 0) fchild_cnt[fparent[F] + 1]++;
  }
  for (int64_t F = 0; F < nfr; ++F) fchild_cnt[F + 1] += fchild_cnt[F];
  S.children.assign(fchild_cnt[nfr], 0);
  {
    std::vector<int32_t> fillc(fchild_cnt.begin(), fchild_cnt.end() - 1);
    for (int64_t F = 0; F < nfr; ++F)
      if (fparent[F] >= 0) S.children[fillc[fparent[F]]++] = (int32_t)F;
  }

  timer.mark("amalgamation + front tree");
  // ---- 8. front row lists, relative maps, levels
  S.sn.assign(nfr, SnInfo{});
  S.slevel.assign(nfr, 0);
  S.rowidx.clear();
  S.relmap.clear();
  int64_t Loff = 0, woff = 0, map_off = 0;
  S.max_front = 0;
  S.max_k = 0;
  S.front_flops = 0.0;
  S.nlevels = nfr > 0 ? 1 : 0;
  {
    std::vector<int32_t> posn(n, -1), stamp(n, -1), mark(n, -1), upd;
    for (int64_t F = 0; F < nfr; ++F) {
      const int32_t top = tops[F];
      const int32_t f = S.front_ptr[F], l = S.front_ptr[F + 1] - 1, k = l - f + 1;
      // update rows: entries of C below the front's columns, plus the
      // children's update rows below them (the multifrontal structure)
      upd.clear();
      for (int32_t j = f; j <= l; ++j)
        for (int64_t p = cp[j]; p < cp[j + 1]; ++p) {
          const int32_t i = cr[p];
          if (i > l && mark[i] != F) {
            mark[i] = (int32_t)F;
            upd.push_back(i);
          }
        }
      for (int32_t ci = fchild_cnt[F]; ci < fchild_cnt[F + 1]; ++ci) {
        const SnInfo& C = S.sn[S.children[ci]];
        const int32_t* crow = S.rowidx.data() + C.rows_off + C.k;
        for (int32_t t = 0; t < C.m; ++t) {
          const int32_t r = crow[t];
          if (r > l && mark[r] != F) {
            mark[r] = (int32_t)F;
            upd.push_back(r);
          }
        }
      }
      std::sort(upd.begin(), upd.end());
      const int32_t m = (int32_t)upd.size();
      if (m != fs_m[top]) {
        err = "front update rows disagree with the column counts";
        return MF_ERR_INTERNAL;
      }
      SnInfo& I = S.sn[F];
      I.first = f;
      I.k = k;
      I.m = m;
      I.parent = fparent[F];
      I.child_begin = fchild_cnt[F];
      I.nchild = fchild_cnt[F + 1] - fchild_cnt[F];
      I.Loff = Loff;
      I.Uoff = 0;
      I.rows_off = (int64_t)S.rowidx.size();
      I.map_off = map_off;
      I.woff = woff;
      const int64_t nf = (int64_t)k + m;
      Loff += nf * k;
      woff += nf;
      map_off += m;
      S.max_front = std::max<int64_t>(S.max_front, nf);
      S.max_k = std::max<int64_t>(S.max_k, k);
      for (int64_t t = 0; t < k; ++t) S.front_flops += (double)(nf - t) * (double)(nf - t);
      for (int32_t j = f; j <= l; ++j) S.rowidx.push_back(j);
      for (int32_t t = 0; t < m; ++t) {
        S.rowidx.push_back(upd[t]);
        posn[upd[t]] = k + t;
        stamp[upd[t]] = (int32_t)F;
      }
      S.relmap.resize(map_off);
      int32_t lev = 0;
      for (int32_t ci = fchild_cnt[F]; ci < fchild_cnt[F + 1]; ++ci) {
        const int32_t c = S.children[ci];
        const SnInfo& C = S.sn[c];
        const int32_t* crow = S.rowidx.data() + C.rows_off + C.k;
        int32_t* cmap = S.relmap.data() + C.map_off;
        for (int32_t t = 0; t < C.m; ++t) {
          const int32_t r = crow[t];
          if (r >= f && r <= l) {
            cmap[t] = r - f;
          } else if (r > l && stamp[r] == F) {
            cmap[t] = posn[r];
          } else {
            err = "update row of a child front outside its parent front";
            return MF_ERR_INTERNAL;
          }
        }
        lev = std::max(lev, S.slevel[c] + 1);
      }
      S.slevel[F] = lev;
      S.nlevels = std::max(S.nlevels, lev + 1);
    }
  }
  timer.mark("front rows + maps");
  S.Lsize = Loff;
  S.Wsize = woff;
  S.Usize = plan_update_memory(S, std::vector<char>(S.sn.size(), 0));
  S.low_cp = std::move(cp);
  S.low_cr = std::move(cr);
  timer.mark("update-memory plan");
  // inverse of the relative maps for the forward solve: for every front row
  // (global index woff + i) the global rows (child woff + child row) of the
  // children's update entries that add into it, children in increasing order
  // (deterministic sums)
  S.ginv_ptr.assign(S.Wsize + 1, 0);
  for (int64_t F = 0; F < nfr; ++F) {
    const SnInfo& P = S.sn[F];
    for (int32_t ci = P.child_begin; ci < P.child_begin + P.nchild; ++ci) {
      const SnInfo& C = S.sn[S.children[ci]];
      const int32_t* cmap = S.relmap.data() + C.map_off;
      for (int32_t t = 0; t < C.m; ++t) S.ginv_ptr[P.woff + cmap[t] + 1]++;
    }
  }
  for (int64_t i = 0; i < S.Wsize; ++i) S.ginv_ptr[i + 1] += S.ginv_ptr[i];
  S.ginv_src.assign(S.ginv_ptr[S.Wsize], 0);
  {
    std::vector<int64_t> fillg(S.ginv_ptr.begin(), S.ginv_ptr.end() - 1);
    for (int64_t F = 0; F < nfr; ++F) {
      const SnInfo& P = S.sn[F];
      for (int32_t ci = P.child_begin; ci < P.child_begin + P.nchild; ++ci) {
        const int32_t c = S.children[ci];
        const SnInfo& C = S.sn[c];
        const int32_t* cmap = S.relmap.data() + C.map_off;
        for (int32_t t = 0; t < C.m; ++t)
          S.ginv_src[fillg[P.woff + cmap[t]]++] = C.woff + C.k + t;
      }
    }
  }

  timer.mark("gather maps");
  // ---- 9. assembly map of the lower triangle of C (incl. diagonal).  Rows
  // are visited in increasing permuted order, so each column's entries come
  // out sorted by row with duplicates adjacent; front-relative rows come from
  // a per-front position marker.
  {
    std::vector<int64_t> ccount(n + 1, 0);
    for (int64_t i = 0; i < n; ++i) {
      const int32_t ro = S.perm[i];
      for (int64_t p = rowptr[ro]; p < rowptr[ro + 1]; ++p)
        if (ip[colind[p]] <= i) ccount[ip[colind[p]] + 1]++;
    }
    for (int64_t j = 0; j < n; ++j) ccount[j + 1] += ccount[j];
    std::vector<int32_t> erow(ccount[n]);
    std::vector<int64_t> esrc(ccount[n]);
    {
      std::vector<int64_t> fillp(ccount.begin(), ccount.end() - 1);
      for (int64_t i = 0; i < n; ++i) {
        const int32_t ro = S.perm[i];
        for (int64_t p = rowptr[ro]; p < rowptr[ro + 1]; ++p) {
          const int32_t j = ip[colind[p]];
          if (j <= i) {
            erow[fillp[j]] = (int32_t)i;
            esrc[fillp[j]++] = p;
          }
        }
      }
    }
    S.acol_ptr.assign(n + 1, 0);
    S.arow.clear();
    S.asrc_ptr.clear();
    S.asrc.clear();
    S.arow.reserve(ccount[n]);
    S.asrc_ptr.reserve(ccount[n] + 1);
    S.asrc.reserve(ccount[n]);
    S.asrc_ptr.push_back(0);
    std::vector<int32_t> posn(n, -1);
    for (int64_t F = 0; F < (int64_t)S.sn.size(); ++F) {
      const SnInfo& I = S.sn[F];
      const int32_t* frows = S.rowidx.data() + I.rows_off;
      for (int32_t r = 0; r < I.k + I.m; ++r) posn[frows[r]] = r;
      for (int32_t j = I.first; j < I.first + I.k; ++j) {
        for (int64_t e = ccount[j]; e < ccount[j + 1]; ++e) {
          const int32_t i = erow[e];
          if (e == ccount[j] || erow[e - 1] != i) {
            const int32_t r = posn[i];
            if (r < 0 || frows[r] != i) {
              err = "entry of A outside its front";
              return MF_ERR_INTERNAL;
            }
            S.arow.push_back(r);
            S.asrc_ptr.push_back(S.asrc_ptr.back());
          }
          S.asrc.push_back(esrc[e]);
          S.asrc_ptr.back()++;
        }
        S.acol_ptr[j + 1] = (int64_t)S.arow.size();
      }
    }
    S.nnz_lower = (int64_t)S.arow.size();
  }
  timer.mark("assembly map");
  return MF_OK;
}

// SpTRSV variant 4 (Sec. 5): the level's partitioned inverse L_l^{-1} as one
// sparse product per level and sweep, on the permuted global vector (no
// front work vectors, no flags).  Forward, level l: for every front s of the
// level, P_s = [L11^{-1}; -L21 L11^{-1}] maps the front's pivot values y(s)
// to its pivot results (replace: F(r) = row of P11 times y(s)) and to
// additions into its update rows (y(r) += row of P21 times y(s)); an update
// row shared by several fronts of the level is one row of the level's
// matrix whose entries are those fronts' rows of P, in front order.  Items:
// one per row of the level's matrix, (global row, first group, end group,
// pivot?), with groups (front, front row) in S.v4_grp.  Backward, level l:
// x(first_s + c) = column c of P_s (rows c .. nf-1) times [F of the pivot
// rows; x of the update rows]; items (front, column).  Every large front
// (with kept diagonal inverses) takes the blocked partitioned inverse;
// the others are returned in `pinv` as empty and get the one-CTA kernel.
template <class Add>
static void build_v4_solves(mf_symbolic& S, const std::vector<std::vector<int32_t>>& bylev,
                            Add& add, std::vector<int32_t>& pinv) {
  const int64_t n = S.n;
  std::vector<int32_t> stamp(n, -1), slot(n, -1);
  std::vector<std::vector<Item>> groups;  // per level row: its groups
  std::vector<Item> it;
  for (int32_t lev = 0; lev < S.nlevels; ++lev) {
    const std::vector<int32_t>& L = bylev[lev];
    std::vector<int32_t> rows;
    std::vector<char> pivot;
    groups.clear();
    for (int32_t s : L) {
      const SnInfo& f = S.sn[s];
      if (S.ioff[s] >= 0) pinv.push_back(s);
      const int nf = f.k + f.m;
      const int32_t* rw = S.rowidx.data() + f.rows_off;
      for (int i = 0; i < nf; ++i) {
        const int32_t r = rw[i];
        if (stamp[r] != lev) {
          stamp[r] = lev;
          slot[r] = (int32_t)rows.size();
          rows.push_back(r);
          pivot.push_back(i < f.k ? 1 : 0);
          groups.emplace_back();
        }
        groups[slot[r]].push_back({s, i, 0, 0});
      }
    }
    it.clear();
    for (size_t q = 0; q < rows.size(); ++q) {
      const int32_t g0 = (int32_t)S.v4_grp.size();
      S.v4_grp.insert(S.v4_grp.end(), groups[q].begin(), groups[q].end());
      it.push_back({rows[q], g0, (int32_t)S.v4_grp.size(), pivot[q]});
    }
    add(S.fwsched, K_V4_FW, lev, 0, it, 0.0);
  }
  for (int32_t lev = S.nlevels - 1; lev >= 0; --lev) {
    it.clear();
    for (int32_t s : bylev[lev])
      for (int c = 0; c < S.sn[s].k; ++c) it.push_back({s, c, 0, 0});
    add(S.bwsched, K_V4_BW, lev, 0, it, 0.0);
  }
}

// Launch schedules of the numeric factorization and of the solves.  Fronts
// of one level are independent (paper Sec. 5: level-set scheduling); small
// fronts are batched one CTA each (grouped by size class), large fronts are
// split into column chunks (assembly), panel steps (POTRF, TRSM) and trailing
// tiles (SYRK), each batched over all large fronts of the level.
// Front-size buckets of the per-bucket trailing-update choice (k + m of a
// large front): <= 512, <= 2048, <= 8192, larger.
int tile_bucket(int nf) { return nf <= 512 ? 0 : nf <= 2048 ? 1 : nf <= 8192 ? 2 : 3; }

void build_schedules(mf_symbolic& S, int small_max, int small_queue, const int32_t* update_tile) {
  S.items.clear();
  S.arange.clear();
  S.fsched.clear();
  S.fsched_tc.clear();
  S.soff.assign(S.sn.size(), 0);
  S.split_rows = 0;
  S.split_rows_b = 0;
  S.max_large = 0;
  S.ioff.assign(S.sn.size(), -1);
  S.ninv = 0;
  S.fwsched.clear();
  S.bwsched.clear();
  const int64_t ns = (int64_t)S.sn.size();
  std::vector<std::vector<int32_t>> bylev(S.nlevels);
  for (int64_t s = 0; s < ns; ++s) bylev[S.slevel[s]].push_back((int32_t)s);
  const int classes[3] = {32, 64, 128};
  auto add = [&](std::vector<Launch>& sched, int32_t kind, int32_t lev, int32_t param,
                 const std::vector<Item>& it, double flops, int side = 0, int join = 0,
                 int area = 0, int tile = 0) {
    if (it.empty()) return;
    Launch L;
    L.tile = (uint8_t)tile;
    L.kind = kind;
    L.level = lev;
    L.count = (int32_t)it.size();
    L.param = param;
    L.item_off = (int64_t)S.items.size();
    L.flops = flops;
    L.side = (int8_t)side;
    L.join = (int8_t)join;
    L.area = (int8_t)area;
    S.items.insert(S.items.end(), it.begin(), it.end());
    sched.push_back(L);
  };
  auto front_flops = [](int64_t nf, int64_t k) {
    double f = 0.0;
    for (int64_t t = 0; t < k; ++t) f += (double)(nf - t) * (double)(nf - t);
    return f;
  };
  std::vector<Item> it;
  // Persistent queue: the small fronts whose whole subtree is small run in
  // one launch before everything else, in ticket order = level order (a
  // front's children always have smaller tickets); each waits for its
  // children's completion flags instead of a level barrier.
  std::vector<char> inq(ns, 0);
  // fronts up to qmax rows join the queue (option 1: the default of 64, which
  // keeps the queue's shared memory small enough for many CTAs per SM)
  const int qmax = std::min(small_max, small_queue == 1 ? 64 : small_queue);
  if (small_queue) {
    std::vector<char>& closed = inq;
    for (int32_t lev = 0; lev < S.nlevels; ++lev)
      for (int32_t s : bylev[lev]) {
        const SnInfo& P = S.sn[s];
        bool ok = P.k + P.m <= qmax;
        for (int32_t ci = P.child_begin; ok && ci < P.child_begin + P.nchild; ++ci)
          ok = closed[S.children[ci]] != 0;
        closed[s] = ok ? 1 : 0;
      }
  }
  // the update-matrix plan follows the execution order of the schedule
  S.Usize = plan_update_memory(S, inq);
  if (small_queue) {
    it.clear();
    double fl = 0.0;
    int32_t maxnf = 0;
    for (int32_t lev = 0; lev < S.nlevels; ++lev)
      for (int32_t s : bylev[lev])
        if (inq[s]) {
          const int nf = S.sn[s].k + S.sn[s].m;
          it.push_back({s, 0, 0, 0});
          fl += front_flops(nf, S.sn[s].k);
          maxnf = std::max(maxnf, nf);
        }
    add(S.fsched, K_SMALL_Q, 0, maxnf, it, fl);
    add(S.fsched_tc, K_SMALL_Q, 0, maxnf, it, fl);
  }
  for (int32_t lev = 0; lev < S.nlevels; ++lev) {
    const std::vector<int32_t>& L = bylev[lev];
    // small fronts by class
    for (int c = 0; c < 3; ++c) {
      const int lo = c == 0 ? 0 : classes[c - 1];
      const int hi = std::min(classes[c], small_max);
      if (hi <= lo) continue;
      it.clear();
      double fl = 0.0;
      for (int32_t s : L) {
        const int nf = S.sn[s].k + S.sn[s].m;
        if (nf > lo && nf <= hi && !inq[s]) {
          it.push_back({s, 0, 0, 0});
          fl += front_flops(nf, S.sn[s].k);
        }
      }
      add(S.fsched, K_SMALL, lev, hi, it, fl);
      add(S.fsched_tc, K_SMALL, lev, hi, it, fl);
    }
    // large fronts
    std::vector<int32_t> G;
    for (int32_t s : L)
      if (S.sn[s].k + S.sn[s].m > small_max) G.push_back(s);
    if (G.empty()) continue;
    it.clear();
    int32_t T = 0;
    for (int32_t s : G) {
      const SnInfo& P = S.sn[s];
      const int nf = P.k + P.m;
      for (int c0 = 0; c0 < nf; c0 += kAsmCols) {
        const int c1 = std::min(c0 + kAsmCols, nf);
        // children whose update columns land in [c0, c1): (child, lo, hi)
        // ranges of their columns, closed by a sentinel
        const int32_t off = (int32_t)S.arange.size();
        for (int32_t ci = P.child_begin; ci < P.child_begin + P.nchild; ++ci) {
          const int32_t c = S.children[ci];
          const SnInfo& C = S.sn[c];
          const int32_t* map = S.relmap.data() + C.map_off;
          const int32_t lo = (int32_t)(std::lower_bound(map, map + C.m, c0) - map);
          const int32_t hi = (int32_t)(std::lower_bound(map, map + C.m, c1) - map);
          if (hi > lo) S.arange.push_back({c, lo, hi, 0});
        }
        S.arange.push_back({-1, 0, 0, 0});
        it.push_back({s, off, c0, c1});
      }
      T = std::max<int32_t>(T, (P.k + kNB - 1) / kNB);
    }
    add(S.fsched, K_ASSEMBLE, lev, 0, it, 0.0);
    add(S.fsched_tc, K_ASSEMBLE, lev, 0, it, 0.0);
    // rows of the split buffer: the level's large fronts side by side, in
    // the eight-slot area on lookahead levels (four slots elsewhere)
    const bool la = (int)G.size() <= kLookaheadFronts;
    int64_t srow = 0;
    for (int32_t s : G) {
      S.soff[s] = srow | (la ? (int64_t)1 << kSoffAreaShift : 0);
      srow += S.sn[s].k + S.sn[s].m;
    }
    if (la) S.split_rows_b = std::max(S.split_rows_b, srow);
    else S.split_rows = std::max(S.split_rows, srow);
    S.max_large = std::max<int64_t>(S.max_large, (int64_t)G.size());
    if (S.keep_inv)
      for (int32_t s : G) {
        S.ioff[s] = S.ninv;
        S.ninv += (S.sn[s].k + kNB - 1) / kNB;
      }
    // per front: the FMA tile of the FP64 / FP32-FMA schedule and, in the
    // tensor-core schedule, tensor cores or that FMA tile (update_tile code
    // of the front's size bucket: 0 default, 1 FMA 64, 2 FMA 128, 3 tensor
    // cores, 4 FMA 32; the FMA schedule takes 32 for 0 and 3, the tile that
    // measured fastest for FP64 on GB300: most CTAs per SM for the
    // read-modify-write of the trailing tiles)
    auto code_of = [&](int32_t s) {
      const int c = update_tile ? update_tile[tile_bucket(S.sn[s].k + S.sn[s].m)] : 0;
      return c < 0 || c > 4 ? 0 : c;
    };
    auto fma_tile = [&](int32_t s) {
      const int c = code_of(s);
      return c == 1 ? 64 : c == 2 ? 128 : 32;
    };
    auto uses_tc = [&](int32_t s) { return code_of(s) == 0 || code_of(s) == 3; };
    for (int32_t t = 0; t < T; ++t) {
      std::vector<Item> ip, it3, itc;
      std::vector<Item> is[3], isf[3];  // FMA tiles 32 / 64 / 128: FP64 and FP32-TC schedules
      double fp = 0, ft = 0, fs[3] = {0, 0, 0}, fsf[3] = {0, 0, 0}, fstc = 0;
      auto tix = [](int T) { return T == 32 ? 0 : T == 64 ? 1 : 2; };
      bool group_end = false;  // a tensor-core front ends its group of panels this step
      for (size_t gi = 0; gi < G.size(); ++gi) {
        const int32_t s = G[gi];
        // slot of the diagonal-block inverse: per level, or kept per block
        const int lpos = S.keep_inv ? (int)(S.ioff[s] + t) : (int)gi;
        const int k = S.sn[s].k, nf = k + S.sn[s].m;
        if (k <= t * kNB) continue;
        const int b = std::min(kNB, k - t * kNB);
        const int p0 = t * kNB + b;
        ip.push_back({s, t, 0, lpos});
        fp += (double)b * b * b / 3.0;
        for (int r0 = p0; r0 < nf; r0 += kTrsmRows) it3.push_back({s, t, r0, lpos});
        ft += (double)(nf - p0) * b * b;
        const int Tf = fma_tile(s), x = tix(Tf);
        const int nt = (nf - p0 + Tf - 1) / Tf;
        for (int I = 0; I < nt; ++I)
          for (int J = 0; J <= I; ++J) is[x].push_back({s, t, I, J});
        const double full = (double)(nf - p0) * (double)(nf - p0 + 1) * b;
        fs[x] += full;
        if (!uses_tc(s)) {  // the tensor-core schedule takes the FMA tile too
          isf[x].insert(isf[x].end(), is[x].end() - (int64_t)nt * (nt + 1) / 2, is[x].end());
          fsf[x] += full;
          continue;
        }
        // tensor-core path: panels in groups of four (g0 .. gl), the
        // trailing matrix read and written once per group (K up to 256).
        // Inside a group the next panel's columns are brought up to date
        // left-looking: after panel t < gl a strip updates the 64 columns of
        // panel t + 1 with panels g0 .. t; after gl one pass updates
        // everything beyond gl with the whole group.  Item field t packs the
        // group's first panel, the number of panels applied and the strip
        // flag.
        const int nt2 = (nf - p0 + kTcTile - 1) / kTcTile;
        const int g0 = t & ~3;
        const int gl = std::min(g0 + 3, (k - 1) / kNB);
        if (t < gl) {
          const int nK = t - g0 + 1;
          const int b1 = std::min(kNB, k - (t + 1) * kNB);
          for (int I = 0; I < nt2; ++I) itc.push_back({s, g0 | (nK << 16) | (1 << 24), I, 0});
          fstc += 2.0 * (double)kNB * nK * ((double)b1 * (nf - p0) - (double)b1 * (b1 - 1) / 2.0);
        } else {
          const int nK = gl - g0 + 1;
          for (int I = 0; I < nt2; ++I)
            for (int J = 0; J <= I; ++J) itc.push_back({s, g0 | (nK << 16), I, J});
          const double Kw = (double)kNB * (nK - 1) + b;
          fstc += Kw * (double)(nf - p0) * (double)(nf - p0 + 1);
          group_end = true;
        }
      }
      static const int kTiles[3] = {32, 64, 128};
      add(S.fsched, K_POTRF, lev, t, ip, fp);
      add(S.fsched, K_TRSM, lev, t, it3, ft);
      add(S.fsched_tc, K_POTRF, lev, t, ip, fp, 0, 0, la);
      add(S.fsched_tc, K_TRSM, lev, t, it3, ft, 0, 0, la);
      if (!la) {
        for (int x = 0; x < 3; ++x) {
          add(S.fsched, K_SYRK, lev, t, is[x], fs[x], 0, 0, 0, kTiles[x]);
          add(S.fsched_tc, K_SYRK, lev, t, isf[x], fsf[x], 0, 0, 0, kTiles[x]);
        }
        add(S.fsched_tc, K_SYRK_TC, lev, t, itc, fstc);
        continue;
      }
      // lookahead: the first tile column of a trailing update (the next
      // panel's columns) runs on the main stream after the side stream has
      // finished the previous bulk; the other tiles run on the side stream
      // while the next panel is factored.  The flop split is by tile count.
      auto split_j0 = [](const std::vector<Item>& v, std::vector<Item>& a, std::vector<Item>& b) {
        for (const Item& x : v) (x.b == 0 ? a : b).push_back(x);
      };
      // FMA tiles: the tile columns covering the next panel (J T < 64) on the
      // critical stream, the rest on the side stream
      auto fma_split = [&](std::vector<Launch>& sched, const std::vector<Item>& v, double fl, int T) {
        std::vector<Item> a, b;
        for (const Item& x : v) (x.b * T < kNB ? a : b).push_back(x);
        const double fa = v.empty() ? 0.0 : fl * (double)a.size() / (double)v.size();
        add(sched, K_SYRK, lev, t, a, fa, 0, 1, 0, T);
        add(sched, K_SYRK, lev, t, b, fl - fa, 1, 0, 0, T);
      };
      for (int x = 0; x < 3; ++x) {
        fma_split(S.fsched, is[x], fs[x], kTiles[x]);
        fma_split(S.fsched_tc, isf[x], fsf[x], kTiles[x]);
      }
      // tensor cores: the strips (next panel only) and the first two tile
      // columns of a group pass (the next group's four panels) on the
      // critical stream, after the previous group's bulk (join); the rest
      // of the pass on the side stream.  A group's bulk on the side stream
      // runs while the next group's panels are factored: their staging slots
      // differ (eight per row on lookahead levels), and their strips touch
      // only columns inside those two tile columns.
      {
        std::vector<Item> a, b;
        for (const Item& x : itc) ((x.t >> 24) != 0 || x.b * kTcTile < 4 * kNB ? a : b).push_back(x);
        const double fa = itc.empty() ? 0.0 : fstc * (double)a.size() / (double)itc.size();
        add(S.fsched_tc, K_SYRK_TC, lev, t, a, fa, 0, group_end ? 1 : 0, 1);
        add(S.fsched_tc, K_SYRK_TC, lev, t, b, fstc - fa, 1, 0, 1);
      }
    }
  }
  // ---- solves.  Per level and sweep, fronts with k + m <= kWarpSolve go to
  // the one-warp kernels (no waits, one launch per row class, 32 H rows with
  // H = 2, 4, 8, 16) unless the class is too sparse to fill the GPU and the
  // front has a long pivot chain (k > 64) or more than 128 rows (one warp
  // would stream all its update rows alone); all other fronts are split into
  // 64-row blocks for the sync-free level kernel.  Level-kernel items are
  // taken in ticket order, so a block only waits on blocks with earlier
  // tickets; they are ordered by depth in their front's chain (every
  // front's first block, then every front's second, ...), so the resident
  // blocks are the frontier of all chains rather than the tail of a few.
  S.blkoff.assign(ns + 1, 0);
  for (int64_t s = 0; s < ns; ++s) S.blkoff[s + 1] = S.blkoff[s] + (S.sn[s].k + kNB - 1) / kNB;
  constexpr size_t kWarpMinFronts = 2048;
  auto warp_class = [](int nf) { return nf <= 64 ? 0 : nf <= 128 ? 1 : nf <= 256 ? 2 : 3; };
  // split a level's fronts into warp classes and level-kernel fronts
  auto split_level = [&](const std::vector<int32_t>& L, std::vector<Item> (&wcls)[4],
                         std::vector<int32_t>& big) {
    std::vector<int32_t> cls[4];
    big.clear();
    for (int32_t s : L) {
      const int nf = S.sn[s].k + S.sn[s].m;
      if (nf <= kWarpSolve) cls[warp_class(nf)].push_back(s);
      else big.push_back(s);
    }
    for (int c = 0; c < 4; ++c) {
      wcls[c].clear();
      const bool sparse = cls[c].size() < kWarpMinFronts;
      for (int32_t s : cls[c]) {
        if (sparse && (S.sn[s].k > 2 * 32 || c >= 2)) big.push_back(s);
        else wcls[c].push_back({s, 0, 0, 0});
      }
    }
  };
  std::vector<int32_t> all_pinv;
  S.v4_grp.clear();
  if (S.v4) {
    build_v4_solves(S, bylev, add, all_pinv);
  } else {
  std::vector<std::vector<Item>> bydepth;
  auto flatten = [&](std::vector<Item>& out) {
    out.clear();
    for (auto& v : bydepth) {
      out.insert(out.end(), v.begin(), v.end());
      v.clear();
    }
  };
  std::vector<Item> wcls[4], upd, pg, pv;
  std::vector<int32_t> big, pfronts;
  // SpTRSV variant 3: large fronts of the factor (those with kept diagonal
  // inverses) that the solve takes as level-kernel fronts use the
  // partitioned inverse instead of the chained pivot blocks
  auto take_pinv = [&](std::vector<int32_t>& B, std::vector<int32_t>& P) {
    P.clear();
    if (!S.pinv) return;
    size_t w = 0;
    for (int32_t s : B) {
      if (S.ioff[s] >= 0) P.push_back(s);
      else B[w++] = s;
    }
    B.resize(w);
  };
  for (int32_t lev = 0; lev < S.nlevels; ++lev) {
    split_level(bylev[lev], wcls, big);
    take_pinv(big, pfronts);
    all_pinv.insert(all_pinv.end(), pfronts.begin(), pfronts.end());
    pg.clear();
    pv.clear();
    for (int32_t s : pfronts) {
      const int k = S.sn[s].k, m = S.sn[s].m;
      for (int r0 = 0; r0 < k; r0 += kNB) {
        pg.push_back({s, 0, r0, std::min(kNB, k - r0)});
        pv.push_back({s, 0, r0, std::min(kNB, k - r0)});
      }
      for (int r0 = 0; r0 < m; r0 += kNB) pv.push_back({s, 1, k + r0, std::min(kNB, m - r0)});
    }
    upd.clear();
    for (int32_t s : big) {
      const int k = S.sn[s].k, m = S.sn[s].m;
      for (int r0 = 0, dpt = 0; r0 < k; r0 += kNB, ++dpt) {
        if ((int)bydepth.size() <= dpt) bydepth.resize(dpt + 1);
        bydepth[dpt].push_back({s, 0, r0, std::min(kNB, k - r0)});
      }
      for (int r0 = 0; r0 < m; r0 += kNB) upd.push_back({s, 1, k + r0, std::min(kNB, m - r0)});
    }
    flatten(it);
    for (int c = 0; c < 4; ++c) add(S.fwsched, K_FW_WARP, lev, 2 << c, wcls[c], 0.0);
    // pivot blocks (chains within a front), then the update-row blocks
    // of the level as a streaming product that never waits
    add(S.fwsched, K_FW_LEVEL, lev, 0, it, 0.0);
    // one CTA per 64 update rows when every front has at most kFwNarrowK
    // pivot columns (tile 2 up to 128 of them, 1 beyond), else four (tile 0)
    {
      int maxk = 0;
      for (const Item& x : upd) maxk = std::max(maxk, S.sn[x.s].k);
      add(S.fwsched, K_FW_GEMV, lev, 0, upd, 0.0, 0, 0, 0, fw_gemv_tile(maxk));
    }
    // variant 3: gather the pivot rows' w, then one product per row block
    add(S.fwsched, K_FW_PGATHER, lev, 0, pg, 0.0);
    add(S.fwsched, K_FW_PINV, lev, 0, pv, 0.0);
  }
  for (int32_t lev = S.nlevels - 1; lev >= 0; --lev) {
    split_level(bylev[lev], wcls, big);
    take_pinv(big, pfronts);
    pg.clear();
    pv.clear();
    for (int32_t s : pfronts) {
      const int k = S.sn[s].k;
      for (int c0 = 0; c0 < k; c0 += kNB) {
        pg.push_back({s, 0, c0, std::min(kNB, k - c0)});
        pv.push_back({s, 0, c0, std::min(kNB, k - c0)});
      }
    }
    for (int32_t s : big) {
      const int k = S.sn[s].k;
      int dpt = 0;
      for (int c0 = ((k - 1) / kNB) * kNB; c0 >= 0; c0 -= kNB, ++dpt) {
        if ((int)bydepth.size() <= dpt) bydepth.resize(dpt + 1);
        bydepth[dpt].push_back({s, 0, c0, std::min(kNB, k - c0)});
      }
    }
    flatten(it);
    upd.clear();
    for (const Item& x : it)
      if (S.sn[x.s].m > 0) upd.push_back(x);
    for (int c = 0; c < 4; ++c) add(S.bwsched, K_BW_WARP, lev, 2 << c, wcls[c], 0.0);
    // update-row products of every column block first (no waiting), then the
    // chained triangles
    // CTAs per 64-column item: the row split of the launch's tallest front
    {
      int maxm = 0;
      for (const Item& x : upd) maxm = std::max(maxm, S.sn[x.s].m);
      add(S.bwsched, K_BW_GEMV, lev, 0, upd, 0.0, 0, 0, 0, bw_gemv_split(maxm));
    }
    add(S.bwsched, K_BW_LEVEL, lev, 1, it, 0.0);
    // variant 3: stage the pivot rows' y, then one product per column block
    add(S.bwsched, K_BW_PCOPY, lev, 0, pg, 0.0);
    add(S.bwsched, K_BW_PINV, lev, 0, pv, 0.0);
  }
  }  // variants 1-3
  // ---- partitioned inverse of the variant-3 fronts, after the whole
  // factorization: P = [L11; L21] X with L11 X = I solved by block rows,
  // right-looking.  Row blocks i of a front are its pivot blocks (i < nb)
  // then its 64-row blocks of update rows.  Init: P = 0 with the kept
  // diagonal inverses on the diagonal blocks.  Step t: every tile (i, j)
  // with i > t >= j takes P(i, j) -= L(i, t) P(t, j); a pivot tile with
  // i = t + 1 is then final after P(i, j) = L_ii^{-1} P(i, j).
  S.pinv_flops = 0.0;
  if (S.pinv && !all_pinv.empty()) {
    std::vector<Item> init;
    int32_t tmax = 0;
    for (int32_t s : all_pinv) {
      const int k = S.sn[s].k;
      for (int j = 0; j * kNB < k; ++j) init.push_back({s, j, 0, 0});
      tmax = std::max(tmax, (k + kNB - 1) / kNB);
    }
    const int32_t plev = S.nlevels;  // after every level of the factorization
    add(S.fsched, K_PINV_INIT, plev, 0, init, 0.0);
    add(S.fsched_tc, K_PINV_INIT, plev, 0, init, 0.0);
    std::vector<Item> st;
    for (int32_t t = 0; t < tmax; ++t) {
      st.clear();
      double fl = 0.0;
      for (int32_t s : all_pinv) {
        const int k = S.sn[s].k, m = S.sn[s].m;
        const int nb = (k + kNB - 1) / kNB, mb = (m + kNB - 1) / kNB;
        if (t >= nb) continue;
        const double bt = std::min(kNB, k - t * kNB);
        for (int i = t + 1; i < nb + mb; ++i) {
          const double ri = i < nb ? std::min(kNB, k - i * kNB) : std::min(kNB, m - (i - nb) * kNB);
          for (int j = 0; j <= t; ++j) {
            const double bj = std::min(kNB, k - j * kNB);
            st.push_back({s, t, i, j});
            fl += 2.0 * ri * bt * bj + (i == t + 1 && i < nb ? 2.0 * ri * ri * bj : 0.0);
          }
        }
      }
      S.pinv_flops += fl;
      add(S.fsched, K_PINV, plev, t, st, fl);
      add(S.fsched_tc, K_PINV, plev, t, st, fl);
    }
  }
  // ---- variant 4: the partitioned inverse of every other front (one CTA
  // each), then P transposed front by front (PT, rows of P contiguous) for
  // the forward products
  if (S.v4) {
    const int32_t plev = S.nlevels;
    std::vector<Item> sm, tr;
    double fl = 0.0;
    for (int64_t s = 0; s < ns; ++s) {
      const SnInfo& P = S.sn[s];
      if (S.ioff[s] < 0) {
        sm.push_back({(int32_t)s, 0, 0, 0});
        fl += (double)P.k * P.k * P.k / 3.0 + (double)P.m * P.k * P.k;
      }
      const int nf = P.k + P.m;
      for (int i = 0; i < nf; i += kNB)
        for (int j = 0; j < P.k; j += kNB) tr.push_back({(int32_t)s, 0, i, j});
    }
    S.pinv_flops += fl;
    int32_t maxnf = 0;
    for (const Item& x : sm) maxnf = std::max(maxnf, S.sn[x.s].k + S.sn[x.s].m);
    add(S.fsched, K_PINV_SMALL, plev, maxnf, sm, fl);
    add(S.fsched_tc, K_PINV_SMALL, plev, maxnf, sm, fl);
    add(S.fsched, K_PT, plev, 0, tr, 0.0);
    add(S.fsched_tc, K_PT, plev, 0, tr, 0.0);
  }
}

// Consistency of the launch schedules, checked on the host: every front's
// work appears exactly once, in launches of its own level, in level order.
//   factor: a small front is one K_SMALL item; a large front has assembly
//   chunks tiling [0, nf), one POTRF item per 64-column panel t, TRSM row
//   blocks tiling [p0, nf) after it, and (FP64 schedule) the trailing tiles
//   0 <= J <= I < nt of every panel exactly once; POTRF(t + 1) comes after
//   TRSM(t) and the first tile column of SYRK(t);
//   partitioned inverse: init column blocks tile [0, nb), and step t holds
//   the tiles t < i < nb + mb, 0 <= j <= t exactly once, steps in order;
//   small-front queue (first launch): each queued front once, after all of
//   its children, which are queued too;
//   solves: a front is one warp item (nf <= 32 H) or its pivot blocks tile
//   [0, k) (and, forward, its update blocks tile [k, nf)).
int check_schedules(const mf_symbolic& S, std::string& err) {
  const int64_t ns = (int64_t)S.sn.size();
  auto fail = [&](const std::string& m) {
    err = m;
    return MF_ERR_INTERNAL;
  };
  auto tiles = [&](const std::vector<std::pair<int, int>>& v, int lo, int hi, int step) {
    // v: (start, length) segments; must tile [lo, hi) in blocks of `step`
    std::vector<std::pair<int, int>> w(v);
    std::sort(w.begin(), w.end());
    int at = lo;
    for (const auto& x : w) {
      if (x.first != at || x.second <= 0 || x.second > step) return false;
      at += x.second;
    }
    return at == hi;
  };
  // the forward gather reads only update rows of the children's work
  // vectors, so the pivot rows of every front's work vector are free: the
  // chained pivot blocks pass their solved values through them
  if (!S.v4 && S.Wsize > 0) {
    std::vector<int32_t> owner(S.Wsize, -1);
    for (int64_t s = 0; s < ns; ++s)
      for (int64_t i = 0; i < (int64_t)S.sn[s].k + S.sn[s].m; ++i) {
        const int64_t g = S.sn[s].woff + i;
        if (g < 0 || g >= S.Wsize || owner[g] >= 0) return fail("work vectors overlap");
        owner[g] = (int32_t)s;
      }
    for (int64_t g : S.ginv_src) {
      if (g < 0 || g >= S.Wsize || owner[g] < 0) return fail("gather source outside a work vector");
      const SnInfo& c = S.sn[owner[g]];
      if (g - c.woff < c.k) return fail("gather source on a pivot row (a value slot)");
    }
  }
  for (const auto* schedp : {&S.fsched, &S.fsched_tc, &S.fwsched, &S.bwsched})
    for (const Launch& L : *schedp) {
      if (L.item_off < 0 || L.count < 0 || L.item_off + L.count > (int64_t)S.items.size())
        return fail("launch items out of range");
      for (int64_t x = L.item_off; x < L.item_off + L.count; ++x)
        if (S.items[x].s < 0 || S.items[x].s >= (L.kind == K_V4_FW ? S.n : ns))
          return fail(L.kind == K_V4_FW ? "row item out of range" : "item names no front");
    }
  auto nb_of = [&](int64_t s) { return (S.sn[s].k + kNB - 1) / kNB; };
  // ---- factor schedules
  for (int tc = 0; tc < 2; ++tc) {
    const std::vector<Launch>& sched = tc ? S.fsched_tc : S.fsched;
    std::vector<int> small(ns, 0);
    std::vector<std::vector<std::pair<int, int>>> asmb(ns);
    std::vector<std::vector<int>> potrf(ns);  // launch index per panel
    std::vector<std::vector<int64_t>> syrk_tiles(ns);
    std::vector<std::vector<std::vector<std::pair<int, int>>>> trsm(ns);
    std::vector<std::vector<int>> trsm_at(ns), syrk0_at(ns);
    std::vector<int> syrk_tile(ns, 0);  // FMA tile of a front (0: none seen)
    std::vector<std::vector<int64_t>> tc_tiles(ns);
    int32_t last_level = -1;
    for (size_t li = 0; li < sched.size(); ++li) {
      const Launch& L = sched[li];
      if (L.kind == K_PINV_INIT || L.kind == K_PINV || L.kind == K_PINV_SMALL || L.kind == K_PT)
        continue;
      if (L.kind == K_SMALL_Q) {
        // the persistent queue comes first; every front in it is small, and
        // every child of a queued front is queued with a smaller ticket
        if (li != 0) return fail("small-front queue not first");
        std::vector<int64_t> ticket(ns, -1);
        for (int64_t x = L.item_off; x < L.item_off + L.count; ++x) {
          const int32_t s = S.items[x].s;
          const SnInfo& f = S.sn[s];
          if (f.k + f.m > L.param || ticket[s] >= 0) return fail("queued front too large or repeated");
          ticket[s] = x - L.item_off;
          small[s]++;
          for (int32_t ci = f.child_begin; ci < f.child_begin + f.nchild; ++ci) {
            const int64_t tc_ = ticket[S.children[ci]];
            if (tc_ < 0 || tc_ >= ticket[s]) return fail("queued front before its children");
          }
        }
        continue;
      }
      if (L.level < last_level) return fail("factor levels out of order");
      last_level = L.level;
      for (int64_t x = L.item_off; x < L.item_off + L.count; ++x) {
        const Item& it = S.items[x];
        const SnInfo& f = S.sn[it.s];
        const int nf = f.k + f.m, nb = (int)nb_of(it.s);
        if (S.slevel[it.s] != L.level) return fail("factor item outside its front's level");
        if (potrf[it.s].empty()) {
          potrf[it.s].assign(nb, -1);
          trsm[it.s].assign(nb, {});
          trsm_at[it.s].assign(nb, -1);
          syrk0_at[it.s].assign(nb, -1);
        }
        switch (L.kind) {
          case K_SMALL:
            if (nf > L.param) return fail("small front above its size class");
            small[it.s]++;
            break;
          case K_ASSEMBLE:
            asmb[it.s].push_back({it.a, it.b - it.a});
            break;
          case K_POTRF:
            if (it.t != L.param || it.t < 0 || it.t >= nb || potrf[it.s][it.t] != -1)
              return fail("POTRF panel repeated or out of range");
            if (it.t > 0 && (trsm_at[it.s][it.t - 1] < 0 ||
                             (nf > it.t * kNB && syrk0_at[it.s][it.t - 1] < 0 && !tc)))
              return fail("POTRF before the previous panel's TRSM / first update column");
            potrf[it.s][it.t] = (int)li;
            break;
          case K_TRSM:
            if (it.t != L.param || it.t < 0 || it.t >= nb || potrf[it.s][it.t] < 0)
              return fail("TRSM before its panel's POTRF");
            trsm[it.s][it.t].push_back({it.a, std::min(kTrsmRows, nf - it.a)});
            trsm_at[it.s][it.t] = (int)li;
            break;
          case K_SYRK: {
            const int t = it.t;
            const int Tl = L.tile ? L.tile : kTile;
            if (Tl != 32 && Tl != 64 && Tl != 128) return fail("SYRK tile size");
            if (syrk_tile[it.s] == 0) syrk_tile[it.s] = Tl;
            if (syrk_tile[it.s] != Tl) return fail("front with two SYRK tile sizes");
            const int p0 = t * kNB + std::min(kNB, f.k - t * kNB);
            const int nt = (nf - p0 + Tl - 1) / Tl;
            if (t != L.param || t < 0 || t >= nb || it.b < 0 || it.b > it.a || it.a >= nt)
              return fail("SYRK tile out of range");
            syrk_tiles[it.s].push_back(((int64_t)t << 40) | ((int64_t)it.a << 20) | it.b);
            // the tile columns covering the next panel
            if (it.b * Tl < kNB) syrk0_at[it.s][t] = (int)li;
            break;
          }
          case K_SYRK_TC:
            // (group first panel, panels, strip, I, J) in 8/4/1/24/24 bits
            tc_tiles[it.s].push_back(((int64_t)(it.t & 0xffff) << 40) |
                                     ((int64_t)((it.t >> 16) & 0xff) << 36) |
                                     ((int64_t)(it.t >> 24) << 35) | ((int64_t)it.a << 17) | it.b);
            break;
          default:
            return fail("unknown factor kind");
        }
      }
    }
    for (int64_t s = 0; s < ns; ++s) {
      const SnInfo& f = S.sn[s];
      const int nf = f.k + f.m, nb = (int)nb_of(s);
      if (small[s]) {
        if (small[s] != 1 || !asmb[s].empty()) return fail("small front scheduled twice");
        continue;
      }
      if (!tiles(asmb[s], 0, nf, kAsmCols)) return fail("assembly chunks do not tile the front");
      if ((int)potrf[s].size() != nb) return fail("large front without panels");
      int64_t want = 0;
      for (int t = 0; t < nb; ++t) {
        if (potrf[s][t] < 0) return fail("panel without POTRF");
        const int p0 = t * kNB + std::min(kNB, f.k - t * kNB);
        if (!tiles(trsm[s][t], p0, nf, kTrsmRows)) return fail("TRSM rows do not tile the panel");
        const int Tl = syrk_tile[s] ? syrk_tile[s] : kTile;
        const int64_t nt = (nf - p0 + Tl - 1) / Tl;
        want += nt * (nt + 1) / 2;
      }
      // tensor-core fronts: per group of four panels g0 .. gl, the strips
      // after each t < gl (panels g0 .. t, the 128-row tiles of the next
      // panel's columns) and the pass after gl (panels g0 .. gl, the lower
      // tiles beyond it), each tile exactly once
      if (tc && !tc_tiles[s].empty()) {
        if (syrk_tile[s]) return fail("front on both trailing-update paths");
        std::vector<int64_t> want_tc;
        for (int g0 = 0; g0 < nb; g0 += 4) {
          const int gl = std::min(g0 + 3, nb - 1);
          for (int t = g0; t <= gl; ++t) {
            const int p0 = t * kNB + std::min(kNB, f.k - t * kNB);
            const int nt2 = (nf - p0 + kTcTile - 1) / kTcTile;
            const int64_t head = ((int64_t)g0 << 40) | ((int64_t)(t - g0 + 1) << 36);
            if (t < gl) {
              for (int I = 0; I < nt2; ++I) want_tc.push_back(head | (1ll << 35) | ((int64_t)I << 17));
            } else {
              for (int I = 0; I < nt2; ++I)
                for (int J = 0; J <= I; ++J) want_tc.push_back(head | ((int64_t)I << 17) | J);
            }
          }
        }
        std::vector<int64_t>& v = tc_tiles[s];
        std::sort(v.begin(), v.end());
        std::sort(want_tc.begin(), want_tc.end());
        if (v != want_tc) return fail("tensor-core strips or group passes missing or repeated");
      }
      // every front of the FMA schedule, and the FMA fronts of the
      // tensor-core schedule, take each trailing tile exactly once
      if (!tc || syrk_tile[s]) {
        std::vector<int64_t>& v = syrk_tiles[s];
        std::sort(v.begin(), v.end());
        if (std::adjacent_find(v.begin(), v.end()) != v.end() || (int64_t)v.size() != want)
          return fail("trailing tiles missing or repeated");
      }
    }
  }
  // ---- solve schedules
  std::vector<int> pinv_front(ns, 0);
  if (S.v4) {
    // forward: every front row once, in a row item of its front's level
    // (pivot rows alone, update rows merged by global row); backward: every
    // pivot column once
    std::vector<int64_t> rowoff(ns + 1, 0);
    for (int64_t s = 0; s < ns; ++s) rowoff[s + 1] = rowoff[s] + S.sn[s].k + S.sn[s].m;
    std::vector<char> seen(rowoff[ns], 0);
    int32_t last = -1;
    for (const Launch& L : S.fwsched) {
      if (L.kind != K_V4_FW || L.level < last) return fail("variant-4 forward schedule");
      last = L.level;
      for (int64_t x = L.item_off; x < L.item_off + L.count; ++x) {
        const Item& it = S.items[x];
        if (it.t < 0 || it.t >= it.a || it.a > (int64_t)S.v4_grp.size())
          return fail("variant-4 row without groups");
        if (it.b && it.a - it.t != 1) return fail("variant-4 pivot row with several groups");
        for (int32_t g = it.t; g < it.a; ++g) {
          const Item& gr = S.v4_grp[g];
          const SnInfo& f = S.sn[gr.s];
          if (S.slevel[gr.s] != L.level || gr.t < 0 || gr.t >= f.k + f.m)
            return fail("variant-4 group outside its level or front");
          if ((gr.t < f.k) != (it.b != 0) || S.rowidx[f.rows_off + gr.t] != it.s)
            return fail("variant-4 group on the wrong row");
          if (seen[rowoff[gr.s] + gr.t]++) return fail("variant-4 front row repeated");
        }
      }
    }
    for (char c : seen)
      if (c != 1) return fail("variant-4 front row missing");
    std::vector<int64_t> cols(ns, 0);
    last = S.nlevels;
    for (const Launch& L : S.bwsched) {
      if (L.kind != K_V4_BW || L.level > last) return fail("variant-4 backward schedule");
      last = L.level;
      for (int64_t x = L.item_off; x < L.item_off + L.count; ++x) {
        const Item& it = S.items[x];
        if (S.slevel[it.s] != L.level || it.t != cols[it.s]) return fail("variant-4 column order");
        cols[it.s]++;
      }
    }
    for (int64_t s = 0; s < ns; ++s) {
      if (cols[s] != S.sn[s].k) return fail("variant-4 pivot column missing");
      pinv_front[s] = S.ioff[s] >= 0;  // the blocked inverse, checked below
    }
    // the partitioned inverse of every front: blocked (kept inverses) or
    // one CTA, then its transpose tile by tile
    for (int tc = 0; tc < 2; ++tc) {
      std::vector<int> once(ns, 0);
      std::vector<int64_t> tiles_(ns, 0);
      for (const Launch& L : tc ? S.fsched_tc : S.fsched)
        for (int64_t x = L.item_off; L.kind >= K_PINV_INIT && x < L.item_off + L.count; ++x) {
          const Item& it = S.items[x];
          if (L.kind == K_PINV_SMALL || (L.kind == K_PINV_INIT && it.t == 0)) once[it.s]++;
          if (L.kind == K_PT) tiles_[it.s]++;
        }
      for (int64_t s = 0; s < ns; ++s) {
        const int64_t nf = S.sn[s].k + S.sn[s].m;
        if (once[s] != 1) return fail("variant-4 front without a partitioned inverse");
        if (tiles_[s] != ((nf + kNB - 1) / kNB) * ((S.sn[s].k + kNB - 1) / kNB))
          return fail("variant-4 transpose tiles");
      }
    }
  }
  for (int bw = 0; bw < 2 && !S.v4; ++bw) {
    const std::vector<Launch>& sched = bw ? S.bwsched : S.fwsched;
    std::vector<int> warp(ns, 0);
    std::vector<std::vector<std::pair<int, int>>> piv(ns), upd(ns), pv(ns), pg(ns), gemv(ns);
    int32_t last_level = bw ? S.nlevels : -1;
    for (const Launch& L : sched) {
      if (bw ? L.level > last_level : L.level < last_level) return fail("solve levels out of order");
      last_level = L.level;
      for (int64_t x = L.item_off; x < L.item_off + L.count; ++x) {
        const Item& it = S.items[x];
        const SnInfo& f = S.sn[it.s];
        if (S.slevel[it.s] != L.level) return fail("solve item outside its front's level");
        switch (L.kind) {
          case K_FW_WARP:
          case K_BW_WARP:
            if (f.k + f.m > 32 * L.param) return fail("front too large for its warp class");
            warp[it.s]++;
            break;
          case K_FW_LEVEL:
          case K_BW_LEVEL:
            piv[it.s].push_back({it.a, it.b});
            break;
          case K_FW_GEMV:
            if (it.a < f.k) return fail("forward update block inside the pivots");
            if (L.tile > fw_gemv_tile(f.k)) return fail("forward update product too narrow for its front");
            upd[it.s].push_back({it.a, it.b});
            break;
          case K_BW_GEMV:
            if (L.tile < bw_gemv_split(f.m)) return fail("backward update split below its front's");
            gemv[it.s].push_back({it.a, it.b});
            break;
          case K_FW_PGATHER:
          case K_BW_PCOPY:
            pg[it.s].push_back({it.a, it.b});
            break;
          case K_FW_PINV:
          case K_BW_PINV:
            pinv_front[it.s] = 1;
            if (it.t == 0) pv[it.s].push_back({it.a, it.b});
            else upd[it.s].push_back({it.a, it.b});
            break;
          default:
            return fail("unknown solve kind");
        }
      }
    }
    for (int64_t s = 0; s < ns; ++s) {
      const SnInfo& f = S.sn[s];
      const int nf = f.k + f.m;
      const bool blocks = !piv[s].empty() || !pv[s].empty();
      if (warp[s] + (blocks ? 1 : 0) != 1) return fail("front solved twice or never");
      if (warp[s]) continue;
      if (!pv[s].empty()) {  // partitioned inverse
        if (S.ioff[s] < 0) return fail("partitioned-inverse front without kept inverses");
        if (!tiles(pv[s], 0, f.k, kNB) || !tiles(pg[s], 0, f.k, kNB))
          return fail("partitioned-inverse blocks do not tile the pivots");
        if (!piv[s].empty() || !gemv[s].empty()) return fail("front in two solve variants");
      } else {
        if (!tiles(piv[s], 0, f.k, kNB)) return fail("pivot blocks do not tile the pivots");
        if (bw && f.m > 0 && !tiles(gemv[s], 0, f.k, kNB))
          return fail("backward update blocks do not tile the pivots");
      }
      if (!bw && !tiles(upd[s], f.k, nf, kNB)) return fail("update blocks do not tile the rows");
    }
  }
  // ---- partitioned inverse pass (both factor schedules)
  for (int tc = 0; tc < 2; ++tc) {
    const std::vector<Launch>& sched = tc ? S.fsched_tc : S.fsched;
    std::vector<std::vector<std::pair<int, int>>> init(ns);
    std::vector<std::vector<int64_t>> steps(ns);
    int32_t last_t = -1;
    bool seen_init = false;
    for (const Launch& L : sched) {
      if (L.kind != K_PINV_INIT && L.kind != K_PINV) continue;
      if (L.kind == K_PINV_INIT) seen_init = true;
      else if (!seen_init || L.param <= last_t) return fail("inverse steps out of order");
      if (L.kind == K_PINV) last_t = L.param;
      for (int64_t x = L.item_off; x < L.item_off + L.count; ++x) {
        const Item& it = S.items[x];
        if (!pinv_front[it.s]) return fail("inverse pass on a front the solve does not use it for");
        const int nb = (int)nb_of(it.s), mb = (S.sn[it.s].m + kNB - 1) / kNB;
        if (L.kind == K_PINV_INIT) {
          init[it.s].push_back({it.t, 1});
        } else {
          if (it.t != L.param || it.t >= nb || it.a <= it.t || it.a >= nb + mb || it.b < 0 ||
              it.b > it.t)
            return fail("inverse tile out of range");
          steps[it.s].push_back(((int64_t)it.t << 40) | ((int64_t)it.a << 20) | it.b);
        }
      }
    }
    for (int64_t s = 0; s < ns; ++s) {
      if (!pinv_front[s]) continue;
      const int64_t nb = nb_of(s), mb = (S.sn[s].m + kNB - 1) / kNB;
      if (!tiles(init[s], 0, (int)nb, 1)) return fail("inverse init does not cover the columns");
      int64_t want = 0;
      for (int64_t t = 0; t < nb; ++t) want += (nb + mb - t - 1) * (t + 1);
      std::vector<int64_t>& v = steps[s];
      std::sort(v.begin(), v.end());
      if (std::adjacent_find(v.begin(), v.end()) != v.end() || (int64_t)v.size() != want)
        return fail("inverse tiles missing or repeated");
    }
  }
  return MF_OK;
}

// Row lists of the fundamental supernodes (the exported pattern of L), built
// on first request: column j's lower entries of C plus the children's update
// rows, merged per supernode in increasing order.
int build_upper_assembly(const mf_symbolic& S, UpperAssembly& out, std::string& err) {
  const int64_t n = S.n;
  out.col_ptr.assign(n + 1, 0);
  out.row.clear();
  out.src_ptr.assign(1, 0);
  out.src.clear();
  std::vector<int32_t> posn(n, -1);
  std::vector<std::pair<int32_t, int64_t>> ent;  // (front row, CSR position)
  for (const SnInfo& I : S.sn) {
    const int32_t* frows = S.rowidx.data() + I.rows_off;
    for (int32_t r = 0; r < I.k + I.m; ++r) posn[frows[r]] = r;
    for (int32_t j = I.first; j < I.first + I.k; ++j) {
      ent.clear();
      const int32_t ro = S.perm[j];
      for (int64_t p = S.rowptr[ro]; p < S.rowptr[ro + 1]; ++p) {
        const int32_t i = S.iperm[S.colind[p]];
        if (i <= j) continue;
        const int32_t r = posn[i];
        if (r < 0 || frows[r] != i) {
          err = "an upper entry of A falls outside its front: the pattern is not structurally symmetric";
          return MF_ERR_INVALID;
        }
        ent.emplace_back(r, p);
      }
      std::sort(ent.begin(), ent.end());
      for (size_t e = 0; e < ent.size(); ++e) {
        if (e == 0 || ent[e].first != ent[e - 1].first) {
          out.row.push_back(ent[e].first);
          out.src_ptr.push_back(out.src_ptr.back());
        }
        out.src.push_back(ent[e].second);
        out.src_ptr.back()++;
      }
      out.col_ptr[j + 1] = (int64_t)out.row.size();
    }
  }
  return MF_OK;
}

void ensure_fundamental_rows(const mf_symbolic& Sc) {
  std::lock_guard<std::mutex> lk(Sc.dev_mu);
  if (!Sc.fs_rows_off.empty() || Sc.nsuper == 0) return;
  mf_symbolic& S = const_cast<mf_symbolic&>(Sc);
  const int64_t n = S.n, ns = S.nsuper;
  std::vector<int32_t> schild_cnt(ns + 1, 0), children;
  for (int64_t s = 0; s < ns; ++s)
    if (S.fs_parent[s] >= 0) schild_cnt[S.fs_parent[s] + 1]++;
  for (int64_t s = 0; s < ns; ++s) schild_cnt[s + 1] += schild_cnt[s];
  children.assign(schild_cnt[ns], 0);
  {
    std::vector<int32_t> fillc(schild_cnt.begin(), schild_cnt.end() - 1);
    for (int64_t s = 0; s < ns; ++s)
      if (S.fs_parent[s] >= 0) children[fillc[S.fs_parent[s]]++] = (int32_t)s;
  }
  std::vector<int32_t> mark(n, -1), upd;
  std::vector<int32_t> fs_m(ns, 0);
  S.fs_rows_off.assign(ns + 1, 0);
  S.fs_rowidx.clear();
  int64_t total = 0;
  for (int64_t s = 0; s < ns; ++s) total += S.colcount[S.sup_ptr[s]];
  S.fs_rowidx.reserve(total);
  for (int64_t s = 0; s < ns; ++s) {
    const int32_t f = S.sup_ptr[s], l = S.sup_ptr[s + 1] - 1;
    upd.clear();
    for (int32_t j = f; j <= l; ++j)
      for (int64_t p = S.low_cp[j]; p < S.low_cp[j + 1]; ++p) {
        const int32_t i = S.low_cr[p];
        if (i > l && mark[i] != s) {
          mark[i] = (int32_t)s;
          upd.push_back(i);
        }
      }
    for (int32_t ci = schild_cnt[s]; ci < schild_cnt[s + 1]; ++ci) {
      const int32_t c = children[ci];
      const int32_t* crow = S.fs_rowidx.data() + S.fs_rows_off[c] + (S.sup_ptr[c + 1] - S.sup_ptr[c]);
      for (int32_t t = 0; t < fs_m[c]; ++t) {
        const int32_t r = crow[t];
        if (r > l && mark[r] != s) {
          mark[r] = (int32_t)s;
          upd.push_back(r);
        }
      }
    }
    std::sort(upd.begin(), upd.end());
    fs_m[s] = (int32_t)upd.size();
    S.fs_rows_off[s] = (int64_t)S.fs_rowidx.size();
    for (int32_t j = f; j <= l; ++j) S.fs_rowidx.push_back(j);
    S.fs_rowidx.insert(S.fs_rowidx.end(), upd.begin(), upd.end());
  }
  S.fs_rows_off[ns] = (int64_t)S.fs_rowidx.size();
}

}  // namespace mf
