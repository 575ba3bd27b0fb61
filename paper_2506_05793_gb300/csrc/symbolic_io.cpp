// symbolic_io.cpp -- save and load a symbolic analysis (restart without
// repeating the host analysis).  The paper has no counterpart; the analysis
// depends on the pattern only (Sec. 3, phase 1), so a program that factors
// the same pattern again after a restart can load it instead.
//
// Format: a fixed header (magic, version, byte-order mark, sizes of the
// record types), then every member of mf_symbolic in declaration order:
// scalars as raw bytes, vectors as a 64-bit count followed by the elements,
// then a 64-bit FNV-1a hash of those member bytes.  The hash rejects an
// accidentally damaged file whose sizes still look consistent (its offsets
// reach device code).  Native byte order: a file is read back on the same
// kind of machine.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "mf_internal.h"

namespace {

constexpr char kMagic[8] = {'M', 'F', 'S', 'Y', 'M', 'B', 'O', 'L'};
constexpr uint32_t kVersion = 5;
constexpr uint64_t kFnvOffset = 1469598103934665603ull;
constexpr uint64_t kFnvPrime = 1099511628211ull;

// FNV-1a, 64 bit, over a byte range, continuing from h.
uint64_t fnv1a(uint64_t h, const void* p, size_t n) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * kFnvPrime;
  return h;
}
constexpr uint32_t kByteOrder = 0x01020304u;

struct Header {
  char magic[8];
  uint32_t version;
  uint32_t byte_order;
  uint32_t size_sninfo, size_item, size_launch, size_pointer;
};

Header make_header() {
  Header h;
  std::memcpy(h.magic, kMagic, sizeof(kMagic));
  h.version = kVersion;
  h.byte_order = kByteOrder;
  h.size_sninfo = sizeof(mf::SnInfo);
  h.size_item = sizeof(mf::Item);
  h.size_launch = sizeof(mf::Launch);
  h.size_pointer = sizeof(void*);
  return h;
}

struct Writer {
  FILE* f;
  bool ok = true;
  uint64_t hash = kFnvOffset;  // of the member bytes
  void raw(const void* p, size_t n) {
    if (ok && n && std::fwrite(p, 1, n, f) != n) ok = false;
    hash = fnv1a(hash, p, n);
  }
  template <typename T>
  void operator()(const T& v) {
    static_assert(std::is_trivially_copyable<T>::value, "raw scalar");
    raw(&v, sizeof(T));
  }
  template <typename T>
  void operator()(const std::vector<T>& v) {
    static_assert(std::is_trivially_copyable<T>::value, "raw elements");
    const uint64_t n = v.size();
    raw(&n, sizeof(n));
    raw(v.data(), n * sizeof(T));
  }
};

struct Reader {
  FILE* f;
  uint64_t left;  // bytes not yet read
  bool ok = true;
  uint64_t hash = kFnvOffset;  // of the member bytes
  void raw(void* p, size_t n) {
    if (!ok) return;
    if (n > left || (n && std::fread(p, 1, n, f) != n)) {
      ok = false;
      return;
    }
    left -= n;
    hash = fnv1a(hash, p, n);
  }
  template <typename T>
  void operator()(T& v) {
    static_assert(std::is_trivially_copyable<T>::value, "raw scalar");
    raw(&v, sizeof(T));
  }
  template <typename T>
  void operator()(std::vector<T>& v) {
    static_assert(std::is_trivially_copyable<T>::value, "raw elements");
    uint64_t n = 0;
    raw(&n, sizeof(n));
    // a count the rest of the file cannot hold is corruption, not a reason
    // to allocate
    if (!ok || n > left / sizeof(T)) {
      ok = false;
      return;
    }
    v.resize(n);
    raw(v.data(), n * sizeof(T));
  }
};

// Every member of the analysis, in one place for both directions.
template <class IO, class S>
void members(IO& io, S& s) {
  io(s.n);
  io(s.nnzA);
  io(s.rowptr);
  io(s.colind);
  io(s.perm);
  io(s.iperm);
  io(s.parent);
  io(s.colcount);
  io(s.sup_ptr);
  io(s.col2sn);
  io(s.fs_rowidx);
  io(s.fs_rows_off);
  io(s.low_cp);
  io(s.low_cr);
  io(s.fs_parent);
  io(s.relax);
  io(s.front_ptr);
  io(s.col2front);
  io(s.front_flops);
  io(s.nsuper);
  io(s.nnzL);
  io(s.nnz_lower);
  io(s.flops);
  io(s.nlevels);
  io(s.max_front);
  io(s.max_k);
  io(s.sn);
  io(s.children);
  io(s.rowidx);
  io(s.relmap);
  io(s.slevel);
  io(s.acol_ptr);
  io(s.arow);
  io(s.asrc_ptr);
  io(s.asrc);
  io(s.Lsize);
  io(s.Usize);
  io(s.Wsize);
  io(s.items);
  io(s.fsched);
  io(s.fsched_tc);
  io(s.soff);
  io(s.split_rows);
  io(s.split_rows_b);
  io(s.max_large);
  io(s.keep_inv);
  io(s.ioff);
  io(s.ninv);
  io(s.pinv);
  io(s.pinv_flops);
  io(s.arange);
  io(s.fwsched);
  io(s.bwsched);
  io(s.blkoff);
  io(s.ginv_ptr);
  io(s.ginv_src);
  io(s.v4);
  io(s.v4_grp);
  io(s.opt_used.small_front_max);
  io(s.opt_used.use_graphs);
  io(s.opt_used.profile);
  io(s.opt_used.relax);
  io(s.opt_used.budget_bytes);
  io(s.opt_used.tc);
  io(s.opt_used.sptrsv);
  io(s.opt_used.small_queue);
  for (int b = 0; b < 4; ++b) io(s.opt_used.update_tile[b]);
}

// Sizes that the rest of the library relies on without checking again.
bool consistent(const mf_symbolic& s) {
  const size_t n = (size_t)s.n;
  if (s.n < 0 || s.rowptr.size() != n + 1 || s.perm.size() != n || s.iperm.size() != n ||
      s.parent.size() != n || s.colcount.size() != n || s.col2front.size() != n)
    return false;
  if ((int64_t)s.colind.size() != s.nnzA || (n && s.rowptr[n] != s.nnzA)) return false;
  if (s.sup_ptr.size() != (size_t)(n ? s.nsuper + 1 : (s.sup_ptr.empty() ? 0 : 1))) return false;
  const size_t nf = s.sn.size();
  if (s.slevel.size() != nf || s.soff.size() != nf || s.ioff.size() != nf ||
      s.blkoff.size() != nf + 1 || s.front_ptr.size() != nf + 1)
    return false;
  if (s.ginv_ptr.size() != (size_t)s.Wsize + 1) return false;
  if (s.acol_ptr.size() != n + 1 || (int64_t)s.arow.size() != s.nnz_lower) return false;
  for (const auto* sched : {&s.fsched, &s.fsched_tc, &s.fwsched, &s.bwsched})
    for (const mf::Launch& L : *sched)
      if (L.item_off < 0 || L.count < 0 || (size_t)(L.item_off + L.count) > s.items.size())
        return false;
  // the backward update-row product launches P = tile CTAs per item
  for (const mf::Launch& L : s.bwsched)
    if (L.kind == mf::K_BW_GEMV && L.tile != 1 && L.tile != 2 && L.tile != 4 && L.tile != 8)
      return false;
  for (const mf::Item& it : s.items)
    if (it.s < -1 || it.s >= (int64_t)nf) return false;
  return true;
}

// Every index that a device kernel dereferences lies inside the array it
// indexes.  The hash only catches accidental damage; this check keeps a
// file made to carry a matching hash from reaching device code with an
// out-of-range index.  Runs after consistent().
bool indices_in_range(const mf_symbolic& s) {
  const int64_t n = s.n, nfr = (int64_t)s.sn.size();
  auto mono = [](const auto& v, int64_t first, int64_t last) {
    if (v.empty() || (int64_t)v.front() != first || (int64_t)v.back() != last) return false;
    for (size_t i = 1; i < v.size(); ++i)
      if (v[i] < v[i - 1]) return false;
    return true;
  };
  std::vector<char> seen(n, 0);
  for (int64_t i = 0; i < n; ++i) {
    const int32_t o = s.perm[i];
    if (o < 0 || o >= n || seen[o] || s.iperm[o] != i) return false;
    seen[o] = 1;
  }
  if (!mono(s.rowptr, 0, s.nnzA)) return false;
  for (int32_t c : s.colind)
    if (c < 0 || c >= n) return false;
  if (!mono(s.front_ptr, 0, n)) return false;
  for (int64_t j = 0; j < n; ++j) {
    const int32_t F = s.col2front[j];
    if (F < 0 || F >= nfr || j < s.front_ptr[F] || j >= s.front_ptr[F + 1]) return false;
  }
  for (int64_t F = 0; F < nfr; ++F) {
    const mf::SnInfo& I = s.sn[F];
    const int64_t nf = (int64_t)I.k + I.m;
    if (I.first != s.front_ptr[F] || I.k != s.front_ptr[F + 1] - s.front_ptr[F] || I.k < 1 ||
        I.m < 0 || I.first + (int64_t)I.k > n)
      return false;
    if (I.parent < -1 || I.parent >= nfr || (I.parent < 0 && I.m != 0)) return false;
    if (I.Loff < 0 || I.Loff + nf * I.k > s.Lsize) return false;
    if (I.m > 0 && (I.Uoff < 0 || I.Uoff + (int64_t)I.m * I.m > s.Usize)) return false;
    if (I.rows_off < 0 || I.rows_off + nf > (int64_t)s.rowidx.size()) return false;
    if (I.woff < 0 || I.woff + nf > s.Wsize) return false;
    if (I.nchild < 0 || I.child_begin < 0 ||
        (int64_t)I.child_begin + I.nchild > (int64_t)s.children.size())
      return false;
    for (int32_t c = 0; c < I.nchild; ++c) {
      const int32_t ch = s.children[I.child_begin + c];
      if (ch < 0 || ch >= nfr || s.sn[ch].parent != F) return false;
    }
    if (I.parent >= 0) {
      const mf::SnInfo& P = s.sn[I.parent];
      if (I.map_off < 0 || I.map_off + I.m > (int64_t)s.relmap.size()) return false;
      for (int32_t i = 0; i < I.m; ++i) {
        const int32_t r = s.relmap[I.map_off + i];
        if (r < 0 || r >= P.k + P.m) return false;
      }
    }
    const int64_t nb = (I.k + mf::kNB - 1) / mf::kNB;
    if (s.ioff[F] != -1 && (s.ioff[F] < 0 || s.ioff[F] + nb > s.ninv)) return false;
    if (s.soff[F] < 0 || (s.soff[F] >> mf::kSoffAreaShift) > 1) return false;
  }
  // panel items of the large fronts: panel index, rows, inverse slot, tile
  // indices and the staging rows (soff) the panel kernels touch
  const int64_t slots = s.keep_inv ? s.ninv : s.max_large;
  for (const auto* sched : {&s.fsched, &s.fsched_tc})
    for (const mf::Launch& L : *sched)
      for (int64_t x = L.item_off; x < L.item_off + L.count; ++x) {
        const mf::Item& it = s.items[x];
        const mf::SnInfo& I = s.sn[it.s];
        const int64_t nf = (int64_t)I.k + I.m, nb = (I.k + mf::kNB - 1) / mf::kNB;
        // tensor-core items pack (first panel, panels, strip) into t
        const int32_t tt = L.kind == mf::K_SYRK_TC ? (it.t & 0xffff) : it.t;
        const int32_t nK = L.kind == mf::K_SYRK_TC ? ((it.t >> 16) & 0xff) : 1;
        switch (L.kind) {
          case mf::K_POTRF:
          case mf::K_TRSM:
          case mf::K_SYRK_TC: {
            if (tt < 0 || tt >= nb || nK < 1 || nK > 4 || tt + nK > nb) return false;
            if (L.kind != mf::K_SYRK_TC && (it.b < 0 || it.b >= slots)) return false;
            if (L.kind == mf::K_TRSM && (it.a < 0 || it.a >= nf)) return false;
            if (L.kind == mf::K_SYRK_TC && ((it.t >> 24) > 1 || it.a < 0 || it.b < 0 || it.b > it.a))
              return false;
            const int64_t so = s.soff[it.s];
            const int64_t srow = so & (((int64_t)1 << mf::kSoffAreaShift) - 1);
            if (srow + nf > ((so >> mf::kSoffAreaShift) ? s.split_rows_b : s.split_rows))
              return false;
            break;
          }
          case mf::K_PINV_SMALL:
            if (nf > mf::kSmallMax || s.ioff[it.s] >= 0) return false;
            break;
          case mf::K_PT:
            if (it.a < 0 || it.a >= nf || it.b < 0 || it.b >= I.k) return false;
            break;
          case mf::K_PINV_INIT:
          case mf::K_PINV:
            if (it.t < 0 || it.t >= nb || it.a < 0 || it.b < 0 || it.b >= nb ||
                it.a >= nb + (I.m + mf::kNB - 1) / mf::kNB || s.ioff[it.s] < 0)
              return false;
            break;
          default:
            break;
        }
      }
  for (int32_t r : s.rowidx)
    if (r < 0 || r >= n) return false;
  if (!mono(s.blkoff, 0, s.blkoff.empty() ? 0 : (int64_t)s.blkoff.back())) return false;
  if (!mono(s.acol_ptr, 0, s.nnz_lower)) return false;
  for (int64_t j = 0; j < n; ++j) {
    const mf::SnInfo& I = s.sn[s.col2front[j]];
    for (int64_t e = s.acol_ptr[j]; e < s.acol_ptr[j + 1]; ++e)
      if (s.arow[e] < 0 || s.arow[e] >= I.k + I.m) return false;
  }
  if (s.asrc_ptr.size() != (size_t)s.nnz_lower + 1 ||
      !mono(s.asrc_ptr, 0, (int64_t)s.asrc.size()))
    return false;
  for (int64_t x : s.asrc)
    if (x < 0 || x >= s.nnzA) return false;
  if (!mono(s.ginv_ptr, 0, (int64_t)s.ginv_src.size())) return false;
  for (int64_t x : s.ginv_src)
    if (x < 0 || x >= s.Wsize) return false;
  for (const mf::Item& r : s.arange) {
    if (r.s < -1 || r.s >= nfr) return false;
    if (r.s >= 0 && (r.t < 0 || r.t > r.a || r.a > s.sn[r.s].m)) return false;
    // a chunk of kAsmCols parent columns receives at most that many columns
    // of a child (the assembly kernel reads one per lane)
    if (r.s >= 0 && r.a - r.t > mf::kAsmCols) return false;
  }
  // variant 4: forward groups name a front row; forward items a global row
  // and a range of groups; backward items a pivot column
  for (const mf::Item& g : s.v4_grp)
    if (g.s < 0 || g.s >= nfr || g.t < 0 || g.t >= s.sn[g.s].k + s.sn[g.s].m) return false;
  for (const mf::Launch& L : s.fwsched)
    if (L.kind == mf::K_V4_FW)
      for (int64_t x = L.item_off; x < L.item_off + L.count; ++x) {
        const mf::Item& it = s.items[x];
        if (it.s < 0 || it.s >= n || it.t < 0 || it.t > it.a || it.a > (int64_t)s.v4_grp.size())
          return false;
      }
  for (const mf::Launch& L : s.bwsched)
    if (L.kind == mf::K_V4_BW)
      for (int64_t x = L.item_off; x < L.item_off + L.count; ++x) {
        const mf::Item& it = s.items[x];
        if (it.t < 0 || it.t >= s.sn[it.s].k) return false;
      }
  for (const auto* sched : {&s.fsched, &s.fsched_tc})
    for (const mf::Launch& L : *sched)
      if (L.kind == mf::K_ASSEMBLE)
        for (int64_t x = L.item_off; x < L.item_off + L.count; ++x) {
          const mf::Item& it = s.items[x];
          // the chunk's child ranges start at arange[t] and end at a sentinel
          if (it.t < 0 || it.t >= (int64_t)s.arange.size()) return false;
          int64_t q = it.t;
          while (q < (int64_t)s.arange.size() && s.arange[q].s >= 0) ++q;
          if (q == (int64_t)s.arange.size()) return false;
          const mf::SnInfo& I = s.sn[it.s];
          if (it.a < 0 || it.a > it.b || it.b > I.k + I.m || it.b - it.a > mf::kAsmCols) return false;
        }
  return true;
}

}  // namespace

extern "C" {

int mf_symbolic_save(const mf_symbolic* s, const char* path) {
  if (!s || !path) return mf::set_error(MF_ERR_INVALID, "NULL argument");
  FILE* f = std::fopen(path, "wb");
  if (!f) return mf::set_error(MF_ERR_INVALID, std::string("cannot open for writing: ") + path);
  const Header h = make_header();
  bool ok = std::fwrite(&h, 1, sizeof(h), f) == sizeof(h);
  Writer w{f};
  w.ok = ok;
  members(w, *s);
  const uint64_t hash = w.hash;
  w.raw(&hash, sizeof(hash));
  const bool closed = std::fclose(f) == 0;
  if (!w.ok || !closed) return mf::set_error(MF_ERR_INVALID, std::string("write failed: ") + path);
  return MF_OK;
}

int mf_symbolic_load(mf_handle* h, const char* path, mf_symbolic** s) {
  if (!h || !path || !s) return mf::set_error(MF_ERR_INVALID, "NULL argument");
  *s = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) return mf::set_error(MF_ERR_INVALID, std::string("cannot open: ") + path);
  std::fseek(f, 0, SEEK_END);
  const long size = std::ftell(f);
  std::fseek(f, 0, SEEK_SET);
  Header hd;
  const Header want = make_header();
  const bool head_ok = size >= (long)sizeof(hd) && std::fread(&hd, 1, sizeof(hd), f) == sizeof(hd);
  Reader r{f, head_ok ? (uint64_t)size - sizeof(hd) : 0};
  if (!head_ok || std::memcmp(&hd, &want, sizeof(hd)) != 0) {
    std::fclose(f);
    return mf::set_error(MF_ERR_INVALID, "not a symbolic analysis of this library version/machine");
  }
  mf_symbolic* S = new (std::nothrow) mf_symbolic();
  if (!S) {
    std::fclose(f);
    return mf::set_error(MF_ERR_OOM, "host allocation failed");
  }
  try {
    members(r, *S);
  } catch (const std::bad_alloc&) {
    r.ok = false;
  }
  const uint64_t hash = r.hash;
  uint64_t stored = 0;
  r.raw(&stored, sizeof(stored));
  if (stored != hash) r.ok = false;
  std::fclose(f);
  if (!r.ok || r.left != 0 || !consistent(*S)) {
    delete S;
    return mf::set_error(MF_ERR_INVALID, std::string("truncated or corrupt file: ") + path);
  }
  std::string why;
  bool ranged = false;
  try {
    ranged = indices_in_range(*S) && mf::check_schedules(*S, why) == MF_OK;
  } catch (const std::bad_alloc&) {
    delete S;
    return mf::set_error(MF_ERR_OOM, "host allocation failed");
  }
  if (!ranged) {
    delete S;
    return mf::set_error(MF_ERR_INVALID,
                         std::string("analysis with an index out of range or an invalid "
                                     "schedule: ") + path + (why.empty() ? "" : " (" + why + ")"));
  }
  *s = S;
  return MF_OK;
}

}  // extern "C"
