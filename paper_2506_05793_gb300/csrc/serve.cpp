// serve.cpp -- continuous-batching request loop over resident factors.
//
// The paper's Tacho serves many subdomain solves per GPU (Sec. 5: several
// MPI ranks share an A100 through MPS; one factorization per nonlinear step,
// many solves per factorization).  Here one process serves a stream of
// requests instead:
//   - factor requests (a prepared symbolic object + values + right-hand
//     sides) create a device factor, factor it and solve; the factor stays
//     resident for later solve-only requests until released;
//   - solve-only requests run against a resident factor.
// Worker threads each own a CUDA stream.  A request is admitted in arrival
// order when a worker is free and, for a factor request, its device bytes
// fit in the remaining budget; a request that cannot be admitted yet does
// not block later ones that can (requests on a busy factor wait for it).
// Work of different workers overlaps on the device.  FP32 factors solve with
// FP64 refinement to a backward error of 1e-13 (FP64 fallback on).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstddef>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "mf_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t id = 0;
  bool is_factor = false;
  const mf_symbolic* sym = nullptr;
  const double* values = nullptr;
  int32_t prec = MF_FP64;
  int64_t factor_id = -1;
  int32_t nrhs = 0;
  const double* B = nullptr;
  int64_t ldb = 0;
  double* X = nullptr;
  int64_t ldx = 0;
  int64_t bytes = 0;  // device bytes a factor request reserves
  Clock::time_point submitted;
};

struct Done {
  bool done = false;
  int32_t status = MF_OK;
  double latency_ms = 0.0;
};

struct Resident {
  mf_factor* f = nullptr;
  int64_t bytes = 0;
  bool ready = false;    // factorization finished
  bool busy = false;     // a request is using it
  bool release = false;  // free once idle
  int32_t prec = MF_FP64;
};

}  // namespace

struct mf_server {
  mf_handle* h = nullptr;
  int64_t budget = 0;
  int64_t reserved = 0;  // bytes of resident or in-flight factors
  int64_t peak = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request> queue;
  std::map<int64_t, Done> done;
  std::map<int64_t, Resident> factors;
  std::vector<double> latencies;
  int64_t completed = 0, failed = 0, solves = 0;
  Clock::time_point t_first, t_last;
  bool any = false;
  int64_t next_req = 1, next_factor = 1;
  bool stop = false;
  std::vector<std::thread> workers;

  // first admissible request in arrival order (under mu)
  bool pick(Request& out) {
    for (size_t q = 0; q < queue.size();) {
      Request& r = queue[q];
      if (r.is_factor) {
        if (budget > 0 && reserved + r.bytes > budget) {
          ++q;
          continue;
        }
        reserved += r.bytes;
        peak = std::max(peak, reserved);
        Resident& res = factors[r.factor_id];
        res.busy = true;
        res.bytes = r.bytes;
        res.prec = r.prec;
      } else {
        auto fr = factors.find(r.factor_id);
        if (fr == factors.end()) {
          const int64_t fid = r.factor_id;
          const bool pending = std::any_of(queue.begin(), queue.end(), [&](const Request& x) {
            return x.is_factor && x.factor_id == fid;
          });
          if (pending) {
            ++q;
            continue;
          }
          // its factorization failed or it was released: fail it now
          Done& d = done[r.id];
          d.done = true;
          d.status = MF_ERR_INVALID;
          ++failed;
          queue.erase(queue.begin() + (std::ptrdiff_t)q);
          cv.notify_all();
          continue;
        }
        if (!fr->second.ready || fr->second.busy) {
          ++q;
          continue;
        }
        fr->second.busy = true;
      }
      out = r;
      queue.erase(queue.begin() + (std::ptrdiff_t)q);
      return true;
    }
    return false;
  }

  void run(int device) {
    cudaSetDevice(device);
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return;
    for (;;) {
      Request rq;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] { return (stop && queue.empty()) || pick(rq); });
        if (stop && rq.id == 0) break;
      }
      int rc = MF_OK;
      mf_factor* f = nullptr;
      if (rq.is_factor) {
        rc = mf_factor_create(h, rq.sym, rq.prec, &f);
        if (rc == MF_OK) rc = mf_factor_numeric(f, rq.values, 0, st, 0);
      } else {
        std::lock_guard<std::mutex> lk(mu);
        f = factors[rq.factor_id].f;
      }
      if (rc == MF_OK && rq.nrhs > 0) {
        const int32_t prec = rq.is_factor ? rq.prec : factors_prec(rq.factor_id);
        if (prec == MF_FP32)
          rc = mf_solve_refined(f, rq.nrhs, rq.B, rq.ldb, rq.X, rq.ldx, 0, 1e-13, 30, 1, nullptr, st);
        else
          rc = mf_solve(f, rq.nrhs, rq.B, rq.ldb, rq.X, rq.ldx, 0, st);
      }
      const Clock::time_point t = Clock::now();
      std::vector<mf_factor*> to_free;
      {
        std::lock_guard<std::mutex> lk(mu);
        Resident& r = factors[rq.factor_id];
        if (rq.is_factor) {
          if (rc == MF_OK) {
            r.f = f;
            r.ready = true;
          } else {
            to_free.push_back(f);
            reserved -= rq.bytes;
            factors.erase(rq.factor_id);
          }
        }
        auto fr = factors.find(rq.factor_id);
        if (fr != factors.end()) {
          fr->second.busy = false;
          if (fr->second.release && !queued_for(rq.factor_id)) {
            to_free.push_back(fr->second.f);
            reserved -= fr->second.bytes;
            factors.erase(fr);
          }
        }
        Done& d = done[rq.id];
        d.done = true;
        d.status = rc;
        d.latency_ms = std::chrono::duration<double, std::milli>(t - rq.submitted).count();
        if (rc == MF_OK) {
          ++completed;
          solves += rq.nrhs > 0 ? 1 : 0;
          latencies.push_back(d.latency_ms);
          if (!any || rq.submitted < t_first) t_first = rq.submitted;
          if (!any || t > t_last) t_last = t;
          any = true;
        } else {
          ++failed;
        }
      }
      for (mf_factor* x : to_free) mf_factor_free(x);
      cv.notify_all();
    }
    cudaStreamDestroy(st);
  }

  // a queued request still needs this factor (under mu)
  bool queued_for(int64_t id) const {
    return std::any_of(queue.begin(), queue.end(),
                       [&](const Request& q) { return q.factor_id == id; });
  }

  int32_t factors_prec(int64_t id) {
    std::lock_guard<std::mutex> lk(mu);
    return factors[id].prec;
  }
};

namespace {
int64_t factor_bytes_of(const mf_symbolic* s, int32_t prec) {
  mf_symbolic_info info;
  mf_symbolic_get_info(s, &info);
  return prec == MF_FP32 ? info.factor_bytes_fp32 : info.factor_bytes_fp64;
}
}  // namespace

extern "C" {

int mf_server_create(mf_handle* h, int32_t workers, int64_t budget_bytes, mf_server** sv) {
  if (!h || !sv || workers < 1 || workers > 64 || budget_bytes < 0)
    return mf::set_error(MF_ERR_INVALID, "invalid server arguments");
  *sv = nullptr;
  mf_server* S = new (std::nothrow) mf_server();
  if (!S) return mf::set_error(MF_ERR_OOM, "host allocation failed");
  S->h = h;
  S->budget = budget_bytes;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) {
    delete S;
    return mf::set_error(MF_ERR_CUDA, "no CUDA device");
  }
  try {
    for (int i = 0; i < workers; ++i) S->workers.emplace_back([S, device] { S->run(device); });
  } catch (...) {
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->stop = true;
    }
    S->cv.notify_all();
    for (auto& t : S->workers) t.join();
    delete S;
    return mf::set_error(MF_ERR_INTERNAL, "could not start worker threads");
  }
  *sv = S;
  return MF_OK;
}

int mf_server_submit_factor(mf_server* sv, const mf_symbolic* s, const double* values, int32_t prec,
                            int32_t nrhs, const double* B, int64_t ldb, double* X, int64_t ldx,
                            int64_t* req, int64_t* factor_id) {
  if (!sv || !s || !values || !req || !factor_id || nrhs < 0 || (prec != MF_FP64 && prec != MF_FP32))
    return mf::set_error(MF_ERR_INVALID, "invalid factor request");
  mf_symbolic_info info;
  mf_symbolic_get_info(s, &info);
  if (nrhs > 0 && (!B || !X || ldb < info.n || ldx < info.n))
    return mf::set_error(MF_ERR_INVALID, "invalid right-hand sides");
  const int64_t bytes = factor_bytes_of(s, prec);
  if (sv->budget > 0 && bytes > sv->budget)
    return mf::set_error(MF_ERR_OOM, "factor larger than the server budget");
  Request r;
  r.is_factor = true;
  r.sym = s;
  r.values = values;
  r.prec = prec;
  r.nrhs = nrhs;
  r.B = B;
  r.ldb = ldb;
  r.X = X;
  r.ldx = ldx;
  r.bytes = bytes;
  r.submitted = Clock::now();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop) return mf::set_error(MF_ERR_INVALID, "server is shutting down");
    r.id = sv->next_req++;
    r.factor_id = sv->next_factor++;
    sv->done[r.id] = Done{};
    sv->queue.push_back(r);
  }
  sv->cv.notify_all();
  *req = r.id;
  *factor_id = r.factor_id;
  return MF_OK;
}

int mf_server_submit_solve(mf_server* sv, int64_t factor_id, int32_t nrhs, const double* B,
                           int64_t ldb, double* X, int64_t ldx, int64_t* req) {
  if (!sv || !req || nrhs < 1 || !B || !X) return mf::set_error(MF_ERR_INVALID, "invalid solve request");
  Request r;
  r.factor_id = factor_id;
  r.nrhs = nrhs;
  r.B = B;
  r.ldb = ldb;
  r.X = X;
  r.ldx = ldx;
  r.submitted = Clock::now();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop) return mf::set_error(MF_ERR_INVALID, "server is shutting down");
    auto fr = sv->factors.find(factor_id);
    const bool pending = std::any_of(sv->queue.begin(), sv->queue.end(), [&](const Request& q) {
      return q.is_factor && q.factor_id == factor_id;
    });
    if ((fr == sv->factors.end() && !pending) || (fr != sv->factors.end() && fr->second.release))
      return mf::set_error(MF_ERR_INVALID, "unknown or released factor");
    r.id = sv->next_req++;
    sv->done[r.id] = Done{};
    sv->queue.push_back(r);
  }
  sv->cv.notify_all();
  *req = r.id;
  return MF_OK;
}

int mf_server_poll(mf_server* sv, int64_t req, int32_t* is_done, int32_t* status, double* latency_ms) {
  if (!sv) return mf::set_error(MF_ERR_INVALID, "NULL server");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->done.find(req);
  if (it == sv->done.end()) return mf::set_error(MF_ERR_INVALID, "unknown request");
  if (is_done) *is_done = it->second.done ? 1 : 0;
  if (status) *status = it->second.status;
  if (latency_ms) *latency_ms = it->second.latency_ms;
  return MF_OK;
}

int mf_server_wait(mf_server* sv, int64_t req, int32_t* status, double* latency_ms) {
  if (!sv) return mf::set_error(MF_ERR_INVALID, "NULL server");
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->done.find(req);
  if (it == sv->done.end()) return mf::set_error(MF_ERR_INVALID, "unknown request");
  sv->cv.wait(lk, [&] { return sv->done[req].done; });
  const Done d = sv->done[req];
  if (status) *status = d.status;
  if (latency_ms) *latency_ms = d.latency_ms;
  return MF_OK;
}

int mf_server_release_factor(mf_server* sv, int64_t factor_id) {
  if (!sv) return mf::set_error(MF_ERR_INVALID, "NULL server");
  mf_factor* f = nullptr;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    auto fr = sv->factors.find(factor_id);
    if (fr == sv->factors.end()) return mf::set_error(MF_ERR_INVALID, "unknown factor");
    if (fr->second.busy || !fr->second.ready || sv->queued_for(factor_id)) {
      fr->second.release = true;  // freed after its last queued request
      return MF_OK;
    }
    f = fr->second.f;
    sv->reserved -= fr->second.bytes;
    sv->factors.erase(fr);
  }
  mf_factor_free(f);
  sv->cv.notify_all();
  return MF_OK;
}

int mf_server_get_stats(mf_server* sv, mf_server_stats* out) {
  if (!sv || !out) return mf::set_error(MF_ERR_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  std::memset(out, 0, sizeof(*out));
  out->completed = sv->completed;
  out->failed = sv->failed;
  out->resident_bytes = sv->reserved;
  out->peak_resident_bytes = sv->peak;
  std::vector<double> l = sv->latencies;
  if (!l.empty()) {
    std::sort(l.begin(), l.end());
    auto pct = [&](double p) {
      const double x = p * (double)(l.size() - 1);
      const size_t i = (size_t)x;
      const double w = x - (double)i;
      return i + 1 < l.size() ? l[i] * (1.0 - w) + l[i + 1] * w : l[i];
    };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    double s = 0.0;
    for (double v : l) s += v;
    out->mean_ms = s / (double)l.size();
    const double span = std::chrono::duration<double>(sv->t_last - sv->t_first).count();
    out->solves_per_s = span > 0 ? (double)sv->solves / span : 0.0;
  }
  return MF_OK;
}

int mf_server_free(mf_server* sv) {
  if (!sv) return MF_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv.notify_all();
  for (auto& t : sv->workers) t.join();
  for (auto& kv : sv->factors)
    if (kv.second.f) mf_factor_free(kv.second.f);
  delete sv;
  return MF_OK;
}

}  // extern "C"
