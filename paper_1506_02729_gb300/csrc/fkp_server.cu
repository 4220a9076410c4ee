// fkp_server.cu - continuous-batching request server over the C ABI.
//
// The method's stated use is covariance estimation from many realisations of
// a survey (~10^4 mocks, Sec. III.C); requests of different sizes and grids
// arrive while others are running.  The server keeps `nslots` worker threads,
// each with its own CUDA stream, and a pool of plans (device workspaces)
// shared by the slots: a request checks out an idle plan of its geometry, or
// a new one is made, and returns it when done, so the fields and buffers stay
// on the device across requests and no allocation (which would synchronize
// the device) happens in steady state.  A request is admitted when its
// estimated device footprint fits next to the pooled plans and the running
// requests; idle plans of other geometries are evicted, least recently used
// first, when that makes room.  The queue is first-in first-out with
// skip-ahead (a smaller request behind a large one starts when it fits).
// Requests on different slots run concurrently on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "fkp_internal.h"

namespace fkp {
namespace {

using Clock = std::chrono::steady_clock;

struct PooledPlan {
  void* plan = nullptr;
  fkp_request_t key{};
  size_t bytes = 0;
  bool busy = false;
  uint64_t last = 0;
};

struct Job {
  uint64_t ticket = 0;
  fkp_request_t req{};
  size_t plan_est = 0, cat_bytes = 0;  // footprint: a new plan (if none is idle) + the call's catalog buffers
  PooledPlan* pp = nullptr;            // plan checked out for this job (null: create one)
  size_t reserved = 0;                 // bytes reserved at admission
  int status = 1;                      // 1 pending, else the call's return code
  std::string msg;                     // the worker's error message when status != 0
  bool done = false;
  Clock::time_point t_submit, t_start, t_end;
};

bool same_key(const fkp_request_t& a, const fkp_request_t& b) {
  return std::memcmp(&a.geom, &b.geom, sizeof(a.geom)) == 0 && std::memcmp(&a.pbins, &b.pbins, sizeof(a.pbins)) == 0 &&
         a.want == b.want &&
         (!(a.want & (FKP_B0 | FKP_B2 | FKP_B4)) || std::memcmp(&a.bshells, &b.bshells, sizeof(a.bshells)) == 0);
}

// Device bytes of a plan for a request (workspace; the same terms as plan
// creation) and of the per-call catalog buffers (tile-sorted copy, and a
// staging copy for host catalogs).
size_t estimate_plan(const fkp_request_t& r) {
  const int N = r.geom.N;
  const size_t N3 = (size_t)N * N * N;
  const bool B = (r.want & (FKP_B0 | FKP_B2 | FKP_B4)) != 0;
  int lmax = 0;
  if (r.want & (FKP_P2 | FKP_P4B | FKP_B2 | FKP_B4B)) lmax = 2;
  if (r.want & (FKP_P4 | FKP_B4 | FKP_P6B | FKP_P8B)) lmax = 4;
  const int nf = lmax >= 4 ? 16 : (lmax >= 2 ? 6 : 1), ng = lmax >= 4 ? 9 : (lmax >= 2 ? 4 : 1);
  const size_t half = field_elems(N) * sizeof(float2);
  // one grid (F, and F^w with B), or one per moment field with each object's x^
  const size_t ngrid = (r.want & FKP_XHAT_OBJECT) ? (size_t)nf : (B ? 2 : 1);
  size_t b = N3 * 8 * ngrid + half * (nf + ng);
  b += sizeof(double) * (BQ_N + 1) * (size_t)r.pbins.nbins * tiles_x(N) * N;
  // per-block tile counts of the gridding: two rows per SM (256 bounds the SM count)
  const size_t nt = (size_t)assign_tiles_per_axis(N);
  b += nt * nt * nt * sizeof(int) * 2 * 256;
  if (B) {
    const int S = r.bshells.nshells;
    const int nl = (r.want & FKP_B4) ? 3 : ((r.want & FKP_B2) ? 2 : 1);
    const double hmax = r.bshells.first + (S - 1.0) * r.bshells.step + 0.5 * r.bshells.width;
    const size_t mm = (size_t)hmax, w2 = 2 * mm + 1, m1 = mm + 1;
    b += 3 * w2 * w2 * m1 * 8 + (size_t)S * N * w2 * m1 * 8 + (size_t)S * N * N * m1 * 8 + (size_t)nl * S * N3 * 4;
    const size_t slices = (N3 + 65535) / 65536, pairs = (size_t)S * (S + 1) / 2;
    b += slices * ((pairs + 255) / 256) * 128 * 256 * 4 + slices * 16384 * 8;
  }
  return b + b / 10 + (64 << 20);
}

size_t estimate_catalog(const fkp_request_t& r) {
  const size_t nobj = (size_t)std::max<int64_t>(0, r.gal.n) + (size_t)std::max<int64_t>(0, r.ran.n);
  return nobj * 20 * 9 / 8 + (r.gal.on_device ? 0 : 20 * (size_t)r.gal.n) +
         (r.ran.on_device ? 0 : 20 * (size_t)r.ran.n);
}

struct Server;

struct Worker {
  Server* srv = nullptr;
  int id = 0;
  cudaStream_t stream = nullptr;
  std::thread th;
};

struct Server {
  void* ctx = nullptr;
  int device = 0;
  size_t budget = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Job*> queue;
  std::map<uint64_t, std::unique_ptr<Job>> jobs;
  std::vector<std::unique_ptr<Worker>> workers;
  std::vector<std::unique_ptr<PooledPlan>> pool;  // every plan, idle or checked out
  uint64_t next_ticket = 1, tick = 0;
  size_t pool_bytes = 0, running_bytes = 0, peak = 0;
  int running = 0, peak_running = 0;
  int64_t submitted = 0, completed = 0, failed = 0, rejected = 0;
  bool stop = false;

  size_t in_use() const { return pool_bytes + running_bytes; }

  // Admits the first queued job that fits, evicting idle plans of other keys
  // (least recently used first) when that makes room.  Evicted plans are
  // handed back in `evict` and destroyed by the caller outside the lock.
  Job* pick(std::vector<std::unique_ptr<PooledPlan>>& evict) {
    for (auto it = queue.begin(); it != queue.end(); ++it) {
      Job* j = *it;
      PooledPlan* idle = nullptr;
      for (auto& p : pool)
        if (!p->busy && same_key(p->key, j->req)) { idle = p.get(); break; }
      const size_t need = j->cat_bytes + (idle ? 0 : j->plan_est);
      if (in_use() + need > budget && running > 0) {
        // how much could evicting idle plans of other keys free?
        size_t freeable = 0;
        for (auto& p : pool)
          if (!p->busy && p.get() != idle) freeable += p->bytes;
        if (in_use() + need - std::min(freeable, in_use()) > budget) continue;
      }
      while (in_use() + need > budget) {
        int victim = -1;
        for (int i = 0; i < (int)pool.size(); ++i)
          if (!pool[i]->busy && pool[i].get() != idle && (victim < 0 || pool[i]->last < pool[victim]->last))
            victim = i;
        if (victim < 0) break;
        pool_bytes -= pool[victim]->bytes;
        evict.push_back(std::move(pool[victim]));
        pool.erase(pool.begin() + victim);
      }
      queue.erase(it);
      if (idle) idle->busy = true;
      j->pp = idle;
      j->reserved = need;
      running_bytes += need;
      peak = std::max(peak, in_use());
      ++running;
      peak_running = std::max(peak_running, running);
      return j;
    }
    return nullptr;
  }

  void run(Worker& w) {
    cudaSetDevice(device);
    for (;;) {
      Job* j = nullptr;
      std::vector<std::unique_ptr<PooledPlan>> evict;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait(lk, [&] {
          if (stop) return true;
          j = pick(evict);
          return j != nullptr;
        });
        if (!j) return;
        j->t_start = Clock::now();
      }
      for (auto& p : evict) fkp_plan_destroy(p->plan);
      evict.clear();
      int rc = FKP_OK;
      PooledPlan* pp = j->pp;
      std::unique_ptr<PooledPlan> fresh;
      if (!pp) {
        fresh = std::make_unique<PooledPlan>();
        const fkp_bshells_t* bs = (j->req.want & (FKP_B0 | FKP_B2 | FKP_B4)) ? &j->req.bshells : nullptr;
        rc = fkp_plan_create(ctx, &j->req.geom, &j->req.pbins, bs, j->req.want, &fresh->plan);
        if (rc) fresh.reset();
        else {
          fresh->key = j->req;
          fresh->busy = true;
          pp = fresh.get();
        }
      }
      if (!rc) {
        if (j->req.want & (FKP_B0 | FKP_B2 | FKP_B4))
          rc = fkp_bispectrum(pp->plan, &j->req.gal, &j->req.ran, j->req.contraction, w.stream, j->req.pout,
                              j->req.bout);
        else
          rc = fkp_power(pp->plan, &j->req.gal, &j->req.ran, w.stream, j->req.pout);
      }
      // a pooled plan is charged at least what admission reserved for it, so
      // that the pool's accounting and the admission estimate agree
      size_t bytes = 0;
      if (pp) fkp_plan_sizes(pp->plan, nullptr, nullptr, &bytes);
      bytes = std::max(bytes, j->plan_est);
      {
        std::lock_guard<std::mutex> lk(mu);
        running_bytes -= j->reserved;
        if (fresh) {
          pool.push_back(std::move(fresh));
        } else if (pp) {
          pool_bytes -= pp->bytes;
        }
        if (pp) {
          pp->bytes = bytes;
          pool_bytes += bytes;
          pp->busy = false;
          pp->last = ++tick;
        }
        j->status = rc;
        if (rc) j->msg = fkp_last_error();
        j->done = true;
        j->t_end = Clock::now();
        --running;
        ++completed;
        if (rc) ++failed;
      }
      cv_done.notify_all();
      cv_work.notify_all();
    }
  }
};

}  // namespace
}  // namespace fkp

using namespace fkp;

extern "C" int fkp_server_create(int device, int nslots, size_t hbm_budget_bytes, void** out) {
  if (!out || nslots < 1 || nslots > 64) return set_error(FKP_EINVAL, "fkp_server_create: need 1..64 slots");
  auto* S = new Server();
  int rc = fkp_context_create(device, 0, &S->ctx);
  if (rc) {
    delete S;
    return rc;
  }
  S->device = device;
  size_t freeb = 0, total = 0;
  cudaSetDevice(device);
  cudaMemGetInfo(&freeb, &total);
  S->budget = hbm_budget_bytes ? hbm_budget_bytes : freeb * 9 / 10;
  for (int i = 0; i < nslots; ++i) {
    auto w = std::make_unique<Worker>();
    w->srv = S;
    w->id = i;
    if (cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking) != cudaSuccess) {
      fkp_context_destroy(S->ctx);
      delete S;
      return set_error(FKP_ECUDA, "cannot create a stream for slot %d", i);
    }
    S->workers.push_back(std::move(w));
  }
  for (auto& w : S->workers) {
    Worker* wp = w.get();
    wp->th = std::thread([S, wp] { S->run(*wp); });
  }
  *out = S;
  return FKP_OK;
}

extern "C" int fkp_server_submit(void* srv, const fkp_request_t* req, uint64_t* ticket) {
  auto* S = static_cast<Server*>(srv);
  if (!S || !req || !ticket) return set_error(FKP_EINVAL, "fkp_server_submit: NULL argument");
  if (req->geom.N < 8 || req->geom.N > 512 || req->pbins.nbins < 1)
    return set_error(FKP_EINVAL, "fkp_server_submit: bad geometry or bins");
  auto j = std::make_unique<Job>();
  j->req = *req;
  j->plan_est = estimate_plan(*req);
  j->cat_bytes = estimate_catalog(*req);
  j->t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(S->mu);
  if (j->plan_est + j->cat_bytes > S->budget) {
    ++S->rejected;
    return set_error(FKP_ENOMEM, "request needs about %.2f GB, over the server's budget of %.2f GB",
                     (j->plan_est + j->cat_bytes) / 1e9, S->budget / 1e9);
  }
  j->ticket = S->next_ticket++;
  *ticket = j->ticket;
  S->queue.push_back(j.get());
  S->jobs[j->ticket] = std::move(j);
  ++S->submitted;
  S->cv_work.notify_all();
  return FKP_OK;
}

extern "C" int fkp_server_poll(void* srv, uint64_t ticket, int* done) {
  auto* S = static_cast<Server*>(srv);
  if (!S || !done) return set_error(FKP_EINVAL, "fkp_server_poll: NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->jobs.find(ticket);
  if (it == S->jobs.end()) return set_error(FKP_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
  *done = it->second->done ? 1 : 0;
  return FKP_OK;
}

extern "C" int fkp_server_wait(void* srv, uint64_t ticket, int timeout_ms, int* status, double* latency_ms) {
  auto* S = static_cast<Server*>(srv);
  if (!S) return set_error(FKP_EINVAL, "fkp_server_wait: NULL server");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->jobs.find(ticket);
  if (it == S->jobs.end()) return set_error(FKP_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
  Job* j = it->second.get();
  const auto pred = [&] { return j->done; };
  if (timeout_ms < 0) S->cv_done.wait(lk, pred);
  else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred))
    return set_error(FKP_ETIMEOUT, "ticket %llu not finished within %d ms", (unsigned long long)ticket, timeout_ms);
  if (status) *status = j->status;
  if (j->status) set_error(j->status, "ticket %llu: %s", (unsigned long long)ticket, j->msg.c_str());
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(j->t_end - j->t_submit).count();
  S->jobs.erase(it);
  return FKP_OK;
}

extern "C" int fkp_server_stats(void* srv, fkp_server_stats_t* st) {
  auto* S = static_cast<Server*>(srv);
  if (!S || !st) return set_error(FKP_EINVAL, "fkp_server_stats: NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  st->submitted = S->submitted;
  st->completed = S->completed;
  st->failed = S->failed;
  st->rejected = S->rejected;
  st->queued = (int64_t)S->queue.size();
  st->running = S->running;
  st->peak_running = S->peak_running;
  st->bytes_in_use = S->in_use();
  st->peak_bytes = S->peak;
  st->budget_bytes = S->budget;
  return FKP_OK;
}

extern "C" void fkp_server_destroy(void* srv) {
  auto* S = static_cast<Server*>(srv);
  if (!S) return;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    // let queued and running requests finish
    S->cv_done.wait(lk, [&] { return S->queue.empty() && S->running == 0; });
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto& w : S->workers) {
    if (w->th.joinable()) w->th.join();
    if (w->stream) cudaStreamDestroy(w->stream);
  }
  for (auto& p : S->pool) fkp_plan_destroy(p->plan);
  fkp_context_destroy(S->ctx);
  delete S;
}
