// The serving loop (meb_server_*): continuous batching of MEB requests on one
// GPU.
//
// Requests arrive on any host thread (meb_server_submit) and are admitted in
// arrival order while the sum of the admitted, unfinished requests' device
// footprints (inputs, outputs and solver scratch, from meb_footprint) stays
// within the budget.  Admitted small requests wait in one queue; each small
// worker owns a context (its own stream, one scratch slot per instance,
// scratch released and stream-ordered after every call) and, whenever it is
// free, launches the queued requests (up to max_group) as one
// meb_solve_batch.  A group launched while others are still on the GPU runs
// beside them: its thread blocks take the SMs the running groups do not use
// or release.  A group holds its worker until its slowest request ends, so
// groups are kept small and workers many: the SMs stay busy while a long
// request finishes.  Large requests (m*d >= large_balls, or d beyond the batch
// solver's limit) go to large workers, one multi-block meb_solve each.  The
// multi-block kernels need many SMs at once while every batch block holds an
// SM for a whole solve, so each side waits for the other: the threshold is
// high (2^27 coordinates, 1 GB of FP64 centres) and everything below it is
// solved one thread block per request.
// Completion frees the request's budget and admits the next ones.
//
// Each request is solved by the same steps whatever else is queued (one
// thread block per request in the batch kernel, or the multi-block path), so
// its results are the same alone and in any mix.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/meb.h"

// meb_api.cu: scratch of a context from a given pool (library-internal)
extern "C" void meb_ctx_use_pool(meb_ctx* ctx, cudaMemPool_t pool);

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t ticket = 0;
  const double* C = nullptr;
  const double* R = nullptr;
  int64_t m = 0;
  int32_t d = 0;
  double* c_out = nullptr;
  int64_t* act = nullptr;
  int64_t cap = 0;
  meb_info* info = nullptr;
  int64_t footprint = 0;
  bool large = false;
  bool done = false;
  int rc = MEB_OK;
  Clock::time_point t_submit, t_done;
};

constexpr int kBatchMaxD = 4096;   // the batch solver's largest d

// The workers allocate and free stream-ordered from a pool of the servers'
// own, one per device for the process.  Freed memory stays in it (up to the
// largest budget of the servers created) instead of going back to the driver
// at every synchronisation, and a later server reuses what an earlier one
// mapped: a server created after another had served (and returned its memory)
// ran at about half the throughput while mapping memory anew.  A block freed
// on one worker's stream is reused by another only once that free has
// completed: with the allocator's internal dependencies a worker's launch
// would wait for another worker's batch, and the workers would run one after
// another.
// The k-th worker stream of the process on `device` (created once, kept for
// later servers): each server's workers reuse the same streams instead of
// creating and destroying their own.
cudaStream_t server_stream(int device, int k) {
  static std::mutex mu;
  static std::unordered_map<int, std::vector<cudaStream_t>> streams;
  std::lock_guard<std::mutex> lk(mu);
  std::vector<cudaStream_t>& v = streams[device];
  while ((int)v.size() <= k) {
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
    v.push_back(s);
  }
  return v[k];
}

cudaMemPool_t server_pool(int device, int64_t budget) {
  static std::mutex mu;
  static std::unordered_map<int, cudaMemPool_t> pools;
  std::lock_guard<std::mutex> lk(mu);
  cudaMemPool_t& p = pools[device];
  if (!p) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
      p = nullptr;
      return nullptr;
    }
    int no = 0, yes = 1;
    cudaMemPoolSetAttribute(p, cudaMemPoolReuseAllowInternalDependencies, &no);
    cudaMemPoolSetAttribute(p, cudaMemPoolReuseAllowOpportunistic, &yes);
    cudaMemPoolSetAttribute(p, cudaMemPoolReuseFollowEventDependencies, &yes);
  }
  uint64_t keep = 0;
  cudaMemPoolGetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
  if ((uint64_t)budget > keep) {
    keep = (uint64_t)budget;
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  return p;
}

}  // namespace

struct meb_server {
  int device = 0;
  meb_server_config cfg{};
  meb_params P{};
  std::mutex mu;
  std::condition_variable cv_work;   // wakes workers: admitted requests or stop
  std::condition_variable cv_done;   // wakes waiters: a request finished
  std::deque<Request*> pending;      // submitted, not admitted (arrival order)
  std::deque<Request*> small_q, large_q;
  std::unordered_map<int64_t, Request*> live;
  int64_t next_ticket = 1;
  int64_t used = 0;
  meb_server_stats st{};
  bool stop = false;
  cudaMemPool_t pool = nullptr;      // the workers' scratch and staging (shared per device)
  std::vector<std::thread> workers;
};

namespace {

int64_t request_footprint(int64_t m, int32_t d, int64_t cap, bool large) {
  int64_t scratch = 0;
  meb_footprint(m, d, large ? 0 : 1, &scratch);
  const int64_t io = 8 * m * (int64_t)(d + 1) + 8 * (int64_t)d + 8 * cap;
  return io + scratch + (1 << 16);   // + the per-call records of a launch
}

// Under the lock: admit in arrival order while the footprints fit.
void admit(meb_server* sv) {
  bool any = false;
  while (!sv->pending.empty()) {
    Request* r = sv->pending.front();
    if (sv->used + r->footprint > sv->cfg.budget_bytes) break;
    sv->used += r->footprint;
    sv->pending.pop_front();
    (r->large ? sv->large_q : sv->small_q).push_back(r);
    any = true;
  }
  sv->st.in_use_bytes = sv->used;
  sv->st.peak_bytes = std::max(sv->st.peak_bytes, sv->used);
  sv->st.pending = (int64_t)sv->pending.size();
  if (any) sv->cv_work.notify_all();
}

// Under the lock: a request finished with rc.
void finish(meb_server* sv, Request* r, int rc) {
  r->rc = rc;
  r->done = true;
  r->t_done = Clock::now();
  sv->used -= r->footprint;
  if (rc == MEB_OK || rc == MEB_ENOTCONV) sv->st.completed++;
  else sv->st.failed++;
}

int rc_of(const meb_info& info) {
  return info.status == -1 ? MEB_EINVAL : info.status == 0 ? MEB_OK : MEB_ENOTCONV;
}

void small_worker(meb_server* sv, int k) {
  cudaSetDevice(sv->device);
  meb_ctx* ctx = nullptr;
  cudaStream_t ws = server_stream(sv->device, k);
  const int crc = ws ? meb_create(&ctx, sv->device, ws) : MEB_ECUDA;
  if (crc == MEB_OK) {
    meb_set_option(ctx, MEB_OPT_BATCH_SLOTS, 1);
    meb_set_option(ctx, MEB_OPT_RELEASE_SCRATCH, 1);
    if (!(sv->cfg.flags & MEB_SERVER_SPIN_WAITS)) meb_set_option(ctx, MEB_OPT_BLOCKING_SYNC, 1);
    meb_ctx_use_pool(ctx, sv->pool);
  }
  std::vector<Request*> group;
  std::vector<meb_batch_item> items;
  std::vector<meb_info> infos;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      sv->cv_work.wait(lk, [&] { return sv->stop || !sv->small_q.empty(); });
      if (sv->small_q.empty()) break;   // stop, and nothing left to run
      group.clear();
      while (!sv->small_q.empty() && (int)group.size() < sv->cfg.max_group) {
        group.push_back(sv->small_q.front());
        sv->small_q.pop_front();
      }
      sv->st.launches++;
    }
    const int n = (int)group.size();
    items.assign(n, meb_batch_item{});
    infos.assign(n, meb_info{});
    for (int k = 0; k < n; k++) {
      const Request* r = group[k];
      items[k].centers = r->C;
      items[k].radii = r->R;
      items[k].m = r->m;
      items[k].d = r->d;
      items[k].c_out = r->c_out;
      items[k].active_idx = r->act;
      items[k].active_cap = r->cap;
    }
    const int rc = ctx ? meb_solve_batch(ctx, n, items.data(), 0.0, &sv->P, 0, infos.data())
                       : crc;
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      for (int k = 0; k < n; k++) {
        Request* r = group[k];
        if (r->info) *r->info = infos[k];
        const bool call_failed = !(rc == MEB_OK || rc == MEB_EINVAL || rc == MEB_ENOTCONV);
        finish(sv, r, call_failed ? rc : rc_of(infos[k]));
      }
      admit(sv);
    }
    sv->cv_done.notify_all();
  }
  if (ctx) meb_destroy(ctx);
}

void large_worker(meb_server* sv, int k) {
  cudaSetDevice(sv->device);
  meb_ctx* ctx = nullptr;
  cudaStream_t ws = server_stream(sv->device, k);
  const int crc = ws ? meb_create(&ctx, sv->device, ws) : MEB_ECUDA;
  if (crc == MEB_OK) {
    meb_set_option(ctx, MEB_OPT_RELEASE_SCRATCH, 1);
    if (!(sv->cfg.flags & MEB_SERVER_SPIN_WAITS)) meb_set_option(ctx, MEB_OPT_BLOCKING_SYNC, 1);
    meb_ctx_use_pool(ctx, sv->pool);
  }
  for (;;) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      sv->cv_work.wait(lk, [&] { return sv->stop || !sv->large_q.empty(); });
      if (sv->large_q.empty()) break;
      r = sv->large_q.front();
      sv->large_q.pop_front();
      sv->st.launches++;
    }
    meb_info info;
    memset(&info, 0, sizeof(info));
    const int rc = ctx ? meb_solve(ctx, r->C, r->R, r->m, r->d, 0.0, &sv->P, 0, r->c_out, r->act,
                                   r->cap, &info)
                       : crc;
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      if (r->info) *r->info = info;
      finish(sv, r, rc);
      admit(sv);
    }
    sv->cv_done.notify_all();
  }
  if (ctx) meb_destroy(ctx);
}

}  // namespace

extern "C" int meb_server_create(meb_server** out, int device, const meb_server_config* cfg,
                                 const meb_params* params) {
  if (!out || !cfg || cfg->budget_bytes <= 0) return MEB_EINVAL;
  *out = nullptr;
  meb_server* sv = new (std::nothrow) meb_server();
  if (!sv) return MEB_ENOMEM;
  sv->device = device;
  sv->cfg = *cfg;
  if (sv->cfg.small_workers <= 0) sv->cfg.small_workers = 64;
  if (sv->cfg.large_workers <= 0) sv->cfg.large_workers = 2;
  if (sv->cfg.large_balls <= 0) sv->cfg.large_balls = (int64_t)1 << 27;
  if (sv->cfg.max_group <= 0) sv->cfg.max_group = 4;
  if (params) sv->P = *params;
  else meb_params_default(&sv->P);
  if (cudaSetDevice(device) != cudaSuccess) {
    delete sv;
    return MEB_ECUDA;
  }
  if (!(sv->cfg.flags & MEB_SERVER_DEVICE_POOL)) {
    sv->pool = server_pool(device, sv->cfg.budget_bytes);
    if (!sv->pool) {
      delete sv;
      return MEB_ECUDA;
    }
  }
  for (int k = 0; k < sv->cfg.small_workers; k++) sv->workers.emplace_back(small_worker, sv, k);
  for (int k = 0; k < sv->cfg.large_workers; k++)
    sv->workers.emplace_back(large_worker, sv, sv->cfg.small_workers + k);
  *out = sv;
  return MEB_OK;
}

extern "C" int meb_server_submit(meb_server* sv, const double* centers, const double* radii,
                                 int64_t m, int32_t d, double* c_out, int64_t* active_idx,
                                 int64_t active_cap, meb_info* info, int64_t* ticket) {
  if (!sv || !centers || !radii || !c_out || !ticket || active_cap < 0 ||
      (active_cap > 0 && !active_idx))
    return MEB_EINVAL;
  if (m < 1 || m > (int64_t)2147483647 - 256 || d < 1 || d > 16384) return MEB_EINVAL;
  Request* r = new (std::nothrow) Request();
  if (!r) return MEB_ENOMEM;
  r->C = centers;
  r->R = radii;
  r->m = m;
  r->d = d;
  r->c_out = c_out;
  r->act = active_idx;
  r->cap = active_cap;
  r->info = info;
  r->large = m * (int64_t)d >= sv->cfg.large_balls || d > kBatchMaxD;
  r->footprint = request_footprint(m, d, active_cap, r->large);
  if (r->footprint > sv->cfg.budget_bytes) {
    delete r;
    return MEB_ENOMEM;
  }
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    r->ticket = sv->next_ticket++;
    sv->live[r->ticket] = r;
    sv->pending.push_back(r);
    sv->st.submitted++;
    admit(sv);
  }
  *ticket = r->ticket;
  return MEB_OK;
}

extern "C" int meb_server_wait(meb_server* sv, int64_t ticket, double timeout_s, int* rc,
                               double* latency_s) {
  if (!sv) return MEB_EINVAL;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->live.find(ticket);
  if (it == sv->live.end()) return MEB_EINVAL;
  Request* r = it->second;
  auto ready = [&] { return r->done; };
  if (timeout_s < 0) sv->cv_done.wait(lk, ready);
  else if (!sv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready))
    return MEB_ETIMEOUT;
  if (rc) *rc = r->rc;
  if (latency_s) *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
  sv->live.erase(it);
  delete r;
  return MEB_OK;
}

extern "C" int meb_server_get_stats(meb_server* sv, meb_server_stats* out) {
  if (!sv || !out) return MEB_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  *out = sv->st;
  out->pending = (int64_t)sv->pending.size();
  return MEB_OK;
}

extern "C" void meb_server_destroy(meb_server* sv) {
  if (!sv) return;
  {
    // every submitted request runs to completion first
    std::unique_lock<std::mutex> lk(sv->mu);
    sv->cv_done.wait(lk, [&] {
      return sv->pending.empty() && sv->small_q.empty() && sv->large_q.empty() && sv->used == 0;
    });
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  for (auto& t : sv->workers) t.join();
  for (auto& kv : sv->live) delete kv.second;
  delete sv;
}
