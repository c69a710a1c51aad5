// C ABI of the serving engine (pf_server_*, declared in include/pf.h): host
// logic only.  Streams of observations arrive at any time; each stream's
// particle state stays resident in one batch pool (batch_api.cuh); a worker
// thread forms each cycle from whatever observations are pending (one per
// stream, continuous batching), launches it as one persistent kernel
// (batch.cuh) followed by the summaries of the stepped streams, and keeps up
// to max_inflight cycles on the device while the next one is formed.
// Streams wait in FIFO order for admission while the pool (the HBM budget)
// or the slots are full, and enter as others close.
//
// Compiled as part of api.cu.
#pragma once
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "batch_api.cuh"

namespace {

double now_us() {
  using namespace std::chrono;
  return (double)duration_cast<nanoseconds>(steady_clock::now().time_since_epoch()).count() * 1e-3;
}

struct SrvObs {
  double y;
  double t_sub;   // submit time (us)
  uint64_t seq;
};

struct SrvStream {
  pf_config cfg;
  int64_t slot = -1;         // batch slot while resident
  std::deque<SrvObs> pending;
  uint64_t next_seq = 0;
  uint32_t inflight = 0;     // observations in cycles not yet retired
  bool queued = false;       // in the ready list
  bool closing = false;
  bool waiting = false;      // in the admission queue
  double t_open = 0;
};

struct SrvItem {
  uint64_t id, seq;
  double t_sub;
  uint32_t slot;
  double y;
};

struct SrvCycle {
  uint32_t r;
  std::vector<SrvItem> items;
  double t_launch;
};

}  // namespace

struct pf_server {
  pf_batch* b = nullptr;
  uint32_t max_inflight = 2;
  bool keep_results = false;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread worker, replayer;
  bool stop = false;
  bool replaying = false;
  pf_status err = PF_OK;
  char err_msg[512] = "";
  std::unordered_map<uint64_t, SrvStream> streams;
  std::deque<uint64_t> waiting;              // admission FIFO
  std::vector<uint64_t> ready;               // resident streams with pending observations
  std::vector<uint64_t> closing;             // streams to release once drained
  std::deque<SrvCycle> inflight;
  double* est_dev[pf_batch::kRing] = {};
  double* est_pin[pf_batch::kRing] = {};
  cudaEvent_t cyc_ev[pf_batch::kRing] = {};
  uint32_t ring = 0;
  std::deque<pf_server_result> results;
  std::vector<float> lat_us;
  std::vector<float> sub_s;                  // submit time of each result, s after the first submit
  double warmup_s = 0;
  // counters
  uint64_t submitted = 0, completed = 0, cycles = 0, particle_steps = 0, admitted = 0,
           admitted_after_wait = 0, streams_opened = 0, streams_closed = 0, items_total = 0;
  uint32_t max_cycle_items = 0;
  double t_first_sub = -1, t_last_done = -1, replay_max_lag_us = 0, wait_us_total = 0;
};

namespace {

pf_status srv_fail(pf_server* s, pf_status st) {
  if (s->err == PF_OK) {
    s->err = st;
    std::snprintf(s->err_msg, sizeof(s->err_msg), "%s", pf_last_error());
  }
  s->cv_done.notify_all();
  return st;
}

void srv_make_ready(pf_server* s, uint64_t id, SrvStream& st) {
  if (st.slot >= 0 && !st.queued && !st.pending.empty()) {
    st.queued = true;
    s->ready.push_back(id);
  }
}

// Admit waiting streams in FIFO order while the pool and the slots have room;
// all streams admitted together share one admission list and init launch.
pf_status srv_admit(pf_server* s) {
  std::vector<uint32_t> slots;
  while (!s->waiting.empty()) {
    const uint64_t id = s->waiting.front();
    auto it = s->streams.find(id);
    if (it == s->streams.end()) {
      s->waiting.pop_front();
      continue;
    }
    SrvStream& st = it->second;
    uint32_t slot = 0;
    if (!batch_reserve(s->b, st.cfg, &slot)) break;
    slots.push_back(slot);
    s->waiting.pop_front();
    st.waiting = false;
    st.slot = slot;
    s->admitted++;
    const double w = now_us() - st.t_open;
    if (w > 1000.0) s->admitted_after_wait++;
    s->wait_us_total += w;
    srv_make_ready(s, id, st);
  }
  return batch_init_slots(s->b, slots.data(), (uint32_t)slots.size());
}

// Release closing streams whose observations are all done.
pf_status srv_release(pf_server* s) {
  size_t keep = 0;
  for (size_t i = 0; i < s->closing.size(); ++i) {
    const uint64_t id = s->closing[i];
    auto it = s->streams.find(id);
    if (it == s->streams.end()) continue;
    SrvStream& st = it->second;
    if (!st.pending.empty() || st.inflight) {
      s->closing[keep++] = id;
      continue;
    }
    if (st.slot >= 0) {
      const pf_status r = pf_batch_remove(s->b, (uint32_t)st.slot);
      if (r != PF_OK) return r;
    }
    s->streams.erase(it);
    s->streams_closed++;
  }
  if (keep != s->closing.size()) s->cv_done.notify_all();
  s->closing.resize(keep);
  return PF_OK;
}

void srv_retire_front(pf_server* s) {
  SrvCycle& c = s->inflight.front();
  const double t = now_us();
  const double* rows = s->est_pin[c.r];
  for (size_t i = 0; i < c.items.size(); ++i) {
    const SrvItem& it = c.items[i];
    const double* v = rows + i * BATCH_EST_ROW;
    const float lat = (float)(t - it.t_sub);
    s->lat_us.push_back(lat);
    s->sub_s.push_back((float)((it.t_sub - s->t_first_sub) * 1e-6));
    auto sit = s->streams.find(it.id);
    if (sit != s->streams.end()) {
      sit->second.inflight--;
      s->particle_steps += sit->second.cfg.n_particles;
    }
    if (s->keep_results) {
      pf_server_result r;
      r.stream_id = it.id;
      r.seq = it.seq;
      r.est.t = (uint64_t)v[0];
      r.est.x_mean = v[1];
      r.est.x_var = v[2];
      r.est.sigma2_mean = v[3];
      r.est.sigma2_var = v[4];
      r.est.tau2_mean = v[5];
      r.est.tau2_var = v[6];
      r.est.log_marglik = v[7];
      r.status = (uint32_t)v[8] ? (int32_t)PF_ERR_NUMERIC : (int32_t)PF_OK;
      r.latency_us = lat;
      s->results.push_back(r);
    }
  }
  s->completed += c.items.size();
  s->t_last_done = t;
  s->inflight.pop_front();
  s->cv_done.notify_all();
}

// Stage and launch one cycle for `items` (sorted largest filter first) on
// ring slot r, then the summaries of the stepped streams and their copy to
// the host.  Called without the lock: only the worker touches the batch.
pf_status srv_launch(pf_server* s, uint32_t r, const std::vector<SrvItem>& items) {
  pf_batch* b = s->b;
  CK(cudaEventSynchronize(b->list_ev[r]));
  BatchItem* li = (BatchItem*)(b->list_pin[r] + 16);
  for (size_t i = 0; i < items.size(); ++i) {
    li[i].slot = items[i].slot;
    li[i].pad = 0;
    li[i].y = items[i].y;
  }
  const uint32_t cnt = (uint32_t)items.size();
  ((uint32_t*)b->list_pin[r])[0] = cnt;
  ((uint32_t*)b->list_pin[r])[1] = big_items(b, li, cnt);
  CK(cudaMemcpyAsync(b->list_dev[r], b->list_pin[r], 16 + (size_t)cnt * sizeof(BatchItem),
                     cudaMemcpyHostToDevice, b->stream));
  CK(cudaEventRecord(b->list_ev[r], b->stream));
  CK(cudaGraphLaunch(b->exec[r], b->stream));
  b->cycles++;
  const unsigned grid = (unsigned)std::min<uint64_t>(cnt, b->grid);
  if (b->fp64) {
    BatchArgs<double> a = batch_args<double>(b);
    set_list(a, b->list_dev[r]);
    a.est = s->est_dev[r];
    CK(batch_estimate_launch<double>(grid, a, b->stream));
  } else {
    BatchArgs<float> a = batch_args<float>(b);
    set_list(a, b->list_dev[r]);
    a.est = s->est_dev[r];
    CK(batch_estimate_launch<float>(grid, a, b->stream));
  }
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(s->est_pin[r], s->est_dev[r], (size_t)cnt * BATCH_EST_ROW * 8,
                     cudaMemcpyDeviceToHost, b->stream));
  CK(cudaEventRecord(s->cyc_ev[r], b->stream));
  return PF_OK;
}

void srv_loop(pf_server* s) {
  std::unique_lock<std::mutex> lk(s->mu);
  std::vector<SrvItem> items;
  while (true) {
    while (!s->inflight.empty() && cudaEventQuery(s->cyc_ev[s->inflight.front().r]) == cudaSuccess)
      srv_retire_front(s);
    pf_status st = srv_release(s);
    if (st == PF_OK) st = srv_admit(s);
    if (st != PF_OK) {
      srv_fail(s, st);
      return;
    }
    bool launched = false;
    if (!s->ready.empty() && s->inflight.size() < s->max_inflight) {
      // one pending observation of every ready stream
      items.clear();
      std::vector<uint64_t> still;
      for (uint64_t id : s->ready) {
        auto it = s->streams.find(id);
        if (it == s->streams.end()) continue;
        SrvStream& ss = it->second;
        const SrvObs o = ss.pending.front();
        ss.pending.pop_front();
        ss.inflight++;
        items.push_back({id, o.seq, o.t_sub, (uint32_t)ss.slot, o.y});
        if (!ss.pending.empty()) still.push_back(id);
        else ss.queued = false;
      }
      s->ready.swap(still);
      const pf_batch* b = s->b;
      std::sort(items.begin(), items.end(), [b](const SrvItem& x, const SrvItem& y2) {
        const uint32_t nx = b->Fh[x.slot].n, ny = b->Fh[y2.slot].n;
        return nx != ny ? nx > ny : x.slot < y2.slot;
      });
      const uint32_t r = s->ring;
      s->ring = (r + 1) % pf_batch::kRing;
      SrvCycle c;
      c.r = r;
      c.items = items;
      c.t_launch = now_us();
      s->cycles++;
      s->items_total += items.size();
      s->max_cycle_items = std::max<uint32_t>(s->max_cycle_items, (uint32_t)items.size());
      lk.unlock();
      st = srv_launch(s, r, items);
      lk.lock();
      if (st != PF_OK) {
        s->b->sticky = PF_ERR_CUDA;
        srv_fail(s, st);
        return;
      }
      s->inflight.push_back(std::move(c));
      launched = true;
    }
    if (launched && s->inflight.size() < s->max_inflight) continue;
    if (!s->inflight.empty()) {
      // wait for the oldest cycle, then form the next from what arrived
      const uint32_t r = s->inflight.front().r;
      lk.unlock();
      const cudaError_t e = cudaEventSynchronize(s->cyc_ev[r]);
      lk.lock();
      if (e != cudaSuccess) {
        s->b->sticky = PF_ERR_CUDA;
        srv_fail(s, set_err(PF_ERR_CUDA, "served cycle: %s", cudaGetErrorString(e)));
        return;
      }
      srv_retire_front(s);
      continue;
    }
    if (s->stop && s->ready.empty()) return;
    s->cv_work.wait_for(lk, std::chrono::milliseconds(2));
  }
}

pf_status srv_open_locked(pf_server* s, uint64_t id, const pf_config* cfg) {
  if (s->streams.count(id)) return set_err(PF_ERR_INVALID, "stream %llu is already open", (unsigned long long)id);
  pf_status st = validate_member(s->b, cfg);
  if (st != PF_OK) return st;
  if (round_pool(cfg->n_particles) > s->b->pool)
    return set_err(PF_ERR_BUSY, "stream of %llu particles can never fit the pool",
                   (unsigned long long)cfg->n_particles);
  SrvStream& ss = s->streams[id];
  ss.cfg = *cfg;
  ss.t_open = now_us();
  ss.waiting = true;
  s->waiting.push_back(id);
  s->streams_opened++;
  s->cv_work.notify_one();
  return PF_OK;
}

pf_status srv_submit_locked(pf_server* s, uint64_t id, double y) {
  auto it = s->streams.find(id);
  if (it == s->streams.end()) return set_err(PF_ERR_INVALID, "stream %llu is not open", (unsigned long long)id);
  SrvStream& ss = it->second;
  if (ss.closing) return set_err(PF_ERR_INVALID, "stream %llu is closing", (unsigned long long)id);
  const double t = now_us();
  if (s->t_first_sub < 0) s->t_first_sub = t;
  ss.pending.push_back({y, t, ss.next_seq++});
  s->submitted++;
  srv_make_ready(s, id, ss);
  s->cv_work.notify_one();
  return PF_OK;
}

pf_status srv_close_locked(pf_server* s, uint64_t id) {
  auto it = s->streams.find(id);
  if (it == s->streams.end()) return set_err(PF_ERR_INVALID, "stream %llu is not open", (unsigned long long)id);
  if (it->second.closing) return PF_OK;
  it->second.closing = true;
  s->closing.push_back(id);
  s->cv_work.notify_one();
  return PF_OK;
}

struct ReplayPlan {
  std::vector<double> t_s;
  std::vector<uint8_t> kind;
  std::vector<uint64_t> id;
  std::vector<double> y;
  std::vector<pf_config> cfgs;
};

void srv_replay(pf_server* s, ReplayPlan* plan) {
  const double t0 = now_us();
  for (size_t i = 0; i < plan->t_s.size(); ++i) {
    const double target = t0 + plan->t_s[i] * 1e6;
    double now = now_us();
    if (now < target - 200.0)
      std::this_thread::sleep_for(std::chrono::microseconds((int64_t)(target - now - 100.0)));
    while ((now = now_us()) < target) {
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->replay_max_lag_us = std::max(s->replay_max_lag_us, now - target);
    if (s->err != PF_OK) break;
    pf_status st = PF_OK;
    const uint64_t id = plan->id[i];
    if (plan->kind[i] == PF_EVENT_OBS) st = srv_submit_locked(s, id, plan->y[i]);
    else if (plan->kind[i] == PF_EVENT_CLOSE) st = srv_close_locked(s, id);
    else if (id < plan->cfgs.size()) st = srv_open_locked(s, id, &plan->cfgs[id]);
    else st = set_err(PF_ERR_INVALID, "open event for stream %llu without a configuration", (unsigned long long)id);
    if (st != PF_OK && st != PF_ERR_BUSY) {
      srv_fail(s, st);
      break;
    }
  }
  std::lock_guard<std::mutex> lk(s->mu);
  s->replaying = false;
  s->cv_done.notify_all();
  delete plan;
}

pf_status srv_check(pf_server* s) {
  if (!s) return set_err(PF_ERR_INVALID, "NULL server handle");
  if (s->err != PF_OK) return set_err(s->err, "server failed: %s", s->err_msg);
  return PF_OK;
}

}  // namespace

extern "C" {

pf_status pf_server_create(const pf_server_opts* opts, pf_server** out) {
  if (!opts || !out) return set_err(PF_ERR_INVALID, "NULL argument");
  *out = nullptr;
  if (opts->max_inflight > (uint32_t)pf_batch::kRing)
    return set_err(PF_ERR_INVALID, "max_inflight must be in [0, %d]", pf_batch::kRing);
  if (opts->max_streams < 1) return set_err(PF_ERR_INVALID, "max_streams must be >= 1");
  if (opts->hbm_budget_bytes == 0) return set_err(PF_ERR_INVALID, "hbm_budget_bytes must be > 0");
  pf_batch_opts bo;
  std::memset(&bo, 0, sizeof(bo));
  bo.max_filters = opts->max_streams;
  bo.hbm_budget_bytes = opts->hbm_budget_bytes;
  bo.scheme = opts->scheme;
  bo.precision = opts->precision;
  bo.adaptive = opts->adaptive;
  bo.stream = opts->stream;
  bo.alloc = opts->alloc;
  bo.free = opts->free;
  bo.alloc_ctx = opts->alloc_ctx;
  pf_server* s = new (std::nothrow) pf_server();
  if (!s) return set_err(PF_ERR_OOM, "host allocation failed");
  pf_status st = pf_batch_create(nullptr, 0, &bo, &s->b);
  if (st != PF_OK) {
    delete s;
    return st;
  }
  s->max_inflight = opts->max_inflight ? opts->max_inflight : 2;
  s->warmup_s = opts->warmup_s > 0 ? opts->warmup_s : 0.0;
  s->keep_results = opts->keep_results != 0;
  if (opts->block || opts->cluster) {
    const uint32_t blk = opts->block ? opts->block : 256;
    const uint32_t cl = opts->cluster ? opts->cluster : 1;
    uint32_t grid = opts->grid;
    if (!grid)
      for (auto& sh : s->b->shapes)
        if (sh.nt == (int)blk && sh.cl == (int)cl) grid = std::max(grid, sh.grid);
    if ((st = pf_batch_set_shape(s->b, blk, grid, cl, opts->big_min)) != PF_OK) {
      pf_batch_destroy(s->b);
      delete s;
      return st;
    }
  }
  auto bail = [&](pf_status e) {
    pf_server_destroy(s);
    return e;
  };
  for (int r = 0; r < pf_batch::kRing; ++r) {
    const size_t bytes = (size_t)opts->max_streams * BATCH_EST_ROW * 8;
    if ((st = batch_alloc(s->b, bytes, (void**)&s->est_dev[r])) != PF_OK) return bail(st);
    if (cudaHostAlloc((void**)&s->est_pin[r], bytes, cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      return bail(set_err(PF_ERR_OOM, "pinned host allocation failed"));
    }
    if (cudaEventCreateWithFlags(&s->cyc_ev[r], cudaEventDisableTiming) != cudaSuccess)
      return bail(set_err(PF_ERR_CUDA, "cudaEventCreate failed"));
  }
  int dev = 0;
  cudaGetDevice(&dev);
  s->worker = std::thread([s, dev]() {
    cudaSetDevice(dev);
    srv_loop(s);
  });
  *out = s;
  return PF_OK;
}

pf_status pf_server_open(pf_server* s, uint64_t id, const pf_config* cfg) {
  pf_status st = srv_check(s);
  if (st != PF_OK) return st;
  if (!cfg) return set_err(PF_ERR_INVALID, "NULL configuration");
  std::lock_guard<std::mutex> lk(s->mu);
  return srv_open_locked(s, id, cfg);
}

pf_status pf_server_submit(pf_server* s, uint64_t id, double y) {
  pf_status st = srv_check(s);
  if (st != PF_OK) return st;
  std::lock_guard<std::mutex> lk(s->mu);
  return srv_submit_locked(s, id, y);
}

pf_status pf_server_close(pf_server* s, uint64_t id) {
  pf_status st = srv_check(s);
  if (st != PF_OK) return st;
  std::lock_guard<std::mutex> lk(s->mu);
  return srv_close_locked(s, id);
}

pf_status pf_server_replay(pf_server* s, uint64_t count, const double* t_s, const uint8_t* kind,
                           const uint64_t* ids, const double* y, const pf_config* cfgs,
                           uint64_t n_cfgs) {
  pf_status st = srv_check(s);
  if (st != PF_OK) return st;
  if (count && (!t_s || !kind || !ids || !y)) return set_err(PF_ERR_INVALID, "NULL event array");
  for (uint64_t i = 1; i < count; ++i)
    if (!(t_s[i] >= t_s[i - 1])) return set_err(PF_ERR_INVALID, "event times must be nondecreasing");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->replaying) return set_err(PF_ERR_BUSY, "a replay is running");
  }
  if (s->replayer.joinable()) s->replayer.join();
  ReplayPlan* plan = new (std::nothrow) ReplayPlan();
  if (!plan) return set_err(PF_ERR_OOM, "host allocation failed");
  plan->t_s.assign(t_s, t_s + count);
  plan->kind.assign(kind, kind + count);
  plan->id.assign(ids, ids + count);
  plan->y.assign(y, y + count);
  if (n_cfgs) plan->cfgs.assign(cfgs, cfgs + n_cfgs);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->replaying = true;
  }
  s->replayer = std::thread(srv_replay, s, plan);
  return PF_OK;
}

pf_status pf_server_drain(pf_server* s, double timeout_s) {
  if (!s) return set_err(PF_ERR_INVALID, "NULL server handle");
  std::unique_lock<std::mutex> lk(s->mu);
  const auto until = std::chrono::steady_clock::now() +
                     std::chrono::microseconds((int64_t)(timeout_s * 1e6));
  while (s->err == PF_OK && (s->replaying || s->completed < s->submitted || !s->closing.empty())) {
    s->cv_work.notify_one();
    s->cv_done.wait_for(lk, std::chrono::milliseconds(10));
    if (std::chrono::steady_clock::now() > until)
      return set_err(PF_ERR_TIMEOUT, "drain: %llu of %llu observations done, %zu streams closing",
                     (unsigned long long)s->completed, (unsigned long long)s->submitted,
                     s->closing.size());
  }
  if (s->err != PF_OK) return set_err(s->err, "server failed: %s", s->err_msg);
  return PF_OK;
}

pf_status pf_server_poll(pf_server* s, pf_server_result* out, uint32_t max, uint32_t* n) {
  if (!s || !n || (max && !out)) return set_err(PF_ERR_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  uint32_t k = 0;
  while (k < max && !s->results.empty()) {
    out[k++] = s->results.front();
    s->results.pop_front();
  }
  *n = k;
  return s->err;
}

pf_status pf_server_get_stats(pf_server* s, pf_server_stats* out) {
  if (!s || !out) return set_err(PF_ERR_INVALID, "NULL argument");
  std::vector<float> lat;
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(out, 0, sizeof(*out));
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->cycles = s->cycles;
  out->particle_steps = s->particle_steps;
  out->streams_opened = s->streams_opened;
  out->streams_closed = s->streams_closed;
  out->admitted = s->admitted;
  out->admitted_after_wait = s->admitted_after_wait;
  out->waiting = (uint32_t)s->waiting.size();
  out->resident = s->b->resident;
  out->pool_particles = s->b->pool;
  out->used_particles = s->b->used;
  out->mean_cycle_streams = s->cycles ? (double)s->items_total / (double)s->cycles : 0.0;
  out->max_cycle_streams = s->max_cycle_items;
  out->mean_admission_wait_us = s->admitted ? s->wait_us_total / (double)s->admitted : 0.0;
  out->replay_max_lag_us = s->replay_max_lag_us;
  if (s->t_first_sub >= 0 && s->t_last_done > s->t_first_sub) {
    out->wall_s = (s->t_last_done - s->t_first_sub) * 1e-6;
    out->particle_steps_per_s = (double)s->particle_steps / out->wall_s;
    out->obs_per_s = (double)s->completed / out->wall_s;
  }
  auto pct = [&](double q) {
    const size_t k = std::min(lat.size() - 1, (size_t)(q * (double)(lat.size() - 1) + 0.5));
    std::nth_element(lat.begin(), lat.begin() + k, lat.end());
    return (double)lat[k];
  };
  lat = s->lat_us;
  if (!lat.empty()) {
    double sum = 0;
    for (float v : lat) sum += v;
    out->mean_us = sum / (double)lat.size();
    out->p50_us = pct(0.50);
    out->p90_us = pct(0.90);
    out->p99_us = pct(0.99);
    out->max_us = (double)*std::max_element(lat.begin(), lat.end());
  }
  // steady state: observations submitted after the warm-up window
  lat.clear();
  for (size_t i = 0; i < s->lat_us.size(); ++i)
    if (s->sub_s[i] >= s->warmup_s) lat.push_back(s->lat_us[i]);
  out->steady_count = lat.size();
  if (!lat.empty()) {
    out->steady_p50_us = pct(0.50);
    out->steady_p90_us = pct(0.90);
    out->steady_p99_us = pct(0.99);
  }
  out->grid = s->b->grid;
  out->block = (uint32_t)s->b->nt;
  out->cluster = (uint32_t)s->b->cl;
  return s->err;
}

pf_status pf_server_destroy(pf_server* s) {
  if (!s) return PF_OK;
  if (s->replayer.joinable()) s->replayer.join();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->ready.clear();
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  if (s->b) {
    cudaStreamSynchronize(s->b->stream);
    for (int r = 0; r < pf_batch::kRing; ++r) {
      if (s->est_pin[r]) cudaFreeHost(s->est_pin[r]);
      if (s->cyc_ev[r]) cudaEventDestroy(s->cyc_ev[r]);
    }
    pf_batch_destroy(s->b);  // frees est_dev with the pool
  }
  cudaGetLastError();
  delete s;
  return PF_OK;
}

}  // extern "C"
