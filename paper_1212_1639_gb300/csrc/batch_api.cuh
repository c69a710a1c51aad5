// C ABI of batched filters (pf_batch_*, declared in include/pf.h): host logic
// only -- the particle pool and its first-fit allocator, slot bookkeeping,
// the size-ordered work list, CUDA-graph replay of the persistent cycle
// kernel, launch-shape selection and error mapping.  Every step of the
// method runs in the kernels of batch.cuh.
//
// Compiled as part of api.cu (it shares that file's error and allocation
// helpers and its kernels' translation unit).
#pragma once
#include <algorithm>
#include <map>
#include <set>

#include "batch_launch.h"

struct pf_batch {
  int scheme = 0;          // as configured (cut-point variants give the same ancestors)
  int pos = 0;             // POS_MULTINOMIAL or POS_SYSTEMATIC
  bool fp64 = false;
  bool adaptive = false;   // the pool carries lambda: filters may resample adaptively
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  pf_alloc_fn alloc = nullptr;
  pf_free_fn free = nullptr;
  void* alloc_ctx = nullptr;
  uint32_t max_filters = 0;
  uint64_t pool = 0;                 // particles in the pool
  uint64_t bytes_per_particle = 0;
  std::vector<void*> allocs;
  void* x[2] = {}; void* s2[2] = {}; void* t2[2] = {}; void* bs[2] = {}; void* bt[2] = {};
  void* ell = nullptr;
  void* lam = nullptr;               // adaptive batches: carried log-weights
  uint64_t* Q = nullptr;
  uint64_t* S = nullptr;
  uint32_t* anc = nullptr;
  BatchFilter* F = nullptr;          // device, one per slot
  std::vector<BatchFilter> Fh;       // host copy of the fields the host owns
  uint32_t* ctr = nullptr;           // device work counters
  // work lists: kRing lists for cycles (pinned staging + device copy), one
  // for init / estimate
  static constexpr int kRing = 4;
  char* list_dev[kRing + 1] = {};
  char* list_pin[kRing + 1] = {};
  cudaEvent_t list_ev[kRing] = {};
  uint32_t ring = 0;
  double* est_dev = nullptr;
  double* est_pin = nullptr;
  // admission lists (slot + record per admitted filter), a ring of pinned
  // staging buffers so that admitting never waits for cycles in flight
  static constexpr int kAdm = 4;
  char* adm_dev[kAdm] = {};
  char* adm_pin[kAdm] = {};
  cudaEvent_t adm_ev[kAdm] = {};
  uint32_t adm_ring = 0;
  cudaGraphExec_t exec[kRing] = {};
  unsigned grid = 0;                 // persistent grid of the cycle kernel
  int nt = 256;                      // its threads per CTA
  int cl = 1;                        // CTAs per cluster (1: no clusters)
  uint32_t big_min = 0;              // cluster launches: filters this large use a whole cluster
  bool autotune = false, tuned = false;
  struct Shape {
    int nt;
    unsigned grid;
    int cl;
    uint32_t big_min;
  };
  std::vector<Shape> shapes;         // candidates of the autotuner
  std::vector<uint32_t> order;       // resident slots, largest filter first
  std::set<uint32_t> free_slots;
  std::map<uint64_t, uint64_t> free_ranges;  // pool offset -> length (particles)
  uint64_t used = 0;                 // particles of resident filters (rounded)
  uint32_t resident = 0;
  uint64_t cycles = 0;
  pf_status sticky = PF_OK;
};

namespace {

constexpr uint64_t kPoolAlign = 32;  // particles: 128-byte aligned filter ranges

size_t list_bytes(uint32_t max_filters) { return 16 + (size_t)max_filters * sizeof(BatchItem); }

pf_status batch_alloc(pf_batch* b, size_t bytes, void** out) {
  bytes = (bytes + 255) & ~size_t(255);
  void* p = nullptr;
  if (b->alloc) {
    p = b->alloc(bytes, b->stream, b->alloc_ctx);
    if (!p) return set_err(PF_ERR_OOM, "allocator callback returned NULL for %zu bytes", bytes);
  } else {
    cudaError_t e = cudaMallocAsync(&p, bytes, b->stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return set_err(e == cudaErrorMemoryAllocation ? PF_ERR_OOM : PF_ERR_CUDA,
                     "cudaMallocAsync(%zu): %s", bytes, cudaGetErrorString(e));
    }
  }
  if (((uintptr_t)p & 15) != 0) return set_err(PF_ERR_INVALID, "allocator returned a pointer not 16-byte aligned");
  b->allocs.push_back(p);
  *out = p;
  return PF_OK;
}

uint64_t batch_bytes_per_particle(bool fp64, bool multi, bool adaptive) {
  const uint64_t rs = fp64 ? 8 : 4;
  // x, sigma^2, tau^2 and b_sigma, b_tau, both parities; l; Q; ancestors; S;
  // lambda
  return 2 * (3 * rs + 2 * 8) + rs + 8 + 4 + (multi ? 8 : 0) + (adaptive ? rs : 0);
}

template <class R>
BatchArgs<R> batch_args(pf_batch* b) {
  typedef typename SuffT<R>::B Bt;
  BatchArgs<R> a;
  for (int p = 0; p < 2; ++p) {
    a.st[p].x = (R*)b->x[p];
    a.st[p].s2 = (R*)b->s2[p];
    a.st[p].t2 = (R*)b->t2[p];
    a.st[p].bs = (Bt*)b->bs[p];
    a.st[p].bt = (Bt*)b->bt[p];
  }
  a.ell = (R*)b->ell;
  a.lam = (R*)b->lam;
  a.Q = b->Q;
  a.S = b->S;
  a.anc = b->anc;
  a.F = b->F;
  a.items = nullptr;
  a.count = nullptr;
  a.ctr = b->ctr;
  a.est = b->est_dev;
  a.inits = nullptr;
  a.commit = 1;
  return a;
}

void set_list(BatchArgs<float>& a, const char* list) {
  a.count = (const uint32_t*)list;
  a.items = (const BatchItem*)(list + 16);
}
void set_list(BatchArgs<double>& a, const char* list) {
  a.count = (const uint32_t*)list;
  a.items = (const BatchItem*)(list + 16);
}

// Launch the cycle kernel for the list at `list` (device) with the batch's
// current launch shape.
pf_status launch_batch_cycle(pf_batch* b, const char* list, int commit, cudaStream_t s) {
  cudaError_t e;
  if (b->fp64) {
    BatchArgs<double> a = batch_args<double>(b);
    set_list(a, list);
    a.commit = commit;
    e = batch_cycle_launch<double>(b->pos, b->nt, b->cl, b->grid, a, s);
  } else {
    BatchArgs<float> a = batch_args<float>(b);
    set_list(a, list);
    a.commit = commit;
    e = batch_cycle_launch<float>(b->pos, b->nt, b->cl, b->grid, a, s);
  }
  if (e != cudaSuccess) return set_err(PF_ERR_CUDA, "batch cycle launch: %s", cudaGetErrorString(e));
  return PF_OK;
}

unsigned resident_grid(const pf_batch* b, int nt, int cl, int sms) {
  return b->fp64 ? batch_cycle_resident<double>(b->pos, nt, cl, sms)
                 : batch_cycle_resident<float>(b->pos, nt, cl, sms);
}

// Candidate launch shapes: 256 or 512 threads per CTA with 1 .. the resident
// maximum of CTAs per SM; and clusters of 2, 4 or 8 CTAs of 256 threads (as
// many as fit) that take filters of at least 1 or 4 tiles per CTA together.
// The first is the default before tuning (256 threads, as many CTAs as fit,
// no clusters).
pf_status batch_shapes(pf_batch* b) {
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (sms < 1) return set_err(PF_ERR_CUDA, "no multiprocessors");
  b->shapes.clear();
  for (int nt : {256, 512}) {
    const unsigned g = resident_grid(b, nt, 1, sms);
    for (unsigned k = g / (unsigned)sms; k >= 1; --k) b->shapes.push_back({nt, k * (unsigned)sms, 1, 0});
  }
  for (int cl : {2, 4, 8}) {
    const unsigned g = resident_grid(b, 256, cl, sms);
    if (g == 0) continue;
    for (uint32_t tiles : {1u, 4u}) b->shapes.push_back({256, g, cl, tiles * (uint32_t)cl * (uint32_t)TILE});
  }
  if (b->shapes.empty()) return set_err(PF_ERR_CUDA, "no launch shape fits");
  b->nt = b->shapes[0].nt;
  b->grid = b->shapes[0].grid;
  b->cl = b->shapes[0].cl;
  b->big_min = b->shapes[0].big_min;
  return PF_OK;
}

// Number of leading items of a size-ordered list that a cluster launch gives
// to whole clusters.
uint32_t big_items(const pf_batch* b, const BatchItem* items, uint32_t cnt) {
  if (b->cl == 1) return 0;
  uint32_t k = 0;
  while (k < cnt && b->Fh[items[k].slot].n >= b->big_min) ++k;
  return k;
}

pf_status check_batch(pf_batch* b) {
  if (!b) return set_err(PF_ERR_INVALID, "NULL batch handle");
  if (b->sticky != PF_OK) return set_err(b->sticky, "batch is in a failed state (%d)", (int)b->sticky);
  return PF_OK;
}

pf_status batch_fail(pf_batch* b, pf_status st) {
  if (st == PF_ERR_CUDA) b->sticky = st;
  return st;
}

pf_status validate_member(const pf_batch* b, const pf_config* c) {
  if (c->n_particles < 1 || c->n_particles > PF_MAX_PARTICLES)
    return set_err(PF_ERR_INVALID, "n_particles must be in [1, 2^26]");
  if (c->scheme != b->scheme) return set_err(PF_ERR_INVALID, "a filter's scheme differs from its batch's");
  if (c->algorithm != PF_PARTICLE_LEARNING)
    return set_err(PF_ERR_INVALID, "batched and served filters run particle learning");
  if (c->precision != (b->fp64 ? PF_FP64 : PF_FP32))
    return set_err(PF_ERR_INVALID, "a filter's precision differs from its batch's");
  if (!c->known_variances && !(c->a_sigma >= 1.0 && c->a_tau >= 1.0))
    return set_err(PF_ERR_INVALID, "prior shapes must be >= 1");
  if (!(c->b_sigma > 0 && c->b_tau > 0 && c->x0_var >= 0))
    return set_err(PF_ERR_INVALID, "prior scales must be > 0 and x0_var >= 0");
  if (c->known_variances && !(c->sigma2 > 0 && c->tau2 > 0))
    return set_err(PF_ERR_INVALID, "known variances must be > 0");
  if (!(c->ess_frac >= 0.0 && c->ess_frac <= 1.0))
    return set_err(PF_ERR_INVALID, "ess_frac must be in [0, 1]");
  if (c->ess_frac > 0.0 && !b->adaptive)
    return set_err(PF_ERR_INVALID, "ess_frac > 0 needs a batch created with adaptive = 1");
  return PF_OK;
}

uint64_t round_pool(uint64_t n) { return (n + kPoolAlign - 1) / kPoolAlign * kPoolAlign; }

// First fit in the pool; returns false when no free range is large enough.
bool pool_take(pf_batch* b, uint64_t len, uint64_t* off) {
  for (auto it = b->free_ranges.begin(); it != b->free_ranges.end(); ++it) {
    if (it->second >= len) {
      *off = it->first;
      const uint64_t rest = it->second - len, roff = it->first + len;
      b->free_ranges.erase(it);
      if (rest) b->free_ranges[roff] = rest;
      return true;
    }
  }
  return false;
}

void pool_give(pf_batch* b, uint64_t off, uint64_t len) {
  auto it = b->free_ranges.emplace(off, len).first;
  auto nx = std::next(it);
  if (nx != b->free_ranges.end() && it->first + it->second == nx->first) {
    it->second += nx->second;
    b->free_ranges.erase(nx);
  }
  if (it != b->free_ranges.begin()) {
    auto pv = std::prev(it);
    if (pv->first + pv->second == it->first) {
      pv->second += it->second;
      b->free_ranges.erase(it);
    }
  }
}

bool larger_first(const pf_batch* b, uint32_t a, uint32_t c) {
  if (b->Fh[a].n != b->Fh[c].n) return b->Fh[a].n > b->Fh[c].n;
  return a < c;
}

// Reserve the lowest free slot and a pool range for one filter and record it
// on the host; false (nothing changed) when either is missing.
bool batch_reserve(pf_batch* b, const pf_config& c, uint32_t* slot_out) {
  if (b->free_slots.empty()) {
    set_err(PF_ERR_BUSY, "no free slot (%u of %u in use)", b->resident, b->max_filters);
    return false;
  }
  const uint64_t len = round_pool(c.n_particles);
  uint64_t off = 0;
  if (!pool_take(b, len, &off)) {
    set_err(PF_ERR_BUSY, "particle pool full: %llu particles requested, %llu of %llu in use",
            (unsigned long long)c.n_particles, (unsigned long long)b->used,
            (unsigned long long)b->pool);
    return false;
  }
  const uint32_t slot = *b->free_slots.begin();
  b->free_slots.erase(b->free_slots.begin());
  BatchFilter f;
  std::memset(&f, 0, sizeof(f));
  f.off = off;
  f.seed = c.seed;
  f.n = (uint32_t)c.n_particles;
  f.filter_id = c.filter_id;
  f.k = cdf_shift(c.n_particles);
  f.learn = c.known_variances ? 0u : 1u;
  f.x0_mean = c.x0_mean; f.x0_var = c.x0_var;
  f.a_sigma = c.a_sigma; f.b_sigma = c.b_sigma;
  f.a_tau = c.a_tau; f.b_tau = c.b_tau;
  f.sigma2 = c.sigma2; f.tau2 = c.tau2;
  f.ess_frac = c.ess_frac;
  f.slam = (double)c.n_particles;  // sum of exp(lambda_i) with lambda = 0
  b->Fh[slot] = f;
  b->used += len;
  b->resident++;
  b->order.insert(std::lower_bound(b->order.begin(), b->order.end(), slot,
                                   [&](uint32_t a2, uint32_t c2) { return larger_first(b, a2, c2); }),
                  slot);
  *slot_out = slot;
  return true;
}

// Undo batch_reserve (host bookkeeping only; device work enqueued later on
// the batch's stream is what reuses the range).
void batch_release(pf_batch* b, uint32_t slot) {
  const uint64_t len = round_pool(b->Fh[slot].n);
  pool_give(b, b->Fh[slot].off, len);
  b->used -= len;
  b->resident--;
  b->order.erase(std::find(b->order.begin(), b->order.end(), slot));
  std::memset(&b->Fh[slot], 0, sizeof(BatchFilter));
  b->free_slots.insert(slot);
}

// One admission list for the reserved slots: their records and one init
// launch.  Waits only for the copy made from the same staging buffer
// pf_batch::kAdm admissions ago.
pf_status batch_init_slots(pf_batch* b, const uint32_t* slots, uint32_t cnt) {
  if (cnt == 0) return PF_OK;
  const uint32_t ar = b->adm_ring;
  CK(cudaEventSynchronize(b->adm_ev[ar]));
  BatchInit* inits = (BatchInit*)(b->adm_pin[ar] + 16);
  for (uint32_t i = 0; i < cnt; ++i) {
    std::memset(&inits[i], 0, sizeof(BatchInit));
    inits[i].slot = slots[i];
    inits[i].rec = b->Fh[slots[i]];
  }
  *(uint32_t*)b->adm_pin[ar] = cnt;
  CK(cudaMemcpyAsync(b->adm_dev[ar], b->adm_pin[ar], 16 + (size_t)cnt * sizeof(BatchInit),
                     cudaMemcpyHostToDevice, b->stream));
  CK(cudaEventRecord(b->adm_ev[ar], b->stream));
  b->adm_ring = (ar + 1) % pf_batch::kAdm;
  const unsigned grid = (unsigned)std::min<uint64_t>(cnt, 4096);
  if (b->fp64) {
    BatchArgs<double> a = batch_args<double>(b);
    a.count = (const uint32_t*)b->adm_dev[ar];
    a.inits = (const BatchInit*)(b->adm_dev[ar] + 16);
    CK(batch_init_launch<double>(grid, a, b->stream));
  } else {
    BatchArgs<float> a = batch_args<float>(b);
    a.count = (const uint32_t*)b->adm_dev[ar];
    a.inits = (const BatchInit*)(b->adm_dev[ar] + 16);
    CK(batch_init_launch<float>(grid, a, b->stream));
  }
  CK(cudaGetLastError());
  return PF_OK;
}

// Admit the filters cfgs[0..cnt) into free slots and enqueue their
// initialisation.  All or nothing: on PF_ERR_BUSY nothing is admitted.
pf_status batch_admit(pf_batch* b, const pf_config* cfgs, uint32_t cnt, uint32_t* slots) {
  for (uint32_t i = 0; i < cnt; ++i) {
    pf_status st = validate_member(b, &cfgs[i]);
    if (st != PF_OK) return st;
  }
  std::vector<uint32_t> got;
  got.reserve(cnt);
  for (uint32_t i = 0; i < cnt; ++i) {
    uint32_t slot = 0;
    if (!batch_reserve(b, cfgs[i], &slot)) {
      for (uint32_t s2 : got) batch_release(b, s2);
      return PF_ERR_BUSY;
    }
    got.push_back(slot);
  }
  if (slots) std::copy(got.begin(), got.end(), slots);
  return batch_init_slots(b, got.data(), cnt);
}

pf_status batch_build_graphs(pf_batch* b) {
  for (int r = 0; r < pf_batch::kRing; ++r) {
    if (b->exec[r]) {
      cudaGraphExecDestroy(b->exec[r]);
      b->exec[r] = nullptr;
    }
    CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    pf_status st = launch_batch_cycle(b, b->list_dev[r], 1, b->stream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (st != PF_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return set_err(PF_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->exec[r], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return set_err(PF_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  }
  return PF_OK;
}

}  // namespace

extern "C" {

pf_status pf_batch_create(const pf_config* cfgs, uint32_t n, const pf_batch_opts* opts,
                          pf_batch** out) {
  if (!out) return set_err(PF_ERR_INVALID, "NULL output");
  *out = nullptr;
  if (!opts) return set_err(PF_ERR_INVALID, "NULL options");
  if (n && !cfgs) return set_err(PF_ERR_INVALID, "NULL filter configurations");
  if (opts->scheme < 0 || opts->scheme > 3) return set_err(PF_ERR_INVALID, "bad scheme");
  if (opts->precision != PF_FP32 && opts->precision != PF_FP64) return set_err(PF_ERR_INVALID, "bad precision");
  const uint32_t maxf = opts->max_filters ? opts->max_filters : n;
  if (maxf < 1 || maxf < n || maxf > (1u << 24))
    return set_err(PF_ERR_INVALID, "max_filters must be in [max(n, 1), 2^24]");
  if ((opts->alloc == nullptr) != (opts->free == nullptr))
    return set_err(PF_ERR_INVALID, "alloc and free must both be set or both NULL");
  pf_batch* b = new (std::nothrow) pf_batch();
  if (!b) return set_err(PF_ERR_OOM, "host allocation failed");
  b->scheme = opts->scheme;
  b->pos = is_multinomial(opts->scheme) ? POS_MULTINOMIAL : POS_SYSTEMATIC;
  b->fp64 = opts->precision == PF_FP64;
  b->adaptive = opts->adaptive != 0;
  b->alloc = opts->alloc;
  b->free = opts->free;
  b->alloc_ctx = opts->alloc_ctx;
  b->max_filters = maxf;
  b->bytes_per_particle = batch_bytes_per_particle(b->fp64, b->pos == POS_MULTINOMIAL, b->adaptive);
  auto bail = [&](pf_status s) {
    pf_batch_destroy(b);
    return s;
  };
  // validate the initial filters before allocating anything
  for (uint32_t i = 0; i < n; ++i) {
    pf_status st = validate_member(b, &cfgs[i]);
    if (st != PF_OK) {
      delete b;
      return st;
    }
  }
  uint64_t need = 0;
  for (uint32_t i = 0; i < n; ++i) need += round_pool(cfgs[i].n_particles);
  uint64_t pool = need;
  if (opts->hbm_budget_bytes) {
    pool = opts->hbm_budget_bytes / b->bytes_per_particle / kPoolAlign * kPoolAlign;
    if (pool < need) {
      delete b;
      return set_err(PF_ERR_BUSY, "budget of %llu bytes holds %llu particles, the initial filters need %llu",
                     (unsigned long long)opts->hbm_budget_bytes, (unsigned long long)pool,
                     (unsigned long long)need);
    }
  }
  if (pool == 0) pool = kPoolAlign;
  b->pool = pool;
  if (opts->stream) {
    b->stream = (cudaStream_t)opts->stream;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete b;
      return set_err(PF_ERR_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
    }
    b->own_stream = true;
  }
  pf_status st;
  const size_t rs = b->fp64 ? 8 : 4;
  for (int p = 0; p < 2; ++p) {
    if ((st = batch_alloc(b, pool * rs, &b->x[p])) != PF_OK) return bail(st);
    if ((st = batch_alloc(b, pool * rs, &b->s2[p])) != PF_OK) return bail(st);
    if ((st = batch_alloc(b, pool * rs, &b->t2[p])) != PF_OK) return bail(st);
    if ((st = batch_alloc(b, pool * 8, &b->bs[p])) != PF_OK) return bail(st);
    if ((st = batch_alloc(b, pool * 8, &b->bt[p])) != PF_OK) return bail(st);
  }
  if ((st = batch_alloc(b, pool * rs, &b->ell)) != PF_OK) return bail(st);
  if (b->adaptive && (st = batch_alloc(b, pool * rs, &b->lam)) != PF_OK) return bail(st);
  if ((st = batch_alloc(b, pool * 8, (void**)&b->Q)) != PF_OK) return bail(st);
  if (b->pos == POS_MULTINOMIAL && (st = batch_alloc(b, pool * 8, (void**)&b->S)) != PF_OK) return bail(st);
  if ((st = batch_alloc(b, pool * 4, (void**)&b->anc)) != PF_OK) return bail(st);
  if ((st = batch_alloc(b, (size_t)maxf * sizeof(BatchFilter), (void**)&b->F)) != PF_OK) return bail(st);
  if ((st = batch_alloc(b, 256, (void**)&b->ctr)) != PF_OK) return bail(st);
  if ((st = batch_alloc(b, (size_t)maxf * BATCH_EST_ROW * 8, (void**)&b->est_dev)) != PF_OK) return bail(st);
  for (int r = 0; r <= pf_batch::kRing; ++r) {
    if ((st = batch_alloc(b, list_bytes(maxf), (void**)&b->list_dev[r])) != PF_OK) return bail(st);
    if (cudaHostAlloc((void**)&b->list_pin[r], list_bytes(maxf), cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      return bail(set_err(PF_ERR_OOM, "pinned host allocation failed"));
    }
  }
  if (cudaHostAlloc((void**)&b->est_pin, (size_t)maxf * BATCH_EST_ROW * 8, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    return bail(set_err(PF_ERR_OOM, "pinned host allocation failed"));
  }
  for (int r = 0; r < pf_batch::kRing; ++r)
    if (cudaEventCreateWithFlags(&b->list_ev[r], cudaEventDisableTiming) != cudaSuccess)
      return bail(set_err(PF_ERR_CUDA, "cudaEventCreate failed"));
  for (int r = 0; r < pf_batch::kAdm; ++r) {
    const size_t ab = 16 + (size_t)maxf * sizeof(BatchInit);
    if ((st = batch_alloc(b, ab, (void**)&b->adm_dev[r])) != PF_OK) return bail(st);
    if (cudaHostAlloc((void**)&b->adm_pin[r], ab, cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      return bail(set_err(PF_ERR_OOM, "pinned host allocation failed"));
    }
    if (cudaEventCreateWithFlags(&b->adm_ev[r], cudaEventDisableTiming) != cudaSuccess)
      return bail(set_err(PF_ERR_CUDA, "cudaEventCreate failed"));
  }
  if (cudaMemsetAsync(b->ctr, 0, 256, b->stream) != cudaSuccess ||
      cudaMemsetAsync(b->F, 0, (size_t)maxf * sizeof(BatchFilter), b->stream) != cudaSuccess)
    return bail(set_err(PF_ERR_CUDA, "batch memset failed"));
  b->Fh.assign(maxf, BatchFilter());
  std::memset(b->Fh.data(), 0, (size_t)maxf * sizeof(BatchFilter));
  b->free_ranges[0] = pool;
  for (uint32_t i = 0; i < maxf; ++i) b->free_slots.insert(b->free_slots.end(), i);
  b->autotune = opts->autotune != 0;
  if ((st = batch_shapes(b)) != PF_OK) return bail(st);
  if ((b->fp64 ? batch_prepare<double>() : batch_prepare<float>()) != cudaSuccess)
    return bail(set_err(PF_ERR_CUDA, "loading the batch kernels failed"));
  if (n && (st = batch_admit(b, cfgs, n, nullptr)) != PF_OK) return bail(st);
  if ((st = batch_build_graphs(b)) != PF_OK) return bail(st);
  *out = b;
  return PF_OK;
}

pf_status pf_batch_add(pf_batch* b, const pf_config* cfg, uint32_t* slot) {
  pf_status st = check_batch(b);
  if (st != PF_OK) return st;
  if (!cfg || !slot) return set_err(PF_ERR_INVALID, "NULL argument");
  st = batch_admit(b, cfg, 1, slot);
  return batch_fail(b, st);
}

pf_status pf_batch_remove(pf_batch* b, uint32_t slot) {
  pf_status st = check_batch(b);
  if (st != PF_OK) return st;
  if (slot >= b->max_filters || b->Fh[slot].n == 0) return set_err(PF_ERR_INVALID, "slot %u is not in use", slot);
  // the slot's range is reused only by later work on the same stream
  batch_release(b, slot);
  return PF_OK;
}

}  // extern "C"

namespace {

// Fill work list r (pinned) with the selected resident filters, largest
// first, and copy it to the device.  Returns the number of items.
pf_status stage_cycle_list(pf_batch* b, uint32_t r, const double* y, const uint8_t* mask,
                           uint32_t* cnt_out) {
  CK(cudaEventSynchronize(b->list_ev[r]));  // the list copied from this buffer has left
  BatchItem* items = (BatchItem*)(b->list_pin[r] + 16);
  uint32_t cnt = 0;
  for (uint32_t s : b->order) {
    if (mask && !mask[s]) continue;
    items[cnt].slot = s;
    items[cnt].pad = 0;
    items[cnt].y = y[s];
    ++cnt;
  }
  *cnt_out = cnt;
  if (cnt == 0) return PF_OK;
  ((uint32_t*)b->list_pin[r])[0] = cnt;
  ((uint32_t*)b->list_pin[r])[1] = big_items(b, items, cnt);
  CK(cudaMemcpyAsync(b->list_dev[r], b->list_pin[r], 16 + (size_t)cnt * sizeof(BatchItem),
                     cudaMemcpyHostToDevice, b->stream));
  CK(cudaEventRecord(b->list_ev[r], b->stream));
  return PF_OK;
}

// Time every candidate launch shape on trial cycles of list r (which commit
// nothing: t, log-ML and the error words stay as they are, and the next real
// cycle rewrites everything else the trials wrote), keep the fastest and
// re-capture the cycle graphs with it.
pf_status batch_tune_list(pf_batch* b, uint32_t r, pf_batch_tuning* out) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const int reps = 2;
  float best = 0.0f;
  size_t best_i = 0;
  pf_status st = PF_OK;
  std::vector<float> ms(b->shapes.size(), 0.0f);
  // the list's large-item count depends on the shape: rewrite it per shape
  BatchItem* items = (BatchItem*)(b->list_pin[r] + 16);
  const uint32_t cnt = ((uint32_t*)b->list_pin[r])[0];
  for (size_t i = 0; i < b->shapes.size() && st == PF_OK; ++i) {
    b->nt = b->shapes[i].nt;
    b->grid = b->shapes[i].grid;
    b->cl = b->shapes[i].cl;
    b->big_min = b->shapes[i].big_min;
    if (i > 0) {
      CK(cudaEventSynchronize(b->list_ev[r]));
      ((uint32_t*)b->list_pin[r])[1] = big_items(b, items, cnt);
      CK(cudaMemcpyAsync(b->list_dev[r], b->list_pin[r], 16, cudaMemcpyHostToDevice, b->stream));
      CK(cudaEventRecord(b->list_ev[r], b->stream));
    }
    st = launch_batch_cycle(b, b->list_dev[r], 0, b->stream);  // warm-up
    if (st == PF_OK) cudaEventRecord(e0, b->stream);
    for (int k = 0; k < reps && st == PF_OK; ++k) st = launch_batch_cycle(b, b->list_dev[r], 0, b->stream);
    if (st != PF_OK) break;
    cudaEventRecord(e1, b->stream);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      st = set_err(PF_ERR_CUDA, "tuning: %s", cudaGetErrorString(e));
      break;
    }
    cudaEventElapsedTime(&ms[i], e0, e1);
    ms[i] /= reps;
    if (i == 0 || ms[i] < best) {
      best = ms[i];
      best_i = i;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != PF_OK) return st;
  b->nt = b->shapes[best_i].nt;
  b->grid = b->shapes[best_i].grid;
  b->cl = b->shapes[best_i].cl;
  b->big_min = b->shapes[best_i].big_min;
  b->tuned = true;
  // the staged list is about to run with the kept shape
  CK(cudaEventSynchronize(b->list_ev[r]));
  ((uint32_t*)b->list_pin[r])[1] = big_items(b, items, cnt);
  CK(cudaMemcpyAsync(b->list_dev[r], b->list_pin[r], 16, cudaMemcpyHostToDevice, b->stream));
  CK(cudaEventRecord(b->list_ev[r], b->stream));
  if (out) {
    std::memset(out, 0, sizeof(*out));
    const size_t m = std::min<size_t>(b->shapes.size(), PF_BATCH_MAX_SHAPES);
    out->n_shapes = (uint32_t)m;
    for (size_t i = 0; i < m; ++i) {
      out->block[i] = (uint32_t)b->shapes[i].nt;
      out->grid[i] = b->shapes[i].grid;
      out->cluster[i] = (uint32_t)b->shapes[i].cl;
      out->big_min[i] = b->shapes[i].big_min;
      out->ms[i] = ms[i];
    }
    out->chosen = (uint32_t)best_i;
  }
  return batch_build_graphs(b);
}

}  // namespace

extern "C" {

pf_status pf_batch_tune(pf_batch* b, const double* y, const uint8_t* mask, pf_batch_tuning* out) {
  pf_status st = check_batch(b);
  if (st != PF_OK) return st;
  if (!y) return set_err(PF_ERR_INVALID, "NULL observations");
  const uint32_t r = b->ring;
  uint32_t cnt = 0;
  if ((st = stage_cycle_list(b, r, y, mask, &cnt)) != PF_OK) return batch_fail(b, st);
  if (cnt == 0) return set_err(PF_ERR_INVALID, "no filter selected");
  b->ring = (r + 1) % pf_batch::kRing;
  return batch_fail(b, batch_tune_list(b, r, out));
}

pf_status pf_batch_set_shape(pf_batch* b, uint32_t block, uint32_t grid, uint32_t cluster,
                             uint32_t big_min) {
  pf_status st = check_batch(b);
  if (st != PF_OK) return st;
  if (cluster == 0) cluster = 1;
  const pf_batch::Shape* fit = nullptr;
  for (auto& sh : b->shapes)
    if (sh.nt == (int)block && sh.cl == (int)cluster && (!fit || sh.grid > fit->grid)) fit = &sh;
  if (!fit)
    return set_err(PF_ERR_INVALID, "unsupported shape: block %u, cluster %u (256 or 512 threads "
                   "without clusters, 256 threads with clusters of 2, 4 or 8)", block, cluster);
  if (grid < cluster || grid > fit->grid || grid % cluster != 0)
    return set_err(PF_ERR_INVALID, "grid must be a multiple of %u in [%u, %u]", cluster, cluster, fit->grid);
  CK(cudaStreamSynchronize(b->stream));
  b->nt = (int)block;
  b->grid = grid;
  b->cl = (int)cluster;
  b->big_min = cluster > 1 ? big_min : 0;
  b->tuned = true;
  return batch_fail(b, batch_build_graphs(b));
}

pf_status pf_batch_step(pf_batch* b, const double* y, const uint8_t* mask) {
  pf_status st = check_batch(b);
  if (st != PF_OK) return st;
  if (!y) return set_err(PF_ERR_INVALID, "NULL observations");
  const uint32_t r = b->ring;
  uint32_t cnt = 0;
  if ((st = stage_cycle_list(b, r, y, mask, &cnt)) != PF_OK) return batch_fail(b, st);
  if (cnt == 0) return PF_OK;
  if (b->autotune && !b->tuned && (st = batch_tune_list(b, r, nullptr)) != PF_OK) return batch_fail(b, st);
  cudaError_t e = cudaGraphLaunch(b->exec[r], b->stream);
  if (e != cudaSuccess) {
    b->sticky = PF_ERR_CUDA;
    return set_err(PF_ERR_CUDA, "batch step: %s", cudaGetErrorString(e));
  }
  b->ring = (r + 1) % pf_batch::kRing;
  b->cycles++;
  return PF_OK;
}

pf_status pf_batch_sync(pf_batch* b) {
  pf_status st = check_batch(b);
  if (st != PF_OK) return st;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    b->sticky = PF_ERR_CUDA;
    return set_err(PF_ERR_CUDA, "stream: %s", cudaGetErrorString(e));
  }
  return PF_OK;
}

pf_status pf_batch_estimate(pf_batch* b, const uint8_t* mask, pf_estimates* out) {
  pf_status st = check_batch(b);
  if (st != PF_OK) return st;
  if (!out) return set_err(PF_ERR_INVALID, "NULL output");
  char* lp = b->list_pin[pf_batch::kRing];
  BatchItem* items = (BatchItem*)(lp + 16);
  uint32_t cnt = 0;
  for (uint32_t s : b->order) {
    if (mask && !mask[s]) continue;
    items[cnt].slot = s;
    items[cnt].pad = 0;
    items[cnt].y = 0.0;
    ++cnt;
  }
  if (cnt == 0) return pf_batch_sync(b);
  *(uint32_t*)lp = cnt;
  CK(cudaMemcpyAsync(b->list_dev[pf_batch::kRing], lp, 16 + (size_t)cnt * sizeof(BatchItem),
                     cudaMemcpyHostToDevice, b->stream));
  const unsigned grid = (unsigned)std::min<uint64_t>(cnt, b->grid);
  cudaError_t e;
  if (b->fp64) {
    BatchArgs<double> a = batch_args<double>(b);
    set_list(a, b->list_dev[pf_batch::kRing]);
    e = batch_estimate_launch<double>(grid, a, b->stream);
  } else {
    BatchArgs<float> a = batch_args<float>(b);
    set_list(a, b->list_dev[pf_batch::kRing]);
    e = batch_estimate_launch<float>(grid, a, b->stream);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->est_pin, b->est_dev, (size_t)cnt * BATCH_EST_ROW * 8, cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    b->sticky = PF_ERR_CUDA;
    return set_err(PF_ERR_CUDA, "batch estimate: %s", cudaGetErrorString(e));
  }
  pf_status worst = PF_OK;
  for (uint32_t i = 0; i < cnt; ++i) {
    const double* v = b->est_pin + (size_t)i * BATCH_EST_ROW;
    pf_estimates& o = out[items[i].slot];
    o.t = (uint64_t)v[0];
    o.x_mean = v[1];
    o.x_var = v[2];
    o.sigma2_mean = v[3];
    o.sigma2_var = v[4];
    o.tau2_mean = v[5];
    o.tau2_var = v[6];
    o.log_marglik = v[7];
    const uint32_t err = (uint32_t)v[8];
    if (err && worst == PF_OK) {
      worst = map_err(err);
      set_err(worst, "filter in slot %u: %s", items[i].slot, pf_last_error());
    }
  }
  return worst;
}

pf_status pf_batch_get_particles(pf_batch* b, uint32_t slot, void* x, void* sigma2, void* tau2,
                                 void* b_sigma, void* b_tau) {
  pf_status st = check_batch(b);
  if (st != PF_OK) return st;
  if (slot >= b->max_filters || b->Fh[slot].n == 0) return set_err(PF_ERR_INVALID, "slot %u is not in use", slot);
  BatchFilter f;
  CK(cudaMemcpyAsync(&f, b->F + slot, sizeof(f), cudaMemcpyDeviceToHost, b->stream));
  CK(cudaStreamSynchronize(b->stream));
  const int p = (int)(f.t & 1);
  const size_t rs = b->fp64 ? 8 : 4;
  void* dst[5] = {x, sigma2, tau2, b_sigma, b_tau};
  char* src[5] = {(char*)b->x[p], (char*)b->s2[p], (char*)b->t2[p], (char*)b->bs[p], (char*)b->bt[p]};
  const size_t sz[5] = {rs, rs, rs, 8, 8};
  for (int i = 0; i < 5; ++i)
    if (dst[i]) CK(cudaMemcpyAsync(dst[i], src[i] + f.off * sz[i], (size_t)f.n * sz[i], cudaMemcpyDefault, b->stream));
  CK(cudaStreamSynchronize(b->stream));
  return PF_OK;
}

pf_status pf_batch_get_ancestors(pf_batch* b, uint32_t slot, uint32_t* anc, uint64_t* Q) {
  pf_status st = check_batch(b);
  if (st != PF_OK) return st;
  if (slot >= b->max_filters || b->Fh[slot].n == 0) return set_err(PF_ERR_INVALID, "slot %u is not in use", slot);
  const BatchFilter& f = b->Fh[slot];
  if (anc) CK(cudaMemcpyAsync(anc, b->anc + f.off, (size_t)f.n * 4, cudaMemcpyDefault, b->stream));
  if (Q) CK(cudaMemcpyAsync(Q, b->Q + f.off, (size_t)f.n * 8, cudaMemcpyDefault, b->stream));
  CK(cudaStreamSynchronize(b->stream));
  return PF_OK;
}

pf_status pf_batch_get_info(pf_batch* b, pf_batch_info* out) {
  if (!b || !out) return set_err(PF_ERR_INVALID, "NULL argument");
  out->max_filters = b->max_filters;
  out->resident = b->resident;
  out->pool_particles = b->pool;
  out->used_particles = b->used;
  out->bytes_per_particle = b->bytes_per_particle;
  out->pool_bytes = b->pool * b->bytes_per_particle;
  out->grid = b->grid;
  out->block = (uint32_t)b->nt;
  out->cluster = (uint32_t)b->cl;
  out->big_min = b->big_min;
  out->tuned = b->tuned ? 1u : 0u;
  out->cycles = b->cycles;
  return PF_OK;
}

pf_status pf_batch_destroy(pf_batch* b) {
  if (!b) return PF_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (int r = 0; r < pf_batch::kRing; ++r) {
    if (b->exec[r]) cudaGraphExecDestroy(b->exec[r]);
    if (b->list_ev[r]) cudaEventDestroy(b->list_ev[r]);
  }
  for (void* p : b->allocs) {
    if (b->alloc && b->free) b->free(p, b->stream, b->alloc_ctx);
    else if (!b->alloc) cudaFreeAsync(p, b->stream);
  }
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (int r = 0; r <= pf_batch::kRing; ++r)
    if (b->list_pin[r]) cudaFreeHost(b->list_pin[r]);
  for (int r = 0; r < pf_batch::kAdm; ++r) {
    if (b->adm_pin[r]) cudaFreeHost(b->adm_pin[r]);
    if (b->adm_ev[r]) cudaEventDestroy(b->adm_ev[r]);
  }
  if (b->est_pin) cudaFreeHost(b->est_pin);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  cudaGetLastError();
  delete b;
  return PF_OK;
}

}  // extern "C"
