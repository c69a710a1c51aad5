// C ABI of the particle-learning library (declared in include/pf.h).
//
// Host logic only: argument checks, device allocation, launch configuration,
// CUDA-graph capture of one cycle, the observation ring, and error mapping.
// Every step of the method runs in the kernels of kernels.cuh.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <chrono>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/pf.h"
#include "../../include/pf_diag.h"
#include "kernels.cuh"

using namespace pfk;

namespace {

thread_local char g_err[512] = "";

pf_status set_err(pf_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return set_err(PF_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));     \
  } while (0)

inline uint64_t cdiv(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

int cdf_shift(uint64_t n) {
  int c = 0;
  while ((1ull << c) < n) ++c;
  return 61 - c;
}

pf_status map_err(uint32_t err) {
  if (err & ERR_TIMEOUT) return set_err(PF_ERR_TIMEOUT, "device look-back wait timed out");
  if (err & ERR_WEIGHTS) return set_err(PF_ERR_NUMERIC, "weights negative, non-finite or all zero");
  if (err & ERR_NUMERIC)
    return set_err(PF_ERR_NUMERIC, "non-finite likelihood, empty CDF or gamma sampler failure");
  return PF_OK;
}

}  // namespace

// Forms of a captured cycle.  A cycle either runs the weights kernel or finds
// its weights computed by the previous cycle's propagation; its propagation
// either stops there or also computes the next cycle's weights.
enum CycleForm : int {
  CF_PLAIN = 0,  // weights, CDF, resampling, propagation
  CF_HEAD = 1,   // weights, CDF, resampling, propagation + next weights
  CF_MID = 2,    // CDF, resampling, propagation + next weights
  CF_TAIL = 3,   // CDF, resampling, propagation
  CF_EST = 4,    // CF_PLAIN, then the summaries and their copy to the host mirror
  CF_COUNT = 5
};
inline bool form_weighs(int form) { return form == CF_PLAIN || form == CF_HEAD || form == CF_EST; }
inline bool form_fuses(int form) { return form == CF_HEAD || form == CF_MID; }

// One captured cycle, with the kernel nodes whose observation arguments each
// launch sets: the weights node (this cycle's y) and the fused propagation
// node (the next cycle's y).
struct CycleGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t wnode = nullptr, pnode = nullptr;
  cudaKernelNodeParams wparams = {}, pparams = {};
  alignas(16) unsigned char wargs[sizeof(FilterArgs<double>)] = {};
  alignas(16) unsigned char pargs[sizeof(FilterArgs<double>)] = {};
  void* wkp[1] = {};
  void* pkp[1] = {};
};

struct pf_filter {
  pf_config cfg;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // multinomial schemes: the exponential spacings need nothing from the
  // cycle's weights or CDF, so they are scanned on a second stream, forked
  // from and joined back into the filter's stream (a parallel branch of the
  // captured graph)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  uint64_t n = 0;
  int k = 0;
  uint32_t ntiles = 0;
  bool fp64 = false, learn = true;
  int scheme = 0;
  unsigned prop_grid = 0;  // persistent propagate grid
  uint64_t w_cap = 1;      // resident CTAs of the weights kernel
  unsigned prop_grid_fuse = 0;  // the same for the propagation that also weighs
  unsigned cdf_grid = 0;   // cooperative CDF + systematic resampling grid (0: not used)
  bool cdf_staged = false; // its CTAs own several tiles: TMA-staged variant
  int cdf_per = 16;         // particles per thread of its tiles (8: 2048-particle tiles)
  bool bootstrap = false;   // Algorithm "Particle Filtering" instead of particle learning
  uint32_t nparts = 0;      // log-ML partials per cycle
  uint64_t* cta_tot = nullptr;
  U128* cta_sq = nullptr;  // adaptive resampling: per-CTA sums of W^2 of the cooperative kernel
  std::vector<void*> allocs;
  void* x[2] = {}; void* s2[2] = {}; void* t2[2] = {}; void* bs[2] = {}; void* bt[2] = {};
  void* ell = nullptr;
  // adaptive resampling (cfg.ess_frac > 0): carried log-weights, the grid of
  // the decision kernel and its per-block partial sums
  bool ess = false;
  void* lam = nullptr;
  unsigned ess_grid = 0;
  U128* ess_part = nullptr;
  uint64_t* Q = nullptr;
  uint64_t* S = nullptr;
  uint32_t* anc = nullptr;
  uint32_t* I = nullptr;
  uint64_t* splits = nullptr;  // merge-path partition
  uint64_t* stat_w[2] = {};
  uint64_t* stat_e[2] = {};
  void* part = nullptr;
  double* part_est = nullptr;
  Ctl* ctl = nullptr;
  Ctl* ctl_host = nullptr;  // pinned mirror for summaries
  Ctl* ctl_host_dev = nullptr;  // its device address (mapped), or NULL
  // pf_step_estimate: the observation and a sequence number in mapped host
  // memory (no graph-node update per call), the summary kernel's copy of the
  // number marking the summaries complete (no stream synchronisation)
  EstIO* io = nullptr;
  EstIO* io_dev = nullptr;
  uint64_t io_seq = 0;
  // captured cycles by CycleForm (the fused forms on first use); each launch
  // sets its observations in the kernel nodes' arguments (no copy on the stream)
  CycleGraph cg[CF_COUNT];
  // the previous cycle computed this cycle's weights for the observation
  // ahead_y, announced by pf_step_ahead
  bool ahead = false;
  double ahead_y = 0.0;
  pf_status sticky = PF_OK;
};

namespace {

pf_status dev_alloc(pf_filter* f, size_t bytes, void** out) {
  bytes = (bytes + 255) & ~size_t(255);
  void* p = nullptr;
  if (f->cfg.alloc) {
    p = f->cfg.alloc(bytes, f->stream, f->cfg.alloc_ctx);
    if (!p) return set_err(PF_ERR_OOM, "allocator callback returned NULL for %zu bytes", bytes);
  } else {
    cudaError_t e = cudaMallocAsync(&p, bytes, f->stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return set_err(e == cudaErrorMemoryAllocation ? PF_ERR_OOM : PF_ERR_CUDA,
                     "cudaMallocAsync(%zu): %s", bytes, cudaGetErrorString(e));
    }
  }
  if (((uintptr_t)p & 15) != 0) return set_err(PF_ERR_INVALID, "allocator returned a pointer not 16-byte aligned");
  f->allocs.push_back(p);
  *out = p;
  return PF_OK;
}

void free_all(pf_filter* f) {
  for (void* p : f->allocs) {
    if (f->cfg.alloc && f->cfg.free) f->cfg.free(p, f->stream, f->cfg.alloc_ctx);
    else if (!f->cfg.alloc) cudaFreeAsync(p, f->stream);
  }
  f->allocs.clear();
}

template <class R>
FilterArgs<R> filter_args(pf_filter* f) {
  typedef typename SuffT<R>::B B;
  FilterArgs<R> a;
  for (int p = 0; p < 2; ++p) {
    a.st[p].x = (R*)f->x[p];
    a.st[p].s2 = (R*)f->s2[p];
    a.st[p].t2 = (R*)f->t2[p];
    a.st[p].bs = (B*)f->bs[p];
    a.st[p].bt = (B*)f->bt[p];
    a.stat_w[p] = f->stat_w[p];
    a.stat_e[p] = f->stat_e[p];
  }
  a.ell = (R*)f->ell;
  a.lam = (R*)f->lam;
  a.ess_frac = f->cfg.ess_frac;
  a.ess_part = f->ess_part;
  a.Q = f->Q;
  a.S = f->S;
  a.anc = f->anc;
  a.I = f->I;
  a.part = f->part;
  a.part_est = f->part_est;
  a.ctl = f->ctl;
  a.ctl_mirror = f->ctl_host_dev;
  a.io = nullptr;
  a.y_src = nullptr;
  a.y_val = 0.0;
  a.n = f->n;
  a.ntiles = f->ntiles;
  a.nparts = f->nparts;
  a.k = f->k;
  a.seed = f->cfg.seed;
  a.filter = f->cfg.filter_id;
  {
    // Philox4x32-10 round keys: the key words bumped by the Weyl constants
    uint32_t k0 = (uint32_t)f->cfg.seed, k1 = (uint32_t)(f->cfg.seed >> 32);
    for (int r = 0; r < 10; ++r) {
      a.rk[2 * r] = k0;
      a.rk[2 * r + 1] = k1;
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
  }
  a.x0_mean = f->cfg.x0_mean;
  a.x0_var = f->cfg.x0_var;
  a.a_sigma = f->cfg.a_sigma;
  a.b_sigma = f->cfg.b_sigma;
  a.a_tau = f->cfg.a_tau;
  a.b_tau = f->cfg.b_tau;
  a.sigma2 = f->cfg.sigma2;
  a.tau2 = f->cfg.tau2;
  return a;
}

// Optional per-kernel event timer (pf_step_profiled).
struct KTimer {
  static constexpr int MAX = 8;
  cudaEvent_t ev[MAX + 1];
  const char* names[MAX];
  int count = 0;
};
inline void mark(KTimer* tm, const char* name, cudaStream_t s) {
  if (!tm || tm->count >= KTimer::MAX) return;
  tm->names[tm->count] = name;
  cudaEventRecord(tm->ev[++tm->count], s);
}

bool is_multinomial(int scheme) { return scheme == PF_MULTINOMIAL || scheme == PF_MULTINOMIAL_CUTPOINT; }
bool is_cutpoint(int scheme) { return scheme == PF_MULTINOMIAL_CUTPOINT || scheme == PF_SYSTEMATIC_CUTPOINT; }

// Resampling kernels shared by the filter cycle and pf_resample: from a
// finished CDF Q (and spacing prefix S) to ancestors.
inline uint32_t merge_chunks(uint64_t n) { return (uint32_t)cdiv(2 * n, MERGE_D); }
inline uint32_t sys_chunks(uint64_t n) { return (uint32_t)cdiv(2 * n, SYS_D); }

pf_status launch_resample(int scheme, const PosArgs& pa, uint64_t n, uint32_t* I,
                          uint64_t* splits, cudaStream_t s, KTimer* tm = nullptr) {
  const bool multi = is_multinomial(scheme);
  if (scheme == PF_STRATIFIED) {
    k_strat<<<(unsigned)cdiv(n, BLOCK), BLOCK, 0, s>>>(pa);
    mark(tm, "stratified", s);
  } else if (!is_cutpoint(scheme) && multi) {
    const uint32_t chunks = merge_chunks(n);
    const unsigned pgrid = (unsigned)cdiv((uint64_t)(chunks + 1) * 32, BLOCK);
    k_partition<POS_MULTINOMIAL><<<pgrid, BLOCK, 0, s>>>(pa, splits, chunks + 1, MERGE_D);
    mark(tm, "partition", s);
    k_merge<POS_MULTINOMIAL><<<chunks, BLOCK, 0, s>>>(pa, splits);
    mark(tm, "merge", s);
  } else if (!is_cutpoint(scheme)) {
    const uint32_t chunks = sys_chunks(n);
    const unsigned pgrid = (unsigned)cdiv((uint64_t)(chunks + 1) * 32, BLOCK);
    k_partition<POS_SYSTEMATIC><<<pgrid, BLOCK, 0, s>>>(pa, splits, chunks + 1, SYS_D);
    mark(tm, "partition", s);
    k_merge_sys<<<chunks, SYS_THREADS, 0, s>>>(pa, splits);
    mark(tm, "merge", s);
  } else {
    const unsigned grid = (unsigned)cdiv(n, BLOCK);
    k_cutpoint_search<<<grid, BLOCK, 0, s>>>(pa.Q, n, I);
    mark(tm, "cutpoint_search", s);
    if (multi) k_cutpoint_method<POS_MULTINOMIAL><<<grid, BLOCK, 0, s>>>(pa);
    else k_cutpoint_method<POS_SYSTEMATIC><<<grid, BLOCK, 0, s>>>(pa);
    mark(tm, "cutpoint_method", s);
  }
  CK(cudaGetLastError());
  return PF_OK;
}

// One cycle (Steps 1-4), enqueued on f->stream; reads t and y on the device.
// With form CF_HEAD / CF_MID the propagation also computes the next cycle's
// weights against y_{t+2} (*ynx_src when set, else ynx_val); with CF_MID /
// CF_TAIL the weights kernel is left out, its work done by the previous cycle.
// The binary32 propagation with or without slots handed out by ticket.
template <bool LEARN, bool FUSE, bool ESS>
void launch_prop2(bool dyn, unsigned grid, cudaStream_t s, const FilterArgs<float>& a) {
  if (dyn) k_propagate2<LEARN, FUSE, ESS, true><<<grid, BLOCK, 0, s>>>(a);
  else k_propagate2<LEARN, FUSE, ESS, false><<<grid, BLOCK, 0, s>>>(a);
}
template <class R>
pf_status enqueue_cycle(pf_filter* f, KTimer* tm = nullptr, const double* y_src = nullptr,
                        double y_val = 0.0, int form = CF_PLAIN, const double* ynx_src = nullptr,
                        double ynx_val = 0.0) {
  cudaStream_t s = f->stream;
  FilterArgs<R> a = filter_args<R>(f);
  a.y_src = y_src;
  a.y_val = y_val;
  a.y_nx_src = ynx_src;
  a.y_nx_val = ynx_val;
  if (form == CF_EST && f->io_dev) {  // pf_step_estimate: y and completion through mapped words
    a.io = f->io_dev;
    a.y_src = &f->io_dev->y;
  }
  const uint64_t n = f->n;
  if (tm) cudaEventRecord(tm->ev[0], s);
  // multinomial: the spacing scan (Section 3.1's sorted uniforms) depends only
  // on the seed, the filter and t, so outside a timed cycle it runs on the
  // side stream beside the weights and the CDF scan
  const bool fork = is_multinomial(f->scheme) && !tm;
  auto spacing = [&](cudaStream_t on) {
    SpacingArgs sp;
    sp.S = f->S;
    sp.stat[0] = f->stat_e[0];
    sp.stat[1] = f->stat_e[1];
    sp.ctl = f->ctl;
    sp.t_dev = &f->ctl->t;
    sp.t_arg = 0;
    sp.n = n;
    sp.seed = f->cfg.seed;
    sp.filter = f->cfg.filter_id;
    k_spacing_scan<<<f->ntiles, BLOCK, 0, on>>>(sp);
  };
  if (fork) {
    CK(cudaEventRecord(f->ev_fork, s));
    CK(cudaStreamWaitEvent(f->side, f->ev_fork, 0));
    spacing(f->side);
    CK(cudaEventRecord(f->ev_join, f->side));
  }
  if (f->bootstrap) {  // Algorithm "Particle Filtering": propagate blind, then weigh
    k_boot_pw<R><<<(unsigned)cdiv(n, BLOCK), BLOCK, 0, s>>>(a);
    mark(tm, "propagate_weights", s);
  } else if (form_weighs(form)) {
    const unsigned wg = weights_grid<R>(n, f->w_cap);
    if (f->ess) k_weights<R, true><<<wg, BLOCK, 0, s>>>(a);
    else k_weights<R><<<wg, BLOCK, 0, s>>>(a);
    mark(tm, "weights", s);
  }
  ScanArgs sa;
  sa.src = f->ell;
  sa.Q = f->Q;
  sa.stat[0] = f->stat_w[0];
  sa.stat[1] = f->stat_w[1];
  sa.part = f->part;
  sa.ctl = f->ctl;
  sa.t_dev = &f->ctl->t;
  sa.t_arg = 0;
  sa.n = n;
  sa.k = f->k;
  sa.spin_limit = SPIN_LIMIT;
  sa.withhold = NO_TILE;
  sa.vec_ok = 1;
  if (!f->cdf_grid) {
    k_scan<FROM_LOGLIK, R><<<f->ntiles, BLOCK, 0, s>>>(sa);
    mark(tm, "scan", s);
  }
  if (f->ess && !f->cdf_grid) {  // adaptive resampling: the decision from the finished CDF
    k_ess<R><<<f->ess_grid, BLOCK, 0, s>>>(a);
    mark(tm, "ess", s);
  }
  if (fork) {
    CK(cudaStreamWaitEvent(s, f->ev_join, 0));
  } else if (is_multinomial(f->scheme)) {
    spacing(s);
    mark(tm, "spacing_scan", s);
  }
  PosArgs pa;
  pa.gate = f->ess ? &f->ctl->resamp : nullptr;
  pa.Q = f->Q;
  pa.S = f->S;
  pa.anc = f->anc;
  pa.I = f->I;
  pa.ctl = f->ctl;
  pa.t_dev = &f->ctl->t;
  pa.t_arg = 0;
  pa.n = n;
  pa.seed = f->cfg.seed;
  pa.filter = f->cfg.filter_id;
  if (f->cdf_grid) {
    // systematic: the CDF and the resampling in one cooperative launch
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(f->cdf_grid, 1, 1);
    cfg.blockDim = dim3(BLOCK, 1, 1);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    U128* const sq = f->cta_sq;
    if (f->cdf_staged) {
      if (f->ess) CK(cudaLaunchKernelEx(&cfg, k_cdf_sys<R, true, 16, true>, a, f->cta_tot, sq));
      else CK(cudaLaunchKernelEx(&cfg, k_cdf_sys<R, true, 16>, a, f->cta_tot, sq));
    } else if (f->cdf_per == 8) {
      if constexpr (sizeof(R) == 4) {
        if (f->ess) CK(cudaLaunchKernelEx(&cfg, k_cdf_sys<float, false, 8, true>, a, f->cta_tot, sq));
        else CK(cudaLaunchKernelEx(&cfg, k_cdf_sys<float, false, 8>, a, f->cta_tot, sq));
      }
    } else {
      if (f->ess) CK(cudaLaunchKernelEx(&cfg, k_cdf_sys<R, false, 16, true>, a, f->cta_tot, sq));
      else CK(cudaLaunchKernelEx(&cfg, k_cdf_sys<R, false, 16>, a, f->cta_tot, sq));
    }
    mark(tm, "cdf_resample", s);
  } else {
    pf_status st = launch_resample(f->scheme, pa, n, f->I, f->splits, s, tm);
    if (st != PF_OK) return st;
  }
  const bool fuse = !f->bootstrap && !f->ess && form_fuses(form);
  const unsigned pg = fuse ? f->prop_grid_fuse : f->prop_grid;
  // binary32: slots handed out by ticket when each warp has many 64-slot units
  const bool dyn = (n + 63) / 64 >= (uint64_t)PROP_DYN * pg * WARPS;
  if (f->bootstrap) {
    k_boot_gather<R><<<(unsigned)cdiv(n, BLOCK), BLOCK, 0, s>>>(a);
    mark(tm, "gather", s);
  } else if (f->ess) {  // adaptive resampling (never fused)
    if constexpr (sizeof(R) == 4) {
      if (f->learn) launch_prop2<true, false, true>(dyn, pg, s, a);
      else launch_prop2<false, false, true>(dyn, pg, s, a);
    } else {
      if (f->learn) k_propagate<R, true, false, true><<<pg, BLOCK, 0, s>>>(a);
      else k_propagate<R, false, false, true><<<pg, BLOCK, 0, s>>>(a);
    }
  } else if constexpr (sizeof(R) == 4) {  // binary32: two slots per thread, paired arithmetic
    if (f->learn) {
      if (fuse) launch_prop2<true, true, false>(dyn, pg, s, a);
      else launch_prop2<true, false, false>(dyn, pg, s, a);
    } else {
      if (fuse) launch_prop2<false, true, false>(dyn, pg, s, a);
      else launch_prop2<false, false, false>(dyn, pg, s, a);
    }
  } else {
    if (f->learn) {
      if (fuse) k_propagate<R, true, true><<<pg, BLOCK, 0, s>>>(a);
      else k_propagate<R, true><<<pg, BLOCK, 0, s>>>(a);
    } else {
      if (fuse) k_propagate<R, false, true><<<pg, BLOCK, 0, s>>>(a);
      else k_propagate<R, false><<<pg, BLOCK, 0, s>>>(a);
    }
  }
  mark(tm, fuse ? "propagate_weights_next" : "propagate", s);
  if (form == CF_EST) {  // the posterior summaries and their 104-byte copy to the pinned mirror
    const unsigned eg = (unsigned)cdiv(n, (uint64_t)BLOCK * EST_PER_THREAD);
    if (f->ess) k_estimate_w<R><<<eg, BLOCK, 0, s>>>(a);
    else k_estimate<R><<<eg, BLOCK, 0, s>>>(a);
    // the kernel writes the mapped mirror itself; otherwise a 104-byte copy
    if (!a.ctl_mirror)
      CK(cudaMemcpyAsync(f->ctl_host, f->ctl, offsetof(Ctl, y), cudaMemcpyDeviceToHost, s));
  }
  CK(cudaGetLastError());
  return PF_OK;
}

// The cooperative CDF + systematic resampling kernel of a configuration.
const void* cdf_fn(bool fp64, bool staged, int per, bool ess) {
  if (per == 8)
    return ess ? (const void*)k_cdf_sys<float, false, 8, true> : (const void*)k_cdf_sys<float, false, 8>;
  if (fp64) {
    if (staged)
      return ess ? (const void*)k_cdf_sys<double, true, 16, true> : (const void*)k_cdf_sys<double, true, 16>;
    return ess ? (const void*)k_cdf_sys<double, false, 16, true> : (const void*)k_cdf_sys<double, false, 16>;
  }
  if (staged)
    return ess ? (const void*)k_cdf_sys<float, true, 16, true> : (const void*)k_cdf_sys<float, true, 16>;
  return ess ? (const void*)k_cdf_sys<float, false, 16, true> : (const void*)k_cdf_sys<float, false, 16>;
}

// The propagation that also computes the next cycle's weights (binary32:
// the form with slots handed out by ticket when dyn).
const void* prop_fuse_fn(const pf_filter* f, bool dyn = false) {
  if (f->fp64)
    return f->learn ? (const void*)k_propagate<double, true, true>
                    : (const void*)k_propagate<double, false, true>;
  if (dyn)
    return f->learn ? (const void*)k_propagate2<true, true, false, true>
                    : (const void*)k_propagate2<false, true, false, true>;
  return f->learn ? (const void*)k_propagate2<true, true> : (const void*)k_propagate2<false, true>;
}

// Capture one cycle of the given form and find the nodes whose arguments
// carry observations.
pf_status build_graph(pf_filter* f, int form) {
  CycleGraph& G = f->cg[form];
  CK(cudaStreamBeginCapture(f->stream, cudaStreamCaptureModeThreadLocal));
  pf_status st = f->fp64 ? enqueue_cycle<double>(f, nullptr, nullptr, 0.0, form)
                         : enqueue_cycle<float>(f, nullptr, nullptr, 0.0, form);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(f->stream, &g);
  if (st != PF_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return set_err(PF_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
  G.graph = g;
  CK(cudaGraphInstantiate(&G.exec, g, 0));
  size_t nn = 0;
  CK(cudaGraphGetNodes(g, nullptr, &nn));
  std::vector<cudaGraphNode_t> nodes(nn);
  CK(cudaGraphGetNodes(g, nodes.data(), &nn));
  const void* wfun =
      f->bootstrap ? (f->fp64 ? (const void*)k_boot_pw<double> : (const void*)k_boot_pw<float>)
      : f->ess     ? (f->fp64 ? (const void*)k_weights<double, true> : (const void*)k_weights<float, true>)
                   : (f->fp64 ? (const void*)k_weights<double> : (const void*)k_weights<float>);
  const void* pfun = prop_fuse_fn(f);
  const void* pfun_dyn = prop_fuse_fn(f, true);
  const size_t asz = f->fp64 ? sizeof(FilterArgs<double>) : sizeof(FilterArgs<float>);
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType ty;
    CK(cudaGraphNodeGetType(nd, &ty));
    if (ty != cudaGraphNodeTypeKernel) continue;
    cudaKernelNodeParams p;
    CK(cudaGraphKernelNodeGetParams(nd, &p));
    if (p.func == wfun && !(form == CF_EST && f->io_dev)) {
      G.wnode = nd;
      G.wparams = p;
      std::memcpy(G.wargs, p.kernelParams[0], asz);
      G.wkp[0] = G.wargs;
      G.wparams.kernelParams = G.wkp;
      G.wparams.extra = nullptr;
    } else if (p.func == pfun || p.func == pfun_dyn) {
      G.pnode = nd;
      G.pparams = p;
      std::memcpy(G.pargs, p.kernelParams[0], asz);
      G.pkp[0] = G.pargs;
      G.pparams.kernelParams = G.pkp;
      G.pparams.extra = nullptr;
    }
  }
  if (form_weighs(form) && !G.wnode && !(form == CF_EST && f->io_dev))
    return set_err(PF_ERR_CUDA, "graph capture: weights node not found");
  if (form_fuses(form) && !f->bootstrap && !G.pnode)
    return set_err(PF_ERR_CUDA, "graph capture: fused propagation node not found");
  return PF_OK;
}

template <class R>
void set_obs(unsigned char* args, bool next, const double* src, double val) {
  FilterArgs<R>* a = reinterpret_cast<FilterArgs<R>*>(args);
  if (next) {
    a->y_nx_src = src;
    a->y_nx_val = val;
  } else {
    a->y_src = src;
    a->y_val = val;
  }
}

// One cycle of the given form: its graph (captured on first use), with this
// cycle's observation in the weights node and the next one in the fused
// propagation node.
pf_status launch_cycle(pf_filter* f, const double* y_src, double y_val, int form = CF_PLAIN,
                       const double* ynx_src = nullptr, double ynx_val = 0.0) {
  // the bootstrap filter's weights follow its own blind propagation;
  // adaptive resampling carries weights the fused propagation does not add
  if ((f->bootstrap || f->ess) && form != CF_EST) form = CF_PLAIN;
  CycleGraph& G = f->cg[form];
  if (!G.exec) {
    pf_status st = build_graph(f, form);
    if (st != PF_OK) return st;
  }
  auto setter = f->fp64 ? set_obs<double> : set_obs<float>;
  if (G.wnode) {
    setter(G.wargs, false, y_src, y_val);
    CK(cudaGraphExecKernelNodeSetParams(G.exec, G.wnode, &G.wparams));
  }
  if (G.pnode) {
    setter(G.pargs, true, ynx_src, ynx_val);
    CK(cudaGraphExecKernelNodeSetParams(G.exec, G.pnode, &G.pparams));
  }
  CK(cudaGraphLaunch(G.exec, f->stream));
  return PF_OK;
}

pf_status check_handle(pf_filter* f) {
  if (!f) return set_err(PF_ERR_INVALID, "NULL filter handle");
  if (f->sticky != PF_OK) return set_err(f->sticky, "filter is in a failed state (%d)", (int)f->sticky);
  return PF_OK;
}

pf_status sync_and_check(pf_filter* f) {
  // t, the error word, counters and the summaries: the fields before the
  // per-cycle constants (104 bytes)
  cudaError_t e = cudaMemcpyAsync(f->ctl_host, f->ctl, offsetof(Ctl, y), cudaMemcpyDeviceToHost, f->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(f->stream);
  if (e != cudaSuccess) {
    f->sticky = PF_ERR_CUDA;
    return set_err(PF_ERR_CUDA, "stream: %s", cudaGetErrorString(e));
  }
  pf_status st = map_err(f->ctl_host->err);
  if (st != PF_OK) f->sticky = st;
  return st;
}

}  // namespace

extern "C" {

const char* pf_last_error(void) { return g_err; }

pf_status pf_create(const pf_config* cfg, pf_filter** out) {
  if (!cfg || !out) return set_err(PF_ERR_INVALID, "NULL argument");
  *out = nullptr;
  if (cfg->n_particles < 1 || cfg->n_particles > PF_MAX_PARTICLES)
    return set_err(PF_ERR_INVALID, "n_particles must be in [1, 2^26]");
  if (cfg->scheme < 0 || cfg->scheme > 4) return set_err(PF_ERR_INVALID, "bad scheme");
  if (cfg->algorithm != PF_PARTICLE_LEARNING && cfg->algorithm != PF_BOOTSTRAP)
    return set_err(PF_ERR_INVALID, "bad algorithm");
  if (cfg->algorithm == PF_BOOTSTRAP && !cfg->known_variances)
    return set_err(PF_ERR_INVALID, "the bootstrap filter takes known variances");
  if (cfg->precision != PF_FP32 && cfg->precision != PF_FP64) return set_err(PF_ERR_INVALID, "bad precision");
  if (!cfg->known_variances && !(cfg->a_sigma >= 1.0 && cfg->a_tau >= 1.0))
    return set_err(PF_ERR_INVALID, "prior shapes must be >= 1");
  if (!(cfg->b_sigma > 0 && cfg->b_tau > 0 && cfg->x0_var >= 0))
    return set_err(PF_ERR_INVALID, "prior scales must be > 0 and x0_var >= 0");
  if (cfg->known_variances && !(cfg->sigma2 > 0 && cfg->tau2 > 0))
    return set_err(PF_ERR_INVALID, "known variances must be > 0");
  if (!(cfg->ess_frac >= 0.0 && cfg->ess_frac <= 1.0))
    return set_err(PF_ERR_INVALID, "ess_frac must be in [0, 1]");
  if (cfg->ess_frac > 0.0 && cfg->algorithm != PF_PARTICLE_LEARNING)
    return set_err(PF_ERR_INVALID, "adaptive resampling runs with particle learning");
  if ((cfg->alloc == nullptr) != (cfg->free == nullptr))
    return set_err(PF_ERR_INVALID, "alloc and free must both be set or both NULL");
  pf_filter* f = new (std::nothrow) pf_filter();
  if (!f) return set_err(PF_ERR_OOM, "host allocation failed");
  f->cfg = *cfg;
  f->n = cfg->n_particles;
  f->k = cdf_shift(f->n);
  f->ntiles = (uint32_t)cdiv(f->n, TILE);
  f->fp64 = cfg->precision == PF_FP64;
  f->learn = !cfg->known_variances;
  f->ess = cfg->ess_frac > 0.0;
  f->bootstrap = cfg->algorithm == PF_BOOTSTRAP;
  f->scheme = cfg->scheme;
  pf_status st = PF_OK;
  auto bail = [&](pf_status s) {
    pf_destroy(f);
    return s;
  };
  if (cfg->stream) {
    f->stream = (cudaStream_t)cfg->stream;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&f->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete f;
      return set_err(PF_ERR_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
    }
    f->own_stream = true;
  }
  const size_t rs = f->fp64 ? 8 : 4;
  const size_t n = f->n;
  for (int p = 0; p < 2; ++p) {
    if ((st = dev_alloc(f, n * rs, &f->x[p])) != PF_OK) return bail(st);
    if ((st = dev_alloc(f, n * rs, &f->s2[p])) != PF_OK) return bail(st);
    if ((st = dev_alloc(f, n * rs, &f->t2[p])) != PF_OK) return bail(st);
    if ((st = dev_alloc(f, n * 8, &f->bs[p])) != PF_OK) return bail(st);
    if ((st = dev_alloc(f, n * 8, &f->bt[p])) != PF_OK) return bail(st);
    if ((st = dev_alloc(f, (size_t)f->ntiles * 8, (void**)&f->stat_w[p])) != PF_OK) return bail(st);
    if ((st = dev_alloc(f, (size_t)f->ntiles * 8, (void**)&f->stat_e[p])) != PF_OK) return bail(st);
  }
  // l is moved by 16-byte bulk copies: its tail is padded to 16 bytes
  if ((st = dev_alloc(f, (n * rs + 15) & ~(size_t)15, &f->ell)) != PF_OK) return bail(st);
  if ((st = dev_alloc(f, n * 8, (void**)&f->Q)) != PF_OK) return bail(st);
  if (is_multinomial(f->scheme)) {
    if ((st = dev_alloc(f, (n + 1) * 8, (void**)&f->S)) != PF_OK) return bail(st);
    if (cudaStreamCreateWithFlags(&f->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&f->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&f->ev_join, cudaEventDisableTiming) != cudaSuccess)
      return bail(set_err(PF_ERR_CUDA, "side stream: %s", cudaGetErrorString(cudaGetLastError())));
  }
  if ((st = dev_alloc(f, n * 4, (void**)&f->anc)) != PF_OK) return bail(st);
  if (is_cutpoint(f->scheme) && (st = dev_alloc(f, n * 4, (void**)&f->I)) != PF_OK) return bail(st);
  if ((st = dev_alloc(f, ((size_t)merge_chunks(n) + 1) * 8, (void**)&f->splits)) != PF_OK) return bail(st);
  // log-ML partials: one per CDF tile (2048-particle tiles need twice as many)
  if ((st = dev_alloc(f, (size_t)f->ntiles * 32, &f->part)) != PF_OK) return bail(st);
  f->nparts = f->ntiles;
  const uint64_t est_blocks = cdiv(n, (uint64_t)BLOCK * EST_PER_THREAD);
  if ((st = dev_alloc(f, est_blocks * 8 * 8, (void**)&f->part_est)) != PF_OK) return bail(st);
  if (f->ess) {
    if ((st = dev_alloc(f, n * rs, &f->lam)) != PF_OK) return bail(st);
    const uint64_t eb = cdiv(n, (uint64_t)BLOCK * ESS_PER_THREAD);
    f->ess_grid = (unsigned)(eb < 1024 ? eb : 1024);
    if ((st = dev_alloc(f, (size_t)f->ess_grid * sizeof(U128), (void**)&f->ess_part)) != PF_OK)
      return bail(st);
  }
  if ((st = dev_alloc(f, sizeof(Ctl), (void**)&f->ctl)) != PF_OK) return bail(st);
  if (cudaHostAlloc((void**)&f->ctl_host, sizeof(Ctl), cudaHostAllocMapped) != cudaSuccess) {
    cudaGetLastError();
    return bail(set_err(PF_ERR_OOM, "pinned host allocation failed"));
  }
  // the summary kernels write the mirror directly when it is mapped
  if (cudaHostGetDevicePointer((void**)&f->ctl_host_dev, f->ctl_host, 0) != cudaSuccess) {
    cudaGetLastError();
    f->ctl_host_dev = nullptr;
  }
  if (f->ctl_host_dev && cudaHostAlloc((void**)&f->io, sizeof(EstIO), cudaHostAllocMapped) == cudaSuccess) {
    std::memset(f->io, 0, sizeof(EstIO));
    if (cudaHostGetDevicePointer((void**)&f->io_dev, f->io, 0) != cudaSuccess) {
      cudaFreeHost(f->io);
      f->io = nullptr;
      f->io_dev = nullptr;
    }
  }
  cudaGetLastError();
  // control block: t = 0, no error, max = -inf, counters 0
  Ctl c0;
  std::memset(&c0, 0, sizeof(c0));
  {
    if (f->fp64) {
      double ninf = -__builtin_inf();
      uint64_t b;
      std::memcpy(&b, &ninf, 8);
      c0.maxenc = (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
    } else {
      float ninf = -__builtin_inff();
      uint32_t b;
      std::memcpy(&b, &ninf, 4);
      c0.maxenc = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
    }
  }
  c0.resamp = 1;
  c0.slam = (double)n;
  *f->ctl_host = c0;
  if (cudaMemcpyAsync(f->ctl, f->ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, f->stream) != cudaSuccess)
    return bail(set_err(PF_ERR_CUDA, "control block upload failed"));
  if (f->ess && cudaMemsetAsync(f->lam, 0, n * rs, f->stream) != cudaSuccess)
    return bail(set_err(PF_ERR_CUDA, "log-weight memset failed"));
  for (int p = 0; p < 2; ++p) {
    if (cudaMemsetAsync(f->stat_w[p], 0, (size_t)f->ntiles * 8, f->stream) != cudaSuccess ||
        cudaMemsetAsync(f->stat_e[p], 0, (size_t)f->ntiles * 8, f->stream) != cudaSuccess)
      return bail(set_err(PF_ERR_CUDA, "status memset failed"));
  }
  const unsigned grid = (unsigned)cdiv(n, BLOCK);
  if (f->fp64) {
    FilterArgs<double> a = filter_args<double>(f);
    if (f->learn) k_init<double, true><<<grid, BLOCK, 0, f->stream>>>(a);
    else k_init<double, false><<<grid, BLOCK, 0, f->stream>>>(a);
  } else {
    FilterArgs<float> a = filter_args<float>(f);
    if (f->learn) k_init<float, true><<<grid, BLOCK, 0, f->stream>>>(a);
    else k_init<float, false><<<grid, BLOCK, 0, f->stream>>>(a);
  }
  if (cudaGetLastError() != cudaSuccess) return bail(set_err(PF_ERR_CUDA, "init kernel launch failed"));
  {
    // persistent propagate grid: resident blocks per SM x SMs, at most one
    // block per BLOCK slots
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e;
    if (f->fp64)
      e = f->learn ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_propagate<double, true>, BLOCK, 0)
                   : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_propagate<double, false>, BLOCK, 0);
    else
      e = f->learn ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_propagate2<true>, BLOCK, 0)
                   : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_propagate2<false>, BLOCK, 0);
    if (e != cudaSuccess || per_sm < 1 || sms < 1) return bail(set_err(PF_ERR_CUDA, "occupancy query failed"));
    const uint64_t want = cdiv(n, f->fp64 ? (uint64_t)BLOCK : 2ull * BLOCK),
                   cap = (uint64_t)per_sm * (uint64_t)sms;
    f->prop_grid = (unsigned)(want < cap ? want : cap);
    int per_sm_f = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_f, prop_fuse_fn(f), BLOCK, 0);
    if (e != cudaSuccess || per_sm_f < 1) return bail(set_err(PF_ERR_CUDA, "occupancy query failed"));
    const uint64_t cap_f = (uint64_t)per_sm_f * (uint64_t)sms;
    int per_sm_w = 0;
    e = f->fp64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_w, k_weights<double>, BLOCK, 0)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_w, k_weights<float>, BLOCK, 0);
    if (e != cudaSuccess || per_sm_w < 1) return bail(set_err(PF_ERR_CUDA, "occupancy query failed"));
    f->w_cap = (uint64_t)per_sm_w * (uint64_t)sms;
    f->prop_grid_fuse = (unsigned)(want < cap_f ? want : cap_f);
    if (f->scheme == PF_SYSTEMATIC) {
      // cooperative grid: every CTA resident at once (it waits on the others).
      // One tile per CTA when the tiles fit at once -- in binary32 2048-particle
      // tiles (8 per thread) if those fit, for twice the parallelism -- else
      // the staged variant over 4096-particle tiles.
      int cdf_sm = 0;
      uint64_t g = 0;
      if (!f->fp64) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cdf_sm, cdf_fn(false, false, 8, f->ess), BLOCK, 0);
        if (e != cudaSuccess || cdf_sm < 1) return bail(set_err(PF_ERR_CUDA, "occupancy query failed"));
        g = (uint64_t)cdf_sm * (uint64_t)sms;
        if (cdiv(n, 8ull * BLOCK) <= g) {
          f->cdf_per = 8;
          f->nparts = (uint32_t)cdiv(n, 8ull * BLOCK);
        }
      }
      if (f->cdf_per == 16) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cdf_sm, cdf_fn(f->fp64, false, 16, f->ess), BLOCK, 0);
        if (e != cudaSuccess || cdf_sm < 1) return bail(set_err(PF_ERR_CUDA, "occupancy query failed"));
        g = (uint64_t)cdf_sm * (uint64_t)sms;
        if (f->ntiles > g) {
          f->cdf_staged = true;
          e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cdf_sm, cdf_fn(f->fp64, true, 16, f->ess), BLOCK, 0);
          if (e != cudaSuccess || cdf_sm < 1) return bail(set_err(PF_ERR_CUDA, "occupancy query failed"));
          g = (uint64_t)cdf_sm * (uint64_t)sms;
        }
      }
      const uint64_t nt = f->cdf_per == 8 ? f->nparts : f->ntiles;
      f->cdf_grid = (unsigned)(nt < g ? nt : g);
      // the staged binary32 kernel leaves one exact log-ML partial per CTA
      if (f->cdf_staged && !f->fp64) f->nparts = f->cdf_grid;
      if ((st = dev_alloc(f, (size_t)f->cdf_grid * 8, (void**)&f->cta_tot)) != PF_OK) return bail(st);
      if (f->ess && (st = dev_alloc(f, (size_t)f->cdf_grid * sizeof(U128), (void**)&f->cta_sq)) != PF_OK)
        return bail(st);
    }
  }
  if ((st = build_graph(f, CF_PLAIN)) != PF_OK) return bail(st);
  *out = f;
  return PF_OK;
}

// The form of a cycle that consumes y: without weights when the previous
// cycle computed them, which requires y to be the observation it announced.
static pf_status form_for(pf_filter* f, double y, bool fuse_next, int* form) {
  if (f->ahead && std::memcmp(&y, &f->ahead_y, sizeof(double)) != 0)
    return set_err(PF_ERR_INVALID,
                   "observation %.17g differs from %.17g, announced by pf_step_ahead", y, f->ahead_y);
  *form = f->ahead ? (fuse_next ? CF_MID : CF_TAIL) : (fuse_next ? CF_HEAD : CF_PLAIN);
  return PF_OK;
}

pf_status pf_step(pf_filter* f, double y) {
  pf_status st = check_handle(f);
  if (st != PF_OK) return st;
  int form = CF_PLAIN;
  if ((st = form_for(f, y, false, &form)) != PF_OK) return st;
  if ((st = launch_cycle(f, nullptr, y, form)) != PF_OK) return f->sticky = st;
  f->ahead = false;
  return PF_OK;
}

pf_status pf_step_ahead(pf_filter* f, double y, double y_next) {
  pf_status st = check_handle(f);
  if (st != PF_OK) return st;
  if (f->bootstrap || f->ess) return pf_step(f, y);
  int form = CF_PLAIN;
  if ((st = form_for(f, y, true, &form)) != PF_OK) return st;
  if ((st = launch_cycle(f, nullptr, y, form, nullptr, y_next)) != PF_OK) return f->sticky = st;
  f->ahead = true;
  f->ahead_y = y_next;
  return PF_OK;
}

pf_status pf_run(pf_filter* f, const double* y, uint32_t n_steps) {
  pf_status st = check_handle(f);
  if (st != PF_OK) return st;
  if (!y && n_steps) return set_err(PF_ERR_INVALID, "NULL observations");
  cudaPointerAttributes attr;
  bool dev = false;
  if (n_steps && cudaPointerGetAttributes(&attr, y) == cudaSuccess)
    dev = attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
  cudaGetLastError();
  if (!dev) {
    for (uint32_t i = 0; i < n_steps; ++i)
      if ((st = pf_step(f, y[i])) != PF_OK) return st;
    return PF_OK;
  }
  // device-resident observations cannot be compared with an announced one
  if (f->ahead && n_steps)
    return set_err(PF_ERR_INVALID,
                   "pf_run with device-resident observations after pf_step_ahead: pass the "
                   "announced observation to pf_step first");
  for (uint32_t i = 0; i < n_steps; ++i)
    if ((st = launch_cycle(f, y + i, 0.0)) != PF_OK) return f->sticky = st;
  return PF_OK;
}

// One cycle enqueued kernel by kernel between CUDA events.
static pf_status step_profiled(pf_filter* f, double y, bool fuse_next, double y_next, float* kernel_ms,
                        const char** kernel_names, int max_kernels, int* n_kernels) {
  pf_status st = check_handle(f);
  if (st != PF_OK) return st;
  if (!kernel_ms || !n_kernels || max_kernels < 1) return set_err(PF_ERR_INVALID, "NULL output");
  if (f->bootstrap || f->ess) fuse_next = false;
  int form = CF_PLAIN;
  if ((st = form_for(f, y, fuse_next, &form)) != PF_OK) return st;
  KTimer tm;
  for (int i = 0; i <= KTimer::MAX; ++i) CK(cudaEventCreate(&tm.ev[i]));
  st = f->fp64 ? enqueue_cycle<double>(f, &tm, nullptr, y, form, nullptr, y_next)
               : enqueue_cycle<float>(f, &tm, nullptr, y, form, nullptr, y_next);
  f->ahead = fuse_next && st == PF_OK;
  f->ahead_y = y_next;
  if (st == PF_OK) st = sync_and_check(f);
  if (st == PF_OK) {
    const int cnt = tm.count < max_kernels ? tm.count : max_kernels;
    for (int i = 0; i < cnt; ++i) {
      cudaEventElapsedTime(&kernel_ms[i], tm.ev[i], tm.ev[i + 1]);
      if (kernel_names) kernel_names[i] = tm.names[i];
    }
    *n_kernels = cnt;
  } else {
    f->sticky = st;
  }
  for (int i = 0; i <= KTimer::MAX; ++i) cudaEventDestroy(tm.ev[i]);
  return st;
}

pf_status pf_step_profiled(pf_filter* f, double y, float* kernel_ms, const char** kernel_names,
                           int max_kernels, int* n_kernels) {
  return step_profiled(f, y, false, 0.0, kernel_ms, kernel_names, max_kernels, n_kernels);
}

pf_status pf_step_ahead_profiled(pf_filter* f, double y, double y_next, float* kernel_ms,
                                 const char** kernel_names, int max_kernels, int* n_kernels) {
  return step_profiled(f, y, true, y_next, kernel_ms, kernel_names, max_kernels, n_kernels);
}

pf_status pf_sync(pf_filter* f) {
  pf_status st = check_handle(f);
  if (st != PF_OK) return st;
  return sync_and_check(f);
}

pf_status pf_estimate(pf_filter* f, pf_estimates* out) {
  pf_status st = check_handle(f);
  if (st != PF_OK) return st;
  if (!out) return set_err(PF_ERR_INVALID, "NULL output");
  const unsigned grid = (unsigned)cdiv(f->n, (uint64_t)BLOCK * EST_PER_THREAD);
  if (f->ess) {  // weighted by the carried log-weights
    if (f->fp64) k_estimate_w<double><<<grid, BLOCK, 0, f->stream>>>(filter_args<double>(f));
    else k_estimate_w<float><<<grid, BLOCK, 0, f->stream>>>(filter_args<float>(f));
  } else if (f->fp64) {
    k_estimate<double><<<grid, BLOCK, 0, f->stream>>>(filter_args<double>(f));
  } else {
    k_estimate<float><<<grid, BLOCK, 0, f->stream>>>(filter_args<float>(f));
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    f->sticky = PF_ERR_CUDA;
    return set_err(PF_ERR_CUDA, "estimate launch: %s", cudaGetErrorString(e));
  }
  if (f->ctl_host_dev) {  // the kernel wrote the mirror
    if (cudaStreamSynchronize(f->stream) != cudaSuccess) {
      f->sticky = PF_ERR_CUDA;
      return set_err(PF_ERR_CUDA, "stream: %s", cudaGetErrorString(cudaGetLastError()));
    }
    if ((st = map_err(f->ctl_host->err)) != PF_OK) return f->sticky = st;
  } else if ((st = sync_and_check(f)) != PF_OK) {
    return st;
  }
  const double* v = f->ctl_host->est;
  out->t = (uint64_t)v[0];
  out->x_mean = v[1];
  out->x_var = v[2];
  out->sigma2_mean = v[3];
  out->sigma2_var = v[4];
  out->tau2_mean = v[5];
  out->tau2_var = v[6];
  out->log_marglik = v[7];
  return PF_OK;
}

pf_status pf_step_estimate(pf_filter* f, double y, pf_estimates* out) {
  pf_status st = check_handle(f);
  if (st != PF_OK) return st;
  if (!out) return set_err(PF_ERR_INVALID, "NULL output");
  if (f->ahead) {  // this cycle's weights are ready: the cycle without them, then the summaries
    if ((st = pf_step(f, y)) != PF_OK) return st;
    return pf_estimate(f, out);
  }
  if (f->io) {
    // the observation and the next sequence number into the mapped words,
    // then the graph; the summaries are complete once the summary kernel has
    // copied the number to seq_out (a bounded wait on the host, then the
    // stream's own synchronisation, which also reports a failed launch)
    const uint64_t want = ++f->io_seq;
    f->io->y = y;
    __atomic_store_n(&f->io->seq_in, (unsigned long long)want, __ATOMIC_RELEASE);
    if ((st = launch_cycle(f, nullptr, y, CF_EST)) != PF_OK) return f->sticky = st;
    const auto t0 = std::chrono::steady_clock::now();
    uint32_t k = 0;
    while (__atomic_load_n(&f->io->seq_out, __ATOMIC_ACQUIRE) != want) {
      if ((++k & 1023u) == 0 &&
          std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(20))
        break;
    }
    if (__atomic_load_n(&f->io->seq_out, __ATOMIC_ACQUIRE) != want) {
      if (cudaStreamSynchronize(f->stream) != cudaSuccess) {
        f->sticky = PF_ERR_CUDA;
        return set_err(PF_ERR_CUDA, "stream: %s", cudaGetErrorString(cudaGetLastError()));
      }
      if (__atomic_load_n(&f->io->seq_out, __ATOMIC_ACQUIRE) != want) {
        f->sticky = PF_ERR_CUDA;
        return set_err(PF_ERR_CUDA, "summaries not published");
      }
    }
  } else {
    if ((st = launch_cycle(f, nullptr, y, CF_EST)) != PF_OK) return f->sticky = st;
    if (cudaStreamSynchronize(f->stream) != cudaSuccess) {
      f->sticky = PF_ERR_CUDA;
      return set_err(PF_ERR_CUDA, "stream: %s", cudaGetErrorString(cudaGetLastError()));
    }
  }
  if ((st = map_err(f->ctl_host->err)) != PF_OK) return f->sticky = st;
  const double* v = f->ctl_host->est;
  out->t = (uint64_t)v[0];
  out->x_mean = v[1];
  out->x_var = v[2];
  out->sigma2_mean = v[3];
  out->sigma2_var = v[4];
  out->tau2_mean = v[5];
  out->tau2_var = v[6];
  out->log_marglik = v[7];
  return PF_OK;
}

pf_status pf_get_particles(pf_filter* f, void* x, void* sigma2, void* tau2, void* b_sigma,
                           void* b_tau) {
  pf_status st = check_handle(f);
  if (st != PF_OK) return st;
  if ((st = sync_and_check(f)) != PF_OK) return st;
  const int p = (int)(f->ctl_host->t & 1);
  const size_t rs = f->fp64 ? 8 : 4;
  void* dst[5] = {x, sigma2, tau2, b_sigma, b_tau};
  void* src[5] = {f->x[p], f->s2[p], f->t2[p], f->bs[p], f->bt[p]};
  const size_t sz[5] = {rs, rs, rs, 8, 8};
  for (int i = 0; i < 5; ++i)
    if (dst[i]) CK(cudaMemcpyAsync(dst[i], src[i], f->n * sz[i], cudaMemcpyDefault, f->stream));
  CK(cudaStreamSynchronize(f->stream));
  return PF_OK;
}

pf_status pf_get_ancestors(pf_filter* f, uint32_t* anc, uint64_t* Q) {
  pf_status st = check_handle(f);
  if (st != PF_OK) return st;
  if ((st = sync_and_check(f)) != PF_OK) return st;
  if (anc) CK(cudaMemcpyAsync(anc, f->anc, f->n * 4, cudaMemcpyDefault, f->stream));
  if (Q) CK(cudaMemcpyAsync(Q, f->Q, f->n * 8, cudaMemcpyDefault, f->stream));
  CK(cudaStreamSynchronize(f->stream));
  return PF_OK;
}

pf_status pf_destroy(pf_filter* f) {
  if (!f) return PF_OK;
  if (f->stream) cudaStreamSynchronize(f->stream);
  for (CycleGraph& G : f->cg) {
    if (G.exec) cudaGraphExecDestroy(G.exec);
    if (G.graph) cudaGraphDestroy(G.graph);
  }
  free_all(f);
  if (f->ctl_host) cudaFreeHost(f->ctl_host);
  if (f->io) cudaFreeHost(f->io);
  if (f->side) {
    cudaStreamSynchronize(f->side);
    cudaStreamDestroy(f->side);
  }
  if (f->ev_fork) cudaEventDestroy(f->ev_fork);
  if (f->ev_join) cudaEventDestroy(f->ev_join);
  if (f->own_stream) cudaStreamDestroy(f->stream);
  cudaGetLastError();
  delete f;
  return PF_OK;
}

// ---------------------------------------------------------------------------
// Checkpoint and resume: a header, then the current parity's x, sigma^2,
// tau^2 (R each), b_sigma, b_tau (8 bytes each), n of each, and with
// adaptive resampling the carried log-weights (R each).
// ---------------------------------------------------------------------------
namespace {

constexpr uint64_t CKPT_MAGIC = 0x54504b434c4c4650ull;  // "PFLLCKPT"
constexpr uint32_t CKPT_VERSION = 2;

struct CkptHeader {
  uint64_t magic;
  uint32_t version;
  uint32_t header_bytes;
  uint64_t n;
  uint64_t seed;
  uint32_t filter_id;
  int32_t scheme, precision, known_variances, algorithm, pad;
  double x0_mean, x0_var, a_sigma, b_sigma, a_tau, b_tau, sigma2, tau2;
  uint64_t t;
  double logml;
  double ess_frac, slam;
  uint64_t total_bytes;
};

size_t ckpt_bytes(uint64_t n, bool fp64, bool ess) {
  const size_t rs = fp64 ? 8 : 4;
  return sizeof(CkptHeader) + (size_t)n * (3 * rs + 16 + (ess ? rs : 0));
}

}  // namespace

pf_status pf_checkpoint_size(pf_filter* f, size_t* bytes) {
  if (!f || !bytes) return set_err(PF_ERR_INVALID, "NULL argument");
  *bytes = ckpt_bytes(f->n, f->fp64, f->ess);
  return PF_OK;
}

pf_status pf_checkpoint(pf_filter* f, void* buf, size_t bytes) {
  pf_status st = check_handle(f);
  if (st != PF_OK) return st;
  if (!buf) return set_err(PF_ERR_INVALID, "NULL buffer");
  const size_t need = ckpt_bytes(f->n, f->fp64, f->ess);
  if (bytes < need) return set_err(PF_ERR_INVALID, "checkpoint needs %zu bytes, got %zu", need, bytes);
  if (f->ahead)
    return set_err(PF_ERR_INVALID, "a pf_step_ahead announcement is pending: pf_step(%.17g) first",
                   f->ahead_y);
  if ((st = sync_and_check(f)) != PF_OK) return st;
  CkptHeader h;
  std::memset(&h, 0, sizeof(h));
  h.magic = CKPT_MAGIC;
  h.version = CKPT_VERSION;
  h.header_bytes = sizeof(CkptHeader);
  h.n = f->n;
  h.seed = f->cfg.seed;
  h.filter_id = f->cfg.filter_id;
  h.scheme = f->cfg.scheme;
  h.precision = f->cfg.precision;
  h.known_variances = f->cfg.known_variances;
  h.algorithm = f->cfg.algorithm;
  h.x0_mean = f->cfg.x0_mean;
  h.x0_var = f->cfg.x0_var;
  h.a_sigma = f->cfg.a_sigma;
  h.b_sigma = f->cfg.b_sigma;
  h.a_tau = f->cfg.a_tau;
  h.b_tau = f->cfg.b_tau;
  h.sigma2 = f->cfg.sigma2;
  h.tau2 = f->cfg.tau2;
  h.t = f->ctl_host->t;
  h.logml = f->ctl_host->logml;
  h.ess_frac = f->cfg.ess_frac;
  if (f->ess) {  // the carried weights' sum lies past the summary part
    CK(cudaMemcpy(&h.slam, &f->ctl->slam, sizeof(double), cudaMemcpyDeviceToHost));
  } else {
    h.slam = (double)f->n;
  }
  h.total_bytes = need;
  char* out = static_cast<char*>(buf);
  CK(cudaMemcpy(out, &h, sizeof(h), cudaMemcpyDefault));
  const int p = (int)(h.t & 1);
  const size_t rs = f->fp64 ? 8 : 4;
  const void* src[5] = {f->x[p], f->s2[p], f->t2[p], f->bs[p], f->bt[p]};
  const size_t sz[5] = {rs, rs, rs, 8, 8};
  size_t off = sizeof(h);
  for (int i = 0; i < 5; ++i) {
    CK(cudaMemcpyAsync(out + off, src[i], f->n * sz[i], cudaMemcpyDefault, f->stream));
    off += f->n * sz[i];
  }
  if (f->ess) CK(cudaMemcpyAsync(out + off, f->lam, f->n * rs, cudaMemcpyDefault, f->stream));
  CK(cudaStreamSynchronize(f->stream));
  return PF_OK;
}

pf_status pf_restore(const pf_config* cfg, const void* buf, size_t bytes, pf_filter** out) {
  if (!buf || !out) return set_err(PF_ERR_INVALID, "NULL argument");
  *out = nullptr;
  if (bytes < sizeof(CkptHeader)) return set_err(PF_ERR_INVALID, "checkpoint truncated (%zu bytes)", bytes);
  CkptHeader h;
  CK(cudaMemcpy(&h, buf, sizeof(h), cudaMemcpyDefault));
  if (h.magic != CKPT_MAGIC) return set_err(PF_ERR_INVALID, "not a filter checkpoint");
  if (h.version != CKPT_VERSION || h.header_bytes != sizeof(CkptHeader))
    return set_err(PF_ERR_INVALID, "checkpoint format version %u, this library reads %u", h.version,
                   CKPT_VERSION);
  if (h.precision != PF_FP32 && h.precision != PF_FP64) return set_err(PF_ERR_INVALID, "bad precision");
  if (h.n < 1 || h.n > PF_MAX_PARTICLES) return set_err(PF_ERR_INVALID, "bad particle count");
  const bool fp64 = h.precision == PF_FP64;
  if (!(h.ess_frac >= 0.0 && h.ess_frac <= 1.0)) return set_err(PF_ERR_INVALID, "bad ess_frac");
  const bool ess = h.ess_frac > 0.0;
  const size_t need = ckpt_bytes(h.n, fp64, ess);
  if (h.total_bytes != need || bytes < need)
    return set_err(PF_ERR_INVALID, "checkpoint truncated or inconsistent (%zu of %zu bytes)", bytes, need);
  if (h.t >= 0xffffffffull) return set_err(PF_ERR_INVALID, "bad cycle count");
  pf_config c;
  std::memset(&c, 0, sizeof(c));
  c.n_particles = h.n;
  c.seed = h.seed;
  c.filter_id = h.filter_id;
  c.scheme = h.scheme;
  c.precision = h.precision;
  c.known_variances = h.known_variances;
  c.algorithm = h.algorithm;
  c.x0_mean = h.x0_mean;
  c.x0_var = h.x0_var;
  c.a_sigma = h.a_sigma;
  c.b_sigma = h.b_sigma;
  c.a_tau = h.a_tau;
  c.b_tau = h.b_tau;
  c.sigma2 = h.sigma2;
  c.tau2 = h.tau2;
  c.ess_frac = h.ess_frac;
  if (cfg) {
    c.stream = cfg->stream;
    c.alloc = cfg->alloc;
    c.free = cfg->free;
    c.alloc_ctx = cfg->alloc_ctx;
  }
  pf_filter* f = nullptr;
  pf_status st = pf_create(&c, &f);
  if (st != PF_OK) return st;
  auto bail = [&](pf_status s) {
    pf_destroy(f);
    return s;
  };
  const int p = (int)(h.t & 1);
  const size_t rs = fp64 ? 8 : 4;
  void* dst[5] = {f->x[p], f->s2[p], f->t2[p], f->bs[p], f->bt[p]};
  const size_t sz[5] = {rs, rs, rs, 8, 8};
  const char* in = static_cast<const char*>(buf);
  size_t off = sizeof(h);
  for (int i = 0; i < 5; ++i) {
    if (cudaMemcpyAsync(dst[i], in + off, h.n * sz[i], cudaMemcpyDefault, f->stream) != cudaSuccess)
      return bail(set_err(PF_ERR_CUDA, "checkpoint upload: %s", cudaGetErrorString(cudaGetLastError())));
    off += h.n * sz[i];
  }
  if (ess && cudaMemcpyAsync(f->lam, in + off, h.n * rs, cudaMemcpyDefault, f->stream) != cudaSuccess)
    return bail(set_err(PF_ERR_CUDA, "checkpoint upload: %s", cudaGetErrorString(cudaGetLastError())));
  // the cycle count, the log marginal likelihood and the carried weights'
  // sum; the rest of the control block is as pf_create left it (no error,
  // max -inf, counters 0)
  if (cudaStreamSynchronize(f->stream) != cudaSuccess)
    return bail(set_err(PF_ERR_CUDA, "stream: %s", cudaGetErrorString(cudaGetLastError())));
  f->ctl_host->t = (uint32_t)h.t;
  f->ctl_host->logml = h.logml;
  f->ctl_host->slam = h.slam;
  if (cudaMemcpyAsync(&f->ctl->t, &f->ctl_host->t, sizeof(uint32_t), cudaMemcpyHostToDevice,
                      f->stream) != cudaSuccess ||
      cudaMemcpyAsync(&f->ctl->logml, &f->ctl_host->logml, sizeof(double), cudaMemcpyHostToDevice,
                      f->stream) != cudaSuccess ||
      cudaMemcpyAsync(&f->ctl->slam, &f->ctl_host->slam, sizeof(double), cudaMemcpyHostToDevice,
                      f->stream) != cudaSuccess ||
      cudaStreamSynchronize(f->stream) != cudaSuccess)
    return bail(set_err(PF_ERR_CUDA, "checkpoint upload: %s", cudaGetErrorString(cudaGetLastError())));
  *out = f;
  return PF_OK;
}

// ---------------------------------------------------------------------------
// Standalone resampling and the paper's cut-point primitives.
// ---------------------------------------------------------------------------
namespace {

struct Scratch {
  uint64_t* Q;
  uint64_t* S;
  uint32_t* I;
  uint64_t* splits;
  uint64_t* stat[2];
  uint64_t* stat_e[2];
  Ctl* ctl;
  void* base;
};

constexpr size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Lay out the scratch of pf_resample / pf_cdf inside one allocation.
size_t scratch_layout(uint64_t n, bool need_Q, bool multi, bool cut, char* base, Scratch* s) {
  const uint64_t ntiles = cdiv(n, TILE);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += align256(bytes);
    return p;
  };
  s->ctl = (Ctl*)take(sizeof(Ctl));
  s->stat[0] = (uint64_t*)take(ntiles * 8);
  s->stat[1] = (uint64_t*)take(ntiles * 8);
  s->stat_e[0] = (uint64_t*)take(ntiles * 8);
  s->stat_e[1] = (uint64_t*)take(ntiles * 8);
  const size_t zero_bytes = off;  // everything above must start at zero
  s->Q = need_Q ? (uint64_t*)take(n * 8) : nullptr;
  s->S = multi ? (uint64_t*)take((n + 1) * 8) : nullptr;
  s->I = cut ? (uint32_t*)take(n * 4) : nullptr;
  s->splits = (uint64_t*)take(((size_t)merge_chunks(n) + 1) * 8);
  s->base = base;
  (void)zero_bytes;
  return off;
}

size_t scratch_zero_bytes(uint64_t n) {
  const uint64_t ntiles = cdiv(n, TILE);
  return align256(sizeof(Ctl)) + 4 * align256(ntiles * 8);
}

// Weights -> Q (and S for multinomial) -> ancestors, on stream s with the
// given scratch (already zeroed in its first scratch_zero_bytes bytes).
// Wait settings of the scan: the normal bound, or a failure-detection test's.
struct WaitDiag {
  uint32_t spin_limit = SPIN_LIMIT;
  uint32_t withhold = NO_TILE;
};

pf_status run_resample(const float* w, uint64_t n, uint64_t seed, uint32_t filter, uint32_t t,
                       int scheme, uint32_t* anc, uint64_t* Q_out, const Scratch& sc,
                       cudaStream_t s, WaitDiag dg = WaitDiag()) {
  const uint32_t ntiles = (uint32_t)cdiv(n, TILE);
  const unsigned gmax = (unsigned)(cdiv(n, BLOCK) < 152 * 8 ? cdiv(n, BLOCK) : 152 * 8);
  k_wmax<<<gmax, BLOCK, 0, s>>>(w, n, sc.ctl);
  ScanArgs sa;
  sa.src = w;
  sa.Q = Q_out ? Q_out : sc.Q;
  sa.stat[0] = sc.stat[0];
  sa.stat[1] = sc.stat[1];
  sa.part = nullptr;
  sa.ctl = sc.ctl;
  sa.t_dev = nullptr;
  sa.t_arg = 0;
  sa.n = n;
  sa.k = cdf_shift(n);
  sa.vec_ok = ((uintptr_t)w & 15) == 0;
  sa.spin_limit = dg.spin_limit;
  sa.withhold = dg.withhold;
  k_scan<FROM_WEIGHTS, float><<<ntiles, BLOCK, 0, s>>>(sa);
  CK(cudaGetLastError());
  if (!anc) return PF_OK;
  if (is_multinomial(scheme)) {
    SpacingArgs sp;
    sp.S = sc.S;
    sp.stat[0] = sc.stat_e[0];
    sp.stat[1] = sc.stat_e[1];
    sp.ctl = sc.ctl;
    sp.t_dev = nullptr;
    sp.t_arg = t;
    sp.n = n;
    sp.seed = seed;
    sp.filter = filter;
    k_spacing_scan<<<ntiles, BLOCK, 0, s>>>(sp);
  }
  PosArgs pa;
  pa.gate = nullptr;
  pa.Q = sa.Q;
  pa.S = sc.S;
  pa.anc = anc;
  pa.I = sc.I;
  pa.ctl = sc.ctl;
  pa.t_dev = nullptr;
  pa.t_arg = t;
  pa.n = n;
  pa.seed = seed;
  pa.filter = filter;
  return launch_resample(scheme, pa, n, sc.I, sc.splits, s);
}

pf_status finish_and_check(const Scratch& sc, cudaStream_t s) {
  Ctl h;
  CK(cudaMemcpyAsync(&h, sc.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (h.maxenc == 0) return set_err(PF_ERR_NUMERIC, "all weights are zero");
  return map_err(h.err);
}

// Scratch of pf_resample / pf_cdf comes from a library-owned stream-ordered
// memory pool per device that keeps up to kScratchKeep bytes of freed scratch
// between calls.  (The device's default pool hands freed memory back at every
// synchronisation, which these calls perform, so each call would map fresh
// memory: about 0.2 ms per call.)  Created on first use on each device.
constexpr uint64_t kScratchKeep = 256ull << 20;
constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxDevices] = {};

pf_status scratch_pool(cudaMemPool_t* out) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return set_err(PF_ERR_CUDA, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    CK(cudaMemPoolCreate(&p, &props));
    uint64_t keep = kScratchKeep;
    CK(cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep));
    g_pool[dev] = p;
  }
  *out = g_pool[dev];
  return PF_OK;
}

// A pinned, mapped 32-bit error word per host thread (calls on one host
// thread are sequential: each synchronises its stream before returning).
pf_status small_err_word(uint32_t** host, uint32_t** dev) {
  thread_local uint32_t* h = nullptr;
  thread_local uint32_t* d = nullptr;
  if (!h) {
    if (cudaHostAlloc((void**)&h, 64, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
      cudaGetLastError();
      h = nullptr;
      return set_err(PF_ERR_OOM, "pinned host allocation failed");
    }
    if (cudaHostGetDevicePointer((void**)&d, h, 0) != cudaSuccess) {
      cudaGetLastError();
      cudaFreeHost(h);
      h = nullptr;
      return set_err(PF_ERR_CUDA, "mapped host memory unavailable");
    }
  }
  *host = h;
  *dev = d;
  return PF_OK;
}

// Systematic and stratified resampling of up to SMALL_N weights: one CTA, one
// launch, no scratch (k_resample_small), the same ancestors as the general path.
pf_status resample_small(const float* w, uint64_t n, uint64_t seed, uint32_t filter, uint32_t t,
                         int scheme, uint32_t* anc, cudaStream_t s) {
  uint32_t *eh = nullptr, *ed = nullptr;
  pf_status st = small_err_word(&eh, &ed);
  if (st != PF_OK) return st;
  *(volatile uint32_t*)eh = 0u;
  if (scheme == PF_STRATIFIED)
    k_resample_small<true><<<1, SMALL_THREADS, 0, s>>>(w, (uint32_t)n, seed, filter, t, anc, ed);
  else
    k_resample_small<false><<<1, SMALL_THREADS, 0, s>>>(w, (uint32_t)n, seed, filter, t, anc, ed);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return map_err(*(volatile uint32_t*)eh);
}

pf_status resample_common(const float* w, uint64_t n, uint64_t seed, uint32_t filter,
                          uint32_t t, int scheme, uint32_t* anc, uint64_t* Q_out, void* stream,
                          WaitDiag dg = WaitDiag()) {
  if (!w || (!anc && !Q_out)) return set_err(PF_ERR_INVALID, "NULL pointer");
  if (n < 1 || n > PF_MAX_PARTICLES) return set_err(PF_ERR_INVALID, "n must be in [1, 2^26]");
  if (scheme < 0 || scheme > 4) return set_err(PF_ERR_INVALID, "bad scheme");
  cudaStream_t s = (cudaStream_t)stream;
  if (anc && !Q_out && n <= SMALL_N && dg.withhold == NO_TILE &&
      (scheme == PF_SYSTEMATIC || scheme == PF_STRATIFIED))
    return resample_small(w, n, seed, filter, t, scheme, anc, s);
  Scratch sc;
  const bool multi = anc && is_multinomial(scheme), cut = anc && is_cutpoint(scheme);
  const size_t bytes = scratch_layout(n, Q_out == nullptr, multi, cut, nullptr, &sc);
  void* base = nullptr;
  cudaMemPool_t pool = nullptr;
  pf_status sp = scratch_pool(&pool);
  if (sp != PF_OK) return sp;
  cudaError_t e = cudaMallocFromPoolAsync(&base, bytes, pool, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_err(PF_ERR_OOM, "cudaMallocFromPoolAsync(%zu): %s", bytes, cudaGetErrorString(e));
  }
  scratch_layout(n, Q_out == nullptr, multi, cut, (char*)base, &sc);
  pf_status st = PF_OK;
  if (cudaMemsetAsync(base, 0, scratch_zero_bytes(n), s) != cudaSuccess)
    st = set_err(PF_ERR_CUDA, "scratch memset failed");
  if (st == PF_OK) st = run_resample(w, n, seed, filter, t, scheme, anc, Q_out, sc, s, dg);
  pf_status st2 = PF_OK;
  if (st == PF_OK) st2 = finish_and_check(sc, s);
  cudaFreeAsync(base, s);
  if (st == PF_OK && cudaStreamSynchronize(s) != cudaSuccess)
    st = set_err(PF_ERR_CUDA, "stream synchronisation failed");
  return st != PF_OK ? st : st2;
}

pf_status read_total(const uint64_t* Q, uint64_t n, cudaStream_t s, uint64_t* T) {
  CK(cudaMemcpyAsync(T, Q + n - 1, 8, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (*T == 0 || *T > (1ull << 62)) return set_err(PF_ERR_INVALID, "CDF total must be in [1, 2^62]");
  return PF_OK;
}

}  // namespace

pf_status pf_resample(const float* w_dev, uint64_t n, uint64_t seed, uint32_t filter_id,
                      uint32_t t, int32_t scheme, uint32_t* anc_dev, void* stream) {
  if (!anc_dev) return set_err(PF_ERR_INVALID, "NULL ancestor output");
  return resample_common(w_dev, n, seed, filter_id, t, scheme, anc_dev, nullptr, stream);
}

pf_status pf_cdf(const float* w_dev, uint64_t n, uint64_t* Q_dev, void* stream) {
  if (!Q_dev) return set_err(PF_ERR_INVALID, "NULL CDF output");
  return resample_common(w_dev, n, 0, 0, 0, PF_SYSTEMATIC, nullptr, Q_dev, stream);
}

pf_status pf_diag_cdf_wait(const float* w_dev, uint64_t n, uint32_t withhold_tile,
                           uint32_t spin_limit, uint64_t* Q_dev, void* stream) {
  if (!Q_dev) return set_err(PF_ERR_INVALID, "NULL CDF output");
  if (spin_limit < 1) return set_err(PF_ERR_INVALID, "spin_limit must be at least 1");
  WaitDiag dg;
  dg.spin_limit = spin_limit;
  dg.withhold = withhold_tile;
  return resample_common(w_dev, n, 0, 0, 0, PF_SYSTEMATIC, nullptr, Q_dev, stream, dg);
}

pf_status pf_cutpoint_search(const uint64_t* Q_dev, uint64_t n, uint32_t* I_dev, void* stream) {
  if (!Q_dev || !I_dev) return set_err(PF_ERR_INVALID, "NULL pointer");
  if (n < 1 || n > PF_MAX_PARTICLES) return set_err(PF_ERR_INVALID, "n must be in [1, 2^26]");
  cudaStream_t s = (cudaStream_t)stream;
  uint64_t T;
  pf_status st = read_total(Q_dev, n, s, &T);
  if (st != PF_OK) return st;
  k_cutpoint_search<<<(unsigned)cdiv(n, BLOCK), BLOCK, 0, s>>>(Q_dev, n, I_dev);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return PF_OK;
}

pf_status pf_cutpoint_method(const uint64_t* Q_dev, uint64_t n, const uint32_t* I_dev,
                             const uint64_t* U_dev, uint64_t m, uint32_t* anc_dev, void* stream) {
  if (!Q_dev || !I_dev || (m && (!U_dev || !anc_dev))) return set_err(PF_ERR_INVALID, "NULL pointer");
  if (n < 1 || n > PF_MAX_PARTICLES || m > PF_MAX_PARTICLES)
    return set_err(PF_ERR_INVALID, "n and m must be at most 2^26 (n >= 1)");
  cudaStream_t s = (cudaStream_t)stream;
  uint64_t T;
  pf_status st = read_total(Q_dev, n, s, &T);
  if (st != PF_OK) return st;
  if (m == 0) return PF_OK;
  k_cutpoint_method_explicit<<<(unsigned)cdiv(m, BLOCK), BLOCK, 0, s>>>(Q_dev, n, I_dev, U_dev, m,
                                                                     anc_dev);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return PF_OK;
}

// ---------------------------------------------------------------------------
// Resampling without any allocation.
//
// For callers that cannot allocate device memory when they resample:
// latency-critical loops that must not risk an allocation's device
// synchronisation or unbounded time, and processes whose device memory is
// fully reserved up front.  Only allocation is avoided: the call still makes
// CUDA runtime calls and synchronises its stream, so it is not for host
// functions enqueued on a stream.  The scratch of this entry point lives in
// one file-scope device array of fixed size, present on every device that
// loads the library for the life of the process.
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {

constexpr uint64_t NOALLOC_N = PF_NOALLOC_MAX_PARTICLES;
constexpr uint64_t NOALLOC_TILES = (NOALLOC_N + TILE - 1) / TILE;
constexpr size_t NOALLOC_BYTES =
    align256(sizeof(Ctl)) + 4 * align256(NOALLOC_TILES * 8) + align256(NOALLOC_N * 8) +
    align256((NOALLOC_N + 1) * 8) + align256(NOALLOC_N * 4) +
    align256(((2 * NOALLOC_N + MERGE_D - 1) / MERGE_D + 1) * 8);

// The scratch itself: one copy per device, shared by every call on it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
char* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch on the current device, looked up once per
// device (the host-side symbol is only a stand-in, not a device address).
pf_status noalloc_scratch(char** out) {
  int dev = -1;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return set_err(PF_ERR_INVALID, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return set_err(PF_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    g_noalloc_ptr[dev] = (char*)p;
  }
  *out = g_noalloc_ptr[dev];
  return PF_OK;
}

}  // namespace

extern "C" pf_status pf_resample_noalloc(const float* w_dev, uint64_t n, uint64_t seed,
                                         uint32_t filter_id, uint32_t t, int32_t scheme,
                                         uint32_t* anc_dev, void* stream) {
  if (!w_dev || !anc_dev) return set_err(PF_ERR_INVALID, "NULL pointer");
  if (n < 1 || n > PF_NOALLOC_MAX_PARTICLES)
    return set_err(PF_ERR_INVALID, "pf_resample_noalloc: n must be in [1, %llu]",
                   (unsigned long long)PF_NOALLOC_MAX_PARTICLES);
  if (scheme < 0 || scheme > 4) return set_err(PF_ERR_INVALID, "bad scheme");
  cudaStream_t s = (cudaStream_t)stream;
  char* base = nullptr;
  pf_status st = noalloc_scratch(&base);
  if (st != PF_OK) return st;
  Scratch sc;
  const size_t bytes =
      scratch_layout(n, true, is_multinomial(scheme), is_cutpoint(scheme), nullptr, &sc);
  if (bytes > NOALLOC_BYTES) return set_err(PF_ERR_INVALID, "scratch layout exceeds the static array");
  scratch_layout(n, true, is_multinomial(scheme), is_cutpoint(scheme), base, &sc);
  // the control block and tile status words must start at zero each call
  CK(cudaMemsetAsync(base, 0, scratch_zero_bytes(n), s));
  if ((st = run_resample(w_dev, n, seed, filter_id, t, scheme, anc_dev, nullptr, sc, s)) != PF_OK)
    return st;
  return finish_and_check(sc, s);
}

#include "batch_api.cuh"
#include "server_api.cuh"
