// Kernels of the particle-learning cycle (sm_103a).
//
// One cycle for observation y = y_{t+1} (paper Section 2, Algorithm
// "Particle Learning"):
//   k_weights       l_i = log p(y | x_i, sigma_i^2, tau_i^2) + log(2 pi)/2, max_i l_i
//   k_scan          W_i = quantised exp(l_i - max), Q = inclusive scan of W
//                   (eq. resample.cdf as exact 64-bit integers), single pass
//                   with decoupled look-back
//   k_spacing_scan  (multinomial) S = inclusive scan of exponential spacings
//   k_merge         ancestors a_j = #{i : Q_i * A <= B_j} by a merge of the
//                   sorted positions B with the CDF
//   k_cutpoint_*    the paper's Section 3.2 algorithms (same ancestors)
//   k_propagate     gather ancestor, draw x, update b_sigma/b_tau, draw theta
//   k_estimate      posterior summaries on demand
//
// Data layout in HBM (structure of arrays, one entry per particle):
//   x, sigma2, tau2 : R (binary32 or binary64), two ping-pong copies
//   b_sigma, b_tau  : uint64 2^-32 fixed point (FP32) / binary64 (FP64)
//   l               : R,    Q : uint64,   S : uint64 (n+1),   anc : uint32
#pragma once
#include <cstddef>
#include <cstdint>

#include "device.cuh"

namespace pfk {

constexpr int BLOCK = 256;
constexpr int WARPS = BLOCK / 32;
constexpr int CHUNK = 128;                 // elements per warp per chunk (4 per lane)
constexpr int CHUNKS = 4;                  // chunks per warp
constexpr int TILE = WARPS * CHUNKS * CHUNK;  // 4096 elements per scan tile
constexpr int MERGE_D = 2048;              // merged elements per merge CTA
constexpr int MERGE_E = MERGE_D / BLOCK;   // merged elements per thread

constexpr uint64_t FLAG_A = 1ull << 62;    // tile aggregate published
constexpr uint64_t FLAG_P = 2ull << 62;    // tile inclusive prefix published
constexpr uint64_t VAL_MASK = (1ull << 62) - 1;
constexpr uint32_t SPIN_LIMIT = 1u << 22;  // bounded look-back wait

enum ErrBits : uint32_t {
  ERR_TIMEOUT = 1u,   // look-back gave up
  ERR_NUMERIC = 2u,   // non-finite max, gamma sampler failure, b overflow
  ERR_WEIGHTS = 4u,   // negative / non-finite / all-zero input weights
};

// Per-filter control block in device memory.
struct Ctl {
  uint32_t t;             // cycles completed
  uint32_t err;           // ErrBits
  unsigned long long maxenc;  // order-encoded max of l (or of the input weights)
  uint32_t ticket_w;      // scan tile ticket
  uint32_t ticket_e;      // spacing scan tile ticket
  uint32_t done_prop;     // last-block counter of k_propagate
  uint32_t done_est;      // last-block counter of k_estimate
  uint32_t gbar;          // grid barrier of k_cdf_sys
  double logml;           // accumulated log marginal likelihood
  double est[8];          // t, x mean/var, sigma2 mean/var, tau2 mean/var, log_marglik
  // per-cycle constants written by k_weights (block 0) for k_propagate:
  double y;               // this cycle's observation y_{t+1}
  double mtd[6];          // Marsaglia-Tsang d, c for sigma^2 and tau^2 ([0..3]) and the
                          // squeeze coefficients K_sigma, K_tau ([4], [5]), binary64
  float yf;               // y rounded to binary32
  float mtf[6];           // the same constants rounded to binary32
  // resampling key constants written by k_partition (block 0) for k_merge:
  // T = Q_{n-1}, A (n or S_n) and the systematic offset r
  uint64_t keyT, keyA, keyR;
  // the next cycle's maximum of l, gathered by a propagation that also
  // computes the next cycle's predictive weights (order-encoded, as maxenc)
  unsigned long long maxenc_nx;
  // adaptive resampling: this cycle's decision (written by k_ess), the
  // last-block counter of k_ess, and sum_i exp(lambda_i) of the carried
  // log-weights (n after a resampling)
  uint32_t resamp;
  uint32_t done_ess;
  double slam;
  // binary32 propagation: the next unit of 64 slots to hand out
  unsigned long long prop_ticket;
  // weights kernel: the next round of WARPS chunks to hand out
  uint32_t w_ticket;
};

// Tile status words carry their value and flag in one aligned 64-bit word and
// nothing else is read through them, so relaxed (single-copy atomic) accesses
// suffice; unlike acquire loads, several can be in flight at once.
__device__ __forceinline__ void st_status(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_status(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_volatile_u32(const uint32_t* p) {
  return *(volatile const uint32_t*)p;
}

template <class T>
__device__ __forceinline__ T shfl_up(T v, int d) {
  return __shfl_up_sync(0xffffffffu, v, d);
}
__device__ __forceinline__ uint64_t warp_incl_scan(uint64_t v, int lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint64_t o = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= d) v += o;
  }
  return v;
}

// ---------------------------------------------------------------------------
// State views.
// ---------------------------------------------------------------------------
template <class R> struct SuffT;
template <> struct SuffT<float> { typedef uint64_t B; };
template <> struct SuffT<double> { typedef double B; };

template <class R>
struct StateV {
  R* x;
  R* s2;
  R* t2;
  typename SuffT<R>::B* bs;
  typename SuffT<R>::B* bt;
};

// Host-mapped words of a synchronous cycle with summaries (pf_step_estimate):
// the observation, and the host's sequence number, which the summary kernel
// copies to seq_out once the summaries are in the host mirror.
struct EstIO {
  double y;
  unsigned long long seq_in;
  unsigned long long seq_out;
  unsigned long long pad;
};

template <class R>
struct FilterArgs {
  StateV<R> st[2];          // ping-pong by cycle parity
  R* ell;
  uint64_t* Q;
  uint64_t* S;              // n+1 spacing prefix (multinomial)
  uint32_t* anc;
  uint32_t* I;              // cut-point table
  uint64_t* stat_w[2];      // scan tile status, by parity
  uint64_t* stat_e[2];      // spacing scan tile status, by parity
  void* part;               // per-tile log-ML partial (U128 for FP32, double for FP64)
  double* part_est;         // per-block estimate partials
  Ctl* ctl;
  // device address of the handle's pinned host mirror of the control block
  // (mapped), or NULL: the summary kernels write the control block's summary
  // prefix there directly, so no copy follows them
  Ctl* ctl_mirror;
  EstIO* io;                // mapped words of pf_step_estimate, or NULL
  // this cycle's observation: *y_src when y_src is set (device-resident
  // observations), else y_val (set per launch in the graph's weights node)
  const double* y_src;
  double y_val;
  // the next cycle's observation y_{t+2}, for a propagation that computes
  // the next cycle's predictive weights (*y_nx_src when set, else y_nx_val)
  const double* y_nx_src;
  double y_nx_val;
  // adaptive resampling: carried log-weights (NULL: resample every cycle),
  // the ESS fraction and k_ess's per-block partial sums of W^2
  R* lam;
  double ess_frac;
  U128* ess_part;
  uint64_t n;
  uint32_t ntiles;
  uint32_t nparts;          // log-ML partials written this cycle (one per CDF tile)
  int k;                    // CDF shift: W <= 2^k
  uint64_t seed;
  uint32_t filter;
  uint32_t rk[20];          // Philox round keys of seed (philox_rk)
  double x0_mean, x0_var, a_sigma, b_sigma, a_tau, b_tau, sigma2, tau2;
};

// ---------------------------------------------------------------------------
// Initialisation (Algorithm "Particle Learning", Step 0).
// ---------------------------------------------------------------------------
template <class R> struct SuffOps;
template <> struct SuffOps<float> {
  static __device__ __forceinline__ uint64_t from_prior(double b) {
    return __double2ull_rz(b * 0x1p32);
  }
  // b + r^2 / 2 in 2^-32 fixed point: trunc(r^2 2^31), which is
  // (r^2 / 2) 2^32 exactly; below 2^32 by one u32 truncation
  static __device__ __forceinline__ uint64_t incr(float v) {
    return v < 0x1p32f ? (uint64_t)__float2uint_rz(v) : f2u64_rz(v);
  }
  static __device__ __forceinline__ uint64_t add_half_square(uint64_t b, float r, bool* fail) {
    const float r2 = r * r;
    const float v = r2 * 0x1p31f;
    if (!(v < 0x1p63f)) {
      *fail = true;
      return b;
    }
    return b + incr(v);
  }
  // b 2^-32 in binary32 from the two 32-bit halves, each converted to
  // nearest, joined by one fused multiply-add
  static __device__ __forceinline__ float bscale(uint64_t b) {
    const float hi = __uint2float_rn((uint32_t)(b >> 32));
    const float lo = __uint2float_rn((uint32_t)b);
    return __fmaf_rn(lo, 0x1p-32f, hi);
  }
  static __device__ __forceinline__ float ig(uint64_t b, float G) { return bscale(b) / G; }
};
template <> struct SuffOps<double> {
  static __device__ __forceinline__ double from_prior(double b) { return b; }
  static __device__ __forceinline__ double add_half_square(double b, double r, bool*) {
    const double r2 = r * r;
    const double h = 0.5 * r2;
    return b + h;
  }
  static __device__ __forceinline__ double ig(double b, double G) { return b / G; }
};

// Constants of Marsaglia-Tsang for shape a, in binary64: d = a - 1/3,
// c = 1/sqrt(9 d) and the squeeze coefficient K = 0.0331 (2/3) / d, with
// 0.0331 (2/3) = 331/15000 rounded to nearest.
__device__ __forceinline__ void mt_constants(double a, double* d, double* c, double* K) {
  const double ONE_THIRD = 0x1.5555555555555p-2;
  const double SQZ = 0x1.698a4eea9073cp-6;
  const double dd = a - ONE_THIRD;
  const double nine_d = 9.0 * dd;
  const double s = sqrt(nine_d);
  *d = dd;
  *c = 1.0 / s;
  *K = SQZ / dd;
}
// This cycle's constants for the propagation (observation and the
// Marsaglia-Tsang constants of the shapes a0 + (t+1)/2), in both precisions.
__device__ __forceinline__ void write_cycle_constants(Ctl* c, double y, double a_sigma,
                                                      double a_tau, uint32_t t1) {
  double ds, cs, ks, dt, ct, kt;
  mt_constants(a_sigma + 0.5 * (double)t1, &ds, &cs, &ks);
  mt_constants(a_tau + 0.5 * (double)t1, &dt, &ct, &kt);
  c->y = y;
  c->yf = (float)y;
  const double v[6] = {ds, cs, dt, ct, ks, kt};
  for (int i = 0; i < 6; ++i) {
    c->mtd[i] = v[i];
    c->mtf[i] = (float)v[i];
  }
}

template <class R, bool LEARN>
__global__ void __launch_bounds__(BLOCK) k_init(FilterArgs<R> a) {
  __shared__ double s_c[7];
  if (threadIdx.x == 0) {
    double ds, cs, ks, dt, ct, kt;
    mt_constants(a.a_sigma, &ds, &cs, &ks);
    mt_constants(a.a_tau, &dt, &ct, &kt);
    s_c[0] = ds; s_c[1] = cs; s_c[2] = dt; s_c[3] = ct;
    s_c[4] = sqrt(a.x0_var);
    s_c[5] = ks; s_c[6] = kt;
  }
  __syncthreads();
  const uint64_t j = (uint64_t)blockIdx.x * BLOCK + threadIdx.x;
  if (j >= a.n) return;
  const StateV<R> st = a.st[0];
  const R x0m = (R)a.x0_mean;
  const R sdx = (R)s_c[4];
  const R Z = bm_normal(draw(a.seed, a.filter, 0, (uint32_t)j, P_INIT_X, 0), (R)0);
  const R p = sdx * Z;
  st.x[j] = x0m + p;
  const auto bs0 = SuffOps<R>::from_prior(a.b_sigma);
  const auto bt0 = SuffOps<R>::from_prior(a.b_tau);
  st.bs[j] = bs0;
  st.bt[j] = bt0;
  if (!LEARN) {
    st.s2[j] = (R)a.sigma2;
    st.t2[j] = (R)a.tau2;
    return;
  }
  bool fail = false;
  const R Gs = gamma_mt<R>((R)s_c[0], (R)s_c[1], (R)s_c[5], a.seed, a.filter, 0, (uint32_t)j,
                          P_INIT_SIGMA, &fail);
  const R Gt = gamma_mt<R>((R)s_c[2], (R)s_c[3], (R)s_c[6], a.seed, a.filter, 0, (uint32_t)j,
                          P_INIT_TAU, &fail);
  st.s2[j] = SuffOps<R>::ig(bs0, Gs);
  st.t2[j] = SuffOps<R>::ig(bt0, Gt);
  if (fail) atomicOr(&a.ctl->err, ERR_NUMERIC);
}

// ---------------------------------------------------------------------------
// Step 1a: predictive log-likelihood and its maximum.
// ---------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ R log_pred(R x, R s2, R t2, R y) {
  const R s = s2 + t2;
  const R dx = y - x;
  const R q = dx * dx;
  const R lg = det_log(s);
  const R r = q / s;
  const R sum = lg + r;
  return (R)-0.5 * sum;
}

__device__ __forceinline__ unsigned long long enc_max(float x) { return enc_f(x); }
__device__ __forceinline__ unsigned long long enc_max(double x) { return enc_d(x); }

template <class R>
__device__ __forceinline__ R block_max(R v, R* s_red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane == 0) s_red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < WARPS ? s_red[lane] : (R)-INFINITY;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  }
  return v;
}

// Persistent over the particles: per pass a warp takes a chunk of 64 16-byte
// vectors of each array (2 x 32 x W_VEC particles), each load and store
// instruction 512 contiguous bytes, two of each in flight per thread and array;
// the rest of the last chunk element by element.  One block maximum and one
// atomic per CTA.
template <class R> struct WVec;
template <> struct WVec<float> {
  static constexpr int N = 4;
  typedef float4 V;
  static __device__ __forceinline__ void get(const V& v, float* o) { o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w; }
  static __device__ __forceinline__ V make(const float* o) { return make_float4(o[0], o[1], o[2], o[3]); }
};
template <> struct WVec<double> {
  static constexpr int N = 2;
  typedef double2 V;
  static __device__ __forceinline__ void get(const V& v, double* o) { o[0] = v.x; o[1] = v.y; }
  static __device__ __forceinline__ V make(const double* o) { return make_double2(o[0], o[1]); }
};
constexpr int W_CTAS_PER_SM = 4;  // 64 registers: the pass's 2 x 3 vectors stay in registers

// With ESS (adaptive resampling) the carried log-weights are added: L = lambda + l.
template <class R, bool ESS = false>
__global__ void __launch_bounds__(BLOCK, W_CTAS_PER_SM) k_weights(FilterArgs<R> a) {
  typedef WVec<R> VW;
  typedef typename VW::V V;
  constexpr int NV = VW::N;
  constexpr uint64_t CHUNK = 64 * NV;  // particles per warp pass
  __shared__ R s_red[WARPS];
  const uint32_t t = a.ctl->t;
  const StateV<R> st = (t & 1) ? a.st[1] : a.st[0];
  // every thread reads y itself (no barrier), so that its first loads of the
  // state overlap that read (y may sit in host memory)
  const double y = a.y_src ? *a.y_src : a.y_val;
  if (blockIdx.x == 0 && threadIdx.x == 0) write_cycle_constants(a.ctl, y, a.a_sigma, a.a_tau, t + 1);
  const R yr = (R)y;
  const uint64_t n = a.n;
  const int lane = threadIdx.x & 31;
  const uint64_t gw = (uint64_t)blockIdx.x * WARPS + (threadIdx.x >> 5);
  const uint64_t nw = (uint64_t)gridDim.x * WARPS;
  R mx = (R)-INFINITY;
  bool bad = false;
  auto weigh = [&](R x, R s2, R t2, R lam) {
    R l = log_pred<R>(x, s2, t2, yr);
    if constexpr (ESS) l = lam + l;
    bad |= !(l < (R)INFINITY);  // NaN or +inf
    mx = fmax(mx, l);
    return l;
  };
  auto chunk = [&](uint64_t cb) {  // the warp's chunk of CHUNK particles from cb
    if (cb + CHUNK <= n) {
      const uint64_t i0 = cb + (uint64_t)lane * NV, i1 = i0 + 32 * NV;
      const V x0 = *reinterpret_cast<const V*>(st.x + i0), x1 = *reinterpret_cast<const V*>(st.x + i1);
      const V s0 = *reinterpret_cast<const V*>(st.s2 + i0), s1 = *reinterpret_cast<const V*>(st.s2 + i1);
      const V u0 = *reinterpret_cast<const V*>(st.t2 + i0), u1 = *reinterpret_cast<const V*>(st.t2 + i1);
      R xv[2 * NV], sv[2 * NV], tv[2 * NV], lm[2 * NV], lv[2 * NV];
      VW::get(x0, xv); VW::get(x1, xv + NV);
      VW::get(s0, sv); VW::get(s1, sv + NV);
      VW::get(u0, tv); VW::get(u1, tv + NV);
      if constexpr (ESS) {
        VW::get(*reinterpret_cast<const V*>(a.lam + i0), lm);
        VW::get(*reinterpret_cast<const V*>(a.lam + i1), lm + NV);
      }
#pragma unroll
      for (int e = 0; e < 2 * NV; ++e) lv[e] = weigh(xv[e], sv[e], tv[e], ESS ? lm[e] : (R)0);
      *reinterpret_cast<V*>(a.ell + i0) = VW::make(lv);
      *reinterpret_cast<V*>(a.ell + i1) = VW::make(lv + NV);
    } else {
      for (uint64_t i = cb + lane; i < n; i += 32)
        a.ell[i] = weigh(st.x[i], st.s2[i], st.t2[i], ESS ? a.lam[i] : (R)0);
    }
  };
  const uint64_t nchunks = (n + CHUNK - 1) / CHUNK;
  if (nchunks >= 4 * nw) {
    // Many chunks per warp: rounds of WARPS chunks (one per warp) go to
    // CTAs by ticket, each ticket taken a round ahead by thread 0, so that
    // CTAs on faster SMs take more rounds (the CTAs' finishing times under
    // the grid stride at N = 2^24 spread from 35 to 43 us).
    __shared__ uint32_t s_round[2];
    const uint64_t nrounds = (nchunks + WARPS - 1) / WARPS;
    uint64_t rd = blockIdx.x;
    uint32_t tk = 0;
    if (threadIdx.x == 0) tk = atomicAdd(&a.ctl->w_ticket, 1u);
    for (uint32_t q = 0; rd < nrounds; ++q) {
      const uint64_t ch = rd * WARPS + (threadIdx.x >> 5);
      if (ch < nchunks) chunk(ch * CHUNK);
      if (threadIdx.x == 0) {
        s_round[q & 1] = gridDim.x + tk;
        tk = atomicAdd(&a.ctl->w_ticket, 1u);
      }
      __syncthreads();
      rd = s_round[q & 1];
    }
  } else {
    for (uint64_t cb = gw * CHUNK; cb < n; cb += nw * CHUNK) chunk(cb);
  }
  if (bad) atomicOr(&a.ctl->err, ERR_NUMERIC);
  mx = block_max<R>(mx, s_red);
  if (threadIdx.x == 0 && mx > (R)-INFINITY) atomicMax(&a.ctl->maxenc, enc_max(mx));
}
// CTAs of the weights kernel for n particles: the resident maximum `cap`, or
// fewer when the particles make fewer chunks than the resident warps.
template <class R>
inline unsigned weights_grid(uint64_t n, uint64_t cap) {
  const uint64_t per_cta = 64ull * WVec<R>::N * WARPS;  // one chunk per warp
  const uint64_t ctas = (n + per_cta - 1) / per_cta;
  return (unsigned)(ctas < cap ? (ctas > 0 ? ctas : 1) : cap);
}

// ---------------------------------------------------------------------------
// Algorithm "Particle Filtering" (the bootstrap filter, known variances),
// Steps 1-2: propagate every particle blind, x_t = x~_{t-1} + sqrt(tau^2) Z
// (Box-Muller's first output of the draw (seed, filter, t, i, BOOT_STATE)),
// in place, then weigh it by p(y_t | x_t) = N(y_t; x_t, sigma^2): the
// predictive-weight kernel's l with tau^2 = 0, and its maximum.  Step 3 is
// the resampling of the particle-learning cycle; k_boot_gather then copies
// the ancestors.
// ---------------------------------------------------------------------------
template <class R>
__global__ void __launch_bounds__(BLOCK) k_boot_pw(FilterArgs<R> a) {
  __shared__ R s_red[WARPS];
  Ctl* c = a.ctl;
  const uint32_t t = c->t;
  const StateV<R> st = (t & 1) ? a.st[1] : a.st[0];
  const double y = a.y_src ? *a.y_src : a.y_val;
  const R yr = (R)y;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    c->y = y;
    c->yf = (float)y;
  }
  R mx = (R)-INFINITY;
  bool bad = false;
  const uint64_t i = (uint64_t)blockIdx.x * BLOCK + threadIdx.x;
  if (i < a.n) {
    const R Z = bm_normal(draw(a.seed, a.filter, t, (uint32_t)i, P_BOOT_STATE, 0), (R)0);
    const R sv = sqrt(st.t2[i]);
    const R xz = sv * Z;
    const R xp = st.x[i] + xz;
    st.x[i] = xp;
    const R l = log_pred<R>(xp, st.s2[i], (R)0, yr);
    bad = !(l < (R)INFINITY);  // NaN or +inf
    mx = l;
    a.ell[i] = l;
  }
  if (bad) atomicOr(&c->err, ERR_NUMERIC);
  mx = block_max<R>(mx, s_red);
  if (threadIdx.x == 0 && mx > (R)-INFINITY) atomicMax(&c->maxenc, enc_max(mx));
}

// ---------------------------------------------------------------------------
// Step 1b: the exact fixed-point CDF by a single-pass decoupled look-back scan
// (Merrill & Garland 2016).  Tiles are claimed through an atomic ticket so a
// tile's predecessors are always resident or finished; the look-back wait is
// bounded and reports ERR_TIMEOUT instead of hanging.
//
// Warp w of a tile owns elements [512 w, 512 w + 512) as 4 chunks of 128;
// lane l owns elements 4l..4l+3 of each chunk, so every load and store
// instruction of the warp covers one contiguous span.
// ---------------------------------------------------------------------------

// Sum of exp(l_i - m) for the log marginal likelihood: exact 2^-96 fixed
// point in FP32 mode (binary32 terms >= 2^-73 are integers there).
struct ESum32 {
  U128 s;
  __device__ __forceinline__ void zero() { s.hi = 0; s.lo = 0; }
  __device__ __forceinline__ void add(float e) {
    // e = 0 or e >= 2^-73: e * 2^96 = mant * 2^(exponent bits - 54), an
    // integer below 2^101 (e < 16 for a thread's partial); added without branches
    const uint32_t b = __float_as_uint(e);
    const uint32_t E = b >> 23;
    const uint64_t mant = E ? (uint64_t)((b & 0x7fffffu) | 0x800000u) : 0ull;
    const int sh = E > 54u ? (int)E - 54 : 0;
    const uint64_t lo = sh < 64 ? mant << sh : 0ull;
    const uint64_t hi = sh == 0 ? 0ull : (sh < 64 ? mant >> (64 - sh) : mant << (sh - 64));
    s = add128(s, U128{hi, lo});
  }
  __device__ __forceinline__ void add(const ESum32& o) { s = add128(s, o.s); }
  __device__ __forceinline__ ESum32 shfl_xor(int m) const {
    ESum32 r;
    r.s.hi = __shfl_xor_sync(0xffffffffu, s.hi, m);
    r.s.lo = __shfl_xor_sync(0xffffffffu, s.lo, m);
    return r;
  }
};
struct ESum64 {
  double s;
  __device__ __forceinline__ void zero() { s = 0.0; }
  __device__ __forceinline__ void add(double e) { s = s + e; }
  __device__ __forceinline__ void add(const ESum64& o) { s = s + o.s; }
  __device__ __forceinline__ ESum64 shfl_xor(int m) const {
    ESum64 r;
    r.s = __shfl_xor_sync(0xffffffffu, s, m);
    return r;
  }
};
template <class R> struct ESumT;
template <> struct ESumT<float> { typedef ESum32 T; };
template <> struct ESumT<double> { typedef ESum64 T; };

// Tile look-back by warp 0.  Returns the exclusive prefix of the tile (in
// lane 0).  `total` is the tile aggregate.  Each round reads a window of 128
// predecessors (four status words per lane, loads issued together), so a
// tile far from the last published prefix needs few round trips.
constexpr int LB_PER_LANE = 4;

__device__ __forceinline__ uint64_t spin_status(const uint64_t* p, bool* timed_out,
                                                uint32_t limit) {
  uint64_t v = ld_status(p);
  uint32_t spins = 0;
  while ((v >> 62) == 0) {
    if (++spins > limit) {
      *timed_out = true;
      return FLAG_P;
    }
    __nanosleep(32);
    v = ld_status(p);
  }
  return v;
}

// limit: polls of one status word before the wait gives up (ERR_TIMEOUT);
// withhold: a tile that publishes nothing (a failure-detection test makes its
// successors' waits run out this way; NO_TILE otherwise).
constexpr uint32_t NO_TILE = 0xffffffffu;
__device__ __forceinline__ uint64_t lookback(uint64_t* stat, uint32_t tile, uint64_t total,
                                             uint32_t* err, uint32_t limit = SPIN_LIMIT,
                                             uint32_t withhold = NO_TILE) {
  const int lane = threadIdx.x & 31;
  if (tile == withhold) return 0;
  if (tile == 0) {
    if (lane == 0) st_status(&stat[0], FLAG_P | total);
    return 0;
  }
  if (lane == 0) st_status(&stat[tile], FLAG_A | total);
  uint64_t excl = 0;
  int64_t look = (int64_t)tile - 1;
  bool timed_out = false;
  while (true) {
    // lane l covers distances LB_PER_LANE*l .. LB_PER_LANE*l + 3 below `look`
    uint64_t v[LB_PER_LANE];
#pragma unroll
    for (int k = 0; k < LB_PER_LANE; ++k) {
      const int64_t idx = look - (LB_PER_LANE * lane + k);
      v[k] = idx >= 0 ? ld_status(&stat[idx]) : FLAG_P;  // before tile 0: a zero prefix
    }
#pragma unroll
    for (int k = 0; k < LB_PER_LANE; ++k) {
      const int64_t idx = look - (LB_PER_LANE * lane + k);
      if ((v[k] >> 62) == 0) v[k] = spin_status(&stat[idx], &timed_out, limit);
    }
    int first_p = LB_PER_LANE;
#pragma unroll
    for (int k = LB_PER_LANE - 1; k >= 0; --k)
      if ((v[k] >> 62) == 2) first_p = k;
    const uint32_t pmask = __ballot_sync(0xffffffffu, first_p < LB_PER_LANE);
    const int stop_lane = pmask ? __ffs(pmask) - 1 : 32;
    uint64_t contrib = 0;
#pragma unroll
    for (int k = 0; k < LB_PER_LANE; ++k) {
      const bool take = lane < stop_lane || (lane == stop_lane && k <= first_p);
      if (take) contrib += v[k] & VAL_MASK;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) contrib += __shfl_xor_sync(0xffffffffu, contrib, o);
    excl += contrib;
    if (pmask) break;
    look -= 32 * LB_PER_LANE;
  }
  if (__any_sync(0xffffffffu, timed_out) && lane == 0) atomicOr(err, ERR_TIMEOUT);
  if (lane == 0) st_status(&stat[tile], FLAG_P | ((excl + total) & VAL_MASK));
  return excl;
}

// Scan sources.
enum ScanMode { FROM_LOGLIK = 0, FROM_WEIGHTS = 1 };

struct ScanArgs {
  const void* src;          // l (R) or w (float)
  uint64_t* Q;
  uint64_t* stat[2];        // tile status by cycle parity; the other parity's
                            // entries are cleared for the next cycle
  void* part;               // per-tile log-ML partial (FROM_LOGLIK)
  Ctl* ctl;
  const uint32_t* t_dev;    // cycle index in device memory, or NULL
  uint32_t t_arg;
  uint64_t n;
  int k;
  int vec_ok;               // src is 16-byte aligned
  uint32_t spin_limit;      // look-back polls before giving up (SPIN_LIMIT)
  uint32_t withhold;        // a tile that publishes nothing (NO_TILE; failure tests)
};

// Thread-blocked scan: thread t of a tile owns the 16 consecutive elements
// [16 t, 16 t + 16), so the running sum is two integer adds per element and
// the warp / block scans run once per 16 elements.
constexpr int SCAN_PER = TILE / BLOCK;  // 16

template <int MODE, class R>
__global__ void __launch_bounds__(BLOCK, 4) k_scan(ScanArgs a) {
  typedef typename ESumT<R>::T ES;
  __shared__ uint64_t s_stage[BLOCK * (SCAN_PER + 1)];
  __shared__ uint32_t s_tile;
  __shared__ uint64_t s_warp_tot[WARPS];
  __shared__ uint64_t s_excl;
  __shared__ ES s_es[WARPS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_tile = atomicAdd(&a.ctl->ticket_w, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint64_t base = (uint64_t)tile * TILE + (uint64_t)threadIdx.x * SCAN_PER;
  const uint32_t par = (a.t_dev ? *a.t_dev : a.t_arg) & 1u;
  uint64_t* const stat = par ? a.stat[1] : a.stat[0];
  uint64_t* const stat_next = par ? a.stat[0] : a.stat[1];

  // the value that quantisation is relative to
  R m = (R)0;
  int escale = 0;
  if (MODE == FROM_LOGLIK) {
    if constexpr (sizeof(R) == 4) m = dec_f((uint32_t)a.ctl->maxenc);
    else m = dec_d(a.ctl->maxenc);
  } else {
    int e;
    (void)frexpf(__uint_as_float((uint32_t)a.ctl->maxenc), &e);
    escale = a.k - e;
  }

  const bool full = base + SCAN_PER <= a.n;
  uint64_t W[SCAN_PER];
  R epart = (R)0;  // this thread's sum of exp(l - m), fixed order
  uint64_t run = 0;
#pragma unroll
  for (int q = 0; q < SCAN_PER / 4; ++q) {
    // four values at a time, consumed as soon as they arrive
    R v[4];
    if (full && a.vec_ok) {
      if constexpr (sizeof(R) == 4) {
        const float4 f = *reinterpret_cast<const float4*>((const float*)a.src + base + 4 * q);
        v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
      } else {
        const double2 f0 = *reinterpret_cast<const double2*>((const double*)a.src + base + 4 * q);
        const double2 f1 = *reinterpret_cast<const double2*>((const double*)a.src + base + 4 * q + 2);
        v[0] = f0.x; v[1] = f0.y; v[2] = f1.x; v[3] = f1.y;
      }
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e)
        v[e] = (base + 4 * q + e < a.n) ? ((const R*)a.src)[base + 4 * q + e] : (R)0;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      uint64_t w = 0;
      if (full || base + 4 * q + e < a.n) {
        if (MODE == FROM_LOGLIK) {
          R ex;
          const R dl = v[e] - m;
          w = quant_exp<R>(dl, a.k, &ex);
          epart = epart + ex;
        } else {
          const float wf = (float)v[e];
          if (!(wf >= 0.0f) || !(wf < INFINITY)) atomicOr(&a.ctl->err, ERR_WEIGHTS);
          else w = f2u64_rz(ldexpf(wf, escale));
        }
      }
      run += w;
      W[4 * q + e] = run;  // inclusive running sum
    }
  }
  // warp exclusive offsets of the thread totals, then the block
  const uint64_t tt = W[SCAN_PER - 1];
  const uint64_t tincl = warp_incl_scan(tt, lane);
  if (lane == 31) s_warp_tot[warp] = tincl;
  if (MODE == FROM_LOGLIK) {
    ES es;
    es.zero();
    es.add(epart);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) es.add(es.shfl_xor(o));
    if (lane == 0) s_es[warp] = es;
  }
  __syncthreads();
  if (warp == 0) {
    uint64_t wt = lane < WARPS ? s_warp_tot[lane] : 0;
    const uint64_t wincl = warp_incl_scan(wt, lane);
    if (lane < WARPS) s_warp_tot[lane] = wincl - wt;  // exclusive warp offsets
  }
  __syncthreads();
  // stage the tile-local inclusive prefix (padded rows of 17 words), so that
  // no per-element state is live across the look-back
  {
    const uint64_t toff = s_warp_tot[warp] + (tincl - tt);
#pragma unroll
    for (int e = 0; e < SCAN_PER; ++e) s_stage[threadIdx.x * (SCAN_PER + 1) + e] = W[e] + toff;
  }
  __syncthreads();
  if (warp == 0) {
    // tile total = last thread's staged inclusive value
    const uint64_t total = s_stage[(BLOCK - 1) * (SCAN_PER + 1) + SCAN_PER - 1];
    const uint64_t excl = lookback(stat, tile, total, &a.ctl->err, a.spin_limit, a.withhold);
    if (lane == 0) {
      s_excl = excl;
      stat_next[tile] = 0;
      if (MODE == FROM_LOGLIK) {
        ES tot = s_es[0];
        for (int w = 1; w < WARPS; ++w) tot.add(s_es[w]);
        reinterpret_cast<ES*>(a.part)[tile] = tot;
      }
    }
  }
  __syncthreads();
  const uint64_t off = s_excl;
  const uint64_t tbase = (uint64_t)tile * TILE;
  if (tbase + TILE <= a.n) {
#pragma unroll
    for (int r = 0; r < TILE / (2 * BLOCK); ++r) {
      const int q = 2 * threadIdx.x + 2 * BLOCK * r;  // even: q and q+1 share a row
      const int si = (q >> 4) * (SCAN_PER + 1) + (q & 15);
      *reinterpret_cast<ulonglong2*>(a.Q + tbase + q) =
          make_ulonglong2(s_stage[si] + off, s_stage[si + 1] + off);
    }
  } else {
    for (int q = threadIdx.x; q < TILE; q += BLOCK)
      if (tbase + q < a.n) a.Q[tbase + q] = s_stage[(q >> 4) * (SCAN_PER + 1) + (q & 15)] + off;
  }
}

// ---------------------------------------------------------------------------
// Multinomial positions: exponential spacings (Carpenter, Clifford &
// Fearnhead 1999).  E_l = floor(-log(u_l) 2^31), u_l from draw
// (seed, filter, t, l >> 2, SPACING) word l & 3; S = inclusive scan of E over
// l = 0..n-1 by the same look-back scan, and S[n] = S[n-1] + E_n.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t spacing_E(uint64_t seed, uint32_t filter, uint32_t t,
                                              uint64_t l, const U4& w) {
  const uint32_t word = (l & 3) == 0 ? w.a : (l & 3) == 1 ? w.b : (l & 3) == 2 ? w.c : w.d;
  const float u = unif_f32(word);
  const float L = det_log(u);
  const float x = -L * 0x1p31f;
  return f2u64_rz(x);
}

struct SpacingArgs {
  uint64_t* S;
  uint64_t* stat[2];
  Ctl* ctl;
  const uint32_t* t_dev;    // cycle index in device memory, or NULL
  uint32_t t_arg;
  uint64_t n;
  uint64_t seed;
  uint32_t filter;
};

static __global__ void __launch_bounds__(BLOCK, 3) k_spacing_scan(SpacingArgs a) {
  __shared__ uint32_t s_tile;
  __shared__ uint64_t s_warp_tot[WARPS];
  __shared__ uint64_t s_excl;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_tile = atomicAdd(&a.ctl->ticket_e, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint32_t t = a.t_dev ? *a.t_dev : a.t_arg;
  const uint64_t wbase = (uint64_t)tile * TILE + (uint64_t)warp * (CHUNKS * CHUNK);
  uint64_t W[CHUNKS][4];
#pragma unroll
  for (int c = 0; c < CHUNKS; ++c) {
    const uint64_t i0 = wbase + (uint64_t)c * CHUNK + 4 * lane;  // multiple of 4
    const U4 w = draw(a.seed, a.filter, t, (uint32_t)(i0 >> 2), P_SPACING, 0);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      uint64_t v = 0;
      if (i0 + e < a.n) {
        const uint32_t word = e == 0 ? w.a : e == 1 ? w.b : e == 2 ? w.c : w.d;
        const float u = unif_f32(word);
        const float L = det_log(u);
        const float x = -L * 0x1p31f;
        v = f2u64_rz(x);
      }
      W[c][e] = v;
    }
  }
  uint64_t carry = 0;
#pragma unroll
  for (int c = 0; c < CHUNKS; ++c) {
    W[c][1] += W[c][0];
    W[c][2] += W[c][1];
    W[c][3] += W[c][2];
    const uint64_t incl = warp_incl_scan(W[c][3], lane);
    const uint64_t excl_l = incl - W[c][3] + carry;
#pragma unroll
    for (int e = 0; e < 4; ++e) W[c][e] += excl_l;
    carry += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (lane == 0) s_warp_tot[warp] = carry;
  __syncthreads();
  if (warp == 0) {
    uint64_t wt = lane < WARPS ? s_warp_tot[lane] : 0;
    const uint64_t wincl = warp_incl_scan(wt, lane);
    if (lane < WARPS) s_warp_tot[lane] = wincl - wt;
    const uint64_t total = __shfl_sync(0xffffffffu, wincl, 31);
    uint64_t* const stat = (t & 1u) ? a.stat[1] : a.stat[0];
    uint64_t* const stat_next = (t & 1u) ? a.stat[0] : a.stat[1];
    const uint64_t excl = lookback(stat, tile, total, &a.ctl->err);
    if (lane == 0) {
      s_excl = excl;
      stat_next[tile] = 0;
    }
  }
  __syncthreads();
  const uint64_t off = s_excl + s_warp_tot[warp];
#pragma unroll
  for (int c = 0; c < CHUNKS; ++c) {
    const uint64_t i0 = wbase + (uint64_t)c * CHUNK + 4 * lane;
    if (i0 + 4 <= a.n) {
      *reinterpret_cast<ulonglong2*>(a.S + i0) = make_ulonglong2(W[c][0] + off, W[c][1] + off);
      *reinterpret_cast<ulonglong2*>(a.S + i0 + 2) = make_ulonglong2(W[c][2] + off, W[c][3] + off);
    }
    if (i0 + 4 > a.n) {
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (i0 + e < a.n) a.S[i0 + e] = W[c][e] + off;
    }
  }
  // S[n] = S[n-1] + E_n, by the thread holding element n-1
  const uint64_t last = a.n - 1;
  const uint64_t lb = last - wbase;  // position of n-1 in this warp's 512 elements
  if (last >= wbase && lb < CHUNKS * CHUNK && ((lb % CHUNK) >> 2) == (uint64_t)lane) {
    const int c = (int)(lb / CHUNK), e = (int)(lb & 3);
    uint64_t v = 0;
#pragma unroll
    for (int cc = 0; cc < CHUNKS; ++cc)
#pragma unroll
      for (int ee = 0; ee < 4; ++ee)
        if (cc == c && ee == e) v = W[cc][ee];
    const uint64_t ln = a.n;
    const U4 w = draw(a.seed, a.filter, t, (uint32_t)(ln >> 2), P_SPACING, 0);
    a.S[ln] = v + off + spacing_E(a.seed, a.filter, t, ln, w);
  }
}

// ---------------------------------------------------------------------------
// Resampling by merge (paper Section 3.1, multinomial with sorted uniforms;
// systematic): the merged order of the CDF keys KQ_i = Q_i * A and the
// position keys KB_j is cut into equal diagonals (merge path, Green, McColl
// & Bader 2012).  Each CTA finds its two diagonal splits with a warp-wide
// 32-ary search, stages both key ranges in shared memory and merges.
// Ties go to the CDF (Q_i * A <= B_j means particle i lies below slot j).
// ---------------------------------------------------------------------------
enum PosKind { POS_MULTINOMIAL = 0, POS_SYSTEMATIC = 1 };

struct PosArgs {
  const uint64_t* Q;
  const uint64_t* S;      // multinomial: spacing prefix, n+1 entries
  uint32_t* anc;
  const uint32_t* I;      // cut-point table (cut-point kernels)
  Ctl* ctl;
  const uint32_t* t_dev;
  uint32_t t_arg;
  uint64_t n;
  uint64_t seed;
  uint32_t filter;
  // adaptive resampling: when set and *gate == 0 this cycle does not
  // resample, and the resampling kernels return at once (NULL: always run)
  const uint32_t* gate;
};

__device__ __forceinline__ bool gated_off(const PosArgs& a) { return a.gate && *a.gate == 0u; }

template <int POS>
struct PosKeys {
  const uint64_t* Q;
  const uint64_t* S;
  uint64_t n, T, A, r;
  __device__ __forceinline__ U128 kq(uint64_t i) const {
    if (POS == POS_SYSTEMATIC) return mul64x32(Q[i], (uint32_t)A);  // A = n < 2^32
    return mul64(Q[i], A);
  }
  __device__ __forceinline__ U128 kb(uint64_t j) const {
    if (POS == POS_SYSTEMATIC) return add128(mul64x32(T, (uint32_t)j), r);
    return mul64(S[j], T);
  }
};

template <int POS>
__device__ __forceinline__ PosKeys<POS> make_keys(const PosArgs& a) {
  PosKeys<POS> K;
  K.Q = a.Q;
  K.S = a.S;
  K.n = a.n;
  K.T = a.Q[a.n - 1];
  const uint32_t t = a.t_dev ? *a.t_dev : a.t_arg;
  if (POS == POS_SYSTEMATIC) {
    K.A = a.n;
    const U4 w = draw(a.seed, a.filter, t, 0, P_SYS_OFFSET, 0);
    const uint64_t R = ((uint64_t)w.b << 32) | w.a;
    K.r = __umul64hi(R, K.T);
  } else {
    K.A = a.S[a.n];
    K.r = 0;
  }
  return K;
}

// Number of CDF elements among the first d merged elements, by warp-wide
// 32-ary search.  P(i) = (KQ_{i-1} <= KB_{d-i}) is true then false in i.
template <int POS>
__device__ __forceinline__ uint64_t warp_split(const PosKeys<POS>& K, uint64_t d) {
  const int lane = threadIdx.x & 31;
  uint64_t lo = d > K.n ? d - K.n : 0;
  uint64_t hi = d < K.n ? d : K.n;
  while (hi > lo) {
    const uint64_t span = hi - lo;
    const uint64_t q = lo + 1 + (span * (uint64_t)lane) / 32;
    const bool p = le128(K.kq(q - 1), K.kb(d - q));
    const uint32_t m = __ballot_sync(0xffffffffu, p);
    if (m == 0) {
      hi = lo;
    } else {
      const int kstar = 31 - __clz(m);  // trues form a prefix: last true lane
      const uint64_t qk = __shfl_sync(0xffffffffu, q, kstar);
      const uint64_t qn = __shfl_sync(0xffffffffu, q, kstar < 31 ? kstar + 1 : 31);
      lo = qk;
      if (kstar < 31) hi = qn - 1;
    }
  }
  return lo;
}

// Merge-path partition: the split of diagonal d = c * MERGE_D, one warp per
// split, all splits searched concurrently.  Block 0 also publishes the key
// constants (T, A, r) for k_merge.
template <int POS>
__global__ void __launch_bounds__(BLOCK) k_partition(PosArgs a, uint64_t* splits,
                                                     uint32_t nsplits, uint32_t tile) {
  if (gated_off(a)) return;
  const PosKeys<POS> K = make_keys<POS>(a);
  const int lane = threadIdx.x & 31;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.ctl->keyT = K.T;
    a.ctl->keyA = K.A;
    a.ctl->keyR = K.r;
  }
  const uint32_t wid = (uint32_t)(((uint64_t)blockIdx.x * BLOCK + threadIdx.x) >> 5);
  if (wid >= nsplits) return;  // uniform per warp
  const uint64_t total = 2 * a.n;
  const uint64_t d = (uint64_t)wid * tile < total ? (uint64_t)wid * tile : total;
  uint64_t sp;
  if (K.T == 0 || K.A == 0) {
    sp = d < a.n ? d : a.n;  // empty CDF: any monotone split; k_merge flags it
  } else {
    sp = warp_split<POS>(K, d);
  }
  if (lane == 0) splits[wid] = sp;
}

template <int POS>
__global__ void __launch_bounds__(BLOCK) k_merge(PosArgs a, const uint64_t* splits) {
  if (gated_off(a)) return;
  __shared__ U128 s_key[MERGE_D];
  PosKeys<POS> K;
  K.Q = a.Q;
  K.S = a.S;
  K.n = a.n;
  K.T = a.ctl->keyT;
  K.A = a.ctl->keyA;
  K.r = a.ctl->keyR;
  if (K.T == 0 || K.A == 0) {  // empty CDF: flag, keep every index in range
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&a.ctl->err, ERR_NUMERIC);
    for (uint64_t j = (uint64_t)blockIdx.x * BLOCK + threadIdx.x; j < a.n;
         j += (uint64_t)gridDim.x * BLOCK)
      a.anc[j] = (uint32_t)j;
    return;
  }
  const uint64_t total = 2 * a.n;
  const uint64_t d0 = (uint64_t)blockIdx.x * MERGE_D;
  const uint64_t d1 = d0 + MERGE_D < total ? d0 + MERGE_D : total;
  const uint64_t i0 = splits[blockIdx.x], i1 = splits[blockIdx.x + 1];
  const uint64_t j0 = d0 - i0, j1 = d1 - i1;
  const int nA = (int)(i1 - i0), nB = (int)(j1 - j0);
  for (int e = threadIdx.x; e < nA; e += BLOCK) s_key[e] = K.kq(i0 + e);
  for (int e = threadIdx.x; e < nB; e += BLOCK) s_key[nA + e] = K.kb(j0 + e);
  __syncthreads();
  // this thread's diagonal range within the CTA's merge
  const int dl0 = threadIdx.x * MERGE_E;
  const int len = nA + nB;
  if (dl0 >= len) return;
  const int dl1 = dl0 + MERGE_E < len ? dl0 + MERGE_E : len;
  // local split on diagonal dl0: largest ia with ia == lo or A[ia-1] <= B[dl0-ia]
  int lo = dl0 > nB ? dl0 - nB : 0;
  int hi = dl0 < nA ? dl0 : nA;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (le128(s_key[mid - 1], s_key[nA + dl0 - mid])) lo = mid;
    else hi = mid - 1;
  }
  int ia = lo, jb = dl0 - lo;
  for (int d = dl0; d < dl1; ++d) {
    const bool takeA = jb >= nB || (ia < nA && le128(s_key[ia], s_key[nA + jb]));
    if (takeA) {
      ++ia;
    } else {
      const uint64_t an = i0 + ia;  // < n whenever T > 0
      a.anc[j0 + jb] = (uint32_t)(an < a.n ? an : a.n - 1);
      ++jb;
    }
  }
}

// ---------------------------------------------------------------------------
// Systematic resampling by a per-thread walk.  Slot j's key is j T + r
// (A = n), so slots are equally spaced and particle i owns the slots
// [R_{i-1}, R_i) with R_i = #{j : j T + r < n Q_i}.  Each CTA takes one
// merge-path tile (particles [i0, i1), slots [j0, j1), j0 <= R_i <= j1 for
// its particles).  Thread t walks 16 consecutive particles: it finds its
// first slot once (a division by T through a 64-bit reciprocal), then emits
// a_j = i while j T + r < n Q_i, stepping the key by T.  A particle owning
// more than SYS_CAP slots records a run that the whole CTA fills.  The
// ancestors are staged in shared memory and written out coalesced.
// ---------------------------------------------------------------------------
constexpr int SYS_D = 8192;
constexpr int SYS_THREADS = 512;
constexpr int SYS_PER = 16;      // particles per thread (SYS_D / SYS_THREADS)
constexpr int SYS_CAP = 8;       // slots emitted one by one per particle
constexpr int SYS_MAX_RUNS = SYS_D / SYS_CAP + 2;
constexpr int BB_RUNS = 512;     // k_cdf_sys: runs per tile held in shared memory

__device__ __forceinline__ U128 sub128(U128 x, uint64_t y) {
  return U128{x.hi - (x.lo < y ? 1ull : 0ull), x.lo - y};
}
__device__ __forceinline__ U128 sub128(U128 x, U128 y) {
  return U128{x.hi - y.hi - (x.lo < y.lo ? 1ull : 0ull), x.lo - y.lo};
}

struct SysDiv {      // reciprocal of T for quotients below 2^32
  uint64_t T, m;     // m = floor((2^64 - 1) / (T >> s))
  int s;             // T >> s lies in [2^31, 2^32) (s = 0 if T < 2^32)
};
__device__ __forceinline__ SysDiv make_sysdiv(uint64_t T) {
  SysDiv d;
  d.T = T;
  const int bits = 64 - __clzll((long long)T);
  d.s = bits > 32 ? bits - 32 : 0;
  d.m = 0xffffffffffffffffull / (T >> d.s);
  return d;
}
// floor(Z / T) for Z < T * 2^32: reciprocal estimate, exact correction.
__device__ __forceinline__ uint64_t sys_floor_div(U128 Z, const SysDiv& d) {
  const uint64_t zs = d.s ? ((Z.lo >> d.s) | (Z.hi << (64 - d.s))) : Z.lo;
  uint64_t q = __umul64hi(zs, d.m);
  U128 P = mul64(q, d.T);
  for (int it = 0; it < 8 && lt128(Z, P); ++it) {
    --q;
    P = sub128(P, d.T);
  }
  for (int it = 0; it < 8; ++it) {
    const U128 P1 = add128(P, d.T);
    if (lt128(Z, P1)) break;
    ++q;
    P = P1;
  }
  return q;
}
// R(Q) = #{j in [0, n) : j T + r < n Q} = clamp(ceil((n Q - r) / T), 0, n).
__device__ __forceinline__ uint64_t sys_first_slot(uint64_t Qi, uint64_t n, uint64_t r,
                                                   const SysDiv& d) {
  const U128 X = mul64x32(Qi, (uint32_t)n);
  if (le128(X, U128{0, r})) return 0;
  const U128 Z = sub128(sub128(X, r), 1ull);  // ceil(Y/T) = floor((Y-1)/T) + 1
  const uint64_t q = sys_floor_div(Z, d) + 1;
  return q < n ? q : n;
}

// Stratified resampling (Section 3.1, one uniform in each of the n equal
// strata): slot j's position is P_j = j T + r_j with its own r_j in [0, T),
// r_j = floor(R_j T / 2^64) from word pair 2 (j mod 2), 2 (j mod 2) + 1 of the
// draw (seed, filter, t, floor(j/2), STRATIFIED); slot j goes to the particle
// i with n Q_{i-1} <= P_j < n Q_i.
__device__ __forceinline__ uint64_t strat_offset(uint64_t T, uint64_t seed, uint32_t filter,
                                                 uint32_t t, uint64_t j) {
  const U4 w = draw(seed, filter, t, (uint32_t)(j >> 1), P_STRATIFIED, 0);
  const uint64_t R = (j & 1) ? (((uint64_t)w.d << 32) | w.c) : (((uint64_t)w.b << 32) | w.a);
  return __umul64hi(R, T);
}
// #{j : P_j < n q}: with c = floor(n q / T), P_c is the only position in
// [c T, c T + T), so the count is c or c + 1.
__device__ __forceinline__ uint64_t strat_first(uint64_t q, uint64_t n, uint64_t T, const SysDiv& dv,
                                                uint64_t seed, uint32_t filter, uint32_t t) {
  const U128 X = mul64x32(q, (uint32_t)n);
  if (X.hi == 0 && X.lo == 0) return 0;
  const uint64_t c = sys_floor_div(X, dv);  // X <= n T < 2^32 T
  if (c >= n) return n;
  const U128 P = add128(mul64x32(T, (uint32_t)c), strat_offset(T, seed, filter, t, c));
  return lt128(P, X) ? c + 1 : c;
}
// One thread per particle: particle i owns the slots [first(n Q_{i-1}),
// first(n Q_i)); the lower end comes from the neighbouring lane.  A warp
// stores the ranges longer than 32 slots together.
static __global__ void __launch_bounds__(BLOCK) k_strat(PosArgs a) {
  if (gated_off(a)) return;
  const uint64_t n = a.n;
  const uint32_t t = a.t_dev ? *a.t_dev : a.t_arg;
  const uint64_t T = a.Q[n - 1];
  const uint64_t i = (uint64_t)blockIdx.x * BLOCK + threadIdx.x;
  const int lane = threadIdx.x & 31;
  if (T == 0) {  // empty CDF (flagged): keep every index in range
    if (i == 0) atomicOr(&a.ctl->err, ERR_NUMERIC);
    if (i < n) a.anc[i] = (uint32_t)i;
    return;
  }
  const SysDiv dv = make_sysdiv(T);
  const uint64_t j1 = i < n ? strat_first(a.Q[i], n, T, dv, a.seed, a.filter, t) : n;
  uint64_t j0 = __shfl_up_sync(0xffffffffu, j1, 1);
  if (lane == 0) j0 = i == 0 ? 0 : (i < n ? strat_first(a.Q[i - 1], n, T, dv, a.seed, a.filter, t) : n);
  const uint64_t cnt = i < n ? j1 - j0 : 0;
  if (cnt <= 32) {
    for (uint64_t q = j0; q < j0 + cnt; ++q) a.anc[q] = (uint32_t)i;
  }
  uint32_t heavy = __ballot_sync(0xffffffffu, cnt > 32);
  while (heavy) {
    const int l = __ffs(heavy) - 1;
    heavy &= heavy - 1;
    const uint64_t s0 = __shfl_sync(0xffffffffu, j0, l), s1 = __shfl_sync(0xffffffffu, j1, l);
    const uint32_t v = (uint32_t)__shfl_sync(0xffffffffu, i, l);
    for (uint64_t q = s0 + lane; q < s1; q += 32) a.anc[q] = v;
  }
}

static __global__ void __launch_bounds__(SYS_THREADS) k_merge_sys(PosArgs a, const uint64_t* splits) {
  if (gated_off(a)) return;
  __shared__ uint32_t s_anc[SYS_D];
  __shared__ uint32_t s_run[SYS_MAX_RUNS][3];
  __shared__ uint32_t s_nruns;
  const uint64_t T = a.ctl->keyT, r = a.ctl->keyR, n = a.n;
  if (T == 0) {  // empty CDF: flag, keep every index in range
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&a.ctl->err, ERR_NUMERIC);
    for (uint64_t j = (uint64_t)blockIdx.x * SYS_THREADS + threadIdx.x; j < n;
         j += (uint64_t)gridDim.x * SYS_THREADS)
      a.anc[j] = (uint32_t)j;
    return;
  }
  const uint64_t total = 2 * n;
  const uint64_t d0 = (uint64_t)blockIdx.x * SYS_D;
  const uint64_t d1 = d0 + SYS_D < total ? d0 + SYS_D : total;
  const uint64_t i0 = splits[blockIdx.x], i1 = splits[blockIdx.x + 1];
  const uint64_t j0 = d0 - i0, j1 = d1 - i1;
  const uint32_t nB = (uint32_t)(j1 - j0);
  if (threadIdx.x == 0) s_nruns = 0;
  __syncthreads();
  const SysDiv dv = make_sysdiv(T);
  auto add_run = [&](uint64_t st, uint64_t en, uint64_t val) {
    const uint32_t k = atomicAdd(&s_nruns, 1u);
    if (k < SYS_MAX_RUNS) {
      s_run[k][0] = (uint32_t)(st - j0);
      s_run[k][1] = (uint32_t)(en - j0);
      s_run[k][2] = (uint32_t)val;
    }
  };
  if (i0 == i1) {
    if (threadIdx.x == 0 && nB) add_run(j0, j1, i0);  // every slot belongs to particle i0
  } else {
    const uint64_t ib = i0 + (uint64_t)threadIdx.x * SYS_PER;
    if (ib < i1) {
      const uint64_t ie = ib + SYS_PER < i1 ? ib + SYS_PER : i1;
      uint64_t j = threadIdx.x == 0 ? j0 : sys_first_slot(a.Q[ib - 1], n, r, dv);
      j = j < j0 ? j0 : (j > j1 ? j1 : j);
      U128 KB = add128(mul64x32(T, (uint32_t)j), r);
      for (uint64_t i = ib; i < ie; ++i) {
        const uint64_t qi = a.Q[i];
        const U128 KQ = mul64x32(qi, (uint32_t)n);
        int emitted = 0;
        while (j < j1 && lt128(KB, KQ)) {
          if (emitted == SYS_CAP) {  // a heavy particle: jump to its last slot
            uint64_t R = sys_first_slot(qi, n, r, dv);
            R = R < j ? j : (R > j1 ? j1 : R);
            add_run(j, R, i);
            j = R;
            KB = add128(mul64x32(T, (uint32_t)j), r);
            break;
          }
          s_anc[j - j0] = (uint32_t)i;
          ++j;
          KB = add128(KB, T);
          ++emitted;
        }
      }
      if (ie == i1 && j < j1) add_run(j, j1, i1);  // remaining slots belong to particle i1
    }
  }
  __syncthreads();
  const uint32_t nr = s_nruns < SYS_MAX_RUNS ? s_nruns : SYS_MAX_RUNS;
  if (s_nruns > SYS_MAX_RUNS && threadIdx.x == 0) atomicOr(&a.ctl->err, ERR_NUMERIC);
  for (uint32_t k = 0; k < nr; ++k) {
    const uint32_t st = s_run[k][0], en = s_run[k][1], v = s_run[k][2];
    for (uint32_t q = st + threadIdx.x; q < en; q += SYS_THREADS) s_anc[q] = v;
  }
  __syncthreads();
  for (uint32_t q = threadIdx.x; q < nB; q += SYS_THREADS) {
    const uint32_t v = s_anc[q];
    a.anc[j0 + q] = v < n ? v : (uint32_t)(n - 1);
  }
}

// ---------------------------------------------------------------------------
// The paper's Section 3.2 algorithms.
// Parallelized Cut-Point Search: thread i computes L_i = ceil(n Q_i / T) and
// writes I_k = i for L_{i-1} <= k < L_i.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t ceil_nq_over_t(uint64_t n, uint64_t q, uint64_t T) {
  const U128 X = mul64(n, q);
  const uint64_t f = div128_small(X, T);
  const U128 p = mul64(f, T);
  return (p.hi == X.hi && p.lo == X.lo) ? f : f + 1;
}

static __global__ void __launch_bounds__(BLOCK) k_cutpoint_search(const uint64_t* Q, uint64_t n,
                                                           uint32_t* I) {
  const uint64_t i = (uint64_t)blockIdx.x * BLOCK + threadIdx.x;
  if (i >= n) return;
  const uint64_t T = Q[n - 1];
  if (T == 0) {
    I[i] = (uint32_t)i;
    return;
  }
  uint64_t Li = ceil_nq_over_t(n, Q[i], T);
  uint64_t Lp = i == 0 ? 0 : ceil_nq_over_t(n, Q[i - 1], T);
  Li = Li < n ? Li : n;  // L_i <= n whenever Q_i <= T
  Lp = Lp < n ? Lp : n;
  for (uint64_t k = Lp; k < Li; ++k) I[k] = (uint32_t)i;
}

// Parallelized Cut-Point Method for the scheme's positions: bucket b_j
// (systematic: j; multinomial: floor(n S_j / S_n)), start at I_{b_j}, climb
// while KQ_k <= KB_j.
template <int POS>
__global__ void __launch_bounds__(BLOCK) k_cutpoint_method(PosArgs a) {
  if (gated_off(a)) return;
  const uint64_t j = (uint64_t)blockIdx.x * BLOCK + threadIdx.x;
  if (j >= a.n) return;
  const PosKeys<POS> K = make_keys<POS>(a);
  if (K.T == 0 || K.A == 0) {
    if (j == 0) atomicOr(&a.ctl->err, ERR_NUMERIC);
    a.anc[j] = (uint32_t)j;
    return;
  }
  uint64_t b = j;
  if (POS == POS_MULTINOMIAL) b = div128_small(mul64(a.n, a.S[j]), K.A);
  uint64_t k = a.I[b < a.n ? b : a.n - 1];
  const U128 kb = K.kb(j);
  while (k < a.n && le128(K.kq(k), kb)) ++k;
  a.anc[j] = (uint32_t)(k < a.n ? k : a.n - 1);
}

// Explicit integer positions U_j in [0, T) (A = 1).
static __global__ void __launch_bounds__(BLOCK) k_cutpoint_method_explicit(
    const uint64_t* Q, uint64_t n, const uint32_t* I, const uint64_t* U, uint64_t m,
    uint32_t* anc) {
  const uint64_t j = (uint64_t)blockIdx.x * BLOCK + threadIdx.x;
  if (j >= m) return;
  const uint64_t T = Q[n - 1];
  const uint64_t u = U[j];
  const uint64_t b = T ? div128_small(mul64(n, u), T) : 0;
  uint64_t k = I[b < n ? b : n - 1];
  while (k < n && Q[k] <= u) ++k;
  anc[j] = (uint32_t)(k < n ? k : n - 1);
}

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (TMA, cp.async.bulk) into shared memory, completed
// on an mbarrier.  Waits are bounded: after SPIN_LIMIT polls they report
// failure instead of hanging.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// make the barrier initialisation visible to the async proxy
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// order this thread's earlier shared-memory accesses before later async-proxy ones
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// copy `bytes` (a multiple of 16; both addresses 16-byte aligned) from global
// to shared memory, completing on `bar`, which expects exactly these bytes
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes,
                                            uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
               ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t addr = smem_u32(bar);
  for (uint32_t i = 0; i < SPIN_LIMIT; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done) : "r"(addr), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}

// copy `bytes` (a multiple of 16; both addresses 16-byte aligned) from
// shared to global memory as one bulk async-group
__device__ __forceinline__ void tma_store_1d(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;"
               ::"l"(dst), "r"(smem_u32(src)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// wait until this thread's bulk stores have read their shared-memory source
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// wait until all but the most recent of this thread's bulk store groups
// have read their shared-memory source
__device__ __forceinline__ void bulk_wait_read1() {
  asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
}
// wait until this thread's bulk stores are complete
__device__ __forceinline__ void bulk_wait_done() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// W = min(floor(e 2^k), 2^k) from e = exp(dl) as quant_exp returns it: e is
// 0 or a normal number p 2^n, so e 2^k and p 2^(n + k) have the same bits
// and the floor is the one quant_exp takes.
__device__ __forceinline__ uint64_t quant_from_e(float e, int k) {
  uint64_t W = 0;
  if (e != 0.0f) {
    const uint32_t eb = __float_as_uint(e);
    const int sh = (int)(eb >> 23) - 150 + k;
    const uint32_t m24 = (eb & 0x7fffffu) | 0x800000u;
    W = sh >= 0 ? ((uint64_t)m24 << sh) : (uint64_t)(m24 >> (-sh < 31 ? -sh : 31));
  }
  const uint64_t cap = 1ull << k;
  return W > cap ? cap : W;
}
__device__ __forceinline__ uint64_t quant_from_e(double e, int k) {
  const uint64_t W = e != 0.0 ? f2u64_rz(e * pow2d(k)) : 0ull;
  const uint64_t cap = 1ull << k;
  return W > cap ? cap : W;
}

// The systematic resampling step writes each particle's slots into a
// shared-memory window (an entry per slot of the tile, the particle's offset
// in the tile + 1; the window starts at the tile's first slot rounded down to
// a multiple of four).  Entry of slot x: x with bits 1-3 XORed by bits 6-8, so
// that threads writing slots about PER apart, and warps reading consecutive
// slots, hit distinct banks.  The four slots 4g .. 4g + 3 keep one aligned
// group of four entries (in the order 0 1 2 3, or 2 3 0 1 when bit 1 is
// flipped), so the window is read out four slots per 8-byte load.
__device__ __forceinline__ uint32_t win_entry(uint32_t x) { return x ^ (((x >> 6) & 7u) << 1); }
// A run of the CTA's run list: slots [s0, s1) of ancestor v; with WRUN set in
// v, window slots (relative to the tile's first slot) of mark v & 0xffff.
constexpr uint32_t WRUN = 0x80000000u;

// Rare paths of the systematic resampling step, kept out of line so that the
// per-particle loop stays small: the slot count of a heavy particle (more than
// three slots), and the slots of a particle that its `inl` in-line window
// writes did not cover -- the rest of a heavy particle's run in the window
// (by the whole CTA when long) and slots past the window (stored directly, or
// by the whole CTA when long).
static __device__ __noinline__ uint32_t sys_heavy_count(int64_t D, SysDiv dv) {
  return (uint32_t)(sys_floor_div(U128{0, (uint64_t)D - 1}, dv) + 1);
}
static __device__ __noinline__ void sys_rest(uint32_t j, uint32_t c, uint32_t S0, uint32_t wslots,
                                             uint16_t mk, uint32_t ig, uint16_t* win, uint32_t* anc,
                                             uint32_t (*runs)[3], uint32_t* nruns, uint32_t inl = 2u) {
  const uint32_t wend = S0 + wslots, e = j + c;
  const uint32_t a = j + inl < e ? j + inl : e;  // window part [a, b)
  const uint32_t b = e < wend ? e : wend;
  if (b > a) {
    bool queued = false;
    if (b - a > (uint32_t)SYS_CAP) {
      const uint32_t kr = atomicAdd(nruns, 1u);
      if (kr < BB_RUNS) {
        runs[kr][0] = a - S0;
        runs[kr][1] = b - S0;
        runs[kr][2] = WRUN | mk;
        queued = true;
      }
    }
    if (!queued)
      for (uint32_t q = a; q < b; ++q) win[win_entry(q - S0)] = mk;
  }
  const uint32_t st = j > wend ? j : wend;  // past the window: [st, e)
  if (e > st) {
    if (e - st > (uint32_t)SYS_CAP) {
      const uint32_t kr = atomicAdd(nruns, 1u);
      if (kr < BB_RUNS) {
        runs[kr][0] = st;
        runs[kr][1] = e;
        runs[kr][2] = ig;
        return;
      }
    }
    for (uint32_t q = st; q < e; ++q) anc[q] = ig;
  }
}

// Correctly rounded conversion of a 128-bit integer to binary64: the top 64
// significant bits with a sticky bit for the rest, rounded once, scaled by an
// exact power of two.
__device__ __forceinline__ double u128_to_f64_rn(U128 v) {
  if (v.hi == 0) return __ull2double_rn(v.lo);
  const int lz = __clzll(v.hi);
  const int sh = 64 - lz;  // 1..64
  uint64_t top, rest;
  if (lz == 0) {
    top = v.hi;
    rest = v.lo;
  } else {
    top = (v.hi << lz) | (v.lo >> sh);
    rest = v.lo << lz;
  }
  const double d = __ull2double_rn(top | (rest != 0 ? 1ull : 0ull));
  return d * __longlong_as_double((long long)(1023 + sh) << 52);
}

// ---------------------------------------------------------------------------
// The CDF and systematic resampling in one cooperative launch (Steps 1b-1c
// of the cycle for the systematic scheme).  Every CTA owns a contiguous range
// of tiles of BLOCK x PER particles (thread t: particles [PER t, PER t + PER)):
//   phase 1  the exact sum of its quantised weights W_i;
//   barrier  all CTAs (the launch is cooperative, so all are resident; the
//            wait is bounded and reports ERR_TIMEOUT);
//   phase 2  its exclusive prefix and T from the CTA sums, then for each of
//            its tiles the block scan of W with a carry -- thread t holds
//            Q_i for its particles and Q before them in registers -- the CDF
//            written out, and systematic resampling from those registers:
//            each particle writes its slots into a shared-memory window, which
//            the CTA then stores out coalesced.
// The quantisation and the log-ML partials (sums over 16 consecutive
// particles in a fixed order; with PER = 8 a lane pair shares one) are those
// of k_scan, and the ancestors those of k_merge_sys: the results are the same
// bits.  Instead of a look-back over tiles in flight, one grid-wide barrier.
// PER = 8 (binary32) doubles the CTAs for the same particles where one tile
// per CTA fits at once; the binary32 tile partials are exact, so the tile
// size does not change them.
// ---------------------------------------------------------------------------
// STAGED: a CTA owns several tiles, copied by TMA into shared memory ahead of
// use.  Phase 1 streams l through a ring of NB1 buffers (NB1 - 1 tiles in
// flight: phase 1 is bound by the bytes in flight, and the CDF rows' space
// is free until phase 2) and writes e = exp(l - m) back in l's place by bulk
// stores, so phase 2 needs no exponentials; phase 2 reads e through a double
// buffer; the CDF goes out through shared-memory rows, coalesced.  Otherwise
// (one tile per CTA) l is read directly and the tile's W stay in shared
// memory between the phases.
//
// With ESS (adaptive resampling) phase 1 also sums W^2 exactly per CTA
// (cta_sq); after the grid barrier every CTA takes k_ess's decision from the
// totals, CTA 0 publishes it, and a cycle that does not resample writes the
// CDF and the log-ML partials but no ancestors.
template <class R, bool STAGED, int PER, bool ESS = false>
__global__ void __launch_bounds__(BLOCK, PER == 8 ? 4 : 3) k_cdf_sys(FilterArgs<R> a, uint64_t* cta_tot,
                                                                    U128* cta_sq) {
  static_assert(PER == 16 || (PER == 8 && !STAGED && sizeof(R) == 4), "tile shapes");
  // staged: phase 1 writes e = exp(l - m) back in l's place and phase 2
  // quantises from e (no second exponential); with ESS, or without
  // write-back, phase 2 quantises from l again
  constexpr bool WB = STAGED && !ESS;
  constexpr int TP = BLOCK * PER;  // particles per tile
  typedef typename ESumT<R>::T ES;
  __shared__ uint64_t s_warp[WARPS + 1];
  __shared__ uint64_t s_pre2[WARPS];
  __shared__ ES s_es[WARPS];
  __shared__ uint64_t s_bc[2];
  __shared__ uint32_t s_run[BB_RUNS][3];
  __shared__ uint32_t s_nruns;
  // one tile per CTA: the tile's quantised weights and log-ML partials, kept
  // from phase 1 for phase 2 (the CTA quantises once).  Staged: phase 1 uses
  // this space as further TMA buffers and phase 2 as the rows of the CDF.
  __shared__ alignas(128) uint64_t s_keep[BLOCK * (PER + 1)];
  __shared__ R s_keep_ep[STAGED ? 1 : BLOCK];
  // staged: l (phase 1) or e (phase 2) of the next tiles arrives by TMA while
  // the CTA works on the current one; in phase 2 the buffer of the current
  // tile, once quantised, is the tile's ancestor window (see below)
  __shared__ alignas(128) R s_ell[2][STAGED ? TP : 4];
  __shared__ alignas(16) uint16_t s_win[STAGED ? 8 : 2 * TP];
  // phase 1's ring of NB1 buffers (s_ell[0], s_ell[1], then s_keep), so that
  // NB1 - 1 tiles are in flight while one is quantised: four 16 KB tiles in
  // binary32, three 32 KB tiles in binary64; phase 2's ring is s_ell
  constexpr int NB1 = STAGED ? 2 + (int)(sizeof(uint64_t) * BLOCK * (PER + 1) / (sizeof(R) * TP)) : 1;
  __shared__ alignas(8) uint64_t s_bar[NB1 + 2];
  __shared__ uint32_t s_S[2];  // the tile's first slot and the slot after its last
  __shared__ U128 s_sq[ESS ? WARPS : 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Ctl* c = a.ctl;
  const uint64_t n = a.n;
  const uint32_t ntiles = (uint32_t)((n + TP - 1) / TP);
  const uint32_t per = (ntiles + gridDim.x - 1) / gridDim.x;
  const uint32_t tb = blockIdx.x * per < ntiles ? blockIdx.x * per : ntiles;
  const uint32_t te = tb + per < ntiles ? tb + per : ntiles;
  const uint32_t t = c->t;
  R m;
  if constexpr (sizeof(R) == 4) m = dec_f((uint32_t)c->maxenc);
  else m = dec_d(c->maxenc);
  const int k = a.k;
  // TMA rings (staged).  Phase 1: the CTA's tile i goes to ring buffer
  // i % NB1 with barrier i % NB1; phase 2: tile i to s_ell[i & 1] with
  // barrier NB1 + (i & 1).  The k-th copy through a barrier completes its
  // phase k, waited for with parity k & 1.
  // After a wait that gave up (s_tmo set, ERR_TIMEOUT raised) the CTA issues
  // no more copies and waits for none; its CDF and ancestors are then
  // invalid, which the error word reports.  Before the CTA exits, thread 0
  // waits once more, bounded, for every copy it issued that it has not seen
  // complete, so that no copy into this CTA's shared memory outlives it.
  __shared__ uint32_t s_tmo;
  if (threadIdx.x == 0) {
    s_tmo = 0;
    if (STAGED) {
      for (int b = 0; b < NB1 + 2; ++b) mbar_init(&s_bar[b], 1);
      mbar_init_fence();
    }
  }
  __syncthreads();
  uint32_t iss_b[NB1 + 2], ok_b[NB1 + 2];  // thread 0: copies issued / seen complete per barrier
#pragma unroll
  for (int b = 0; b < NB1 + 2; ++b) iss_b[b] = ok_b[b] = 0;
  // phase 1's ring buffer b
  auto ring1 = [&](uint32_t b) -> R* {
    return b < 2 ? s_ell[b] : reinterpret_cast<R*>(s_keep) + (b - 2) * TP;
  };
  // thread 0: copy tile `tile` of l (or e) into dst through barrier bi; dst
  // is free (any bulk store from it has read it)
  auto issue = [&](uint32_t bi, R* dst, uint32_t tile) {
    if (*(volatile uint32_t*)&s_tmo) return;
    const uint64_t first = (uint64_t)tile * TP;
    const uint64_t cnt = n - first < (uint64_t)TP ? n - first : (uint64_t)TP;
    const uint32_t bytes = (uint32_t)((cnt * sizeof(R) + 15) & ~(uint64_t)15);
    fence_proxy_async_smem();  // (phase 2: the buffer held the previous tile's window)
    tma_load_1d(dst, a.ell + first, bytes, &s_bar[bi]);
    ++iss_b[bi];
  };
  // every thread: wait for the k-th copy through barrier bi
  auto take = [&](uint32_t bi, uint32_t k) {
    if (!*(volatile uint32_t*)&s_tmo) {
      if (mbar_wait(&s_bar[bi], k & 1)) {
        if (threadIdx.x == 0) ++ok_b[bi];
      } else {
        s_tmo = 1u;
        atomicOr(&c->err, ERR_TIMEOUT);
      }
    }
  };
  auto drain_copies = [&]() {  // thread 0, at exit
    if constexpr (STAGED) {
      if (!*(volatile uint32_t*)&s_tmo) return;
      for (int b = 0; b < NB1 + 2; ++b)
        for (uint32_t k = ok_b[b]; k < iss_b[b]; ++k) (void)mbar_wait(&s_bar[b], k & 1);
    }
  };
  // this thread's 16 weights of tile `tile` quantised, as inclusive running
  // sums W, the partial sum of e = exp(l - m) and the largest e.  mode 0:
  // from l in buf; 1: from l in buf (shared memory), writing e back in its
  // place; 2: from e in buf (written back by phase 1).
  auto quantP = [&](uint32_t tile, const R* buf, uint64_t* W, R* epart, R* emx, int mode) {
    R exs[PER];
    R mx = (R)0;
    const uint64_t base = (uint64_t)tile * TP + (uint64_t)threadIdx.x * PER;
    R* const row = const_cast<R*>(buf) + threadIdx.x * PER;
    const bool full = base + PER <= n;
    uint64_t run = 0;
    R ep = (R)0;
#pragma unroll
    for (int q = 0; q < PER / 4; ++q) {
      R v[4];
      if (full) {
        if constexpr (sizeof(R) == 4) {
          const float4 f = *reinterpret_cast<const float4*>(row + 4 * q);
          v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
        } else {
          const double2 f0 = *reinterpret_cast<const double2*>(row + 4 * q);
          const double2 f1 = *reinterpret_cast<const double2*>(row + 4 * q + 2);
          v[0] = f0.x; v[1] = f0.y; v[2] = f1.x; v[3] = f1.y;
        }
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) v[e] = (base + 4 * q + e < n) ? row[4 * q + e] : (R)0;
      }
      R ex4[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        uint64_t w = 0;
        R ex = (R)0;
        if (full || base + 4 * q + e < n) {
          if (mode == 2) {
            ex = v[e];
            w = quant_from_e(ex, k);
          } else {
            const R dl = v[e] - m;
            w = quant_exp<R>(dl, k, &ex);
          }
          ep = ep + ex;
          mx = ex > mx ? ex : mx;
        }
        ex4[e] = ex;
        exs[4 * q + e] = ex;
        run += w;
        W[4 * q + e] = run;  // inclusive running sum
      }
      if (mode == 1) {
        if constexpr (sizeof(R) == 4) {
          *reinterpret_cast<float4*>(row + 4 * q) = make_float4(ex4[0], ex4[1], ex4[2], ex4[3]);
        } else {
          *reinterpret_cast<double2*>(row + 4 * q) = make_double2(ex4[0], ex4[1]);
          *reinterpret_cast<double2*>(row + 4 * q + 2) = make_double2(ex4[2], ex4[3]);
        }
      }
    }
    if constexpr (PER == 8) {
      // the log-ML partials are sums over 16 consecutive particles in
      // order: the odd lane continues the even lane's sum over its own 8
      const R prev = __shfl_xor_sync(0xffffffffu, ep, 1);
      R acc = prev;
#pragma unroll
      for (int e = 0; e < PER; ++e) acc = acc + exs[e];  // e = 0 past n: adds nothing
      ep = (threadIdx.x & 1) ? acc : (R)0;
    }
    *epart = ep;
    *emx = mx;
  };
  // block sum of one value per thread, returned to every thread
  auto block_sum = [&](uint64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_warp[warp] = v;
    __syncthreads();
    uint64_t tot = 0;
    for (int w = 0; w < WARPS; ++w) tot += s_warp[w];
    __syncthreads();
    return tot;
  };

  // block sum of one 128-bit value per thread, returned to every thread
  auto block_sum128 = [&](U128 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      U128 u;
      u.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
      u.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
      v = add128(v, u);
    }
    if (lane == 0) s_sq[warp] = v;
    __syncthreads();
    U128 tot{0, 0};
    for (int w = 0; w < WARPS; ++w) tot = add128(tot, s_sq[w]);
    __syncthreads();
    return tot;
  };

  // phase 1: this CTA's sum of W (and with ESS of W^2)
  uint64_t mine = 0;
  R emx_keep = (R)0;
  U128 sq{0, 0};
  auto add_sq = [&](const uint64_t* W) {
    if constexpr (ESS) {
      uint64_t prev = 0;
#pragma unroll
      for (int e = 0; e < PER; ++e) {
        const uint64_t w = W[e] - prev;
        prev = W[e];
        sq = add128(sq, mul64(w, w));
      }
    }
  };
  if constexpr (STAGED) {
    if (threadIdx.x == 0)
      for (uint32_t b = 0; b + 1 < (uint32_t)NB1 && tb + b < te; ++b) issue(b, ring1(b), tb + b);
    uint32_t i = 0;
    for (uint32_t tile = tb; tile < te; ++tile, ++i) {
      const uint32_t b = i % NB1;
      R* const buf = ring1(b);
      take(b, i / NB1);
      uint64_t W[PER];
      R ep;
      // (with ESS l stays in place: a propagation that does not resample
      // carries L - m from it, so phase 2 quantises from l again)
      R emx;
      quantP(tile, buf, W, &ep, &emx, WB ? 1 : 0);
      if (WB) fence_proxy_async_smem();  // e in buf, for the bulk store below
      mine += W[PER - 1];
      add_sq(W);
      __syncthreads();
      if (threadIdx.x == 0) {
        if (WB) {
          // e goes back to l's place in global memory for phase 2, which
          // then needs no exponentials
          const uint64_t first = (uint64_t)tile * TP;
          const uint64_t cnt = n - first < (uint64_t)TP ? n - first : (uint64_t)TP;
          tma_store_1d(a.ell + first, buf, (uint32_t)((cnt * sizeof(R) + 15) & ~(uint64_t)15));
        }
        if (tile + NB1 - 1 < te) {
          // the previous tile's buffer takes the tile NB1 - 1 ahead, once
          // its bulk store has read it (this tile's may still be reading)
          if (WB) bulk_wait_read1();
          const uint32_t nb = (i + NB1 - 1) % NB1;
          issue(nb, ring1(nb), tile + NB1 - 1);
        }
      }
    }
  } else {
    // at most one tile: l read directly, its W (and this thread's largest e)
    // kept for phase 2
    for (uint32_t tile = tb; tile < te; ++tile) {
      uint64_t W[PER];
      R ep;
      quantP(tile, a.ell + (uint64_t)tile * TP, W, &ep, &emx_keep, 0);
      mine += W[PER - 1];
      add_sq(W);
#pragma unroll
      for (int e = 0; e < PER; ++e) s_keep[threadIdx.x * (PER + 1) + e] = W[e];
      s_keep_ep[threadIdx.x] = ep;
    }
  }
  mine = block_sum(mine);
  if constexpr (ESS) sq = block_sum128(sq);
  if (threadIdx.x == 0) {
    st_status(&cta_tot[blockIdx.x], mine);
    if constexpr (ESS) {
      st_status(&cta_sq[blockIdx.x].hi, sq.hi);
      st_status(&cta_sq[blockIdx.x].lo, sq.lo);
    }
    __threadfence();
    atomicAdd(&c->gbar, 1u);
    if (STAGED && tb < te) {  // phase 2's first tile from HBM: e stored, complete
      bulk_wait_done();
      issue(NB1, s_ell[0], tb);
    }
    uint32_t spins = 0;
    while (ld_volatile_u32(&c->gbar) < gridDim.x) {
      if (++spins > SPIN_LIMIT) {
        atomicOr(&c->err, ERR_TIMEOUT);
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
  }
  __syncthreads();

  // phase 2: this CTA's exclusive prefix and the total T
  uint64_t pre = 0, all = 0;
  for (uint32_t b = threadIdx.x; b < gridDim.x; b += BLOCK) {
    const uint64_t v = ld_status(&cta_tot[b]);
    all += v;
    if (b < blockIdx.x) pre += v;
  }
  // both block sums in one pass (two block barriers)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    pre += __shfl_xor_sync(0xffffffffu, pre, o);
    all += __shfl_xor_sync(0xffffffffu, all, o);
  }
  if (lane == 0) {
    s_warp[warp] = pre;
    s_pre2[warp] = all;
  }
  __syncthreads();
  pre = 0;
  uint64_t T = 0;
  for (int w = 0; w < WARPS; ++w) {
    pre += s_warp[w];
    T += s_pre2[w];
  }
  __syncthreads();
  // adaptive resampling: the decision of k_ess, from the same exact sums
  bool rs = true;
  if constexpr (ESS) {
    U128 B{0, 0};
    for (uint32_t b = threadIdx.x; b < gridDim.x; b += BLOCK) {
      U128 v;
      v.hi = ld_status(&cta_sq[b].hi);
      v.lo = ld_status(&cta_sq[b].lo);
      B = add128(B, v);
    }
    B = block_sum128(B);
    const double A = __ull2double_rn(T);
    const double Bd = u128_to_f64_rn(B);
    const double lhs = A * A;
    const double f = a.ess_frac * (double)n;
    const double rhs = f * Bd;
    rs = lhs < rhs;
    if (blockIdx.x == 0 && threadIdx.x == 0) c->resamp = rs ? 1u : 0u;
  }
  const U4 wr = draw(a.seed, a.filter, t, 0, P_SYS_OFFSET, 0);
  const uint64_t r = __umul64hi(((uint64_t)wr.b << 32) | wr.a, T);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    c->keyT = T;
    c->keyA = n;
    c->keyR = r;
    if (T == 0) atomicOr(&c->err, ERR_NUMERIC);
  }
  const SysDiv dv = make_sysdiv(T > 0 ? T : 1);
  // a particle with n W_i <= 2 T owns at most two slots, and e_i <= thr
  // implies it: W_i <= e_i 2^k <= thr 2^k <= 2 T / n, every rounding of
  // thr = T (1 / n) 2^(1 - k) taken downward
  R thr;
  if constexpr (sizeof(R) == 4)
    thr = __fmul_rd(__fmul_rd(__ull2float_rd(T), __frcp_rd(__ull2float_ru(n))), pow2f(1 - k));
  else
    thr = __dmul_rd(__dmul_rd(__ull2double_rd(T), __drcp_rd((double)n)), pow2d(1 - k));
  if (threadIdx.x == 0) s_nruns = 0;
  __syncthreads();
  uint64_t carry = pre;
  uint32_t i2 = 0;
  // the log-ML partial of the CTA's tiles (thread 0)
  constexpr bool CTA_PART = STAGED && sizeof(R) == 4;
  ES cta_es;
  cta_es.zero();
  for (uint32_t tile = tb; tile < te; ++tile, ++i2) {
    uint64_t W[PER];
    R ep, emx = emx_keep;
    if constexpr (!STAGED) {  // this thread's own entries: no barrier needed
#pragma unroll
      for (int e = 0; e < PER; ++e) W[e] = s_keep[threadIdx.x * (PER + 1) + e];
      ep = s_keep_ep[threadIdx.x];
    } else {
      // the next tile into the other buffer (the previous tile's window,
      // stored out), then this one
      if (threadIdx.x == 0 && tile + 1 < te) issue(NB1 + ((i2 + 1) & 1), s_ell[(i2 + 1) & 1], tile + 1);
      take(NB1 + (i2 & 1), i2 >> 1);
      quantP(tile, s_ell[i2 & 1], W, &ep, &emx, WB ? 2 : 0);
    }
    // the tile's first slot S0 = R(carry)
    // (a later tile starts where the previous one ended: no division)
    if (threadIdx.x == 0) s_S[0] = tile == tb ? (uint32_t)sys_first_slot(carry, n, r, dv) : s_S[1];
    // The ancestors of the tile's slots [S0, S1) are built in a shared-memory
    // window of one 16-bit entry per slot (a free l buffer when staged), at
    // least two per particle of the tile, then stored out coalesced.
    constexpr uint32_t WIN_SLOTS = STAGED ? TP * sizeof(R) / 2 : 2 * TP;
    static_assert(WIN_SLOTS % 512 == 0 && WIN_SLOTS >= 2 * TP, "window");
    uint16_t* const win = STAGED ? reinterpret_cast<uint16_t*>(s_ell[i2 & 1]) : s_win;
    {
      ES es;
      es.zero();
      es.add(ep);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) es.add(es.shfl_xor(o));
      if (lane == 0) s_es[warp] = es;
    }
    // block exclusive scan of the thread totals
    const uint64_t tt = W[PER - 1];
    const uint64_t incl = warp_incl_scan(tt, lane);
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const uint64_t wt = lane < WARPS ? s_warp[lane] : 0;
      const uint64_t wi = warp_incl_scan(wt, lane);
      if (lane < WARPS) s_warp[lane] = wi - wt;
      if (lane == WARPS - 1) s_bc[0] = wi;
      if (lane == 0) {
        ES tot = s_es[0];
        for (int w = 1; w < WARPS; ++w) tot.add(s_es[w]);
        // staged binary32: one exact partial per CTA (the sum of its tiles'),
        // so that the propagation's final fold reads one per CTA
        if constexpr (CTA_PART) cta_es.add(tot);
        else reinterpret_cast<ES*>(a.part)[tile] = tot;
      }
    }
    __syncthreads();
    const uint64_t o = carry + s_warp[warp] + (incl - tt);  // Q just before this thread's particles
    const uint64_t tile_tot = s_bc[0];
    const uint64_t tbase = (uint64_t)tile * TP;
    const uint64_t base = tbase + (uint64_t)threadIdx.x * PER;
    const uint32_t S0 = s_S[0];
    const uint32_t S0a = S0 & ~3u;  // the window's base: slots in aligned groups of four
    // The CDF: this thread's values go to its shared-memory row (read by the
    // resampling step below); staged (several tiles per CTA, where the store
    // instructions add up) the rows are written out coalesced below,
    // otherwise the values are stored directly.
    uint64_t* const qrow = s_keep + threadIdx.x * (PER + 1);
#pragma unroll
    for (int e = 0; e < PER; ++e) qrow[e] = o + W[e];
    if constexpr (!STAGED) {
      if (base + PER <= n) {
#pragma unroll
        for (int e = 0; e < PER; e += 2)
          *reinterpret_cast<ulonglong2*>(a.Q + base + e) = make_ulonglong2(o + W[e], o + W[e + 1]);
      } else {
#pragma unroll
        for (int e = 0; e < PER; ++e)
          if (base + e < n) a.Q[base + e] = o + W[e];
      }
    }
    // Systematic resampling, one step per particle: with D = n Q_i - (j T + r)
    // for particle i and its first slot j, i owns the c = ceil(D / T) slots
    // j .. j + c - 1 (none if D <= 0); D then drops by c T into (-T, 0] and
    // the next particle adds n w_{i+1} <= n 2^k <= 2^61 (T <= 2^61 too), so
    // D is an int64.  A particle writes its offset in the tile + 1 into the
    // window entries of its slots: the first three by predicated stores, any
    // others (a heavy particle) and slots past the window out of line, in
    // runs of the CTA when long.  c comes from three comparisons unless it is
    // above 3 (a heavy particle, divided out): no branch for up to three slots,
    // which covers all but a few particles in a hundred even when an outlying
    // observation concentrates the weights.  Every slot of [S0, S1) is
    // written exactly once, so the window needs no clearing.  A rolled loop
    // over the row: the step's code stays small.
    // a warp none of whose particles can own more than two slots takes the
    // lean step; any other warp counts up to three slots without a branch
    const bool light = !__any_sync(0xffffffffu, emx > thr);
    if (rs && T > 0 && base < n) {
      const uint32_t ecount = base + PER <= n ? (uint32_t)PER : (uint32_t)(n - base);
      uint32_t j = threadIdx.x == 0 ? S0 : (base == 0 ? 0u : (uint32_t)sys_first_slot(o, n, r, dv));
      const U128 X = mul64x32(o, (uint32_t)n);
      const U128 KB = add128(mul64x32(T, j), r);
      int64_t D = (int64_t)(X.lo - KB.lo);  // n Q - (j T + r) just before this thread's particles
      const int64_t Ti = (int64_t)T, T2 = 2 * Ti, T3 = 3 * Ti;
      const uint32_t off0 = (uint32_t)(base - tbase) + 1u;
      const uint32_t n32 = (uint32_t)n;
      uint64_t qprev = o;
      if (light) {
#pragma unroll 1
        for (uint32_t e = 0; e < ecount; ++e) {
          const uint64_t q = qrow[e];
          const uint64_t w = q - qprev;
          D += (int64_t)((uint64_t)(uint32_t)w * n32 + (((w >> 32) * n32) << 32));  // w n mod 2^64
          qprev = q;
          const uint32_t c = (uint32_t)(D > 0) + (uint32_t)(D > Ti);
          const uint16_t mk = (uint16_t)(off0 + e);
          const uint32_t x = j - S0a;
          if (c >= 1u && x < WIN_SLOTS) win[win_entry(x)] = mk;
          if (c >= 2u && x + 1u < WIN_SLOTS) win[win_entry(x + 1u)] = mk;
          if (x + c > WIN_SLOTS)
            sys_rest(j, c, S0a, WIN_SLOTS, mk, (uint32_t)base + e, win, a.anc, s_run, &s_nruns, 2u);
          D -= c == 1u ? Ti : (int64_t)c * Ti;
          j += c;
        }
      } else {
#pragma unroll 1
      for (uint32_t e = 0; e < ecount; ++e) {
        const uint64_t q = qrow[e];
        const uint64_t w = q - qprev;
        D += (int64_t)((uint64_t)(uint32_t)w * n32 + (((w >> 32) * n32) << 32));  // w n mod 2^64
        qprev = q;
        uint32_t c = (uint32_t)(D > 0) + (uint32_t)(D > Ti) + (uint32_t)(D > T2);
        if (D > T3) c = sys_heavy_count(D, dv);
        const uint16_t mk = (uint16_t)(off0 + e);
        const uint32_t x = j - S0a;
        if (c >= 1u && x < WIN_SLOTS) win[win_entry(x)] = mk;
        if (c >= 2u && x + 1u < WIN_SLOTS) win[win_entry(x + 1u)] = mk;
        if (c >= 3u && x + 2u < WIN_SLOTS) win[win_entry(x + 2u)] = mk;
        if (c > 3u || x + c > WIN_SLOTS)
          sys_rest(j, c, S0a, WIN_SLOTS, mk, (uint32_t)base + e, win, a.anc, s_run, &s_nruns, 3u);
        D -= c == 1u ? Ti : (int64_t)c * Ti;
        j += c;
      }
      }
      if (base + PER >= n || threadIdx.x == BLOCK - 1) s_S[1] = j;  // the tile's end slot
    }
    __syncthreads();
    // window runs of heavy particles, by the whole CTA
    const uint32_t nr = s_nruns < BB_RUNS ? s_nruns : BB_RUNS;
    bool wr = false;
    for (uint32_t q = 0; q < nr; ++q) {
      const uint32_t v = s_run[q][2];
      if (!(v & WRUN)) continue;
      wr = true;
      for (uint32_t x = s_run[q][0] + threadIdx.x; x < s_run[q][1]; x += BLOCK)
        win[win_entry(x)] = (uint16_t)v;
    }
    if (wr) __syncthreads();  // (wr is the same in every thread)
    if constexpr (STAGED) {  // the CDF rows, written out coalesced
      const uint64_t tcnt = n - tbase < (uint64_t)TP ? n - tbase : (uint64_t)TP;
      for (uint32_t p = 2 * threadIdx.x; p < tcnt; p += 2 * BLOCK) {
        const uint64_t q0 = s_keep[(p / PER) * (PER + 1) + (p % PER)];
        if (p + 1 < tcnt) {
          const uint64_t q1 = s_keep[(p / PER) * (PER + 1) + (p % PER) + 1];
          *reinterpret_cast<ulonglong2*>(a.Q + tbase + p) = make_ulonglong2(q0, q1);
        } else {
          a.Q[tbase + p] = q0;
        }
      }
    }
    // the window's slots [S0, wend), stored out coalesced, four per 16-byte
    // store (the partial groups at either end slot by slot)
    {
      const uint32_t S1 = s_S[1];
      const uint32_t wend = (rs && T > 0) ? (S1 - S0a < WIN_SLOTS ? S1 : S0a + WIN_SLOTS) : S0;
      const uint32_t tb32 = (uint32_t)tbase - 1u;
      const uint32_t ng = wend > S0 ? (wend - S0a + 3u) >> 2 : 0u;
      for (uint32_t g = threadIdx.x; g < ng; g += BLOCK) {
        const uint32_t x0 = g << 2;
        const uint32_t sw = ((x0 >> 6) & 7u) << 1;
        const uint2 v = *reinterpret_cast<const uint2*>(win + (x0 ^ (sw & 12u)));
        const uint32_t lo = (sw & 2u) ? v.y : v.x, hi = (sw & 2u) ? v.x : v.y;
        const uint32_t slot = S0a + x0;
        const uint4 o4 = make_uint4(tb32 + (lo & 0xffffu), tb32 + (lo >> 16), tb32 + (hi & 0xffffu),
                                    tb32 + (hi >> 16));
        if (slot >= S0 && slot + 4u <= wend) {
          *reinterpret_cast<uint4*>(a.anc + slot) = o4;
        } else {
          if (slot >= S0 && slot < wend) a.anc[slot] = o4.x;
          if (slot + 1u >= S0 && slot + 1u < wend) a.anc[slot + 1u] = o4.y;
          if (slot + 2u >= S0 && slot + 2u < wend) a.anc[slot + 2u] = o4.z;
          if (slot + 3u >= S0 && slot + 3u < wend) a.anc[slot + 3u] = o4.w;
        }
      }
    }
    // runs past the window, by the whole CTA
    for (uint32_t q = 0; q < nr; ++q) {
      const uint32_t st = s_run[q][0], en = s_run[q][1], v = s_run[q][2];
      if (v & WRUN) continue;
      for (uint32_t jj = st + threadIdx.x; jj < en; jj += BLOCK) a.anc[jj] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) s_nruns = 0;
    carry += tile_tot;
  }
  if (CTA_PART && threadIdx.x == 0) reinterpret_cast<ES*>(a.part)[blockIdx.x] = cta_es;
  if (T == 0) {  // empty CDF (flagged): keep every index in range
    for (uint64_t j = (uint64_t)blockIdx.x * BLOCK + threadIdx.x; j < n;
         j += (uint64_t)gridDim.x * BLOCK)
      a.anc[j] = (uint32_t)j;
  }
  if (STAGED && threadIdx.x == 0) {
    drain_copies();
    bulk_wait_done();
  }
}

// ---------------------------------------------------------------------------
// Steps 2-4: propagate x, update the sufficient statistics, draw theta.
// The last block to finish folds the log-ML partials, resets the per-cycle
// counters and advances t.
// ---------------------------------------------------------------------------
template <class R> struct ResidObs;
template <> struct ResidObs<float> {
  static __device__ __forceinline__ float f(double, float yr, float xj) { return yr - xj; }
};
template <> struct ResidObs<double> {
  static __device__ __forceinline__ double f(double y, double, double xj) { return y - xj; }
};

__device__ __forceinline__ double esum_value(const ESum32& e) {
  return __ull2double_rn(e.s.hi) * 0x1p-32 + __ull2double_rn(e.s.lo) * 0x1p-96;
}
__device__ __forceinline__ double esum_value(const ESum64& e) { return e.s; }

// ---------------------------------------------------------------------------
// Adaptive resampling decision (not in the paper, which resamples every
// cycle): ESS = (sum W)^2 / sum W^2 of the quantised weights against
// ess_frac * n (Kong, Liu & Wong 1994).  sum W^2 is summed exactly in 128
// bits from the finished CDF (W_i = Q_i - Q_{i-1}); sum W = Q_{n-1}.  The
// comparison is A * A < (ess_frac * n) * B in binary64, A and B the two sums
// each rounded to nearest once.  The last block writes the decision.
// ---------------------------------------------------------------------------
constexpr int ESS_PER_THREAD = 8;

template <class R>
__global__ void __launch_bounds__(BLOCK) k_ess(FilterArgs<R> a) {
  __shared__ U128 s_red[WARPS];
  __shared__ bool s_last;
  const uint64_t n = a.n;
  U128 acc{0, 0};
  const uint64_t stride = (uint64_t)gridDim.x * BLOCK;
  // ESS_PER_THREAD strided elements per pass, their loads issued together
  for (uint64_t i0 = (uint64_t)blockIdx.x * BLOCK + threadIdx.x; i0 < n;
       i0 += stride * ESS_PER_THREAD) {
    uint64_t q[ESS_PER_THREAD], qp[ESS_PER_THREAD];
#pragma unroll
    for (int e = 0; e < ESS_PER_THREAD; ++e) {
      const uint64_t i = i0 + (uint64_t)e * stride;
      q[e] = i < n ? a.Q[i] : 0ull;
      qp[e] = (i < n && i > 0) ? a.Q[i - 1] : 0ull;
    }
#pragma unroll
    for (int e = 0; e < ESS_PER_THREAD; ++e) {
      const uint64_t W = q[e] - qp[e];
      acc = add128(acc, mul64(W, W));
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    U128 v;
    v.hi = __shfl_xor_sync(0xffffffffu, acc.hi, o);
    v.lo = __shfl_xor_sync(0xffffffffu, acc.lo, o);
    acc = add128(acc, v);
  }
  if (lane == 0) s_red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    U128 b = s_red[0];
    for (int w = 1; w < WARPS; ++w) b = add128(b, s_red[w]);
    a.ess_part[blockIdx.x] = b;
    __threadfence();
    s_last = atomicAdd(&a.ctl->done_ess, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // fold the block partials across the block: an exact integer sum, so the
  // order does not matter
  U128 B{0, 0};
  for (uint32_t b = threadIdx.x; b < gridDim.x; b += BLOCK) {
    U128 v;
    v.hi = __ldcg(&a.ess_part[b].hi);
    v.lo = __ldcg(&a.ess_part[b].lo);
    B = add128(B, v);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    U128 v;
    v.hi = __shfl_xor_sync(0xffffffffu, B.hi, o);
    v.lo = __shfl_xor_sync(0xffffffffu, B.lo, o);
    B = add128(B, v);
  }
  if (lane == 0) s_red[warp] = B;
  __syncthreads();
  if (threadIdx.x != 0) return;
  B = s_red[0];
  for (int w = 1; w < WARPS; ++w) B = add128(B, s_red[w]);
  const double A = __ull2double_rn(a.Q[n - 1]);
  const double Bd = u128_to_f64_rn(B);
  const double lhs = A * A;
  const double f = a.ess_frac * (double)n;
  const double rhs = f * Bd;
  a.ctl->resamp = lhs < rhs ? 1u : 0u;
  a.ctl->done_ess = 0;
}

// Run by the last warp of k_propagate: fold the per-tile log-ML partials
// (lane-strided, then butterfly: a fixed order), accumulate the increment
// m + log(sum_i e_i) - log n - log(2 pi)/2, reset the per-cycle counters and
// advance t.
//
// With FUSE the propagation has also computed the next cycle's weights: the
// maximum it gathered becomes the next cycle's, and the constants that the
// weights kernel would write for the next cycle (observation y_{t+2},
// Marsaglia-Tsang constants of the shapes a0 + (t+2)/2) are written here, once
// every warp has read this cycle's.
//
// With ESS (adaptive resampling) the increment is normalised by the carried
// weights, log sum_i exp(lambda_i), instead of log n, and that sum for the
// next cycle is n after a resampling, else this cycle's sum of exp(L_i - m).
template <class R, bool FUSE = false, bool ESS = false>
__device__ void fold_cycle_warp(const FilterArgs<R>& a, uint32_t t) {
  typedef typename ESumT<R>::T ES;
  const int lane = threadIdx.x & 31;
  ES acc;
  acc.zero();
  const ES* const part = reinterpret_cast<const ES*>(a.part);
  if constexpr (sizeof(R) == 4) {
    // exact fixed-point partials: any grouping gives the same sum, so each
    // lane issues eight loads at once
    for (uint32_t b = lane; b < a.nparts; b += 256) {
      ES v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        v[q].zero();
        if (b + 32u * q < a.nparts) v[q] = part[b + 32u * q];
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) acc.add(v[q]);
    }
  } else {
    for (uint32_t b = lane; b < a.nparts; b += 32) acc.add(part[b]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc.add(acc.shfl_xor(o));
  if (lane == 0) {
    Ctl* c = a.ctl;
    const double m = sizeof(R) == 4 ? (double)dec_f((uint32_t)c->maxenc) : dec_d(c->maxenc);
    const double LOG_2PI = 0x1.d67f1c864beb5p+0;
    if constexpr (ESS) {
      const double S = esum_value(acc);
      const double inc = m + log(S) - log(c->slam) - 0.5 * LOG_2PI;
      c->logml = c->logml + inc;
      c->slam = c->resamp ? (double)a.n : S;
    } else {
      const double inc = m + log(esum_value(acc)) - log((double)a.n) - 0.5 * LOG_2PI;
      c->logml = c->logml + inc;
    }
    const unsigned long long ninf =
        sizeof(R) == 4 ? (unsigned long long)enc_f(-INFINITY) : enc_d(-INFINITY);
    if constexpr (FUSE) {
      // every warp's maximum was published before its completion count
      __threadfence();
      c->maxenc = atomicExch(&c->maxenc_nx, ninf);
      const double y = a.y_nx_src ? *a.y_nx_src : a.y_nx_val;
      write_cycle_constants(c, y, a.a_sigma, a.a_tau, t + 2);
    } else {
      c->maxenc = ninf;
    }
    c->ticket_w = 0;
    c->ticket_e = 0;
    c->done_prop = 0;
    c->gbar = 0;
    c->prop_ticket = 0;
    c->w_ticket = 0;
    __threadfence();
    c->t = t + 1;
  }
}

// A gamma draw that missed the Marsaglia-Tsang squeeze on its first attempt,
// finished after the warp's fast path (same arithmetic, later in time).
template <class R>
struct GammaItem {
  typename SuffT<R>::B b;  // updated sufficient statistic (the IG scale)
  R Z, U;                  // attempt-0 normal and uniform
  uint32_t j;              // slot
  uint32_t which;          // 0: sigma^2, 1: tau^2
};

// Per-warp queue of such draws.  A warp pushes at most 64 per pass and
// finishes them 32 at a time (one per lane) once 32 are queued, so no block
// barrier is needed and the lanes of a finishing round are all busy.
constexpr uint32_t WQ_CAP = 96;

template <class Item>
__device__ __forceinline__ void wq_push(Item* q, uint32_t& qn, bool dfr, const Item& itm,
                                        int lane) {
  const uint32_t m = __ballot_sync(0xffffffffu, dfr);
  if (dfr) q[qn + __popc(m & ((1u << lane) - 1u))] = itm;
  qn += __popc(m);
}

// Finish queued draws, 32 per round, while at least `lo` (>= 1) are queued;
// after each round (its writes ordered by the warp barrier) `post` runs on the
// lanes whose item has bit 1 of `which` set.
template <class R, class Fin, class Post>
__device__ __forceinline__ void wq_drain_post(GammaItem<R>* q, uint32_t& qn, uint32_t lo,
                                              int lane, Fin fin, Post post) {
  __syncwarp();
  while (qn >= lo) {
    const uint32_t take = qn < 32u ? qn : 32u;
    const uint32_t base = qn - take;
    const bool mine = (uint32_t)lane < take;
    GammaItem<R> itm;
    if (mine) {
      itm = q[base + lane];
      fin(itm);
    }
    __syncwarp();
    if (mine && (itm.which & 2u)) post(itm);
    qn = base;
    __syncwarp();
  }
}

// Finish queued draws, 32 per round, while at least `lo` (>= 1) are queued.
template <class Item, class Fin>
__device__ __forceinline__ void wq_drain(Item* q, uint32_t& qn, uint32_t lo, int lane, Fin fin) {
  __syncwarp();
  while (qn >= lo) {
    const uint32_t take = qn < 32u ? qn : 32u;
    const uint32_t base = qn - take;
    if ((uint32_t)lane < take) fin(q[base + lane]);
    qn = base;
    __syncwarp();
  }
}

// The next cycle's weight of one slot: l = log p(y_{t+2} | x, sigma^2, tau^2),
// the weights kernel's arithmetic; its maximum and finiteness are tracked.
template <class R>
__device__ __forceinline__ void weigh_next(R* ell, uint64_t j, R x, R s2, R t2, R yn, R& mx,
                                           bool& bad) {
  const R l = log_pred<R>(x, s2, t2, yn);
  ell[j] = l;
  bad |= !(l < (R)INFINITY);
  mx = fmax(mx, l);
}

// log_pred on two slots with paired operations; per lane the same IEEE
// operations in the same order, so the same bits.
__device__ __forceinline__ float2 log_pred2(float2 x, float2 s2, float2 t2, float yn) {
  const float2 s = add2(s2, t2);
  const float2 dx = sub2(splat2(yn), x);
  const float2 q = mul2(dx, dx);
  const float2 lg = det_log2(s);
  const float2 r = make_float2(q.x / s.x, q.y / s.y);
  const float2 sum = add2(lg, r);
  return mul2(splat2(-0.5f), sum);
}

// Store a next-cycle weight computed elsewhere and track it.
template <class R>
__device__ __forceinline__ void keep_next(R* ell, uint64_t j, R l, R& mx, bool& bad) {
  ell[j] = l;
  bad |= !(l < (R)INFINITY);
  mx = fmax(mx, l);
}

// Publish a warp's maximum of the next cycle's weights (lane 0 only), before
// the warp's completion count.
template <class R>
__device__ __forceinline__ void publish_next_max(Ctl* c, R mx, int lane) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) {
    if (mx > (R)-INFINITY) atomicMax(&c->maxenc_nx, enc_max(mx));
    __threadfence();
  }
}

// One ancestor's record, gathered ahead of its use.
template <class R>
struct Gathered {
  R x, s2, t2;
  typename SuffT<R>::B bs, bt;
};
template <class R>
__device__ __forceinline__ Gathered<R> gather_rec(const StateV<R>& src, uint32_t an) {
  Gathered<R> g;
  g.x = src.x[an];
  g.s2 = src.s2[an];
  g.t2 = src.t2[an];
  g.bs = src.bs[an];
  g.bt = src.bt[an];
  return g;
}

// Persistent grid: thread (block b, lane t) handles slots j = b*BLOCK + t +
// k * stride.  The ancestor index is loaded two slots ahead and the ancestor's
// record one slot ahead, so the dependent index -> gather latency overlaps the
// arithmetic of the current slot.
//
// With FUSE the kernel also computes the next cycle's predictive weights
// l_j = log p(y_{t+2} | x'_j, sigma^2'_j, tau^2'_j) and their maximum, which
// the next cycle then uses instead of running the weights kernel.  A slot
// whose gamma draw missed the squeeze is weighed by the drain round that
// finishes its last queued draw (bit 1 of `which` on that item), reading its
// new state back after the round's warp barrier.  Every value is the one the
// weights kernel would give.
template <class R, bool LEARN, bool FUSE = false, bool ESS = false>
__global__ void __launch_bounds__(BLOCK, 5) k_propagate(FilterArgs<R> a) {
  typedef GammaItem<R> Item;
  __shared__ Item s_q[WARPS][WQ_CAP];
  const Ctl* c = a.ctl;
  const uint32_t t = c->t;
  const StateV<R> src = (t & 1) ? a.st[1] : a.st[0];
  const StateV<R> dst = (t & 1) ? a.st[0] : a.st[1];
  const double y = c->y;
  R yr, ds, cs, dt, ct, ks, kt;
  if constexpr (sizeof(R) == 4) {
    yr = c->yf; ds = c->mtf[0]; cs = c->mtf[1]; dt = c->mtf[2]; ct = c->mtf[3];
    ks = c->mtf[4]; kt = c->mtf[5];
  } else {
    yr = y; ds = c->mtd[0]; cs = c->mtd[1]; dt = c->mtd[2]; ct = c->mtd[3];
    ks = c->mtd[4]; kt = c->mtd[5];
  }
  const int lane = threadIdx.x & 31;
  Item* const wq = s_q[threadIdx.x >> 5];
  uint32_t qn = 0;  // warp-uniform
  const uint64_t n = a.n;
  const uint64_t stride = (uint64_t)gridDim.x * BLOCK;
  const uint64_t iters = (n + stride - 1) / stride;
  auto clampi = [&](uint32_t v) { return v < n ? v : (uint32_t)(n - 1); };
  // adaptive resampling: without a resampling every slot is its own ancestor
  bool rs = true;
  R mR = 0;
  if constexpr (ESS) {
    rs = c->resamp != 0;
    if constexpr (sizeof(R) == 4) mR = dec_f((uint32_t)c->maxenc);
    else mR = dec_d(c->maxenc);
  }
  auto ancx = [&](uint64_t k) -> uint32_t {
    if constexpr (ESS) {
      if (!rs) return (uint32_t)k;
    }
    return clampi(a.anc[k]);
  };
  // the carried log-weight of slot j: 0 after a resampling, else L_j - m
  auto carry = [&](uint64_t k) {
    if (rs) {
      a.lam[k] = (R)0;
    } else {
      a.lam[k] = a.ell[k] - mR;
      a.anc[k] = (uint32_t)k;
    }
  };
  bool fail = false;
  // next cycle's weights (FUSE)
  R yn = 0;
  if constexpr (FUSE) yn = (R)(a.y_nx_src ? *a.y_nx_src : a.y_nx_val);
  R mxn = (R)-INFINITY;
  bool badn = false;
  auto finish = [&](const Item& itm) {
    const bool sig = (itm.which & 1u) == 0;
    const R G = gamma_mt_from<R>(sig ? ds : dt, sig ? cs : ct, sig ? ks : kt, itm.Z, itm.U, a.seed,
                                 a.filter, t, itm.j, sig ? P_GAMMA_SIGMA : P_GAMMA_TAU, &fail);
    const R v = SuffOps<R>::ig(itm.b, G);
    if (sig) dst.s2[itm.j] = v;
    else dst.t2[itm.j] = v;
  };
  auto weigh_late = [&](const Item& itm) {  // FUSE: the slot's state is final
    weigh_next<R>(a.ell, itm.j, dst.x[itm.j], dst.s2[itm.j], dst.t2[itm.j], yn, mxn, badn);
  };
  uint64_t j = (uint64_t)blockIdx.x * BLOCK + threadIdx.x;
  uint32_t an = j < n ? ancx(j) : 0;
  uint32_t an_next = j + stride < n ? ancx(j + stride) : 0;
  Gathered<R> cur = gather_rec<R>(src, an);
  for (uint64_t it = 0; it < iters; ++it, j += stride) {
    // prefetch: the index two slots ahead, the record one slot ahead
    const uint32_t an_next2 = j + 2 * stride < n ? ancx(j + 2 * stride) : 0;
    const Gathered<R> nxt = gather_rec<R>(src, an_next);
    bool defer_s = false, defer_t = false;
    typename SuffT<R>::B bsn = 0, btn = 0;
    R Zs = 0, Us = 0, Zt = 0, Ut = 0;
    R xj = 0, s2n = 0, t2n = 0;
    if (j < n) {
      const R xa = cur.x, sa = cur.s2, ta = cur.t2;
      // V and mu share one correctly rounded reciprocal of s
      const R s = sa + ta;
      const R ri = (R)1 / s;
      const R p = sa * ta;
      const R V = p * ri;
      const R n2 = yr * ta;
      const R nn = fmaR(xa, sa, n2);
      const R mu = nn * ri;
      const R sv = sqrt(V);
      R Z;
      theta_draws_rk<R>(a.rk, a.filter, t, (uint32_t)j, &Z, &Zs, &Us, &Zt, &Ut);
      xj = fmaR(sv, Z, mu);
      dst.x[j] = xj;
      if (LEARN) {
        const R rs = ResidObs<R>::f(y, yr, xj);
        const R rt = xj - xa;
        bsn = SuffOps<R>::add_half_square(cur.bs, rs, &fail);
        btn = SuffOps<R>::add_half_square(cur.bt, rt, &fail);
        dst.bs[j] = bsn;
        dst.bt[j] = btn;
        R Gs, Gt;
        if (gamma_mt_squeeze<R>(ds, cs, ks, Zs, Us, &Gs)) dst.s2[j] = s2n = SuffOps<R>::ig(bsn, Gs);
        else defer_s = true;
        if (gamma_mt_squeeze<R>(dt, ct, kt, Zt, Ut, &Gt)) dst.t2[j] = t2n = SuffOps<R>::ig(btn, Gt);
        else defer_t = true;
      } else {
        dst.s2[j] = s2n = sa;
        dst.t2[j] = t2n = ta;
        dst.bs[j] = cur.bs;
        dst.bt[j] = cur.bt;
      }
      if (FUSE && !defer_s && !defer_t) weigh_next<R>(a.ell, j, xj, s2n, t2n, yn, mxn, badn);
      if constexpr (ESS) carry(j);
    }
    if constexpr (LEARN && FUSE) {
      // the sigma^2 item sits below the tau^2 item of its slot, so it is
      // finished in the same round or a later one: it weighs the slot when
      // both were deferred
      wq_push(wq, qn, defer_s, Item{bsn, Zs, Us, (uint32_t)j, 2u}, lane);
      wq_push(wq, qn, defer_t, Item{btn, Zt, Ut, (uint32_t)j, defer_s ? 1u : 3u}, lane);
      wq_drain_post(wq, qn, 32u, lane, finish, weigh_late);
    } else if constexpr (LEARN) {
      // queue the draws that missed the squeeze; the warp finishes them 32
      // at a time
      wq_push(wq, qn, defer_s, Item{bsn, Zs, Us, (uint32_t)j, 0u}, lane);
      wq_push(wq, qn, defer_t, Item{btn, Zt, Ut, (uint32_t)j, 1u}, lane);
      wq_drain(wq, qn, 32u, lane, finish);
    }
    cur = nxt;
    an_next = an_next2;
  }
  if constexpr (LEARN && FUSE) wq_drain_post(wq, qn, 1u, lane, finish, weigh_late);
  else if (LEARN) wq_drain(wq, qn, 1u, lane, finish);
  (void)an;
  if (__any_sync(0xffffffffu, fail || badn) && lane == 0) atomicOr(&a.ctl->err, ERR_NUMERIC);
  // Without FUSE the fold reads only what earlier kernels wrote (tile
  // partials, the control block), so the completion count needs no fence;
  // every warp has read t before its increment.  With FUSE each warp's
  // maximum is fenced before its count.
  if constexpr (FUSE) publish_next_max<R>(a.ctl, mxn, lane);
  bool last = false;
  if (lane == 0) last = atomicAdd(&a.ctl->done_prop, 1u) == gridDim.x * WARPS - 1;
  last = __shfl_sync(0xffffffffu, last, 0);
  if (last) fold_cycle_warp<R, FUSE, ESS>(a, t);
}

// ---------------------------------------------------------------------------
// k_propagate for binary32 state, two slots per thread per pass: the pair
// 2i, 2i + 1, which shares its second draw (theta_draws2), shares each paired
// FADD2 / FMUL2 / FFMA2, while divisions, square roots, comparisons and the
// fixed-point statistics run per lane.  Per slot the operations are those of
// the scalar propagation, in the same order, so the results are the same bits.
// ---------------------------------------------------------------------------
constexpr uint32_t WQ2_CAP = 160;  // 31 queued + 4 pushes of 32 per pass
// k_propagate2's units of 64 slots: with DYN handed out by ticket, PROP_GRAB
// at a time; the launch takes DYN when there are at least PROP_DYN per warp
constexpr uint32_t PROP_GRAB = 4;
constexpr uint32_t PROP_DYN = 16;

// With FUSE, the next cycle's weights as in k_propagate, the two slots of a
// pass weighed by paired operations.
// 3 CTAs per SM (up to 85 registers, no spills): measured faster at N = 2^24
// than 4 CTAs at 64 registers, where the plain form spills.
template <bool LEARN, bool FUSE = false, bool ESS = false, bool DYN = false>
__global__ void __launch_bounds__(BLOCK, 3) k_propagate2(FilterArgs<float> a) {
  typedef GammaItem<float> Item;
  __shared__ Item s_q[WARPS][WQ2_CAP];
  const Ctl* c = a.ctl;
  const uint32_t t = c->t;
  const StateV<float> src = (t & 1) ? a.st[1] : a.st[0];
  const StateV<float> dst = (t & 1) ? a.st[0] : a.st[1];
  const float yr = c->yf, ds = c->mtf[0], cs = c->mtf[1], dt = c->mtf[2], ct = c->mtf[3];
  const float ks = c->mtf[4], kt = c->mtf[5];
  const int lane = threadIdx.x & 31;
  Item* const wq = s_q[threadIdx.x >> 5];
  uint32_t qn = 0;  // warp-uniform
  const uint64_t n = a.n;
  auto clampi = [&](uint32_t v) { return v < n ? v : (uint32_t)(n - 1); };
  // adaptive resampling: without a resampling every slot is its own ancestor
  bool rs = true;
  float mR = 0.0f;
  if constexpr (ESS) {
    rs = c->resamp != 0;
    mR = dec_f((uint32_t)c->maxenc);
  }
  // the carried log-weight of slot j: 0 after a resampling, else L_j - m
  auto carry = [&](uint64_t k) {
    if (rs) {
      a.lam[k] = 0.0f;
    } else {
      a.lam[k] = a.ell[k] - mR;
      a.anc[k] = (uint32_t)k;
    }
  };
  bool fail = false;
  // next cycle's weights (FUSE)
  float yn = 0.0f;
  if constexpr (FUSE) yn = (float)(a.y_nx_src ? *a.y_nx_src : a.y_nx_val);
  float mxn = -INFINITY;
  bool badn = false;
  auto finish = [&](const Item& itm) {
    const bool sig = (itm.which & 1u) == 0;
    const float G = gamma_mt_from<float>(sig ? ds : dt, sig ? cs : ct, sig ? ks : kt, itm.Z,
                                         itm.U, a.seed, a.filter, t, itm.j,
                                         sig ? P_GAMMA_SIGMA : P_GAMMA_TAU, &fail);
    const float v = SuffOps<float>::ig(itm.b, G);
    if (sig) dst.s2[itm.j] = v;
    else dst.t2[itm.j] = v;
  };
  auto weigh_late = [&](const Item& itm) {  // FUSE: the slot's state is final
    weigh_next<float>(a.ell, itm.j, dst.x[itm.j], dst.s2[itm.j], dst.t2[itm.j], yn, mxn, badn);
  };
  // Slots go out in units of 64: lane l of a warp takes the pair j0 = 64 u +
  // 2 l, j1 = j0 + 1 of unit u (the two slots that share a draw), so its
  // ancestor load and its stores are 8 or 16 bytes wide.  Without DYN, pass
  // p of warp w (of the grid's W) is unit p W + w.  With DYN (many units per
  // warp) a warp takes PROP_GRAB consecutive units per ticket, each ticket
  // taken a batch ahead of its use, so that a warp on a slower SM (or with
  // more draws that missed the squeeze) takes fewer of them and the kernel
  // ends with its work: under the fixed assignment the CTAs' finishing times
  // at N = 2^24 spread from 187 to 234 us.  A slot's arithmetic does not
  // depend on the warp that computes it.
  const uint64_t nunits = (n + 63) / 64;
  const uint64_t stride = (uint64_t)gridDim.x * BLOCK * 2;  // slots per pass
  const uint64_t iters = (n + stride - 1) / stride;
  unsigned long long tick = 0;  // lane 0: the ticket of the next batch
  uint64_t u = 0;
  uint64_t j0 = 2 * ((uint64_t)blockIdx.x * BLOCK + threadIdx.x);
  if constexpr (DYN) {
    if (lane == 0) tick = atomicAdd(&a.ctl->prop_ticket, (unsigned long long)PROP_GRAB);
    u = __shfl_sync(0xffffffffu, tick, 0);
    if (lane == 0) tick = atomicAdd(&a.ctl->prop_ticket, (unsigned long long)PROP_GRAB);
    j0 = u * 64 + 2 * (uint64_t)lane;
  }
  (void)nunits; (void)iters; (void)u;
  // the ancestors of the pair starting at slot j (even; clamped into range)
  auto anc_pair = [&](uint64_t j) -> uint2 {
    if constexpr (ESS) {  // (past the end: the last slot, a valid address)
      if (!rs) return make_uint2(clampi((uint32_t)j), clampi((uint32_t)j + 1u));
    }
    if (j + 1 < n) {
      const uint2 v = *reinterpret_cast<const uint2*>(a.anc + j);
      return make_uint2(clampi(v.x), clampi(v.y));
    }
    return make_uint2(j < n ? clampi(a.anc[j]) : 0u, 0u);
  };
  uint2 an = anc_pair(j0);
  Gathered<float> c0 = gather_rec<float>(src, an.x);
  Gathered<float> c1 = gather_rec<float>(src, an.y);
  for (uint64_t it = 0; DYN ? u < nunits : it < iters; ++it) {  // (the same in every lane)
    // the next pair: the next pass's; with DYN the next unit of the batch,
    // or the first of the batch taken a batch ago (then the ticket of the
    // batch after it)
    uint64_t jn = j0 + stride;
    uint64_t un = u + 1;
    if constexpr (DYN) {
      if (un % PROP_GRAB == 0) {
        un = __shfl_sync(0xffffffffu, tick, 0);
        if (lane == 0 && un < nunits) tick = atomicAdd(&a.ctl->prop_ticket, (unsigned long long)PROP_GRAB);
      }
      jn = un * 64 + 2 * (uint64_t)lane;
    }
    const uint64_t j1 = j0 + 1;
    const bool v0 = j0 < n, v1 = j1 < n;
    // the next unit's records, gathered ahead
    const uint2 na = anc_pair(jn);
    const Gathered<float> n0 = gather_rec<float>(src, na.x);
    const Gathered<float> n1 = gather_rec<float>(src, na.y);
    // the last unit may be partial: a warp skips it when no lane has a slot
    if (__any_sync(0xffffffffu, v0)) {
      const float2 xa = make_float2(c0.x, c1.x), sa = make_float2(c0.s2, c1.s2);
      const float2 ta = make_float2(c0.t2, c1.t2);
      // V and mu share one correctly rounded reciprocal of s = sigma^2 + tau^2
      const float2 sm = addp(sa, ta);
      const float2 ri = make_float2(__frcp_rn(sm.x), __frcp_rn(sm.y));
      const float2 V = mul2(mul2(sa, ta), ri);
      const float2 nn = fma2(xa, sa, mul2(splat2(yr), ta));
      const float2 mu = mul2(nn, ri);
      const float2 sv = make_float2(sqrtf(V.x), sqrtf(V.y));
      float2 Z, Zs, Us, Zt, Ut;
      theta_draws2(a.rk, a.filter, t, (uint32_t)(j0 >> 1), &Z, &Zs, &Us, &Zt, &Ut);
      const float2 xj = fma2(sv, Z, mu);
      if (v1) {
        *reinterpret_cast<float2*>(dst.x + j0) = xj;
      } else if (v0) {
        dst.x[j0] = xj.x;
      }
      bool ds0 = false, dt0 = false, ds1 = false, dt1 = false;
      uint64_t bs0 = 0, bt0 = 0, bs1 = 0, bt1 = 0;
      if (LEARN) {
        const float2 rs = addp(splat2(yr), make_float2(-xj.x, -xj.y));
        const float2 rt = addp(xj, make_float2(-xa.x, -xa.y));
        // b + r^2 / 2 in 2^-32 fixed point, per SuffOps<float>::add_half_square
        const float2 ws = mul2(mul2(rs, rs), splat2(0x1p31f));
        const float2 wt = mul2(mul2(rt, rt), splat2(0x1p31f));
        bool f0 = false, f1 = false;
        auto addb = [&](uint64_t b, float v, bool* f) -> uint64_t {
          if (!(v < 0x1p63f)) {
            *f = true;
            return b;
          }
          return b + SuffOps<float>::incr(v);
        };
        bs0 = addb(c0.bs, ws.x, &f0);
        bt0 = addb(c0.bt, wt.x, &f0);
        bs1 = addb(c1.bs, ws.y, &f1);
        bt1 = addb(c1.bt, wt.y, &f1);
        fail |= (v0 && f0) || (v1 && f1);
        if (v1) {
          *reinterpret_cast<ulonglong2*>(dst.bs + j0) = make_ulonglong2(bs0, bs1);
          *reinterpret_cast<ulonglong2*>(dst.bt + j0) = make_ulonglong2(bt0, bt1);
        } else if (v0) {
          dst.bs[j0] = bs0;
          dst.bt[j0] = bt0;
        }
        // Marsaglia-Tsang squeeze for sigma^2 (x lanes: slot j0, j1) and tau^2
        const float2 vs = fma2(splat2(cs), Zs, splat2(1.0f)), vt = fma2(splat2(ct), Zt, splat2(1.0f));
        const float2 v3s = mul2(mul2(vs, vs), vs), v3t = mul2(mul2(vt, vt), vt);
        const float2 Z2s = mul2(Zs, Zs), Z2t = mul2(Zt, Zt);
        const float2 thrs = fma2(splat2(-ks), mul2(Z2s, Z2s), splat2(1.0f));
        const float2 thrt = fma2(splat2(-kt), mul2(Z2t, Z2t), splat2(1.0f));
        const float2 Gs = mul2(splat2(ds), v3s), Gt = mul2(splat2(dt), v3t);
        const bool as0 = vs.x > 0.0f && Us.x < thrs.x, as1 = vs.y > 0.0f && Us.y < thrs.y;
        const bool at0 = vt.x > 0.0f && Ut.x < thrt.x, at1 = vt.y > 0.0f && Ut.y < thrt.y;
        // inverse gamma: (b 2^-32) / G, per SuffOps<float>::ig.  The divisions
        // run for every lane (no branch around them); a draw that missed the
        // squeeze stores nothing here and is finished from the warp's queue.
        const float2 bsf = fma2(make_float2(__uint2float_rn((uint32_t)bs0), __uint2float_rn((uint32_t)bs1)),
                                splat2(0x1p-32f),
                                make_float2(__uint2float_rn((uint32_t)(bs0 >> 32)),
                                            __uint2float_rn((uint32_t)(bs1 >> 32))));
        const float2 btf = fma2(make_float2(__uint2float_rn((uint32_t)bt0), __uint2float_rn((uint32_t)bt1)),
                                splat2(0x1p-32f),
                                make_float2(__uint2float_rn((uint32_t)(bt0 >> 32)),
                                            __uint2float_rn((uint32_t)(bt1 >> 32))));
        const float q0 = bsf.x / Gs.x, r0 = btf.x / Gt.x, q1 = bsf.y / Gs.y, r1 = btf.y / Gt.y;
        ds0 = v0 && !as0; dt0 = v0 && !at0; ds1 = v1 && !as1; dt1 = v1 && !at1;
        if (v1 && as0 && as1) {
          *reinterpret_cast<float2*>(dst.s2 + j0) = make_float2(q0, q1);
        } else {
          if (v0 && as0) dst.s2[j0] = q0;
          if (v1 && as1) dst.s2[j1] = q1;
        }
        if (v1 && at0 && at1) {
          *reinterpret_cast<float2*>(dst.t2 + j0) = make_float2(r0, r1);
        } else {
          if (v0 && at0) dst.t2[j0] = r0;
          if (v1 && at1) dst.t2[j1] = r1;
        }
        // 1 for a deferred draw: the paired weight of that slot is discarded,
        // and a normal operand keeps the log and the division on their fast paths
        const float s20 = as0 ? q0 : 1.0f, t20 = at0 ? r0 : 1.0f;
        const float s21 = as1 ? q1 : 1.0f, t21 = at1 ? r1 : 1.0f;
        // queue the draws that missed the squeeze (rare: K Z^4 is small for
        // the shapes of a running filter); the warp finishes them 32 at a time
        const bool any_def = __any_sync(0xffffffffu, ds0 || dt0 || ds1 || dt1);
        if constexpr (FUSE) {
          // both slots weighed paired; a slot with a deferred draw is weighed
          // by the drain round that finishes it (its sigma^2 item lies below
          // its tau^2 item, so it weighs when both were deferred)
          const float2 l = log_pred2(xj, make_float2(s20, s21), make_float2(t20, t21), yn);
          if (v0 && !ds0 && !dt0) keep_next(a.ell, j0, l.x, mxn, badn);
          if (v1 && !ds1 && !dt1) keep_next(a.ell, j1, l.y, mxn, badn);
          if (any_def) {
            wq_push(wq, qn, ds0, Item{bs0, Zs.x, Us.x, (uint32_t)j0, 2u}, lane);
            wq_push(wq, qn, dt0, Item{bt0, Zt.x, Ut.x, (uint32_t)j0, ds0 ? 1u : 3u}, lane);
            wq_push(wq, qn, ds1, Item{bs1, Zs.y, Us.y, (uint32_t)j1, 2u}, lane);
            wq_push(wq, qn, dt1, Item{bt1, Zt.y, Ut.y, (uint32_t)j1, ds1 ? 1u : 3u}, lane);
            wq_drain_post(wq, qn, 32u, lane, finish, weigh_late);
          }
        } else {
          (void)s20; (void)t20; (void)s21; (void)t21;
          if (any_def) {
            wq_push(wq, qn, ds0, Item{bs0, Zs.x, Us.x, (uint32_t)j0, 0u}, lane);
            wq_push(wq, qn, dt0, Item{bt0, Zt.x, Ut.x, (uint32_t)j0, 1u}, lane);
            wq_push(wq, qn, ds1, Item{bs1, Zs.y, Us.y, (uint32_t)j1, 0u}, lane);
            wq_push(wq, qn, dt1, Item{bt1, Zt.y, Ut.y, (uint32_t)j1, 1u}, lane);
            wq_drain(wq, qn, 32u, lane, finish);
          }
        }
      } else {
        if (v0) { dst.s2[j0] = sa.x; dst.t2[j0] = ta.x; dst.bs[j0] = c0.bs; dst.bt[j0] = c0.bt; }
        if (v1) { dst.s2[j1] = sa.y; dst.t2[j1] = ta.y; dst.bs[j1] = c1.bs; dst.bt[j1] = c1.bt; }
        if constexpr (FUSE) {
          const float2 l = log_pred2(xj, sa, ta, yn);
          if (v0) keep_next(a.ell, j0, l.x, mxn, badn);
          if (v1) keep_next(a.ell, j1, l.y, mxn, badn);
        }
      }
      if constexpr (ESS) {
        if (v0) carry(j0);
        if (v1) carry(j1);
      }
    }
    c0 = n0;
    c1 = n1;
    u = un;
    j0 = jn;
  }
  if constexpr (LEARN && FUSE) wq_drain_post(wq, qn, 1u, lane, finish, weigh_late);
  else if (LEARN) wq_drain(wq, qn, 1u, lane, finish);
  if (__any_sync(0xffffffffu, fail || badn) && lane == 0) atomicOr(&a.ctl->err, ERR_NUMERIC);
  if constexpr (FUSE) publish_next_max<float>(a.ctl, mxn, lane);
  bool last = false;
  if (lane == 0) last = atomicAdd(&a.ctl->done_prop, 1u) == gridDim.x * WARPS - 1;
  last = __shfl_sync(0xffffffffu, last, 0);
  if (last) fold_cycle_warp<float, FUSE, ESS>(a, t);
}

// ---------------------------------------------------------------------------
// The bootstrap filter's Step 3 completed: the resampled particles are the
// propagated ones at the ancestors (in place in the current buffer), copied
// into the other buffer; the last warp folds the log-ML increment and
// advances t, as in the propagation kernels.
// ---------------------------------------------------------------------------
template <class R>
__global__ void __launch_bounds__(BLOCK) k_boot_gather(FilterArgs<R> a) {
  const uint32_t t = a.ctl->t;
  const StateV<R> src = (t & 1) ? a.st[1] : a.st[0];
  const StateV<R> dst = (t & 1) ? a.st[0] : a.st[1];
  const uint64_t n = a.n;
  const uint64_t j = (uint64_t)blockIdx.x * BLOCK + threadIdx.x;
  if (j < n) {
    uint32_t an = a.anc[j];
    an = an < n ? an : (uint32_t)(n - 1);
    dst.x[j] = src.x[an];
    dst.s2[j] = src.s2[an];
    dst.t2[j] = src.t2[an];
    dst.bs[j] = src.bs[an];
    dst.bt[j] = src.bt[an];
  }
  const int lane = threadIdx.x & 31;
  bool last = false;
  if (lane == 0) last = atomicAdd(&a.ctl->done_prop, 1u) == gridDim.x * WARPS - 1;
  last = __shfl_sync(0xffffffffu, last, 0);
  if (last) fold_cycle_warp<R>(a, t);
}

// ---------------------------------------------------------------------------
// Posterior summaries (on demand): population means and variances of x,
// sigma^2 and tau^2, from sums of v - c and (v - c)^2 with c the value of
// particle 0 (a shift against cancellation).  Each thread sums its
// EST_PER_THREAD consecutive particles (vector loads) and each warp its
// lanes by a shuffle tree in the working precision; the warps of a block are
// joined in binary64, and the last block to finish folds the block partials
// in binary64 (each thread a fixed stride of blocks, then a shuffle tree):
// the result is run-to-run deterministic and binary64 arithmetic runs per
// block, not per particle (binary64 is a small fraction of the binary32 rate
// on this part).
// ---------------------------------------------------------------------------
constexpr int EST_PER_THREAD = 16;

// The control block's prefix up to the per-cycle constants (t, error word,
// counters, log-ML, summaries) written to the mapped host mirror, one 8-byte
// word per thread (called by every thread of the block, after a barrier that
// follows the writes to the control block); the host reads the mirror after
// synchronising with the stream, which orders these writes.
constexpr int SUMMARY_WORDS = (int)(offsetof(Ctl, y) / 8);
__device__ __forceinline__ void publish_summary(const Ctl* c, Ctl* mirror) {
  static_assert(offsetof(Ctl, y) % 8 == 0 && SUMMARY_WORDS <= 32, "prefix of whole words");
  if (!mirror || threadIdx.x >= SUMMARY_WORDS) return;
  reinterpret_cast<unsigned long long*>(mirror)[threadIdx.x] =
      __ldcg(reinterpret_cast<const unsigned long long*>(c) + threadIdx.x);
}
// After publish_summary, by the whole block: the host's sequence number to
// io->seq_out, ordered after every mirror word (each writer's system-scope
// fence, the block barrier, a release store).
__device__ __forceinline__ void publish_done(EstIO* io) {
  if (!io) return;
  __threadfence_system();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long sq = *reinterpret_cast<volatile unsigned long long*>(&io->seq_in);
    asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(&io->seq_out), "l"(sq) : "memory");
  }
}

// Means and variances from the shifted sums (sum of v - c, sum of (v - c)^2
// per quantity) over n particles, one reciprocal of n.
__device__ __forceinline__ void est_finish(const double* tot, double n, const double* cs,
                                           double* out) {
  const double inv_n = 1.0 / n;
  for (int q = 0; q < 3; ++q) {
    const double m1 = tot[2 * q] * inv_n;
    const double m2 = tot[2 * q + 1] * inv_n;
    out[2 * q] = cs[q] + m1;
    out[2 * q + 1] = m2 - m1 * m1;
  }
}

template <class R>
__device__ __forceinline__ void est_add(R* loc, R v0, R v1, R v2, R c0, R c1, R c2) {
  const R dx = v0 - c0, ds = v1 - c1, dt = v2 - c2;
  loc[0] += dx; loc[1] += dx * dx;
  loc[2] += ds; loc[3] += ds * ds;
  loc[4] += dt; loc[5] += dt * dt;
}

template <class R>
__global__ void __launch_bounds__(BLOCK) k_estimate(FilterArgs<R> a) {
  __shared__ double s_sum[6][WARPS];
  __shared__ bool s_last;
  const uint32_t t = a.ctl->t;
  const StateV<R> st = (t & 1) ? a.st[1] : a.st[0];
  const R c0 = st.x[0], c1 = st.s2[0], c2 = st.t2[0];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  {
    R loc[6] = {0, 0, 0, 0, 0, 0};
    const uint64_t base = ((uint64_t)blockIdx.x * BLOCK + threadIdx.x) * EST_PER_THREAD;
    if constexpr (sizeof(R) == 4) {
      if (base + EST_PER_THREAD <= a.n) {
        float4 X[EST_PER_THREAD / 4], S[EST_PER_THREAD / 4], T[EST_PER_THREAD / 4];
#pragma unroll
        for (int q = 0; q < EST_PER_THREAD / 4; ++q) {
          X[q] = *reinterpret_cast<const float4*>(st.x + base + 4 * q);
          S[q] = *reinterpret_cast<const float4*>(st.s2 + base + 4 * q);
          T[q] = *reinterpret_cast<const float4*>(st.t2 + base + 4 * q);
        }
#pragma unroll
        for (int q = 0; q < EST_PER_THREAD / 4; ++q) {
          est_add<float>(loc, X[q].x, S[q].x, T[q].x, c0, c1, c2);
          est_add<float>(loc, X[q].y, S[q].y, T[q].y, c0, c1, c2);
          est_add<float>(loc, X[q].z, S[q].z, T[q].z, c0, c1, c2);
          est_add<float>(loc, X[q].w, S[q].w, T[q].w, c0, c1, c2);
        }
      } else {
        for (uint64_t i = base; i < a.n; ++i) est_add<R>(loc, st.x[i], st.s2[i], st.t2[i], c0, c1, c2);
      }
    } else {
#pragma unroll 4
      for (int e = 0; e < EST_PER_THREAD; ++e) {
        const uint64_t i = base + e;
        if (i < a.n) est_add<R>(loc, st.x[i], st.s2[i], st.t2[i], c0, c1, c2);
      }
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      R v = loc[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) s_sum[q][warp] = (double)v;
    }
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double v = 0;
    for (int w = 0; w < WARPS; ++w) v += s_sum[threadIdx.x][w];
    a.part_est[(uint64_t)blockIdx.x * 6 + threadIdx.x] = v;
  }
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(&a.ctl->done_est, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // fold the block partials: thread i sums blocks i, i + BLOCK, ... (a fixed
  // assignment), then a shuffle tree per warp and the warps in order
  {
    double v[6] = {0, 0, 0, 0, 0, 0};
    for (uint32_t b = threadIdx.x; b < gridDim.x; b += BLOCK) {
#pragma unroll
      for (int q = 0; q < 6; ++q) v[q] += __ldcg(a.part_est + (uint64_t)b * 6 + q);
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    }
    __syncthreads();  // s_sum is reused
    if (lane == 0) {
#pragma unroll
      for (int q = 0; q < 6; ++q) s_sum[q][warp] = v[q];
    }
  }
  __syncthreads();
  __shared__ double s_tot[6];
  if (threadIdx.x < 6) {  // the warps in order, one quantity per thread
    double v = 0;
    for (int w = 0; w < WARPS; ++w) v += s_sum[threadIdx.x][w];
    s_tot[threadIdx.x] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double cs[3] = {(double)c0, (double)c1, (double)c2};
    a.ctl->est[0] = (double)t;
    est_finish(s_tot, (double)a.n, cs, a.ctl->est + 1);
    a.ctl->est[7] = a.ctl->logml;
    a.ctl->done_est = 0;
  }
  __syncthreads();
  publish_summary(a.ctl, a.ctl_mirror);
  publish_done(a.io);
}

// Posterior summaries under adaptive resampling: the particles weighted by
// w_i = exp(lambda_i) (the CDF's deterministic exp).  Per block: sums of w,
// w (v - c) and w (v - c)^2 with c the value of particle 0, in binary64; the
// last block folds the block partials in block order.
template <class R>
__global__ void __launch_bounds__(BLOCK) k_estimate_w(FilterArgs<R> a) {
  __shared__ double s_sum[7][WARPS];
  __shared__ bool s_last;
  const uint32_t t = a.ctl->t;
  const StateV<R> st = (t & 1) ? a.st[1] : a.st[0];
  const R c0 = st.x[0], c1 = st.s2[0], c2 = st.t2[0];
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  const uint64_t base = ((uint64_t)blockIdx.x * BLOCK + threadIdx.x) * EST_PER_THREAD;
  for (int e = 0; e < EST_PER_THREAD; ++e) {
    const uint64_t i = base + e;
    if (i < a.n) {
      R wr;
      (void)quant_exp<R>(a.lam[i], a.k, &wr);
      const double w = (double)wr;
      const double dx = (double)(st.x[i] - c0), ds = (double)(st.s2[i] - c1),
                   dt = (double)(st.t2[i] - c2);
      acc[0] += w;
      acc[1] += w * dx; acc[2] += w * (dx * dx);
      acc[3] += w * ds; acc[4] += w * (ds * ds);
      acc[5] += w * dt; acc[6] += w * (dt * dt);
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    double v = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_sum[q][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < 7) {
    double v = 0;
    for (int w = 0; w < WARPS; ++w) v += s_sum[threadIdx.x][w];
    a.part_est[(uint64_t)blockIdx.x * 7 + threadIdx.x] = v;
  }
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(&a.ctl->done_est, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x < 7) {
    double v = 0;
    for (uint32_t b = 0; b < gridDim.x; ++b) v += __ldcg(a.part_est + (uint64_t)b * 7 + threadIdx.x);
    s_sum[threadIdx.x][0] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double sw = s_sum[0][0];
    const double cs[3] = {(double)c0, (double)c1, (double)c2};
    a.ctl->est[0] = (double)t;
    for (int q = 0; q < 3; ++q) {
      const double m1 = s_sum[1 + 2 * q][0] / sw;
      const double m2 = s_sum[2 + 2 * q][0] / sw;
      a.ctl->est[1 + 2 * q] = cs[q] + m1;
      a.ctl->est[2 + 2 * q] = m2 - m1 * m1;
    }
    a.ctl->est[7] = a.ctl->logml;
    a.ctl->done_est = 0;
  }
  __syncthreads();
  publish_summary(a.ctl, a.ctl_mirror);
  publish_done(a.io);
}

// ---------------------------------------------------------------------------
// Resampling of a small weight vector (n <= SMALL_N) in one CTA, for
// pf_resample's systematic and stratified schemes: the same quantisation
// (W_i = floor(w_i 2^(k - e)), max w = f 2^e), the same exact CDF and the same
// positions as the multi-kernel path, so the same ancestors -- one launch
// instead of four, no scratch.  Thread t owns particles [PER t, PER t + PER);
// particle i owns the slots [first(Q_{i-1}), first(Q_i)) with first() the
// number of slot positions below n Q (systematic: j T + r; stratified:
// j T + r_j).  Errors go to *err (negative / non-finite / all-zero weights:
// ERR_WEIGHTS).
// ---------------------------------------------------------------------------
constexpr int SMALL_THREADS = 1024;
constexpr int SMALL_PER = 16;
constexpr uint64_t SMALL_N = (uint64_t)SMALL_THREADS * SMALL_PER;

template <bool STRAT>
__global__ void __launch_bounds__(SMALL_THREADS) k_resample_small(const float* w, uint32_t n,
                                                                   uint64_t seed, uint32_t filter,
                                                                   uint32_t t, uint32_t* anc,
                                                                   uint32_t* err) {
  constexpr int NW = SMALL_THREADS / 32;
  __shared__ uint32_t s_max[NW];
  __shared__ uint64_t s_tot[NW];
  __shared__ int s_bad[NW];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // per = ceil(n / threads) particles per thread, so that small n uses every thread
  const uint32_t per = (n + SMALL_THREADS - 1) / SMALL_THREADS;
  const uint32_t base = (uint32_t)threadIdx.x * per;
  float v[SMALL_PER];
  uint32_t mx = 0;
  bool bad = false;
#pragma unroll
  for (int e = 0; e < SMALL_PER; ++e) {
    v[e] = ((uint32_t)e < per && base + e < n) ? w[base + e] : 0.0f;
    if (!(v[e] >= 0.0f) || !(v[e] < INFINITY)) bad = true;
    else mx = max(mx, __float_as_uint(v[e]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const bool wbad = __any_sync(0xffffffffu, bad);
  if (lane == 0) { s_max[warp] = mx; s_bad[warp] = wbad; }
  __syncthreads();
  mx = 0;
  bool any_bad = false;
  for (int i = 0; i < NW; ++i) { mx = max(mx, s_max[i]); any_bad |= s_bad[i] != 0; }
  if (any_bad || mx == 0) {  // (every thread takes the same branch)
    if (threadIdx.x == 0) *err = ERR_WEIGHTS;
    for (uint32_t i = threadIdx.x; i < n; i += SMALL_THREADS) anc[i] = i;
    return;
  }
  int e2;
  (void)frexpf(__uint_as_float(mx), &e2);
  int k = 0;
  {
    uint32_t c = 0, m1 = n - 1;
    while (m1) { ++c; m1 >>= 1; }
    k = 61 - (int)c;  // cdf_shift(n)
  }
  const int escale = k - e2;
  uint64_t Qi[SMALL_PER];
  uint64_t run = 0;
#pragma unroll
  for (int e = 0; e < SMALL_PER; ++e) {
    if ((uint32_t)e < per && base + e < n) run += f2u64_rz(ldexpf(v[e], escale));
    Qi[e] = run;
  }
  // block exclusive scan of the thread totals
  const uint64_t incl = warp_incl_scan(run, lane);
  if (lane == 31) s_tot[warp] = incl;
  __syncthreads();
  uint64_t pre = 0, T = 0;
  for (int i = 0; i < NW; ++i) {
    const uint64_t v2 = s_tot[i];
    if (i < warp) pre += v2;
    T += v2;
  }
  const uint64_t o = pre + incl - run;  // Q just before this thread's particles
  const SysDiv dv = make_sysdiv(T);
  uint64_t r = 0;
  if (!STRAT) {
    const U4 wr = draw(seed, filter, t, 0, P_SYS_OFFSET, 0);
    r = __umul64hi(((uint64_t)wr.b << 32) | wr.a, T);
  }
  auto first = [&](uint64_t q) -> uint64_t {
    if constexpr (STRAT) return strat_first(q, n, T, dv, seed, filter, t);
    else return sys_first_slot(q, n, r, dv);
  };
  // the first slot of each own particle's successor: f[e] = first(Q_{base+e});
  // the slots of particle base + e are [f[e-1], f[e]), f[-1] from the lane below
  uint64_t f[SMALL_PER];
#pragma unroll
  for (int e = 0; e < SMALL_PER; ++e)
    f[e] = ((uint32_t)e < per && base + e < n) ? first(o + Qi[e]) : 0;
  uint64_t flast = 0;  // first(Q of this thread's last particle): the next thread's start
  {
    const uint32_t cnt = base < n ? (n - base < per ? n - base : per) : 0u;
#pragma unroll
    for (int e = 0; e < SMALL_PER; ++e)
      if ((uint32_t)e + 1 == cnt) flast = f[e];
    if (cnt == 0) flast = n;
  }
  uint64_t fprev = __shfl_up_sync(0xffffffffu, flast, 1);
  if (lane == 0) fprev = threadIdx.x == 0 ? 0 : (base < n ? first(o) : n);
#pragma unroll
  for (int e = 0; e < SMALL_PER; ++e) {
    if ((uint32_t)e >= per) break;  // (per is the same in every thread)
    const uint32_t i = base + e;
    const uint64_t fe = i < n ? f[e] : fprev;
    const uint64_t cnt = fe - fprev;
    if (cnt <= 32)
      for (uint64_t q = fprev; q < fe; ++q) anc[q] = i;
    uint32_t heavy = __ballot_sync(0xffffffffu, cnt > 32);
    while (heavy) {  // long runs by the whole warp
      const int l = __ffs(heavy) - 1;
      heavy &= heavy - 1;
      const uint64_t s0 = __shfl_sync(0xffffffffu, fprev, l), s1 = __shfl_sync(0xffffffffu, fe, l);
      const uint32_t vi = __shfl_sync(0xffffffffu, i, l);
      for (uint64_t q = s0 + lane; q < s1; q += 32) anc[q] = vi;
    }
    fprev = fe;
  }
}

// Maximum of binary32 input weights (pf_resample): non-negative floats order
// as their bit patterns.
static __global__ void __launch_bounds__(BLOCK) k_wmax(const float* w, uint64_t n, Ctl* ctl) {
  __shared__ uint32_t s_red[WARPS];
  uint32_t mx = 0;
  bool bad = false;
  for (uint64_t i = (uint64_t)blockIdx.x * BLOCK + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * BLOCK) {
    const float v = w[i];
    if (!(v >= 0.0f) || !(v < INFINITY)) bad = true;
    else mx = max(mx, __float_as_uint(v));
  }
  if (bad) atomicOr(&ctl->err, ERR_WEIGHTS);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) s_red[warp] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < WARPS; ++i) mx = max(mx, s_red[i]);
    mx = max(mx, s_red[0]);
    atomicMax(&ctl->maxenc, (unsigned long long)mx);
  }
}

}  // namespace pfk
