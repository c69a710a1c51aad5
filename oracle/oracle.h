// CPU oracle for the particle-learning cycle of McAlinn & Nakatsuma,
// "Parallel Resampling for Fully Parallelized Particle Filters" (arXiv 1212.1639).
//
// TEST INFRASTRUCTURE ONLY.  This code is the plain, slow, single-threaded
// reference that the CUDA path is checked against.  Only tests/,
// __graft_entry__.smoke() and bench.py's cpu_baseline / reference leg may load
// it.  It shares no code, header, table or constant generator with the CUDA
// library; where both must compute the same bits (Philox, the deterministic
// elementary functions, the fixed-point CDF) each side implements the same
// published definition in its own code.
//
// Every floating-point step is written as an explicit sequence of IEEE-754
// operations -- each a separately rounded add, multiply, divide or square
// root, or a fused multiply-add where the code calls std::fma -- and the file
// is compiled with -ffp-contract=off, so that the compiler fuses nothing
// else: the same sequence in the CUDA library (built with -fmad=false, fused
// multiply-adds written explicitly) gives the same bits.
//
// Parity status: every function here is pinned by tests under tests/ (see the
// "pin" line in each function's comment) except where marked
// "parity unpinned".
#pragma once
#include <cstddef>
#include <cstdint>
#include <vector>

namespace oracle {

typedef unsigned __int128 u128;

// ---------------------------------------------------------------------------
// Counter-based RNG: Philox4x32-10 and Philox4x64-10 as defined by Salmon,
// Moraes, Dror & Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11).
// pin: 4x32 against triton's interpreter implementation, 4x64 against numpy's
// Philox bit generator (tests/test_oracle_rng.py).
// ---------------------------------------------------------------------------
struct W4 { uint32_t w[4]; };
W4 philox4x32_10(const uint32_t ctr[4], const uint32_t key[2]);
void philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);

// Draw purposes: the fourth counter word is purpose | attempt << 8.
enum Purpose : uint32_t {
  P_INIT_X = 1, P_INIT_SIGMA = 2, P_INIT_TAU = 3,
  P_STATE = 4, P_GAMMA_SIGMA = 5, P_GAMMA_TAU = 6,
  P_SYS_OFFSET = 7, P_SPACING = 8, P_STRATIFIED = 9, P_BOOT_STATE = 10,
};

// One 128-bit draw addressed by (seed, filter, t, j, purpose, attempt):
// counter = (j, t, filter, purpose | attempt << 8), key = (seed lo, seed hi).
W4 draw(uint64_t seed, uint32_t filter, uint32_t t, uint32_t j, uint32_t purpose,
        uint32_t attempt);

// Uniforms on (0,1), exactly representable (no rounding in the conversion).
float unif_f32(uint32_t w);                     // (2*(w>>9)+1) * 2^-24
double unif_f64(uint32_t lo, uint32_t hi);      // (2*(R>>12)+1) * 2^-53, R = hi:lo
double unif_f64_32(uint32_t w);                 // (2*w+1) * 2^-33

// ---------------------------------------------------------------------------
// Deterministic elementary functions (same operation sequence on CPU and GPU).
// pin: against libm within a few ulp over dense samples
// (tests/test_oracle_detmath.py).
// ---------------------------------------------------------------------------
template <class R> R det_log(R x);          // x > 0 (binary32: +inf, NaN returned unchanged)
template <class R> R det_exp_core(R r);     // Taylor polynomial of exp on |r| <= ~0.35
template <class R> R det_cos2pi(R u);       // cos(2*pi*u) for u in [0, 1]
template <class R> void det_sincos2pi(R u, R* s, R* c);  // both, same reduction

// Quantised weight of the fixed-point CDF: for dl = l_i - max_j l_j <= 0,
// *e = exp(dl) as evaluated by the deterministic exp (0 below dl = -50),
// return floor(*e * 2^k) clamped to 2^k.
template <class R> uint64_t quant_exp(R dl, int k, R* e);

// Standard normal by Box-Muller (first output) from one 128-bit draw, both
// outputs (cos and sin branches), and the extra uniform the gamma sampler
// needs from the same draw.
template <class R> R bm_normal(const W4& w);
template <class R> void bm_normal2(const W4& w, R* zc, R* zs);
template <class R> R extra_uniform(const W4& w);

// Gamma(a, 1) by Marsaglia & Tsang (2000), a >= 1, with d = a - 1/3,
// c = 1/sqrt(9 d) and the squeeze coefficient K = 0.0331 (2/3) / d given in
// the working precision: v = fma(c, Z, 1); accept d v^3 when v > 0 and
// U < fma(-K, Z^4, 1) (the squeeze), else when
// log U < fma(d, (1 - v^3) + log v^3, Z^2 / 2).  Attempt k uses its own draw
// (purpose, attempt k); after 16 rejections *fail is set and d returned.
// pin: gamma KS / moments (tests/test_oracle_rng.py); the squeeze bound
// 1 - K Z^4 <= exp(g(Z)) over a dense grid of d and Z
// (tests/test_oracle_rng.py::test_gamma_squeeze_is_a_lower_bound).
template <class R> R gamma_mt(R d, R c, R K, uint64_t seed, uint32_t filter, uint32_t t,
                              uint32_t j, uint32_t purpose, int* fail);
// The same with the first attempt's (Z, U) given; attempts k >= 1 use draw
// (purpose, k).
template <class R> R gamma_mt_from(R d, R c, R K, R Z0, R U0, uint64_t seed, uint32_t filter,
                                   uint32_t t, uint32_t j, uint32_t purpose, int* fail);

// The draws of one propagation step for slot j: two 128-bit draws,
// A = (j, t, STATE, attempt 0) and B = (j, t, STATE, attempt 1).  Box-Muller
// on A gives the state normal (cos branch) and the first normal of the
// sigma^2 gamma draw (sin branch); A's extra uniform is that draw's first
// uniform; B gives the tau^2 gamma draw's first normal and uniform.
template <class R> void theta_draws(uint64_t seed, uint32_t filter, uint32_t t, uint32_t j,
                                    R* Zx, R* Zs, R* Us, R* Zt, R* Ut);

// Shape constants of Marsaglia-Tsang for shape a, in double: d = a - 1/3,
// c = 1/sqrt(9 d) and the squeeze coefficient K = 0.0331 (2/3) / d.
void mt_constants(double a, double* d, double* c, double* K);

// ---------------------------------------------------------------------------
// Fixed-point CDF (the resampling CDF q(i) of the paper's Section 3.1 in
// exact integers) and resampling.
// ---------------------------------------------------------------------------
int cdf_shift(uint64_t n);  // k = 61 - ceil(log2 n)

// Inclusive prefix sum Q_i = sum_{l<=i} W_l (exact u64).
void cdf_scan(const uint64_t* W, uint64_t n, uint64_t* Q);

// W_i = floor(w_i * 2^(k - e)) where max_i w_i = f * 2^e, f in [0.5, 1).
// Returns 0 on success, -1 if any w_i is negative / not finite or all are 0.
int quantize_weights_f32(const float* w, uint64_t n, uint64_t* W);

// Resampling positions.  Slot j's position in CDF units is B_j / A (a
// rational number in [0, T)); its ancestor is the first i with Q_i > B_j / A,
// i.e. the number of i with Q_i * A <= B_j.
struct Positions {
  std::vector<u128> B;           // n keys, strictly increasing
  u128 A;
  std::vector<uint64_t> bucket;  // floor(n * B_j / (A * T)): the cut-point bucket
};
// Systematic (paper Section 3.1): B_j = j*T + r, A = n, with r = floor(R*T/2^64)
// and R the 64-bit draw (seed, filter, t, 0, SYS_OFFSET).
Positions systematic_positions(uint64_t n, uint64_t T, uint64_t seed, uint32_t filter,
                               uint32_t t);
Positions systematic_positions_with_offset(uint64_t n, uint64_t T, uint64_t r);
uint64_t systematic_offset(uint64_t T, uint64_t seed, uint32_t filter, uint32_t t);
// Stratified (paper Section 3.1, "Stratified Resampling"): one uniform in
// each of the n equal strata, B_j = j*T + r_j, A = n, r_j = floor(R_j*T/2^64)
// with R_j the 64-bit word pair 2(j mod 2), 2(j mod 2)+1 of the draw
// (seed, filter, t, floor(j/2), STRATIFIED).
uint64_t stratified_offset(uint64_t T, uint64_t seed, uint32_t filter, uint32_t t, uint64_t j);
Positions stratified_positions(uint64_t n, uint64_t T, uint64_t seed, uint32_t filter,
                               uint32_t t);
// Multinomial with sorted uniforms: order statistics of n iid uniforms
// generated directly in ascending order by exponential spacings
// (Carpenter, Clifford & Fearnhead 1999): E_0..E_n iid Exp(1) in 2^-31 fixed
// point, S_j = E_0 + ... + E_j, B_j = S_j * T, A = S_n.
void spacing_prefix(uint64_t n, uint64_t seed, uint32_t filter, uint32_t t,
                    std::vector<uint64_t>* S /* n+1 entries */);
Positions multinomial_positions(uint64_t n, uint64_t T, uint64_t seed, uint32_t filter,
                                uint32_t t);

// Ancestor search strategies (all must agree exactly):
// sequential walk over sorted positions (paper Section 3.1, multinomial with
// sorted uniforms), naive O(n^2) search (paper Section 3.1), and the
// cut-point method seeded by the cut-point table (paper Section 3.2).
void walk(const uint64_t* Q, uint64_t n, const Positions& P, uint32_t* anc);
void naive_search(const uint64_t* Q, uint64_t n, const Positions& P, uint32_t* anc);
// Parallelized Cut-Point Search (paper Section 3.2) in 0-based form:
// L_i = ceil(n * Q_i / T); I_k = i for k in [L_{i-1}, L_i).
void cutpoint_search(const uint64_t* Q, uint64_t n, uint64_t* L, uint32_t* I);
// Cut-Point Method: bucket b_j = floor(n * B_j / (A * T)), start at I_{b_j},
// climb while Q_k * A <= B_j.
void cutpoint_method(const uint64_t* Q, uint64_t n, const uint32_t* I, const Positions& P,
                     uint32_t* anc);

enum Scheme {
  MULTINOMIAL = 0, SYSTEMATIC = 1, MULTINOMIAL_CUTPOINT = 2, SYSTEMATIC_CUTPOINT = 3,
  STRATIFIED = 4
};

// Ancestors of one resampling step from a finished CDF.
void resample(const uint64_t* Q, uint64_t n, int scheme, uint64_t seed, uint32_t filter,
              uint32_t t, uint32_t* anc);

// ---------------------------------------------------------------------------
// Particle learning for the local-level model y_t = x_t + v_t,
// x_t = x_{t-1} + w_t, v ~ N(0, sigma^2), w ~ N(0, tau^2)  (paper Section 4),
// with conjugate inverse-gamma learning of sigma^2 and tau^2 (paper Section 2,
// Algorithm "Particle Learning").
// ---------------------------------------------------------------------------
struct Config {
  uint64_t n, seed;
  uint32_t filter_id;
  int32_t scheme;
  int32_t precision;  // 0 = FP32 state (paper's sp), 1 = FP64 state (paper's dp)
  double x0_mean, x0_var, a_sigma, b_sigma, a_tau, b_tau;
  int32_t known_variances;
  double sigma2, tau2;
  int32_t algorithm;  // 0 = particle learning, 1 = bootstrap filter (known variances)
  // Adaptive resampling (particle learning only): 0 = resample every cycle
  // (the paper's setting); in (0, 1], resample only when the effective
  // sample size of the combined weights is below ess_frac * n, else carry
  // the log-weights to the next cycle.
  double ess_frac;
};

struct Estimates {
  double t, x_mean, x_var, sigma2_mean, sigma2_var, tau2_mean, tau2_var, log_marglik;
};

class FilterBase {
 public:
  virtual ~FilterBase() {}
  virtual int step(double y) = 0;
  virtual Estimates estimate() const = 0;
  virtual void state_as_double(double* x, double* s2, double* t2, double* bs, double* bt) const = 0;
  virtual void state_raw(void* x, void* s2, void* t2, void* bs, void* bt) const = 0;
  virtual const std::vector<uint32_t>& last_ancestors() const = 0;
  virtual const std::vector<uint64_t>& last_cdf() const = 0;
  virtual bool last_resampled() const = 0;
};

FilterBase* make_filter(const Config& cfg);

// Adaptive resampling decision (Kong, Liu & Wong 1994; Liu & Chen 1998):
// resample iff ESS = (sum W)^2 / sum W^2 < ess_frac * n for the quantised
// weights W, evaluated as A * A < (ess_frac * n) * B in binary64 with
// A = sum W and B = sum W^2 exact integers, each rounded to nearest once.
// pin: exact rational comparison away from ties (tests/test_oracle_pl.py).
bool ess_resample(const uint64_t* W, uint64_t n, double ess_frac);

// Kalman filter for the local-level model with known variances (the closed
// form of the Bayes filter, paper Section 2).  Outputs the filtered mean and
// variance of x_t for t = 1..T and the exact log-likelihood.
void kalman(const double* y, uint32_t T, double m0, double P0, double sigma2, double tau2,
            double* mean, double* var, double* loglik);

}  // namespace oracle
