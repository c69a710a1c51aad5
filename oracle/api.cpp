// CPU oracle, part 4: flat C entry points for the ctypes wrapper in
// oracle/oracle.py.  TEST INFRASTRUCTURE ONLY (see oracle.h).
#include <cstring>
#include <vector>

#include "oracle.h"

namespace oracle {
template <class R>
int suffstat_known_states(const Config& cfg, const double* xpath, const double* y, uint32_t T,
                          double* bs_out, double* bt_out, double* s2_out, double* t2_out);
}

using namespace oracle;

extern "C" {

void or_philox4x32(const uint32_t* ctr, const uint32_t* key, uint32_t* out, uint64_t count) {
  for (uint64_t i = 0; i < count; ++i) {
    W4 w = philox4x32_10(ctr + 4 * i, key + 2 * i);
    std::memcpy(out + 4 * i, w.w, sizeof(w.w));
  }
}

void or_philox4x64(const uint64_t* ctr, const uint64_t* key, uint64_t* out, uint64_t count) {
  for (uint64_t i = 0; i < count; ++i) philox4x64_10(ctr + 4 * i, key + 2 * i, out + 4 * i);
}

void or_draw(uint64_t seed, uint32_t filter, uint32_t t, uint32_t j0, uint32_t count,
             uint32_t purpose, uint32_t attempt, uint32_t* out) {
  for (uint32_t i = 0; i < count; ++i) {
    W4 w = draw(seed, filter, t, j0 + i, purpose, attempt);
    std::memcpy(out + 4 * i, w.w, sizeof(w.w));
  }
}

void or_unif_f32(const uint32_t* w, uint64_t n, float* out) {
  for (uint64_t i = 0; i < n; ++i) out[i] = unif_f32(w[i]);
}

void or_det_log_f32(const float* in, float* out, uint64_t n) {
  for (uint64_t i = 0; i < n; ++i) out[i] = det_log<float>(in[i]);
}
void or_det_log_f64(const double* in, double* out, uint64_t n) {
  for (uint64_t i = 0; i < n; ++i) out[i] = det_log<double>(in[i]);
}
void or_det_exp_core_f32(const float* in, float* out, uint64_t n) {
  for (uint64_t i = 0; i < n; ++i) out[i] = det_exp_core<float>(in[i]);
}
void or_det_exp_core_f64(const double* in, double* out, uint64_t n) {
  for (uint64_t i = 0; i < n; ++i) out[i] = det_exp_core<double>(in[i]);
}
void or_det_cos2pi_f32(const float* in, float* out, uint64_t n) {
  for (uint64_t i = 0; i < n; ++i) out[i] = det_cos2pi<float>(in[i]);
}
void or_det_cos2pi_f64(const double* in, double* out, uint64_t n) {
  for (uint64_t i = 0; i < n; ++i) out[i] = det_cos2pi<double>(in[i]);
}
void or_det_sincos2pi_f32(const float* in, float* s, float* c, uint64_t n) {
  for (uint64_t i = 0; i < n; ++i) det_sincos2pi<float>(in[i], &s[i], &c[i]);
}
void or_det_sincos2pi_f64(const double* in, double* s, double* c, uint64_t n) {
  for (uint64_t i = 0; i < n; ++i) det_sincos2pi<double>(in[i], &s[i], &c[i]);
}
void or_quant_exp_f32(const float* dl, uint64_t n, int k, uint64_t* W, float* e) {
  for (uint64_t i = 0; i < n; ++i) W[i] = quant_exp<float>(dl[i], k, &e[i]);
}
void or_quant_exp_f64(const double* dl, uint64_t n, int k, uint64_t* W, double* e) {
  for (uint64_t i = 0; i < n; ++i) W[i] = quant_exp<double>(dl[i], k, &e[i]);
}

void or_normals_f32(uint64_t seed, uint32_t filter, uint32_t t, uint32_t purpose, uint64_t n,
                    float* out) {
  for (uint64_t j = 0; j < n; ++j)
    out[j] = bm_normal<float>(draw(seed, filter, t, (uint32_t)j, purpose, 0));
}
void or_normals_f64(uint64_t seed, uint32_t filter, uint32_t t, uint32_t purpose, uint64_t n,
                    double* out) {
  for (uint64_t j = 0; j < n; ++j)
    out[j] = bm_normal<double>(draw(seed, filter, t, (uint32_t)j, purpose, 0));
}

// The propagation draws of slots 0..n-1: out[5 j + (0..4)] = Zx, Zs, Us, Zt, Ut.
void or_theta_draws_f32(uint64_t seed, uint32_t filter, uint32_t t, uint64_t n, float* out) {
  for (uint64_t j = 0; j < n; ++j) {
    float* o = out + 5 * j;
    theta_draws<float>(seed, filter, t, (uint32_t)j, o, o + 1, o + 2, o + 3, o + 4);
  }
}
void or_theta_draws_f64(uint64_t seed, uint32_t filter, uint32_t t, uint64_t n, double* out) {
  for (uint64_t j = 0; j < n; ++j) {
    double* o = out + 5 * j;
    theta_draws<double>(seed, filter, t, (uint32_t)j, o, o + 1, o + 2, o + 3, o + 4);
  }
}

int or_gamma_f32(double a, uint64_t seed, uint32_t filter, uint32_t t, uint32_t purpose,
                 uint64_t n, float* out) {
  double d, c, K;
  mt_constants(a, &d, &c, &K);
  int fail = 0;
  for (uint64_t j = 0; j < n; ++j)
    out[j] = gamma_mt<float>((float)d, (float)c, (float)K, seed, filter, t, (uint32_t)j, purpose,
                             &fail);
  return fail;
}
int or_gamma_f64(double a, uint64_t seed, uint32_t filter, uint32_t t, uint32_t purpose,
                 uint64_t n, double* out) {
  double d, c, K;
  mt_constants(a, &d, &c, &K);
  int fail = 0;
  for (uint64_t j = 0; j < n; ++j)
    out[j] = gamma_mt<double>(d, c, K, seed, filter, t, (uint32_t)j, purpose, &fail);
  return fail;
}

void or_mt_constants(double a, double* out) { mt_constants(a, &out[0], &out[1], &out[2]); }

int or_cdf_shift(uint64_t n) { return cdf_shift(n); }
void or_cdf_scan(const uint64_t* W, uint64_t n, uint64_t* Q) { cdf_scan(W, n, Q); }
int or_quantize_weights_f32(const float* w, uint64_t n, uint64_t* W) {
  return quantize_weights_f32(w, n, W);
}

uint64_t or_systematic_offset(uint64_t T, uint64_t seed, uint32_t filter, uint32_t t) {
  return systematic_offset(T, seed, filter, t);
}
uint64_t or_stratified_offset(uint64_t T, uint64_t seed, uint32_t filter, uint32_t t, uint64_t j) {
  return stratified_offset(T, seed, filter, t, j);
}
void or_spacing_prefix(uint64_t n, uint64_t seed, uint32_t filter, uint32_t t, uint64_t* S) {
  std::vector<uint64_t> v;
  spacing_prefix(n, seed, filter, t, &v);
  std::memcpy(S, v.data(), (n + 1) * sizeof(uint64_t));
}

// positions: 0 = multinomial (spacings), 1 = systematic, 2 = stratified
// method: 0 = sequential walk, 1 = naive O(n^2), 2 = cut-point method
void or_resample_method(const uint64_t* Q, uint64_t n, int positions, int method,
                        uint64_t seed, uint32_t filter, uint32_t t, uint32_t* anc) {
  uint64_t T = Q[n - 1];
  Positions P = positions == 1   ? systematic_positions(n, T, seed, filter, t)
                : positions == 2 ? stratified_positions(n, T, seed, filter, t)
                                 : multinomial_positions(n, T, seed, filter, t);
  if (method == 0) {
    walk(Q, n, P, anc);
  } else if (method == 1) {
    naive_search(Q, n, P, anc);
  } else {
    std::vector<uint64_t> L(n);
    std::vector<uint32_t> I(n);
    cutpoint_search(Q, n, L.data(), I.data());
    cutpoint_method(Q, n, I.data(), P, anc);
  }
}

void or_systematic_with_offset(const uint64_t* Q, uint64_t n, uint64_t r, uint32_t* anc) {
  Positions P = systematic_positions_with_offset(n, Q[n - 1], r);
  walk(Q, n, P, anc);
}

void or_cutpoint_search(const uint64_t* Q, uint64_t n, uint64_t* L, uint32_t* I) {
  cutpoint_search(Q, n, L, I);
}

// Cut-point method for explicit integer positions U_j in [0, T) (A = 1).
void or_cutpoint_method_int(const uint64_t* Q, uint64_t n, const uint32_t* I,
                            const uint64_t* U, uint64_t m, uint32_t* anc, uint64_t* bucket) {
  uint64_t T = Q[n - 1];
  Positions P;
  P.A = 1;
  P.B.resize(m);
  P.bucket.resize(m);
  for (uint64_t j = 0; j < m; ++j) {
    P.B[j] = U[j];
    P.bucket[j] = (uint64_t)(((u128)n * U[j]) / T);
    bucket[j] = P.bucket[j];
  }
  for (uint64_t j = 0; j < m; ++j) {
    uint64_t k = I[P.bucket[j]];
    while (k < n && (u128)Q[k] <= P.B[j]) ++k;
    anc[j] = (uint32_t)k;
  }
}

void or_resample_cdf(const uint64_t* Q, uint64_t n, int scheme, uint64_t seed,
                     uint32_t filter, uint32_t t, uint32_t* anc) {
  resample(Q, n, scheme, seed, filter, t, anc);
}

// pf_resample semantics: quantise FP32 weights, scan, resample.
int or_resample_weights(const float* w, uint64_t n, int scheme, uint64_t seed,
                        uint32_t filter, uint32_t t, uint32_t* anc) {
  std::vector<uint64_t> W(n), Q(n);
  if (quantize_weights_f32(w, n, W.data()) != 0) return 1;
  cdf_scan(W.data(), n, Q.data());
  resample(Q.data(), n, scheme, seed, filter, t, anc);
  return 0;
}

typedef struct {
  uint64_t n, seed;
  uint32_t filter_id;
  int32_t scheme;
  int32_t precision;
  int32_t known_variances;
  double x0_mean, x0_var, a_sigma, b_sigma, a_tau, b_tau, sigma2, tau2;
  int32_t algorithm;
  double ess_frac;
} or_config;

static Config to_cfg(const or_config* c) {
  Config cfg;
  cfg.n = c->n; cfg.seed = c->seed; cfg.filter_id = c->filter_id; cfg.scheme = c->scheme;
  cfg.precision = c->precision; cfg.known_variances = c->known_variances;
  cfg.x0_mean = c->x0_mean; cfg.x0_var = c->x0_var; cfg.a_sigma = c->a_sigma;
  cfg.b_sigma = c->b_sigma; cfg.a_tau = c->a_tau; cfg.b_tau = c->b_tau;
  cfg.sigma2 = c->sigma2; cfg.tau2 = c->tau2;
  cfg.algorithm = c->algorithm;
  cfg.ess_frac = c->ess_frac;
  return cfg;
}

void* or_pl_create(const or_config* c) { return make_filter(to_cfg(c)); }
int or_pl_step(void* h, double y) { return ((FilterBase*)h)->step(y); }
void or_pl_estimate(void* h, double* out) {
  Estimates e = ((FilterBase*)h)->estimate();
  std::memcpy(out, &e, sizeof(e));
}
void or_pl_state(void* h, double* x, double* s2, double* t2, double* bs, double* bt) {
  ((FilterBase*)h)->state_as_double(x, s2, t2, bs, bt);
}
void or_pl_state_raw(void* h, void* x, void* s2, void* t2, void* bs, void* bt) {
  ((FilterBase*)h)->state_raw(x, s2, t2, bs, bt);
}
void or_pl_ancestors(void* h, uint32_t* anc) {
  const std::vector<uint32_t>& a = ((FilterBase*)h)->last_ancestors();
  std::memcpy(anc, a.data(), a.size() * sizeof(uint32_t));
}
void or_pl_cdf(void* h, uint64_t* Q) {
  const std::vector<uint64_t>& q = ((FilterBase*)h)->last_cdf();
  std::memcpy(Q, q.data(), q.size() * sizeof(uint64_t));
}
void or_pl_destroy(void* h) { delete (FilterBase*)h; }
int or_pl_resampled(void* h) { return ((FilterBase*)h)->last_resampled() ? 1 : 0; }
int or_ess_resample(const uint64_t* W, uint64_t n, double ess_frac) {
  return ess_resample(W, n, ess_frac) ? 1 : 0;
}

int or_suffstat_known_states(const or_config* c, const double* xpath, const double* y,
                             uint32_t T, double* bs, double* bt, double* s2, double* t2) {
  Config cfg = to_cfg(c);
  if (cfg.precision == 0)
    return suffstat_known_states<float>(cfg, xpath, y, T, bs, bt, s2, t2);
  return suffstat_known_states<double>(cfg, xpath, y, T, bs, bt, s2, t2);
}

void or_kalman(const double* y, uint32_t T, double m0, double P0, double sigma2, double tau2,
               double* mean, double* var, double* loglik) {
  kalman(y, T, m0, P0, sigma2, tau2, mean, var, loglik);
}

}  // extern "C"
