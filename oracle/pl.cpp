// CPU oracle, part 3: particle learning for the local-level model and the
// Kalman filter.  TEST INFRASTRUCTURE ONLY (see oracle.h).
//
// The cycle follows Algorithm "Particle Learning" of the paper (Section 2):
//   Step 1  resample z_t with weights w proportional to p(y_{t+1} | z_t),
//   Step 2  propagate x_{t+1} ~ p(x_{t+1} | z~_t, y_{t+1}),
//   Step 3  update the sufficient statistics s_{t+1} = S(s~_t, x_{t+1}, y_{t+1}),
//   Step 4  draw theta ~ p(theta | s_{t+1}),
// specialised to the model of Section 4 by the conjugate derivation of
// Carvalho, Johannes, Lopes & Polson (2010):
//   p(y_{t+1} | x_t, theta)      = N(y; x_t, sigma^2 + tau^2)
//   p(x_{t+1} | x_t, theta, y)    = N(mu, V), V = sigma^2 tau^2 / (sigma^2 + tau^2),
//                                   mu = (x_t sigma^2 + y tau^2) / (sigma^2 + tau^2)
//                                   (evaluated with r = 1/(sigma^2 + tau^2):
//                                   V = (sigma^2 tau^2) r, mu = fma(x_t, sigma^2, y tau^2) r,
//                                   x_{t+1} = fma(sqrt V, Z, mu))
//   b_sigma <- b_sigma + (y - x_{t+1})^2 / 2,  b_tau <- b_tau + (x_{t+1} - x_t)^2 / 2
//   sigma^2 ~ IG(a_sigma0 + (t+1)/2, b_sigma), tau^2 ~ IG(a_tau0 + (t+1)/2, b_tau).
// pin: Kalman filter with known variances, conjugate inverse-gamma posterior
// with known states, prior means (tests/test_oracle_pl.py).
//
// Adaptive resampling (cfg.ess_frac > 0; not in the paper, which resamples
// every cycle): the filter carries log-weights lambda_i (0 after a
// resampling).  Step 1 combines them with the predictive weights,
// L_i = lambda_i + log p(y_{t+1} | z_t^(i)), builds the CDF from L and
// resamples only when the effective sample size of those weights is below
// ess_frac * n; otherwise every particle is its own ancestor and carries
// lambda'_i = L_i - max L.  This is the fully adapted auxiliary particle filter
// with an ESS trigger (Pitt & Shephard 1999; Kong, Liu & Wong 1994).  The log
// marginal likelihood increment is log sum_i e^{L_i} - log sum_i e^{lambda_i}
// (log n after a resampling), and the posterior summaries are weighted by
// e^{lambda_i}.
// pin: Kalman filter with known variances (adaptive and never-resampling
// forms), equality with the always-resampling filter when ess_frac = 1.
#include <cmath>
#include <limits>

#include "oracle.h"

namespace oracle {

static const double LOG_2PI = 0x1.d67f1c864beb5p+0;

// Sufficient-statistic storage: 2^-32 fixed point (exact sums) for FP32
// state, binary64 for FP64 state.
template <class R> struct Suff;
template <> struct Suff<float> {
  typedef uint64_t B;
  static B from_prior(double b) { return (uint64_t)(b * 0x1p32); }
  static double as_double(B b) { return (double)b * 0x1p-32; }
  // b + (resid^2)/2 with resid in the working precision: resid^2 2^31 is
  // (resid^2 / 2) 2^32 exactly (a power-of-two scaling), truncated.
  static B add_half_square(B b, float resid, int* fail) {
    float r2 = resid * resid;
    float v = r2 * 0x1p31f;
    if (!(v < 0x1p63f)) {
      *fail = 1;
      return b;
    }
    return b + (uint64_t)v;
  }
  // The inverse-gamma draw b 2^-32 / G.  b 2^-32 in binary32 is taken from
  // the two 32-bit halves, each converted to nearest, joined by one fused
  // multiply-add: fma(lo, 2^-32, hi).
  static float ig(B b, float G) {
    float hi = (float)(uint32_t)(b >> 32);
    float lo = (float)(uint32_t)b;
    float bs = std::fma(lo, 0x1p-32f, hi);
    return bs / G;
  }
};
template <> struct Suff<double> {
  typedef double B;
  static B from_prior(double b) { return b; }
  static double as_double(B b) { return b; }
  static B add_half_square(B b, double resid, int*) {
    double r2 = resid * resid;
    double h = 0.5 * r2;
    return b + h;
  }
  static double ig(B b, double G) { return b / G; }
};

// Exact sum of exp(l_i - m) for the log marginal likelihood: 2^-96 fixed
// point for binary32 terms (every term >= 2^-73 or 0 is then an integer),
// plain sequential binary64 sum for binary64 terms.
struct ExpSumF32 {
  u128 s = 0;
  void add(float e) {
    if (e == 0.0f) return;
    int ex;
    float f = std::frexp(e, &ex);  // e = f 2^ex, f in [0.5, 1)
    uint64_t mant = (uint64_t)(f * 0x1p24f);
    s += (u128)mant << (ex + 72);
  }
  double value() const {
    double hi = std::ldexp((double)(uint64_t)(s >> 64), -32);
    double lo = std::ldexp((double)(uint64_t)s, -96);
    return hi + lo;
  }
};
struct ExpSumF64 {
  double s = 0.0;
  void add(double e) { s += e; }
  double value() const { return s; }
};
template <class R> struct ExpSum;
template <> struct ExpSum<float> { typedef ExpSumF32 T; };
template <> struct ExpSum<double> { typedef ExpSumF64 T; };

// log p(y | x, sigma^2, tau^2) + log(2 pi)/2 = -(log s + (y - x)^2 / s) / 2,
// s = sigma^2 + tau^2.
template <class R> static inline R log_pred(R x, R s2, R t2, R y) {
  R s = s2 + t2;
  R dx = y - x;
  R q = dx * dx;
  R lg = det_log(s);
  R r = q / s;
  R a = lg + r;
  return (R)-0.5 * a;
}

bool ess_resample(const uint64_t* W, uint64_t n, double ess_frac) {
  uint64_t T = 0;
  u128 B = 0;
  for (uint64_t i = 0; i < n; ++i) {
    T += W[i];
    B += (u128)W[i] * W[i];
  }
  const double A = (double)T;    // correctly rounded conversions
  const double Bd = (double)B;
  const double lhs = A * A;
  const double f = ess_frac * (double)n;
  const double rhs = f * Bd;
  return lhs < rhs;
}

template <class R> class Filter : public FilterBase {
  typedef typename Suff<R>::B B;

 public:
  explicit Filter(const Config& c) : cfg(c), n(c.n), t(0), k(cdf_shift(c.n)), logml(0.0) {
    x.resize(n); s2.resize(n); t2.resize(n); bs.resize(n); bt.resize(n);
    anc.resize(n); Q.resize(n);
    ess = cfg.ess_frac > 0.0 && cfg.algorithm == 0;
    if (ess) lam.assign(n, (R)0);
    slam = (double)n;
    const R x0m = (R)cfg.x0_mean;
    const R sdx = (R)std::sqrt(cfg.x0_var);
    double ds, cs, ks, dt, ct, kt;
    mt_constants(cfg.a_sigma, &ds, &cs, &ks);
    mt_constants(cfg.a_tau, &dt, &ct, &kt);
    for (uint64_t j = 0; j < n; ++j) {
      W4 w = draw(cfg.seed, cfg.filter_id, 0, (uint32_t)j, P_INIT_X, 0);
      R Z = bm_normal<R>(w);
      R p = sdx * Z;
      x[j] = x0m + p;
      if (cfg.known_variances) {
        s2[j] = (R)cfg.sigma2;
        t2[j] = (R)cfg.tau2;
        bs[j] = Suff<R>::from_prior(cfg.b_sigma);
        bt[j] = Suff<R>::from_prior(cfg.b_tau);
      } else {
        bs[j] = Suff<R>::from_prior(cfg.b_sigma);
        bt[j] = Suff<R>::from_prior(cfg.b_tau);
        R Gs = gamma_mt<R>((R)ds, (R)cs, (R)ks, cfg.seed, cfg.filter_id, 0, (uint32_t)j,
                           P_INIT_SIGMA, &fail);
        R Gt = gamma_mt<R>((R)dt, (R)ct, (R)kt, cfg.seed, cfg.filter_id, 0, (uint32_t)j,
                           P_INIT_TAU, &fail);
        s2[j] = Suff<R>::ig(bs[j], Gs);
        t2[j] = Suff<R>::ig(bt[j], Gt);
      }
    }
  }

  int step(double y) override {
    if (cfg.algorithm == 1) return step_bootstrap(y);
    const R yr = (R)y;
    // Step 1: predictive weights and the resampling CDF (with adaptive
    // resampling: combined with the carried log-weights).
    std::vector<R> ell(n);
    for (uint64_t i = 0; i < n; ++i) {
      ell[i] = log_pred<R>(x[i], s2[i], t2[i], yr);
      if (ess) ell[i] = lam[i] + ell[i];
    }
    R m = ell[0];
    for (uint64_t i = 1; i < n; ++i)
      if (ell[i] > m) m = ell[i];
    if (!std::isfinite((double)m)) return 4;
    std::vector<uint64_t> W(n);
    typename ExpSum<R>::T S;
    for (uint64_t i = 0; i < n; ++i) {
      R e;
      R dl = ell[i] - m;
      W[i] = quant_exp<R>(dl, k, &e);
      S.add(e);
    }
    cdf_scan(W.data(), n, Q.data());
    if (ess) {
      logml += (double)m + std::log(S.value()) - std::log(slam) - 0.5 * LOG_2PI;
      resampled = ess_resample(W.data(), n, cfg.ess_frac);
      if (resampled) {
        resample(Q.data(), n, cfg.scheme, cfg.seed, cfg.filter_id, t, anc.data());
        for (uint64_t j = 0; j < n; ++j) lam[j] = (R)0;
        slam = (double)n;
      } else {
        for (uint64_t j = 0; j < n; ++j) {
          anc[j] = (uint32_t)j;
          lam[j] = ell[j] - m;
        }
        slam = S.value();
      }
    } else {
      logml += (double)m + std::log(S.value()) - std::log((double)n) - 0.5 * LOG_2PI;
      resample(Q.data(), n, cfg.scheme, cfg.seed, cfg.filter_id, t, anc.data());
    }

    // Steps 2-4: propagate, update sufficient statistics, draw theta.
    double ds, cs, ks, dt, ct, kt;
    mt_constants(cfg.a_sigma + 0.5 * (double)(t + 1), &ds, &cs, &ks);
    mt_constants(cfg.a_tau + 0.5 * (double)(t + 1), &dt, &ct, &kt);
    std::vector<R> xn(n), s2n(n), t2n(n);
    std::vector<B> bsn(n), btn(n);
    for (uint64_t j = 0; j < n; ++j) {
      const uint32_t a = anc[j];
      const R xa = x[a], sa = s2[a], ta = t2[a];
      // V = sigma^2 tau^2 / s and mu = (x sigma^2 + y tau^2) / s share one
      // correctly rounded reciprocal of s = sigma^2 + tau^2
      R s = sa + ta;
      R rs_inv = (R)1 / s;
      R p = sa * ta;
      R V = p * rs_inv;
      R n2 = yr * ta;
      R nn = std::fma(xa, sa, n2);
      R mu = nn * rs_inv;
      R sv = std::sqrt(V);
      R Z, Zs, Us, Zt, Ut;
      theta_draws<R>(cfg.seed, cfg.filter_id, t, (uint32_t)j, &Z, &Zs, &Us, &Zt, &Ut);
      R xj = std::fma(sv, Z, mu);
      xn[j] = xj;
      if (cfg.known_variances) {
        s2n[j] = sa; t2n[j] = ta; bsn[j] = bs[a]; btn[j] = bt[a];
        continue;
      }
      R rs = resid_obs(y, yr, xj);
      R rt = xj - xa;
      bsn[j] = Suff<R>::add_half_square(bs[a], rs, &fail);
      btn[j] = Suff<R>::add_half_square(bt[a], rt, &fail);
      R Gs = gamma_mt_from<R>((R)ds, (R)cs, (R)ks, Zs, Us, cfg.seed, cfg.filter_id, t,
                              (uint32_t)j, P_GAMMA_SIGMA, &fail);
      R Gt = gamma_mt_from<R>((R)dt, (R)ct, (R)kt, Zt, Ut, cfg.seed, cfg.filter_id, t,
                              (uint32_t)j, P_GAMMA_TAU, &fail);
      s2n[j] = Suff<R>::ig(bsn[j], Gs);
      t2n[j] = Suff<R>::ig(btn[j], Gt);
    }
    x.swap(xn); s2.swap(s2n); t2.swap(t2n); bs.swap(bsn); bt.swap(btn);
    ++t;
    return fail ? 4 : 0;
  }

  // Algorithm "Particle Filtering" (paper Section 2) for the local-level
  // model with known sigma^2, tau^2 (the bootstrap filter):
  //   Step 1  propagate x_t ~ p(x_t | x~_{t-1}) = N(x~_{t-1}, tau^2),
  //   Step 2  weights w_t proportional to p(y_t | x_t) = N(y_t; x_t, sigma^2),
  //   Step 3  resample x~_t from x_t with the weights w_t.
  // The normal of step 1 is Box-Muller's first output from the draw
  // (seed, filter, t, i, BOOT_STATE).  The weights, the CDF, the log
  // marginal likelihood increment and the resampling are those of particle
  // learning with sigma^2 + tau^2 replaced by sigma^2.
  // pin: the Kalman filter (tests/test_oracle_pl.py).
  int step_bootstrap(double y) {
    const R yr = (R)y;
    std::vector<R> ell(n);
    for (uint64_t i = 0; i < n; ++i) {
      W4 w = draw(cfg.seed, cfg.filter_id, t, (uint32_t)i, P_BOOT_STATE, 0);
      R Z = bm_normal<R>(w);
      R sv = std::sqrt(t2[i]);
      R xz = sv * Z;
      x[i] = x[i] + xz;
      ell[i] = log_pred<R>(x[i], s2[i], (R)0, yr);
    }
    R m = ell[0];
    for (uint64_t i = 1; i < n; ++i)
      if (ell[i] > m) m = ell[i];
    if (!std::isfinite((double)m)) return 4;
    std::vector<uint64_t> W(n);
    typename ExpSum<R>::T S;
    for (uint64_t i = 0; i < n; ++i) {
      R e;
      R dl = ell[i] - m;
      W[i] = quant_exp<R>(dl, k, &e);
      S.add(e);
    }
    cdf_scan(W.data(), n, Q.data());
    logml += (double)m + std::log(S.value()) - std::log((double)n) - 0.5 * LOG_2PI;
    resample(Q.data(), n, cfg.scheme, cfg.seed, cfg.filter_id, t, anc.data());
    std::vector<R> xn(n), s2n(n), t2n(n);
    std::vector<B> bsn(n), btn(n);
    for (uint64_t j = 0; j < n; ++j) {
      const uint32_t a = anc[j];
      xn[j] = x[a]; s2n[j] = s2[a]; t2n[j] = t2[a]; bsn[j] = bs[a]; btn[j] = bt[a];
    }
    x.swap(xn); s2.swap(s2n); t2.swap(t2n); bs.swap(bsn); bt.swap(btn);
    ++t;
    return 0;
  }

  // y - x_{t+1}: in binary32 from the rounded observation, in binary64 from y.
  static R resid_obs(double y, R yr, R xj);

  Estimates estimate() const override {
    Estimates E;
    E.t = (double)t;
    if (ess) {
      // weights e^{lambda_i}, by the deterministic exp of the CDF
      std::vector<double> w(n);
      for (uint64_t i = 0; i < n; ++i) {
        R e;
        (void)quant_exp<R>(lam[i], k, &e);
        w[i] = (double)e;
      }
      wmoments(x, w, &E.x_mean, &E.x_var);
      wmoments(s2, w, &E.sigma2_mean, &E.sigma2_var);
      wmoments(t2, w, &E.tau2_mean, &E.tau2_var);
    } else {
      moments(x, &E.x_mean, &E.x_var);
      moments(s2, &E.sigma2_mean, &E.sigma2_var);
      moments(t2, &E.tau2_mean, &E.tau2_var);
    }
    E.log_marglik = logml;
    return E;
  }

  void state_as_double(double* xo, double* s2o, double* t2o, double* bso,
                       double* bto) const override {
    for (uint64_t i = 0; i < n; ++i) {
      xo[i] = x[i]; s2o[i] = s2[i]; t2o[i] = t2[i];
      bso[i] = Suff<R>::as_double(bs[i]); bto[i] = Suff<R>::as_double(bt[i]);
    }
  }
  void state_raw(void* xo, void* s2o, void* t2o, void* bso, void* bto) const override {
    R* xr = (R*)xo; R* sr = (R*)s2o; R* tr = (R*)t2o; B* br = (B*)bso; B* cr = (B*)bto;
    for (uint64_t i = 0; i < n; ++i) {
      xr[i] = x[i]; sr[i] = s2[i]; tr[i] = t2[i]; br[i] = bs[i]; cr[i] = bt[i];
    }
  }
  const std::vector<uint32_t>& last_ancestors() const override { return anc; }
  const std::vector<uint64_t>& last_cdf() const override { return Q; }
  bool last_resampled() const override { return resampled; }

 private:
  // Weighted mean and variance, two-pass, in binary64.
  static void wmoments(const std::vector<R>& v, const std::vector<double>& w, double* mean,
                       double* var) {
    double sw = 0.0, s = 0.0;
    for (size_t i = 0; i < v.size(); ++i) {
      sw += w[i];
      s += w[i] * (double)v[i];
    }
    double mu = s / sw;
    double q = 0.0;
    for (size_t i = 0; i < v.size(); ++i) {
      double d = (double)v[i] - mu;
      q += w[i] * (d * d);
    }
    *mean = mu;
    *var = q / sw;
  }

  // Population mean and variance, two-pass, in binary64.
  static void moments(const std::vector<R>& v, double* mean, double* var) {
    double s = 0.0;
    for (R a : v) s += (double)a;
    double mu = s / (double)v.size();
    double q = 0.0;
    for (R a : v) {
      double d = (double)a - mu;
      q += d * d;
    }
    *mean = mu;
    *var = q / (double)v.size();
  }

  Config cfg;
  uint64_t n;
  uint32_t t;
  int k;
  double logml;
  int fail = 0;
  bool ess = false;        // adaptive resampling
  bool resampled = true;   // the last cycle resampled
  double slam;             // sum_i e^{lambda_i} of the carried log-weights
  std::vector<R> lam;      // carried log-weights (adaptive resampling)
  std::vector<R> x, s2, t2;
  std::vector<B> bs, bt;
  std::vector<uint32_t> anc;
  std::vector<uint64_t> Q;
};

template <> float Filter<float>::resid_obs(double, float yr, float xj) { return yr - xj; }
template <> double Filter<double>::resid_obs(double y, double, double xj) { return y - xj; }

FilterBase* make_filter(const Config& cfg) {
  if (cfg.precision == 0) return new Filter<float>(cfg);
  return new Filter<double>(cfg);
}

// Known-state learning: apply Steps 3-4 of the cycle to a given state path
// x_0..x_T and observations y_1..y_T for every particle (identity ancestors).
template <class R>
int suffstat_known_states(const Config& cfg, const double* xpath, const double* y, uint32_t T,
                          double* bs_out, double* bt_out, double* s2_out, double* t2_out) {
  typedef typename Suff<R>::B B;
  int fail = 0;
  for (uint64_t j = 0; j < cfg.n; ++j) {
    B bs = Suff<R>::from_prior(cfg.b_sigma), bt = Suff<R>::from_prior(cfg.b_tau);
    R s2v = 0, t2v = 0;
    for (uint32_t t = 0; t < T; ++t) {
      R xa = (R)xpath[t], xj = (R)xpath[t + 1];
      R rs = Filter<R>::resid_obs(y[t], (R)y[t], xj);
      R rt = xj - xa;
      bs = Suff<R>::add_half_square(bs, rs, &fail);
      bt = Suff<R>::add_half_square(bt, rt, &fail);
      double ds, cs, ks, dt, ct, kt;
      mt_constants(cfg.a_sigma + 0.5 * (double)(t + 1), &ds, &cs, &ks);
      mt_constants(cfg.a_tau + 0.5 * (double)(t + 1), &dt, &ct, &kt);
      R Zx, Zs, Us, Zt, Ut;
      theta_draws<R>(cfg.seed, cfg.filter_id, t, (uint32_t)j, &Zx, &Zs, &Us, &Zt, &Ut);
      R Gs = gamma_mt_from<R>((R)ds, (R)cs, (R)ks, Zs, Us, cfg.seed, cfg.filter_id, t,
                              (uint32_t)j, P_GAMMA_SIGMA, &fail);
      R Gt = gamma_mt_from<R>((R)dt, (R)ct, (R)kt, Zt, Ut, cfg.seed, cfg.filter_id, t,
                              (uint32_t)j, P_GAMMA_TAU, &fail);
      s2v = Suff<R>::ig(bs, Gs);
      t2v = Suff<R>::ig(bt, Gt);
    }
    bs_out[j] = Suff<R>::as_double(bs);
    bt_out[j] = Suff<R>::as_double(bt);
    s2_out[j] = s2v;
    t2_out[j] = t2v;
  }
  return fail ? 4 : 0;
}
template int suffstat_known_states<float>(const Config&, const double*, const double*, uint32_t,
                                          double*, double*, double*, double*);
template int suffstat_known_states<double>(const Config&, const double*, const double*,
                                           uint32_t, double*, double*, double*, double*);

// Kalman filter (closed form of the prediction / filtering equations of the
// paper's Section 2 for the linear Gaussian local-level model).
void kalman(const double* y, uint32_t T, double m0, double P0, double sigma2, double tau2,
            double* mean, double* var, double* loglik) {
  double m = m0, P = P0, ll = 0.0;
  for (uint32_t t = 0; t < T; ++t) {
    double Pp = P + tau2;
    double F = Pp + sigma2;
    double v = y[t] - m;
    double K = Pp / F;
    m = m + K * v;
    P = Pp - K * Pp;
    ll += -0.5 * (std::log(F) + LOG_2PI + v * v / F);
    mean[t] = m;
    var[t] = P;
  }
  *loglik = ll;
}

}  // namespace oracle
