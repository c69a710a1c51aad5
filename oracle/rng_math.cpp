// CPU oracle, part 1: counter-based RNG, deterministic elementary functions,
// normal and gamma draws.  TEST INFRASTRUCTURE ONLY (see oracle.h).
#include <cmath>
#include <cstring>

#include "oracle.h"

namespace oracle {

// ---------------------------------------------------------------------------
// Philox (Salmon et al. 2011).  One round maps counter (c0, c1, c2, c3) with
// round key (k0, k1) to
//   (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0));
// between rounds the key is bumped by the Weyl constants (W0, W1).
// ---------------------------------------------------------------------------
W4 philox4x32_10(const uint32_t ctr[4], const uint32_t key[2]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)M0 * c0;
    uint64_t p1 = (uint64_t)M1 * c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += W0;
    k1 += W1;
  }
  W4 out = {{c0, c1, c2, c3}};
  return out;
}

void philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
  uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    u128 p0 = (u128)M0 * c0;
    u128 p1 = (u128)M1 * c2;
    uint64_t n0 = (uint64_t)(p1 >> 64) ^ c1 ^ k0;
    uint64_t n1 = (uint64_t)p1;
    uint64_t n2 = (uint64_t)(p0 >> 64) ^ c3 ^ k1;
    uint64_t n3 = (uint64_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += W0;
    k1 += W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

W4 draw(uint64_t seed, uint32_t filter, uint32_t t, uint32_t j, uint32_t purpose,
        uint32_t attempt) {
  uint32_t ctr[4] = {j, t, filter, purpose | (attempt << 8)};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  return philox4x32_10(ctr, key);
}

float unif_f32(uint32_t w) {
  // 2*(w>>9)+1 < 2^24 is exact in binary32; the scaling is exact.
  return (float)(2u * (w >> 9) + 1u) * 0x1p-24f;
}
double unif_f64(uint32_t lo, uint32_t hi) {
  uint64_t R = ((uint64_t)hi << 32) | lo;
  return (double)(2ull * (R >> 12) + 1ull) * 0x1p-53;
}
double unif_f64_32(uint32_t w) { return (double)(2ull * w + 1ull) * 0x1p-33; }

// ---------------------------------------------------------------------------
// Deterministic elementary functions.
//
// log, binary64: x = f * 2^e with f in [sqrt(1/2), sqrt(2)); log f = 2 atanh(z),
//   z = (f - 1)/(f + 1), by the odd series 2z (1 + z^2/3 + z^4/5 + ...)
//   (terms through z^20/21); log x = e * ln2 + log f.
// log, binary32 (no division): the same reduction, u = f - 1 (exact), and
//   log(1 + u) = u + u^2 q(u) with q a degree-8 polynomial fitted for minimal
//   maximum relative error of log(1 + u) on [sqrt(1/2) - 1, sqrt(2) - 1]
//   (Lawson's iteratively reweighted least squares, coefficients rounded to
//   binary32); log x = e ln2_hi + (e ln2_lo + log f) by two fused
//   multiply-adds.  Error at most 0.93 ulp over every positive normal
//   binary32 (checked exhaustively against long double log).
// exp: Taylor polynomial sum_{k<=D} r^k/k! (D = 7 / 13) on the reduced
//   argument of a Cody & Waite (1980) reduction r = (x - n ln2_hi) - n ln2_lo.
// cos(2 pi u): reduce u to w = |u - rint(u)| in [0, 1/2]; by octant use
//   cos(2 pi w), sin(2 pi (1/4 - w)) or -cos(2 pi (1/2 - w)), each a Taylor
//   polynomial on |x| <= pi/4 (cos through x^10 / x^16, sin through x^9 / x^17).
// All constants are the exact values rounded to nearest in the working format.
// ---------------------------------------------------------------------------
template <class R> struct K;
template <> struct K<float> {
  static constexpr float LN2 = 0x1.62e430p-1f;
  static constexpr float LN2_HI = 0x1.62e400p-1f;  // ln2 truncated to 16 bits
  static constexpr float LN2_LO = 0x1.7f7d1cp-20f; // ln2 - LN2_HI
  static constexpr float INV_LN2 = 0x1.715476p+0f;
  static constexpr float TWO_PI = 0x1.921fb6p+2f;
  static constexpr float SQRT_HALF = 0x1.6a09e6p-1f;
  static constexpr int LOG_K = 4;
  static constexpr int EXP_D = 7;
  static constexpr int COS_K = 5;
  static constexpr int SIN_K = 4;
};
template <> struct K<double> {
  static constexpr double LN2 = 0x1.62e42fefa39efp-1;
  static constexpr double LN2_HI = 0x1.62e42fefa2000p-1;  // ln2 truncated to 40 bits
  static constexpr double LN2_LO = 0x1.9ef35793c7673p-41;
  static constexpr double INV_LN2 = 0x1.71547652b82fep+0;
  static constexpr double TWO_PI = 0x1.921fb54442d18p+2;
  static constexpr double SQRT_HALF = 0x1.6a09e667f3bcdp-1;
  static constexpr int LOG_K = 10;
  static constexpr int EXP_D = 13;
  static constexpr int COS_K = 8;
  static constexpr int SIN_K = 8;
};

// 1/k! rounded to nearest, k = 0..17.
static const float INV_FACT_F[18] = {
    0x1p+0f, 0x1p+0f, 0x1p-1f, 0x1.555556p-3f, 0x1.555556p-5f, 0x1.111112p-7f,
    0x1.6c16c2p-10f, 0x1.a01a02p-13f, 0x1.a01a02p-16f, 0x1.71de3ap-19f, 0x1.27e4fcp-22f,
    0x1.ae6456p-26f, 0x1.1eed8ep-29f, 0x1.612462p-33f, 0x1.93974ap-37f, 0x1.ae7f3ep-41f,
    0x1.ae7f3ep-45f, 0x1.952c78p-49f};
static const double INV_FACT_D[18] = {
    0x1p+0, 0x1p+0, 0x1p-1, 0x1.5555555555555p-3, 0x1.5555555555555p-5,
    0x1.1111111111111p-7, 0x1.6c16c16c16c17p-10, 0x1.a01a01a01a01ap-13,
    0x1.a01a01a01a01ap-16, 0x1.71de3a556c734p-19, 0x1.27e4fb7789f5cp-22,
    0x1.ae64567f544e4p-26, 0x1.1eed8eff8d898p-29, 0x1.6124613a86d09p-33,
    0x1.93974a8c07c9dp-37, 0x1.ae7f3e733b81fp-41, 0x1.ae7f3e733b81fp-45,
    0x1.952c77030ad4ap-49};
// 1/(2m+1) rounded to nearest, m = 0..10.
static const float INV_ODD_F[11] = {
    0x1p+0f, 0x1.555556p-2f, 0x1.99999ap-3f, 0x1.24924ap-3f, 0x1.c71c72p-4f, 0x1.745d18p-4f,
    0x1.3b13b2p-4f, 0x1.111112p-4f, 0x1.e1e1e2p-5f, 0x1.af286cp-5f, 0x1.861862p-5f};
static const double INV_ODD_D[11] = {
    0x1p+0, 0x1.5555555555555p-2, 0x1.999999999999ap-3, 0x1.2492492492492p-3,
    0x1.c71c71c71c71cp-4, 0x1.745d1745d1746p-4, 0x1.3b13b13b13b14p-4,
    0x1.1111111111111p-4, 0x1.e1e1e1e1e1e1ep-5, 0x1.af286bca1af28p-5,
    0x1.8618618618618p-5};

template <class R> static inline R inv_fact(int k);
template <> inline float inv_fact<float>(int k) { return INV_FACT_F[k]; }
template <> inline double inv_fact<double>(int k) { return INV_FACT_D[k]; }
template <class R> static inline R inv_odd(int m);
template <> inline float inv_odd<float>(int m) { return INV_ODD_F[m]; }
template <> inline double inv_odd<double>(int m) { return INV_ODD_D[m]; }

template <class R> R det_log(R x) {
  int e;
  R f = std::frexp(x, &e);  // x = f * 2^e, f in [0.5, 1)
  if (f < K<R>::SQRT_HALF) {
    f = f * (R)2;
    e = e - 1;
  }
  R num = f - (R)1;  // exact (Sterbenz)
  R den = f + (R)1;
  R z = num / den;
  R z2 = z * z;
  R p = inv_odd<R>(K<R>::LOG_K);
  for (int m = K<R>::LOG_K - 1; m >= 0; --m) p = std::fma(p, z2, inv_odd<R>(m));
  R two_z = z * (R)2;
  R logf = two_z * p;
  R elog2 = (R)e * K<R>::LN2;
  return elog2 + logf;
}

// q(u) of the binary32 log, c_0 .. c_8 (coefficient of u^j).
static const float LOGQ_F[9] = {-0x1.fffff8p-2f, 0x1.55555p-2f,   -0x1.000426p-2f,
                                0x1.99a3f6p-3f,  -0x1.542766p-3f, 0x1.22715ep-3f,
                                -0x1.0f3756p-3f, 0x1.0849bep-3f,  -0x1.38339ap-4f};

// x > 0 (normal or subnormal); +inf and NaN are returned unchanged.
template <> float det_log<float>(float x) {
  if (!(x < INFINITY)) return x;
  uint32_t b;
  std::memcpy(&b, &x, 4);
  int e = 0;
  if ((b & 0x7f800000u) == 0) {  // subnormal: scale by 2^23 (exact)
    const float xs = x * 0x1p23f;
    std::memcpy(&b, &xs, 4);
    e = -23;
  }
  e += (int)(b >> 23) - 127;
  uint32_t m = (b & 0x7fffffu) | 0x3f800000u;  // f = x 2^-e in [1, 2)
  if (m >= 0x3fb504f3u) {                       // f >= sqrt(2) rounded: halve it
    m -= 0x00800000u;
    e += 1;
  }
  float f;
  std::memcpy(&f, &m, 4);
  const float u = f - 1.0f;  // exact (Sterbenz)
  float q = LOGQ_F[8];
  for (int j = 7; j >= 0; --j) q = std::fma(q, u, LOGQ_F[j]);
  const float u2 = u * u;
  const float lf = std::fma(u2, q, u);
  const float ef = (float)e;  // exact
  const float lo = std::fma(ef, K<float>::LN2_LO, lf);
  return std::fma(ef, K<float>::LN2_HI, lo);
}

template <class R> R det_exp_core(R r) {
  R p = inv_fact<R>(K<R>::EXP_D);
  for (int k = K<R>::EXP_D - 1; k >= 0; --k) p = std::fma(p, r, inv_fact<R>(k));
  return p;
}

template <class R> static inline R cos_poly(R x) {
  R x2 = x * x;
  int kk = K<R>::COS_K;
  R p = (kk & 1) ? -inv_fact<R>(2 * kk) : inv_fact<R>(2 * kk);
  for (int m = kk - 1; m >= 0; --m) {
    R c = (m & 1) ? -inv_fact<R>(2 * m) : inv_fact<R>(2 * m);
    p = std::fma(p, x2, c);
  }
  return p;
}
template <class R> static inline R sin_poly(R x) {
  R x2 = x * x;
  int kk = K<R>::SIN_K;
  R p = (kk & 1) ? -inv_fact<R>(2 * kk + 1) : inv_fact<R>(2 * kk + 1);
  for (int m = kk - 1; m >= 0; --m) {
    R c = (m & 1) ? -inv_fact<R>(2 * m + 1) : inv_fact<R>(2 * m + 1);
    p = std::fma(p, x2, c);
  }
  return x * p;
}

template <class R> R det_cos2pi(R u) {
  R v = u - std::rint(u);
  R w = std::fabs(v);  // in [0, 1/2]
  if (w <= (R)0.125) {
    R x = K<R>::TWO_PI * w;
    return cos_poly(x);
  } else if (w <= (R)0.375) {
    R a = (R)0.25 - w;  // exact
    R x = K<R>::TWO_PI * a;
    return sin_poly(x);
  } else {
    R a = (R)0.5 - w;  // exact
    R x = K<R>::TWO_PI * a;
    return -cos_poly(x);
  }
}

// sin(2 pi u) and cos(2 pi u) together, same reduction as det_cos2pi:
// with w = |u - rint(u)|, the octant picks the argument x = 2 pi a and which
// of the two polynomials gives each value; sin takes the sign of u - rint(u).
template <class R> void det_sincos2pi(R u, R* s, R* c) {
  R v = u - std::rint(u);
  R w = std::fabs(v);
  R sv, cv;
  if (w <= (R)0.125) {
    R x = K<R>::TWO_PI * w;
    sv = sin_poly(x);
    cv = cos_poly(x);
  } else if (w <= (R)0.375) {
    R a = (R)0.25 - w;
    R x = K<R>::TWO_PI * a;
    sv = cos_poly(x);
    cv = sin_poly(x);
  } else {
    R a = (R)0.5 - w;
    R x = K<R>::TWO_PI * a;
    sv = sin_poly(x);
    cv = -cos_poly(x);
  }
  *s = v < (R)0 ? -sv : sv;
  *c = cv;
}

template <class R> static inline R pow2(int n) { return std::ldexp((R)1, n); }

template <class R> uint64_t quant_exp(R dl, int k, R* e) {
  const R CUTOFF = (R)-50;
  if (!(dl >= CUTOFF)) {
    *e = (R)0;
    return 0;
  }
  R t = dl * K<R>::INV_LN2;
  R nr = std::rint(t);
  int n = (int)nr;
  R a = nr * K<R>::LN2_HI;
  R b = dl - a;
  R c = nr * K<R>::LN2_LO;
  R r = b - c;
  R p = det_exp_core(r);
  *e = p * pow2<R>(n);
  int sc = n + k;
  uint64_t W = 0;
  if (sc >= 0) {
    R v = p * pow2<R>(sc);
    W = (uint64_t)v;  // truncation; v < 2^62
  }
  uint64_t cap = 1ull << k;
  return W > cap ? cap : W;
}

template <class R> R bm_normal(const W4& w);
template <> float bm_normal<float>(const W4& w) {
  float u1 = unif_f32(w.w[0]);
  float u2 = unif_f32(w.w[1]);
  float L = det_log(u1);
  float m2 = L * -2.0f;
  float r = std::sqrt(m2);
  float c = det_cos2pi(u2);
  return r * c;
}
template <> double bm_normal<double>(const W4& w) {
  double u1 = unif_f64(w.w[0], w.w[1]);
  double u2 = unif_f64_32(w.w[2]);
  double L = det_log(u1);
  double m2 = L * -2.0;
  double r = std::sqrt(m2);
  double c = det_cos2pi(u2);
  return r * c;
}
template <> void bm_normal2<float>(const W4& w, float* zc, float* zs) {
  float u1 = unif_f32(w.w[0]);
  float u2 = unif_f32(w.w[1]);
  float L = det_log(u1);
  float m2 = L * -2.0f;
  float r = std::sqrt(m2);
  float sn, cs;
  det_sincos2pi(u2, &sn, &cs);
  *zc = r * cs;
  *zs = r * sn;
}
template <> void bm_normal2<double>(const W4& w, double* zc, double* zs) {
  double u1 = unif_f64(w.w[0], w.w[1]);
  double u2 = unif_f64_32(w.w[2]);
  double L = det_log(u1);
  double m2 = L * -2.0;
  double r = std::sqrt(m2);
  double sn, cs;
  det_sincos2pi(u2, &sn, &cs);
  *zc = r * cs;
  *zs = r * sn;
}
template <> float extra_uniform<float>(const W4& w) { return unif_f32(w.w[2]); }
template <> double extra_uniform<double>(const W4& w) { return unif_f64_32(w.w[3]); }

void mt_constants(double a, double* d, double* c, double* K) {
  const double ONE_THIRD = 0x1.5555555555555p-2;
  // 0.0331 * 2/3 = 331/15000 rounded to nearest: the squeeze coefficient
  // K = 0.0331 (2/3) / d equals Marsaglia & Tsang's 0.0331 at d = 2/3 (a = 1)
  const double SQZ = 0x1.698a4eea9073cp-6;
  double dd = a - ONE_THIRD;
  double nine_d = 9.0 * dd;
  double s = std::sqrt(nine_d);
  *d = dd;
  *c = 1.0 / s;
  *K = SQZ / dd;
}

// Marsaglia & Tsang (2000): with v = (1 + c Z)^3, accept d v when v > 0 and
// log U < Z^2/2 + d (1 - v + log v).  The squeeze U < 1 - K Z^4 accepts
// without logarithms; it is valid (implies the full test) because
// 1 - e^{g(Z)} <= K Z^4 for every Z (g the right-hand side above): the
// supremum of (1 - e^g) d / Z^4 over Z is 0.02205 at d = 2/3 and falls as d
// grows (to 1/108), so K = 0.0331 (2/3) / d bounds it for all d >= 2/3.  A
// draw the squeeze misses takes the full test, so the accepted draws, and
// the sampler's law, are exactly Marsaglia-Tsang's; the d-scaled squeeze only
// takes the logarithms far less often (pin: tests/test_oracle_rng.py).
template <class R> R gamma_mt_from(R d, R c, R K, R Z0, R U0, uint64_t seed, uint32_t filter,
                                   uint32_t t, uint32_t j, uint32_t purpose, int* fail) {
  for (uint32_t attempt = 0; attempt < 16; ++attempt) {
    R Z = Z0, U = U0;
    if (attempt > 0) {
      W4 w = draw(seed, filter, t, j, purpose, attempt);
      Z = bm_normal<R>(w);
      U = extra_uniform<R>(w);
    }
    R v = std::fma(c, Z, (R)1);
    if (!(v > (R)0)) continue;
    R vv = v * v;
    R v3 = vv * v;
    R Z2 = Z * Z;
    R z4 = Z2 * Z2;
    R thr = std::fma(-K, z4, (R)1);
    if (U < thr) return d * v3;
    R lhs = det_log(U);
    R a1 = (R)1 - v3;
    R a2 = det_log(v3);
    R a3 = a1 + a2;
    R a5 = (R)0.5 * Z2;
    R rhs = std::fma(d, a3, a5);
    if (lhs < rhs) return d * v3;
  }
  *fail = 1;
  return d;
}

template <class R> R gamma_mt(R d, R c, R K, uint64_t seed, uint32_t filter, uint32_t t,
                              uint32_t j, uint32_t purpose, int* fail) {
  W4 w = draw(seed, filter, t, j, purpose, 0);
  return gamma_mt_from<R>(d, c, K, bm_normal<R>(w), extra_uniform<R>(w), seed, filter, t, j,
                          purpose, fail);
}

// The draws of one propagation step for slot j (Algorithm "Particle
// Learning", Steps 2 and 4): the state normal Zx, and the first normal and
// uniform of the sigma^2 and tau^2 gamma draws.  Draw A = (j, t, STATE, 0):
// its Box-Muller pair gives Zx (cos) and Zs (sin), its word 2 gives Us.
// binary32: slots 2i and 2i + 1 share draw B = (i, t, STATE, 1): the two
// outputs of its Box-Muller pair are their tau^2 normals (cos to the even
// slot, sin to the odd one) and its words 2 and 3 their uniforms -- three
// 128-bit draws and three Box-Muller transforms per two slots.  binary64
// (whose Box-Muller takes three words and whose uniform takes the fourth):
// B = (j, t, STATE, 1) per slot, its first output and its uniform.
template <class R> void theta_draws(uint64_t seed, uint32_t filter, uint32_t t, uint32_t j,
                                    R* Zx, R* Zs, R* Us, R* Zt, R* Ut) {
  W4 A = draw(seed, filter, t, j, P_STATE, 0);
  bm_normal2<R>(A, Zx, Zs);
  *Us = extra_uniform<R>(A);
  if (sizeof(R) == 4) {
    W4 B = draw(seed, filter, t, j >> 1, P_STATE, 1);
    R zc, zs;
    bm_normal2<R>(B, &zc, &zs);
    *Zt = (j & 1) ? zs : zc;
    *Ut = (R)unif_f32((j & 1) ? B.w[3] : B.w[2]);
  } else {
    W4 B = draw(seed, filter, t, j, P_STATE, 1);
    *Zt = bm_normal<R>(B);
    *Ut = extra_uniform<R>(B);
  }
}

template double det_log<double>(double);
template float det_exp_core<float>(float);
template double det_exp_core<double>(double);
template float det_cos2pi<float>(float);
template double det_cos2pi<double>(double);
template uint64_t quant_exp<float>(float, int, float*);
template uint64_t quant_exp<double>(double, int, double*);
template float gamma_mt<float>(float, float, float, uint64_t, uint32_t, uint32_t, uint32_t,
                               uint32_t, int*);
template double gamma_mt<double>(double, double, double, uint64_t, uint32_t, uint32_t, uint32_t,
                                 uint32_t, int*);
template float gamma_mt_from<float>(float, float, float, float, float, uint64_t, uint32_t,
                                    uint32_t, uint32_t, uint32_t, int*);
template double gamma_mt_from<double>(double, double, double, double, double, uint64_t,
                                      uint32_t, uint32_t, uint32_t, uint32_t, int*);
template void det_sincos2pi<float>(float, float*, float*);
template void det_sincos2pi<double>(double, double*, double*);
template void theta_draws<float>(uint64_t, uint32_t, uint32_t, uint32_t, float*, float*, float*,
                                 float*, float*);
template void theta_draws<double>(uint64_t, uint32_t, uint32_t, uint32_t, double*, double*,
                                  double*, double*, double*);

}  // namespace oracle
