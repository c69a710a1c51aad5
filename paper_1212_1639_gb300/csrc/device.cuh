// Device building blocks of the particle-learning cycle (sm_103a).
//
// This translation-unit-shared header holds the per-element arithmetic that
// every kernel uses: the counter-based RNG, exactly representable uniforms,
// deterministic elementary functions, Box-Muller normals, the Marsaglia-Tsang
// gamma sampler and 128-bit integer helpers.
//
// Determinism contract.  The library is compiled with -fmad=false, IEEE
// division and square root, and no flush-to-zero, and every floating-point
// expression below is written as one IEEE operation per statement: a
// separately rounded add, multiply, divide or square root, or an explicit
// fused multiply-add (__fmaf_rn / __fma_rn / fma.rn.f32x2) where the
// definition fuses.  Given the
// same inputs the results are therefore bit-identical on any IEEE-754
// machine that evaluates the same operation sequence, which is what makes the
// quantised CDF (and hence every ancestor index) a deterministic function of
// the particle state.
#pragma once
#include <cstdint>

namespace pfk {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC'11): ten rounds of the Philox S-box on a 128-bit
// counter with a 64-bit key bumped by the golden-ratio Weyl constants.
// ---------------------------------------------------------------------------
struct U4 {
  uint32_t a, b, c, d;
};

__device__ __forceinline__ U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                     uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    // one 32 x 32 -> 64-bit product each: its halves are the S-box outputs
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return U4{c0, c1, c2, c3};
}

// Philox4x32-10 with its ten round keys given (they depend only on the
// 64-bit key, so a kernel can take them precomputed as parameters instead of
// bumping the key twice per round in every draw): rk[2r], rk[2r+1] are the
// key words of round r.
__device__ __forceinline__ U4 philox_rk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        const uint32_t* rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c0 = hi1 ^ c1 ^ rk[2 * r];
    c1 = lo1;
    c2 = hi0 ^ c3 ^ rk[2 * r + 1];
    c3 = lo0;
  }
  return U4{c0, c1, c2, c3};
}

enum Purpose : uint32_t {
  P_INIT_X = 1, P_INIT_SIGMA = 2, P_INIT_TAU = 3,
  P_STATE = 4, P_GAMMA_SIGMA = 5, P_GAMMA_TAU = 6,
  P_SYS_OFFSET = 7, P_SPACING = 8, P_STRATIFIED = 9, P_BOOT_STATE = 10,
};

// Draw (seed, filter, t, j, purpose, attempt): counter (j, t, filter,
// purpose | attempt << 8), key (seed lo, seed hi).
__device__ __forceinline__ U4 draw(uint64_t seed, uint32_t filter, uint32_t t, uint32_t j,
                                   uint32_t purpose, uint32_t attempt) {
  return philox(j, t, filter, purpose | (attempt << 8), (uint32_t)seed, (uint32_t)(seed >> 32));
}

// Uniforms on (0,1) whose conversion is exact: (2 (w >> 9) + 1) 2^-24.
// m = w >> 9 < 2^23 is converted exactly by the 2^23 bias trick.
__device__ __forceinline__ float unif_f32(uint32_t w) {
  const float fm = __uint_as_float(0x4B000000u | (w >> 9)) - 8388608.0f;  // = m exactly
  const float a = fm * 0x1p-23f;
  return a + 0x1p-24f;  // exact: 24 significant bits
}
__device__ __forceinline__ double unif_f64(uint32_t lo, uint32_t hi) {
  const uint64_t R = ((uint64_t)hi << 32) | lo;
  return __ull2double_rn(2ull * (R >> 12) + 1ull) * 0x1p-53;
}
__device__ __forceinline__ double unif_f64_32(uint32_t w) {
  return __ull2double_rn(2ull * w + 1ull) * 0x1p-33;
}

// ---------------------------------------------------------------------------
// Deterministic elementary functions.
//  log x : x = f 2^e, f in [sqrt(1/2), sqrt(2)).
//          binary64: log f = 2 atanh(z), z = (f-1)/(f+1), series through
//          z^20/21; log x = e ln2 + log f.
//          binary32 (no division): u = f - 1 (exact), log f = u + u^2 q(u)
//          with q of degree 8, coefficients fitted for the least maximum
//          relative error of log(1 + u) on [sqrt(1/2) - 1, sqrt(2) - 1] and
//          rounded to binary32 (at most 0.93 ulp over all binary32);
//          log x = e ln2_hi + (e ln2_lo + log f), two fused multiply-adds.
//  exp r : Taylor polynomial through r^D/D! (D = 7 / 13) on a Cody-Waite
//          reduced argument.
//  cos(2 pi u): octant reduction of u in [0,1] and Taylor polynomials of cos
//          (through x^10 / x^16) and sin (through x^9 / x^17) on |x| <= pi/4.
// Constants are the exact values rounded to nearest in the working format.
// ---------------------------------------------------------------------------
template <class R> struct Cst;
template <> struct Cst<float> {
  static constexpr float LN2 = 0x1.62e430p-1f;
  static constexpr float LN2_HI = 0x1.62e400p-1f;
  static constexpr float LN2_LO = 0x1.7f7d1cp-20f;
  static constexpr float INV_LN2 = 0x1.715476p+0f;
  static constexpr float TWO_PI = 0x1.921fb6p+2f;
  static constexpr float SQRT_HALF = 0x1.6a09e6p-1f;
};
template <> struct Cst<double> {
  static constexpr double LN2 = 0x1.62e42fefa39efp-1;
  static constexpr double LN2_HI = 0x1.62e42fefa2000p-1;
  static constexpr double LN2_LO = 0x1.9ef35793c7673p-41;
  static constexpr double INV_LN2 = 0x1.71547652b82fep+0;
  static constexpr double TWO_PI = 0x1.921fb54442d18p+2;
  static constexpr double SQRT_HALF = 0x1.6a09e667f3bcdp-1;
};

// Exact small-integer to binary32 conversion (|e| < 2^22) by the 1.5 * 2^23 bias.
__device__ __forceinline__ float small_int_to_f32(int e) {
  return __int_as_float(0x4B400000 + e) - 12582912.0f;
}

// q(u) of the binary32 log: coefficients of u^0 .. u^8
__device__ __forceinline__ float logq_f(int j) {
  constexpr float C[9] = {-0x1.fffff8p-2f, 0x1.55555p-2f,   -0x1.000426p-2f,
                          0x1.99a3f6p-3f,  -0x1.542766p-3f, 0x1.22715ep-3f,
                          -0x1.0f3756p-3f, 0x1.0849bep-3f,  -0x1.38339ap-4f};
  return C[j];
}
// reduction of the binary32 log: x = f 2^e with f = as_float(m) in
// [sqrt(1/2), sqrt(2)) (subnormals scaled by 2^23 first)
__device__ __forceinline__ uint32_t log_reduce(float x, int* e_out) {
  uint32_t b = __float_as_uint(x);
  int e = 0;
  if ((b & 0x7f800000u) == 0) {  // subnormal (or zero): scale by 2^23, exact
    b = __float_as_uint(__fmul_rn(x, 0x1p23f));
    e = -23;
  }
  e += (int)(b >> 23) - 127;
  uint32_t m = (b & 0x7fffffu) | 0x3f800000u;  // [1, 2)
  if (m >= 0x3fb504f3u) {                       // at or above sqrt(2) rounded: halve
    m -= 0x00800000u;
    e += 1;
  }
  *e_out = e;
  return m;
}

// log of x > 0 (normal or subnormal); +inf and NaN are returned unchanged.
__device__ __forceinline__ float det_log(float x) {
  int e;
  const uint32_t m = log_reduce(x, &e);
  const float u = __fsub_rn(__uint_as_float(m), 1.0f);  // exact
  float q = logq_f(8);
#pragma unroll
  for (int j = 7; j >= 0; --j) q = __fmaf_rn(q, u, logq_f(j));
  const float u2 = __fmul_rn(u, u);
  const float lf = __fmaf_rn(u2, q, u);
  const float ef = small_int_to_f32(e);
  const float lo = __fmaf_rn(ef, Cst<float>::LN2_LO, lf);
  const float r = __fmaf_rn(ef, Cst<float>::LN2_HI, lo);
  return x < INFINITY ? r : x;
}
__device__ __forceinline__ double det_log(double x) {
  int e;
  double f = frexp(x, &e);
  if (f < Cst<double>::SQRT_HALF) {
    f = f * 2.0;
    e = e - 1;
  }
  const double num = f - 1.0;
  const double den = f + 1.0;
  const double z = num / den;
  const double z2 = z * z;
  // 1/(2m+1), m = 10 .. 0
  const double c[11] = {0x1.8618618618618p-5, 0x1.af286bca1af28p-5, 0x1.e1e1e1e1e1e1ep-5,
                        0x1.1111111111111p-4, 0x1.3b13b13b13b14p-4, 0x1.745d1745d1746p-4,
                        0x1.c71c71c71c71cp-4, 0x1.2492492492492p-3, 0x1.999999999999ap-3,
                        0x1.5555555555555p-2, 0x1p+0};
  double p = c[0];
#pragma unroll
  for (int m = 1; m < 11; ++m) p = __fma_rn(p, z2, c[m]);
  const double two_z = z * 2.0;
  const double lf = two_z * p;
  const double el = (double)e * Cst<double>::LN2;
  return el + lf;
}

// Taylor polynomial of exp on the reduced argument.
__device__ __forceinline__ float det_exp_core(float r) {
  const float c[8] = {0x1.a01a02p-13f, 0x1.6c16c2p-10f, 0x1.111112p-7f, 0x1.555556p-5f,
                      0x1.555556p-3f, 0x1p-1f, 0x1p+0f, 0x1p+0f};  // 1/7! .. 1/0!
  float p = c[0];
#pragma unroll
  for (int k = 1; k < 8; ++k) p = __fmaf_rn(p, r, c[k]);
  return p;
}
__device__ __forceinline__ double det_exp_core(double r) {
  const double c[14] = {0x1.6124613a86d09p-33, 0x1.1eed8eff8d898p-29, 0x1.ae64567f544e4p-26,
                        0x1.27e4fb7789f5cp-22, 0x1.71de3a556c734p-19, 0x1.a01a01a01a01ap-16,
                        0x1.a01a01a01a01ap-13, 0x1.6c16c16c16c17p-10, 0x1.1111111111111p-7,
                        0x1.5555555555555p-5,  0x1.5555555555555p-3,  0x1p-1,
                        0x1p+0,                0x1p+0};  // 1/13! .. 1/0!
  double p = c[0];
#pragma unroll
  for (int k = 1; k < 14; ++k) p = __fma_rn(p, r, c[k]);
  return p;
}

__device__ __forceinline__ float cos_poly(float x) {
  const float x2 = x * x;
  // (-1)^m / (2m)!, m = 5 .. 0
  const float c[6] = {-0x1.27e4fcp-22f, 0x1.a01a02p-16f, -0x1.6c16c2p-10f, 0x1.555556p-5f,
                      -0x1p-1f, 0x1p+0f};
  float p = c[0];
#pragma unroll
  for (int m = 1; m < 6; ++m) p = __fmaf_rn(p, x2, c[m]);
  return p;
}
__device__ __forceinline__ float sin_poly(float x) {
  const float x2 = x * x;
  // (-1)^m / (2m+1)!, m = 4 .. 0
  const float c[5] = {0x1.71de3ap-19f, -0x1.a01a02p-13f, 0x1.111112p-7f, -0x1.555556p-3f,
                      0x1p+0f};
  float p = c[0];
#pragma unroll
  for (int m = 1; m < 5; ++m) p = __fmaf_rn(p, x2, c[m]);
  return x * p;
}
__device__ __forceinline__ double cos_poly(double x) {
  const double x2 = x * x;
  // (-1)^m / (2m)!, m = 8 .. 0
  const double c[9] = {0x1.ae7f3e733b81fp-45, -0x1.93974a8c07c9dp-37, 0x1.1eed8eff8d898p-29,
                       -0x1.27e4fb7789f5cp-22, 0x1.a01a01a01a01ap-16, -0x1.6c16c16c16c17p-10,
                       0x1.5555555555555p-5, -0x1p-1, 0x1p+0};
  double p = c[0];
#pragma unroll
  for (int m = 1; m < 9; ++m) p = __fma_rn(p, x2, c[m]);
  return p;
}
__device__ __forceinline__ double sin_poly(double x) {
  const double x2 = x * x;
  // (-1)^m / (2m+1)!, m = 8 .. 0
  const double c[9] = {0x1.952c77030ad4ap-49, -0x1.ae7f3e733b81fp-41, 0x1.6124613a86d09p-33,
                       -0x1.ae64567f544e4p-26, 0x1.71de3a556c734p-19, -0x1.a01a01a01a01ap-13,
                       0x1.1111111111111p-7, -0x1.5555555555555p-3, 0x1p+0};
  double p = c[0];
#pragma unroll
  for (int m = 1; m < 9; ++m) p = __fma_rn(p, x2, c[m]);
  return x * p;
}

// sin and cos of 2 pi u for u in [0, 1]: v = u - rint(u), w = |v|; the
// octant of w selects the reduced argument a (w, 1/4 - w or 1/2 - w, all
// exact) and which polynomial gives each value; sin takes the sign of v.
// Both polynomials are always evaluated, so the selection is branch-free.
template <class R>
__device__ __forceinline__ void det_sincos2pi(R u, R* s_out, R* c_out) {
  const R ru = u > (R)0.5 ? (R)1 : (R)0;  // rint(u) for u in [0, 1] (0.5 rounds to even 0)
  const R v = u - ru;
  const R w = fabs(v);
  const bool o1 = w <= (R)0.125;
  const bool o3 = w > (R)0.375;
  const R a = o1 ? w : (o3 ? (R)0.5 - w : (R)0.25 - w);
  const R x = Cst<R>::TWO_PI * a;
  const R S = sin_poly(x);
  const R C = cos_poly(x);
  const R sv = (o1 || o3) ? S : C;
  const R cv = o1 ? C : (o3 ? -C : S);
  *s_out = v < (R)0 ? -sv : sv;
  *c_out = cv;
}
template <class R>
__device__ __forceinline__ R det_cos2pi(R u) {
  R s, c;
  det_sincos2pi(u, &s, &c);
  return c;
}

__device__ __forceinline__ float pow2f(int n) {  // n in [-126, 127]
  return __int_as_float((n + 127) << 23);
}
__device__ __forceinline__ double pow2d(int n) {  // n in [-1022, 1023]
  return __longlong_as_double((long long)(n + 1023) << 52);
}
__device__ __forceinline__ float pow2(int n, float) { return pow2f(n); }
__device__ __forceinline__ double pow2(int n, double) { return pow2d(n); }

__device__ __forceinline__ uint64_t f2u64_rz(float v);
__device__ __forceinline__ uint64_t f2u64_rz(double v);

// Quantised CDF weight: e = exp(dl) (0 below dl = -50) and
// W = min(floor(e * 2^k), 2^k) for dl <= 0.
template <class R>
__device__ __forceinline__ uint64_t quant_exp(R dl, int k, R* e_out) {
  if (!(dl >= (R)-50)) {
    *e_out = (R)0;
    return 0;
  }
  const R t = dl * Cst<R>::INV_LN2;
  R nr;
  int n;
  if constexpr (sizeof(R) == 4) {
    // round to nearest even by the 1.5 * 2^23 bias (|t| < 2^22)
    const float biased = t + 12582912.0f;
    nr = biased - 12582912.0f;
    n = __float_as_int(biased) - 0x4B400000;
  } else {
    nr = rint(t);
    n = (int)nr;
  }
  const R a = nr * Cst<R>::LN2_HI;
  const R b = dl - a;
  const R c = nr * Cst<R>::LN2_LO;
  const R r = b - c;
  const R p = det_exp_core(r);
  *e_out = p * pow2(n, (R)0);
  const int sc = n + k;
  uint64_t W = 0;
  if constexpr (sizeof(R) == 4) {
    // floor(p * 2^sc) straight from p's bits: p = m24 2^(E - 23)
    const uint32_t pb = __float_as_uint(p);
    const int sh = (int)(pb >> 23) - 150 + sc;
    const uint32_t m24 = (pb & 0x7fffffu) | 0x800000u;
    if (sc >= 0) W = sh >= 0 ? ((uint64_t)m24 << sh) : (uint64_t)(m24 >> (-sh < 31 ? -sh : 31));
  } else {
    if (sc >= 0) {
      const R v = p * pow2(sc, (R)0);
      W = f2u64_rz(v);
    }
  }
  const uint64_t cap = 1ull << k;
  return W > cap ? cap : W;
}

// Box-Muller, first output, from one 128-bit draw; and the extra uniform.
__device__ __forceinline__ float bm_normal_f(const U4& w) {
  const float u1 = unif_f32(w.a);
  const float u2 = unif_f32(w.b);
  const float L = det_log(u1);
  const float m2 = L * -2.0f;
  const float r = sqrtf(m2);
  const float c = det_cos2pi(u2);
  return r * c;
}
__device__ __forceinline__ double bm_normal_d(const U4& w) {
  const double u1 = unif_f64(w.a, w.b);
  const double u2 = unif_f64_32(w.c);
  const double L = det_log(u1);
  const double m2 = L * -2.0;
  const double r = sqrt(m2);
  const double c = det_cos2pi(u2);
  return r * c;
}
__device__ __forceinline__ void bm_normal2_f(const U4& w, float* zc, float* zs) {
  const float u1 = unif_f32(w.a);
  const float u2 = unif_f32(w.b);
  const float L = det_log(u1);
  const float m2 = L * -2.0f;
  const float r = sqrtf(m2);
  float sn, cs;
  det_sincos2pi(u2, &sn, &cs);
  *zc = r * cs;
  *zs = r * sn;
}
__device__ __forceinline__ void bm_normal2_d(const U4& w, double* zc, double* zs) {
  const double u1 = unif_f64(w.a, w.b);
  const double u2 = unif_f64_32(w.c);
  const double L = det_log(u1);
  const double m2 = L * -2.0;
  const double r = sqrt(m2);
  double sn, cs;
  det_sincos2pi(u2, &sn, &cs);
  *zc = r * cs;
  *zs = r * sn;
}
__device__ __forceinline__ void bm_normal2(const U4& w, float* zc, float* zs) { bm_normal2_f(w, zc, zs); }
__device__ __forceinline__ void bm_normal2(const U4& w, double* zc, double* zs) { bm_normal2_d(w, zc, zs); }
__device__ __forceinline__ float bm_normal(const U4& w, float) { return bm_normal_f(w); }
__device__ __forceinline__ double bm_normal(const U4& w, double) { return bm_normal_d(w); }
__device__ __forceinline__ float extra_uniform(const U4& w, float) { return unif_f32(w.c); }
__device__ __forceinline__ double extra_uniform(const U4& w, double) { return unif_f64_32(w.d); }

__device__ __forceinline__ float fmaR(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmaR(double a, double b, double c) { return __fma_rn(a, b, c); }

// Gamma(a, 1) for a >= 1 by Marsaglia & Tsang (2000), d = a - 1/3,
// c = 1/sqrt(9d), v = fma(c, Z, 1): accept d v^3 when v > 0 and either the
// squeeze U < fma(-K, Z^4, 1) holds (K = 0.0331 (2/3) / d, a bound that
// implies the full test for every d >= 2/3 and equals Marsaglia & Tsang's
// 0.0331 at d = 2/3) or the full test
// log U < fma(d, (1 - v^3) + log v^3, Z^2 / 2) does.  Attempt k uses draw
// (purpose, k); after 16 rejections *fail is set and d is returned.
template <class R>
__device__ __forceinline__ R gamma_mt_from(R d, R c, R K, R Z0, R U0, uint64_t seed,
                                           uint32_t filter, uint32_t t, uint32_t j,
                                           uint32_t purpose, bool* fail) {
  for (uint32_t attempt = 0; attempt < 16; ++attempt) {
    R Z = Z0, U = U0;
    if (attempt > 0) {
      const U4 w = draw(seed, filter, t, j, purpose, attempt);
      Z = bm_normal(w, (R)0);
      U = extra_uniform(w, (R)0);
    }
    const R v = fmaR(c, Z, (R)1);
    if (!(v > (R)0)) continue;
    const R vv = v * v;
    const R v3 = vv * v;
    const R Z2 = Z * Z;
    const R z4 = Z2 * Z2;
    const R thr = fmaR(-K, z4, (R)1);
    if (U < thr) return d * v3;
    const R lhs = det_log(U);
    const R a1 = (R)1 - v3;
    const R a2 = det_log(v3);
    const R a3 = a1 + a2;
    const R a5 = (R)0.5 * Z2;
    const R rhs = fmaR(d, a3, a5);
    if (lhs < rhs) return d * v3;
  }
  *fail = true;
  return d;
}
// Marsaglia-Tsang attempt 0 restricted to the squeeze: returns true and
// *G = d v^3 when v > 0 and U < fma(-K, Z^4, 1) (the same test, in the same
// order, as the first step of gamma_mt_from); otherwise the draw must be
// finished by gamma_mt_from with the same (Z, U).
template <class R>
__device__ __forceinline__ bool gamma_mt_squeeze(R d, R c, R K, R Z, R U, R* G) {
  const R v = fmaR(c, Z, (R)1);
  if (!(v > (R)0)) return false;
  const R vv = v * v;
  const R v3 = vv * v;
  const R Z2 = Z * Z;
  const R z4 = Z2 * Z2;
  const R thr = fmaR(-K, z4, (R)1);
  if (!(U < thr)) return false;
  *G = d * v3;
  return true;
}

template <class R>
__device__ __forceinline__ R gamma_mt(R d, R c, R K, uint64_t seed, uint32_t filter, uint32_t t,
                                      uint32_t j, uint32_t purpose, bool* fail) {
  const U4 w = draw(seed, filter, t, j, purpose, 0);
  return gamma_mt_from<R>(d, c, K, bm_normal(w, (R)0), extra_uniform(w, (R)0), seed, filter, t,
                          j, purpose, fail);
}

// The draws of one propagation step for slot j: A = (j, t, STATE, 0) gives
// the state normal (cos branch) and the sigma^2 gamma draw's first normal
// (sin branch) and uniform (word 2).  The tau^2 gamma draw's first normal and
// uniform: in binary32, slots 2i and 2i + 1 share B = (i, t, STATE, 1) -- the
// cos output of its Box-Muller pair and word 2 go to the even slot, the sin
// output and word 3 to the odd one; in binary64 (whose Box-Muller takes three
// words), B = (j, t, STATE, 1), its first output and its uniform.
template <class R>
__device__ __forceinline__ void theta_draws_from(const U4& A, const U4& B, uint32_t j, R* Zx,
                                                 R* Zs, R* Us, R* Zt, R* Ut) {
  bm_normal2(A, Zx, Zs);
  *Us = extra_uniform(A, (R)0);
  if constexpr (sizeof(R) == 4) {
    R zc, zs;
    bm_normal2(B, &zc, &zs);
    *Zt = (j & 1u) ? zs : zc;
    *Ut = unif_f32((j & 1u) ? B.d : B.c);
  } else {
    *Zt = bm_normal(B, (R)0);
    *Ut = extra_uniform(B, (R)0);
  }
}
template <class R>
__device__ __forceinline__ uint32_t theta_b_index(uint32_t j) {
  return sizeof(R) == 4 ? (j >> 1) : j;
}
template <class R>
__device__ __forceinline__ void theta_draws(uint64_t seed, uint32_t filter, uint32_t t,
                                            uint32_t j, R* Zx, R* Zs, R* Us, R* Zt, R* Ut) {
  const U4 A = draw(seed, filter, t, j, P_STATE, 0);
  const U4 B = draw(seed, filter, t, theta_b_index<R>(j), P_STATE, 1);
  theta_draws_from<R>(A, B, j, Zx, Zs, Us, Zt, Ut);
}
// The same draws with the Philox round keys given (philox_rk).
template <class R>
__device__ __forceinline__ void theta_draws_rk(const uint32_t* rk, uint32_t filter, uint32_t t,
                                               uint32_t j, R* Zx, R* Zs, R* Us, R* Zt, R* Ut) {
  const U4 A = philox_rk(j, t, filter, P_STATE, rk);
  const U4 B = philox_rk(theta_b_index<R>(j), t, filter, P_STATE | (1u << 8), rk);
  theta_draws_from<R>(A, B, j, Zx, Zs, Us, Zt, Ut);
}

// ---------------------------------------------------------------------------
// Paired binary32 arithmetic for two particles at once (sm_100+ FADD2 /
// FMUL2 / FFMA2: one instruction, two independently rounded IEEE results).
// Each function below performs, lane by lane, exactly the operation sequence
// of its scalar counterpart above, so the two lanes' results are the scalar
// results bit for bit.  Division, square root, comparisons and integer
// conversions stay per lane.
// ---------------------------------------------------------------------------
// Additions stay scalar, one add.rn per lane: ptxas contracts a paired
// mul.rn feeding a paired addition (add.rn.f32x2, or an fma.rn.f32x2 with a
// unit factor) into one fused FFMA2 -- a different rounding -- even with
// contraction disabled, which scalar add.rn never allows.  Products and
// true fused multiply-adds (the Horner steps) are paired.
__device__ __forceinline__ float2 splat2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
      "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
  return make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y));
}
// A paired addition (FADD2).  Only for operands that are not the result of a
// paired multiplication (loads, integer-built values, fused multiply-adds),
// which ptxas could otherwise contract into one FFMA2.
__device__ __forceinline__ float2 addp(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return make_float2(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y));
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

__device__ __forceinline__ float2 unif_f32_2(uint32_t w0, uint32_t w1) {
  const float2 fm = sub2(make_float2(__uint_as_float(0x4B000000u | (w0 >> 9)),
                                     __uint_as_float(0x4B000000u | (w1 >> 9))),
                         splat2(8388608.0f));
  const float2 a = mul2(fm, splat2(0x1p-23f));
  return add2(a, splat2(0x1p-24f));
}

// det_log on two positive values
__device__ __forceinline__ float2 det_log2(float2 x) {
  int e0, e1;
  const uint32_t m0 = log_reduce(x.x, &e0), m1 = log_reduce(x.y, &e1);
  const float2 u = addp(make_float2(__uint_as_float(m0), __uint_as_float(m1)), splat2(-1.0f));
  float2 q = splat2(logq_f(8));
#pragma unroll
  for (int j = 7; j >= 0; --j) q = fma2(q, u, splat2(logq_f(j)));
  const float2 u2 = mul2(u, u);
  const float2 lf = fma2(u2, q, u);
  const float2 ef = make_float2(small_int_to_f32(e0), small_int_to_f32(e1));
  const float2 lo = fma2(ef, splat2(Cst<float>::LN2_LO), lf);
  const float2 r = fma2(ef, splat2(Cst<float>::LN2_HI), lo);
  return make_float2(x.x < INFINITY ? r.x : x.x, x.y < INFINITY ? r.y : x.y);
}

__device__ __forceinline__ float2 cos_poly2(float2 x) {
  const float2 x2 = mul2(x, x);
  float2 p = splat2(-0x1.27e4fcp-22f);
  p = fma2(p, x2, splat2(0x1.a01a02p-16f));
  p = fma2(p, x2, splat2(-0x1.6c16c2p-10f));
  p = fma2(p, x2, splat2(0x1.555556p-5f));
  p = fma2(p, x2, splat2(-0x1p-1f));
  p = fma2(p, x2, splat2(0x1p+0f));
  return p;
}
__device__ __forceinline__ float2 sin_poly2(float2 x) {
  const float2 x2 = mul2(x, x);
  float2 p = splat2(0x1.71de3ap-19f);
  p = fma2(p, x2, splat2(-0x1.a01a02p-13f));
  p = fma2(p, x2, splat2(0x1.111112p-7f));
  p = fma2(p, x2, splat2(-0x1.555556p-3f));
  p = fma2(p, x2, splat2(0x1p+0f));
  return mul2(x, p);
}

// det_sincos2pi on two values of [0, 1]
__device__ __forceinline__ void det_sincos2pi2(float2 u, float2* s_out, float2* c_out) {
  const float2 ru = make_float2(u.x > 0.5f ? 1.0f : 0.0f, u.y > 0.5f ? 1.0f : 0.0f);
  const float2 v = sub2(u, ru);
  const float2 w = make_float2(fabsf(v.x), fabsf(v.y));
  const float2 h = sub2(splat2(0.5f), w);
  const float2 q = sub2(splat2(0.25f), w);
  const bool o1x = w.x <= 0.125f, o3x = w.x > 0.375f;
  const bool o1y = w.y <= 0.125f, o3y = w.y > 0.375f;
  const float2 a = make_float2(o1x ? w.x : (o3x ? h.x : q.x), o1y ? w.y : (o3y ? h.y : q.y));
  const float2 x = mul2(splat2(Cst<float>::TWO_PI), a);
  const float2 S = sin_poly2(x);
  const float2 C = cos_poly2(x);
  const float svx = (o1x || o3x) ? S.x : C.x, svy = (o1y || o3y) ? S.y : C.y;
  *s_out = make_float2(v.x < 0.0f ? -svx : svx, v.y < 0.0f ? -svy : svy);
  *c_out = make_float2(o1x ? C.x : (o3x ? -C.x : S.x), o1y ? C.y : (o3y ? -C.y : S.y));
}

// the propagation draws (theta_draws_rk) of the two slots 2i, 2i + 1 of a
// pair: A of each slot through one paired Box-Muller transform, the pair's
// shared B through one scalar transform whose two outputs both serve
__device__ __forceinline__ void theta_draws2(const uint32_t* rk, uint32_t filter, uint32_t t,
                                             uint32_t i, float2* Zx, float2* Zs, float2* Us,
                                             float2* Zt, float2* Ut) {
  const U4 A0 = philox_rk(2u * i, t, filter, P_STATE, rk);
  const U4 A1 = philox_rk(2u * i + 1u, t, filter, P_STATE, rk);
  const U4 B = philox_rk(i, t, filter, P_STATE | (1u << 8), rk);
  {
    const float2 u1 = unif_f32_2(A0.a, A1.a);
    const float2 u2 = unif_f32_2(A0.b, A1.b);
    const float2 L = det_log2(u1);
    const float2 m2 = mul2(L, splat2(-2.0f));
    const float2 r = make_float2(sqrtf(m2.x), sqrtf(m2.y));
    float2 sn, cs;
    det_sincos2pi2(u2, &sn, &cs);
    *Zx = mul2(r, cs);
    *Zs = mul2(r, sn);
    *Us = unif_f32_2(A0.c, A1.c);
  }
  {
    float zc, zs;
    bm_normal2_f(B, &zc, &zs);
    *Zt = make_float2(zc, zs);
    *Ut = unif_f32_2(B.c, B.d);
  }
}

// ---------------------------------------------------------------------------
// 128-bit unsigned helpers (hi, lo).
// ---------------------------------------------------------------------------
struct U128 {
  uint64_t hi, lo;
};
__device__ __forceinline__ U128 mul64(uint64_t a, uint64_t b) {
  return U128{__umul64hi(a, b), a * b};
}
// a * b for b < 2^32: two 32x32 -> 64 products instead of a 64x64 multiply.
__device__ __forceinline__ U128 mul64x32(uint64_t a, uint32_t b) {
  const uint64_t p0 = (uint64_t)(uint32_t)a * b;
  const uint64_t p1 = (a >> 32) * (uint64_t)b;
  const uint64_t lo = p0 + (p1 << 32);
  return U128{(p1 >> 32) + (lo < p0 ? 1ull : 0ull), lo};
}
__device__ __forceinline__ U128 add128(U128 x, uint64_t y) {
  const uint64_t lo = x.lo + y;
  return U128{x.hi + (lo < y ? 1ull : 0ull), lo};
}
__device__ __forceinline__ U128 add128(U128 x, U128 y) {
  const uint64_t lo = x.lo + y.lo;
  return U128{x.hi + y.hi + (lo < y.lo ? 1ull : 0ull), lo};
}
__device__ __forceinline__ bool le128(U128 x, U128 y) {
  return x.hi < y.hi || (x.hi == y.hi && x.lo <= y.lo);
}
__device__ __forceinline__ bool lt128(U128 x, U128 y) {
  return x.hi < y.hi || (x.hi == y.hi && x.lo < y.lo);
}
__device__ __forceinline__ U128 shl128(uint64_t v, int s) {  // v << s, 0 <= s < 128
  if (s == 0) return U128{0, v};
  if (s < 64) return U128{v >> (64 - s), v << s};
  return U128{v << (s - 64), 0};
}

// floor(X / d) for X = (xh, xl) when the quotient is below 2^53: binary64
// estimate, then exact correction with 128-bit products.
__device__ __forceinline__ uint64_t div128_small(U128 X, uint64_t d) {
  const double xd = __ull2double_rn(X.hi) * 0x1p64 + __ull2double_rn(X.lo);
  const double qd = xd / __ull2double_rn(d);
  uint64_t q = qd <= 0.0 ? 0ull : __double2ull_rz(qd);
  for (int it = 0; it < 8; ++it) {
    const U128 p = mul64(q, d);
    if (!le128(p, X)) {
      --q;
      continue;
    }
    const U128 p1 = add128(p, d);
    if (le128(p1, X)) {
      ++q;
      continue;
    }
    break;
  }
  return q;
}

// Conversions between binary32 and uint64 with integer instructions only
// (the hardware 64-bit conversions issue on the binary64 pipe, which is a
// small fraction of the binary32 rate on this part).  Results equal the C
// conversions: truncation toward zero, and round-to-nearest-even.
__device__ __forceinline__ uint64_t f2u64_rz(float v) {  // v >= 0, finite, < 2^64
  const uint32_t b = __float_as_uint(v);
  const int e = (int)(b >> 23) - 127;
  if (e < 0) return 0;
  const uint64_t m = (b & 0x7fffffu) | 0x800000u;
  return e >= 23 ? (m << (e - 23)) : (m >> (23 - e));
}
// u64 -> binary32, round to nearest even.  Values below 2^32 convert in one
// hardware u32 conversion.  Above, the top 32 bits m = b >> s (s = 32 minus
// the leading zeros of the high word) carry 8 bits below the binary32
// rounding position; OR-ing "any lower bit set" into m's last bit keeps
// every tie and sticky decision of the 64-bit value, so converting m and
// scaling by 2^s (exact) rounds b correctly.
__device__ __forceinline__ float u64_to_f32_rn(uint64_t b) {
  const uint32_t hi = (uint32_t)(b >> 32);
  if (hi == 0) return __uint2float_rn((uint32_t)b);
  const int s = 32 - __clz(hi);  // 1 .. 32
  const uint32_t m = (uint32_t)(b >> s);
  const uint32_t sticky = (b & ((1ull << s) - 1ull)) != 0ull ? 1u : 0u;
  const float f = __uint2float_rn(m | sticky);
  return f * __int_as_float((127 + s) << 23);  // * 2^s, exact
}
__device__ __forceinline__ uint64_t f2u64_rz(double v) { return __double2ull_rz(v); }

// Order-preserving encodings for atomicMax on floating point.
__device__ __forceinline__ uint32_t enc_f(float x) {
  const uint32_t b = __float_as_uint(x);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float dec_f(uint32_t e) {
  return __uint_as_float((e & 0x80000000u) ? (e & 0x7fffffffu) : ~e);
}
__device__ __forceinline__ unsigned long long enc_d(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double dec_d(unsigned long long e) {
  return __longlong_as_double((long long)((e & 0x8000000000000000ull) ? (e & 0x7fffffffffffffffull) : ~e));
}

}  // namespace pfk
