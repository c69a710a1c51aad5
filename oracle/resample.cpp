// CPU oracle, part 2: the resampling CDF in exact fixed point, resampling
// positions, and the ancestor searches of the paper's Section 3.
// TEST INFRASTRUCTURE ONLY (see oracle.h).
#include <algorithm>
#include <cmath>

#include "oracle.h"

namespace oracle {

int cdf_shift(uint64_t n) {
  int c = 0;
  while ((1ull << c) < n) ++c;  // c = ceil(log2 n)
  return 61 - c;
}

// Eq. (resample.cdf): q(i) proportional to the running sum of the weights.
// pin: equality with Python's exact integer cumulative sum, and the
// worked example of Table 1 (tests/test_oracle_resample.py).
void cdf_scan(const uint64_t* W, uint64_t n, uint64_t* Q) {
  uint64_t run = 0;
  for (uint64_t i = 0; i < n; ++i) {
    run += W[i];
    Q[i] = run;
  }
}

int quantize_weights_f32(const float* w, uint64_t n, uint64_t* W) {
  float mx = 0.0f;
  for (uint64_t i = 0; i < n; ++i) {
    if (!(w[i] >= 0.0f) || !std::isfinite(w[i])) return -1;
    if (w[i] > mx) mx = w[i];
  }
  if (!(mx > 0.0f)) return -1;
  int e;
  (void)std::frexp(mx, &e);
  int k = cdf_shift(n);
  for (uint64_t i = 0; i < n; ++i) {
    float v = std::ldexp(w[i], k - e);
    W[i] = (uint64_t)v;
  }
  return 0;
}

static inline uint64_t mulhi64(uint64_t a, uint64_t b) {
  return (uint64_t)(((u128)a * b) >> 64);
}

uint64_t systematic_offset(uint64_t T, uint64_t seed, uint32_t filter, uint32_t t) {
  W4 w = draw(seed, filter, t, 0, P_SYS_OFFSET, 0);
  uint64_t R = ((uint64_t)w.w[1] << 32) | w.w[0];
  return mulhi64(R, T);
}

Positions systematic_positions_with_offset(uint64_t n, uint64_t T, uint64_t r) {
  Positions P;
  P.A = (u128)n;
  P.B.resize(n);
  P.bucket.resize(n);
  for (uint64_t j = 0; j < n; ++j) {
    P.B[j] = (u128)j * T + r;
    P.bucket[j] = j;  // floor((j T + r) / T) = j since r < T
  }
  return P;
}

Positions systematic_positions(uint64_t n, uint64_t T, uint64_t seed, uint32_t filter,
                               uint32_t t) {
  return systematic_positions_with_offset(n, T, systematic_offset(T, seed, filter, t));
}

uint64_t stratified_offset(uint64_t T, uint64_t seed, uint32_t filter, uint32_t t, uint64_t j) {
  W4 w = draw(seed, filter, t, (uint32_t)(j >> 1), P_STRATIFIED, 0);
  const int h = (int)(j & 1) * 2;
  uint64_t R = ((uint64_t)w.w[h + 1] << 32) | w.w[h];
  return mulhi64(R, T);
}

// Stratified resampling: slot j's uniform lies in the j-th of n equal strata.
// pin: every slot stays in its stratum, offspring within one of the exact
// mean on either side, mean offspring over seeds equal to n W_i / T, and the
// naive search agrees (tests/test_oracle_resample.py).
Positions stratified_positions(uint64_t n, uint64_t T, uint64_t seed, uint32_t filter,
                               uint32_t t) {
  Positions P;
  P.A = (u128)n;
  P.B.resize(n);
  P.bucket.resize(n);
  for (uint64_t j = 0; j < n; ++j) {
    P.B[j] = (u128)j * T + stratified_offset(T, seed, filter, t, j);
    P.bucket[j] = j;  // r_j < T
  }
  return P;
}

void spacing_prefix(uint64_t n, uint64_t seed, uint32_t filter, uint32_t t,
                    std::vector<uint64_t>* S) {
  S->assign(n + 1, 0);
  uint64_t run = 0;
  for (uint64_t l = 0; l <= n; ++l) {
    W4 w = draw(seed, filter, t, (uint32_t)(l >> 2), P_SPACING, 0);
    float u = unif_f32(w.w[l & 3]);
    float L = det_log(u);
    float x = -L * 0x1p31f;  // exact scaling of -log(u) to 2^-31 fixed point
    uint64_t E = (uint64_t)x;
    run += E;
    (*S)[l] = run;
  }
}

Positions multinomial_positions(uint64_t n, uint64_t T, uint64_t seed, uint32_t filter,
                                uint32_t t) {
  std::vector<uint64_t> S;
  spacing_prefix(n, seed, filter, t, &S);
  Positions P;
  P.A = (u128)S[n];
  P.B.resize(n);
  P.bucket.resize(n);
  for (uint64_t j = 0; j < n; ++j) {
    P.B[j] = (u128)S[j] * T;
    P.bucket[j] = (uint64_t)(((u128)n * S[j]) / S[n]);  // floor(n S_j / S_n)
  }
  return P;
}

// Multinomial resampling with sorted uniforms (paper Section 3.1): the search
// for each sorted position starts where the previous one stopped.
void walk(const uint64_t* Q, uint64_t n, const Positions& P, uint32_t* anc) {
  uint64_t i = 0;
  for (uint64_t j = 0; j < n; ++j) {
    while (i < n && (u128)Q[i] * P.A <= P.B[j]) ++i;
    anc[j] = (uint32_t)i;
  }
}

// Naive multinomial search (paper Section 3.1): every position scans from 0.
void naive_search(const uint64_t* Q, uint64_t n, const Positions& P, uint32_t* anc) {
  for (uint64_t j = 0; j < n; ++j) {
    uint64_t i = 0;
    while (i < n && (u128)Q[i] * P.A <= P.B[j]) ++i;
    anc[j] = (uint32_t)i;
  }
}

// Algorithm "Parallelized Cut-Point Search" (paper Section 3.2), 0-based:
// thread i computes L_i = ceil(n Q_i / T) and writes I_k = i for every k with
// L_{i-1} <= k < L_i.  I_k is then the first index whose CDF value exceeds k/n
// (the definition of the cut-point).
void cutpoint_search(const uint64_t* Q, uint64_t n, uint64_t* L, uint32_t* I) {
  uint64_t T = Q[n - 1];
  for (uint64_t i = 0; i < n; ++i) {
    u128 num = (u128)n * Q[i];
    u128 q = num / T;
    L[i] = (uint64_t)(q * T == num ? q : q + 1);
  }
  for (uint64_t i = 0; i < n; ++i) {
    uint64_t lo = (i == 0) ? 0 : L[i - 1];
    for (uint64_t k = lo; k < L[i]; ++k) I[k] = (uint32_t)i;
  }
}

// Algorithm "Cut-Point Method" (paper Section 3.2) for given positions:
// start at the cut-point of the position's bucket and climb the CDF.
void cutpoint_method(const uint64_t* Q, uint64_t n, const uint32_t* I, const Positions& P,
                     uint32_t* anc) {
  for (uint64_t j = 0; j < n; ++j) {
    uint64_t k = I[P.bucket[j]];
    while (k < n && (u128)Q[k] * P.A <= P.B[j]) ++k;
    anc[j] = (uint32_t)k;
  }
}

void resample(const uint64_t* Q, uint64_t n, int scheme, uint64_t seed, uint32_t filter,
              uint32_t t, uint32_t* anc) {
  uint64_t T = Q[n - 1];
  if (scheme == STRATIFIED) {
    Positions P = stratified_positions(n, T, seed, filter, t);
    walk(Q, n, P, anc);
    return;
  }
  if (scheme == SYSTEMATIC || scheme == SYSTEMATIC_CUTPOINT) {
    Positions P = systematic_positions(n, T, seed, filter, t);
    if (scheme == SYSTEMATIC) {
      walk(Q, n, P, anc);
    } else {
      std::vector<uint64_t> L(n);
      std::vector<uint32_t> I(n);
      cutpoint_search(Q, n, L.data(), I.data());
      cutpoint_method(Q, n, I.data(), P, anc);
    }
  } else {
    Positions P = multinomial_positions(n, T, seed, filter, t);
    if (scheme == MULTINOMIAL) {
      walk(Q, n, P, anc);
    } else {
      std::vector<uint64_t> L(n);
      std::vector<uint32_t> I(n);
      cutpoint_search(Q, n, L.data(), I.data());
      cutpoint_method(Q, n, I.data(), P, anc);
    }
  }
}

}  // namespace oracle
