// Batched particle learning: many independent filters of uneven size, one
// persistent launch per cycle.
//
// Each CTA takes whole filters from a work list ordered by size (largest
// first) and runs the complete cycle of a filter with block barriers only:
//   1. predictive weights l_i and their maximum (Algorithm "Particle
//      Learning", Step 1),
//   2. the exact fixed-point CDF (Section 3) by a chunked block scan with a
//      carry between chunks,
//   3. resampling (Section 3.1): systematic by a per-thread walk over equally
//      spaced slot keys, multinomial by exponential spacings (a second
//      chunked block scan) and the same walk over the sorted position keys,
//   4. propagation of x, the sufficient statistics and theta (Steps 2-4),
//      with the block's queue of gamma draws that missed the squeeze,
// then folds the filter's log marginal likelihood increment and advances its
// cycle counter.
//
// Every per-particle operation (weights, quantisation, draws keyed by the
// filter's seed and id, the resampling keys, the propagation arithmetic) is
// the one of the single-filter kernels, and the per-thread partial sums of the
// log-ML and of the summaries are taken over the same particle groups and
// folded in the same order, so a filter in a batch reproduces a standalone
// filter with the same configuration bit for bit.
#pragma once
#include "kernels.cuh"

namespace pfk {

// Per-filter state of a batch, one per slot (device array).
struct BatchFilter {
  uint64_t off;        // first particle in the pooled arrays (multiple of 32)
  uint64_t seed;       // Philox key
  uint32_t n;          // particles (0: free slot)
  uint32_t filter_id;  // third Philox counter word
  uint32_t t;          // cycles completed
  uint32_t err;        // ErrBits
  int32_t k;           // CDF shift: W <= 2^k
  uint32_t learn;      // 0: sigma^2, tau^2 known (held at their given values)
  double x0_mean, x0_var, a_sigma, b_sigma, a_tau, b_tau, sigma2, tau2;
  double logml;        // accumulated log marginal likelihood
  // adaptive resampling (ess_frac > 0): resample only when the ESS of the
  // combined weights falls below ess_frac n; slam = sum_i exp(lambda_i) of the
  // carried log-weights (n after a resampling)
  double ess_frac;
  double slam;
};

// One entry of an admission list: the slot and its new record.
struct BatchInit {
  uint32_t slot;
  uint32_t pad[3];
  BatchFilter rec;
};

// One entry of a cycle's work list.
struct BatchItem {
  uint32_t slot;
  uint32_t pad;
  double y;            // this filter's observation for the cycle
};

template <class R>
struct BatchArgs {
  StateV<R> st[2];          // pooled particles, ping-pong by each filter's parity
  R* ell;                   // per particle
  R* lam;                   // per particle: carried log-weights lambda of adaptive
                            // filters (batches created for them; else NULL)
  uint64_t* Q;              // per particle
  uint64_t* S;              // per particle (multinomial spacing prefix S_0..S_{n-1})
  uint32_t* anc;            // per particle
  BatchFilter* F;           // per slot
  const BatchItem* items;   // work list, largest filters first
  const uint32_t* count;    // [0] number of items, [1] large items (cluster launches)
  uint32_t* ctr;            // [0] next large item, [1] finished CTAs, [2] next other item;
                            // all 0 between launches
  double* est;              // k_batch_estimate: BATCH_EST_ROW doubles per item, in list order
  const BatchInit* inits;   // k_batch_init: the admitted filters (count in *count)
  int commit;               // 0: a trial cycle that leaves t, log-ML and err untouched
};

constexpr int BB = BLOCK;                 // threads per CTA of the init and summary kernels
constexpr int BATCH_EST_ROW = 9;          // t, 6 summaries, log-ML, error bits
constexpr int BB_CAP = 32;                // slots emitted per particle before a run
constexpr int BB_MAX_RUNS = 1024;         // runs per tile held in shared memory

// Exclusive block prefix of one value per thread (NW warps), and the block
// total.
template <int NW>
__device__ __forceinline__ uint64_t block_excl_scan(uint64_t v, uint64_t* s_warp,
                                                    uint64_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t incl = warp_incl_scan(v, lane);
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const uint64_t w = lane < NW ? s_warp[lane] : 0;
    const uint64_t wi = warp_incl_scan(w, lane);
    if (lane < NW) s_warp[lane] = wi - w;
    if (lane == NW - 1) s_warp[NW] = wi;
  }
  __syncthreads();
  const uint64_t excl = s_warp[warp] + incl - v;
  *total = s_warp[NW];
  __syncthreads();  // s_warp is reused by the next call
  return excl;
}

// Maximum over the block (NW warps), returned to every thread.
template <class R, int NW>
__device__ __forceinline__ R block_max_all(R v, R* s_red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane == 0) s_red[warp] = v;
  __syncthreads();
  R m = s_red[0];
  for (int i = 1; i < NW; ++i) m = fmax(m, s_red[i]);
  __syncthreads();  // s_red is reused by the next call
  return m;
}

// #{j in [lo, n) : S_j T < key} for nondecreasing S, by bisection.
__device__ __forceinline__ uint64_t multi_first_slot(const uint64_t* S, uint64_t n, uint64_t T,
                                                     U128 key, uint64_t lo) {
  uint64_t hi = n;
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    if (lt128(mul64(S[mid], T), key)) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// Thread-block clusters (sm_90+): a large filter is processed by the CTAs of
// one cluster together.  They exchange per-round totals through distributed
// shared memory and meet at cluster barriers (release / acquire at cluster
// scope, which also orders their global-memory writes).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// Barrier over the G CTAs processing one filter (G = 1: the CTA itself).
__device__ __forceinline__ void group_sync(uint32_t G) {
  if (G > 1)
    asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
                 "barrier.cluster.wait.acquire.aligned;" ::: "memory");
  else
    __syncthreads();
}
__device__ __forceinline__ uint32_t dsm_addr(const void* p, uint32_t rank) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
// Read a shared variable of CTA `rank` of this cluster.
template <class T>
__device__ __forceinline__ T dsm_ld(const T* p, uint32_t rank) {
  static_assert(sizeof(T) == 4 || sizeof(T) % 8 == 0, "4-byte or 8-byte words");
  T v;
  if constexpr (sizeof(T) == 4) {
    uint32_t u;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(u) : "r"(dsm_addr(p, rank)) : "memory");
    memcpy(&v, &u, 4);
  } else {
#pragma unroll
    for (int i = 0; i < (int)(sizeof(T) / 8); ++i) {
      uint64_t u;
      asm volatile("ld.shared::cluster.u64 %0, [%1];"
                   : "=l"(u) : "r"(dsm_addr((const char*)p + 8 * i, rank)) : "memory");
      memcpy((char*)&v + 8 * i, &u, 8);
    }
  }
  return v;
}

// Shared memory of the cycle kernel.
template <class R, int NT>
struct BatchSmem {
  typedef typename ESumT<R>::T ES;
  uint64_t warp[NT / 32 + 1];
  R red[NT / 32];
  ES es[NT / 32];
  ES fold[32];                   // log-ML tile partials, lane-strided (group rank 0)
  uint32_t run[BB_MAX_RUNS][3];
  GammaItem<R> wq[NT / 32][WQ_CAP];   // per-warp queues of deferred gamma draws
  double c[6];
  uint32_t nruns;
  // read by the other CTAs of a group (distributed shared memory)
  R gmax;                        // this CTA's maximum of l
  uint64_t utot[2];              // this round's pass total, by round parity
  ES ues[2][NT / BLOCK];         // this round's tile partials, by round parity
  uint64_t SN;                   // S_n, if this CTA produced it
  uint32_t fail;
  U128 sq;                       // this CTA's exact sum of W^2 (adaptive filters)
  uint32_t work;                 // the group leader's claimed item
  // broadcasts within the CTA
  uint64_t roff, rsum;
  R m;
  uint32_t wb;
  U128 sqw[NT / 32];             // per-warp sums of W^2 (adaptive filters)
  uint32_t rk[20];               // Philox round keys of the filter's seed (binary32 propagation)
};

// One cycle of one filter by a group of G CTAs (G = 1: one CTA; G > 1: the
// CTAs of a cluster, this one being `rank`).  The particles are cut into
// passes of NT / 256 scan tiles; round j gives pass j G + rank to this CTA.
// Thread t of a pass owns its particles [16 t, 16 t + 16) -- the
// single-filter scan's ownership -- and the tile partials of the log-ML are
// folded in tile order, so the result does not depend on G.
template <class R, int POS, int NT, uint32_t G>
__device__ __forceinline__ void batch_filter(const BatchArgs<R>& a, const BatchItem item,
                                             BatchSmem<R, NT>& sm, const uint32_t rank) {
  typedef typename ESumT<R>::T ES;
  constexpr int NW = NT / 32;
  constexpr int TPP = NT / BLOCK;          // scan tiles per pass
  constexpr uint64_t PASS = (uint64_t)TPP * TILE;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  BatchFilter* F = &a.F[item.slot];
  const uint64_t off = F->off, n = F->n, seed = F->seed;
  const uint32_t fid = F->filter_id, t = F->t;
  const int k = F->k;
  const bool learn = F->learn != 0;
  const bool ess = F->ess_frac > 0.0;  // adaptive resampling (the same for the whole group)
  const StateV<R> src = (t & 1) ? a.st[1] : a.st[0];
  const StateV<R> dst = (t & 1) ? a.st[0] : a.st[1];
  const double y = item.y;
  const R yr = (R)y;
  if (threadIdx.x == 0) {
    // Marsaglia-Tsang constants of the shapes a0 + (t+1)/2
    double ds, cs, ks, dt, ct, kt;
    mt_constants(F->a_sigma + 0.5 * (double)(t + 1), &ds, &cs, &ks);
    mt_constants(F->a_tau + 0.5 * (double)(t + 1), &dt, &ct, &kt);
    sm.c[0] = ds; sm.c[1] = cs; sm.c[2] = dt; sm.c[3] = ct; sm.c[4] = ks; sm.c[5] = kt;
  }
  if (rank == 0 && threadIdx.x < 32) sm.fold[threadIdx.x].zero();
  bool fail = false;
  const uint64_t passes = (n + PASS - 1) / PASS;
  const uint64_t rounds = (passes + G - 1) / G;

  // 1. weights and their maximum, four particles per thread
  R mx = (R)-INFINITY;
  for (uint64_t jr = 0; jr < rounds; ++jr) {
    const uint64_t lo = (jr * G + rank) * PASS;
    const uint64_t hi = lo + PASS < n ? lo + PASS : n;
    for (uint64_t i = lo + 4 * (uint64_t)threadIdx.x; i < hi; i += 4 * NT) {
      if (i + 4 <= hi) {
        R xv[4], sv[4], tv[4], lv[4], lam4[4];
        if constexpr (sizeof(R) == 4) {
          const float4 X = *reinterpret_cast<const float4*>(src.x + off + i);
          const float4 Sg = *reinterpret_cast<const float4*>(src.s2 + off + i);
          const float4 Tu = *reinterpret_cast<const float4*>(src.t2 + off + i);
          xv[0] = X.x; xv[1] = X.y; xv[2] = X.z; xv[3] = X.w;
          sv[0] = Sg.x; sv[1] = Sg.y; sv[2] = Sg.z; sv[3] = Sg.w;
          tv[0] = Tu.x; tv[1] = Tu.y; tv[2] = Tu.z; tv[3] = Tu.w;
          if (ess) {
            const float4 Lm = *reinterpret_cast<const float4*>(a.lam + off + i);
            lam4[0] = Lm.x; lam4[1] = Lm.y; lam4[2] = Lm.z; lam4[3] = Lm.w;
          }
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            xv[e] = src.x[off + i + e]; sv[e] = src.s2[off + i + e]; tv[e] = src.t2[off + i + e];
            if (ess) lam4[e] = a.lam[off + i + e];
          }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          lv[e] = log_pred<R>(xv[e], sv[e], tv[e], yr);
          if (ess) lv[e] = lam4[e] + lv[e];  // adaptive filters: L = lambda + l
          fail |= !(lv[e] < (R)INFINITY);  // NaN or +inf
          mx = fmax(mx, lv[e]);
        }
        if constexpr (sizeof(R) == 4) {
          *reinterpret_cast<float4*>(a.ell + off + i) = make_float4(lv[0], lv[1], lv[2], lv[3]);
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) a.ell[off + i + e] = lv[e];
        }
      } else {
        for (uint64_t q = i; q < hi; ++q) {
          R l = log_pred<R>(src.x[off + q], src.s2[off + q], src.t2[off + q], yr);
          if (ess) l = a.lam[off + q] + l;
          fail |= !(l < (R)INFINITY);
          mx = fmax(mx, l);
          a.ell[off + q] = l;
        }
      }
    }
  }
  R m = block_max_all<R, NW>(mx, sm.red);
  if (G > 1) {
    if (threadIdx.x == 0) sm.gmax = m;
    group_sync(G);
    if (threadIdx.x == 0) {
      R v = m;
      for (uint32_t r = 0; r < G; ++r) v = fmax(v, dsm_ld(&sm.gmax, r));
      sm.m = v;
    }
    __syncthreads();
    m = sm.m;
  }
  if (!(m > (R)-INFINITY)) fail = true;

  // One round of an exclusive scan over the group: this CTA's pass total
  // goes out, its offset within the round and the round total come back.
  uint32_t par = 0;  // parity of the exchange buffers, alternating every round
  auto round_offsets = [&](uint64_t total, uint64_t* roff, uint64_t* rsum) {
    if (G == 1) {
      *roff = 0;
      *rsum = total;
      return;
    }
    if (threadIdx.x == 0) sm.utot[par] = total;
    group_sync(G);
    if (warp == 0) {
      const uint64_t v = (uint32_t)lane < G ? dsm_ld(&sm.utot[par], (uint32_t)lane) : 0ull;
      const uint64_t incl = warp_incl_scan(v, lane);
      if ((uint32_t)lane == rank) sm.roff = incl - v;
      if (lane == 31) sm.rsum = incl;
    }
  };

  // 2. quantised weights and their inclusive scan, round by round (with
  // adaptive resampling also the exact sum of W^2)
  uint64_t carry = 0;
  U128 sq{0, 0};
  for (uint64_t jr = 0; jr < rounds; ++jr, par ^= 1u) {
    const uint64_t pidx = jr * G + rank;
    const uint64_t c0 = pidx * PASS;
    const uint64_t base = c0 + (uint64_t)threadIdx.x * SCAN_PER;
    const bool full = base + SCAN_PER <= n;
    uint64_t W[SCAN_PER];
    R epart = (R)0;  // this thread's sum of exp(l - m), fixed order
    uint64_t run = 0;
#pragma unroll
    for (int q = 0; q < SCAN_PER / 4; ++q) {
      R v[4];
      if (full) {
        if constexpr (sizeof(R) == 4) {
          const float4 f = *reinterpret_cast<const float4*>(a.ell + off + base + 4 * q);
          v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
        } else {
          const double2 f0 = *reinterpret_cast<const double2*>(a.ell + off + base + 4 * q);
          const double2 f1 = *reinterpret_cast<const double2*>(a.ell + off + base + 4 * q + 2);
          v[0] = f0.x; v[1] = f0.y; v[2] = f1.x; v[3] = f1.y;
        }
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          v[e] = (base + 4 * q + e < n) ? a.ell[off + base + 4 * q + e] : (R)0;
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        uint64_t wq = 0;
        if (full || base + 4 * q + e < n) {
          R ex;
          const R dl = v[e] - m;
          wq = quant_exp<R>(dl, k, &ex);
          epart = epart + ex;
          if (ess) sq = add128(sq, mul64(wq, wq));
        }
        run += wq;
        W[4 * q + e] = run;  // inclusive running sum
      }
    }
    {
      ES es;
      es.zero();
      es.add(epart);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) es.add(es.shfl_xor(o));
      if (lane == 0) sm.es[warp] = es;
    }
    uint64_t total;
    const uint64_t excl = block_excl_scan<NW>(run, sm.warp, &total);  // its barriers publish sm.es
    if (threadIdx.x == 0) {
      // each tile's partial: its 8 warps in order
#pragma unroll
      for (int tp = 0; tp < TPP; ++tp) {
        ES tot = sm.es[tp * WARPS];
        for (int q = 1; q < WARPS; ++q) tot.add(sm.es[tp * WARPS + q]);
        sm.ues[par][tp] = tot;
      }
    }
    uint64_t roff, rsum;
    round_offsets(total, &roff, &rsum);
    if (threadIdx.x == 0 && rank == 0) {
      // the round's tile partials into the fold, in tile order: tiles
      // lane-strided over 32 accumulators, as the single-filter fold does
      for (uint32_t r = 0; r < G; ++r) {
#pragma unroll
        for (int tp = 0; tp < TPP; ++tp) {
          const uint64_t tile = (jr * G + r) * TPP + tp;
          if (tile * TILE >= n) continue;
          const ES pt = G == 1 ? sm.ues[par][tp] : dsm_ld(&sm.ues[par][tp], r);
          sm.fold[tile & 31].add(pt);
        }
      }
    }
    if (G > 1) {
      __syncthreads();
      roff = sm.roff;
      rsum = sm.rsum;
    }
    const uint64_t o = carry + roff + excl;
#pragma unroll
    for (int e = 0; e < SCAN_PER; ++e)
      if (full || base + e < n) a.Q[off + base + e] = o + W[e];
    carry += rsum;
  }
  const uint64_t T = carry;
  if (T == 0) fail = true;

  // adaptive resampling: the decision of the single-filter kernels (k_ess,
  // k_cdf_sys with ESS) from the same exact sums, T = sum W and B = sum W^2
  // (B summed warps in order, then the group's CTAs in rank order: an exact
  // integer sum, identical in every CTA of the group)
  bool resamp = true;
  if (ess) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      U128 u;
      u.hi = __shfl_xor_sync(0xffffffffu, sq.hi, o);
      u.lo = __shfl_xor_sync(0xffffffffu, sq.lo, o);
      sq = add128(sq, u);
    }
    if (lane == 0) sm.sqw[warp] = sq;
    __syncthreads();
    if (threadIdx.x == 0) {
      U128 b = sm.sqw[0];
      for (int w = 1; w < NW; ++w) b = add128(b, sm.sqw[w]);
      sm.sq = b;
    }
    group_sync(G);
    U128 B = sm.sq;
    if (G > 1) {
      B = dsm_ld(&sm.sq, 0u);
      for (uint32_t r2 = 1; r2 < G; ++r2) B = add128(B, dsm_ld(&sm.sq, r2));
    }
    const double Ad = __ull2double_rn(T);
    const double Bd = u128_to_f64_rn(B);
    const double lhs = Ad * Ad;
    const double f = F->ess_frac * (double)n;
    const double rhs = f * Bd;
    resamp = lhs < rhs;
  }

  // 3. resampling: slot keys B_j against the CDF keys Q_i A (ties go to the
  // CDF); thread t walks the particles [16 t, 16 t + 16) of each of this
  // CTA's passes from its first slot; a particle with more than BB_CAP slots
  // leaves a run for the whole CTA
  uint64_t A = n, r = 0;
  if (!resamp) {
    // an adaptive filter that keeps its particles this cycle: no keys
  } else if (POS == POS_SYSTEMATIC) {
    const U4 wr = draw(seed, fid, t, 0, P_SYS_OFFSET, 0);
    const uint64_t Rw = ((uint64_t)wr.b << 32) | wr.a;
    r = __umul64hi(Rw, T);
    group_sync(G);  // Q complete
  } else {
    // spacings S_l = E_0 + ... + E_l for l = 0..n (Carpenter, Clifford &
    // Fearnhead 1999), the same rounds; S_n stays in shared memory
    const uint64_t passes_e = (n + 1 + PASS - 1) / PASS;
    const uint64_t rounds_e = (passes_e + G - 1) / G;
    uint64_t cs = 0;
    for (uint64_t jr = 0; jr < rounds_e; ++jr, par ^= 1u) {
      const uint64_t base = (jr * G + rank) * PASS + (uint64_t)threadIdx.x * SCAN_PER;
      uint64_t Ev[SCAN_PER];
      uint64_t run = 0;
#pragma unroll
      for (int q = 0; q < SCAN_PER / 4; ++q) {
        const uint64_t l0 = base + 4 * q;  // multiple of 4
        U4 wd = {0, 0, 0, 0};
        if (l0 <= n) wd = draw(seed, fid, t, (uint32_t)(l0 >> 2), P_SPACING, 0);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          uint64_t E = 0;
          if (l0 + e <= n) E = spacing_E(seed, fid, t, l0 + e, wd);
          run += E;
          Ev[4 * q + e] = run;
        }
      }
      uint64_t total;
      const uint64_t excl = block_excl_scan<NW>(run, sm.warp, &total);
      uint64_t roff, rsum;
      round_offsets(total, &roff, &rsum);
      if (G > 1) {
        __syncthreads();
        roff = sm.roff;
        rsum = sm.rsum;
      }
      const uint64_t o = cs + roff + excl;
#pragma unroll
      for (int e = 0; e < SCAN_PER; ++e) {
        const uint64_t l = base + e;
        if (l < n) a.S[off + l] = o + Ev[e];
        else if (l == n) sm.SN = o + Ev[e];
      }
      cs += rsum;
    }
    group_sync(G);  // Q, S and S_n complete
    if (threadIdx.x == 0) {
      const uint32_t owner = (uint32_t)((n / PASS) % G);
      sm.roff = G == 1 ? sm.SN : dsm_ld(&sm.SN, owner);
    }
    __syncthreads();
    A = sm.roff;
  }
  const SysDiv dv = make_sysdiv(T > 0 ? T : 1);
  const uint64_t* Sf = a.S + off;
  if (threadIdx.x == 0) sm.nruns = 0;
  __syncthreads();
  for (uint64_t jr = 0; resamp && jr < rounds; ++jr) {
    const uint64_t ib = (jr * G + rank) * PASS + (uint64_t)threadIdx.x * SCAN_PER;
    if (T > 0 && ib < n) {
      const uint64_t ie = ib + SCAN_PER < n ? ib + SCAN_PER : n;
      uint64_t j = 0;
      const uint64_t qp = ib > 0 ? a.Q[off + ib - 1] : 0;
      if (ib > 0) {
        j = POS == POS_SYSTEMATIC ? sys_first_slot(qp, n, r, dv)
                                  : multi_first_slot(Sf, n, T, mul64(qp, A), 0);
      }
      if constexpr (POS == POS_SYSTEMATIC) {
        // one step per particle: with D = n Q_i - (j T + r), particle i owns
        // the c = ceil(D / T) slots from j (none if D <= 0); D stays an int64
        // (in (-T, 0] between particles, n w_i <= 2^61, T <= 2^61)
        const U128 X = mul64x32(qp, (uint32_t)n);
        const U128 KB = add128(mul64x32(T, (uint32_t)j), r);
        int64_t D = (int64_t)(X.lo - KB.lo);
        const int64_t Ti = (int64_t)T;
        uint64_t qprev = qp;
        for (uint64_t i = ib; i < ie; ++i) {
          const uint64_t qi = a.Q[off + i];
          D += (int64_t)((qi - qprev) * n);
          qprev = qi;
          uint32_t c = (uint32_t)(D > 0) + (uint32_t)(D > Ti);
          if (D > 2 * Ti) c = (uint32_t)(sys_floor_div(U128{0, (uint64_t)D - 1}, dv) + 1);
          if (c > (uint32_t)BB_CAP) {  // a heavy particle: hand its slots to the CTA
            const uint32_t kr = atomicAdd(&sm.nruns, 1u);
            if (kr < BB_MAX_RUNS) {
              sm.run[kr][0] = (uint32_t)j;
              sm.run[kr][1] = (uint32_t)(j + c);
              sm.run[kr][2] = (uint32_t)i;
            } else {
              for (uint64_t q = j; q < j + c; ++q) a.anc[off + q] = (uint32_t)i;
            }
          } else {
            for (uint32_t q = 0; q < c; ++q) a.anc[off + j + q] = (uint32_t)i;
          }
          D -= (int64_t)c * Ti;
          j += c;
        }
      } else {  // multinomial: slot by slot over the positions S_j T
        for (uint64_t i = ib; i < ie; ++i) {
          const uint64_t qi = a.Q[off + i];
          const U128 KQ = mul64(qi, A);
          int emitted = 0;
          while (j < n) {
            const U128 KB = mul64(Sf[j], T);
            if (!lt128(KB, KQ)) break;
            if (emitted == BB_CAP) {  // a heavy particle: hand its other slots to the CTA
              uint64_t R2 = multi_first_slot(Sf, n, T, KQ, j);
              R2 = R2 < j ? j : R2;
              const uint32_t kr = atomicAdd(&sm.nruns, 1u);
              if (kr < BB_MAX_RUNS) {
                sm.run[kr][0] = (uint32_t)j;
                sm.run[kr][1] = (uint32_t)R2;
                sm.run[kr][2] = (uint32_t)i;
              } else {
                for (uint64_t q = j; q < R2; ++q) a.anc[off + q] = (uint32_t)i;
              }
              j = R2;
              break;
            }
            a.anc[off + j] = (uint32_t)i;
            ++j;
            ++emitted;
          }
        }
      }
    }
    __syncthreads();
    const uint32_t nr = sm.nruns < BB_MAX_RUNS ? sm.nruns : BB_MAX_RUNS;
    for (uint32_t q = 0; q < nr; ++q) {
      const uint32_t st = sm.run[q][0], en = sm.run[q][1], v = sm.run[q][2];
      for (uint32_t jj = st + threadIdx.x; jj < en; jj += NT) a.anc[off + jj] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) sm.nruns = 0;
    __syncthreads();
  }
  if (T == 0 || !resamp) {
    // an empty CDF (flagged): keep every index in range; an adaptive filter
    // that keeps its particles: every slot is its own ancestor
    for (uint64_t j = rank * NT + threadIdx.x; j < n; j += (uint64_t)G * NT)
      a.anc[off + j] = (uint32_t)j;
  }
  // the Philox round keys of the filter's seed: the key words bumped by the
  // Weyl constants, round by round (read after the barrier below)
  if (sizeof(R) == 4 && threadIdx.x < 10) {
    sm.rk[2 * threadIdx.x] = (uint32_t)seed + threadIdx.x * 0x9E3779B9u;
    sm.rk[2 * threadIdx.x + 1] = (uint32_t)(seed >> 32) + threadIdx.x * 0xBB67AE85u;
  }
  group_sync(G);  // every ancestor written

  // 4. propagation, one slot per thread per pass (slot blocks of NT dealt
  // round-robin over the group); draws that miss the squeeze go to the
  // warp's queue, which the warp finishes 32 at a time
  const R ds = (R)sm.c[0], cs = (R)sm.c[1], dt = (R)sm.c[2], ct = (R)sm.c[3];
  const R ks = (R)sm.c[4], kt = (R)sm.c[5];
  GammaItem<R>* const wq = sm.wq[warp];
  uint32_t qn = 0;  // warp-uniform
  auto finish = [&](const GammaItem<R>& itm) {
    const bool sig = itm.which == 0;
    const R G2 = gamma_mt_from<R>(sig ? ds : dt, sig ? cs : ct, sig ? ks : kt, itm.Z, itm.U, seed,
                                  fid, t, itm.j, sig ? P_GAMMA_SIGMA : P_GAMMA_TAU, &fail);
    const R v = SuffOps<R>::ig(itm.b, G2);
    if (sig) dst.s2[off + itm.j] = v;
    else dst.t2[off + itm.j] = v;
  };
  // the filter's state, and the record of a slot's ancestor (gathered one
  // pass ahead, so that its latency overlaps the current pass)
  StateV<R> fsrc = src;
  fsrc.x += off; fsrc.s2 += off; fsrc.t2 += off; fsrc.bs += off; fsrc.bt += off;
  auto gather_slot = [&](uint64_t jj) {
    uint32_t an = jj < n ? (resamp ? a.anc[off + jj] : (uint32_t)jj) : 0u;
    an = an < n ? an : (uint32_t)(n - 1);
    return gather_rec<R>(fsrc, an);
  };
  if constexpr (sizeof(R) == 4) {
    // binary32: the slot pair 2k, 2k + 1 per thread (pair blocks of NT dealt
    // round-robin over the group), the two slots sharing draw B (reading 19)
    // and each paired FMUL2 / FFMA2: the operations of the single-filter
    // paired propagation, lane by lane the scalar ones, so the same bits
    const uint64_t np = (n + 1) / 2, ppstride = (uint64_t)G * NT;
    // the ancestors of a pair (clamped into range), loaded a pass ahead
    auto anc_of = [&](uint64_t jj) -> uint32_t {
      uint32_t an = jj < n ? (resamp ? a.anc[off + jj] : (uint32_t)jj) : 0u;
      return an < n ? an : (uint32_t)(n - 1);
    };
    uint64_t kq = (uint64_t)rank * NT + threadIdx.x;
    uint32_t a0 = anc_of(2 * kq), a1 = anc_of(2 * kq + 1);
    for (uint64_t k0 = (uint64_t)rank * NT; k0 < np; k0 += ppstride) {
      const uint64_t kp = k0 + threadIdx.x;
      const uint64_t j0 = 2 * kp, j1 = j0 + 1;
      const bool v0 = j0 < n, v1 = j1 < n;
      const Gathered<float> c0 = gather_rec<float>(fsrc, a0), c1 = gather_rec<float>(fsrc, a1);
      a0 = anc_of(2 * (kp + ppstride));
      a1 = anc_of(2 * (kp + ppstride) + 1);
      bool ds0 = false, dt0 = false, ds1 = false, dt1 = false;
      uint64_t bs0 = 0, bt0 = 0, bs1 = 0, bt1 = 0;
      float2 Zs = make_float2(0.0f, 0.0f), Us = Zs, Zt = Zs, Ut = Zs;
      if (v0) {
        const float2 xa = make_float2(c0.x, c1.x), sa = make_float2(c0.s2, c1.s2);
        const float2 ta = make_float2(c0.t2, c1.t2);
        // V and mu share one correctly rounded reciprocal of s = sigma^2 + tau^2
        const float2 sp = addp(sa, ta);
        const float2 ri = make_float2(__frcp_rn(sp.x), __frcp_rn(sp.y));
        const float2 V = mul2(mul2(sa, ta), ri);
        const float2 nn = fma2(xa, sa, mul2(splat2(yr), ta));
        const float2 mu = mul2(nn, ri);
        const float2 sv = make_float2(sqrtf(V.x), sqrtf(V.y));
        float2 Z;
        theta_draws2(sm.rk, fid, t, (uint32_t)kp, &Z, &Zs, &Us, &Zt, &Ut);
        const float2 xj = fma2(sv, Z, mu);
        const uint64_t d = off + j0;  // even: filter offsets are multiples of 32
        if (v1) *reinterpret_cast<float2*>(dst.x + d) = xj;
        else dst.x[d] = xj.x;
        if (learn) {
          const float2 rsd = addp(splat2(yr), make_float2(-xj.x, -xj.y));
          const float2 rtd = addp(xj, make_float2(-xa.x, -xa.y));
          // b + r^2 / 2 in 2^-32 fixed point, per SuffOps<float>::add_half_square
          const float2 ws = mul2(mul2(rsd, rsd), splat2(0x1p31f));
          const float2 wt = mul2(mul2(rtd, rtd), splat2(0x1p31f));
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
          fail |= f0 || (v1 && f1);
          if (v1) {
            *reinterpret_cast<ulonglong2*>(dst.bs + d) = make_ulonglong2(bs0, bs1);
            *reinterpret_cast<ulonglong2*>(dst.bt + d) = make_ulonglong2(bt0, bt1);
          } else {
            dst.bs[d] = bs0;
            dst.bt[d] = bt0;
          }
          // Marsaglia-Tsang squeeze for sigma^2 and tau^2 (x lanes: slot j0, y: j1)
          const float2 vs = fma2(splat2(cs), Zs, splat2(1.0f)), vt = fma2(splat2(ct), Zt, splat2(1.0f));
          const float2 v3s = mul2(mul2(vs, vs), vs), v3t = mul2(mul2(vt, vt), vt);
          const float2 Z2s = mul2(Zs, Zs), Z2t = mul2(Zt, Zt);
          const float2 thrs = fma2(splat2(-ks), mul2(Z2s, Z2s), splat2(1.0f));
          const float2 thrt = fma2(splat2(-kt), mul2(Z2t, Z2t), splat2(1.0f));
          const float2 Gs = mul2(splat2(ds), v3s), Gt = mul2(splat2(dt), v3t);
          const bool as0 = vs.x > 0.0f && Us.x < thrs.x, as1 = vs.y > 0.0f && Us.y < thrs.y;
          const bool at0 = vt.x > 0.0f && Ut.x < thrt.x, at1 = vt.y > 0.0f && Ut.y < thrt.y;
          // inverse gamma (b 2^-32) / G, per SuffOps<float>::ig, every lane
          const float2 bsf = fma2(make_float2(__uint2float_rn((uint32_t)bs0), __uint2float_rn((uint32_t)bs1)),
                                  splat2(0x1p-32f),
                                  make_float2(__uint2float_rn((uint32_t)(bs0 >> 32)),
                                              __uint2float_rn((uint32_t)(bs1 >> 32))));
          const float2 btf = fma2(make_float2(__uint2float_rn((uint32_t)bt0), __uint2float_rn((uint32_t)bt1)),
                                  splat2(0x1p-32f),
                                  make_float2(__uint2float_rn((uint32_t)(bt0 >> 32)),
                                              __uint2float_rn((uint32_t)(bt1 >> 32))));
          const float q0 = bsf.x / Gs.x, r0 = btf.x / Gt.x, q1 = bsf.y / Gs.y, r1 = btf.y / Gt.y;
          ds0 = !as0; dt0 = !at0; ds1 = v1 && !as1; dt1 = v1 && !at1;
          if (v1 && as0 && as1) {
            *reinterpret_cast<float2*>(dst.s2 + d) = make_float2(q0, q1);
          } else {
            if (as0) dst.s2[d] = q0;
            if (v1 && as1) dst.s2[d + 1] = q1;
          }
          if (v1 && at0 && at1) {
            *reinterpret_cast<float2*>(dst.t2 + d) = make_float2(r0, r1);
          } else {
            if (at0) dst.t2[d] = r0;
            if (v1 && at1) dst.t2[d + 1] = r1;
          }
        } else {
          dst.s2[d] = sa.x;
          dst.t2[d] = ta.x;
          dst.bs[d] = c0.bs;
          dst.bt[d] = c0.bt;
          if (v1) {
            dst.s2[d + 1] = sa.y;
            dst.t2[d + 1] = ta.y;
            dst.bs[d + 1] = c1.bs;
            dst.bt[d + 1] = c1.bt;
          }
        }
        // adaptive filters: the carried log-weight, 0 after a resampling, else
        // L_j - m (a trial cycle leaves it alone)
        if (ess && a.commit) {
          a.lam[d] = resamp ? (R)0 : a.ell[d] - m;
          if (v1) a.lam[d + 1] = resamp ? (R)0 : a.ell[d + 1] - m;
        }
      }
      // queue the draws that missed the squeeze (rare), a slot's two at a
      // time so that the queue never holds more than 95; the warp finishes
      // them 32 at a time
      if (__any_sync(0xffffffffu, ds0 || dt0 || ds1 || dt1)) {
        wq_push(wq, qn, ds0, GammaItem<R>{bs0, Zs.x, Us.x, (uint32_t)j0, 0u}, lane);
        wq_push(wq, qn, dt0, GammaItem<R>{bt0, Zt.x, Ut.x, (uint32_t)j0, 1u}, lane);
        wq_drain(wq, qn, 32u, lane, finish);
        wq_push(wq, qn, ds1, GammaItem<R>{bs1, Zs.y, Us.y, (uint32_t)j1, 0u}, lane);
        wq_push(wq, qn, dt1, GammaItem<R>{bt1, Zt.y, Ut.y, (uint32_t)j1, 1u}, lane);
        wq_drain(wq, qn, 32u, lane, finish);
      }
    }
  } else {
  const uint64_t pstride = (uint64_t)G * NT;
  Gathered<R> cur = gather_slot((uint64_t)rank * NT + threadIdx.x);
  for (uint64_t j0 = (uint64_t)rank * NT; j0 < n; j0 += pstride) {
    const uint64_t j = j0 + threadIdx.x;
    const Gathered<R> nxt = gather_slot(j + pstride);
    bool defer_s = false, defer_t = false;
    typename SuffT<R>::B bsn = 0, btn = 0;
    R Zs = 0, Us = 0, Zt = 0, Ut = 0;
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
      theta_draws<R>(seed, fid, t, (uint32_t)j, &Z, &Zs, &Us, &Zt, &Ut);
      const R xj = fmaR(sv, Z, mu);
      const uint64_t d = off + j;
      dst.x[d] = xj;
      if (learn) {
        const R rs = ResidObs<R>::f(y, yr, xj);
        const R rt = xj - xa;
        bsn = SuffOps<R>::add_half_square(cur.bs, rs, &fail);
        btn = SuffOps<R>::add_half_square(cur.bt, rt, &fail);
        dst.bs[d] = bsn;
        dst.bt[d] = btn;
        R Gs, Gt;
        if (gamma_mt_squeeze<R>(ds, cs, ks, Zs, Us, &Gs)) dst.s2[d] = SuffOps<R>::ig(bsn, Gs);
        else defer_s = true;
        if (gamma_mt_squeeze<R>(dt, ct, kt, Zt, Ut, &Gt)) dst.t2[d] = SuffOps<R>::ig(btn, Gt);
        else defer_t = true;
      } else {
        dst.s2[d] = sa;
        dst.t2[d] = ta;
        dst.bs[d] = cur.bs;
        dst.bt[d] = cur.bt;
      }
      // adaptive filters: the carried log-weight, 0 after a resampling, else
      // L_j - m (a trial cycle leaves it alone)
      if (ess && a.commit) a.lam[d] = resamp ? (R)0 : a.ell[d] - m;
    }
    // queue the draws that missed the squeeze (rare); the warp finishes them
    // 32 at a time
    if (__any_sync(0xffffffffu, defer_s || defer_t)) {
      wq_push(wq, qn, defer_s, GammaItem<R>{bsn, Zs, Us, (uint32_t)j, 0u}, lane);
      wq_push(wq, qn, defer_t, GammaItem<R>{btn, Zt, Ut, (uint32_t)j, 1u}, lane);
      wq_drain(wq, qn, 32u, lane, finish);
    }
    cur = nxt;
  }
  }
  wq_drain(wq, qn, 1u, lane, finish);

  // fold the cycle into the filter's log-ML (the single-filter fold's
  // butterfly over the 32 tile accumulators) and advance t
  bool any_fail = __syncthreads_or(fail);
  if (G > 1) {
    if (threadIdx.x == 0) sm.fail = any_fail ? 1u : 0u;
    group_sync(G);
  }
  if (rank == 0 && warp == 0) {
    if (G > 1) {
      const uint32_t f = (uint32_t)lane < G ? dsm_ld(&sm.fail, (uint32_t)lane) : 0u;
      any_fail = __any_sync(0xffffffffu, f != 0u);
    }
    ES acc = sm.fold[lane];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc.add(acc.shfl_xor(o));
    if (lane == 0 && a.commit) {
      const double LOG_2PI = 0x1.d67f1c864beb5p+0;
      const double md = (double)m;
      if (ess) {
        // normalised by the carried weights: log sum_i exp(lambda_i), which
        // is n after a resampling, else this cycle's sum of exp(L_i - m)
        const double S = esum_value(acc);
        const double inc = md + log(S) - log(F->slam) - 0.5 * LOG_2PI;
        F->logml = F->logml + inc;
        F->slam = resamp ? (double)n : S;
      } else {
        const double inc = md + log(esum_value(acc)) - log((double)n) - 0.5 * LOG_2PI;
        F->logml = F->logml + inc;
      }
      if (any_fail) F->err |= ERR_NUMERIC;
      F->t = t + 1;
    }
  }
  __syncthreads();
}

// The persistent cycle kernel.  With CL > 1 (launched as clusters of CL
// CTAs) each cluster first takes the large filters -- the first count[1]
// items of the size-ordered list -- one at a time and processes each with
// all its CTAs; then every CTA takes the remaining filters one at a time on
// its own.  count[0] is the number of items.
template <class R, int POS, int NT, int CL>
__global__ void __launch_bounds__(NT, NT == 256 ? (POS == POS_SYSTEMATIC && CL == 1 ? 4 : 3) : 1)
k_batch_cycle(BatchArgs<R> a) {
  __shared__ BatchSmem<R, NT> sm;
  const uint32_t count = a.count[0];
  uint32_t nbig = 0;
  if constexpr (CL > 1) {
    nbig = a.count[1] < count ? a.count[1] : count;
    const uint32_t rank = cluster_ctarank();
    while (true) {
      if (rank == 0 && threadIdx.x == 0) sm.work = atomicAdd(&a.ctr[0], 1u);
      group_sync(CL);
      if (threadIdx.x == 0) sm.wb = dsm_ld(&sm.work, 0u);
      __syncthreads();
      const uint32_t w = sm.wb;
      group_sync(CL);  // the leader's claim is read before it changes or the leader exits
      if (w >= nbig) break;
      batch_filter<R, POS, NT, (uint32_t)CL>(a, a.items[w], sm, rank);
    }
  }
  while (true) {
    if (threadIdx.x == 0) sm.wb = nbig + atomicAdd(&a.ctr[2], 1u);
    __syncthreads();
    const uint32_t w = sm.wb;
    __syncthreads();
    if (w >= count) break;
    batch_filter<R, POS, NT, 1u>(a, a.items[w], sm, 0u);
  }
  // the last CTA out resets the work counters for the next launch
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&a.ctr[1], 1u) == gridDim.x - 1) {
      a.ctr[0] = 0;
      a.ctr[1] = 0;
      a.ctr[2] = 0;
    }
  }
}

// Admission: write each admitted filter's record into its slot and
// initialise its particles (Step 0), one filter per CTA pass; the same draws
// and arithmetic as k_init.
template <class R>
__global__ void __launch_bounds__(BB) k_batch_init(BatchArgs<R> a) {
  __shared__ double s_c[7];
  const uint32_t count = *a.count;
  for (uint32_t w = blockIdx.x; w < count; w += gridDim.x) {
    const BatchFilter* rec = &a.inits[w].rec;
    BatchFilter* F = &a.F[a.inits[w].slot];
    const uint64_t off = rec->off, n = rec->n, seed = rec->seed;
    const uint32_t fid = rec->filter_id;
    const bool learn = rec->learn != 0;
    const bool ess = rec->ess_frac > 0.0;
    __syncthreads();
    if (threadIdx.x == 0) {
      *F = *rec;
      double ds, cs, ks, dt, ct, kt;
      mt_constants(rec->a_sigma, &ds, &cs, &ks);
      mt_constants(rec->a_tau, &dt, &ct, &kt);
      s_c[0] = ds; s_c[1] = cs; s_c[2] = dt; s_c[3] = ct;
      s_c[4] = sqrt(rec->x0_var);
      s_c[5] = ks; s_c[6] = kt;
    }
    __syncthreads();
    const StateV<R> st = a.st[0];
    const R x0m = (R)rec->x0_mean;
    const R sdx = (R)s_c[4];
    const auto bs0 = SuffOps<R>::from_prior(rec->b_sigma);
    const auto bt0 = SuffOps<R>::from_prior(rec->b_tau);
    bool fail = false;
    for (uint64_t j = threadIdx.x; j < n; j += BB) {
      const uint64_t g = off + j;
      const R Z = bm_normal(draw(seed, fid, 0, (uint32_t)j, P_INIT_X, 0), (R)0);
      const R p = sdx * Z;
      st.x[g] = x0m + p;
      st.bs[g] = bs0;
      st.bt[g] = bt0;
      if (ess) a.lam[g] = (R)0;  // adaptive filters start with equal weights
      if (!learn) {
        st.s2[g] = (R)rec->sigma2;
        st.t2[g] = (R)rec->tau2;
        continue;
      }
      const R Gs = gamma_mt<R>((R)s_c[0], (R)s_c[1], (R)s_c[5], seed, fid, 0, (uint32_t)j,
                               P_INIT_SIGMA, &fail);
      const R Gt = gamma_mt<R>((R)s_c[2], (R)s_c[3], (R)s_c[6], seed, fid, 0, (uint32_t)j,
                               P_INIT_TAU, &fail);
      st.s2[g] = SuffOps<R>::ig(bs0, Gs);
      st.t2[g] = SuffOps<R>::ig(bt0, Gt);
    }
    if (__syncthreads_or(fail) && threadIdx.x == 0) F->err |= ERR_NUMERIC;
  }
}

// Posterior summaries of one adaptive filter (item w of the list) by one CTA:
// the particles weighted by w_i = exp(lambda_i), in the single-filter weighted
// estimate's groups (BLOCK x EST_PER_THREAD per virtual block, consecutive
// particles per thread, binary64 per particle, shifted by particle 0), each
// group's sums by the same shuffle tree and warps in order, the group sums
// folded in group order -- so the summaries equal a standalone filter's.
template <class R>
__device__ __forceinline__ void batch_estimate_weighted(const BatchArgs<R>& a,
                                                        const BatchFilter* F, uint32_t w,
                                                        const StateV<R>& st, R c0, R c1, R c2,
                                                        double (*s_sum)[WARPS], double* s_tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr uint64_t GROUP = (uint64_t)BLOCK * EST_PER_THREAD;
  const uint64_t off = F->off, n = F->n;
  const int k = F->k;
  if (threadIdx.x < 7) s_tot[threadIdx.x] = 0.0;
  const uint64_t nblk = (n + GROUP - 1) / GROUP;
  for (uint64_t b = 0; b < nblk; ++b) {
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    const uint64_t base = b * GROUP + (uint64_t)threadIdx.x * EST_PER_THREAD;
    for (int e = 0; e < EST_PER_THREAD; ++e) {
      const uint64_t i = base + e;
      if (i < n) {
        R wr;
        (void)quant_exp<R>(a.lam[off + i], k, &wr);
        const double wd = (double)wr;
        const double dx = (double)(st.x[off + i] - c0), ds = (double)(st.s2[off + i] - c1),
                     dt = (double)(st.t2[off + i] - c2);
        acc[0] += wd;
        acc[1] += wd * dx; acc[2] += wd * (dx * dx);
        acc[3] += wd * ds; acc[4] += wd * (ds * ds);
        acc[5] += wd * dt; acc[6] += wd * (dt * dt);
      }
    }
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
      for (int ww = 0; ww < WARPS; ++ww) v += s_sum[threadIdx.x][ww];
      s_tot[threadIdx.x] += v;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double sw = s_tot[0];
    const double cs[3] = {(double)c0, (double)c1, (double)c2};
    double* o = a.est + (uint64_t)w * BATCH_EST_ROW;
    o[0] = (double)F->t;
    for (int q = 0; q < 3; ++q) {
      const double m1 = s_tot[1 + 2 * q] / sw;
      const double m2 = s_tot[2 + 2 * q] / sw;
      o[1 + 2 * q] = cs[q] + m1;
      o[2 + 2 * q] = m2 - m1 * m1;
    }
    o[7] = F->logml;
    o[8] = (double)F->err;
  }
  __syncthreads();
}

// Posterior summaries of the listed filters, one filter per CTA pass.  The
// particles are taken in the single-filter estimate's groups (BLOCK x
// EST_PER_THREAD per virtual block, consecutive particles per thread, shifted
// by particle 0), summed by the same shuffle trees, and the group sums are
// folded in its order (thread i takes groups i, i + BB, ..., then a shuffle
// tree and the warps in order), so the summaries equal a standalone filter's.
template <class R>
__global__ void __launch_bounds__(BB) k_batch_estimate(BatchArgs<R> a) {
  static_assert(BB == BLOCK, "the fold mirrors the single-filter estimate's");
  __shared__ double s_sum[7][WARPS];
  __shared__ double s_col[6][BB];
  __shared__ double s_tot[7];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t count = *a.count;
  constexpr uint64_t GROUP = (uint64_t)BLOCK * EST_PER_THREAD;
  for (uint32_t w = blockIdx.x; w < count; w += gridDim.x) {
    const BatchFilter* F = &a.F[a.items[w].slot];
    const uint64_t off = F->off, n = F->n;
    const uint32_t t = F->t;
    const StateV<R> st = (t & 1) ? a.st[1] : a.st[0];
    const R c0 = st.x[off], c1 = st.s2[off], c2 = st.t2[off];
    __syncthreads();
    if (F->ess_frac > 0.0) {
      batch_estimate_weighted<R>(a, F, w, st, c0, c1, c2, s_sum, s_tot);
      continue;
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) s_col[q][threadIdx.x] = 0.0;
    const uint64_t nblk = (n + GROUP - 1) / GROUP;
    for (uint64_t b = 0; b < nblk; ++b) {
      {
        R loc[6] = {0, 0, 0, 0, 0, 0};
        const uint64_t base = b * GROUP + (uint64_t)threadIdx.x * EST_PER_THREAD;
        for (int e = 0; e < EST_PER_THREAD; ++e) {
          const uint64_t i = base + e;
          if (i < n) est_add<R>(loc, st.x[off + i], st.s2[off + i], st.t2[off + i], c0, c1, c2);
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
        for (int ww = 0; ww < WARPS; ++ww) v += s_sum[threadIdx.x][ww];
        s_col[threadIdx.x][b % BB] += v;
      }
      __syncthreads();
    }
    {
      double v[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        v[q] = s_col[q][threadIdx.x];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
      }
      if (lane == 0) {
#pragma unroll
        for (int q = 0; q < 6; ++q) s_sum[q][warp] = v[q];
      }
    }
    __syncthreads();
    if (threadIdx.x < 6) {  // the warps in order, one quantity per thread
      double v = 0;
      for (int ww = 0; ww < WARPS; ++ww) v += s_sum[threadIdx.x][ww];
      s_tot[threadIdx.x] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const double* tot = s_tot;
      const double cs[3] = {(double)c0, (double)c1, (double)c2};
      double* o = a.est + (uint64_t)w * BATCH_EST_ROW;
      o[0] = (double)t;
      est_finish(tot, (double)n, cs, o + 1);
      o[7] = F->logml;
      o[8] = (double)F->err;
    }
  }
}

}  // namespace pfk
