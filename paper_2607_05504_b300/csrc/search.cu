// Search radius h_SI of every active particle (Sec. 4.2: N_ngb = 32 +- 5,
// Sec. 4.5: iterative search over all particles, active and inactive), and
// its neighbour list N(i) = {j != i : r_ij^2 < h_i^2}.
//
// One warp per active particle i:
//   1. Bounds.  Separations are first taken in FP32 from the FP32 copies of
//      the positions relative to the halo's centre c (within
//      2^-24 (1 + 2^-28) |x - c| of x - c; |x| below for x - c), so the true
//      separation r of a candidate with FP32 separation s lies in
//      [lo(s), hi(s)], lo(s) = s (1 - c) - e, hi(s) = s (1 + c) + e with
//      c = 2^-20 + 2^-21 and e = 2^-21 (max|x_i| + L) (generous over the
//      rounding of coordinates, differences, squares, sums).  Every test
//      "surely inside / surely outside radius H" becomes one comparison of
//      the FP32 squared separation with a threshold computed once per H.
//   2. Radius T, such that K = N_ngb + tol + 1 particles have r <= T.
//      With the context's search hint on, and when i has an h from an
//      earlier search (h_prev, kept in the h output between steps): first
//      T = G h_prev (G = 9/8), kept only when the gather below finds K
//      entries surely within it; the standard SPH practice of starting from
//      the last smoothing length, used here to size the gather only.
//      Else, when the warp's previous query in this step is i's predecessor
//      in the active list (a warp takes runs of consecutive active queries,
//      neighbours in key order and so in space) and lies in i's halo: first
//      T = G' h_pred (G' = 6/5) from that query's h, judged the same way.
//      h varies little between neighbours: on the 2^20 Hernquist halo's
//      10 %-active steps the 71st nearest particle lies within 1.2 h_pred
//      for 98 % of the queries.
//      Otherwise (the plain form carries no h between steps), from the
//      key-order window of
//      128-1024 particles around i (a launch shape, 384 by default; at least
//      K + 1 particles, so 256 where 128 would be too few): an upper bound
//      (within ~2 % above) of the K-th smallest hi.  A halo with at most K
//      particles besides i has no bound: T is infinite and the whole halo
//      (fewer than SEARCH_CAP) is gathered.  Every certified T gives the
//      same h and neighbour list (step 4 counts exactly below T).
//   3. Gather: every particle whose lower bound is <= T goes into a
//      shared-memory list (FP32 squared separation, index).  If more than
//      SEARCH_CAP qualify, T shrinks (count-verified) and the gather repeats.
//   4. Bisection on the neighbour count c(h) = #{j : r^2 < h h}, in the same
//      order of exactly rounded operations from the same start h0 as a
//      direct count: for h > T the count is at least K (above the band);
//      otherwise entries surely inside count, entries surely outside do not,
//      and the rare entries in between are decided on the exact FP64 r^2,
//      computed in the fixed order (dx dx + dy dy) + dz dz.  Doubling and
//      halving h are exact exponent steps; midpoints are one FP64 addition.
//   5. The members of N(i) are written to the neighbour list of i (when the
//      list is complete and fits); otherwise the list is marked for a direct
//      tree walk in the pair kernel.
// No result depends on the FP32 values: they only decide what is certain.
#include "traverse.cuh"

namespace sidm {

namespace {

// One block of 32 warps per SM (64 registers a thread fill the register
// file): the walks that run together on an SM are those of one range of
// consecutive queries (below), and share their leaves and boxes in L1.
constexpr int SW = 32;                // warps per block
constexpr int CLAIM_MAX_SPINS = 1 << 22;
constexpr int ST = SW * WARP;
constexpr float REL = 9.5367431640625e-07f;   // 2^-20
constexpr float ABS = 4.76837158203125e-07f;  // 2^-21
constexpr float CREL = REL + ABS;             // relative part of the bounds
constexpr float SQ = 4.76837158203125e-07f;   // 2^-21: slack on squared thresholds
// The gather walk visits leaves without stacking them, so its stack holds at
// most 31 entries for each internal level below the root except the lowest,
// plus one: 31 * 4 + 1 = 125 for the 6 levels of n < 2^30.  128 entries (2 KB
// per block) beside the candidate lists keep a block's shared memory at
// 18 KB.
constexpr int WALK_STACK = 128;
#ifndef LIST_REGS
#define LIST_REGS 4                            // candidates per lane held in registers
#endif
#ifndef SEARCH_HINT_GROW
#define SEARCH_HINT_GROW 1.125f                // first gather radius / h of the last search
#endif
#ifndef SEARCH_RUN_GROW
#define SEARCH_RUN_GROW 1.2f                   // first gather radius / h of the run's last query
#endif
#ifndef SEARCH_LEAF_BATCH
#define SEARCH_LEAF_BATCH 2                    // leaves per L2 round trip in the gather walk
#endif

struct SearchArgs {
  Sorted so;
  Forest f;
  int64_t n;
  const int32_t* act_list;
  double box;
  int n_ngb, tol;
  double fixed_h;
  int kernel;            // SIDM_KERNEL_*: normalisation bound stored with h
  int split;             // 1: FP32 counts and lists, no FP64 re-tests
  double* h_user;
  int32_t* nb_list;     // [n_act][nb_stride]
  int32_t* nb_count;    // [n_act]: count, or -1 (walk the tree)
  int nb_stride;
  int range;             // runs per range a block claims
  int run;               // consecutive queries a warp takes in a row (a run)
  int all;               // 1: every particle is a query (overlap estimator), s = query index
  int hint;              // 1: the first gather radius from the particle's last h
  DevStats* st;
  int* work;
};

__device__ __forceinline__ int warp_sum(int v) {
  return __reduce_add_sync(0xffffffffu, v);   // one warp reduction instruction (sm_80+)
}

// FP32 squared-separation thresholds for a radius H given by its FP32
// bounds Hlo <= H <= Hhi:  s2 < in2 -> r < H surely;  s2 >= out2 -> r >= H surely.
// Directed-rounding multiplies only (native; directed divisions and roots
// are not): 1/(1 + c) > 1 - c and 1/(1 - c) < 1 + 2c bound the divisions
// from the safe side; SQ covers the rounding of s2 itself.
constexpr float ONE_M_CREL = 1.0f - CREL;         // exact in FP32
constexpr float ONE_P_2CREL = 1.0f + 2.0f * CREL;  // exact in FP32
constexpr float ULP1 = 1.1920928955078125e-07f;    // 2^-23
__device__ __forceinline__ float thr_in2(float Hlo, float eq) {
  const float x = __fmul_rd(__fsub_rd(Hlo, eq), ONE_M_CREL);
  return x > 0.0f ? __fmul_rd(__fmul_rd(x, x), 1.0f - SQ) : 0.0f;
}
__device__ __forceinline__ float thr_out2(float Hhi, float eq) {
  const float x = __fmul_ru(__fadd_ru(Hhi, eq), ONE_P_2CREL);
  return __fmul_ru(__fmul_ru(x, x), 1.0f + SQ);
}
// upper bound hi(s) of the true separation for FP32 squared separation s2
// (sqrtf rounds to nearest: within 2^-24 of the root; 2^-23 covers it)
__device__ __forceinline__ float upper_from_s2(float s2, float eq) {
  const float r = __fmul_ru(sqrtf(s2), 1.0f + ULP1);
  return __fmul_ru(__fadd_ru(__fmul_ru(r, 1.0f + CREL), eq), 1.0f + SQ);
}

// FP32 bounds of a positive double by bit manipulation (exact, no FP64 ops)
__device__ __forceinline__ void float_bounds(double h, float* lo, float* hi) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(h);
  const int e = (int)((b >> 52) & 0x7FF) - 1023;
  if (e < -125 || e > 126) {
    *lo = hw_f32_rd(h);
    *hi = hw_f32_ru(h);
    return;
  }
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  const unsigned int fb = ((unsigned int)(e + 127) << 23) | (unsigned int)(m >> 29);
  *lo = __uint_as_float(fb);
  *hi = (m & 0x1FFFFFFFull) ? __uint_as_float(fb + 1u) : *lo;
}

// exact 2 h and h / 2 (exponent steps; FP64 multiply where that is not exact)
__device__ __forceinline__ double twice(double h) {
  const long long b = __double_as_longlong(h);
  const int ef = (int)((b >> 52) & 0x7FF);
  if (ef >= 1 && ef < 2046) return __longlong_as_double(b + (1ll << 52));
  return hw_mul(h, 2.0);
}
__device__ __forceinline__ double half_of(double h) {
  const long long b = __double_as_longlong(h);
  const int ef = (int)((b >> 52) & 0x7FF);
  if (ef > 1 && ef < 2047) return __longlong_as_double(b - (1ll << 52));
  return hw_mul(h, 0.5);
}

// Radius from the key-order window [w0, w0 + W) around s (warp-collective):
// an upper bound (within ~2 % above) of the K-th smallest separation from s
// over the window's particles.  Out of line: it is the rare path once most
// queries start from their last h, and its registers stay out of the walk's.
template <bool PERIODIC, int NWIN>
__device__ __noinline__ float window_radius(const float4* __restrict__ f, int64_t s, int64_t w0,
                                            int64_t W, float4 fi, float boxf, int K, float eq) {
  const int lane = threadIdx.x & 31;
  float wv[NWIN];
  float a1 = INFINITY, a2 = INFINITY, a3 = INFINITY;   // the lane's three smallest
#pragma unroll
  for (int k = 0; k < NWIN; ++k) {
    wv[k] = INFINITY;
    const int64_t j = w0 + k * 32 + lane;
    if (j < w0 + W && j != s) {
      const float v = sep2f<PERIODIC>(fi, f[j], boxf);
      wv[k] = v;
      a3 = fminf(a3, fmaxf(a2, v));
      a2 = fminf(a2, fmaxf(a1, v));
      a1 = fminf(a1, v);
    }
  }
  // Separations are non-negative, so their bit patterns order as integers.
  // Bracket of the K-th smallest t: with m = ceil(K / 32) <= 3 and every
  // lane holding m values, each lane has m values at or below its m-th
  // smallest a_m, so #{wv <= max over lanes of a_m} >= 32 m >= K, and at most
  // m - 1 values below its a_m, so #{wv < min over lanes of a_m} <= 32 (m - 1)
  // < K.  Otherwise the window's extremes bracket t.
  const float am = K <= 32 ? a1 : (K <= 64 ? a2 : a3);
  uint32_t blo, bhi;
  const uint32_t am_hi = __reduce_max_sync(0xffffffffu, __float_as_uint(am));
  if (K <= 96 && am_hi < __float_as_uint(INFINITY)) {
    blo = __reduce_min_sync(0xffffffffu, __float_as_uint(am));
    bhi = am_hi;
  } else {
    float vmax = 0.0f;
#pragma unroll
    for (int k = 0; k < NWIN; ++k) vmax = wv[k] < INFINITY ? fmaxf(vmax, wv[k]) : vmax;
    blo = __reduce_min_sync(0xffffffffu, __float_as_uint(a1));
    bhi = __reduce_max_sync(0xffffffffu, __float_as_uint(vmax));
  }
  // bit-pattern bisection for t with #{wv <= t} >= K; stop within 2^-6
  if (blo > 0) --blo;
  for (int it = 0; it < 32 && bhi - blo > (1u << 17); ++it) {
    const uint32_t mid = blo + ((bhi - blo) >> 1);
    const float tm = __uint_as_float(mid);
    int c = 0;
#pragma unroll
    for (int k = 0; k < NWIN; ++k) c += wv[k] <= tm ? 1 : 0;
    c = warp_sum(c);
    if (c >= K) bhi = mid; else blo = mid;
  }
  return upper_from_s2(__uint_as_float(bhi), eq);
}

// NWIN: the key-order window of the search radius is 32 NWIN particles.
// The block's next run (a run: `run` consecutive queries, taken in a row by
// one warp): ranges of L consecutive runs (key order, so neighbouring in
// space) are claimed a range at a time by the block, and its warps take the
// runs of the current range one by one, so that the walks
// running together on an SM share their leaves in L1 (on the 2^20 halo the
// search took 0.507 ms per step this way against 0.550 with each warp of
// 4-warp blocks claiming its own next query from the global counter).
// s_claim = (range << 32) | next place in it; s_next = the range after it,
// claimed ahead (-1 while that claim is in flight).  The warp that takes
// the place just past the range's end installs the next range; warps that
// come after it wait for the new range.  Called by lane 0.
__device__ __forceinline__ int64_t claim_in_block(unsigned long long* s_claim, int* s_next,
                                                  int* work, int64_t n_act, int64_t L,
                                                  uint32_t* status) {
  const int64_t nseg = (n_act + L - 1) / L;
  int budget = CLAIM_MAX_SPINS;   // every wait below draws on it
  while (budget-- > 0) {
    const unsigned long long old = atomicAdd(s_claim, 1ull);
    const int64_t seg = (int64_t)(old >> 32);
    const int64_t pos = (int64_t)(uint32_t)old;
    if (seg >= nseg) return n_act;
    const int64_t first = seg * L;
    const int64_t len = n_act - first < L ? n_act - first : L;
    if (pos < len) return first + pos;
    if (pos == len) {
      int nxt = atomicAdd(s_next, 0);
      while (nxt < 0 && budget-- > 0) nxt = atomicAdd(s_next, 0);
      if (nxt < 0) break;
      atomicExch(s_next, -1);
      atomicExch(s_claim, (unsigned long long)nxt << 32);
      atomicExch(s_next, nxt < nseg ? atomicAdd(work, 1) : nxt);
      continue;
    }
    while (budget-- > 0 && (int64_t)(atomicAdd(s_claim, 0ull) >> 32) == seg) {
    }
  }
  *status |= ST_ERR_CLAIM;
  return n_act;
}

template <bool PERIODIC, int NWIN>
__global__ void __launch_bounds__(ST, 1) search_kernel(SearchArgs A) {
  // per warp: its candidate list and walk stack (dynamic shared memory,
  // SEARCH_SMEM bytes)
  extern __shared__ __align__(16) unsigned char s_dyn[];
  float(*s_r2)[SEARCH_CAP] = reinterpret_cast<float(*)[SEARCH_CAP]>(s_dyn);
  int32_t(*s_j)[SEARCH_CAP] =
      reinterpret_cast<int32_t(*)[SEARCH_CAP]>(s_dyn + (size_t)SW * SEARCH_CAP * 4);
  int(*s_stack)[WALK_STACK] =
      reinterpret_cast<int(*)[WALK_STACK]>(s_dyn + (size_t)SW * SEARCH_CAP * 8);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  float* lst_r2 = s_r2[warp];
  int32_t* lst_j = s_j[warp];
  int* stack = s_stack[warp];
  const Sorted& so = A.so;
  const int64_t n_act = A.all ? A.n : (int64_t)A.st->n_active;
  const double box = A.box, half = 0.5 * A.box;
  const float boxf = (float)A.box;
  const int K = A.n_ngb + A.tol + 1;
  const int lo_band = A.n_ngb - A.tol, hi_band = A.n_ngb + A.tol;
  uint32_t status = 0;
  int nonconv = 0;

  __shared__ unsigned long long s_claim;
  __shared__ int s_next;
  __shared__ long long s_qnext[SW], s_qend[SW];
  __shared__ float s_hpred[SW];
  __shared__ int s_halopred[SW];
  if (threadIdx.x == 0) {
    const int a = atomicAdd(A.work, 2);   // the block's first range and the one after
    s_claim = (unsigned long long)a << 32;
    s_next = a + 1;
  }
  __syncthreads();
  // Runs of A.run consecutive queries are the unit of the claims; lane 0
  // keeps the warp's place in its run (next query, end) and the run's
  // previous h (an FP32 upper bound; 0: none yet) and halo in shared memory,
  // so that the loop below carries no state from one query to the next.
  const int64_t n_runs = (n_act + A.run - 1) / A.run;
  if (lane == 0) {
    s_qnext[warp] = 0;
    s_qend[warp] = 0;
  }
  for (;;) {
    int64_t qc = 0;
    if (lane == 0) {
      if (s_qnext[warp] < s_qend[warp]) {
        qc = s_qnext[warp]++;
      } else {
        const int64_t run = claim_in_block(&s_claim, &s_next, A.work, n_runs, A.range, &status);
        qc = run < n_runs ? run * A.run : n_act;
        s_qnext[warp] = qc + 1;
        s_qend[warp] = qc + A.run < n_act ? qc + A.run : n_act;
        s_hpred[warp] = 0.0f;
        s_halopred[warp] = -1;
      }
    }
    __syncwarp();
    const int64_t qi = __shfl_sync(0xffffffffu, qc, 0);
    if (qi >= n_act) break;
    const int64_t s = A.all ? qi : (int64_t)A.act_list[qi];
    const int halo_s = so.halo[s];
    const Halo& H = A.f.halos[halo_s];
    const int64_t hs = H.start, hn = H.n;   // the query's halo: [hs, hs + hn)
    const float4* hpos = so.f + hs;         // its FP32 positions
    const int sl = (int)(s - hs);           // the query's halo-local index
    const float4 fi = so.f[s];
    const float eq = ABS * (fmaxf(fmaxf(fabsf(fi.x), fabsf(fi.y)), fabsf(fi.z)) + boxf);
    double h;
    int len = 0;
    float T0 = INFINITY;  // radius when no bound is known (fixed h: h itself)
    // the key-order window bounds T only when it holds K particles besides i
    const int64_t W = (int64_t)NWIN * 32 < hn ? (int64_t)NWIN * 32 : hn;
    const bool window_bound = !(A.fixed_h > 0.0) && W - 1 >= K;
    if (A.fixed_h > 0.0) {
      h = A.fixed_h;
      float hl, hu;
      float_bounds(h, &hl, &hu);
      T0 = hu;
    }
    // h of the particle's last search (0 before its first): the first
    // gather tries G h_prev, kept only if K entries are surely within it
    double hp = 0.0;
    if (SEARCH_HINT_GROW > 0.0f && A.hint && window_bound) hp = A.h_user[so.orig[s]];
    bool use_hint = hp > 0.0 && hp < INFINITY;
    float T = T0;         // every j with r <= T (and more) is in the list
    if (use_hint) {
      float hpl, hpu;
      float_bounds(hp, &hpl, &hpu);
      T = __fmul_ru(hpu, SEARCH_HINT_GROW);
    }
    // else the h of the run's previous query, a neighbour in space (lane 0
    // records this query's halo now and its h at the end)
    const float h_pred = s_hpred[warp];
    if (!use_hint && window_bound && s_halopred[warp] == halo_s && h_pred > 0.0f &&
        h_pred < INFINITY) {
      use_hint = true;
      T = __fmul_ru(h_pred, SEARCH_RUN_GROW);
    }
    __syncwarp();
    if (lane == 0) s_halopred[warp] = halo_s;

    // ---- 2-3. radius T and gather of every j whose lower bound is <= T
    bool t_bound = false;  // K particles besides i lie within T
    bool complete = true;
    for (;;) {
      if (use_hint) {
        // T: the hinted radius, set above
      } else if (window_bound) {
        int64_t w0 = s - W / 2;
        if (w0 > hs + hn - W) w0 = hs + hn - W;
        if (w0 < hs) w0 = hs;
        T = window_radius<PERIODIC, NWIN>(so.f, s, w0, W, fi, boxf, K, eq);
      } else {
        T = T0;
      }
      bool ok = true;
      for (int attempt = 0;; ++attempt) {
        len = 0;
        const float g2 = T < INFINITY ? thr_out2(T * (1.0f + REL), eq) : INFINITY;
        const float rad = (T + 2.0f * eq) * (1.0f + 4.0f * REL);
        const float rad2 = rad < INFINITY ? rad * rad : INFINITY;
        ok = traverse<PERIODIC, false, SEARCH_LEAF_BATCH, WALK_STACK>(
            A.f, H, hpos, fi, rad2, boxf, stack,
            [&](const int* kk, const bool* valid, const float4* pj, const bool* on) {
          // every slot's separation first (independent work), then the appends
          float s2[SEARCH_LEAF_BATCH];
          bool keep[SEARCH_LEAF_BATCH];
#pragma unroll
          for (int b = 0; b < SEARCH_LEAF_BATCH; ++b) {
            s2[b] = sep2f<PERIODIC>(fi, pj[b], boxf);
            keep[b] = valid[b] && kk[b] != sl && s2[b] < g2;
          }
#pragma unroll
          for (int b = 0; b < SEARCH_LEAF_BATCH; ++b) {
            if (!on[b]) break;
            const uint32_t m = __ballot_sync(0xffffffffu, keep[b]);
            if (keep[b]) {
              const int at = len + __popc(m & lt);
              if (at < SEARCH_CAP) {
                lst_r2[at] = s2[b];
                lst_j[at] = (int32_t)(hs + kk[b]);
              }
            }
            len += __popc(m);
          }
        });
        __syncwarp();
        // the hinted radius is judged once, below
        if (use_hint) break;
        if (!ok) { status |= ST_ERR_STACK; complete = false; break; }
        if (len <= SEARCH_CAP) break;
        // too many candidates.  With a fixed h the pair kernel walks the tree
        // itself; otherwise shrink T, keeping a new T only once at least K
        // particles are certainly within it.
        if (A.fixed_h > 0.0) {
          complete = false;
          len = SEARCH_CAP;
          break;
        }
        if (attempt >= RADIUS_MAX_ITERS) {
          status |= ST_ERR_SEARCH_CAP;
          complete = false;
          len = SEARCH_CAP;
          break;
        }
        float Tn = T * cbrtf(0.5f * (float)SEARCH_CAP / (float)len);
        bool verified = false;
        for (int inner = 0; inner < RADIUS_MAX_ITERS; ++inner) {
          const float in2 = thr_in2(Tn, eq);
          const float radn = (Tn + 2.0f * eq) * (1.0f + 4.0f * REL);
          int c = 0;
          const bool ok2 = traverse<PERIODIC, false, SEARCH_LEAF_BATCH, WALK_STACK>(
              A.f, H, hpos, fi, radn * radn, boxf, stack,
              [&](const int* kk, const bool* valid, const float4* pj, const bool* on) {
#pragma unroll
            for (int b = 0; b < SEARCH_LEAF_BATCH; ++b) {
              const bool in = valid[b] && kk[b] != sl && sep2f<PERIODIC>(fi, pj[b], boxf) < in2;
              c += __popc(__ballot_sync(0xffffffffu, in));   // invalid slots add 0
            }
          });
          if (!ok2) { status |= ST_ERR_STACK; break; }
          if (c >= K) { verified = true; break; }
          Tn = sqrtf(Tn * T);   // too small: move towards the valid T
        }
        if (!verified) {
          status |= ST_ERR_RADIUS;
          complete = false;
          len = SEARCH_CAP;
          break;
        }
        T = Tn;
      }
      if (use_hint) {
        // kept when the whole list fits and K entries are surely within T
        use_hint = false;
        if (ok && len <= SEARCH_CAP) {
          const float in2 = thr_in2(T, eq);
          int c = 0;
          for (int k = lane; k < len; k += 32) c += lst_r2[k] < in2 ? 1 : 0;
          if (warp_sum(c) >= K) { t_bound = true; break; }
        }
        continue;   // the window's radius instead
      }
      t_bound = window_bound;
      break;
    }

    // ---- 4. bisection on the exact neighbour count
    const double xi = so.x[s], yi = so.y[s], zi = so.z[s];
    auto exact_r2 = [&](int k) {
      const int64_t j = lst_j[k];
      return sep2(xi, yi, zi, so.x[j], so.y[j], so.z[j], box, half);
    };
    // #{r^2 < h h} over the list (exact); requires h <= T (1 + 2^-22)
    // FP32-split form: the counts compare FP32 r^2 with the FP32 h^2 directly
    auto thresholds = [&](double hv, float hl, float hu, float* in2, float* out2) {
      if (A.split) {
        const float hf = (float)hv;
        *in2 = *out2 = hf * hf;
      } else {
        *in2 = thr_in2(hl, eq);
        *out2 = thr_out2(hu, eq);
      }
    };
    // a short list (the usual case) is held in registers for the bisection
    const bool in_regs = len <= LIST_REGS * 32;
    float rv[LIST_REGS];
#pragma unroll
    for (int i = 0; i < LIST_REGS; ++i) {
      const int k = lane + 32 * i;
      rv[i] = (in_regs && k < len) ? lst_r2[k] : INFINITY;
    }
    auto count_below = [&](double hv, float hl, float hu) {
      float in2, out2;
      thresholds(hv, hl, hu, &in2, &out2);
      int c = 0;
      bool amb = false;
      if (in_regs) {
#pragma unroll
        for (int i = 0; i < LIST_REGS; ++i) {
          c += rv[i] < in2 ? 1 : 0;
          amb |= (rv[i] >= in2) && (rv[i] < out2);
        }
      } else {
        for (int k = lane; k < len; k += 32) {
          const float v = lst_r2[k];
          c += v < in2 ? 1 : 0;
          amb |= (v >= in2) && (v < out2);
        }
      }
      if (__any_sync(0xffffffffu, amb)) {
        const double hh = hv * hv;
        for (int k = lane; k < len; k += 32) {
          const float v = lst_r2[k];
          if (v >= in2 && v < out2) c += exact_r2(k) < hh ? 1 : 0;
        }
      }
      return warp_sum(c);
    };
    if (!(A.fixed_h > 0.0)) {
      h = H.h0;
      double blo = 0.0, bhi = 0.0;
      bool have_hi = false, conv = false;
      // h > T means c(h) >= K: K particles lie within T.  h and T are
      // positive, so their bit patterns compare as integers.
      const long long t_bits =
          t_bound ? __double_as_longlong((double)T) : 0x7FFFFFFFFFFFFFFFll;
      int it = 0;
      // While h > T and no lower end is known, each step sets bhi = h and
      // halves h (the midpoint of 0 and h): the opening run from h0 down to
      // the first h0 2^-k <= T follows from the exponents.  Taken at once
      // when every halving is an exact exponent step, as in the loop.
      {
        const long long hb = __double_as_longlong(h);
        if (hb > t_bits) {
          int k = (int)((hb >> 52) & 0x7FF) - (int)((t_bits >> 52) & 0x7FF);
          long long hk = hb - ((long long)k << 52);   // h0 2^-k: T's exponent
          if (hk > t_bits) {
            ++k;
            hk -= 1ll << 52;
          }
          if (((hk >> 52) & 0x7FF) >= 1 && k < BISECT_MAX_EVALS) {
            bhi = __longlong_as_double(hk + (1ll << 52));
            have_hi = true;
            h = __longlong_as_double(hk);
            it = k;
          }
        }
      }
      for (; it < BISECT_MAX_EVALS; ++it) {
        int c;
        if (__double_as_longlong(h) > t_bits) {
          c = hi_band + 1;
        } else {
          float hl, hu;
          float_bounds(h, &hl, &hu);
          c = count_below(h, hl, hu);
        }
        if (c >= lo_band && c <= hi_band) { conv = true; break; }
        if (c < lo_band) {
          blo = h;
          h = have_hi ? half_of(blo + bhi) : twice(h);
        } else {
          bhi = h;
          have_hi = true;
          h = half_of(blo + bhi);
        }
      }
      if (!conv) ++nonconv;
    }

    // ---- 5. neighbour list
    float hl, hu;
    float_bounds(h, &hl, &hu);
    int* out = A.nb_list + qi * (int64_t)A.nb_stride;
    int cnt = -1;
    const bool list_covers = complete && (!t_bound || !(hl > T));
    if (list_covers) {
      float in2, out2;
      thresholds(h, hl, hu, &in2, &out2);
      cnt = 0;
      for (int k0 = 0; k0 < len; k0 += 32) {
        const int k = k0 + lane;
        bool in = false;
        if (k < len) {
          const float v = lst_r2[k];
          if (v < in2) in = true;
          else if (v < out2) in = hw_within(so.x, so.y, so.z, s, lst_j[k], box, h);
        }
        const uint32_t m = __ballot_sync(0xffffffffu, in);
        if (in) {
          const int at = cnt + __popc(m & lt);
          if (at < A.nb_stride) out[at] = lst_j[k];
        }
        cnt += __popc(m);
      }
      if (cnt > A.nb_stride) cnt = -1;
    }
    if (lane == 0) {
      A.nb_count[qi] = cnt;
      so.h[s] = h;
      // bounds used by the pair kernel: 1/h from below, K/h^3 from above
      // K = 8/pi or 3/(4 pi) (the FP64 constants) rounded up to FP32
      const float knorm_up = A.kernel == SIDM_KERNEL_TOPHAT ? 0x1.e8ec8cp-3f : 0x1.45f308p+1f;
      // (__frcp_rn is within 2^-24 of the reciprocal; 2^-23 covers it)
      const float h3 = __fmul_rd(__fmul_rd(hl, hl), hl);
      so.hb[s] = make_float4(hl, hu, __fmul_rd(__frcp_rn(hu), 1.0f - ULP1),
                             __fmul_ru(__fmul_ru(knorm_up, __frcp_rn(h3)), 1.0f + ULP1));
      A.h_user[so.orig[s]] = h;
      s_hpred[warp] = hu;
    }
    __syncwarp();
  }
  if (lane == 0) {
    if (nonconv) {
      atomicAdd(&A.st->n_nonconv, (unsigned long long)nonconv);
      status |= ST_H_NONCONV;
    }
    if (status) atomicOr(&A.st->status, status);
  }
}

}  // namespace

constexpr size_t SEARCH_SMEM = (size_t)SW * (SEARCH_CAP * 8 + WALK_STACK * 4);   // 131 KB
template <bool PERIODIC, int NWIN>
void launch_one(const SearchArgs& a, unsigned blocks, cudaStream_t s) {
  // above the default 48 KB of dynamic shared memory (set for the current
  // device at every launch, so that every device of the process has it)
  cudaFuncSetAttribute(search_kernel<PERIODIC, NWIN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)SEARCH_SMEM);
  search_kernel<PERIODIC, NWIN><<<blocks, ST, SEARCH_SMEM, s>>>(a);
}

template <bool PERIODIC>
void launch_search_window(const SearchArgs& a, int window, unsigned blocks, cudaStream_t s) {
  if (window <= 128) launch_one<PERIODIC, 4>(a, blocks, s);
  else if (window <= 256) launch_one<PERIODIC, 8>(a, blocks, s);
  else if (window <= 384) launch_one<PERIODIC, 12>(a, blocks, s);
  else if (window <= 512) launch_one<PERIODIC, 16>(a, blocks, s);
  else if (window <= 768) launch_one<PERIODIC, 24>(a, blocks, s);
  else launch_one<PERIODIC, 32>(a, blocks, s);
}

int launch_search(const Sorted& so, const Forest& f, int64_t n, const int32_t* act_list,
                  double box, int n_ngb, int tol, double fixed_h, int kernel, int split,
                  double* h_user, int32_t* nb_list, int32_t* nb_count, int nb_stride,
                  DevStats* st, int* work, int sms, const LaunchTuning& t, int all,
                  int hint, cudaStream_t s) {
  if (n <= 0) return 0;
  const int range = 32 * t.search_chunk;   // runs per range
  const int run = t.search_run;
  SearchArgs a{so, f, n, act_list, box, n_ngb, tol, fixed_h, kernel, split, h_user,
               nb_list, nb_count, nb_stride, range, run, all, hint, st, work};
  // one block per SM is resident; more blocks per SM start as those finish
  int64_t blocks = (int64_t)sms * t.search_blocks_per_sm;
  const int64_t need = (n + (int64_t)range * run - 1) / ((int64_t)range * run);
  if (blocks > need) blocks = need;
  // the window must hold K = N_ngb + tol + 1 particles besides the query for
  // its radius to bound the K-th neighbour (K <= 255, so 256 always does)
  int window = t.search_window;
  if (window - 1 < n_ngb + tol + 1 && window < 256) window = 256;
  if (box > 0.0) launch_search_window<true>(a, window, (unsigned)blocks, s);
  else launch_search_window<false>(a, window, (unsigned)blocks, s);
  return 1;
}

}  // namespace sidm
