// Application of the accepted pairs (Sec. 4.1 kick, Sec. 4.4 multiple
// scatters with immediate updates).
//
// The canonical result is the sequential pass over the accepted pairs in
// ascending (ord, a, b) order, each kick reading the velocities left by the
// earlier ones.  The resolver reaches the same result in rounds: in a round
// every unapplied pair that precedes all other unapplied pairs at both of its
// particles is applied.  Such pairs share no particle, and every particle
// still meets its pairs in key order, so the velocities equal those of the
// sequential pass bit for bit.  (This is the single-device counterpart of the
// paper's rule that no particle is modified concurrently, Sec. 4.5.)
//
// Direction: Marsaglia (1972) -- x1, x2 uniform in (-1, 1) from the Philox
// streams 1, 2, ... of the pair, accepted when 0 < s = x1^2 + x2^2 < 1, then
// e = (2 x1 sqrt(1-s), 2 x2 sqrt(1-s), 1 - 2 s).
// Kick: v_com = (m_a v_a + m_b v_b)/M, g = |v_a - v_b|,
//       v_a' = v_com + (m_b g / M) e,  v_b' = v_com - (m_a g / M) e.
#include "sidm_internal.cuh"

namespace sidm {

namespace {

constexpr int RT = 1024;

__device__ __forceinline__ bool key_less(const PairRec& x, const PairRec& y) {
  if (x.ord != y.ord) return x.ord < y.ord;
  if (x.a != y.a) return x.a < y.a;
  return x.b < y.b;
}

// true if no other unapplied pair at particle e precedes pair p.  Records
// with equal keys (a caller may pass the same pair twice) precede one
// another in record order, so they are applied one after the other, in the
// order given, and never in the same round.
__device__ bool first_at(int64_t p, const PairRec& rp, int32_t e, const int32_t* head,
                         const int32_t* next, const PairRec* pairs, const volatile uint8_t* flags) {
  for (int32_t slot = head[e]; slot >= 0; slot = next[slot]) {
    const int64_t q = slot >> 1;
    if (q == p || (flags[q] & 1)) continue;
    const PairRec rq = pairs[q];
    if (key_less(rq, rp) || (q < p && !key_less(rp, rq))) return false;
  }
  return true;
}

// The mass terms of a pair, fixed before its turn: M = m_a + m_b and, where
// M lies in [2^-500, 2^500), its correctly rounded reciprocal y = 1/M.
struct KickTerms {
  double ma, mb, M, y, eps;
  bool rcp;      // y is set, and divisions by M start from it
  bool elastic;  // eps == 1: the product with eps is the identity
};

// biased binary64 exponent in [523, 1522], i.e. |v| in [2^-500, 2^500)
// (positive only when `positive`)
__device__ __forceinline__ bool in_rcp_range(double v, bool positive) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned e = positive ? (unsigned)(b >> 52) : (unsigned)(b >> 52) & 0x7FFu;
  return e - 523u < 1000u;
}

__device__ __forceinline__ KickTerms kick_terms(double ma, double mb, double eps) {
  KickTerms t;
  t.ma = ma;
  t.mb = mb;
  t.M = ma + mb;
  t.eps = eps;
  t.rcp = in_rcp_range(t.M, true);
  t.y = t.rcp ? 1.0 / t.M : 0.0;
  t.elastic = eps == 1.0;
  return t;
}

// x / M, correctly rounded, with the division replaced where it is safe.
// From y = RN(1/M), Markstein's correction (P. Markstein, IBM J. Res. Dev.
// 34 (1990) 111) gives q = RN(q0 + RN(x - M q0) y), q0 = RN(x y), by two
// FMAs.  q is then checked, not trusted: the FMA remainder r = RN(x - M q)
// is M (x/M - q) rounded once, and q is kept when |r| < M s/2, s being the
// spacing of the doubles next to q on the side of x/M (ulp(q), or half of
// it toward zero from a power of two).  M s/2 is M times a power of two,
// a double, and rounding is monotone, so a kept q lies within half a
// spacing of x/M: it is the correctly rounded quotient (a quotient of two
// doubles is never a midpoint).  Otherwise, or when x or M lies outside
// [2^-500, 2^500) (where a step could under- or overflow), the division.
__device__ __forceinline__ double div_m(double x, const KickTerms& t) {
  if (t.rcp && in_rcp_range(x, false)) {
    const double q0 = __dmul_rn(x, t.y);
    const double q = __fma_rn(__fma_rn(-t.M, q0, x), t.y, q0);
    const double r = __fma_rn(-t.M, q, x);
    const unsigned long long qb = (unsigned long long)__double_as_longlong(q);
    const unsigned long long rb = (unsigned long long)__double_as_longlong(r);
    const bool toward0 = ((qb ^ rb) >> 63) != 0;               // M > 0: sign(r) = sign(x/M - q)
    const bool pow2 = (qb & 0xFFFFFFFFFFFFFull) == 0;
    // M s/2 = M 2^(E(q) - 53) (one less toward zero from a power of two):
    // an exponent shift of M, in range since M q ~ x
    const long long k = (long long)((qb >> 52) & 0x7FFu) - 1076 - ((toward0 && pow2) ? 1 : 0);
    const unsigned long long half_gap =
        (unsigned long long)__double_as_longlong(t.M) + ((unsigned long long)k << 52);
    if ((rb & 0x7FFFFFFFFFFFFFFFull) < half_gap) return q;
  }
  return x / t.M;
}

// The kick of Eqs. 12-13 in the operation order
//   v_com = ((m_a v_a) + (m_b v_b)) / M,  g = sqrt((dx dx + dy dy) + dz dz) eps,
//   v_a' = v_com + ((m_b g) / M) e,  v_b' = v_com - ((m_a g) / M) e,
// with M = m_a + m_b and eps the outgoing / incoming relative speed (1:
// elastic; the product with 1 is exact and skipped); every operation rounds
// once.
__device__ __forceinline__ void kick_values(const KickTerms& t, const double* e, double* a,
                                            double* b) {
  double c[3], d[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    c[k] = div_m((t.ma * a[k]) + (t.mb * b[k]), t);
    d[k] = a[k] - b[k];
  }
  double g = sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
  if (!t.elastic) g = g * t.eps;
  const double fa = div_m(t.mb * g, t), fb = div_m(t.ma * g, t);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    a[k] = c[k] + fa * e[k];
    b[k] = c[k] - fb * e[k];
  }
}

__device__ void kick(const PairRec& r, double* vel, const double* mass, uint32_t k0, uint32_t k1,
                     uint32_t step, double eps, unsigned* dirfail) {
  double e0 = 0.0, e1 = 0.0, e2 = 1.0;
  bool found = false;
  for (uint32_t t = 0; t < DIRECTION_TRIES && !found; ++t) {
    const U4 w = philox10(k0, k1, step, 1u + t, r.a, r.b);
    const double x1 = 2.0 * unit53(w.x, w.y) - 1.0;
    const double x2 = 2.0 * unit53(w.z, w.w) - 1.0;
    const double s = x1 * x1 + x2 * x2;
    if (s > 0.0 && s < 1.0) {
      const double k = 2.0 * sqrt(1.0 - s);
      e0 = x1 * k;
      e1 = x2 * k;
      e2 = 1.0 - 2.0 * s;
      found = true;
    }
  }
  if (!found) atomicAdd(dirfail, 1u);
  double* va = vel + 3 * (int64_t)r.ia;
  double* vb = vel + 3 * (int64_t)r.ib;
  const KickTerms kt = kick_terms(mass[r.ia], mass[r.ib], eps);
  const double e[3] = {e0, e1, e2};
  double a[3] = {va[0], va[1], va[2]}, b[3] = {vb[0], vb[1], vb[2]};
  kick_values(kt, e, a, b);
  va[0] = a[0];
  va[1] = a[1];
  va[2] = a[2];
  vb[0] = b[0];
  vb[1] = b[1];
  vb[2] = b[2];
}

__global__ void __launch_bounds__(RT) resolve_kernel(const PairRec* __restrict__ pairs,
                                                     int64_t cap, double* vel,
                                                     const double* __restrict__ mass,
                                                     int32_t* head, int32_t* next, uint8_t* flags,
                                                     int32_t* mult, uint32_t k0, uint32_t k1,
                                                     uint32_t step, DevStats* st) {
  __shared__ unsigned s_dirfail;
  __shared__ int s_max;
  const int t = threadIdx.x;
  if (t == 0) { s_dirfail = 0; s_max = 0; }
  const unsigned long long nall = st->n_acc;
  if (nall > (unsigned long long)cap) {
    if (t == 0) atomicOr(&st->status, (unsigned)ST_ERR_PAIR_OVERFLOW);
    return;
  }
  const int64_t na = (int64_t)nall;
  for (int64_t p = t; p < na; p += RT) {
    flags[p] = 0;
    const int32_t ea = pairs[p].ia, eb = pairs[p].ib;
    next[2 * p] = atomicExch(&head[ea], (int32_t)(2 * p));
    next[2 * p + 1] = atomicExch(&head[eb], (int32_t)(2 * p + 1));
    atomicAdd(&mult[ea], 1);
    atomicAdd(&mult[eb], 1);
  }
  __syncthreads();
  int rounds = 0;
  bool done = false;
  for (; rounds < RESOLVE_MAX_ROUNDS; ++rounds) {
    int left = 0;
    for (int64_t p = t; p < na; p += RT) {
      if (flags[p] & 1) continue;
      left = 1;
      const PairRec rp = pairs[p];
      if (first_at(p, rp, rp.ia, head, next, pairs, flags) &&
          first_at(p, rp, rp.ib, head, next, pairs, flags))
        flags[p] = 2;
    }
    if (!__syncthreads_or(left)) { done = true; break; }
    for (int64_t p = t; p < na; p += RT) {
      if (flags[p] == 2) {
        kick(pairs[p], vel, mass, k0, k1, step, 1.0, &s_dirfail);
        flags[p] = 1;
      }
    }
    __syncthreads();
  }
  if (!done) {
    // the cap was reached with pairs left
    int left = 0;
    for (int64_t p = t; p < na; p += RT) left |= !(flags[p] & 1);
    if (__syncthreads_or(left) && t == 0) atomicOr(&st->status, (unsigned)ST_ERR_ROUNDS);
  }
  int mm = 0;
  for (int64_t p = t; p < na; p += RT) mm = max(mm, max(mult[pairs[p].ia], mult[pairs[p].ib]));
  atomicMax(&s_max, mm);
  __syncthreads();
  for (int64_t p = t; p < na; p += RT) {
    head[pairs[p].ia] = -1;
    head[pairs[p].ib] = -1;
    mult[pairs[p].ia] = 0;
    mult[pairs[p].ib] = 0;
  }
  if (t == 0) {
    st->n_rounds = (unsigned long long)rounds;
    st->max_mult = (unsigned long long)s_max;
    if (s_dirfail) {
      st->n_dirfail = s_dirfail;
      atomicOr(&st->status, (unsigned)ST_DIR_FAIL);
    }
  }
}

// ---- step path: dataflow application ------------------------------------
//
// 1. count: accepted pairs per particle.
// 2. split: a pair whose two particles take part in no other accepted pair
//    commutes with every other kick and is applied at once; the others are
//    "pending".  Each particle of a pending pair gets a segment of its pairs.
// 3. fill + sort: the segments are filled and sorted by key (ord, a, b), and
//    every particle gets a cursor at its first segment entry.
// 4. dataflow: a pending pair is ready when it sits at the cursor of both of
//    its particles, i.e. when every earlier pair of both particles has been
//    applied.  Ready pairs are applied and advance the two cursors (release
//    pattern after the kick: one fence.acq_rel, then relaxed stores; the
//    cursors are polled with acquire loads, which order the velocity reads
//    after the earlier kicks without a fence), so every
//    particle meets its pairs in key order -- the sequential result.  The
//    grid is launched cooperatively (all blocks resident); the globally first
//    unapplied pair is always ready, so the passes make progress.  A bounded
//    number of passes guards against a stuck state (error flag).
// 5. reset the per-particle arrays that were touched.

constexpr int GT = 256;
constexpr int DATAFLOW_MAX_PASSES = 1 << 22;

// A pair or deferred-draw buffer that overflowed makes the step invalid:
// then nothing is applied.
__device__ __forceinline__ bool step_overflowed(const DevStats* st, int64_t cap) {
  return st->n_acc > (unsigned long long)cap || st->n_deferred > (unsigned long long)cap;
}

__device__ __forceinline__ void st_relaxed(int32_t* p, int v) {
  asm volatile("st.relaxed.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_acquire(const int32_t* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void fence_acq_rel() {
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

// Isotropic direction of pair r (Marsaglia, Philox streams 1, 2, ...); it
// depends only on the pair's key, so it is drawn before the pair's turn.
__device__ __forceinline__ void pair_direction(const PairRec& r, uint32_t k0, uint32_t k1,
                                               uint32_t step, double* e, unsigned* dirfail) {
  e[0] = 0.0;
  e[1] = 0.0;
  e[2] = 1.0;
  bool found = false;
  for (uint32_t t = 0; t < DIRECTION_TRIES && !found; ++t) {
    const U4 w = philox10(k0, k1, step, 1u + t, r.a, r.b);
    const double x1 = 2.0 * unit53(w.x, w.y) - 1.0;
    const double x2 = 2.0 * unit53(w.z, w.w) - 1.0;
    const double s = x1 * x1 + x2 * x2;
    if (s > 0.0 && s < 1.0) {
      const double k = 2.0 * sqrt(1.0 - s);
      e[0] = x1 * k;
      e[1] = x2 * k;
      e[2] = 1.0 - 2.0 * s;
      found = true;
    }
  }
  if (!found) atomicAdd(dirfail, 1u);
}

// The kick of a pending pair with direction e, the velocities read and
// written through L2 (other SMs apply the neighbouring kicks).
__device__ __forceinline__ void kick_l2(const PairRec& r, double* vel, const KickTerms& kt,
                                        const double* e) {
  double* va = vel + 3 * (int64_t)r.ia;
  double* vb = vel + 3 * (int64_t)r.ib;
  double a[3] = {__ldcg(va), __ldcg(va + 1), __ldcg(va + 2)};
  double b[3] = {__ldcg(vb), __ldcg(vb + 1), __ldcg(vb + 2)};
  kick_values(kt, e, a, b);
  __stcg(va, a[0]);
  __stcg(va + 1, a[1]);
  __stcg(va + 2, a[2]);
  __stcg(vb, b[0]);
  __stcg(vb + 1, b[1]);
  __stcg(vb + 2, b[2]);
}

__global__ void __launch_bounds__(GT) count_kernel(const PairRec* __restrict__ pairs, int64_t cap,
                                                   int32_t* mult, const DevStats* st) {
  const unsigned long long nall = st->n_acc;
  if (step_overflowed(st, cap)) return;
  for (int64_t p = blockIdx.x * (int64_t)GT + threadIdx.x; p < (int64_t)nall;
       p += (int64_t)gridDim.x * GT) {
    atomicAdd(&mult[pairs[p].ia], 1);
    atomicAdd(&mult[pairs[p].ib], 1);
  }
}

// Claims a segment for particle e (the first claimant allocates mult[e]
// slots); called by the whole warp, `want` per lane.  The slot and touched
// counters take one atomic per warp.
__device__ __forceinline__ void claim_segments(bool want, int32_t e, const int32_t* mult,
                                               int32_t* seg_off, int32_t* touched, DevStats* st) {
  const int lane = threadIdx.x & 31;
  const bool first = want && atomicCAS(&seg_off[e], -1, -2) == -1;
  const int cnt = first ? mult[e] : 0;
  int incl = cnt;
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  const uint32_t fm = __ballot_sync(0xffffffffu, first);
  if (!fm) return;
  unsigned long long bs = 0, bt = 0;
  if (lane == 0) {
    bs = atomicAdd(&st->n_seg, (unsigned long long)total);
    bt = atomicAdd(&st->n_touched, (unsigned long long)__popc(fm));
  }
  bs = __shfl_sync(0xffffffffu, bs, 0);
  bt = __shfl_sync(0xffffffffu, bt, 0);
  if (first) {
    seg_off[e] = (int32_t)(bs + (unsigned long long)(incl - cnt));
    touched[bt + __popc(fm & ((1u << lane) - 1u))] = e;
  }
}

__global__ void __launch_bounds__(GT, 4) split_kernel(const PairRec* __restrict__ pairs, int64_t cap,
                                                   double* vel, const double* __restrict__ mass,
                                                   ResolveBuffers b,
                                                   const int32_t* __restrict__ halo_of,
                                                   const Halo* __restrict__ halos, DevStats* st) {
  __shared__ unsigned s_dirfail;
  __shared__ int s_max;
  if (threadIdx.x == 0) { s_dirfail = 0; s_max = 0; }
  __syncthreads();
  const unsigned long long nall = st->n_acc;
  const int lane = threadIdx.x & 31;
  int mm = 0;
  if (!step_overflowed(st, cap)) {
    const int64_t na = (int64_t)nall;
    const int64_t stride = (int64_t)gridDim.x * GT;
    for (int64_t base = blockIdx.x * (int64_t)GT + (threadIdx.x & ~31); base < na; base += stride) {
      const int64_t p = base + lane;
      bool pend = false;
      PairRec r{};
      if (p < na) {
        r = pairs[p];
        const int ma = b.mult[r.ia], mb = b.mult[r.ib];
        mm = max(mm, max(ma, mb));
        if (ma == 1 && mb == 1) {
          const Halo& H = halos[halo_of[r.ia]];
          kick(r, vel, mass, (uint32_t)H.seed, (uint32_t)(H.seed >> 32), H.step, H.eps,
               &s_dirfail);
        } else {
          pend = true;
          b.flags[p] = 0;
        }
      }
      claim_segments(pend, r.ia, b.mult, b.seg_off, b.touched, st);
      claim_segments(pend, r.ib, b.mult, b.seg_off, b.touched, st);
      const uint32_t m = __ballot_sync(0xffffffffu, pend);
      if (m) {
        unsigned long long at = 0;
        const int leader = __ffs(m) - 1;
        if (lane == leader) at = atomicAdd(&st->n_pending, (unsigned long long)__popc(m));
        at = __shfl_sync(0xffffffffu, at, leader);
        if (pend) b.pending[at + __popc(m & ((1u << lane) - 1u))] = (int32_t)p;
      }
    }
  }
  atomicMax(&s_max, mm);
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_max) atomicMax(&st->max_mult, (unsigned long long)s_max);
    if (s_dirfail) {
      atomicAdd(&st->n_dirfail, (unsigned long long)s_dirfail);
      atomicOr(&st->status, (unsigned)ST_DIR_FAIL);
    }
  }
}

__global__ void __launch_bounds__(GT) fill_kernel(const PairRec* __restrict__ pairs, int64_t cap,
                                                  ResolveBuffers b, const DevStats* st) {
  if (step_overflowed(st, cap)) return;
  const int64_t np = (int64_t)st->n_pending;
  for (int64_t k = blockIdx.x * (int64_t)GT + threadIdx.x; k < np; k += (int64_t)gridDim.x * GT) {
    const int32_t p = b.pending[k];
    const int32_t ea = pairs[p].ia, eb = pairs[p].ib;
    const int32_t sa = b.seg_off[ea] + atomicAdd(&b.fill[ea], 1);
    const int32_t sb = b.seg_off[eb] + atomicAdd(&b.fill[eb], 1);
    b.seg[sa] = p;
    b.seg_e[sa] = ea;
    b.seg[sb] = p;
    b.seg_e[sb] = eb;
  }
}

// Place of each pending pair in its particles' key order: one thread per
// segment slot counts the pairs of the same particle with a smaller key.
// (Keys (ord, a, b) are distinct, so the places are 0 .. mult-1.)
__global__ void __launch_bounds__(GT) rank_kernel(const PairRec* __restrict__ pairs, int64_t cap,
                                                  ResolveBuffers b, const DevStats* st) {
  if (step_overflowed(st, cap)) return;
  const int64_t ns = (int64_t)st->n_seg;
  for (int64_t t = blockIdx.x * (int64_t)GT + threadIdx.x; t < ns; t += (int64_t)gridDim.x * GT) {
    const int32_t e = b.seg_e[t], p = b.seg[t];
    const int32_t* sg = b.seg + b.seg_off[e];
    const int len = b.mult[e];
    const PairRec rp = pairs[p];
    int rank = 0;
    for (int k = 0; k < len; ++k) rank += key_less(pairs[sg[k]], rp) ? 1 : 0;
    if (rp.ia == e) b.pos_a[p] = rank;
    else b.pos_b[p] = rank;
  }
}

__global__ void __launch_bounds__(GT) dataflow_kernel(const PairRec* __restrict__ pairs, int64_t cap,
                                                      int max_passes, double* vel,
                                                      const double* __restrict__ mass,
                                                      ResolveBuffers b,
                                                      const int32_t* __restrict__ halo_of,
                                                      const Halo* __restrict__ halos,
                                                      DevStats* st) {
  __shared__ unsigned s_dirfail;
  __shared__ int s_passes;
  if (threadIdx.x == 0) { s_dirfail = 0; s_passes = 0; }
  __syncthreads();
  if (!step_overflowed(st, cap)) {
    const int64_t np = (int64_t)st->n_pending;
    const int64_t gsize = (int64_t)gridDim.x * GT;
    const int64_t t0 = blockIdx.x * (int64_t)GT + threadIdx.x;
    // the thread's first pair, prepared (mass terms, direction) before its
    // turn; a turn is two acquire loads of the cursors
    bool first = t0 < np;
    PairRec r0{};
    int pa0 = 0, pb0 = 0;
    KickTerms kt0{};
    double e0[3];
    if (first) {
      const int32_t p = b.pending[t0];
      r0 = pairs[p];
      pa0 = b.pos_a[p];
      pb0 = b.pos_b[p];
      const Halo& H = halos[halo_of[r0.ia]];
      kt0 = kick_terms(mass[r0.ia], mass[r0.ib], H.eps);
      pair_direction(r0, (uint32_t)H.seed, (uint32_t)(H.seed >> 32), H.step, e0, &s_dirfail);
    }
    int pass = 0;
    bool left = first;
    for (; left && pass < max_passes; ++pass) {
      left = false;
      if (first) {
        const int ca = ld_acquire(&b.cursor[r0.ia]);
        const int cb = ld_acquire(&b.cursor[r0.ib]);
        if (ca == pa0 && cb == pb0) {
          kick_l2(r0, vel, kt0, e0);
          fence_acq_rel();   // release: one fence covers both cursor stores
          st_relaxed(&b.cursor[r0.ia], pa0 + 1);
          st_relaxed(&b.cursor[r0.ib], pb0 + 1);
          first = false;
        } else {
          left = true;
        }
      }
      // further pairs of this thread (more pending pairs than threads)
      for (int64_t k = t0 + gsize; k < np; k += gsize) {
        const int32_t p = b.pending[k];
        if (b.flags[p]) continue;
        const PairRec r = pairs[p];
        const int pa = b.pos_a[p], pb = b.pos_b[p];
        const int ca = ld_acquire(&b.cursor[r.ia]);
        const int cb = ld_acquire(&b.cursor[r.ib]);
        if (ca == pa && cb == pb) {
          const Halo& H = halos[halo_of[r.ia]];
          double e[3];
          pair_direction(r, (uint32_t)H.seed, (uint32_t)(H.seed >> 32), H.step, e, &s_dirfail);
          kick_l2(r, vel, kick_terms(mass[r.ia], mass[r.ib], H.eps), e);
          fence_acq_rel();
          st_relaxed(&b.cursor[r.ia], pa + 1);
          st_relaxed(&b.cursor[r.ib], pb + 1);
          b.flags[p] = 1;
        } else {
          left = true;
        }
      }
    }
    if (left) atomicOr(&st->status, (unsigned)ST_ERR_ROUNDS);
    atomicMax(&s_passes, pass);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicMax(&st->n_rounds, (unsigned long long)s_passes);
    if (s_dirfail) {
      atomicAdd(&st->n_dirfail, (unsigned long long)s_dirfail);
      atomicOr(&st->status, (unsigned)ST_DIR_FAIL);
    }
  }
}

__global__ void __launch_bounds__(GT) reset_kernel(const PairRec* __restrict__ pairs, int64_t cap,
                                                   ResolveBuffers b, const DevStats* st) {
  const unsigned long long nall = st->n_acc;
  if (step_overflowed(st, cap)) return;
  const int64_t stride = (int64_t)gridDim.x * GT;
  const int64_t t0 = blockIdx.x * (int64_t)GT + threadIdx.x;
  for (int64_t p = t0; p < (int64_t)nall; p += stride) {
    b.mult[pairs[p].ia] = 0;
    b.mult[pairs[p].ib] = 0;
  }
  const int64_t nt = (int64_t)st->n_touched;
  for (int64_t k = t0; k < nt; k += stride) {
    const int32_t e = b.touched[k];
    b.seg_off[e] = -1;
    b.fill[e] = 0;
    b.cursor[e] = 0;
  }
}

int dataflow_grid(int sms) {
  static int per_sm = -1;
  if (per_sm < 0) {
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, dataflow_kernel, GT, 0) != cudaSuccess ||
        v < 1)
      v = 1;
    per_sm = v;
  }
  return per_sm * sms;
}

}  // namespace

int launch_resolve(PairRec* pairs, int64_t pair_cap, int max_passes, double* vel,
                   const double* mass, const int32_t* halo_of, const Halo* halos,
                   const ResolveBuffers& b, DevStats* st, int sms, cudaStream_t s) {
  const unsigned g = (unsigned)(sms * 4);
  count_kernel<<<g, GT, 0, s>>>(pairs, pair_cap, b.mult, st);
  split_kernel<<<g, GT, 0, s>>>(pairs, pair_cap, vel, mass, b, halo_of, halos, st);
  fill_kernel<<<g, GT, 0, s>>>(pairs, pair_cap, b, st);
  rank_kernel<<<g, GT, 0, s>>>(pairs, pair_cap, b, st);
  // cooperative launch: every block resident, as the passes wait on each other
  ResolveBuffers bb = b;
  PairRec* pp = pairs;
  int64_t cap = pair_cap;
  int mp = max_passes > 0 ? max_passes : DATAFLOW_MAX_PASSES;
  void* args[] = {(void*)&pp,   (void*)&cap,     (void*)&mp,    (void*)&vel, (void*)&mass,
                  (void*)&bb,   (void*)&halo_of, (void*)&halos, (void*)&st};
  if (cudaLaunchCooperativeKernel((const void*)dataflow_kernel, dim3(dataflow_grid(sms)),
                                  dim3(GT), args, 0, s) != cudaSuccess)
    return -1;
  reset_kernel<<<g, GT, 0, s>>>(pairs, pair_cap, b, st);
  return 6;
}


// The same kernel for the no-allocation entry point: every scratch pointer
// (head, next, flags, mult, st) is supplied by the caller.
void launch_resolve_with_scratch(const PairRec* pairs, int64_t pair_cap, double* vel,
                                 const double* mass, int32_t* head, int32_t* next, uint8_t* flags,
                                 int32_t* mult, uint64_t seed, uint32_t step, DevStats* st,
                                 cudaStream_t s) {
  resolve_kernel<<<1, RT, 0, s>>>(pairs, pair_cap, vel, mass, head, next, flags, mult,
                                  (uint32_t)seed, (uint32_t)(seed >> 32), step, st);
}

}  // namespace sidm
