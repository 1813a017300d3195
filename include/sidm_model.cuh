/*
 * sidm_model.cuh -- device-side interface for the physics of one scatter
 * (CUDA C++, header-only; compile with nvcc for sm_103a, -fmad=false when
 * results must be bit-reproducible).
 *
 * The paper's module is extended with new pairwise interactions by writing
 * four functions, without touching the neighbour search or the parallel
 * scheme (Sec. 4.6):
 *   scatter(state_i, state_j) -> (state_i', state_j')   the interaction;
 *   get_state(particle) -> state                         read a particle;
 *   set_state(particle, state)                           write it back;
 *   overwrite_state(state_in, state_out) -> state        what a particle that
 *                                                       took part carries on.
 * Here a model is a struct M with
 *   typename M::State      the per-particle state the interaction uses;
 *   typename M::Particles  device pointers into the caller's particle arrays;
 *   __device__ State get_state(const Particles&, int32_t i) const;
 *   __device__ void set_state(const Particles&, int32_t i, const State&) const;
 *   __device__ void scatter(State& a, State& b, const PairInfo&) const;
 *   __device__ State overwrite_state(const State& in, const State& out) const;
 * and, optionally, a split of scatter into work that may run before the
 * pair's turn and the part that needs the current states:
 *   typename M::Prepared;
 *   __device__ Prepared prepare(const PairInfo&, const Particles&) const;
 *   __device__ void scatter_prepared(State& a, State& b, const Prepared&) const;
 *
 * The library decides which pairs scatter (one draw per unordered pair from
 * the start-of-step states, Philox stream 0) and in which order they act:
 * ascending (ord, a, b), every particle meeting its pairs in that order, so
 * that each interaction sees the states the earlier ones left (Sec. 4.4,
 * Sec. 4.5).  For each accepted pair it reads both states with get_state,
 * calls scatter on copies, and writes overwrite_state(in, out) back with
 * set_state.  Pairs that share no particle run concurrently; a particle is
 * never in two interactions at once.  get_state and set_state of one
 * particle may run on different SMs one after the other; the library orders
 * them with release / acquire operations, so plain loads and stores are
 * correct (L2-only loads and stores, ld.cg / st.cg, avoid L1 traffic that
 * another SM would invalidate).
 *
 * apply_pairs<M>() applies a list of accepted pairs with model M in that
 * order; the scattering step of libsidm.so applies its own accepted pairs
 * through the same templates with the built-in model IsotropicKick (elastic,
 * or inelastic with the halo's eps).
 */
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <type_traits>

#include "sidm.h"

namespace sidm_model {

// ---------------------------------------------------------------- Philox
// Philox-4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): 10 rounds, each two
// 32x32 -> 64-bit products of counter words 0 and 2 with fixed multipliers;
// the high halves are xor-ed with counter words 1, 3 and the key, the key is
// advanced by two Weyl increments between rounds.
__host__ __device__ __forceinline__ uint4 philox4x32_10(uint32_t k0, uint32_t k1, uint32_t c0,
                                                       uint32_t c1, uint32_t c2, uint32_t c3) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
    const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
  }
  return make_uint4(c0, c1, c2, c3);
}

// 53 random bits -> [0, 1), exact in FP64: top 27 bits of one word, top 26 of the other.
__host__ __device__ __forceinline__ double unit53(uint32_t a, uint32_t b) {
  return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6)) * 0x1.0p-53;
}

// ----------------------------------------------------- one accepted pair
struct PairInfo {
  uint32_t a, b;        // ids, a < b
  int32_t ia, ib;       // indices of the a- and b-particle in the caller's arrays
  uint32_t k0, k1;      // Philox key: the seed of the pair's halo
  uint32_t step;        // Philox counter word 0: the step counter (mod 2^32)
  unsigned* warnings;   // a model counts here events the caller should hear of
                        // (reported as SIDM_WARN_DIRECTION)
  // Words of the pair's random stream t >= 1 (stream 0 drew the acceptance):
  // Philox counter (step, t, a, b).
  __device__ __forceinline__ uint4 words(uint32_t t) const {
    return philox4x32_10(k0, k1, step, t, a, b);
  }
};

// ------------------------------------------------ the built-in model
// Isotropic scattering in the centre-of-momentum frame (Sec. 4.1): the pair
// keeps v_com = (m_a v_a + m_b v_b) / M and leaves along +-e, e uniform on
// the sphere, with relative speed eps |v_a - v_b| (eps = 1: elastic):
//   v_a' = v_com + ((m_b g) / M) e,  v_b' = v_com - ((m_a g) / M) e,
// every operation rounded once in that order.  e by Marsaglia (1972): x1, x2
// from streams 1, 2, ... until 0 < s = x1^2 + x2^2 < 1, then
// e = (2 x1 sqrt(1 - s), 2 x2 sqrt(1 - s), 1 - 2 s); after 64 failed tries
// e = +z and a warning is counted.
namespace detail {

// The mass terms of a pair: M = m_a + m_b and, where M lies in
// [2^-500, 2^500), its correctly rounded reciprocal y = 1/M.
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
// [2^-500, 2^500) (where a step could under- or overflow), the division;
// a zero x is returned as it is.
__device__ __forceinline__ double div_m(double x, const KickTerms& t) {
  // +-0 / M = +-0 exactly for M positive and in range
  if (t.rcp && ((unsigned long long)__double_as_longlong(x) << 1) == 0ull) return x;
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
  return __ddiv_rn(x, t.M);
}

// The kick of Eqs. 12-13 in the operation order
//   v_com = ((m_a v_a) + (m_b v_b)) / M,  g = sqrt((dx dx + dy dy) + dz dz) eps,
//   v_a' = v_com + ((m_b g) / M) e,  v_b' = v_com - ((m_a g) / M) e,
// (eps = 1: the product with 1 is exact and skipped); every operation rounds
// once.
__device__ __forceinline__ void kick_values(const KickTerms& t, const double* e, double* a,
                                            double* b) {
  double c[3], d[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    c[k] = div_m(__dadd_rn(__dmul_rn(t.ma, a[k]), __dmul_rn(t.mb, b[k])), t);
    d[k] = __dsub_rn(a[k], b[k]);
  }
  double g = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])),
                                  __dmul_rn(d[2], d[2])));
  if (!t.elastic) g = __dmul_rn(g, t.eps);
  const double fa = div_m(__dmul_rn(t.mb, g), t), fb = div_m(__dmul_rn(t.ma, g), t);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    a[k] = __dadd_rn(c[k], __dmul_rn(fa, e[k]));
    b[k] = __dsub_rn(c[k], __dmul_rn(fb, e[k]));
  }
}

}  // namespace detail

struct IsotropicKick {
  double eps = 1.0;     // outgoing / incoming relative speed (1: elastic)

  struct State {
    double v[3];
    double m;
  };
  struct Particles {
    double* vel;        // n x 3, row-major
    const double* mass; // n
  };
  struct Prepared {
    detail::KickTerms kt;
    double e[3];
  };

  static constexpr int DIRECTION_TRIES = 64;

  // e uniform on the sphere from the pair's streams 1, 2, ... (Marsaglia)
  __device__ __forceinline__ static void direction(const PairInfo& p, double* e) {
    e[0] = 0.0;
    e[1] = 0.0;
    e[2] = 1.0;
    for (uint32_t t = 0; t < DIRECTION_TRIES; ++t) {
      const uint4 w = p.words(1u + t);
      const double x1 = __dsub_rn(__dmul_rn(2.0, unit53(w.x, w.y)), 1.0);
      const double x2 = __dsub_rn(__dmul_rn(2.0, unit53(w.z, w.w)), 1.0);
      const double s = __dadd_rn(__dmul_rn(x1, x1), __dmul_rn(x2, x2));
      if (s > 0.0 && s < 1.0) {
        const double k = __dmul_rn(2.0, __dsqrt_rn(__dsub_rn(1.0, s)));
        e[0] = __dmul_rn(x1, k);
        e[1] = __dmul_rn(x2, k);
        e[2] = __dsub_rn(1.0, __dmul_rn(2.0, s));
        return;
      }
    }
    if (p.warnings) atomicAdd(p.warnings, 1u);
  }

  __device__ __forceinline__ State get_state(const Particles& P, int32_t i) const {
    const double* v = P.vel + 3 * (int64_t)i;
    return State{{__ldcg(v), __ldcg(v + 1), __ldcg(v + 2)}, __ldg(P.mass + i)};
  }
  __device__ __forceinline__ void set_state(const Particles& P, int32_t i, const State& s) const {
    double* v = P.vel + 3 * (int64_t)i;
    __stcg(v, s.v[0]);
    __stcg(v + 1, s.v[1]);
    __stcg(v + 2, s.v[2]);
  }
  __device__ __forceinline__ Prepared prepare(const PairInfo& p, const Particles& P) const {
    Prepared r;
    r.kt = detail::kick_terms(__ldg(P.mass + p.ia), __ldg(P.mass + p.ib), eps);
    direction(p, r.e);
    return r;
  }
  __device__ __forceinline__ void scatter_prepared(State& a, State& b, const Prepared& r) const {
    detail::kick_values(r.kt, r.e, a.v, b.v);
  }
  __device__ __forceinline__ void scatter(State& a, State& b, const PairInfo& p) const {
    double e[3];
    direction(p, e);
    detail::kick_values(detail::kick_terms(a.m, b.m, eps), e, a.v, b.v);
  }
  __device__ __forceinline__ State overwrite_state(const State&, const State& out) const {
    return out;
  }

  // The prepared kick with its arithmetic spread over a group of GROUP
  // lanes (lanes GROUP g .. GROUP g + GROUP - 1 of a warp, all of them
  // calling together).  Lane s of the group:
  //   s = 0, 1, 2: component s of the a-side (m_a v_a, v_com, v_a');
  //   s = 5, 6, 7: component s - 5 of the b-side (m_b v_b, v_com, v_b');
  //   s = 3: (m_b g) / M;  s = 4: (m_a g) / M;
  // every lane the differences and the square root.  A warp's FP64
  // instruction costs the same for one lane or 32, so the pair's FP64
  // instruction stream shrinks from ~62 to ~23.  Each value is made by the
  // operations of kick_values in the same order (v_b' = v_com - (f_b e) as
  // v_com + (f_b (-e)), which rounds identically), so the result is
  // bit-identical.  The group holds the pair (ia, ib, r) when `active`;
  // otherwise it only takes part in the shuffles.  Loads and stores as
  // get_state / set_state.
  static constexpr int GROUP = 8;
  __device__ __forceinline__ void scatter_group(const Particles& P, int32_t ia, int32_t ib,
                                                const Prepared& r, bool active) const {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, sub = lane & (GROUP - 1), base = lane & ~(GROUP - 1);
    const bool side_a = sub < 3, side_b = sub >= 5, comp = side_a || side_b;
    const int k = side_a ? sub : (side_b ? sub - 5 : 0);
    const detail::KickTerms& t = r.kt;
    double a = 0.0, b = 0.0;
    if (active) {
      a = __ldcg(P.vel + 3 * (int64_t)ia + k);
      b = __ldcg(P.vel + 3 * (int64_t)ib + k);
    }
    const double d = __dsub_rn(a, b);
    const double sq = __dmul_rn(d, d);
    const double s0 = __shfl_sync(full, sq, base), s1 = __shfl_sync(full, sq, base + 1),
                 s2 = __shfl_sync(full, sq, base + 2);
    double g = __dsqrt_rn(__dadd_rn(__dadd_rn(s0, s1), s2));
    if (!t.elastic) g = __dmul_rn(g, t.eps);
    // one product per lane: m_a v_a (a-side), m_b v_b (b-side), m_b g, m_a g
    const double pm = __dmul_rn(side_a || sub == 4 ? t.ma : t.mb, comp ? (side_a ? a : b) : g);
    // the partner's product (a-side lane s <-> b-side lane s + 5)
    const double po = __shfl_sync(full, pm, side_a ? lane + 5 : (side_b ? lane - 5 : lane));
    // x = m_a v_a + m_b v_b on both sides; m g + 0 (exact) on lanes 3, 4
    const double x = __dadd_rn(side_b ? po : pm, comp ? (side_b ? pm : po) : 0.0);
    // x / M, correctly rounded (div_m: Markstein's step, checked)
    const double q0 = __dmul_rn(x, t.y);
    double q = __fma_rn(__fma_rn(-t.M, q0, x), t.y, q0);
    {
      const double rr = __fma_rn(-t.M, q, x);
      const unsigned long long qb = (unsigned long long)__double_as_longlong(q);
      const unsigned long long rb = (unsigned long long)__double_as_longlong(rr);
      const bool toward0 = ((qb ^ rb) >> 63) != 0;
      const bool pow2 = (qb & 0xFFFFFFFFFFFFFull) == 0;
      const long long kk = (long long)((qb >> 52) & 0x7FFu) - 1076 - ((toward0 && pow2) ? 1 : 0);
      const unsigned long long half_gap =
          (unsigned long long)__double_as_longlong(t.M) + ((unsigned long long)kk << 52);
      // a zero numerator is its own quotient (M is positive and in range
      // when t.rcp); a group without a pair needs no quotient.  Either way
      // the division below is skipped: a lane that takes it holds the
      // whole warp for the division's ~650 cycles.
      const bool xzero = ((unsigned long long)__double_as_longlong(x) << 1) == 0ull;
      if (t.rcp && xzero) q = x;
      const bool ok = !active || (t.rcp && (xzero || (detail::in_rcp_range(x, false) &&
                                                      (rb & 0x7FFFFFFFFFFFFFFFull) < half_gap)));
      if (!ok) q = __ddiv_rn(x, t.M);
    }
    const double fa = __shfl_sync(full, q, base + 3), fb = __shfl_sync(full, q, base + 4);
    const double ek = k == 0 ? r.e[0] : (k == 1 ? r.e[1] : r.e[2]);
    const double nv = __dadd_rn(q, __dmul_rn(side_a ? fa : fb, side_a ? ek : -ek));
    if (active && comp) __stcg(P.vel + 3 * (int64_t)(side_a ? ia : ib) + k, nv);
  }
};

// ------------------------------------------------- application order
// Model-independent detection of the optional prepare / scatter_prepared.
template <class M, class = void>
struct has_prepare : std::false_type {};
template <class M>
struct has_prepare<M, std::void_t<typename M::Prepared,
                                  decltype(std::declval<const M&>().prepare(
                                      std::declval<const PairInfo&>(),
                                      std::declval<const typename M::Particles&>()))>>
    : std::true_type {};

// Detection of the optional group form of scatter_prepared (scatter_group,
// with GROUP lanes per pair).
template <class M, class = void>
struct has_group : std::false_type {};
template <class M>
struct has_group<M, std::void_t<decltype(M::GROUP),
                                decltype(std::declval<const M&>().scatter_group(
                                    std::declval<const typename M::Particles&>(), int32_t(0),
                                    int32_t(0), std::declval<const typename M::Prepared&>(),
                                    true))>> : std::true_type {};

}  // namespace sidm_model

#include "sidm_model_apply.cuh"
