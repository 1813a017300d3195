// Candidate pairs, their probabilities and the one draw per unordered pair.
//
// One warp per active particle i, one lane per neighbour j in N(i) (from the
// neighbour list of the search kernel; a direct tree walk with radius h_i if
// the list was not complete).  For each j:
//   * (v sigma/m)(v_ij) enters the maximum of Eq. 18 (start-of-step
//     velocities);
//   * i owns the unordered pair unless j is active, sees i (r^2 < h_j^2) and
//     has the smaller id -- every pair is evaluated exactly once;
//   * the owner forms P_pair = P(i|j) + [j active, i in N(j)] P(j|i) with
//     P(i|j) = 1/2 m_j (sigma/m) |v_i - v_j| W(r, h_i) dt_i (Eqs. 10, 11, 14), and
//     draws u from Philox-4x32-10 with counter (step, 0, min id, max id);
//     u < P_pair accepts; words 2, 3 form the order key.
//
// Exactness with little FP64: P_pair is first bounded from above in FP32
// from the FP32 copies of positions, velocities, masses, dt and h (every
// factor rounded or widened upwards, then a relative margin), and u from
// below by its top 24 bits.  Only when that lower bound of u lies below the
// bound of P_pair (about the acceptance probability) is P_pair evaluated in
// FP64 in the oracle's operation order, and the draw decided on that value.
// The FP64 state of the query is read only on these rare paths.  The owner test r^2 < h_j^2 and the maximum of Eq. 18 likewise
// use FP32 intervals and fall back to FP64 only where an interval straddles
// the decision.  All results equal those of a pure FP64 evaluation.
#include "traverse.cuh"

namespace sidm {

namespace {

constexpr int PW = 4;
constexpr int PT = PW * WARP;
constexpr int XT = 256;                            // thread-per-item passes
constexpr int MAXR = 8;                            // neighbour rounds of 32 (stride <= 256)
constexpr float U = 5.9604644775390625e-08f;       // 2^-24
constexpr float REL = 9.5367431640625e-07f;        // 2^-20
constexpr float ABS = 4.76837158203125e-07f;       // 2^-21
constexpr float SLACK = 3.814697265625e-06f;       // 2^-18
constexpr float FLT_TINY = 7.888609052210118e-31f;  // 2^-100

struct PairKArgs {
  Sorted so;
  Forest f;
  int64_t n;
  const int32_t* act_list;
  const int32_t* nb_list;
  const int32_t* nb_count;
  int nb_stride;
  PairArgs a;
  PairRec* pairs;
  double* dtlim_user;
  DevStats* st;
  int* work;
  int chunk;          // queries claimed per work-counter increment
};

__device__ __forceinline__ double warp_maxd(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_maxf(float v) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_sumd(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// FP32 kernel shape, clamped to [0, 1]; non-increasing in q.
__device__ __forceinline__ float shape_f(int kernel, float q) {
  if (kernel == SIDM_KERNEL_TOPHAT) return 1.0f;
  q = fminf(fmaxf(q, 0.0f), 1.0f);
  if (q <= 0.5f) return 1.0f - 6.0f * (q * q) + 6.0f * (q * q * q);
  const float u = 1.0f - q;
  return 2.0f * (u * u * u);
}

// FP32 estimate of a tabulated sigma/m (statistics and the split form)
__device__ __forceinline__ float table_f(const SigmaTable& T, float v) {
  const int n = T.n;
  if (!(v > T.v_rd[0])) return T.s_rd[0];
  if (v >= T.v_rd[n - 1]) return T.s_rd[n - 1];
  int lo = 0, hi = n - 1;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (T.v_rd[mid] <= v) lo = mid;
    else hi = mid;
  }
  const float l0 = __log2f(T.v_rd[lo]), l1 = __log2f(T.v_rd[lo + 1]);
  const float t = fminf(fmaxf((__log2f(v) - l0) / (l1 - l0), 0.0f), 1.0f);
  return T.s_rd[lo] + t * (T.s_rd[lo + 1] - T.s_rd[lo]);
}

__device__ __forceinline__ float sigma_f(int kind, float s0, float w, const SigmaTable& T,
                                         float v) {
  if (kind == SIDM_SIGMA_TABLE) return table_f(T, v);
  if (kind == SIDM_SIGMA_YUKAWA) {
    const float t = 1.0f + (v * v) / (w * w);
    return s0 / (t * t);
  }
  return s0;
}

// Bounds of a tabulated sigma/m over v in [vl, vu] from node values alone:
// nodes a..b cover every segment that may hold such a v (a: the last node
// surely <= vl, b: the first node surely >= vu), and sigma/m on a segment
// lies between its two node values.
__device__ __forceinline__ void table_bounds(const SigmaTable& T, float vl, float vu, float* smin,
                                             float* smax) {
  const int n = T.n;
  int a = 0, hi = n;  // a: largest k with v_ru[k] <= vl (0 if none)
  while (hi - a > 1) {
    const int mid = (a + hi) >> 1;
    if (T.v_ru[mid] <= vl) a = mid;
    else hi = mid;
  }
  int lo = -1, b = n - 1;  // b: smallest k with v_rd[k] >= vu (n - 1 if none)
  while (b - lo > 1) {
    const int mid = (lo + b) >> 1;
    if (T.v_rd[mid] >= vu) b = mid;
    else lo = mid;
  }
  if (b < a) b = a;
  float mn = INFINITY, mx = 0.0f;
  for (int k = a; k <= b; ++k) {
    mn = fminf(mn, T.s_rd[k]);
    mx = fmaxf(mx, T.s_ru[k]);
  }
  *smin = mn;
  *smax = mx;
}

// g(v) = v sigma/m(v) for v in [vl, vu]: lower and upper bounds.  Constant
// sigma: g is increasing.  Yukawa-like: g rises up to v = w / sqrt(3) and
// falls after it.  Table: v times the node-value bounds.
__device__ __forceinline__ void g_bounds(int kind, float s0, float w, const SigmaTable& T,
                                         float vl, float vu, float* glo, float* ghi) {
  if (kind == SIDM_SIGMA_TABLE) {
    float smin, smax;
    table_bounds(T, vl, vu, &smin, &smax);
    *ghi = __fmul_ru(__fmul_ru(vu, smax), 1.0f + SLACK);
    *glo = __fmul_rd(__fmul_rd(vl, smin), 1.0f - SLACK);
  } else if (kind == SIDM_SIGMA_YUKAWA) {
    const float vp = w * 0.57735026918962576f;
    const float gl = vl * sigma_f(kind, s0, w, T, vl), gu = vu * sigma_f(kind, s0, w, T, vu);
    float hi;
    if (vu <= vp * (1.0f - SLACK)) hi = gu;
    else if (vl >= vp * (1.0f + SLACK)) hi = gl;
    else hi = vp * sigma_f(kind, s0, w, T, vp);
    *ghi = fmaxf(hi, fmaxf(gl, gu)) * (1.0f + SLACK);
    *glo = fminf(gl, gu) * (1.0f - SLACK);
  } else {
    *ghi = vu * s0 * (1.0f + SLACK);
    *glo = vl * s0 * (1.0f - SLACK);
  }
}

// Bounds of g_ij for the overlap estimator from the FP32 bounds of h_i,
// h_j and r_ij: a = min(h)/H and s = r/H lie in intervals; the exact value
// interpolates four table nodes of a cell those intervals reach (one cell
// of margin covers the FP64 rounding of a and s), so it is at most their
// largest rounded-up value, over H^3 from below.  gest: an FP32 estimate
// (statistics and the split form).
constexpr float ULP1 = 1.1920928955078125e-07f;  // 2^-23
__device__ __forceinline__ void overlap_bounds(const OverlapTable& T, float4 hbi, float4 hbj,
                                               float rlo, float rhi, float r, float* gup,
                                               float* gest) {
  const float Hlo = __fadd_rd(hbi.x, hbj.x), Hhi = __fadd_ru(hbi.y, hbj.y);
  const float ilo = __fmul_rd(__frcp_rn(Hhi), 1.0f - ULP1);  // <= 1/H
  const float ihi = __fmul_ru(__frcp_rn(Hlo), 1.0f + ULP1);  // >= 1/H
  const float alo = __fmul_rd(fminf(hbi.x, hbj.x), ilo), ahi = __fmul_ru(fminf(hbi.y, hbj.y), ihi);
  const float slo = __fmul_rd(rlo, ilo), shi = __fmul_ru(rhi, ihi);
  const int na = T.na, ns = T.ns;
  const float fa2 = 2.0f * (float)na, fs1 = (float)ns;
  int a0 = (int)fminf(__fmul_rd(alo, fa2), (float)na) - 1;
  int a1 = (int)fminf(__fmul_ru(ahi, fa2), (float)na) + 1;
  int s0 = (int)fminf(__fmul_rd(slo, fs1), (float)ns) - 1;
  int s1 = (int)fminf(__fmul_ru(shi, fs1), (float)ns) + 1;
  a0 = max(a0, 0);
  a1 = min(a1, na - 1);
  s0 = max(s0, 0);
  s1 = min(s1, ns - 1);
  float gmax = 0.0f;
  for (int ia = a0; ia <= a1 + 1; ++ia)
    for (int is = s0; is <= s1 + 1; ++is) gmax = fmaxf(gmax, T.g_ru[ia * (ns + 1) + is]);
  *gup = __fmul_ru(gmax, __fmul_ru(__fmul_ru(ihi, ihi), ihi));
  // estimate at the midpoint
  const float H = 0.5f * (Hlo + Hhi);
  const float a = fminf(0.5f * (hbi.x + hbi.y), 0.5f * (hbj.x + hbj.y)) / H, sv = r / H;
  float est = 0.0f;
  if (sv < 1.0f) {
    const float fa = a * fa2, fs = sv * fs1;
    const int ia = min((int)fa, na - 1), is = min((int)fs, ns - 1);
    const float ta = fa - (float)ia, ts = fs - (float)is;
    const float* r0 = T.g_ru + ia * (ns + 1);
    const float* r1 = r0 + (ns + 1);
    est = (1.0f - ta) * ((1.0f - ts) * r0[is] + ts * r0[is + 1]) +
          ta * ((1.0f - ts) * r1[is] + ts * r1[is + 1]);
  }
  *gest = est / (H * H * H);
}

// What one warp knows about its query particle i.
struct Query {
  int64_t s;            // key-order index
  uint32_t idi;
  int32_t oi;           // user-order index
  float4 fi, vmi, hbi;  // FP32 position + dt, velocity + mass, h bounds
  float eq, vmax_i;
  uint32_t k0, k1, step;
  int kind;
  float s0f, wf;
};

__device__ __forceinline__ Query load_query(const Sorted& so, const Forest& f, int64_t s,
                                            float boxf) {
  Query Q;
  Q.s = s;
  const Halo& H = f.halos[so.halo[s]];
  Q.k0 = (uint32_t)H.seed;
  Q.k1 = (uint32_t)(H.seed >> 32);
  Q.step = H.step;
  Q.kind = H.sigma_kind;
  Q.s0f = f64_to_f32_ru(H.sigma0);
  Q.wf = f64_to_f32_rn(H.w);
  Q.idi = so.id[s];
  Q.oi = so.orig[s];
  Q.fi = so.f[s];
  Q.vmi = so.vm[s];
  Q.hbi = so.hb[s];
  Q.eq = ABS * (fmaxf(fmaxf(fabsf(Q.fi.x), fabsf(Q.fi.y)), fabsf(Q.fi.z)) + boxf);
  Q.vmax_i = fmaxf(fmaxf(fabsf(Q.vmi.x), fabsf(Q.vmi.y)), fabsf(Q.vmi.z));
  return Q;
}

// Everything about one neighbour j of the query (valid lanes only); the
// accepted pair is appended by the whole warp.  Returns bounds of
// g = v sigma/m(v) in glo/ghi and adds the pair's probability (FP32
// estimate, or the exact value where it was computed) to *psum.
__device__ __forceinline__ void visit(const PairKArgs& A, const Query& Q, int64_t j, bool valid,
                                      float* glo_out, float* ghi_out, float* psum,
                                      unsigned long long* cand, unsigned long long* pge1,
                                      uint32_t* status) {
  const Sorted& so = A.so;
  const PairArgs& P = A.a;
  const int kern = P.kernel;
  const int lane = threadIdx.x & 31;
  const float boxf = (float)P.box;
  bool acc = false, defer = false;
  PairRec rec;
  int2 drec;
  float glo = 0.0f, ghi = 0.0f;
  if (valid) {
    const float4 fj = so.f[j];
    const float4 vmj = so.vm[j];
    const uint32_t idj = so.id[j];
    const bool actj = so.act[j] != 0;
    const float4 hbj = so.hb[j];  // meaningful when j is active
    // separation interval
    const float r2f = sep2f(Q.fi, fj, boxf);
    const float r = sqrtf(r2f);
    const float e = Q.eq + ABS * r;
    const float rlo = fmaxf(r * (1.0f - REL) - e, 0.0f);
    const float rhi = r * (1.0f + REL) + e;
    // relative speed interval
    const float dvx = Q.vmi.x - vmj.x, dvy = Q.vmi.y - vmj.y, dvz = Q.vmi.z - vmj.z;
    const float vr = sqrtf(dvx * dvx + dvy * dvy + dvz * dvz);
    const float vmax_j = fmaxf(fmaxf(fabsf(vmj.x), fabsf(vmj.y)), fabsf(vmj.z));
    const float dv = 4.0f * U * (3.0f * (Q.vmax_i + vmax_j) + vr) + 4.0f * U * vr;
    const float vl = fmaxf(vr - dv, 0.0f), vu = vr + dv;
    g_bounds(Q.kind, Q.s0f, Q.wf, P.table, vl, vu, &glo, &ghi);
    const float gest = vr * sigma_f(Q.kind, Q.s0f, Q.wf, P.table, vr);
    if (P.split) glo = ghi = gest;
    // does j see i?  (j active and r^2 < h_j^2: decided exactly, or in FP32
    // by the split form, as its neighbour lists are)
    bool sees = false;
    if (P.ov.na > 0) {
      sees = actj;  // overlap membership r < h_i + h_j is symmetric
    } else if (actj) {
      if (P.split) {
        const float hjf = f64_to_f32_rn(so.h[j]);
        sees = r2f < hjf * hjf;
      } else if (rhi < hbj.x) {
        sees = true;
      } else if (rlo < hbj.y) {
        sees = hw_within(so.x, so.y, so.z, Q.s, j, P.box, so.h[j]);
      }
    }
    if (!(sees && idj < Q.idi)) {
      // FP32 upper bound of P_pair.  The bound holds only while no product
      // of the chain leaves the normal FP32 range; below 2^-100 the FP64
      // path decides.
      float pu, pc;
      bool tiny;
      if (P.ov.na > 0) {
        // kernel overlap: the same g_ij bounds both directed terms
        float gup, gov;
        overlap_bounds(P.ov, Q.hbi, hbj, rlo, rhi, r, &gup, &gov);
        const float t1 = 0.5f * vmj.w, t2 = t1 * ghi, t3 = t2 * gup;
        pu = t3 * Q.fi.w;
        tiny = !(fminf(fminf(t1, t2), fminf(t3, pu)) >= FLT_TINY);
        pc = 0.5f * vmj.w * gest * gov * Q.fi.w;
        if (sees) {
          const float s1 = 0.5f * Q.vmi.w, s2 = s1 * ghi, s3 = s2 * gup, puj = s3 * fj.w;
          tiny = tiny || !(fminf(fminf(s1, s2), fminf(s3, puj)) >= FLT_TINY);
          pu += puj;
          pc += 0.5f * Q.vmi.w * gest * gov * fj.w;
        }
      } else {
      const float fi_up = shape_f(kern, __fmul_rd(rlo, Q.hbi.z)) * (1.0f + SLACK) + REL;
      const float t1 = 0.5f * vmj.w, t2 = t1 * ghi, t3 = t2 * Q.hbi.w, t4 = t3 * fi_up;
      pu = t4 * Q.fi.w;
      tiny = !(fminf(fminf(t1, t2), fminf(fminf(t3, t4), pu)) >= FLT_TINY);
      pc = 0.5f * vmj.w * gest * Q.hbi.w * shape_f(kern, r * Q.hbi.z) * Q.fi.w;
      if (sees) {
        const float fj_up = shape_f(kern, __fmul_rd(rlo, hbj.z)) * (1.0f + SLACK) + REL;
        const float s1 = 0.5f * Q.vmi.w, s2 = s1 * ghi, s3 = s2 * hbj.w, s4 = s3 * fj_up;
        const float puj = s4 * fj.w;
        tiny = tiny || !(fminf(fminf(s1, s2), fminf(fminf(s3, s4), puj)) >= FLT_TINY);
        pu += puj;
        pc += 0.5f * Q.vmi.w * gest * hbj.w * shape_f(kern, r * hbj.z) * fj.w;
      }
      }
      if (pu == 0.0f) {
        // A zero bound is an underflow unless P_pair is exactly zero: no
        // cross section, zero masses in every term, or two bit-equal
        // velocities (g(0) = 0, e.g. targets at rest).  Exact zeros are
        // rejected for any u >= 0 and need no FP64 pass.
        bool exact_zero = (Q.kind != SIDM_SIGMA_TABLE && Q.s0f == 0.0f) ||
                          (vmj.w == 0.0f && (!sees || Q.vmi.w == 0.0f));
        if (!exact_zero && vr == 0.0f) {
          const unsigned long long* bx = (const unsigned long long*)so.vx;
          const unsigned long long* by = (const unsigned long long*)so.vy;
          const unsigned long long* bz = (const unsigned long long*)so.vz;
          exact_zero = bx[Q.s] == bx[j] && by[Q.s] == by[j] && bz[Q.s] == bz[j];
        }
        tiny = !exact_zero;
      }
      pu *= (1.0f + SLACK);
      const bool i_is_a = Q.idi < idj;
      const uint32_t a = i_is_a ? Q.idi : idj, b = i_is_a ? idj : Q.idi;
      const U4 w = philox10(Q.k0, Q.k1, Q.step, 0u, a, b);
      // u lies in [u_lo, u_lo + 2^-24): its top 24 bits, exactly
      const float u_lo = __uint2float_rz(w.x >> 8) * U;
      if (P.split) {
        // split form: FP32 decision unless u may lie within 1e-5 of P
        const float d = pc - u_lo;
        defer = d > -1e-5f && d < 1e-5f + U;
        if (!defer) {
          if (pc >= 1.0f) ++*pge1;
          acc = d > 0.0f;
        }
      } else {
        // at or above the bound of P_pair the draw is surely rejected
        defer = tiny || u_lo < pu;
      }
      // the exact FP64 decision is left to the thread-per-pair pass
      if (defer) drec = make_int2((int)Q.s, (int)j | (sees ? (int)0x80000000u : 0));
      else *psum += pc;
      if (acc) {
        rec.ord = ((unsigned long long)w.z << 32) | (unsigned long long)w.w;
        rec.a = a;
        rec.b = b;
        const int32_t oj = so.orig[j];
        rec.ia = i_is_a ? Q.oi : oj;
        rec.ib = i_is_a ? oj : Q.oi;
      }
      ++*cand;
    }
  }
  const uint32_t dm = __ballot_sync(0xffffffffu, defer);
  if (dm) {
    unsigned long long base = 0;
    const int leader = __ffs(dm) - 1;
    if (lane == leader) base = atomicAdd(&A.st->n_deferred, (unsigned long long)__popc(dm));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (defer) {
      const unsigned long long at = base + __popc(dm & ((1u << lane) - 1u));
      if (at < (unsigned long long)P.pair_cap) P.deferred[at] = drec;
      else *status |= ST_ERR_PAIR_OVERFLOW;
    }
  }
  const uint32_t m = __ballot_sync(0xffffffffu, acc);
  if (m) {
    unsigned long long base = 0;
    const int leader = __ffs(m) - 1;
    if (lane == leader) base = atomicAdd(&A.st->n_acc, (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (acc) {
      const unsigned long long at = base + __popc(m & ((1u << lane) - 1u));
      if (at < (unsigned long long)P.pair_cap) A.pairs[at] = rec;
      else *status |= ST_ERR_PAIR_OVERFLOW;
    }
  }
  *glo_out = glo;
  *ghi_out = ghi;
}

// exact g = |v_i - v_j| sigma/m(|v_i - v_j|) in FP64 (i, j in key order)
__device__ __forceinline__ double exact_g(const PairKArgs& A, int64_t s, int64_t j) {
  const Sorted& so = A.so;
  const double ddx = so.vx[s] - so.vx[j], ddy = so.vy[s] - so.vy[j], ddz = so.vz[s] - so.vz[j];
  const double vrel = sqrt((ddx * ddx + ddy * ddy) + ddz * ddz);
  const Halo& H = A.f.halos[so.halo[s]];
  return vrel * sigma_over_m(H.sigma_kind, H.sigma0, H.w, A.a.table, vrel);
}

// Eq. 18: dt_lim,i = 2 C_SIDM / (m_i W(0, h_i) (v sigma/m)_max,i)
__device__ __forceinline__ void write_limit(const PairKArgs& A, int64_t s, double vs_max) {
  const Sorted& so = A.so;
  const double den = (so.m[s] * kernel_norm(A.a.kernel, so.h[s])) * vs_max;
  A.dtlim_user[so.orig[s]] = vs_max > 0.0 ? (A.a.c_sidm * 2.0) / den : INFINITY;
}

__device__ __forceinline__ void flush_counters(const PairKArgs& A, unsigned long long cand,
                                               unsigned long long pge1, double sum_p,
                                               uint32_t status) {
  for (int o = 16; o > 0; o >>= 1) {
    cand += __shfl_xor_sync(0xffffffffu, cand, o);
    pge1 += __shfl_xor_sync(0xffffffffu, pge1, o);
  }
  sum_p = warp_sumd(sum_p);
  status = __reduce_or_sync(0xffffffffu, status);
  if ((threadIdx.x & 31) == 0) {
    if (cand) atomicAdd(&A.st->n_cand, cand);
    if (pge1) {
      atomicAdd(&A.st->n_pge1, pge1);
      status |= ST_P_GE_1;
    }
    if (sum_p != 0.0) atomicAdd(&A.st->sum_p, sum_p);
    if (status) atomicOr(&A.st->status, status);
  }
}

// Queries with a complete neighbour list (the usual case).
// 7 resident blocks of 4 warps per SM (72 registers): the kernel waits on
// dependent L2 gathers, and 7 blocks hide them better than 6 at 80 registers
// (pair phase 0.238 -> 0.228 ms on the 2^20 halo)
#ifndef PAIRS_MIN_BLOCKS
#define PAIRS_MIN_BLOCKS 7
#endif
__global__ void __launch_bounds__(PT, PAIRS_MIN_BLOCKS) pairs_kernel(PairKArgs A) {
  __shared__ float s_ghi[PW][MAXR * WARP];
  if (A.a.ov.na > 0) return;  // the overlap estimator's queries all walk the tree
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* ghi_row = s_ghi[warp];
  const int64_t n_act = (int64_t)A.st->n_active;
  const float boxf = (float)A.a.box;
  unsigned long long cand = 0, pge1 = 0;
  double sum_p = 0.0;
  uint32_t status = 0;

  int q = 0, q_end = 0;
  for (;;) {
    if (q >= q_end) {
      if (lane == 0) q = atomicAdd(A.work, A.chunk);
      q = __shfl_sync(0xffffffffu, q, 0);
      q_end = q + A.chunk;
    }
    if (q >= n_act) break;
    const int64_t qi = q++;
    const int cnt = A.nb_count[qi];
    if (cnt < 0) continue;  // left to the tree-walk kernel
    const Query Q = load_query(A.so, A.f, A.act_list[qi], boxf);
    const int32_t* row = A.nb_list + qi * (int64_t)A.nb_stride;
    const int nr = (cnt + 31) >> 5;
    float mlo = 0.0f, psum = 0.0f;
    for (int r = 0; r < nr; ++r) {
      const int k = r * 32 + lane;
      const bool valid = k < cnt;
      const int32_t j = valid ? row[k] : -1;
      float gl, gh;
      visit(A, Q, j, valid, &gl, &gh, &psum, &cand, &pge1, &status);
      mlo = fmaxf(mlo, gl);
      ghi_row[k] = valid ? gh : -1.0f;
    }
    sum_p += (double)psum;
    // Eq. 18 maximum: only j whose upper bound of g reaches the largest lower
    // bound can give it; up to LIM_CAND of them are kept for the exact pass
    mlo = warp_maxf(mlo);
    __syncwarp();
    int nc = 0;
    for (int r = 0; r < nr; ++r) {
      const int k = r * 32 + lane;
      const bool c = k < cnt && ghi_row[k] >= mlo;
      const uint32_t m = __ballot_sync(0xffffffffu, c);
      const int at = nc + __popc(m & ((1u << lane) - 1u));
      if (c && at < LIM_CAND) A.a.lim_cand[qi * LIM_CAND + at] = row[k];
      nc += __popc(m);
    }
    if (lane == 0) {
      A.a.lim_cnt[qi] = nc <= LIM_CAND ? nc : -1;
      A.a.lim_g[qi] = mlo;
    }
    __syncwarp();
  }
  flush_counters(A, cand, pge1, sum_p, status);
}

// Queries whose neighbour list was not complete: walk the tree with radius
// h_i and decide membership exactly.
// One query whose neighbour list was incomplete: walk the tree with radius
// h_i and decide membership exactly (the whole warp).
__device__ void walk_query(const PairKArgs& A, int64_t qi, int* stack, unsigned long long* cand,
                           unsigned long long* pge1, double* sum_p, uint32_t* status) {
  const Sorted& so = A.so;
  const int lane = threadIdx.x & 31;
  const double box = A.a.box;
  const float boxf = (float)A.a.box;
  const Query Q = load_query(so, A.f, A.act_list[qi], boxf);
  const int64_t s = Q.s;
  const Halo& H = A.f.halos[so.halo[s]];
  const int64_t hs = H.start;
  const double hi = so.h[s];
  const bool ov = A.a.ov.na > 0;
  const float rad = (f64_to_f32_ru(hi) + 2.0f * Q.eq) * (1.0f + 4.0f * REL);
  double mine = 0.0;
  float psum = 0.0f;
  const int sl = (int)(s - hs);
  auto leaf = [&](int k, bool valid, const float4& pj) {
    const int64_t j = hs + k;
    bool in = false;
    if (valid && k != sl) {
      const float r = sqrtf(sep2f(Q.fi, pj, boxf));
      const float e = Q.eq + ABS * r;
      const float rlo = fmaxf(r * (1.0f - REL) - e, 0.0f);
      if (ov) {
        // overlap neighbours: r_ij < h_i + h_j, decided exactly near the edge
        const float4 hbj = so.hb[j];
        const float rhi = r * (1.0f + REL) + e;
        if (rhi < __fadd_rd(Q.hbi.x, hbj.x)) {
          in = true;
        } else if (rlo < __fadd_ru(Q.hbi.y, hbj.y)) {
          in = hw_within_sum(so.x, so.y, so.z, s, j, box, hi, so.h[j]);
        }
      } else if (A.a.split) {
        const float hf = (float)hi;
        in = r * r < hf * hf;
      } else if (rlo < Q.hbi.y) {
        in = hw_within(so.x, so.y, so.z, s, j, box, hi);
      }
    }
    float gl, gh;
    visit(A, Q, j, in, &gl, &gh, &psum, cand, pge1, status);
    if (in) mine = fmax(mine, A.a.split ? (double)gl : exact_g(A, s, j));
  };
  bool ok;
  if (ov)  // the radius at each node is widened by the node's largest h
    ok = A.a.box > 0.0
        ? traverse<true, true>(A.f, H, so.f + hs, Q.fi, 0.0f, boxf, stack, leaf, rad)
        : traverse<false, true>(A.f, H, so.f + hs, Q.fi, 0.0f, boxf, stack, leaf, rad);
  else
    ok = A.a.box > 0.0
        ? traverse<true>(A.f, H, so.f + hs, Q.fi, rad * rad, boxf, stack, leaf)
        : traverse<false>(A.f, H, so.f + hs, Q.fi, rad * rad, boxf, stack, leaf);
  if (!ok) *status |= ST_ERR_STACK;
  *sum_p += (double)psum;
  mine = warp_maxd(mine);
  if (lane == 0) write_limit(A, s, mine);
  __syncwarp();
}

// Queries whose neighbour list was not complete (rare): the warps scan the
// query list 32 entries at a time.
__global__ void __launch_bounds__(PT) pairs_walk_kernel(PairKArgs A) {
  __shared__ int s_stack[PW][SEARCH_STACK];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n_act = (int64_t)A.st->n_active;
  unsigned long long cand = 0, pge1 = 0;
  double sum_p = 0.0;
  uint32_t status = 0;
  const int64_t w0 = ((int64_t)blockIdx.x * PW + warp) * 32, ws = (int64_t)gridDim.x * PW * 32;
  for (int64_t q0 = w0; q0 < n_act; q0 += ws) {
    // every query walks for the overlap estimator (its neighbours need h_j)
    const bool need = q0 + lane < n_act && (A.a.ov.na > 0 || A.nb_count[q0 + lane] < 0);
    uint32_t todo = __ballot_sync(0xffffffffu, need);
    while (todo) {
      const int64_t qi = q0 + __ffs(todo) - 1;
      todo &= todo - 1;
      walk_query(A, qi, s_stack[warp], &cand, &pge1, &sum_p, &status);
    }
  }
  flush_counters(A, cand, pge1, sum_p, status);
}

// The draws the warp pass could not decide in FP32, one thread each: the
// exact FP64 P_pair in the oracle's operation order (with P(j|i) when j
// sees i), the draw and, if accepted, the pair record.
__global__ void __launch_bounds__(XT) pairs_exact_kernel(PairKArgs A) {
  const Sorted& so = A.so;
  const PairArgs& P = A.a;
  const int kern = P.kernel;
  const int lane = threadIdx.x & 31;
  const unsigned long long nd_all = A.st->n_deferred;
  const int64_t nd = (int64_t)(nd_all < (unsigned long long)P.pair_cap ? nd_all : P.pair_cap);
  const double box = P.box, half = 0.5 * P.box;
  unsigned long long pge1 = 0;
  double sum_p = 0.0;
  uint32_t status = 0;
  const int64_t stride = (int64_t)gridDim.x * XT;
  for (int64_t base = blockIdx.x * (int64_t)XT + (threadIdx.x & ~31); base < nd; base += stride) {
    const int64_t d = base + lane;
    bool acc = false;
    PairRec rec;
    if (d < nd) {
      const int2 r = P.deferred[d];
      const int64_t s = r.x, j = r.y & 0x7fffffff;
      const bool sees = r.y < 0;
      const uint32_t idi = so.id[s], idj = so.id[j];
      const Halo& H = A.f.halos[so.halo[s]];
      const bool i_is_a = idi < idj;
      const uint32_t a = i_is_a ? idi : idj, b = i_is_a ? idj : idi;
      const U4 w = philox10((uint32_t)H.seed, (uint32_t)(H.seed >> 32), H.step, 0u, a, b);
      const double r2 = sep2(so.x[s], so.y[s], so.z[s], so.x[j], so.y[j], so.z[j], box, half);
      const double ddx = so.vx[s] - so.vx[j], ddy = so.vy[s] - so.vy[j],
                   ddz = so.vz[s] - so.vz[j];
      const double vrel = sqrt((ddx * ddx + ddy * ddy) + ddz * ddz);
      const double sg = sigma_over_m(H.sigma_kind, H.sigma0, H.w, P.table, vrel);
      const double hi = so.h[s];
      double p_i, p_j = 0.0;
      if (P.ov.na > 0) {
        // kernel overlap (Eq. 15): the same g_ij for both directed terms
        const double g = overlap_g(P.ov, hi, so.h[j], r2);
        p_i = ((((0.5 * so.m[j]) * sg) * vrel) * g) * so.dt[s];
        if (sees) p_j = ((((0.5 * so.m[s]) * sg) * vrel) * g) * so.dt[j];
      } else {
        const double qq = sqrt(r2) / hi;
        p_i = ((((0.5 * so.m[j]) * sg) * vrel) * (kernel_norm(kern, hi) *
                                                   kernel_shape(kern, qq))) * so.dt[s];
        if (sees) {
          const double hj = so.h[j];
          const double qj = sqrt(r2) / hj;
          p_j = ((((0.5 * so.m[s]) * sg) * vrel) * (kernel_norm(kern, hj) *
                                                     kernel_shape(kern, qj))) * so.dt[j];
        }
      }
      const double pp = i_is_a ? (p_i + p_j) : (p_j + p_i);
      if (pp >= 1.0) ++pge1;
      sum_p += pp;
      if (unit53(w.x, w.y) < pp) {
        acc = true;
        rec.ord = ((unsigned long long)w.z << 32) | (unsigned long long)w.w;
        rec.a = a;
        rec.b = b;
        const int32_t oi = so.orig[s], oj = so.orig[j];
        rec.ia = i_is_a ? oi : oj;
        rec.ib = i_is_a ? oj : oi;
      }
    }
    const uint32_t m = __ballot_sync(0xffffffffu, acc);
    if (m) {
      unsigned long long at0 = 0;
      const int leader = __ffs(m) - 1;
      if (lane == leader) at0 = atomicAdd(&A.st->n_acc, (unsigned long long)__popc(m));
      at0 = __shfl_sync(0xffffffffu, at0, leader);
      if (acc) {
        const unsigned long long at = at0 + __popc(m & ((1u << lane) - 1u));
        if (at < (unsigned long long)P.pair_cap) A.pairs[at] = rec;
        else status |= ST_ERR_PAIR_OVERFLOW;
      }
    }
  }
  flush_counters(A, 0ull, pge1, sum_p, status);
}

// Eq. 18 limits of the queries with complete neighbour lists, one thread each:
// the exact maximum of v sigma/m over the kept candidates (over the whole
// list when there were more), or the FP32 maximum in the split form.
__global__ void __launch_bounds__(XT) limits_kernel(PairKArgs A) {
  if (A.a.ov.na > 0) return;  // the tree walks wrote every limit
  const int64_t n_act = (int64_t)A.st->n_active;
  const int64_t stride = (int64_t)gridDim.x * XT;
  for (int64_t qi = blockIdx.x * (int64_t)XT + threadIdx.x; qi < n_act; qi += stride) {
    const int cnt = A.nb_count[qi];
    if (cnt < 0) continue;  // the tree-walk kernel wrote this limit
    const int64_t s = A.act_list[qi];
    double vs = 0.0;
    if (A.a.split) {
      vs = (double)A.a.lim_g[qi];
    } else {
      const int nc = A.a.lim_cnt[qi];
      if (nc >= 0) {
        for (int r = 0; r < nc; ++r) vs = fmax(vs, exact_g(A, s, A.a.lim_cand[qi * LIM_CAND + r]));
      } else {
        const int32_t* row = A.nb_list + qi * (int64_t)A.nb_stride;
        for (int k = 0; k < cnt; ++k) vs = fmax(vs, exact_g(A, s, row[k]));
      }
    }
    write_limit(A, s, vs);
  }
}

}  // namespace

int launch_pairs(const Sorted& so, const Forest& f, int64_t n, const int32_t* act_list,
                 const int32_t* nb_list, const int32_t* nb_count, int nb_stride,
                 const PairArgs& a, PairRec* pairs, double* dtlim_user, DevStats* st, int* work,
                 int sms, const LaunchTuning& t, cudaStream_t s) {
  if (n <= 0) return 0;
  PairKArgs k{so, f, n, act_list, nb_list, nb_count, nb_stride, a, pairs, dtlim_user, st, work,
              t.pairs_chunk};
  int64_t blocks = (int64_t)sms * t.pairs_blocks_per_sm;
  const int64_t need = (n + PW - 1) / PW;
  if (blocks > need) blocks = need;
  pairs_kernel<<<(unsigned)blocks, PT, 0, s>>>(k);
  pairs_walk_kernel<<<(unsigned)sms, PT, 0, s>>>(k);
  pairs_exact_kernel<<<(unsigned)(sms * 4), XT, 0, s>>>(k);
  int64_t lb = (n + XT - 1) / XT;
  if (lb > (int64_t)sms * 8) lb = (int64_t)sms * 8;
  limits_kernel<<<(unsigned)lb, XT, 0, s>>>(k);
  return 4;
}

}  // namespace sidm
