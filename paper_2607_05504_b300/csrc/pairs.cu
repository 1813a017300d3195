// Candidate pairs, their probabilities and the one draw per unordered pair.
//
// One warp per active particle i, one lane per neighbour j in N(i) (from the
// neighbour list of the search kernel; a direct tree walk with radius h_i if
// the list was not complete).  For each j:
//   * (v sigma/m)(v_ij) enters the maximum of Eq. 9 (start-of-step
//     velocities);
//   * i owns the unordered pair unless j is active, sees i (r^2 < h_j^2) and
//     has the smaller id -- every pair is evaluated exactly once;
//   * the owner forms P_pair = P(i|j) + [j active, i in N(j)] P(j|i) with
//     P(i|j) = 1/2 m_j (sigma/m) |v_i - v_j| W(r, h_i) dt_i (Eqs. 2-4), and
//     draws u from Philox-4x32-10 with counter (step, 0, min id, max id);
//     u < P_pair accepts; words 2, 3 form the order key.
//
// Exactness with little FP64: P_pair is first bounded from above in FP32
// from the FP32 copies of positions, velocities, masses, dt and h (every
// factor rounded or widened upwards, then a relative margin).  Only when
// u lies below that bound (about the acceptance probability) is P_pair
// evaluated in FP64 in the oracle's operation order, and the draw decided on
// that value.  The owner test r^2 < h_j^2 and the maximum of Eq. 9 likewise
// use FP32 intervals and fall back to FP64 only where an interval straddles
// the decision.  All results equal those of a pure FP64 evaluation.
#include "traverse.cuh"

namespace sidm {

namespace {

constexpr int PW = 4;
constexpr int PT = PW * WARP;
constexpr int CHUNK = 4;
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

__device__ __forceinline__ float sigma_f(int kind, float s0, float w, float v) {
  if (kind == SIDM_SIGMA_YUKAWA) {
    const float t = 1.0f + (v * v) / (w * w);
    return s0 / (t * t);
  }
  return s0;
}

// g(v) = v sigma/m(v) for v in [vl, vu]: lower and upper bounds.  Constant
// sigma: g is increasing.  Yukawa-like: g rises up to v = w / sqrt(3) and
// falls after it.
__device__ __forceinline__ void g_bounds(int kind, float s0, float w, float vl, float vu,
                                         float* glo, float* ghi) {
  if (kind == SIDM_SIGMA_YUKAWA) {
    const float vp = w * 0.57735026918962576f;
    const float gl = vl * sigma_f(kind, s0, w, vl), gu = vu * sigma_f(kind, s0, w, vu);
    float hi;
    if (vu <= vp * (1.0f - SLACK)) hi = gu;
    else if (vl >= vp * (1.0f + SLACK)) hi = gl;
    else hi = vp * sigma_f(kind, s0, w, vp);
    *ghi = fmaxf(hi, fmaxf(gl, gu)) * (1.0f + SLACK);
    *glo = fminf(gl, gu) * (1.0f - SLACK);
  } else {
    *ghi = vu * s0 * (1.0f + SLACK);
    *glo = vl * s0 * (1.0f - SLACK);
  }
}

__global__ void __launch_bounds__(PT) pairs_kernel(PairKArgs A) {
  __shared__ int s_stack[PW][SEARCH_STACK];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  int* stack = s_stack[warp];
  const Sorted& so = A.so;
  const PairArgs& P = A.a;
  const int64_t n_act = (int64_t)A.st->n_active;
  const double box = P.box, half = 0.5 * P.box;
  const float boxf = (float)P.box;
  const int kern = P.kernel;
  const float knorm_up = __double2float_ru(kern == SIDM_KERNEL_TOPHAT
                                               ? 3.0 / (4.0 * 3.141592653589793)
                                               : 8.0 / 3.141592653589793);
  unsigned long long cand = 0, pge1 = 0;
  double sum_p = 0.0;
  uint32_t status = 0;

  int q = 0, q_end = 0;
  for (;;) {
    if (q >= q_end) {
      if (lane == 0) q = atomicAdd(A.work, CHUNK);
      q = __shfl_sync(0xffffffffu, q, 0);
      q_end = q + CHUNK;
    }
    if (q >= n_act) break;
    const int64_t qi = q++;
    const int64_t s = A.act_list[qi];
    // the query's halo: its particles, cross-section model, random key and step
    const Halo& H = A.f.halos[so.halo[s]];
    const int64_t hs = H.start, hn = H.n;
    const uint32_t k0 = (uint32_t)H.seed, k1 = (uint32_t)(H.seed >> 32);
    const uint32_t step = H.step;
    const int kind = H.sigma_kind;
    const double sigma0 = H.sigma0, wv = H.w;
    const float s0f = __double2float_ru(sigma0);
    const float wf = (float)wv;
    const double xi = so.x[s], yi = so.y[s], zi = so.z[s];
    const double vxi = so.vx[s], vyi = so.vy[s], vzi = so.vz[s];
    const double mi = so.m[s], hi = so.h[s], dti = so.dt[s];
    const uint32_t idi = so.id[s];
    const int32_t oi = so.orig[s];
    const float4 fi = so.f[s];
    const float4 vmi = so.vm[s];
    const float2 hbi = so.hb[s];
    const double hhi = hi * hi;
    const double wni = kernel_norm(kern, hi);
    const float wni_up = __double2float_ru(wni);
    const float eq = ABS * (fmaxf(fmaxf(fabsf(fi.x), fabsf(fi.y)), fabsf(fi.z)) + boxf);
    const float vmax_i = fmaxf(fmaxf(fabsf(vmi.x), fabsf(vmi.y)), fabsf(vmi.z));

    // Everything about one neighbour j (valid lanes only); the accepted pair
    // is appended by the whole warp.  Returns bounds of g = v sigma/m(v).
    auto visit = [&](int64_t j, bool valid, float* glo_out, float* ghi_out) {
      bool acc = false;
      PairRec rec;
      float glo = 0.0f, ghi = 0.0f;
      if (valid) {
        const float4 fj = so.f[j];
        const float4 vmj = so.vm[j];
        const uint32_t idj = so.id[j];
        const bool actj = so.act[j] != 0;
        // separation interval
        const float r2f = sep2f(fi, fj, boxf);
        const float r = sqrtf(r2f);
        const float e = eq + ABS * r;
        const float rlo = fmaxf(r * (1.0f - REL) - e, 0.0f);
        const float rhi = r * (1.0f + REL) + e;
        // relative speed interval
        const float dvx = vmi.x - vmj.x, dvy = vmi.y - vmj.y, dvz = vmi.z - vmj.z;
        const float vr = sqrtf(dvx * dvx + dvy * dvy + dvz * dvz);
        const float vmax_j = fmaxf(fmaxf(fabsf(vmj.x), fabsf(vmj.y)), fabsf(vmj.z));
        const float dv = 4.0f * U * (3.0f * (vmax_i + vmax_j) + vr) + 4.0f * U * vr;
        const float vl = fmaxf(vr - dv, 0.0f), vu = vr + dv;
        g_bounds(kind, s0f, wf, vl, vu, &glo, &ghi);
        if (P.split) {
          const float g = vr * sigma_f(kind, s0f, wf, vr);
          glo = ghi = g;
        }
        // does j see i?  (j active and r^2 < h_j^2: decided exactly, or in
        // FP32 by the split form, as its neighbour lists are)
        bool sees = false;
        float2 hbj = make_float2(0.f, 0.f);
        if (actj) {
          hbj = so.hb[j];
          if (P.split) {
            const float hjf = (float)so.h[j];
            sees = r2f < hjf * hjf;
          } else if (rhi < hbj.x) {
            sees = true;
          } else if (rlo < hbj.y) {
            const double hj = so.h[j];
            sees = sep2(xi, yi, zi, so.x[j], so.y[j], so.z[j], box, half) < hj * hj;
          }
        }
        if (!(sees && idj < idi)) {
          // FP32 upper bound of P_pair.  The bound holds only while no product
          // leaves the normal FP32 range; below 2^-100 the FP64 path decides.
          const float qi_lo = rlo / hbi.y;
          const float fi_up = shape_f(kern, qi_lo) * (1.0f + SLACK) + REL;
          const float t1 = 0.5f * vmj.w, t2 = t1 * ghi, t3 = t2 * wni_up, t4 = t3 * fi_up;
          float pu = t4 * fi.w;
          bool tiny = !(fminf(fminf(t1, t2), fminf(fminf(t3, t4), pu)) >= FLT_TINY);
          float pc = 0.5f * vmj.w * (vr * sigma_f(kind, s0f, wf, vr)) * wni_up *
                     shape_f(kern, r / hbi.y) * fi.w;
          if (sees) {
            const float hl = hbj.x;
            const float wnj_up = knorm_up / (hl * hl * hl) * (1.0f + SLACK);
            const float qj_lo = rlo / hbj.y;
            const float fj_up = shape_f(kern, qj_lo) * (1.0f + SLACK) + REL;
            const float s1 = 0.5f * vmi.w, s2 = s1 * ghi, s3 = s2 * wnj_up, s4 = s3 * fj_up;
            const float puj = s4 * fj.w;
            tiny = tiny || !(fminf(fminf(fminf(s1, s2), fminf(s3, s4)),
                                   fminf(puj, hl * hl * hl)) >= FLT_TINY);
            pu += puj;
            pc += 0.5f * vmi.w * (vr * sigma_f(kind, s0f, wf, vr)) * wnj_up *
                  shape_f(kern, r / hbj.y) * fj.w;
          }
          pu *= (1.0f + SLACK);
          const bool i_is_a = idi < idj;
          const uint32_t a = i_is_a ? idi : idj, b = i_is_a ? idj : idi;
          const U4 w = philox10(k0, k1, step, 0u, a, b);
          const double u = unit53(w.x, w.y);
          double pp = (double)pc;
          // plain form: FP64 whenever u is under the FP32 upper bound;
          // split form: FP64 re-test only when |P - u| < 1e-5
          const bool need64 = P.split ? (fabs((double)pc - u) < 1e-5) : (tiny || u < (double)pu);
          if (P.split && !need64) {
            if (pc >= 1.0f) ++pge1;
            if (u < pp) {
              acc = true;
              rec.ord = ((unsigned long long)w.z << 32) | (unsigned long long)w.w;
              rec.a = a;
              rec.b = b;
              const int32_t oj = so.orig[j];
              rec.ia = i_is_a ? oi : oj;
              rec.ib = i_is_a ? oj : oi;
            }
          }
          if (need64) {
            // exact FP64 probability, in the oracle's operation order
            const double r2 = sep2(xi, yi, zi, so.x[j], so.y[j], so.z[j], box, half);
            const double ddx = vxi - so.vx[j], ddy = vyi - so.vy[j], ddz = vzi - so.vz[j];
            const double vrel = sqrt((ddx * ddx + ddy * ddy) + ddz * ddz);
            const double sg = sigma_over_m(kind, sigma0, wv, vrel);
            const double mj = so.m[j];
            const double qq = sqrt(r2) / hi;
            const double p_i = ((((0.5 * mj) * sg) * vrel) * (wni * kernel_shape(kern, qq))) * dti;
            double p_j = 0.0;
            if (sees) {
              const double hj = so.h[j];
              const double qj = sqrt(r2) / hj;
              p_j = ((((0.5 * mi) * sg) * vrel) * (kernel_norm(kern, hj) * kernel_shape(kern, qj))) *
                    so.dt[j];
            }
            pp = i_is_a ? (p_i + p_j) : (p_j + p_i);
            if (pp >= 1.0) ++pge1;
            if (u < pp) {
              acc = true;
              rec.ord = ((unsigned long long)w.z << 32) | (unsigned long long)w.w;
              rec.a = a;
              rec.b = b;
              const int32_t oj = so.orig[j];
              rec.ia = i_is_a ? oi : oj;
              rec.ib = i_is_a ? oj : oi;
            }
          }
          ++cand;
          sum_p += pp;
        }
      }
      const uint32_t m = __ballot_sync(0xffffffffu, acc);
      if (m) {
        unsigned long long base = 0;
        const int leader = __ffs(m) - 1;
        if (lane == leader) base = atomicAdd(&A.st->n_acc, (unsigned long long)__popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (acc) {
          const unsigned long long at = base + __popc(m & lt);
          if (at < (unsigned long long)P.pair_cap) A.pairs[at] = rec;
          else status |= ST_ERR_PAIR_OVERFLOW;
        }
      }
      *glo_out = glo;
      *ghi_out = ghi;
    };

    // exact g = |v_i - v_j| sigma/m(|v_i - v_j|) in FP64
    auto exact_g = [&](int64_t j) {
      const double ddx = vxi - so.vx[j], ddy = vyi - so.vy[j], ddz = vzi - so.vz[j];
      const double vrel = sqrt((ddx * ddx + ddy * ddy) + ddz * ddz);
      return vrel * sigma_over_m(kind, sigma0, wv, vrel);
    };

    double vs_max = 0.0;
    const int cnt = A.nb_count[qi];
    if (cnt >= 0) {
      const int32_t* row = A.nb_list + qi * (int64_t)A.nb_stride;
      const int nr = (cnt + 31) >> 5;
      float glo[MAXR], ghi[MAXR];
      int32_t jr[MAXR];
#pragma unroll
      for (int r = 0; r < MAXR; ++r) {
        glo[r] = 0.0f;
        ghi[r] = -1.0f;
        jr[r] = -1;
        if (r < nr) {
          const int k = r * 32 + lane;
          const bool valid = k < cnt;
          const int32_t j = valid ? row[k] : -1;
          jr[r] = j;
          visit(j, valid, &glo[r], &ghi[r]);
          if (!valid) ghi[r] = -1.0f;
        }
      }
      // exact maximum of g: only j whose upper bound reaches the largest lower bound
      float mlo = 0.0f;
#pragma unroll
      for (int r = 0; r < MAXR; ++r) mlo = fmaxf(mlo, glo[r]);
      mlo = warp_maxf(mlo);
      double mine = 0.0;
#pragma unroll
      for (int r = 0; r < MAXR; ++r)
        if (jr[r] >= 0 && ghi[r] >= mlo) mine = fmax(mine, P.split ? (double)glo[r] : exact_g(jr[r]));
      vs_max = warp_maxd(mine);
    } else {
      // direct walk with radius h_i (list incomplete): exact membership
      const float rad = (__double2float_ru(hi) + 2.0f * eq) * (1.0f + 4.0f * REL);
      double mine = 0.0;
      const bool ok = traverse(A.f, H, fi, rad * rad, boxf, stack, [&](int leaf) {
        const int64_t jl = (int64_t)leaf * LEAF + lane;
        const int64_t j = hs + jl;
        bool in = false;
        if (jl < hn && j != s) {
          const float r = sqrtf(sep2f(fi, so.f[j], boxf));
          const float e = eq + ABS * r;
          const float rlo = fmaxf(r * (1.0f - REL) - e, 0.0f);
          if (P.split) {
            const float hf = (float)hi;
            in = r * r < hf * hf;
          } else if (rlo < hbi.y) {
            in = sep2(xi, yi, zi, so.x[j], so.y[j], so.z[j], box, half) < hhi;
          }
        }
        float gl, gh;
        visit(j, in, &gl, &gh);
        if (in) mine = fmax(mine, P.split ? (double)gl : exact_g(j));
      });
      if (!ok) status |= ST_ERR_STACK;
      vs_max = warp_maxd(mine);
    }
    if (lane == 0) {
      const double den = (mi * wni) * vs_max;
      A.dtlim_user[oi] = vs_max > 0.0 ? (P.c_sidm * 2.0) / den : INFINITY;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    cand += __shfl_xor_sync(0xffffffffu, cand, o);
    pge1 += __shfl_xor_sync(0xffffffffu, pge1, o);
  }
  sum_p = warp_sumd(sum_p);
  status = __reduce_or_sync(0xffffffffu, status);
  if (lane == 0) {
    if (cand) atomicAdd(&A.st->n_cand, cand);
    if (pge1) {
      atomicAdd(&A.st->n_pge1, pge1);
      status |= ST_P_GE_1;
    }
    if (sum_p != 0.0) atomicAdd(&A.st->sum_p, sum_p);
    if (status) atomicOr(&A.st->status, status);
  }
}

}  // namespace

int launch_pairs(const Sorted& so, const Forest& f, int64_t n, const int32_t* act_list,
                 const int32_t* nb_list, const int32_t* nb_count, int nb_stride,
                 const PairArgs& a, PairRec* pairs, double* dtlim_user, DevStats* st, int* work,
                 int sms, cudaStream_t s) {
  if (n <= 0) return 0;
  PairKArgs k{so, f, n, act_list, nb_list, nb_count, nb_stride, a, pairs, dtlim_user, st, work};
  int64_t blocks = (int64_t)sms * 8;
  const int64_t need = (n + PW - 1) / PW;
  if (blocks > need) blocks = need;
  pairs_kernel<<<(unsigned)blocks, PT, 0, s>>>(k);
  return 1;
}

}  // namespace sidm
