// Candidate pairs, their probabilities and the one draw per unordered pair.
//
// One warp per active particle i walks the tree with radius h_i and takes
// every j != i with exact r^2 < h_i h_i (its neighbour set N(i)).  For each:
//   * (v sigma/m) = |v_i - v_j| sigma/m(|v_i - v_j|) enters the maximum of
//     Eq. 9 (start-of-step velocities);
//   * i owns the unordered pair unless j is active, sees i (r^2 < h_j h_j)
//     and has the smaller id -- so that each pair is evaluated exactly once;
//   * the owner forms P_pair = P(i|j) + [j active, i in N(j)] P(j|i) with
//     P(i|j) = 1/2 m_j (sigma/m) |v_i - v_j| W(r, h_i) dt_i (Eqs. 2-4);
//   * Philox-4x32-10 with key (seed) and counter (step, 0, min id, max id)
//     gives u = 53 bits / 2^53 and the 64-bit order key; u < P_pair accepts.
// Accepted pairs are appended to a buffer; the Eq. 9 limit of i is written.
#include "traverse.cuh"

namespace sidm {

namespace {

constexpr int PW = 4;
constexpr int PT = PW * WARP;
constexpr int CHUNK = 8;

struct PairKArgs {
  Sorted so;
  Tree t;
  int64_t n;
  const int32_t* act_list;
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
__device__ __forceinline__ double warp_sumd(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(PT) pairs_kernel(PairKArgs A) {
  __shared__ int s_stack[PW][SEARCH_STACK];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  int* stack = s_stack[warp];
  const Sorted& so = A.so;
  const PairArgs& P = A.a;
  const int64_t n = A.n;
  const int64_t n_act = (int64_t)A.st->n_active;
  const double box = P.box, half = 0.5 * P.box;
  const float boxf = (float)P.box;
  const uint32_t k0 = (uint32_t)P.seed, k1 = (uint32_t)(P.seed >> 32);
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
    const int64_t s = A.act_list[q++];
    const double xi = so.x[s], yi = so.y[s], zi = so.z[s];
    const double vxi = so.vx[s], vyi = so.vy[s], vzi = so.vz[s];
    const double mi = so.m[s], hi = so.h[s], dti = so.dt[s];
    const uint32_t idi = so.id[s];
    const int32_t oi = so.orig[s];
    const float4 fi = so.f[s];
    const double hhi = hi * hi;
    const double wni = kernel_norm(P.kernel, hi);
    double vs_max = 0.0;
    const float rad2 = test_radius2(hi, fi, boxf);
    const bool ok = traverse(A.t, fi, rad2, boxf, stack, [&](int leaf) {
      const int64_t j = (int64_t)leaf * LEAF + lane;
      bool acc = false;
      PairRec rec;
      if (j < n && j != s && sep2f(fi, so.f[j], boxf) <= rad2) {
        const double r2 = sep2(xi, yi, zi, so.x[j], so.y[j], so.z[j], box, half);
        if (r2 < hhi) {
          const double dvx = vxi - so.vx[j], dvy = vyi - so.vy[j], dvz = vzi - so.vz[j];
          const double vrel = sqrt((dvx * dvx + dvy * dvy) + dvz * dvz);
          const double sg = sigma_over_m(P.sigma_kind, P.sigma0, P.w, vrel);
          vs_max = fmax(vs_max, vrel * sg);
          const uint32_t idj = so.id[j];
          const bool actj = so.act[j] != 0;
          double hj = 0.0;
          bool j_sees_i = false;
          if (actj) {
            hj = so.h[j];
            j_sees_i = r2 < hj * hj;
          }
          if (!(j_sees_i && idj < idi)) {
            const double mj = so.m[j];
            const double qi = sqrt(r2) / hi;
            const double p_i = ((((0.5 * mj) * sg) * vrel) * (wni * kernel_shape(P.kernel, qi))) * dti;
            double p_j = 0.0;
            if (j_sees_i) {
              const double qj = sqrt(r2) / hj;
              p_j = ((((0.5 * mi) * sg) * vrel) *
                     (kernel_norm(P.kernel, hj) * kernel_shape(P.kernel, qj))) * so.dt[j];
            }
            const bool i_is_a = idi < idj;
            const double pp = i_is_a ? (p_i + p_j) : (p_j + p_i);
            ++cand;
            if (pp >= 1.0) ++pge1;
            sum_p += pp;
            const uint32_t a = i_is_a ? idi : idj, b = i_is_a ? idj : idi;
            const U4 w = philox10(k0, k1, P.step, 0u, a, b);
            const double u = unit53(w.x, w.y);
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
    });
    if (!ok) status |= ST_ERR_STACK;
    vs_max = warp_maxd(vs_max);
    if (lane == 0) {
      const double den = (mi * wni) * vs_max;
      A.dtlim_user[oi] = vs_max > 0.0 ? (P.c_sidm * 2.0) / den : INFINITY;
    }
  }
  // per-warp reduction of the counters
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

int launch_pairs(const Sorted& so, const Tree& t, int64_t n, const int32_t* act_list,
                  const PairArgs& a, PairRec* pairs, double* dtlim_user, DevStats* st, int* work,
                  cudaStream_t s) {
  if (n <= 0) return 0;
  PairKArgs k{so, t, n, act_list, a, pairs, dtlim_user, st, work};
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t blocks = (int64_t)sms * 8;
  const int64_t need = (n + PW - 1) / PW;
  if (blocks > need) blocks = need;
  pairs_kernel<<<(unsigned)blocks, PT, 0, s>>>(k);
  return 1;
}

}  // namespace sidm
