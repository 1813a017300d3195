// Search radius h_SI of every active particle (Sec. 4.2: "N_ngb = 32 +- 5",
// Sec. 4.5: iterative search over all particles, active and inactive).
//
// One warp per active particle i, taken from a work counter:
//   1. an upper bound R^2 on the squared distance of the K-th nearest other
//      particle, K = N_ngb + tol + 1: the K-th smallest exact squared distance
//      among the key-order window of 32*ceil((K+1)/32) particles around i
//      (K distinct particles lie within it, so the true K-th is no farther);
//   2. all particles with exact r^2 <= R^2 are gathered into shared memory
//      (FP32 box/distance filters, FP64 confirmation); if there are more than
//      SEARCH_CAP, R^2 is shrunk by a bracketed search on the count;
//   3. the bisection on the neighbour count c(h) = #{j != i : r^2 < h h}
//      runs on the gathered list.  For h h <= R^2 the list holds every
//      qualifying particle, so c(h) is exact; for h h > R^2, c(h) >= K lies
//      above the band, which is all the bisection needs to know.
// The bisection is the same sequence of exactly rounded operations from the
// same start h0 as a direct count over all particles, hence the same h.
#include "traverse.cuh"

namespace sidm {

namespace {

constexpr int SW = 4;                 // warps per block
constexpr int ST = SW * WARP;
constexpr int MAX_WIN = 8;            // window of up to 8*32 particles
constexpr int CHUNK = 8;              // queries taken per work-counter increment

struct SearchArgs {
  Sorted so;
  Tree t;
  int64_t n;
  const int32_t* act_list;
  const StepParams* p;
  double box;
  int n_ngb, tol;
  double fixed_h;
  double* h_user;
  DevStats* st;
  int* work;
};

__device__ __forceinline__ int warp_sum(int v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(ST) search_kernel(SearchArgs A) {
  __shared__ double s_list[SW][SEARCH_CAP];
  __shared__ int s_stack[SW][SEARCH_STACK];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  double* list = s_list[warp];
  int* stack = s_stack[warp];
  const Sorted& so = A.so;
  const int64_t n = A.n;
  const int64_t n_act = (int64_t)A.st->n_active;
  const double box = A.box, half = 0.5 * A.box;
  const float boxf = (float)A.box;
  const int K = A.n_ngb + A.tol + 1;
  const double h0 = A.p->h0;
  uint32_t status = 0;
  int nonconv = 0;

  int q = 0, q_end = 0;
  for (;;) {
    if (q >= q_end) {
      if (lane == 0) q = atomicAdd(A.work, CHUNK);
      q = __shfl_sync(0xffffffffu, q, 0);
      q_end = q + CHUNK;
    }
    if (q >= n_act) break;
    const int64_t s = A.act_list[q++];
    double h;
    if (A.fixed_h > 0.0) {
      h = A.fixed_h;
    } else {
      const double xi = so.x[s], yi = so.y[s], zi = so.z[s];
      const float4 fi = so.f[s];

      // ---- 1. upper bound R2 of the K-th nearest squared distance
      double R2 = INFINITY;
      if (n - 1 >= K) {
        const int nw = (K + 1 + 31) / 32;
        const int64_t W = (int64_t)nw * 32;
        int64_t w0 = s - W / 2;
        if (w0 > n - W) w0 = n - W;
        if (w0 < 0) w0 = 0;
        double v[MAX_WIN];
#pragma unroll
        for (int k = 0; k < MAX_WIN; ++k) {
          v[k] = INFINITY;
          const int64_t j = w0 + k * 32 + lane;
          if (k < nw && j < n && j != s) v[k] = sep2(xi, yi, zi, so.x[j], so.y[j], so.z[j], box, half);
        }
        int rank[MAX_WIN];
#pragma unroll
        for (int k = 0; k < MAX_WIN; ++k) rank[k] = 0;
        for (int kk = 0; kk < nw; ++kk) {
          for (int src = 0; src < 32; ++src) {
            double vv = 0.0;
#pragma unroll
            for (int k = 0; k < MAX_WIN; ++k)
              if (k == kk) vv = __shfl_sync(0xffffffffu, v[k], src);
            const int g2 = kk * 32 + src;
#pragma unroll
            for (int k = 0; k < MAX_WIN; ++k) {
              const int g = k * 32 + lane;
              if (k < nw && (vv < v[k] || (vv == v[k] && g2 < g))) ++rank[k];
            }
          }
        }
        double mine = INFINITY;
#pragma unroll
        for (int k = 0; k < MAX_WIN; ++k)
          if (k < nw && rank[k] == K - 1) mine = v[k];
        const uint32_t who = __ballot_sync(0xffffffffu, mine < INFINITY);
        const double pick = __shfl_sync(0xffffffffu, mine, who ? __ffs(who) - 1 : 0);
        R2 = who ? pick : INFINITY;
      }

      // ---- 2. gather every particle with r2 <= R2 (shrink R2 on overflow)
      int len = 0;
      bool full = false;
      double lo2 = 0.0, hi2 = R2;   // count(lo2) < K (or lo2 = 0), count(hi2) > cap
      bool have_lo = false;
      int c_hi = 0;
      for (int iter = 0; iter <= RADIUS_MAX_ITERS; ++iter) {
        len = 0;
        full = false;
        const float rad2 = (R2 < INFINITY) ? test_radius2(sqrt(R2), fi, boxf) : INFINITY;
        const double R2c = R2;
        const bool ok = traverse(A.t, fi, rad2, boxf, stack, [&](int leaf) {
          const int64_t j = (int64_t)leaf * LEAF + lane;
          bool keep = false;
          double r2 = 0.0;
          if (j < n && j != s && sep2f(fi, so.f[j], boxf) <= rad2) {
            r2 = sep2(xi, yi, zi, so.x[j], so.y[j], so.z[j], box, half);
            keep = r2 <= R2c;
          }
          const uint32_t m = __ballot_sync(0xffffffffu, keep);
          if (keep) {
            const int at = len + __popc(m & lt);
            if (at < SEARCH_CAP) list[at] = r2;
          }
          len += __popc(m);
        });
        if (!ok) { status |= ST_ERR_STACK; break; }
        __syncwarp();
        if (len <= SEARCH_CAP) break;
        full = true;
        // too many candidates: shrink the radius (bracketed, geometric)
        hi2 = R2;
        c_hi = len;
        if (iter == RADIUS_MAX_ITERS) { status |= ST_ERR_RADIUS; break; }
        if (have_lo) {
          R2 = sqrt(lo2) * sqrt(hi2);
        } else {
          R2 = hi2 * cbrt(((double)SEARCH_CAP * 0.5 / (double)c_hi) * ((double)SEARCH_CAP * 0.5 / (double)c_hi));
        }
        // if the shrunk radius holds fewer than K, raise the lower bracket
        for (int inner = 0; inner < RADIUS_MAX_ITERS; ++inner) {
          int cnt = 0;
          const float r2t = test_radius2(sqrt(R2), fi, boxf);
          const double R2t = R2;
          const bool ok2 = traverse(A.t, fi, r2t, boxf, stack, [&](int leaf) {
            const int64_t j = (int64_t)leaf * LEAF + lane;
            bool keep = false;
            if (j < n && j != s && sep2f(fi, so.f[j], boxf) <= r2t)
              keep = sep2(xi, yi, zi, so.x[j], so.y[j], so.z[j], box, half) <= R2t;
            cnt += __popc(__ballot_sync(0xffffffffu, keep));
          });
          if (!ok2) { status |= ST_ERR_STACK; break; }
          if (cnt >= K) break;
          lo2 = R2;
          have_lo = true;
          R2 = sqrt(lo2) * sqrt(hi2);
        }
      }
      if (full && len > SEARCH_CAP) status |= ST_ERR_SEARCH_CAP;
      if (len > SEARCH_CAP) len = SEARCH_CAP;

      // ---- 3. bisection on the neighbour count
      const int lo_band = A.n_ngb - A.tol, hi_band = A.n_ngb + A.tol;
      h = h0;
      double blo = 0.0, bhi = 0.0;
      bool have_hi = false, conv = false;
      for (int it = 0; it < BISECT_MAX_EVALS; ++it) {
        const double hh = h * h;
        int c;
        if (hh > R2) {
          c = hi_band + 1;  // at least K particles within h
        } else {
          int mine = 0;
          for (int k = lane; k < len; k += 32) mine += list[k] < hh ? 1 : 0;
          c = warp_sum(mine);
        }
        if (c >= lo_band && c <= hi_band) { conv = true; break; }
        if (c < lo_band) {
          blo = h;
          h = have_hi ? 0.5 * (blo + bhi) : 2.0 * h;
        } else {
          bhi = h;
          have_hi = true;
          h = 0.5 * (blo + bhi);
        }
      }
      if (!conv) ++nonconv;
      __syncwarp();
    }
    if (lane == 0) {
      so.h[s] = h;
      A.h_user[so.orig[s]] = h;
    }
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

int launch_search(const Sorted& so, const Tree& t, int64_t n, const int32_t* act_list,
                   const StepParams* p, double box, int n_ngb, int tol, double fixed_h,
                   double* h_user, DevStats* st, int* work, cudaStream_t s) {
  if (n <= 0) return 0;
  SearchArgs a{so, t, n, act_list, p, box, n_ngb, tol, fixed_h, h_user, st, work};
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t blocks = (int64_t)sms * 8;
  const int64_t need = (n + SW - 1) / SW;
  if (blocks > need) blocks = need;
  search_kernel<<<(unsigned)blocks, ST, 0, s>>>(a);
  return 1;
}

}  // namespace sidm
