// Search radius h_SI of every active particle (Sec. 4.2: N_ngb = 32 +- 5,
// Sec. 4.5: iterative search over all particles, active and inactive), and
// its neighbour list N(i) = {j != i : r_ij^2 < h_i^2}.
//
// One warp per active particle i:
//   1. Bounds.  Every separation is first taken in FP32 from the FP32 copies
//      of the positions.  Those copies lie within 2^-24 |x| of the FP64
//      values, so the true separation r lies in [lo, hi] with
//      lo = r32 (1 - 2^-20) - E, hi = r32 (1 + 2^-20) + E,
//      E = 2^-21 (max|x_i| + L) + 2^-21 r32 (generous over the rounding of
//      coordinates, differences, squares, sums and the square root).
//   2. Radius T: in the key-order window of 256 particles around i, the
//      K-th smallest upper bound hi, K = N_ngb + tol + 1 (found by
//      bisection on the float bit pattern).  K particles have r <= T.
//   3. Gather: every particle with lo <= T goes into a shared-memory list as
//      (lo, hi, index).  If more than SEARCH_CAP qualify, T shrinks
//      (count-verified) and the gather repeats.
//   4. Bisection on the neighbour count c(h) = #{j : r^2 < h h}, in the same
//      order of exactly rounded operations from the same start h0 as a
//      direct count: for h h > T^2 the count is at least K (above the band);
//      otherwise entries with hi below h count, entries with lo at or above h
//      do not, and the rare entries whose bounds straddle h are decided on the
//      exact FP64 r^2, computed in the fixed order (dx dx + dy dy) + dz dz.
//   5. The members of N(i) are written to the neighbour list of i (when the
//      list is complete and fits); otherwise the list is marked for a direct
//      tree walk in the pair kernel.
// No result depends on the FP32 values: they only decide what is certain.
#include "traverse.cuh"

namespace sidm {

namespace {

constexpr int SW = 4;                 // warps per block
constexpr int ST = SW * WARP;
constexpr int NWIN = 8;               // window of 8 * 32 particles
constexpr int CHUNK = 4;              // queries per work-counter increment
constexpr float REL = 9.5367431640625e-07f;   // 2^-20
constexpr float ABS = 4.76837158203125e-07f;  // 2^-21

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
  int32_t* nb_list;     // [n_act][nb_stride]
  int32_t* nb_count;    // [n_act]: count, or -1 (walk the tree)
  int nb_stride;
  DevStats* st;
  int* work;
};

__device__ __forceinline__ int warp_sum(int v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

struct Bounds {
  float lo, hi;
};

// Separation bounds of particle j from the query (FP32), see the header.
__device__ __forceinline__ Bounds sep_bounds(const float4& q, const float4& b, float box,
                                             float eq) {
  const float r = sqrtf(sep2f(q, b, box));
  const float e = eq + ABS * r;
  Bounds o;
  o.lo = fmaxf(r * (1.0f - REL) - e, 0.0f);
  o.hi = r * (1.0f + REL) + e;
  return o;
}

__global__ void __launch_bounds__(ST) search_kernel(SearchArgs A) {
  __shared__ float s_lo[SW][SEARCH_CAP];
  __shared__ float s_hi[SW][SEARCH_CAP];
  __shared__ int32_t s_j[SW][SEARCH_CAP];
  __shared__ int s_stack[SW][SEARCH_STACK];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  float* lst_lo = s_lo[warp];
  float* lst_hi = s_hi[warp];
  int32_t* lst_j = s_j[warp];
  int* stack = s_stack[warp];
  const Sorted& so = A.so;
  const int64_t n = A.n;
  const int64_t n_act = (int64_t)A.st->n_active;
  const double box = A.box, half = 0.5 * A.box;
  const float boxf = (float)A.box;
  const int K = A.n_ngb + A.tol + 1;
  const int lo_band = A.n_ngb - A.tol, hi_band = A.n_ngb + A.tol;
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
    const int64_t qi = q++;
    const int64_t s = A.act_list[qi];
    const double xi = so.x[s], yi = so.y[s], zi = so.z[s];
    const float4 fi = so.f[s];
    const float eq = ABS * (fmaxf(fmaxf(fabsf(fi.x), fabsf(fi.y)), fabsf(fi.z)) + boxf);
    double h;
    int len = 0;
    float T = INFINITY;  // gather radius (all j with lo <= T are in the list)

    if (A.fixed_h > 0.0) {
      h = A.fixed_h;
      // gather N(i) directly with radius h
      T = __double2float_ru(h) * (1.0f + REL);
    } else if (n - 1 >= K) {
      // ---- 2. radius T from the key-order window
      const int64_t W = (int64_t)NWIN * 32 < n ? (int64_t)NWIN * 32 : n;
      int64_t w0 = s - W / 2;
      if (w0 > n - W) w0 = n - W;
      if (w0 < 0) w0 = 0;
      float hv[NWIN];
      float vmin = INFINITY, vmax = 0.0f;
#pragma unroll
      for (int k = 0; k < NWIN; ++k) {
        hv[k] = INFINITY;
        const int64_t j = w0 + k * 32 + lane;
        if (j < w0 + W && j != s) {
          hv[k] = sep_bounds(fi, so.f[j], boxf, eq).hi;
          vmin = fminf(vmin, hv[k]);
          vmax = fmaxf(vmax, hv[k]);
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        vmin = fminf(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
        vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
      }
      // smallest T (bit pattern bisection) with #{hv <= T} >= K
      uint32_t blo = __float_as_uint(vmin), bhi = __float_as_uint(vmax);
      if (blo > 0) --blo;                        // count(blo) < K unless ties
      for (int it = 0; it < 40 && bhi - blo > 1; ++it) {
        const uint32_t mid = blo + ((bhi - blo) >> 1);
        const float tm = __uint_as_float(mid);
        int c = 0;
#pragma unroll
        for (int k = 0; k < NWIN; ++k) c += hv[k] <= tm ? 1 : 0;
        c = warp_sum(c);
        if (c >= K) bhi = mid; else blo = mid;
      }
      T = __uint_as_float(bhi);
    }

    // ---- 3. gather every j with lo <= T (shrink T while the list overflows)
    bool complete = true;
    for (int attempt = 0;; ++attempt) {
      len = 0;
      const float Tg = T * (1.0f + REL);
      // covers every particle whose lower bound can be <= Tg (see the header)
      const float rad = (T + 2.0f * eq) * (1.0f + 4.0f * REL);
      const float rad2 = rad < INFINITY ? rad * rad : INFINITY;
      const bool ok = traverse(A.t, fi, rad2, boxf, stack, [&](int leaf) {
        const int64_t j = (int64_t)leaf * LEAF + lane;
        bool keep = false;
        Bounds b{0.f, 0.f};
        if (j < n && j != s) {
          b = sep_bounds(fi, so.f[j], boxf, eq);
          keep = b.lo <= Tg;
        }
        const uint32_t m = __ballot_sync(0xffffffffu, keep);
        if (keep) {
          const int at = len + __popc(m & lt);
          if (at < SEARCH_CAP) {
            lst_lo[at] = b.lo;
            lst_hi[at] = b.hi;
            lst_j[at] = (int32_t)j;
          }
        }
        len += __popc(m);
      });
      __syncwarp();
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
        int c = 0;
        const float radn = (Tn + 2.0f * eq) * (1.0f + 4.0f * REL);
        const bool ok2 = traverse(A.t, fi, radn * radn, boxf, stack, [&](int leaf) {
          const int64_t j = (int64_t)leaf * LEAF + lane;
          bool in = false;
          if (j < n && j != s) in = sep_bounds(fi, so.f[j], boxf, eq).hi <= Tn;
          c += __popc(__ballot_sync(0xffffffffu, in));
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

    // ---- 4. bisection on the exact neighbour count
    const double R2 = (double)T * (double)T;   // K particles have r^2 < R2 (exact product)
    auto exact_r2 = [&](int k) {
      const int64_t j = lst_j[k];
      return sep2(xi, yi, zi, so.x[j], so.y[j], so.z[j], box, half);
    };
    // count of r^2 < h h over the list (exact), for h h <= R2
    auto count_below = [&](double hh, float hl, float hu) {
      int c = 0;
      for (int k = lane; k < len; k += 32) {
        const float lo = lst_lo[k], hi = lst_hi[k];
        if (hi < hl) ++c;
        else if (lo < hu) c += exact_r2(k) < hh ? 1 : 0;
      }
      return warp_sum(c);
    };
    if (!(A.fixed_h > 0.0)) {
      h = h0;
      double blo = 0.0, bhi = 0.0;
      bool have_hi = false, conv = false;
      for (int it = 0; it < BISECT_MAX_EVALS; ++it) {
        const double hh = h * h;
        int c;
        if (n - 1 >= K && hh > R2) {
          c = hi_band + 1;
        } else {
          c = count_below(hh, __double2float_rd(h), __double2float_ru(h));
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
    }

    // ---- 5. neighbour list
    const double hh = h * h;
    const float hl = __double2float_rd(h), hu = __double2float_ru(h);
    int* out = A.nb_list + qi * (int64_t)A.nb_stride;
    int cnt = -1;
    const bool list_covers = complete && (n - 1 < K || A.fixed_h > 0.0 || hh <= R2);
    if (list_covers) {
      cnt = 0;
      for (int k0 = 0; k0 < len; k0 += 32) {
        const int k = k0 + lane;
        bool in = false;
        if (k < len) {
          const float lo = lst_lo[k], hi = lst_hi[k];
          if (hi < hl) in = true;
          else if (lo < hu) in = exact_r2(k) < hh;
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
      so.hb[s] = make_float2(hl, hu);
      A.h_user[so.orig[s]] = h;
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

int launch_search(const Sorted& so, const Tree& t, int64_t n, const int32_t* act_list,
                  const StepParams* p, double box, int n_ngb, int tol, double fixed_h,
                  double* h_user, int32_t* nb_list, int32_t* nb_count, int nb_stride,
                  DevStats* st, int* work, int sms, cudaStream_t s) {
  if (n <= 0) return 0;
  SearchArgs a{so, t, n, act_list, p, box, n_ngb, tol, fixed_h, h_user,
               nb_list, nb_count, nb_stride, st, work};
  int64_t blocks = (int64_t)sms * 8;
  const int64_t need = (n + SW - 1) / SW;
  if (blocks > need) blocks = need;
  search_kernel<<<(unsigned)blocks, ST, 0, s>>>(a);
  return 1;
}

}  // namespace sidm
