// Warp-cooperative traversal of the 32-ary box tree: one warp serves one
// query sphere; at an internal node every lane tests one child box, at a
// leaf every lane holds one particle.  Box tests are conservative (FP32
// boxes rounded outward, radius inflated by the caller), so no particle
// whose exact FP64 separation qualifies is ever pruned.
#pragma once

#include "sidm_internal.cuh"

namespace sidm {

template <bool PERIODIC>
__device__ __forceinline__ float axis_gap2(float lo, float hi, float q, float box) {
  float d = fmaxf(fmaxf(lo - q, q - hi), 0.f);
  if (PERIODIC) {
    const float q1 = q + box, q2 = q - box;
    d = fminf(d, fmaxf(fmaxf(lo - q1, q1 - hi), 0.f));
    d = fminf(d, fmaxf(fmaxf(lo - q2, q2 - hi), 0.f));
  }
  return d * d;
}

template <bool PERIODIC>
__device__ __forceinline__ bool box_hits(const float4& lo, const float4& hi, const float4& q,
                                         float rad2, float box) {
  return axis_gap2<PERIODIC>(lo.x, hi.x, q.x, box) + axis_gap2<PERIODIC>(lo.y, hi.y, q.y, box) +
             axis_gap2<PERIODIC>(lo.z, hi.z, q.z, box) <= rad2;
}

// FP32 squared separation with a minimum image taken as min(|d|, L - |d|).
template <bool PERIODIC>
__device__ __forceinline__ float sep2f(const float4& a, const float4& b, float box) {
  float dx = fabsf(b.x - a.x), dy = fabsf(b.y - a.y), dz = fabsf(b.z - a.z);
  if (PERIODIC) {
    dx = fminf(dx, box - dx);
    dy = fminf(dy, box - dy);
    dz = fminf(dz, box - dz);
  }
  // fused: two roundings fewer than the plain expression, inside the same
  // error bound
  return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, dx * dx));
}

// The same with the boundary kind known only at run time.
__device__ __forceinline__ float sep2f(const float4& a, const float4& b, float box) {
  return box > 0.f ? sep2f<true>(a, b, box) : sep2f<false>(a, b, box);
}

// Visits every leaf of halo H whose box meets the sphere (depth first over
// the internal nodes, one stack entry at a time: the stack never holds more
// than 31 entries per level plus one).  leaf_fn(k, valid, pj) is called by the whole warp for
// each leaf reached: lane l holds the halo-local particle k = 32 leaf + l,
// valid when k < H.n, with FP32 position pj (hpos = key-order FP32
// positions of the halo's particles).  Returns false if the stack
// overflowed (visit incomplete).
// HMAX: the radius at a node is widened by the node's largest h (the w of
// its upper corner), the overlap walk's h_i + h_j bound; `rad` is then the
// query's own radius and rad2 is ignored.
// LB > 0: the leaves under a node are visited as soon as their boxes are
// tested, LB at a time, with their particle loads issued together (one L2
// round trip per LB leaves); leaf_fn then takes the batch as arrays,
// leaf_fn(k[LB], valid[LB], pj[LB], on[LB]) with on[b] warp-uniform (batch
// slot b holds a leaf), so that it can compute every slot before its
// ballots.  LB = 0: hit leaves go on the stack like the other nodes and
// leaf_fn(k, valid, pj) sees one leaf (smallest code).
// CAP: stack entries; the walk reports an overflow (returns false) rather
// than exceed it.
template <bool PERIODIC, bool HMAX = false, int LB = 0, int CAP = SEARCH_STACK, class LeafFn>
__device__ __forceinline__ bool traverse(const Forest& f, const Halo& H,
                                         const float4* __restrict__ hpos, const float4& q,
                                         float rad2, float box, int* stack, LeafFn&& leaf_fn,
                                         float rad = 0.0f) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  const int levels = H.levels;
  if (levels <= 0) return true;
  const int hn = (int)H.n;
  int top = 1;
  if (lane == 0) stack[0] = (levels - 1) << 28;
  __syncwarp();
  while (top > 0) {
    --top;
    const int node = stack[top];
    __syncwarp();  // read before the children overwrite the slot
    const int level = node >> 28;
    const int k = ((node & 0x0FFFFFFF) << 5) + lane;
    if (level == 0) {
      const bool valid = k < hn;
      float4 pj = make_float4(0.f, 0.f, 0.f, 0.f);
      if (valid) pj = hpos[k];
      if constexpr (LB > 0) {
        int kk[LB];
        bool vv[LB], on[LB];
        float4 pp[LB];
#pragma unroll
        for (int b = 0; b < LB; ++b) {
          kk[b] = k;
          vv[b] = b == 0 && valid;
          on[b] = b == 0;
          pp[b] = pj;
        }
        leaf_fn(kk, vv, pp, on);
      } else {
        leaf_fn(k, valid, pj);
      }
    } else {
      bool hit = false;
      if (k < (int)H.node_cnt[level - 1]) {
        const int64_t nd = H.node_off[level - 1] + k;
        const float4 lo = f.lo[nd], hi = f.hi[nd];
        float r2 = rad2;
        if (HMAX) {
          const float rr = __fmul_ru(__fadd_ru(rad, hi.w), 1.0f + 3.814697265625e-06f);
          r2 = __fmul_ru(rr, rr);
        }
        hit = box_hits<PERIODIC>(lo, hi, q, r2, box);
      }
      const uint32_t m = __ballot_sync(0xffffffffu, hit);
      bool visited = false;
      if constexpr (LB > 0) {
        if (level == 1) {
          // the children are leaves: visit the hit ones now, LB at a time
          const int lbase = (node & 0x0FFFFFFF) << 5;
          uint32_t mm = m;
          while (mm) {
            int kk[LB];
            bool on[LB], valid[LB];
            float4 pj[LB];
#pragma unroll
            for (int b = 0; b < LB; ++b) {
              on[b] = mm != 0u;                       // warp-uniform
              const int c = on[b] ? __ffs(mm) - 1 : 0;
              mm &= mm - 1u;
              kk[b] = ((lbase + c) << 5) + lane;
              valid[b] = on[b] && kk[b] < hn;
              pj[b] = valid[b] ? hpos[kk[b]] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            leaf_fn(kk, valid, pj, on);
          }
          visited = true;
        }
      }
      if (!visited) {
        const int cnt = __popc(m);
        if (top + cnt > CAP) return false;
        if (hit) stack[top + __popc(m & lt)] = ((level - 1) << 28) | k;
        top += cnt;
        __syncwarp();
      }
    }
  }
  return true;
}

}  // namespace sidm
