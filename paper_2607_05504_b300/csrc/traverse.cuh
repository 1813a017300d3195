// Warp-cooperative traversal of the 32-ary box tree: one warp serves one
// query sphere; at an internal node every lane tests one child box, at a
// leaf every lane holds one particle.  Box tests are conservative (FP32
// boxes rounded outward, radius inflated by the caller), so no particle
// whose exact FP64 separation qualifies is ever pruned.
#pragma once

#include "sidm_internal.cuh"

namespace sidm {

__device__ __forceinline__ float axis_gap2(float lo, float hi, float q, float box) {
  float d = fmaxf(fmaxf(lo - q, q - hi), 0.f);
  if (box > 0.f) {
    const float q1 = q + box, q2 = q - box;
    d = fminf(d, fmaxf(fmaxf(lo - q1, q1 - hi), 0.f));
    d = fminf(d, fmaxf(fmaxf(lo - q2, q2 - hi), 0.f));
  }
  return d * d;
}

__device__ __forceinline__ bool box_hits(const float4& lo, const float4& hi, float qx, float qy,
                                         float qz, float rad2, float box) {
  return axis_gap2(lo.x, hi.x, qx, box) + axis_gap2(lo.y, hi.y, qy, box) +
             axis_gap2(lo.z, hi.z, qz, box) <= rad2;
}

// FP32 squared separation with a minimum image taken as min(|d|, L - |d|).
__device__ __forceinline__ float sep2f(const float4& a, const float4& b, float box) {
  float dx = fabsf(b.x - a.x), dy = fabsf(b.y - a.y), dz = fabsf(b.z - a.z);
  if (box > 0.f) {
    dx = fminf(dx, box - dx);
    dy = fminf(dy, box - dy);
    dz = fminf(dz, box - dz);
  }
  return dx * dx + dy * dy + dz * dz;
}

// Squared FP32 test radius covering radius R around a query at q: the FP32
// copies of the coordinates are within 2^-24 |x| of the FP64 values, so a
// particle within R in FP64 is within (R + eps)(1 + 2^-20) in FP32 with
// eps = 2^-20 (max|q| + R + L).
__device__ __forceinline__ float test_radius2(double R, const float4& q, float box) {
  const float Rf = __double2float_ru(R);
  const float qm = fmaxf(fmaxf(fabsf(q.x), fabsf(q.y)), fabsf(q.z));
  const float eps = (qm + Rf + box) * 9.5367431640625e-07f;  // 2^-20
  const float r = (Rf + eps) * (1.0f + 9.5367431640625e-07f);
  return r * r;
}

// Visits every leaf of halo H whose box meets the sphere; leaf_fn(leaf) is
// called by the whole warp with the halo-local leaf index (particles
// H.start + 32 leaf + lane, below H.start + H.n).  Returns false if the
// stack overflowed (visit incomplete).
template <class LeafFn>
__device__ __forceinline__ bool traverse(const Forest& f, const Halo& H, const float4& q,
                                         float rad2, float box, int* stack, LeafFn&& leaf_fn) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  if (H.levels <= 0) return true;
  int top = 1;
  if (lane == 0) stack[0] = (H.levels - 1) << 28;
  __syncwarp();
  bool ok = true;
  while (top > 0) {
    --top;
    const int node = stack[top];
    __syncwarp();
    const int level = node >> 28, idx = node & 0x0FFFFFFF;
    if (level == 0) {
      leaf_fn(idx);
    } else {
      const int64_t child = (int64_t)idx * 32 + lane;
      bool hit = false;
      if (child < H.node_cnt[level - 1]) {
        const int64_t c = H.node_off[level - 1] + child;
        hit = box_hits(f.lo[c], f.hi[c], q.x, q.y, q.z, rad2, box);
      }
      const uint32_t m = __ballot_sync(0xffffffffu, hit);
      const int k = __popc(m);
      if (top + k > SEARCH_STACK) {
        ok = false;
        break;
      }
      if (hit) stack[top + __popc(m & lt)] = ((level - 1) << 28) | (int)child;
      top += k;
      __syncwarp();
    }
  }
  __syncwarp();
  return ok;
}

}  // namespace sidm
