// Per-step neighbour structure: bounding box, spatial keys, key-order copy of
// the particle state, and a 32-ary tree of conservative FP32 boxes over runs
// of 32 key-consecutive particles.
//
// The structure replaces the paper's dedicated DM-only octree (Sec. 4.3): it
// is rebuilt every step from scratch (sort + linear passes), so it needs no
// drifted bounds.  Its only role is to prune the neighbour search; every
// result of the step is independent of the particle order it produces.
#include "sidm_internal.cuh"

namespace sidm {

namespace {

constexpr int BT = 256;

__device__ __forceinline__ double warp_min(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_minf(float v) {
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_maxf(float v) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__global__ void bbox_init_kernel(unsigned long long* mm) {
  if (threadIdx.x < 3) mm[threadIdx.x] = ~0ull;
  else if (threadIdx.x < 6) mm[threadIdx.x] = 0ull;
}

__global__ void __launch_bounds__(BT) bbox_kernel(const double* __restrict__ pos, int64_t n,
                                                  unsigned long long* mm) {
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = blockIdx.x * (int64_t)BT + threadIdx.x; i < n; i += (int64_t)gridDim.x * BT) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double x = pos[3 * i + k];
      lo[k] = fmin(lo[k], x);
      hi[k] = fmax(hi[k], x);
    }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    lo[k] = warp_min(lo[k]);
    hi[k] = warp_max(hi[k]);
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (lo[k] <= hi[k]) {
        atomicMin(&mm[k], dbl_to_ordered(lo[k]));
        atomicMax(&mm[3 + k], dbl_to_ordered(hi[k]));
      }
    }
  }
}

// Start radius h0 = l_ext * 2^-e (e from the host: the largest e with
// 8^e N_ngb <= 4 n), and the key transform parameters.
__global__ void params_kernel(const unsigned long long* mm, StepParams* p, double box, int e) {
  if (threadIdx.x != 0) return;
  double lo[3], hi[3];
  for (int k = 0; k < 3; ++k) {
    lo[k] = ordered_to_dbl(mm[k]);
    hi[k] = ordered_to_dbl(mm[3 + k]);
    p->lo[k] = lo[k];
    p->hi[k] = hi[k];
  }
  double l_ext = box;
  if (!(box > 0.0)) {
    l_ext = 0.0;
    for (int k = 0; k < 3; ++k) l_ext = fmax(l_ext, hi[k] - lo[k]);
  }
  p->l_ext = l_ext;
  p->h0 = ldexp(l_ext, -e);
  float r2 = 0.f;
  for (int k = 0; k < 3; ++k) {
    p->centre[k] = (float)(0.5 * (lo[k] + hi[k]));
    const float d = (float)(hi[k] - lo[k]);
    r2 += d * d;
  }
  const float R = 0.5f * sqrtf(r2) * 1.001f + 1e-30f;
  const float sc = R * (1.0f / 1024.0f);
  p->key_radius = R;
  p->key_scale = sc;
  p->key_inv_norm = 1.0f / asinhf(R / sc);
}

__device__ __forceinline__ uint32_t spread10(uint32_t v) {
  v &= 0x3FFu;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

// 30-bit Morton key.  Periodic box: 1024 cells per axis.  Open boundaries:
// the offset from the box centre is compressed radially by
// asinh(r/s)/asinh(R/s) (s = R/1024) before 1024 cells per axis, so that
// cells stay small relative to the interparticle spacing from the dense
// centre of a halo to its outskirts.  Keys only shape the traversal cost.
__global__ void __launch_bounds__(BT) keys_kernel(const double* __restrict__ pos, int64_t n,
                                                  const StepParams* __restrict__ p, double box,
                                                  uint32_t* __restrict__ keys,
                                                  int32_t* __restrict__ vals) {
  const int64_t i = blockIdx.x * (int64_t)BT + threadIdx.x;
  if (i >= n) return;
  uint32_t c[3];
  if (box > 0.0) {
    const double inv = 1024.0 / box;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double q = pos[3 * i + k] * inv;
      q = fmin(fmax(q, 0.0), 1023.0);
      c[k] = (uint32_t)q;
    }
  } else {
    float d[3];
    float r2 = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      d[k] = (float)pos[3 * i + k] - p->centre[k];
      r2 += d[k] * d[k];
    }
    const float r = sqrtf(r2);
    const float u = asinhf(r / p->key_scale) * p->key_inv_norm;
    const float f = r > 0.f ? u / r : 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float q = (d[k] * f + 1.0f) * 512.0f;
      q = fminf(fmaxf(q, 0.0f), 1023.0f);
      c[k] = (uint32_t)q;
    }
  }
  keys[i] = spread10(c[0]) | (spread10(c[1]) << 1) | (spread10(c[2]) << 2);
  vals[i] = (int32_t)i;
}

__global__ void __launch_bounds__(BT) permute_kernel(
    const int32_t* __restrict__ perm, int64_t n, const double* __restrict__ pos,
    const double* __restrict__ vel, const double* __restrict__ mass,
    const uint32_t* __restrict__ ids, const uint8_t* __restrict__ act,
    const int8_t* __restrict__ bins, double dt_max, Sorted so, int32_t* __restrict__ act_list,
    DevStats* st) {
  const int64_t s = blockIdx.x * (int64_t)BT + threadIdx.x;
  bool a = false;
  if (s < n) {
    const int64_t o = perm[s];
    const double x = pos[3 * o], y = pos[3 * o + 1], z = pos[3 * o + 2];
    so.x[s] = x;
    so.y[s] = y;
    so.z[s] = z;
    const double dt = ldexp(dt_max, -(int)bins[o]);
    const double vx = vel[3 * o], vy = vel[3 * o + 1], vz = vel[3 * o + 2], m = mass[o];
    so.f[s] = make_float4((float)x, (float)y, (float)z, __double2float_ru(dt));
    so.vx[s] = vx;
    so.vy[s] = vy;
    so.vz[s] = vz;
    so.vm[s] = make_float4((float)vx, (float)vy, (float)vz, __double2float_ru(m));
    so.m[s] = m;
    so.id[s] = ids[o];
    a = act[o] != 0;
    so.act[s] = a ? 1 : 0;
    so.dt[s] = dt;
    so.h[s] = 0.0;
    so.orig[s] = (int32_t)o;
  }
  const unsigned ballot = __ballot_sync(0xffffffffu, a);
  if (ballot == 0) return;
  const int lane = threadIdx.x & 31;
  unsigned long long base = 0;
  if (lane == __ffs(ballot) - 1) base = atomicAdd(&st->n_active, (unsigned long long)__popc(ballot));
  base = __shfl_sync(0xffffffffu, base, __ffs(ballot) - 1);
  if (a) act_list[base + __popc(ballot & ((1u << lane) - 1u))] = (int32_t)s;
}

// Leaves: conservative FP32 box of 32 consecutive particles (min rounded
// down, max rounded up from the FP64 coordinates).
__global__ void __launch_bounds__(BT) leaf_kernel(Sorted so, int64_t n, float4* lo, float4* hi,
                                                  int64_t nleaves) {
  const int64_t leaf = (blockIdx.x * (int64_t)BT + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (leaf >= nleaves) return;
  const int64_t s = leaf * LEAF + lane;
  double x0 = INFINITY, y0 = INFINITY, z0 = INFINITY, x1 = -INFINITY, y1 = -INFINITY, z1 = -INFINITY;
  if (s < n) {
    x0 = x1 = so.x[s];
    y0 = y1 = so.y[s];
    z0 = z1 = so.z[s];
  }
  x0 = warp_min(x0); y0 = warp_min(y0); z0 = warp_min(z0);
  x1 = warp_max(x1); y1 = warp_max(y1); z1 = warp_max(z1);
  if (lane == 0) {
    lo[leaf] = make_float4(__double2float_rd(x0), __double2float_rd(y0), __double2float_rd(z0), 0.f);
    hi[leaf] = make_float4(__double2float_ru(x1), __double2float_ru(y1), __double2float_ru(z1), 0.f);
  }
}

__global__ void __launch_bounds__(BT) node_kernel(const float4* clo, const float4* chi,
                                                  int64_t nchild, float4* lo, float4* hi,
                                                  int64_t nnode) {
  const int64_t node = (blockIdx.x * (int64_t)BT + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (node >= nnode) return;
  const int64_t c = node * 32 + lane;
  float x0 = INFINITY, y0 = INFINITY, z0 = INFINITY, x1 = -INFINITY, y1 = -INFINITY, z1 = -INFINITY;
  if (c < nchild) {
    const float4 a = clo[c], b = chi[c];
    x0 = a.x; y0 = a.y; z0 = a.z;
    x1 = b.x; y1 = b.y; z1 = b.z;
  }
  x0 = warp_minf(x0); y0 = warp_minf(y0); z0 = warp_minf(z0);
  x1 = warp_maxf(x1); y1 = warp_maxf(y1); z1 = warp_maxf(z1);
  if (lane == 0) {
    lo[node] = make_float4(x0, y0, z0, 0.f);
    hi[node] = make_float4(x1, y1, z1, 0.f);
  }
}

inline unsigned blocks_for(int64_t threads) { return (unsigned)((threads + BT - 1) / BT); }

}  // namespace

int launch_bbox(const double* pos, int64_t n, unsigned long long* mm, cudaStream_t s) {
  bbox_init_kernel<<<1, 32, 0, s>>>(mm);
  if (n <= 0) return 1;
  int64_t b = blocks_for(n);
  if (b > 148 * 8) b = 148 * 8;
  bbox_kernel<<<(unsigned)b, BT, 0, s>>>(pos, n, mm);
  return 2;
}

int launch_params(const unsigned long long* mm, StepParams* p, double box, int64_t n, int n_ngb,
                  cudaStream_t s) {
  // largest e (<= 60) with 8^e * n_ngb <= 4 n
  int e = 0;
  while (e < 60 && std::ldexp((double)n_ngb, 3 * (e + 1)) <= 4.0 * (double)n) ++e;
  params_kernel<<<1, 32, 0, s>>>(mm, p, box, e);
  return 1;
}

int launch_keys(const double* pos, int64_t n, const StepParams* p, double box, uint32_t* keys,
                int32_t* vals, cudaStream_t s) {
  if (n <= 0) return 0;
  keys_kernel<<<blocks_for(n), BT, 0, s>>>(pos, n, p, box, keys, vals);
  return 1;
}

int launch_permute(const int32_t* perm, int64_t n, const double* pos, const double* vel,
                   const double* mass, const uint32_t* ids, const uint8_t* act,
                   const int8_t* bins, double dt_max, Sorted so, int32_t* act_list,
                   DevStats* st, cudaStream_t s) {
  if (n <= 0) return 0;
  permute_kernel<<<blocks_for(n), BT, 0, s>>>(perm, n, pos, vel, mass, ids, act, bins, dt_max, so,
                                              act_list, st);
  return 1;
}

int tree_levels_for(int64_t n, int64_t count[MAX_LEVELS]) {
  int64_t c = (n + LEAF - 1) / LEAF;
  if (c < 1) c = 1;
  int l = 0;
  count[l++] = c;
  while (c > 1 && l < MAX_LEVELS) {
    c = (c + 31) / 32;
    count[l++] = c;
  }
  return l;
}

int launch_tree(const Sorted& so, int64_t n, Tree& t, cudaStream_t s) {
  leaf_kernel<<<blocks_for(t.count[0] * 32), BT, 0, s>>>(so, n, t.lo, t.hi, t.count[0]);
  for (int l = 1; l < t.levels; ++l) {
    node_kernel<<<blocks_for(t.count[l] * 32), BT, 0, s>>>(
        t.lo + t.offset[l - 1], t.hi + t.offset[l - 1], t.count[l - 1], t.lo + t.offset[l],
        t.hi + t.offset[l], t.count[l]);
  }
  return t.levels;
}

}  // namespace sidm
