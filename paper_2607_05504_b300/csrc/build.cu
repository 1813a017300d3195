// Per-step neighbour structure of every halo: bounding box, spatial keys,
// key-order copy of the particle state, and a 32-ary tree of conservative
// FP32 boxes over runs of 32 key-consecutive particles.
//
// The structure replaces the paper's dedicated DM-only octree (Sec. 4.3): it
// is rebuilt every step from scratch (sort + linear passes), so it needs no
// drifted bounds.  Its only role is to prune the neighbour search; every
// result of the step is independent of the particle order it produces.
// Keys carry the halo index above the spatial bits, so each halo stays a
// contiguous run [start, start + n) in key order, with a tree of its own.
#include "sidm_internal.cuh"

#include <cmath>

namespace sidm {

namespace {

constexpr int BT = 256;
constexpr int BB_ITEMS = 16;
#ifndef BB_GROUP
#define BB_GROUP 4      // loads in flight per thread (1: 0.051 ms, 4: 0.043 ms for the key phase)
#endif

__device__ __forceinline__ float warp_minf(float v) {
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_maxf(float v) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// halo k with node_off[level] of k <= g (the largest such k)
__device__ __forceinline__ int find_halo_level(const Halo* halos, int n_halos, int level,
                                               int64_t g) {
  int lo = 0, hi = n_halos - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (halos[mid].node_off[level] <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void bbox_init_kernel(Halo* halos, int n_halos) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_halos) return;
  for (int a = 0; a < 3; ++a) {
    halos[k].mm[a] = ~0ull;
    halos[k].mm[3 + a] = 0ull;
  }
}

// lo / hi: running extrema as order-preserving integers of the doubles
// (integer min/max: exact, and off B300's slow FP64 pipe)
constexpr unsigned long long ORD_NONE_LO = ~0ull, ORD_NONE_HI = 0ull;
__device__ __forceinline__ void bbox_flush(Halo* halos, int k, const unsigned long long* lo,
                                           const unsigned long long* hi) {
  for (int a = 0; a < 3; ++a) {
    if (lo[a] <= hi[a]) {
      atomicMin(&halos[k].mm[a], lo[a]);
      atomicMax(&halos[k].mm[3 + a], hi[a]);
    }
  }
}
__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w < v ? w : v;
  }
  return v;
}
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// Bounding box of every halo: blocks walk contiguous chunks; a thread flushes
// its running box when the halo changes, warps combine at chunk ends, and
// the warps of a block combine in shared memory, so that a chunk inside one
// halo costs one flush (atomics on the same six words serialise).
__global__ void __launch_bounds__(BT) bbox_kernel(const double* __restrict__ pos,
                                                  const int32_t* __restrict__ halo_of, int64_t n,
                                                  Halo* halos) {
  constexpr int NW = BT / 32;
  __shared__ unsigned long long s_lo[NW][3], s_hi[NW][3];
  __shared__ int s_k[NW];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t chunk_len = (int64_t)BT * BB_ITEMS;
  for (int64_t c0 = blockIdx.x * chunk_len; c0 < n; c0 += (int64_t)gridDim.x * chunk_len) {
    int cur = -1;
    unsigned long long lo[3] = {ORD_NONE_LO, ORD_NONE_LO, ORD_NONE_LO};
    unsigned long long hi[3] = {ORD_NONE_HI, ORD_NONE_HI, ORD_NONE_HI};
    // BB_GROUP items' loads are issued together before any is used
    for (int j0 = 0; j0 < BB_ITEMS; j0 += BB_GROUP) {
      int kg[BB_GROUP];
      double pg[BB_GROUP][3];
#pragma unroll
      for (int g = 0; g < BB_GROUP; ++g) {
        const int64_t i = c0 + (int64_t)(j0 + g) * BT + threadIdx.x;
        kg[g] = -1;
        if (i < n) {
          kg[g] = halo_of[i];
          pg[g][0] = pos[3 * i];
          pg[g][1] = pos[3 * i + 1];
          pg[g][2] = pos[3 * i + 2];
        }
      }
#pragma unroll
      for (int g = 0; g < BB_GROUP; ++g) {
        const int k = kg[g];
        if (k < 0) break;
        if (k != cur) {
          if (cur >= 0) bbox_flush(halos, cur, lo, hi);
          cur = k;
          for (int a = 0; a < 3; ++a) { lo[a] = ORD_NONE_LO; hi[a] = ORD_NONE_HI; }
        }
        for (int a = 0; a < 3; ++a) {
          const unsigned long long x = dbl_to_ordered(pg[g][a]);
          lo[a] = x < lo[a] ? x : lo[a];
          hi[a] = x > hi[a] ? x : hi[a];
        }
      }
    }
    const int k0 = __shfl_sync(0xffffffffu, cur, 0);
    const bool same = __all_sync(0xffffffffu, cur == k0 || cur < 0) && k0 >= 0;
    if (same) {
      for (int a = 0; a < 3; ++a) {
        lo[a] = warp_min_u64(lo[a]);
        hi[a] = warp_max_u64(hi[a]);
      }
    } else if (cur >= 0) {
      bbox_flush(halos, cur, lo, hi);   // a warp across a halo boundary (rare)
    }
    if (lane == 0) {
      s_k[warp] = same ? k0 : -1;
      for (int a = 0; a < 3; ++a) {
        s_lo[warp][a] = lo[a];
        s_hi[warp][a] = hi[a];
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      // runs of warps in the same halo, one flush per run
      int kk = -1;
      unsigned long long alo[3], ahi[3];
      for (int w = 0; w < NW; ++w) {
        const int kw = s_k[w];
        if (kw < 0) continue;
        if (kw != kk) {
          if (kk >= 0) bbox_flush(halos, kk, alo, ahi);
          kk = kw;
          for (int a = 0; a < 3; ++a) { alo[a] = s_lo[w][a]; ahi[a] = s_hi[w][a]; }
        } else {
          for (int a = 0; a < 3; ++a) {
            alo[a] = s_lo[w][a] < alo[a] ? s_lo[w][a] : alo[a];
            ahi[a] = s_hi[w][a] > ahi[a] ? s_hi[w][a] : ahi[a];
          }
        }
      }
      if (kk >= 0) bbox_flush(halos, kk, alo, ahi);
    }
    __syncthreads();   // the next chunk reuses the shared arrays
  }
}

// Per halo: extent, start radius h0 = l_ext 2^-e0, key transform.
__global__ void params_kernel(Halo* halos, int n_halos, double box) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_halos) return;
  Halo& H = halos[k];
  if (H.n <= 0) return;
  double lo[3], hi[3];
  for (int a = 0; a < 3; ++a) {
    lo[a] = ordered_to_dbl(H.mm[a]);
    hi[a] = ordered_to_dbl(H.mm[3 + a]);
  }
  double l_ext = box;
  if (!(box > 0.0)) {
    l_ext = 0.0;
    for (int a = 0; a < 3; ++a) l_ext = fmax(l_ext, hi[a] - lo[a]);
  }
  H.l_ext = l_ext;
  H.h0 = ldexp(l_ext, -H.e0);
  float r2 = 0.f;
  for (int a = 0; a < 3; ++a) {
    // open boundaries: the middle of the bounding box (key transform and
    // origin of the FP32 copies); periodic: 0 (the copies stay absolute)
    H.centre[a] = box > 0.0 ? 0.0f : (float)(0.5 * (lo[a] + hi[a]));
    const float d = (float)(hi[a] - lo[a]);
    r2 += d * d;
  }
  const float R = 0.5f * sqrtf(r2) * 1.001f + 1e-30f;
  const float sc = R * (1.0f / 1024.0f);
  H.key_scale = sc;
  H.key_inv_norm = 1.0f / asinhf(R / sc);
}

__device__ __forceinline__ uint32_t spread10(uint32_t v) {
  v &= 0x3FFu;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

// Index of cell (x0, x1, x2), each coordinate of `bits` bits, along a 3-D
// Hilbert curve (Skilling, "Programming the Hilbert curve", AIP Conf. Proc.
// 707, 2004): the coordinates are transformed in place into the curve's
// "transposed" index, whose bits are then interleaved, axis 0 first.
// Consecutive cells along the curve are face neighbours, so runs of
// key-ordered particles (tree leaves, the search window) stay compact.
__device__ __forceinline__ uint32_t hilbert_key(uint32_t x0, uint32_t x1, uint32_t x2, int bits) {
  if (bits <= 0) return 0u;
  const uint32_t M = 1u << (bits - 1);
  // inverse undo: walk the bits from the top, reflecting or exchanging
  for (uint32_t Q = M; Q > 1; Q >>= 1) {
    const uint32_t P = Q - 1;
    if (x0 & Q) x0 ^= P;
    if (x1 & Q) {
      x0 ^= P;
    } else {
      const uint32_t t = (x0 ^ x1) & P;
      x0 ^= t;
      x1 ^= t;
    }
    if (x2 & Q) {
      x0 ^= P;
    } else {
      const uint32_t t = (x0 ^ x2) & P;
      x0 ^= t;
      x2 ^= t;
    }
  }
  // Gray encode
  x1 ^= x0;
  x2 ^= x1;
  uint32_t t = 0;
  for (uint32_t Q = M; Q > 1; Q >>= 1)
    if (x2 & Q) t ^= Q - 1;
  x0 ^= t;
  x1 ^= t;
  x2 ^= t;
  return (spread10(x0) << 2) | (spread10(x1) << 1) | spread10(x2);
}

// Key = halo index above a Hilbert key with mb = key_axis_bits(halo_bits) bits per
// axis.  Periodic box: 2^mb cells per axis.  Open boundaries: the offset
// from the halo's centre is compressed radially by asinh(r/s)/asinh(R/s)
// (s = R/1024) before 2^mb cells per axis, so that cells stay small relative
// to the interparticle spacing from a halo's dense centre to its outskirts.
// Keys only shape the traversal cost.
__global__ void __launch_bounds__(BT) keys_kernel(const double* __restrict__ pos,
                                                  const int32_t* __restrict__ halo_of, int64_t n,
                                                  const Halo* __restrict__ halos, int halo_bits,
                                                  double box, uint32_t* __restrict__ keys,
                                                  int32_t* __restrict__ vals) {
  const int64_t i = blockIdx.x * (int64_t)BT + threadIdx.x;
  if (i >= n) return;
  const int k = halo_of[i];
  const int mb = key_axis_bits(halo_bits);
  const float cells = (float)(1u << mb);
  uint32_t c[3];
  if (box > 0.0) {
    const double inv = (double)(1u << mb) / box;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      double q = pos[3 * i + a] * inv;
      q = fmin(fmax(q, 0.0), (double)cells - 1.0);
      c[a] = (uint32_t)q;
    }
  } else {
    const Halo& H = halos[k];
    float d[3];
    float r2 = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      d[a] = (float)pos[3 * i + a] - H.centre[a];
      r2 += d[a] * d[a];
    }
    const float r = sqrtf(r2);
    const float u = asinhf(r / H.key_scale) * H.key_inv_norm;
    const float f = r > 0.f ? u / r : 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float q = (d[a] * f + 1.0f) * (0.5f * cells);
      q = fminf(fmaxf(q, 0.0f), cells - 1.0f);
      c[a] = (uint32_t)q;
    }
  }
  keys[i] = ((uint32_t)k << (3 * mb)) | hilbert_key(c[0], c[1], c[2], mb);
  vals[i] = (int32_t)i;
}

// Key-order copy of everything but the velocities (which the search does not
// read: they are copied by permute_vel_kernel just before the pair kernels).
__global__ void __launch_bounds__(BT) permute_kernel(
    const int32_t* __restrict__ perm, int64_t n, const double* __restrict__ pos,
    const double* __restrict__ mass,
    const uint32_t* __restrict__ ids, const int32_t* __restrict__ halo_of,
    const uint8_t* __restrict__ act, const int8_t* __restrict__ bins,
    const Halo* __restrict__ halos, Sorted so, int32_t* __restrict__ act_list, DevStats* st) {
  const int64_t s = blockIdx.x * (int64_t)BT + threadIdx.x;
  bool a = false;
  if (s < n) {
    int64_t o = perm[s];
    if (o < 0 || o >= n) {   // only after a failed sort (the step is then invalid)
      atomicOr(&st->status, (unsigned)ST_ERR_SORT);
      o = s;
    }
    const int k = halo_of[o];
    const double x = pos[3 * o], y = pos[3 * o + 1], z = pos[3 * o + 2];
    so.x[s] = x;
    so.y[s] = y;
    so.z[s] = z;
    const double dt = scale_pow2_down(halos[k].dt_max, (int)bins[o]);
    const double m = mass[o];
    // FP32 copies relative to the halo's centre c (a float, so exact in
    // FP64): their rounding, 2^-24 (1 + 2^-28) |x - c| with the FP64
    // difference, scales with the halo's extent instead of its distance from
    // the origin.  Every FP32 test compares particles of one halo, and a
    // common translation changes none of their separations.
    const float* c = halos[k].centre;
    so.f[s] = make_float4(f64_to_f32_rn(x - (double)c[0]), f64_to_f32_rn(y - (double)c[1]),
                          f64_to_f32_rn(z - (double)c[2]), f64_to_f32_ru(dt));
    so.m[s] = m;
    so.id[s] = ids[o];
    a = act[o] != 0;
    so.act[s] = a ? 1 : 0;
    so.dt[s] = dt;
    so.h[s] = 0.0;
    so.orig[s] = (int32_t)o;
    so.halo[s] = k;
  }
  const unsigned ballot = __ballot_sync(0xffffffffu, a);
  if (ballot == 0) return;
  const int lane = threadIdx.x & 31;
  unsigned long long base = 0;
  if (lane == __ffs(ballot) - 1) base = atomicAdd(&st->n_active, (unsigned long long)__popc(ballot));
  base = __shfl_sync(0xffffffffu, base, __ffs(ballot) - 1);
  if (a) act_list[base + __popc(ballot & ((1u << lane) - 1u))] = (int32_t)s;
}

// Leaves: conservative FP32 box of up to 32 consecutive particles of a halo
// (min rounded down, max rounded up from the FP64 coordinates).
// Leaf boxes from the FP32 copies f of the positions relative to the
// halo's centre, u = x - c: |u - f| <= 2^-24 (1 + 2^-28) |u|, below
// 2^-23 |f| for normal values, so widening the FP32 extrema by 2^-23 of
// their magnitude (plus the smallest normal, for values near zero), with
// directed rounding, gives boxes that contain every u.  No FP64 arithmetic.
__device__ __forceinline__ float widen_down(float v) {
  return __fsub_rd(v, __fadd_ru(__fmul_ru(fabsf(v), 1.1920928955078125e-07f), 1.17549435e-38f));
}
__device__ __forceinline__ float widen_up(float v) {
  return __fadd_ru(v, __fadd_ru(__fmul_ru(fabsf(v), 1.1920928955078125e-07f), 1.17549435e-38f));
}
__global__ void __launch_bounds__(BT) leaf_kernel(Sorted so, Forest f) {
  const int64_t g = (blockIdx.x * (int64_t)BT + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g >= f.level_nodes[0]) return;
  const int k = find_halo_level(f.halos, f.n_halos, 0, g);
  const Halo& H = f.halos[k];
  const int64_t local = g - H.node_off[0];
  const int64_t s = H.start + local * LEAF + lane;
  float x0 = INFINITY, y0 = INFINITY, z0 = INFINITY, x1 = -INFINITY, y1 = -INFINITY, z1 = -INFINITY;
  if (local * LEAF + lane < H.n) {
    const float4 p = so.f[s];
    x0 = x1 = p.x;
    y0 = y1 = p.y;
    z0 = z1 = p.z;
  }
  x0 = warp_minf(x0); y0 = warp_minf(y0); z0 = warp_minf(z0);
  x1 = warp_maxf(x1); y1 = warp_maxf(y1); z1 = warp_maxf(z1);
  if (lane == 0) {
    f.lo[g] = make_float4(widen_down(x0), widen_down(y0), widen_down(z0), 0.f);
    f.hi[g] = make_float4(widen_up(x1), widen_up(y1), widen_up(z1), 0.f);
  }
}
__global__ void __launch_bounds__(BT) node_kernel(Forest f, int level, int64_t level_base) {
  const int64_t g = level_base + ((blockIdx.x * (int64_t)BT + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (g >= level_base + f.level_nodes[level]) return;
  const int k = find_halo_level(f.halos, f.n_halos, level, g);
  const Halo& H = f.halos[k];
  const int64_t local = g - H.node_off[level];
  const int64_t c = local * 32 + lane;
  float x0 = INFINITY, y0 = INFINITY, z0 = INFINITY, x1 = -INFINITY, y1 = -INFINITY, z1 = -INFINITY;
  if (c < H.node_cnt[level - 1]) {
    const int64_t cg = H.node_off[level - 1] + c;
    const float4 a = f.lo[cg], b = f.hi[cg];
    x0 = a.x; y0 = a.y; z0 = a.z;
    x1 = b.x; y1 = b.y; z1 = b.z;
  }
  x0 = warp_minf(x0); y0 = warp_minf(y0); z0 = warp_minf(z0);
  x1 = warp_maxf(x1); y1 = warp_maxf(y1); z1 = warp_maxf(z1);
  if (lane == 0) {
    f.lo[g] = make_float4(x0, y0, z0, 0.f);
    f.hi[g] = make_float4(x1, y1, z1, 0.f);
  }
}

inline unsigned blocks_for(int64_t threads) { return (unsigned)((threads + BT - 1) / BT); }

}  // namespace

int launch_bbox(const double* pos, const int32_t* halo_of, int64_t n, Halo* halos, int n_halos,
                cudaStream_t s) {
  bbox_init_kernel<<<(unsigned)((n_halos + 127) / 128), 128, 0, s>>>(halos, n_halos);
  if (n <= 0) return 1;
  int64_t b = (n + (int64_t)BT * BB_ITEMS - 1) / ((int64_t)BT * BB_ITEMS);
  if (b > 148 * 8) b = 148 * 8;
  bbox_kernel<<<(unsigned)b, BT, 0, s>>>(pos, halo_of, n, halos);
  return 2;
}

int launch_params(Halo* halos, int n_halos, double box, cudaStream_t s) {
  params_kernel<<<(unsigned)((n_halos + 127) / 128), 128, 0, s>>>(halos, n_halos, box);
  return 1;
}

// Largest h (rounded up, from the search) under every node, stored in the w
// of the node's upper corner: the overlap walk widens its radius by it.
__global__ void __launch_bounds__(BT) hmax_leaf_kernel(Sorted so, Forest f) {
  const int64_t g = (blockIdx.x * (int64_t)BT + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g >= f.level_nodes[0]) return;
  const int k = find_halo_level(f.halos, f.n_halos, 0, g);
  const Halo& H = f.halos[k];
  const int64_t local = g - H.node_off[0];
  float m = 0.0f;
  if (local * LEAF + lane < H.n) m = so.hb[H.start + local * LEAF + lane].y;
  m = warp_maxf(m);
  if (lane == 0) f.hi[g].w = m;
}
__global__ void __launch_bounds__(BT) hmax_node_kernel(Forest f, int level, int64_t level_base) {
  const int64_t g = level_base + ((blockIdx.x * (int64_t)BT + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (g >= level_base + f.level_nodes[level]) return;
  const int k = find_halo_level(f.halos, f.n_halos, level, g);
  const Halo& H = f.halos[k];
  const int64_t c = (g - H.node_off[level]) * 32 + lane;
  float m = 0.0f;
  if (c < H.node_cnt[level - 1]) m = f.hi[H.node_off[level - 1] + c].w;
  m = warp_maxf(m);
  if (lane == 0) f.hi[g].w = m;
}

int launch_hmax(const Sorted& so, const Forest& f, cudaStream_t s) {
  if (f.level_nodes[0] <= 0) return 0;
  int launches = 0;
  hmax_leaf_kernel<<<blocks_for(f.level_nodes[0] * 32), BT, 0, s>>>(so, f);
  ++launches;
  int64_t base = f.level_nodes[0];
  for (int l = 1; l < f.max_levels; ++l) {
    if (f.level_nodes[l] > 0) {
      hmax_node_kernel<<<blocks_for(f.level_nodes[l] * 32), BT, 0, s>>>(f, l, base);
      ++launches;
    }
    base += f.level_nodes[l];
  }
  return launches;
}

// Key-order velocities: FP64 copies and the FP32 copy with the mass rounded up.
__global__ void __launch_bounds__(BT) permute_vel_kernel(int64_t n,
                                                         const double* __restrict__ vel,
                                                         Sorted so) {
  const int64_t s = blockIdx.x * (int64_t)BT + threadIdx.x;
  if (s >= n) return;
  const int64_t o = so.orig[s];   // range-checked by permute_kernel
  const double vx = vel[3 * o], vy = vel[3 * o + 1], vz = vel[3 * o + 2];
  so.vx[s] = vx;
  so.vy[s] = vy;
  so.vz[s] = vz;
  so.vm[s] = make_float4(f64_to_f32_rn(vx), f64_to_f32_rn(vy), f64_to_f32_rn(vz),
                         f64_to_f32_ru(so.m[s]));
}

int launch_keys(const double* pos, const int32_t* halo_of, int64_t n, const Halo* halos,
                int halo_bits, double box, uint32_t* keys, int32_t* vals, cudaStream_t s) {
  if (n <= 0) return 0;
  keys_kernel<<<blocks_for(n), BT, 0, s>>>(pos, halo_of, n, halos, halo_bits, box, keys, vals);
  return 1;
}

int launch_permute_vel(int64_t n, const double* vel, const Sorted& so, cudaStream_t s) {
  if (n <= 0) return 0;
  permute_vel_kernel<<<blocks_for(n), BT, 0, s>>>(n, vel, so);
  return 1;
}

int launch_permute(const int32_t* perm, int64_t n, const double* pos,
                   const double* mass, const uint32_t* ids, const int32_t* halo_of,
                   const uint8_t* act, const int8_t* bins, const Halo* halos, Sorted so,
                   int32_t* act_list, DevStats* st, cudaStream_t s) {
  if (n <= 0) return 0;
  permute_kernel<<<blocks_for(n), BT, 0, s>>>(perm, n, pos, mass, ids, halo_of, act, bins,
                                              halos, so, act_list, st);
  return 1;
}

int tree_levels_for(int64_t n, int64_t count[MAX_LEVELS]) {
  if (n <= 0) return 0;
  int64_t c = (n + LEAF - 1) / LEAF;
  int l = 0;
  count[l++] = c;
  while (c > 1 && l < MAX_LEVELS) {
    c = (c + 31) / 32;
    count[l++] = c;
  }
  return l;
}

int launch_forest(const Sorted& so, const Forest& f, cudaStream_t s) {
  if (f.level_nodes[0] <= 0) return 0;
  leaf_kernel<<<blocks_for(f.level_nodes[0] * 32), BT, 0, s>>>(so, f);
  int launches = 1;
  int64_t base = f.level_nodes[0];
  for (int l = 1; l < f.max_levels; ++l) {
    if (f.level_nodes[l] > 0) {
      node_kernel<<<blocks_for(f.level_nodes[l] * 32), BT, 0, s>>>(f, l, base);
      ++launches;
    }
    base += f.level_nodes[l];
  }
  return launches;
}

}  // namespace sidm
