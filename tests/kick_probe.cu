// Device probes of the built-in kick (include/sidm_model.cuh), compiled by
// tests/test_gpu_group_kick.py:
//   probe_group_differing: IsotropicKick::scatter_group (one pair over a
//     group of eight lanes) against scatter_prepared (one lane) on random
//     pairs -- masses, velocities and eps over wide ranges -- returns the
//     number of pairs whose new velocities differ in any bit;
//   probe_cycles: clock64 cycles, on one warp of an otherwise idle GPU, of a
//     dependent FP64 FMA, of two independent ones, of a dependent FP32 FMA,
//     of __dsqrt_rn, and of a whole prepared kick (loads, arithmetic, stores)
//     on one lane and on a group of eight.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sidm_model.cuh"

using sidm_model::IsotropicKick;
using sidm_model::PairInfo;

namespace {

__device__ __forceinline__ double rnd(uint32_t seed, uint64_t i, uint32_t w, double lo,
                                      double hi) {
  const uint4 r = sidm_model::philox4x32_10(seed, 0x5eedu, (uint32_t)i, (uint32_t)(i >> 32), w,
                                            0u);
  return lo + (hi - lo) * sidm_model::unit53(r.x, r.y);
}

// one pair per group of eight lanes; vel holds 2 particles x 3 per pair
__global__ void group_vs_lane(uint64_t first, uint64_t n, uint32_t seed, double* vel,
                              unsigned long long* differing) {
  const int lane = threadIdx.x & 31, sub = lane & 7;
  const uint64_t g = first + (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) / 8;
  const bool active = g < first + n;
  const uint64_t slot = g - first;
  const double ma = exp2(rnd(seed, g, 0, -10.0, 10.0)), mb = exp2(rnd(seed, g, 1, -10.0, 10.0));
  const double eps = (g & 7) == 0 ? rnd(seed, g, 2, 0.1, 1.0) : 1.0;
  double va[3], vb[3];
  for (int k = 0; k < 3; ++k) {
    va[k] = rnd(seed, g, 3 + k, -1.0, 1.0) * exp2(rnd(seed, g, 6 + k, -30.0, 30.0));
    vb[k] = rnd(seed, g, 9 + k, -1.0, 1.0) * exp2(rnd(seed, g, 12 + k, -30.0, 30.0));
  }
  IsotropicKick m;
  m.eps = eps;
  double* v = vel + 6 * slot;
  if (active && sub == 0)
    for (int k = 0; k < 3; ++k) {
      v[k] = va[k];
      v[3 + k] = vb[k];
    }
  __syncwarp();
  // the masses enter through the prepared terms only
  const IsotropicKick::Particles P{v, nullptr};
  const PairInfo info{(uint32_t)g, (uint32_t)g + 1u, 0, 1, seed, 77u, 5u, nullptr};
  // the pair's direction and mass terms, as the library prepares them
  IsotropicKick::Prepared prep;
  prep.kt = sidm_model::detail::kick_terms(ma, mb, eps);
  IsotropicKick::direction(info, prep.e);
  m.scatter_group(P, 0, 1, prep, active);
  __syncwarp();
  if (active && sub == 0) {
    IsotropicKick::State a{{va[0], va[1], va[2]}, ma}, b{{vb[0], vb[1], vb[2]}, mb};
    m.scatter_prepared(a, b, prep);
    bool same = true;
    for (int k = 0; k < 3; ++k)
      same = same && __double_as_longlong(a.v[k]) == __double_as_longlong(v[k]) &&
             __double_as_longlong(b.v[k]) == __double_as_longlong(v[3 + k]);
    if (!same) atomicAdd(differing, 1ull);
  }
}

__device__ __forceinline__ long long clk() {
  long long t;
  asm volatile("mov.u64 %0, %%clock64;" : "=l"(t)::"memory");
  return t;
}

__global__ void cycles(double* vel, const double* mass, long long* out, int reps) {
  const int lane = threadIdx.x & 31;
  __shared__ volatile double sink[32];
  double x = 1.5 + lane * 1e-3, y = 2.5 + lane * 1e-3;
  float xf = 1.5f;
  long long t0 = clk();
  for (int i = 0; i < reps; ++i) x = __fma_rn(x, 1.0000000001, 1e-9);
  sink[lane] = x;
  long long t1 = clk();
  for (int i = 0; i < reps; ++i) {
    x = __fma_rn(x, 1.0000000001, 1e-9);
    y = __fma_rn(y, 1.0000000001, 1e-9);
  }
  sink[lane] = x + y;
  long long t2 = clk();
  for (int i = 0; i < reps; ++i) xf = __fmaf_rn(xf, 1.0001f, 1e-3f);
  sink[lane] = xf;
  long long t3 = clk();
  for (int i = 0; i < reps; ++i) x = __dsqrt_rn(x + 1.0);
  sink[lane] = x;
  long long t4 = clk();
  if (lane == 0) {
    out[0] = (t1 - t0) / reps;
    out[1] = (t2 - t1) / reps;
    out[2] = (t3 - t2) / reps;
    out[3] = (t4 - t3) / reps;
  }
  IsotropicKick m;
  const IsotropicKick::Particles P{vel, mass};
  const PairInfo info{1u, 2u, 0, 1, 7u, 9u, 3u, nullptr};
  const IsotropicKick::Prepared prep = m.prepare(info, P);
  long long one = 0, grp = 0;
  for (int r = 0; r < 16; ++r) {
    __syncwarp();
    const long long a0 = clk();
    if (lane == 0) {
      IsotropicKick::State ia = m.get_state(P, 0), ib = m.get_state(P, 1);
      m.scatter_prepared(ia, ib, prep);
      m.set_state(P, 0, ia);
      m.set_state(P, 1, ib);
    }
    __threadfence();
    __syncwarp();
    const long long a1 = clk();
    m.scatter_group(P, 0, 1, prep, lane < 8);
    __threadfence();
    __syncwarp();
    const long long a2 = clk();
    one += a1 - a0;
    grp += a2 - a1;
  }
  if (lane == 0) {
    out[4] = one / 16;
    out[5] = grp / 16;
  }
}

}  // namespace

extern "C" int probe_group_differing(uint64_t n, uint32_t seed, unsigned long long* differing) {
  const uint64_t chunk = 1ull << 20;
  double* vel = nullptr;
  unsigned long long* d = nullptr;
  if (cudaMalloc(&vel, 6 * chunk * sizeof(double)) != cudaSuccess) return -1;
  if (cudaMalloc(&d, sizeof(*d)) != cudaSuccess) return -1;
  cudaMemset(d, 0, sizeof(*d));
  for (uint64_t first = 0; first < n; first += chunk) {
    const uint64_t m = n - first < chunk ? n - first : chunk;
    group_vs_lane<<<(unsigned)((m * 8 + 255) / 256), 256>>>(first, m, seed, vel, d);
  }
  const cudaError_t e = cudaMemcpy(differing, d, sizeof(*d), cudaMemcpyDeviceToHost);
  cudaFree(vel);
  cudaFree(d);
  return e == cudaSuccess && cudaGetLastError() == cudaSuccess ? 0 : -1;
}

extern "C" int probe_cycles(long long* out) {
  double *vel = nullptr, *mass = nullptr;
  long long* o = nullptr;
  const double hv[6] = {0.31, -0.72, 0.15, -0.44, 0.29, 0.83}, hm[2] = {1.0, 1.2};
  if (cudaMalloc(&vel, sizeof(hv)) != cudaSuccess || cudaMalloc(&mass, sizeof(hm)) != cudaSuccess ||
      cudaMalloc(&o, 6 * sizeof(long long)) != cudaSuccess)
    return -1;
  cudaMemcpy(vel, hv, sizeof(hv), cudaMemcpyHostToDevice);
  cudaMemcpy(mass, hm, sizeof(hm), cudaMemcpyHostToDevice);
  cycles<<<1, 32>>>(vel, mass, o, 64);   // warm-up
  cycles<<<1, 32>>>(vel, mass, o, 512);
  const cudaError_t e = cudaMemcpy(out, o, 6 * sizeof(long long), cudaMemcpyDeviceToHost);
  cudaFree(vel);
  cudaFree(mass);
  cudaFree(o);
  return e == cudaSuccess ? 0 : -1;
}
