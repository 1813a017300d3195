// Total kinetic energy and momentum with compensated (Neumaier) sums, for the
// conservation statistics of a step (momentum and energy are conserved to
// round-off by elastic scatters, Sec. 4.4).  Deterministic for a given n:
// fixed grid, fixed per-thread ranges, fixed combination order.
#include "sidm_internal.cuh"

namespace sidm {

namespace {

constexpr int CT = 256;
constexpr int CB = 296;

struct NSum {
  double s = 0.0, c = 0.0;
  __device__ void add(double x) {
    const double t = s + x;
    if (fabs(s) >= fabs(x)) c += (s - t) + x;
    else c += (x - t) + s;
    s = t;
  }
};

__global__ void __launch_bounds__(CT) conserved_partial_kernel(const double* __restrict__ vel,
                                                               const double* __restrict__ mass,
                                                               int64_t n, double* partial) {
  __shared__ double sh[CT][4];
  NSum acc[4];
  for (int64_t i = blockIdx.x * (int64_t)CT + threadIdx.x; i < n; i += (int64_t)CB * CT) {
    const double m = mass[i];
    const double vx = vel[3 * i], vy = vel[3 * i + 1], vz = vel[3 * i + 2];
    acc[0].add(0.5 * m * ((vx * vx + vy * vy) + vz * vz));
    acc[1].add(m * vx);
    acc[2].add(m * vy);
    acc[3].add(m * vz);
  }
  for (int k = 0; k < 4; ++k) sh[threadIdx.x][k] = acc[k].s + acc[k].c;
  __syncthreads();
  if (threadIdx.x < 4) {
    NSum t;
    for (int j = 0; j < CT; ++j) t.add(sh[j][threadIdx.x]);
    partial[blockIdx.x * 4 + threadIdx.x] = t.s + t.c;
  }
}

__global__ void conserved_final_kernel(const double* partial, double* out4) {
  if (threadIdx.x < 4) {
    NSum t;
    for (int j = 0; j < CB; ++j) t.add(partial[j * 4 + threadIdx.x]);
    out4[threadIdx.x] = t.s + t.c;
  }
}

}  // namespace

int conserved_blocks() { return CB; }

int launch_conserved(const double* vel, const double* mass, int64_t n, double* partial,
                      double* out4, cudaStream_t s) {
  conserved_partial_kernel<<<CB, CT, 0, s>>>(vel, mass, n, partial);
  conserved_final_kernel<<<1, 32, 0, s>>>(partial, out4);
  return 2;
}

}  // namespace sidm
