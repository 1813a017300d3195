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

// Particles whose velocities the last step changed: the two particles of
// every accepted pair, each listed once (the first pair to reach it claims
// it by stamping it with the call's number), with their current velocities.
// Nothing changed if the step overflowed its pair buffers.
__global__ void __launch_bounds__(CT) changed_kernel(const PairRec* __restrict__ pairs,
                                                     int64_t cap, const DevStats* st,
                                                     uint32_t stamp, uint32_t* stamps,
                                                     const double* __restrict__ vel,
                                                     int32_t* idx_out, double* vel_out,
                                                     unsigned long long* count) {
  const unsigned long long na = st->n_acc;
  if (na > (unsigned long long)cap || st->n_deferred > (unsigned long long)cap) return;
  const int lane = threadIdx.x & 31;
  // whole warps step through the pairs, so that each list append takes one
  // atomic per warp
  for (int64_t base = blockIdx.x * (int64_t)CT + (threadIdx.x & ~31); base < (int64_t)na;
       base += (int64_t)gridDim.x * CT) {
    const int64_t p = base + lane;
    const bool valid = p < (int64_t)na;
    int32_t e2[2] = {0, 0};
    if (valid) {
      e2[0] = pairs[p].ia;
      e2[1] = pairs[p].ib;
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int32_t e = e2[q];
      const bool first = valid && atomicExch(&stamps[e], stamp) != stamp;
      const uint32_t m = __ballot_sync(0xffffffffu, first);
      if (!m) continue;
      unsigned long long at = 0;
      if (lane == 0) at = atomicAdd(count, (unsigned long long)__popc(m));
      at = __shfl_sync(0xffffffffu, at, 0);
      if (first) {
        const unsigned long long k = at + __popc(m & ((1u << lane) - 1u));
        idx_out[k] = e;
        vel_out[3 * k] = vel[3 * (int64_t)e];
        vel_out[3 * k + 1] = vel[3 * (int64_t)e + 1];
        vel_out[3 * k + 2] = vel[3 * (int64_t)e + 2];
      }
    }
  }
}

// The same particles written straight into a host copy of the velocities
// (pinned host memory the device can address): each changed particle's
// three components go to its own place, once, so nothing is staged and no
// host loop runs.
__global__ void __launch_bounds__(CT) changed_to_host_kernel(const PairRec* __restrict__ pairs,
                                                             int64_t cap, const DevStats* st,
                                                             uint32_t stamp, uint32_t* stamps,
                                                             const double* __restrict__ vel,
                                                             double* host_vel) {
  const unsigned long long na = st->n_acc;
  if (na > (unsigned long long)cap || st->n_deferred > (unsigned long long)cap) return;
  for (int64_t t = blockIdx.x * (int64_t)CT + threadIdx.x; t < 2 * (int64_t)na;
       t += (int64_t)gridDim.x * CT) {
    const PairRec& r = pairs[t >> 1];
    const int32_t e = (t & 1) ? r.ib : r.ia;
    if (atomicExch(&stamps[e], stamp) == stamp) continue;
    const double* v = vel + 3 * (int64_t)e;
    double* d = host_vel + 3 * (int64_t)e;
    d[0] = v[0];
    d[1] = v[1];
    d[2] = v[2];
  }
}

int launch_changed(const PairRec* pairs, int64_t cap, const DevStats* st, uint32_t stamp,
                   uint32_t* stamps, const double* vel, int32_t* idx_out, double* vel_out,
                   unsigned long long* count, int sms, cudaStream_t s) {
  changed_kernel<<<(unsigned)(sms * 4), CT, 0, s>>>(pairs, cap, st, stamp, stamps, vel, idx_out,
                                                    vel_out, count);
  return 1;
}

int launch_changed_to_host(const PairRec* pairs, int64_t cap, const DevStats* st,
                           uint32_t stamp, uint32_t* stamps, const double* vel,
                           double* host_vel, int sms, cudaStream_t s) {
  changed_to_host_kernel<<<(unsigned)(sms * 4), CT, 0, s>>>(pairs, cap, st, stamp, stamps, vel,
                                                            host_vel);
  return 1;
}

}  // namespace sidm
