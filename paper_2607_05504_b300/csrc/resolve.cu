// Application of the accepted pairs (Sec. 4.1 kick, Sec. 4.4 multiple
// scatters with immediate updates).
//
// The canonical result is the sequential pass over the accepted pairs in
// ascending (ord, a, b) order, each kick reading the velocities left by the
// earlier ones.  The resolver reaches the same result in rounds: in a round
// every unapplied pair that precedes all other unapplied pairs at both of its
// particles is applied.  Such pairs share no particle, and every particle
// still meets its pairs in key order, so the velocities equal those of the
// sequential pass bit for bit.  (This is the single-device counterpart of the
// paper's rule that no particle is modified concurrently, Sec. 4.5.)
//
// Direction: Marsaglia (1972) -- x1, x2 uniform in (-1, 1) from the Philox
// streams 1, 2, ... of the pair, accepted when 0 < s = x1^2 + x2^2 < 1, then
// e = (2 x1 sqrt(1-s), 2 x2 sqrt(1-s), 1 - 2 s).
// Kick: v_com = (m_a v_a + m_b v_b)/M, g = |v_a - v_b|,
//       v_a' = v_com + (m_b g / M) e,  v_b' = v_com - (m_a g / M) e.
#include "sidm_internal.cuh"

namespace sidm {

namespace {

constexpr int RT = 1024;

__device__ __forceinline__ bool key_less(const PairRec& x, const PairRec& y) {
  if (x.ord != y.ord) return x.ord < y.ord;
  if (x.a != y.a) return x.a < y.a;
  return x.b < y.b;
}

// true if no other unapplied pair at particle e precedes pair p
__device__ bool first_at(int64_t p, const PairRec& rp, int32_t e, const int32_t* head,
                         const int32_t* next, const PairRec* pairs, const volatile uint8_t* flags) {
  for (int32_t slot = head[e]; slot >= 0; slot = next[slot]) {
    const int64_t q = slot >> 1;
    if (q == p || (flags[q] & 1)) continue;
    if (key_less(pairs[q], rp)) return false;
  }
  return true;
}

__device__ void kick(const PairRec& r, double* vel, const double* mass, uint32_t k0, uint32_t k1,
                     uint32_t step, unsigned* dirfail) {
  double e0 = 0.0, e1 = 0.0, e2 = 1.0;
  bool found = false;
  for (uint32_t t = 0; t < DIRECTION_TRIES && !found; ++t) {
    const U4 w = philox10(k0, k1, step, 1u + t, r.a, r.b);
    const double x1 = 2.0 * unit53(w.x, w.y) - 1.0;
    const double x2 = 2.0 * unit53(w.z, w.w) - 1.0;
    const double s = x1 * x1 + x2 * x2;
    if (s > 0.0 && s < 1.0) {
      const double k = 2.0 * sqrt(1.0 - s);
      e0 = x1 * k;
      e1 = x2 * k;
      e2 = 1.0 - 2.0 * s;
      found = true;
    }
  }
  if (!found) atomicAdd(dirfail, 1u);
  double* va = vel + 3 * (int64_t)r.ia;
  double* vb = vel + 3 * (int64_t)r.ib;
  const double ma = mass[r.ia], mb = mass[r.ib];
  const double M = ma + mb;
  const double ax = va[0], ay = va[1], az = va[2];
  const double bx = vb[0], by = vb[1], bz = vb[2];
  const double cx = ((ma * ax) + (mb * bx)) / M;
  const double cy = ((ma * ay) + (mb * by)) / M;
  const double cz = ((ma * az) + (mb * bz)) / M;
  const double dx = ax - bx, dy = ay - by, dz = az - bz;
  const double g = sqrt((dx * dx + dy * dy) + dz * dz);
  const double fa = (mb * g) / M, fb = (ma * g) / M;
  va[0] = cx + fa * e0;
  va[1] = cy + fa * e1;
  va[2] = cz + fa * e2;
  vb[0] = cx - fb * e0;
  vb[1] = cy - fb * e1;
  vb[2] = cz - fb * e2;
}

__global__ void __launch_bounds__(RT) resolve_kernel(const PairRec* __restrict__ pairs,
                                                     int64_t cap, double* vel,
                                                     const double* __restrict__ mass,
                                                     int32_t* head, int32_t* next, uint8_t* flags,
                                                     int32_t* mult, uint32_t k0, uint32_t k1,
                                                     uint32_t step, DevStats* st) {
  __shared__ unsigned s_dirfail;
  __shared__ int s_max;
  const int t = threadIdx.x;
  if (t == 0) { s_dirfail = 0; s_max = 0; }
  const unsigned long long nall = st->n_acc;
  if (nall > (unsigned long long)cap) {
    if (t == 0) atomicOr(&st->status, (unsigned)ST_ERR_PAIR_OVERFLOW);
    return;
  }
  const int64_t na = (int64_t)nall;
  for (int64_t p = t; p < na; p += RT) {
    flags[p] = 0;
    const int32_t ea = pairs[p].ia, eb = pairs[p].ib;
    next[2 * p] = atomicExch(&head[ea], (int32_t)(2 * p));
    next[2 * p + 1] = atomicExch(&head[eb], (int32_t)(2 * p + 1));
    atomicAdd(&mult[ea], 1);
    atomicAdd(&mult[eb], 1);
  }
  __syncthreads();
  int rounds = 0;
  bool done = false;
  for (; rounds < RESOLVE_MAX_ROUNDS; ++rounds) {
    int left = 0;
    for (int64_t p = t; p < na; p += RT) {
      if (flags[p] & 1) continue;
      left = 1;
      const PairRec rp = pairs[p];
      if (first_at(p, rp, rp.ia, head, next, pairs, flags) &&
          first_at(p, rp, rp.ib, head, next, pairs, flags))
        flags[p] = 2;
    }
    if (!__syncthreads_or(left)) { done = true; break; }
    for (int64_t p = t; p < na; p += RT) {
      if (flags[p] == 2) {
        kick(pairs[p], vel, mass, k0, k1, step, &s_dirfail);
        flags[p] = 1;
      }
    }
    __syncthreads();
  }
  if (!done) {
    // the cap was reached with pairs left
    int left = 0;
    for (int64_t p = t; p < na; p += RT) left |= !(flags[p] & 1);
    if (__syncthreads_or(left) && t == 0) atomicOr(&st->status, (unsigned)ST_ERR_ROUNDS);
  }
  int mm = 0;
  for (int64_t p = t; p < na; p += RT) mm = max(mm, max(mult[pairs[p].ia], mult[pairs[p].ib]));
  atomicMax(&s_max, mm);
  __syncthreads();
  for (int64_t p = t; p < na; p += RT) {
    head[pairs[p].ia] = -1;
    head[pairs[p].ib] = -1;
    mult[pairs[p].ia] = 0;
    mult[pairs[p].ib] = 0;
  }
  if (t == 0) {
    st->n_rounds = (unsigned long long)rounds;
    st->max_mult = (unsigned long long)s_max;
    if (s_dirfail) {
      st->n_dirfail = s_dirfail;
      atomicOr(&st->status, (unsigned)ST_DIR_FAIL);
    }
  }
}

// ---- step path: isolated pairs in parallel, the rest in rounds ----------
//
// A pair whose two particles take part in no other accepted pair commutes
// with every other kick, so it is applied at once by any thread.  Only the
// remaining ("pending") pairs go through the rounds, and each round visits
// only the pairs still pending.

constexpr int GT = 256;

__global__ void __launch_bounds__(GT) count_kernel(const PairRec* __restrict__ pairs, int64_t cap,
                                                   int32_t* mult, const DevStats* st) {
  const unsigned long long nall = st->n_acc;
  if (nall > (unsigned long long)cap) return;
  for (int64_t p = blockIdx.x * (int64_t)GT + threadIdx.x; p < (int64_t)nall;
       p += (int64_t)gridDim.x * GT) {
    atomicAdd(&mult[pairs[p].ia], 1);
    atomicAdd(&mult[pairs[p].ib], 1);
  }
}

__global__ void __launch_bounds__(GT) split_kernel(const PairRec* __restrict__ pairs, int64_t cap,
                                                   double* vel, const double* __restrict__ mass,
                                                   int32_t* head, int32_t* next, uint8_t* flags,
                                                   const int32_t* __restrict__ mult,
                                                   int32_t* pending, uint32_t k0, uint32_t k1,
                                                   uint32_t step, DevStats* st) {
  __shared__ unsigned s_dirfail;
  __shared__ int s_max;
  if (threadIdx.x == 0) { s_dirfail = 0; s_max = 0; }
  __syncthreads();
  const unsigned long long nall = st->n_acc;
  const int lane = threadIdx.x & 31;
  int mm = 0;
  if (nall <= (unsigned long long)cap) {
    const int64_t na = (int64_t)nall;
    const int64_t stride = (int64_t)gridDim.x * GT;
    // uniform trip count per warp (ballots below)
    for (int64_t base = blockIdx.x * (int64_t)GT + (threadIdx.x & ~31); base < na; base += stride) {
      const int64_t p = base + lane;
      bool pend = false;
      if (p < na) {
        const PairRec r = pairs[p];
        const int ma = mult[r.ia], mb = mult[r.ib];
        mm = max(mm, max(ma, mb));
        if (ma == 1 && mb == 1) {
          kick(r, vel, mass, k0, k1, step, &s_dirfail);
        } else {
          pend = true;
          flags[p] = 0;
          next[2 * p] = atomicExch(&head[r.ia], (int32_t)(2 * p));
          next[2 * p + 1] = atomicExch(&head[r.ib], (int32_t)(2 * p + 1));
        }
      }
      const uint32_t m = __ballot_sync(0xffffffffu, pend);
      if (m) {
        unsigned long long at = 0;
        const int leader = __ffs(m) - 1;
        if (lane == leader) at = atomicAdd(&st->n_pending, (unsigned long long)__popc(m));
        at = __shfl_sync(0xffffffffu, at, leader);
        if (pend) pending[at + __popc(m & ((1u << lane) - 1u))] = (int32_t)p;
      }
    }
  }
  atomicMax(&s_max, mm);
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_max) atomicMax(&st->max_mult, (unsigned long long)s_max);
    if (s_dirfail) {
      atomicAdd(&st->n_dirfail, (unsigned long long)s_dirfail);
      atomicOr(&st->status, (unsigned)ST_DIR_FAIL);
    }
  }
}

__global__ void __launch_bounds__(RT) rounds_kernel(const PairRec* __restrict__ pairs, int64_t cap,
                                                    double* vel, const double* __restrict__ mass,
                                                    const int32_t* head, const int32_t* next,
                                                    uint8_t* flags, int32_t* pend_a,
                                                    int32_t* pend_b, uint32_t k0, uint32_t k1,
                                                    uint32_t step, DevStats* st) {
  __shared__ unsigned s_dirfail;
  __shared__ int s_n;
  const int t = threadIdx.x;
  if (t == 0) s_dirfail = 0;
  __syncthreads();
  if (st->n_acc > (unsigned long long)cap) return;
  int npend = (int)st->n_pending;
  int32_t* cur = pend_a;
  int32_t* nxt = pend_b;
  int rounds = 0;
  while (npend > 0 && rounds < RESOLVE_MAX_ROUNDS) {
    for (int k = t; k < npend; k += RT) {
      const int64_t p = cur[k];
      const PairRec rp = pairs[p];
      if (first_at(p, rp, rp.ia, head, next, pairs, flags) &&
          first_at(p, rp, rp.ib, head, next, pairs, flags))
        flags[p] = 2;
    }
    if (t == 0) s_n = 0;
    __syncthreads();
    for (int k = t; k < npend; k += RT) {
      const int64_t p = cur[k];
      if (flags[p] == 2) {
        kick(pairs[p], vel, mass, k0, k1, step, &s_dirfail);
        flags[p] = 1;
      } else {
        nxt[atomicAdd(&s_n, 1)] = (int32_t)p;
      }
    }
    __syncthreads();
    npend = s_n;
    int32_t* tmp = cur; cur = nxt; nxt = tmp;
    ++rounds;
    __syncthreads();
  }
  if (t == 0) {
    if (npend > 0) atomicOr(&st->status, (unsigned)ST_ERR_ROUNDS);
    st->n_rounds = (unsigned long long)rounds;
    if (s_dirfail) {
      atomicAdd(&st->n_dirfail, (unsigned long long)s_dirfail);
      atomicOr(&st->status, (unsigned)ST_DIR_FAIL);
    }
  }
}

__global__ void __launch_bounds__(GT) reset_kernel(const PairRec* __restrict__ pairs, int64_t cap,
                                                   int32_t* head, int32_t* mult,
                                                   const DevStats* st) {
  const unsigned long long nall = st->n_acc;
  if (nall > (unsigned long long)cap) return;
  for (int64_t p = blockIdx.x * (int64_t)GT + threadIdx.x; p < (int64_t)nall;
       p += (int64_t)gridDim.x * GT) {
    head[pairs[p].ia] = -1;
    head[pairs[p].ib] = -1;
    mult[pairs[p].ia] = 0;
    mult[pairs[p].ib] = 0;
  }
}

}  // namespace

int launch_resolve(PairRec* pairs, int64_t pair_cap, double* vel, const double* mass,
                   int32_t* head, int32_t* next, uint8_t* flags, int32_t* mult, int32_t* pending,
                   uint64_t seed, uint32_t step, DevStats* st, int sms, cudaStream_t s) {
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  const unsigned g = (unsigned)(sms * 4);
  count_kernel<<<g, GT, 0, s>>>(pairs, pair_cap, mult, st);
  split_kernel<<<g, GT, 0, s>>>(pairs, pair_cap, vel, mass, head, next, flags, mult, pending, k0,
                                k1, step, st);
  rounds_kernel<<<1, RT, 0, s>>>(pairs, pair_cap, vel, mass, head, next, flags, pending,
                                 pending + pair_cap, k0, k1, step, st);
  reset_kernel<<<g, GT, 0, s>>>(pairs, pair_cap, head, mult, st);
  return 4;
}

// The same kernel for the no-allocation entry point: every scratch pointer
// (head, next, flags, mult, st) is supplied by the caller.
void launch_resolve_with_scratch(const PairRec* pairs, int64_t pair_cap, double* vel,
                                 const double* mass, int32_t* head, int32_t* next, uint8_t* flags,
                                 int32_t* mult, uint64_t seed, uint32_t step, DevStats* st,
                                 cudaStream_t s) {
  resolve_kernel<<<1, RT, 0, s>>>(pairs, pair_cap, vel, mass, head, next, flags, mult,
                                  (uint32_t)seed, (uint32_t)(seed >> 32), step, st);
}

}  // namespace sidm
