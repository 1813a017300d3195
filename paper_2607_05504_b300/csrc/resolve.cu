// Application of the accepted pairs (Sec. 4.1 kick, Sec. 4.4 multiple
// scatters with immediate updates).
//
// The canonical result is the sequential pass over the accepted pairs in
// ascending (ord, a, b) order, each kick reading the velocities left by the
// earlier ones.  The step applies its pairs with the application templates of
// sidm_model.cuh (split into isolated pairs and per-particle dataflow) and the
// built-in model IsotropicKick, with each halo's random key, step counter and
// eps.  The no-allocation entry point uses a single-block variant in rounds:
// in a round every unapplied pair that precedes all other unapplied pairs at
// both of its particles is applied; such pairs share no particle, and every
// particle still meets its pairs in key order, so the velocities equal those
// of the sequential pass bit for bit.  (This is the single-device counterpart
// of the paper's rule that no particle is modified concurrently, Sec. 4.5.)
#include "sidm_internal.cuh"

namespace sidm {

namespace {

using sidm_model::IsotropicKick;
using sidm_model::PairInfo;

constexpr int RT = 1024;

// The step's pairs: the model and the random key of each pair come from the
// halo of its particles.
struct HaloBinder {
  IsotropicKick::Particles parts;
  const int32_t* halo_of;
  const Halo* halos;
  double* mirror;        // device address of a pinned host copy of the velocities, or null
  // a particle's final velocity of the step into the host copy, read back
  // from L2 (the kick stores there); three 8-byte stores
  __device__ __forceinline__ void publish(int32_t e) const {
    if (!mirror) return;
    const double* v = parts.vel + 3 * (int64_t)e;
    const double v0 = __ldcg(v), v1 = __ldcg(v + 1), v2 = __ldcg(v + 2);
    double* d = mirror + 3 * (int64_t)e;
    d[0] = v0;
    d[1] = v1;
    d[2] = v2;
  }
  __device__ __forceinline__ IsotropicKick model(const PairRec& r) const {
    IsotropicKick m;
    m.eps = halos[halo_of[r.ia]].eps;
    return m;
  }
  __device__ __forceinline__ PairInfo info(const PairRec& r, unsigned* warn) const {
    const Halo& H = halos[halo_of[r.ia]];
    return PairInfo{r.a, r.b, r.ia, r.ib, (uint32_t)H.seed, (uint32_t)(H.seed >> 32), H.step,
                    warn};
  }
};

// true if no other unapplied pair at particle e precedes pair p.  Records
// with equal keys (a caller may pass the same pair twice) precede one
// another in record order, so they are applied one after the other, in the
// order given, and never in the same round.
__device__ bool first_at(int64_t p, const PairRec& rp, int32_t e, const int32_t* head,
                         const int32_t* next, const PairRec* pairs, const volatile uint8_t* flags) {
  for (int32_t slot = head[e]; slot >= 0; slot = next[slot]) {
    const int64_t q = slot >> 1;
    if (q == p || (flags[q] & 1)) continue;
    const PairRec rq = pairs[q];
    if (sidm_model::detail::key_less(rq, rp) || (q < p && !sidm_model::detail::key_less(rp, rq)))
      return false;
  }
  return true;
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
  const IsotropicKick model;   // elastic
  const IsotropicKick::Particles parts{vel, mass};
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
        const PairRec r = pairs[p];
        sidm_model::detail::interact(model, parts,
                                     PairInfo{r.a, r.b, r.ia, r.ib, k0, k1, step, &s_dirfail});
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

}  // namespace

int launch_resolve(PairRec* pairs, int64_t pair_cap, int max_passes, double* vel,
                   const double* mass, const int32_t* halo_of, const Halo* halos,
                   double* mirror, const ResolveBuffers& b, DevStats* st, int sms,
                   cudaStream_t s) {
  const HaloBinder bind{IsotropicKick::Particles{vel, mass}, halo_of, halos, mirror};
  return sidm_model::detail::launch_apply(pairs, pair_cap, max_passes, bind, b, st, sms, s);
}

// Kicks for the no-allocation entry point: every scratch pointer (head,
// next, flags, mult, st) is supplied by the caller.
void launch_resolve_with_scratch(const PairRec* pairs, int64_t pair_cap, double* vel,
                                 const double* mass, int32_t* head, int32_t* next, uint8_t* flags,
                                 int32_t* mult, uint64_t seed, uint32_t step, DevStats* st,
                                 cudaStream_t s) {
  resolve_kernel<<<1, RT, 0, s>>>(pairs, pair_cap, vel, mass, head, next, flags, mult,
                                  (uint32_t)seed, (uint32_t)(seed >> 32), step, st);
}


}  // namespace sidm
