/*
 * sidm_model_apply.cuh -- applies accepted pairs with a model of
 * sidm_model.cuh in the canonical order (part of sidm_model.cuh; include
 * that header).
 *
 * The result is that of one pass over the pairs in ascending (ord, a, b)
 * order (records with equal keys in the order given), each interaction on
 * the states the earlier ones left (Sec. 4.4).  On the device:
 *   1. count: pairs per particle;
 *   2. split: a pair whose particles are in no other pair ("isolated")
 *      commutes with all the others; the rest are "pending", and each of
 *      their particles gets a segment for its pairs;
 *   3. fill + rank: segments filled, each pending pair's place in key order
 *      at both of its particles;
 *   4. dataflow: a pending pair is applied once it sits at the cursor of both
 *      of its particles (every earlier pair of both applied); the kick's
 *      stores, one release fence, then the cursor stores; cursors are polled
 *      with acquire loads.  The grid is launched cooperatively (all blocks
 *      resident), the globally first unapplied pair is always ready, and a
 *      bounded number of passes guards against a stuck state (error flag).
 *      The isolated pairs are applied in the same kernel by the warps that
 *      hold no pending pair, while the chains of pending pairs run (or, when
 *      every warp holds one, by every thread after its pending pairs);
 *   5. reset of the per-particle arrays that were touched.
 * A binder may define publish(e): it is called once for every particle an
 * application changes, right after that particle's last interaction of the
 * application (its state is then final), by the thread that applied it;
 * the step uses it to copy velocities into a host-side mirror.
 * This is the single-device counterpart of the paper's rule that no particle
 * is modified concurrently (Sec. 4.5).
 */
#pragma once

namespace sidm_model {
namespace detail {

// status bits (the values of libsidm's step status)
constexpr unsigned kDirFail = 4u;
constexpr unsigned kErrPairOverflow = 1u << 11;
constexpr unsigned kErrRounds = 1u << 12;
constexpr unsigned kErrInvalid = 1u << 14;
constexpr int kThreads = 256;
constexpr int kMaxPasses = 1 << 22;

// per-particle and per-pair work arrays of one application
struct Buffers {
  int32_t* mult;      // [n] accepted pairs per particle (0 between calls)
  int32_t* seg_off;   // [n] start of the particle's pair segment (-1 between calls)
  int32_t* fill;      // [n] segment fill counter (0 between calls)
  int32_t* cursor;    // [n] first unapplied entry of the segment (0 between calls)
  int32_t* seg;       // [2 cap] pair ids, one segment per particle
  int32_t* seg_e;     // [2 cap] the particle of each segment slot
  int32_t* touched;   // [2 cap] particles that own a segment
  int32_t* pending;   // [cap] pairs that share a particle with another pair
  uint8_t* flags;     // [cap] applied flags
  int32_t* pos_a;     // [cap] place of the pair in the sorted segment of its particle a
  int32_t* pos_b;     // [cap] ... and of its particle b
};

// Counters of one application (libsidm's step statistics carry the same
// names; any struct with these fields serves).
struct Counters {
  unsigned long long n_acc, n_deferred, n_pending, n_seg, n_touched, max_mult, n_rounds,
      n_dirfail;
  unsigned int status;
  unsigned int pad;
};

__device__ __forceinline__ bool key_less(const sidm_pair& x, const sidm_pair& y) {
  if (x.ord != y.ord) return x.ord < y.ord;
  if (x.a != y.a) return x.a < y.a;
  return x.b < y.b;
}

template <class S>
__device__ __forceinline__ bool overflowed(const S* st, int64_t cap) {
  return st->n_acc > (unsigned long long)cap || st->n_deferred > (unsigned long long)cap;
}

__device__ __forceinline__ void st_relaxed(int32_t* p, int v) {
  asm volatile("st.relaxed.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_acquire(const int32_t* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void fence_acq_rel() {
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

// A trivially copyable value of lane src, word by word.
template <class T>
__device__ __forceinline__ T shfl_value(const T& v, int src) {
  constexpr int W = (int)((sizeof(T) + 3) / 4);
  uint32_t w[W] = {};
  memcpy(w, &v, sizeof(T));
#pragma unroll
  for (int i = 0; i < W; ++i) w[i] = __shfl_sync(0xffffffffu, w[i], src);
  T out;
  memcpy(&out, w, sizeof(T));
  return out;
}

// Detection of the binder's optional publish(e) (see the top of this file).
template <class B, class = void>
struct has_publish : std::false_type {};
template <class B>
struct has_publish<B, std::void_t<decltype(std::declval<const B&>().publish(int32_t(0)))>>
    : std::true_type {};

// publish(e) of a particle whose pair at place `place` of its segment of
// `mult` pairs has just been applied, if that was its last pair
template <class B>
__device__ __forceinline__ void publish_if_last(const B& bind, int32_t e, int place, int mult) {
  if constexpr (has_publish<B>::value) {
    if (place + 1 == mult) bind.publish(e);
  }
}

// One interaction through the model: states in, scatter on copies,
// overwrite_state(in, out) back.
template <class M>
__device__ __forceinline__ void interact(const M& m, const typename M::Particles& P,
                                         const PairInfo& p) {
  const typename M::State ia = m.get_state(P, p.ia), ib = m.get_state(P, p.ib);
  typename M::State oa = ia, ob = ib;
  m.scatter(oa, ob, p);
  m.set_state(P, p.ia, m.overwrite_state(ia, oa));
  m.set_state(P, p.ib, m.overwrite_state(ib, ob));
}

template <class S>
__global__ void __launch_bounds__(kThreads) count_kernel(const sidm_pair* __restrict__ pairs,
                                                         int64_t cap, int32_t* mult, const S* st) {
  const unsigned long long nall = st->n_acc;
  if (overflowed(st, cap)) return;
  for (int64_t p = blockIdx.x * (int64_t)kThreads + threadIdx.x; p < (int64_t)nall;
       p += (int64_t)gridDim.x * kThreads) {
    atomicAdd(&mult[pairs[p].ia], 1);
    atomicAdd(&mult[pairs[p].ib], 1);
  }
}

// Claims a segment for particle e (the first claimant allocates mult[e]
// slots); called by the whole warp, `want` per lane.  The slot and touched
// counters take one atomic per warp.
template <class S>
__device__ __forceinline__ void claim_segments(bool want, int32_t e, const int32_t* mult,
                                               int32_t* seg_off, int32_t* touched, S* st) {
  const int lane = threadIdx.x & 31;
  const bool first = want && atomicCAS(&seg_off[e], -1, -2) == -1;
  const int cnt = first ? mult[e] : 0;
  int incl = cnt;
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  const uint32_t fm = __ballot_sync(0xffffffffu, first);
  if (!fm) return;
  unsigned long long bs = 0, bt = 0;
  if (lane == 0) {
    bs = atomicAdd(&st->n_seg, (unsigned long long)total);
    bt = atomicAdd(&st->n_touched, (unsigned long long)__popc(fm));
  }
  bs = __shfl_sync(0xffffffffu, bs, 0);
  bt = __shfl_sync(0xffffffffu, bt, 0);
  if (first) {
    seg_off[e] = (int32_t)(bs + (unsigned long long)(incl - cnt));
    touched[bt + __popc(fm & ((1u << lane) - 1u))] = e;
  }
}

// Marks the pending pairs and claims their particles' segments (B, the
// binder, is the dataflow kernel's; the isolated pairs are applied there).
template <class B, class S>
__global__ void __launch_bounds__(kThreads, 4) split_kernel(const sidm_pair* __restrict__ pairs,
                                                            int64_t cap, B bind, Buffers b,
                                                            S* st) {
  __shared__ int s_max;
  if (threadIdx.x == 0) s_max = 0;
  __syncthreads();
  const unsigned long long nall = st->n_acc;
  const int lane = threadIdx.x & 31;
  int mm = 0;
  if (!overflowed(st, cap)) {
    const int64_t na = (int64_t)nall;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    for (int64_t base = blockIdx.x * (int64_t)kThreads + (threadIdx.x & ~31); base < na;
         base += stride) {
      const int64_t p = base + lane;
      bool pend = false;
      sidm_pair r{};
      if (p < na) {
        r = pairs[p];
        const int ma = b.mult[r.ia], mb = b.mult[r.ib];
        mm = max(mm, max(ma, mb));
        if (ma != 1 || mb != 1) {   // isolated pairs wait for the dataflow kernel
          pend = true;
          b.flags[p] = 0;
        }
      }
      claim_segments(pend, r.ia, b.mult, b.seg_off, b.touched, st);
      claim_segments(pend, r.ib, b.mult, b.seg_off, b.touched, st);
      const uint32_t m = __ballot_sync(0xffffffffu, pend);
      if (m) {
        unsigned long long at = 0;
        const int leader = __ffs(m) - 1;
        if (lane == leader) at = atomicAdd(&st->n_pending, (unsigned long long)__popc(m));
        at = __shfl_sync(0xffffffffu, at, leader);
        if (pend) b.pending[at + __popc(m & ((1u << lane) - 1u))] = (int32_t)p;
      }
    }
  }
  atomicMax(&s_max, mm);
  __syncthreads();
  if (threadIdx.x == 0 && s_max) atomicMax(&st->max_mult, (unsigned long long)s_max);
}

template <class S>
__global__ void __launch_bounds__(kThreads) fill_kernel(const sidm_pair* __restrict__ pairs,
                                                        int64_t cap, Buffers b, const S* st) {
  if (overflowed(st, cap)) return;
  const int64_t np = (int64_t)st->n_pending;
  for (int64_t k = blockIdx.x * (int64_t)kThreads + threadIdx.x; k < np;
       k += (int64_t)gridDim.x * kThreads) {
    const int32_t p = b.pending[k];
    const int32_t ea = pairs[p].ia, eb = pairs[p].ib;
    const int32_t sa = b.seg_off[ea] + atomicAdd(&b.fill[ea], 1);
    const int32_t sb = b.seg_off[eb] + atomicAdd(&b.fill[eb], 1);
    b.seg[sa] = p;
    b.seg_e[sa] = ea;
    b.seg[sb] = p;
    b.seg_e[sb] = eb;
  }
}

// Place of each pending pair in its particles' key order: one thread per
// segment slot counts the pairs of the same particle that come first --
// smaller key, or an equal key in an earlier record -- so the places are
// 0 .. mult-1 and records with equal keys keep the order they were given in.
template <class S>
__global__ void __launch_bounds__(kThreads) rank_kernel(const sidm_pair* __restrict__ pairs,
                                                        int64_t cap, Buffers b, const S* st) {
  if (overflowed(st, cap)) return;
  const int64_t ns = (int64_t)st->n_seg;
  for (int64_t t = blockIdx.x * (int64_t)kThreads + threadIdx.x; t < ns;
       t += (int64_t)gridDim.x * kThreads) {
    const int32_t e = b.seg_e[t], p = b.seg[t];
    const int32_t* sg = b.seg + b.seg_off[e];
    const int len = b.mult[e];
    const sidm_pair rp = pairs[p];
    int rank = 0;
    for (int k = 0; k < len; ++k) {
      const int32_t q = sg[k];
      const sidm_pair rq = pairs[q];
      rank += (key_less(rq, rp) || (q < p && !key_less(rp, rq))) ? 1 : 0;
    }
    if (rp.ia == e) b.pos_a[p] = rank;
    else b.pos_b[p] = rank;
  }
}

// A pending pair, its data gathered (and, where the model allows, its
// interaction prepared) before its turn; a turn is two acquire loads of the
// cursors, then the interaction through L2 and the release of both cursors.
// apply_ready is called by the whole warp each pass, `ready` set on the
// lanes whose pair has its turn: it applies those pairs, then releases
// their cursors (one fence, then relaxed stores).
template <class B, bool PREP = has_prepare<decltype(std::declval<B>().model(sidm_pair{}))>::value>
struct Turn;

template <class B>
struct Turn<B, true> {
  using M = decltype(std::declval<B>().model(sidm_pair{}));
  sidm_pair r;
  int pa, pb;
  int ma = 0, mb = 0;   // pairs of each particle (read only for publish)
  typename M::Prepared prep;
  M m;
  __device__ void load(const B& bind, const sidm_pair& rr, const Buffers& b, int32_t p,
                       unsigned* dirfail) {
    r = rr;
    pa = b.pos_a[p];
    pb = b.pos_b[p];
    if constexpr (has_publish<B>::value) {
      ma = b.mult[r.ia];
      mb = b.mult[r.ib];
    }
    m = bind.model(r);
    prep = m.prepare(bind.info(r, dirfail), bind.parts);
  }
  __device__ void release(const Buffers& b) const {
    st_relaxed(&b.cursor[r.ia], pa + 1);
    st_relaxed(&b.cursor[r.ib], pb + 1);
  }
  __device__ void publish(const B& bind) const {
    publish_if_last(bind, r.ia, pa, ma);
    publish_if_last(bind, r.ib, pb, mb);
  }
  __device__ void apply_ready(const B& bind, const Buffers& b, bool ready, unsigned*) const {
    if constexpr (has_group<M>::value) {
      // the ready pairs of the warp, 32 / GROUP at a time, each by a group
      // of GROUP lanes (M::scatter_group)
      constexpr int G = M::GROUP, NG = 32 / G;
      const int lane = threadIdx.x & 31, grp = lane / G;
      __syncwarp();   // the owners' acquire loads come before the group's loads
      uint32_t rm = __ballot_sync(0xffffffffu, ready);
      while (rm) {
        uint32_t mine = rm;
        for (int i = 0; i < grp; ++i) mine &= mine - 1u;
        const int owner = mine ? __ffs(mine) - 1 : -1;
        uint32_t rest = rm;
#pragma unroll
        for (int i = 0; i < NG; ++i) rest &= rest - 1u;
        const int src = owner >= 0 ? owner : lane;
        const int32_t ia = __shfl_sync(0xffffffffu, r.ia, src);
        const int32_t ib = __shfl_sync(0xffffffffu, r.ib, src);
        const typename M::Prepared pr = shfl_value(prep, src);
        const M mo = shfl_value(m, src);
        mo.scatter_group(bind.parts, ia, ib, pr, owner >= 0);
        __syncwarp();   // the group's stores come before the owner's release
        if ((rm & ~rest) & (1u << lane)) {
          fence_acq_rel();
          release(b);
          publish(bind);
        }
        rm = rest;
      }
    } else if (ready) {
      const typename M::State ia = m.get_state(bind.parts, r.ia),
                              ib = m.get_state(bind.parts, r.ib);
      typename M::State oa = ia, ob = ib;
      m.scatter_prepared(oa, ob, prep);
      m.set_state(bind.parts, r.ia, m.overwrite_state(ia, oa));
      m.set_state(bind.parts, r.ib, m.overwrite_state(ib, ob));
      fence_acq_rel();   // release: one fence covers both cursor stores
      release(b);
      publish(bind);
    }
  }
};

template <class B>
struct Turn<B, false> {
  sidm_pair r;
  int pa, pb;
  int ma = 0, mb = 0;   // pairs of each particle (read only for publish)
  __device__ void load(const B&, const sidm_pair& rr, const Buffers& b, int32_t p, unsigned*) {
    r = rr;
    pa = b.pos_a[p];
    pb = b.pos_b[p];
    if constexpr (has_publish<B>::value) {
      ma = b.mult[r.ia];
      mb = b.mult[r.ib];
    }
  }
  __device__ void apply_ready(const B& bind, const Buffers& b, bool ready,
                              unsigned* dirfail) const {
    if (!ready) return;
    interact(bind.model(r), bind.parts, bind.info(r, dirfail));
    fence_acq_rel();
    st_relaxed(&b.cursor[r.ia], pa + 1);
    st_relaxed(&b.cursor[r.ib], pb + 1);
    publish_if_last(bind, r.ia, pa, ma);
    publish_if_last(bind, r.ib, pb, mb);
  }
};

// The isolated pairs among accepted pairs first, first + stride, ...: each
// is applied by its thread (its particles are in no other pair).
template <class B>
__device__ __forceinline__ void apply_isolated(const sidm_pair* __restrict__ pairs, int64_t na,
                                               int64_t first, int64_t stride, const B& bind,
                                               const Buffers& b, unsigned* dirfail) {
  for (int64_t p = first; p < na; p += stride) {
    const sidm_pair r = pairs[p];
    if (b.mult[r.ia] == 1 && b.mult[r.ib] == 1) {
      interact(bind.model(r), bind.parts, bind.info(r, dirfail));
      publish_if_last(bind, r.ia, 0, 1);
      publish_if_last(bind, r.ib, 0, 1);
    }
  }
}

template <class B, class S>
__global__ void __launch_bounds__(kThreads) dataflow_kernel(const sidm_pair* __restrict__ pairs,
                                                            int64_t cap, int max_passes, B bind,
                                                            Buffers b, S* st) {
  __shared__ unsigned s_dirfail;
  __shared__ int s_passes;
  if (threadIdx.x == 0) { s_dirfail = 0; s_passes = 0; }
  __syncthreads();
  if (!overflowed(st, cap)) {
    const int64_t np = (int64_t)st->n_pending;
    const int64_t na = (int64_t)st->n_acc;
    const int64_t gsize = (int64_t)gridDim.x * kThreads;
    // pending pair k to block k mod G: the pairs (and their FP64 kicks)
    // spread over every SM, each warp still holding 32 of them
    const int64_t t0 = threadIdx.x * (int64_t)gridDim.x + blockIdx.x;
    // warps 0 .. busy-1 of every block hold the pending pairs; the others
    // apply the isolated pairs meanwhile
    constexpr int kWarps = kThreads / 32;
    const int warp = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31);
    const int64_t busy = (np + 32 * (int64_t)gridDim.x - 1) / (32 * (int64_t)gridDim.x);
    if (busy < kWarps && warp >= busy)
      apply_isolated(pairs, na, ((warp - busy) * 32 + lane) * (int64_t)gridDim.x + blockIdx.x,
                     (kWarps - busy) * 32 * (int64_t)gridDim.x, bind, b, &s_dirfail);
    // the thread's first pair, prepared before its turn
    bool first = t0 < np;
    Turn<B> f0;
    if (first) {
      const int32_t p = b.pending[t0];
      f0.load(bind, pairs[p], b, p, &s_dirfail);
    }
    // passes of the whole warp (apply_ready may work across its lanes)
    int pass = 0;
    bool left = first;
    for (; pass < max_passes; ++pass) {
      if (!__any_sync(0xffffffffu, left)) break;
      left = false;
      bool ready = false;
      if (first) {
        const int ca = ld_acquire(&b.cursor[f0.r.ia]);
        const int cb = ld_acquire(&b.cursor[f0.r.ib]);
        ready = ca == f0.pa && cb == f0.pb;
        left = !ready;
      }
      f0.apply_ready(bind, b, ready, &s_dirfail);
      if (ready) first = false;
      // further pairs of this thread (more pending pairs than threads)
      for (int64_t k = t0 + gsize; k < np; k += gsize) {
        const int32_t p = b.pending[k];
        if (b.flags[p]) continue;
        const sidm_pair r = pairs[p];
        const int pa = b.pos_a[p], pb = b.pos_b[p];
        const int ca = ld_acquire(&b.cursor[r.ia]);
        const int cb = ld_acquire(&b.cursor[r.ib]);
        if (ca == pa && cb == pb) {
          interact(bind.model(r), bind.parts, bind.info(r, &s_dirfail));
          fence_acq_rel();
          st_relaxed(&b.cursor[r.ia], pa + 1);
          st_relaxed(&b.cursor[r.ib], pb + 1);
          b.flags[p] = 1;
          if constexpr (has_publish<B>::value) {
            publish_if_last(bind, r.ia, pa, b.mult[r.ia]);
            publish_if_last(bind, r.ib, pb, b.mult[r.ib]);
          }
        } else {
          left = true;
        }
      }
    }
    if (left) atomicOr(&st->status, kErrRounds);
    atomicMax(&s_passes, pass);
    if (busy >= kWarps) apply_isolated(pairs, na, t0, gsize, bind, b, &s_dirfail);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicMax(&st->n_rounds, (unsigned long long)s_passes);
    if (s_dirfail) {
      atomicAdd(&st->n_dirfail, (unsigned long long)s_dirfail);
      atomicOr(&st->status, kDirFail);
    }
  }
}

template <class S>
__global__ void __launch_bounds__(kThreads) reset_kernel(const sidm_pair* __restrict__ pairs,
                                                         int64_t cap, Buffers b, const S* st) {
  const unsigned long long nall = st->n_acc;
  if (overflowed(st, cap)) return;
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  const int64_t t0 = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  for (int64_t p = t0; p < (int64_t)nall; p += stride) {
    b.mult[pairs[p].ia] = 0;
    b.mult[pairs[p].ib] = 0;
  }
  const int64_t nt = (int64_t)st->n_touched;
  for (int64_t k = t0; k < nt; k += stride) {
    const int32_t e = b.touched[k];
    b.seg_off[e] = -1;
    b.fill[e] = 0;
    b.cursor[e] = 0;
  }
}

template <class B, class S>
int dataflow_grid(int sms) {
  static int per_sm = -1;   // per instantiation
  if (per_sm < 0) {
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, dataflow_kernel<B, S>, kThreads, 0) !=
            cudaSuccess ||
        v < 1)
      v = 1;
    per_sm = v;
  }
  return per_sm * sms;
}

// The whole sequence on stream s; returns the number of kernels launched,
// or -1 if the cooperative launch was refused.
template <class B, class S>
int launch_apply(const sidm_pair* pairs, int64_t cap, int max_passes, const B& bind,
                 const Buffers& b, S* st, int sms, cudaStream_t s) {
  const unsigned g = (unsigned)(sms * 4);
  count_kernel<S><<<g, kThreads, 0, s>>>(pairs, cap, b.mult, st);
  split_kernel<B, S><<<g, kThreads, 0, s>>>(pairs, cap, bind, b, st);
  fill_kernel<S><<<g, kThreads, 0, s>>>(pairs, cap, b, st);
  rank_kernel<S><<<g, kThreads, 0, s>>>(pairs, cap, b, st);
  // cooperative launch: every block resident, as the passes wait on each other
  const sidm_pair* pp = pairs;
  int64_t cp = cap;
  int mp = max_passes > 0 ? max_passes : kMaxPasses;
  B bb = bind;
  Buffers buf = b;
  S* sp = st;
  void* args[] = {(void*)&pp, (void*)&cp, (void*)&mp, (void*)&bb, (void*)&buf, (void*)&sp};
  if (cudaLaunchCooperativeKernel((const void*)dataflow_kernel<B, S>,
                                  dim3(dataflow_grid<B, S>(sms)), dim3(kThreads), args, 0,
                                  s) != cudaSuccess)
    return -1;
  reset_kernel<S><<<g, kThreads, 0, s>>>(pairs, cap, b, st);
  return 6;
}

// ---- apply_pairs: the caller's pairs, one random key and step
template <class M>
struct FixedBinder {
  M m;
  typename M::Particles parts;
  uint32_t k0, k1, step;
  __device__ __forceinline__ M model(const sidm_pair&) const { return m; }
  __device__ __forceinline__ PairInfo info(const sidm_pair& r, unsigned* warn) const {
    return PairInfo{r.a, r.b, r.ia, r.ib, k0, k1, step, warn};
  }
};

template <class S>
__global__ void check_kernel(const sidm_pair* __restrict__ pairs, int64_t n_pairs, int64_t n,
                             S* c) {
  bool bad = false;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n_pairs;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ia = pairs[p].ia, ib = pairs[p].ib;
    if (ia < 0 || ia >= n || ib < 0 || ib >= n || ia == ib) bad = true;
  }
  if (bad) atomicOr(&c->status, kErrInvalid);
}

template <class S>
__global__ void arm_kernel(int64_t n_pairs, S* c) {
  // an invalid record leaves the count at 0: nothing is applied
  c->n_acc = (c->status & kErrInvalid) ? 0ull : (unsigned long long)n_pairs;
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace detail

// Scratch bytes apply_pairs needs for n particles and n_pairs pairs.
inline size_t apply_pairs_scratch_bytes(int64_t n, int64_t n_pairs) {
  using detail::align256;
  const size_t a = (size_t)(n > 0 ? n : 1), p = (size_t)(n_pairs > 0 ? n_pairs : 1);
  return align256(sizeof(detail::Counters)) + 4 * align256(4 * a) + 3 * align256(8 * p) +
         3 * align256(4 * p) + align256(p);
}

// Applies n_pairs accepted pairs (device records; ia, ib index the model's
// particle arrays, a < b the ids that key the random streams) with model m in
// ascending (ord, a, b) order, records with equal keys in the order given.
// seed, step: the Philox key and counter word 0 of the draws (step mod 2^32).
// scratch: device memory of at least apply_pairs_scratch_bytes(n, n_pairs),
// 256-byte aligned, owned by the caller; nothing is allocated.  Waits for
// the stream; returns SIDM_OK, SIDM_WARN_DIRECTION (the model counted a
// warning), SIDM_ERR_INVALID_ARG (bad sizes or pointers, scratch too small,
// or a record whose index lies outside [0, n) or names one particle twice:
// then nothing is applied), SIDM_ERR_DEVICE_LIMIT (the bounded wait of the
// application gave up; some interactions are applied) or SIDM_ERR_CUDA.
template <class M>
int apply_pairs(const M& m, const typename M::Particles& parts, const sidm_pair* pairs,
                int64_t n_pairs, int64_t n, uint64_t seed, uint64_t step, void* scratch,
                size_t scratch_bytes, cudaStream_t s, int max_passes = 0) {
  using namespace detail;
  if (n < 0 || n_pairs < 0 || n >= ((int64_t)1 << 31) || n_pairs >= ((int64_t)1 << 30))
    return SIDM_ERR_INVALID_ARG;
  if (n_pairs == 0) return SIDM_OK;
  if (!pairs || !scratch || ((uintptr_t)scratch & 255) ||
      scratch_bytes < apply_pairs_scratch_bytes(n, n_pairs))
    return SIDM_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SIDM_ERR_CUDA;
  const size_t a = (size_t)n, p = (size_t)n_pairs;
  char* at = (char*)scratch;
  auto take = [&](size_t bytes) {
    char* r = at;
    at += align256(bytes);
    return (void*)r;
  };
  Counters* c = (Counters*)take(sizeof(Counters));
  Buffers b;
  b.mult = (int32_t*)take(4 * a);
  b.seg_off = (int32_t*)take(4 * a);
  b.fill = (int32_t*)take(4 * a);
  b.cursor = (int32_t*)take(4 * a);
  b.seg = (int32_t*)take(8 * p);
  b.seg_e = (int32_t*)take(8 * p);
  b.touched = (int32_t*)take(8 * p);
  b.pending = (int32_t*)take(4 * p);
  b.pos_a = (int32_t*)take(4 * p);
  b.pos_b = (int32_t*)take(4 * p);
  b.flags = (uint8_t*)take(p);
  if (cudaMemsetAsync(c, 0, sizeof(Counters), s) != cudaSuccess ||
      cudaMemsetAsync(b.mult, 0, 4 * a, s) != cudaSuccess ||
      cudaMemsetAsync(b.seg_off, 0xFF, 4 * a, s) != cudaSuccess ||
      cudaMemsetAsync(b.fill, 0, 4 * a, s) != cudaSuccess ||
      cudaMemsetAsync(b.cursor, 0, 4 * a, s) != cudaSuccess)
    return SIDM_ERR_CUDA;
  check_kernel<Counters><<<sms * 4, kThreads, 0, s>>>(pairs, n_pairs, n, c);
  arm_kernel<Counters><<<1, 1, 0, s>>>(n_pairs, c);
  FixedBinder<M> bind{m, parts, (uint32_t)seed, (uint32_t)(seed >> 32), (uint32_t)step};
  if (launch_apply(pairs, n_pairs, max_passes, bind, b, c, sms, s) < 0) return SIDM_ERR_CUDA;
  if (cudaGetLastError() != cudaSuccess) return SIDM_ERR_CUDA;
  unsigned status = 0;
  if (cudaMemcpyAsync(&status, &c->status, sizeof(status), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return SIDM_ERR_CUDA;
  if (status & kErrInvalid) return SIDM_ERR_INVALID_ARG;
  if (status & (kErrRounds | kErrPairOverflow)) return SIDM_ERR_DEVICE_LIMIT;
  return (status & kDirFail) ? SIDM_WARN_DIRECTION : SIDM_OK;
}

}  // namespace sidm_model
