// C ABI of the SIDM scattering-step library: context, buffers, haloes,
// validation and the order of the kernels of one step.
//
// Step (all on the context's stream, no host round trip unless statistics
// are requested):
//   halo table upload -> bounding box per halo -> start radius / key
//   transform per halo -> halo-prefixed spatial keys -> radix sort ->
//   key-order copy of the state + active list -> 32-ary box tree per halo ->
//   h_SI per active particle -> candidate pairs, probabilities and draws,
//   Eq. 18 limits -> canonical application of the accepted kicks.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "sidm_internal.cuh"

using namespace sidm;

struct sidm_ctx {
  sidm_config cfg{};
  int device = 0;
  int sms = 148;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int64_t n = 0, cap = 0, pair_cap = 0;
  uint64_t step = 0;
  bool loaded = false;

  // user order
  double *pos = nullptr, *vel = nullptr, *mass = nullptr, *h_user = nullptr, *dtlim = nullptr;
  uint32_t* ids = nullptr;
  int32_t* halo_of = nullptr;   // halo of each particle
  uint8_t* act = nullptr;
  int8_t* bins = nullptr;
  // sort
  uint32_t *keys = nullptr, *keys_alt = nullptr;
  int32_t *vals = nullptr, *vals_alt = nullptr;
  void* sort_tmp = nullptr;
  // key order
  Sorted so{};
  int32_t* act_list = nullptr;
  int32_t* nb_list = nullptr;   // [n][nb_stride] neighbour lists of the active particles
  int32_t* nb_count = nullptr;  // [n] list length, or -1
  int2* deferred = nullptr;     // [pair_cap] draws for the exact FP64 pass
  int32_t* lim_cand = nullptr;  // [n][LIM_CAND] Eq. 18 candidates of each query
  int32_t* lim_cnt = nullptr;   // [n]
  float* lim_g = nullptr;       // [n]
  int nb_stride = 0;
  // haloes and their trees
  std::vector<Halo> halos;      // host copy (layout + per-step parameters)
  Halo* d_halos = nullptr;
  int halo_cap = 0;
  Forest forest{};
  int64_t node_cap = 0;
  float4 *node_lo = nullptr, *node_hi = nullptr;
  // per step
  DevStats* dstats = nullptr;
  unsigned* latched = nullptr;
  int* work = nullptr;
  PairRec* pairs = nullptr;
  ResolveBuffers rb{};          // per-particle segments and cursors of the resolver
  double *cons_partial = nullptr, *cons = nullptr;
  // pinned host staging
  DevStats* h_stats = nullptr;
  double* h_cons = nullptr;
  unsigned* h_latched = nullptr;
  std::vector<void*> allocs;
  // tabulated sigma/m (one device buffer, see SigmaTable)
  SigmaTable table{};
  void* table_mem = nullptr;
  // table of the kernel-overlap estimator
  OverlapTable ov{};
  void* ov_mem = nullptr;
  // launch shapes and the captured step
  LaunchTuning tune{};
  uint64_t layout_version = 1;  // bumped whenever buffers, haloes or tuning change
  // captured steps: [0] refit only, [1] full rebuild (keys + sort); each in
  // two parts, [.][0] up to the search and [.][1] from the key-order
  // velocities on, so that a velocity upload can run beside the first part
  cudaGraphExec_t graph_exec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  uint64_t graph_version[2] = {0, 0};  // layout each graph was captured for
  int64_t graph_launches[2] = {0, 0};  // kernels in each graph (both parts)
  int graph_state = 0;          // 0 off, 1 captured, -1 capture refused (direct launches)
  // velocity uploads on a side stream: they overlap the first part of the
  // next step; every use of the velocities waits for them (join_velocities)
  cudaStream_t vstream = nullptr;
  cudaEvent_t ev_vfree = nullptr;   // the stream's earlier work on the velocities
  cudaEvent_t ev_vdone = nullptr;   // the upload
  bool vel_pending = false;
  // particles changed by the last step (sidm_get_changed)
  uint32_t* chg_stamps = nullptr;   // [n] number of the call that listed the particle
  int32_t* chg_idx = nullptr;       // [n]
  double* chg_vel = nullptr;        // [3 n]
  unsigned long long* chg_count = nullptr;
  unsigned long long* h_chg_count = nullptr;   // pinned
  uint32_t chg_call = 0;
  int32_t* h_chg_idx = nullptr;     // pinned staging of sidm_update_velocities
  double* h_chg_vel = nullptr;
  int64_t h_chg_cap = 0;
  // pinned host copy of the velocities kept current by the kicks
  // (sidm_set_velocity_mirror): its device address and its length in particles
  double* mirror = nullptr;
  int64_t mirror_n = 0;
  bool stepped = false;             // a step ran since the particles were loaded
  // key order kept between full rebuilds
  uint64_t order_version = 0;   // layout of the last full rebuild
  int64_t since_rebuild = 0;    // steps since it
  // sizing only (sidm_context_bytes): dalloc counts bytes and allocates nothing
  bool dry_run = false;
  int64_t dry_bytes = 0;
  // instrumentation
  int64_t launches = 0;
  cudaEvent_t ev[SIDM_N_PHASES + 1] = {};
  bool have_events = false;
  bool timed_step = false;
};

namespace {

int cuda_fail(cudaError_t e) {
  if (e == cudaErrorMemoryAllocation) return SIDM_ERR_OOM;
  return SIDM_ERR_CUDA;
}

#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_);   \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

// Device memory of the context: the caller's allocator when the config
// names one (e.g. a caching allocator of the host framework), else
// cudaMalloc.  Sizes are rounded up to 256 bytes.
cudaError_t raw_alloc(sidm_ctx* c, void** p, size_t bytes) {
  bytes = (std::max<size_t>(bytes, 1) + 255) & ~(size_t)255;
  if (c->cfg.alloc) {
    *p = c->cfg.alloc(bytes, (void*)c->stream, c->cfg.alloc_user);
    return *p ? cudaSuccess : cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

void raw_free(sidm_ctx* c, void* p) {
  if (!p) return;
  if (c->cfg.free) c->cfg.free(p, (void*)c->stream, c->cfg.alloc_user);
  else cudaFree(p);
}

template <class T>
cudaError_t dalloc(sidm_ctx* c, T** p, size_t count) {
  const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  if (c->dry_run) {
    c->dry_bytes += (int64_t)((bytes + 255) & ~(size_t)255);
    *p = nullptr;
    return cudaSuccess;
  }
  void* q = nullptr;
  cudaError_t e = raw_alloc(c, &q, bytes);
  if (e != cudaSuccess) return e;
  c->allocs.push_back(q);
  *p = (T*)q;
  return cudaSuccess;
}

void drop_graph(sidm_ctx* c) {
  for (int k = 0; k < 2; ++k) {
    for (int part = 0; part < 2; ++part) {
      if (c->graph_exec[k][part]) cudaGraphExecDestroy(c->graph_exec[k][part]);
      c->graph_exec[k][part] = nullptr;
    }
    c->graph_version[k] = 0;
  }
}

// Orders the context's stream after a pending velocity upload.
cudaError_t join_velocities(sidm_ctx* c) {
  if (!c->vel_pending) return cudaSuccess;
  c->vel_pending = false;
  return cudaStreamWaitEvent(c->stream, c->ev_vdone, 0);
}

void free_buffers(sidm_ctx* c) {
  drop_graph(c);
  ++c->layout_version;
  for (void* p : c->allocs) raw_free(c, p);
  c->allocs.clear();
  c->cap = 0;
  c->pair_cap = 0;
  c->halo_cap = 0;
  c->node_cap = 0;
  c->d_halos = nullptr;
  c->node_lo = c->node_hi = nullptr;
}

__global__ void fill_kernel(double* p, int64_t n, double v) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

__global__ void fill_halo_kernel(int32_t* halo_of, int64_t start, int64_t n, int k) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) halo_of[start + i] = k;
}

__global__ void latch_kernel(const DevStats* st, unsigned* latched) {
  if (threadIdx.x == 0 && st->status) atomicOr(latched, st->status);
}

void fill(double* p, int64_t n, double v, cudaStream_t s) {
  if (n > 0) fill_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, n, v);
}

int64_t pair_capacity_for(const sidm_config& cfg, int64_t want) {
  return cfg.pair_capacity > 0 ? cfg.pair_capacity : 2 * want + 4096;
}

// Every buffer sized by the particle capacity (dalloc only: with dry_run
// set it just counts the bytes).
int alloc_capacity(sidm_ctx* c, int64_t want) {
  const int64_t pc = pair_capacity_for(c->cfg, want);
  CK(dalloc(c, &c->pos, 3 * want));
  CK(dalloc(c, &c->vel, 3 * want));
  CK(dalloc(c, &c->mass, want));
  CK(dalloc(c, &c->h_user, want));
  CK(dalloc(c, &c->dtlim, want));
  CK(dalloc(c, &c->ids, want));
  CK(dalloc(c, &c->halo_of, want));
  CK(dalloc(c, &c->act, want));
  CK(dalloc(c, &c->bins, want));
  CK(dalloc(c, &c->keys, want));
  CK(dalloc(c, &c->keys_alt, want));
  CK(dalloc(c, &c->vals, want));
  CK(dalloc(c, &c->vals_alt, want));
  CK(dalloc(c, (char**)&c->sort_tmp, radix_sort_temp_bytes(want)));
  Sorted& so = c->so;
  CK(dalloc(c, &so.x, want));
  CK(dalloc(c, &so.y, want));
  CK(dalloc(c, &so.z, want));
  CK(dalloc(c, &so.vx, want));
  CK(dalloc(c, &so.vy, want));
  CK(dalloc(c, &so.vz, want));
  CK(dalloc(c, &so.m, want));
  CK(dalloc(c, &so.h, want));
  CK(dalloc(c, &so.dt, want));
  CK(dalloc(c, &so.f, want));
  CK(dalloc(c, &so.vm, want));
  CK(dalloc(c, &so.hb, want));
  CK(dalloc(c, &so.id, want));
  CK(dalloc(c, &so.act, want));
  CK(dalloc(c, &so.orig, want));
  CK(dalloc(c, &so.halo, want));
  CK(dalloc(c, &c->act_list, want));
  c->nb_stride = c->cfg.n_ngb + c->cfg.ngb_tol;
  CK(dalloc(c, &c->nb_count, want));
  CK(dalloc(c, &c->nb_list, want * (int64_t)c->nb_stride));
  CK(dalloc(c, &c->dstats, 1));
  CK(dalloc(c, &c->latched, 1));
  CK(dalloc(c, &c->work, 8));
  CK(dalloc(c, &c->pairs, pc));
  CK(dalloc(c, &c->deferred, pc));
  CK(dalloc(c, &c->lim_cand, want * (int64_t)LIM_CAND));
  CK(dalloc(c, &c->lim_cnt, want));
  CK(dalloc(c, &c->lim_g, want));
  ResolveBuffers& rb = c->rb;
  CK(dalloc(c, &rb.mult, want));
  CK(dalloc(c, &rb.seg_off, want));
  CK(dalloc(c, &rb.fill, want));
  CK(dalloc(c, &rb.cursor, want));
  CK(dalloc(c, &rb.seg, 2 * pc));
  CK(dalloc(c, &rb.seg_e, 2 * pc));
  CK(dalloc(c, &rb.touched, 2 * pc));
  CK(dalloc(c, &rb.pending, pc));
  CK(dalloc(c, &rb.flags, pc));
  CK(dalloc(c, &rb.pos_a, pc));
  CK(dalloc(c, &rb.pos_b, pc));
  CK(dalloc(c, &c->cons_partial, 4 * conserved_blocks()));
  CK(dalloc(c, &c->cons, 8));
  CK(dalloc(c, &c->chg_stamps, want));
  CK(dalloc(c, &c->chg_idx, want));
  CK(dalloc(c, &c->chg_vel, 3 * want));
  CK(dalloc(c, &c->chg_count, 1));
  return SIDM_OK;
}

int ensure_capacity(sidm_ctx* c, int64_t n) {
  int64_t want = std::max<int64_t>(n, c->cfg.n_max);
  if (want <= c->cap && c->allocs.size()) return SIDM_OK;
  CK(cudaStreamSynchronize(c->stream));
  free_buffers(c);
  want = std::max<int64_t>(want, 64);
  const int64_t pc = pair_capacity_for(c->cfg, want);
  const int ra = alloc_capacity(c, want);
  if (ra != SIDM_OK) return ra;
  ResolveBuffers& rb = c->rb;
  CK(cudaMemsetAsync(c->chg_stamps, 0, want * sizeof(uint32_t), c->stream));
  CK(cudaMemsetAsync(rb.mult, 0, want * sizeof(int32_t), c->stream));
  CK(cudaMemsetAsync(rb.seg_off, 0xFF, want * sizeof(int32_t), c->stream));
  CK(cudaMemsetAsync(rb.fill, 0, want * sizeof(int32_t), c->stream));
  CK(cudaMemsetAsync(rb.cursor, 0, want * sizeof(int32_t), c->stream));
  CK(cudaMemsetAsync(c->latched, 0, sizeof(unsigned), c->stream));
  c->cap = want;
  c->pair_cap = pc;
  return SIDM_OK;
}

// Plain device buffers outside the capacity set (grown on demand).
template <class T>
cudaError_t grow(sidm_ctx* c, T** p, int64_t* have, int64_t need) {
  if (*p && *have >= need) return cudaSuccess;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return e;
  if (*p) {
    auto it = std::find(c->allocs.begin(), c->allocs.end(), (void*)*p);
    if (it != c->allocs.end()) c->allocs.erase(it);
    raw_free(c, *p);
    *p = nullptr;
  }
  return dalloc(c, p, (size_t)need);
}

// largest e (<= 60) with 8^e * n_ngb <= 4 n
int start_exponent(int64_t n, int n_ngb) {
  int e = 0;
  while (e < 60 && std::ldexp((double)n_ngb, 3 * (e + 1)) <= 4.0 * (double)n) ++e;
  return e;
}

// Halo layout from segment offsets (host): particle ranges, tree levels and
// node offsets (level-major), start-radius exponents; fills halo_of.
int layout_haloes(sidm_ctx* c, int n_halos, const int64_t* off) {
  // a new layout (particle ranges) invalidates the key order and the captured steps
  bool same = (int)c->halos.size() == n_halos;
  for (int k = 0; same && k < n_halos; ++k)
    same = c->halos[k].start == off[k] && c->halos[k].n == off[k + 1] - off[k];
  if (!same) ++c->layout_version;
  std::vector<Halo>& H = c->halos;
  H.assign(n_halos, Halo{});
  Forest& f = c->forest;
  std::memset(f.level_nodes, 0, sizeof(f.level_nodes));
  f.max_levels = 0;
  for (int k = 0; k < n_halos; ++k) {
    Halo& h = H[k];
    h.start = off[k];
    h.n = off[k + 1] - off[k];
    h.levels = tree_levels_for(h.n, h.node_cnt);
    for (int l = h.levels; l < MAX_LEVELS; ++l) h.node_cnt[l] = 0;
    h.e0 = start_exponent(h.n, c->cfg.n_ngb);
    for (int l = 0; l < MAX_LEVELS; ++l) f.level_nodes[l] += h.node_cnt[l];
    f.max_levels = std::max(f.max_levels, h.levels);
  }
  int64_t base = 0;
  for (int l = 0; l < MAX_LEVELS; ++l) {
    int64_t run = base;
    for (int k = 0; k < n_halos; ++k) {
      H[k].node_off[l] = run;
      run += H[k].node_cnt[l];
    }
    base += f.level_nodes[l];
  }
  int bits = 0;
  while ((1 << bits) < n_halos) ++bits;
  f.n_halos = n_halos;
  f.halo_bits = n_halos > 1 ? bits : 0;
  int64_t have = c->node_cap;
  CK(grow(c, &c->node_lo, &have, std::max<int64_t>(base, 1)));
  have = c->node_cap;
  CK(grow(c, &c->node_hi, &have, std::max<int64_t>(base, 1)));
  c->node_cap = std::max<int64_t>(c->node_cap, std::max<int64_t>(base, 1));
  int64_t hc = c->halo_cap;
  CK(grow(c, &c->d_halos, &hc, std::max(n_halos, 1)));
  c->halo_cap = std::max(c->halo_cap, std::max(n_halos, 1));
  f.lo = c->node_lo;
  f.hi = c->node_hi;
  f.halos = c->d_halos;
  for (int k = 0; k < n_halos; ++k)
    if (H[k].n > 0)
      fill_halo_kernel<<<(unsigned)((H[k].n + 255) / 256), 256, 0, c->stream>>>(
          c->halo_of, H[k].start, H[k].n, k);
  CK(cudaGetLastError());
  return SIDM_OK;
}

// Uploads the halo table (pageable copy: the host vector may change after).
int upload_haloes(sidm_ctx* c) {
  if (c->halos.empty()) return SIDM_OK;
  CK(cudaMemcpyAsync(c->d_halos, c->halos.data(), c->halos.size() * sizeof(Halo),
                     cudaMemcpyHostToDevice, c->stream));
  return SIDM_OK;
}

cudaMemcpyKind copy_kind_in(int ptr_kind) {
  return ptr_kind == SIDM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
}
cudaMemcpyKind copy_kind_out(int ptr_kind) {
  return ptr_kind == SIDM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int status_from_bits(unsigned bits) {
  if (bits & ST_ERR_MASK) return SIDM_ERR_DEVICE_LIMIT;
  int w = 0;
  if (bits & ST_H_NONCONV) w |= SIDM_WARN_H_NOT_CONVERGED;
  if (bits & ST_P_GE_1) w |= SIDM_WARN_P_GE_1;
  if (bits & ST_DIR_FAIL) w |= SIDM_WARN_DIRECTION;
  return w;
}

// Waits for the stream and returns (and clears) the latched device status.
int wait_and_collect(sidm_ctx* c) {
  CK(cudaMemcpyAsync(c->h_latched, c->latched, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemsetAsync(c->latched, 0, sizeof(unsigned), c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return status_from_bits(*c->h_latched);
}

bool valid_sigma(const sidm_ctx* c, const sidm_sigma_model& s) {
  if (!std::isfinite(s.inelastic) || !(s.inelastic <= 1.0)) return false;
  if (s.kind == SIDM_SIGMA_TABLE) return c->table.n >= 2;
  return (s.sigma0 >= 0.0) && std::isfinite(s.sigma0) &&
         (s.kind == SIDM_SIGMA_CONST || (s.kind == SIDM_SIGMA_YUKAWA && s.w > 0.0 && std::isfinite(s.w)));
}

void set_step_params(Halo& h, double dt_max, const sidm_sigma_model& s, uint64_t seed,
                     uint64_t step) {
  h.dt_max = dt_max;
  h.sigma_kind = s.kind;
  h.sigma0 = s.sigma0;
  h.w = s.kind == SIDM_SIGMA_YUKAWA ? s.w : 1.0;
  h.eps = 1.0 - s.inelastic;
  h.seed = seed;
  h.step = (uint32_t)step;
}

// The kernels of one step over every halo (the halo table is set).
// The kernels of one step, from the reset of the step counters to the
// status latch.  They read only device buffers of the context (the ingest
// copies and the halo table upload come before), so the sequence can be
// captured once into a CUDA graph and replayed while the particle count,
// the halo layout, the buffers and the launch shapes stay the same.
// part 0: from the counter reset to the search (positions only); part 1:
// from the key-order velocities to the status latch.
int launch_core(sidm_ctx* c, bool prof, bool rebuild, int64_t* launches, int part) {
  const int64_t n = c->n;
  cudaStream_t s = c->stream;
  int64_t L = 0;
  if (part == 0) {
    CK(cudaMemsetAsync(c->dstats, 0, sizeof(DevStats), s));
    CK(cudaMemsetAsync(c->work, 0, 8 * sizeof(int), s));
  }
  auto mark = [&](int k) {
    if (prof) cudaEventRecord(c->ev[k], s);
  };
  const int nh = (int)c->halos.size();
  const Forest& F = c->forest;
  if (n > 0 && part == 0) {
    mark(0);
    L += launch_bbox(c->pos, c->halo_of, n, c->d_halos, nh, s);
    L += launch_params(c->d_halos, nh, c->cfg.box, s);
    // the key's width sets the sort's passes; an odd count starts from the
    // alternate buffers, so that the sorted order lands in keys / vals
    const int key_bits = F.halo_bits + 3 * key_axis_bits(F.halo_bits);
    const bool odd = (sort_passes(key_bits) & 1) != 0;
    uint32_t* k_in = odd ? c->keys_alt : c->keys;
    int32_t* v_in = odd ? c->vals_alt : c->vals;
    uint32_t* k_out = odd ? c->keys : c->keys_alt;
    int32_t* v_out = odd ? c->vals : c->vals_alt;
    if (rebuild)
      L += launch_keys(c->pos, c->halo_of, n, c->d_halos, F.halo_bits, c->cfg.box, k_in, v_in, s);
    mark(1);
    if (rebuild) {
      const int sl = radix_sort_pairs(k_in, v_in, k_out, v_out, n, key_bits, c->sort_tmp,
                                      &c->dstats->status, s);
      if (sl < 0) return SIDM_ERR_CUDA;
      L += sl;
    }
    mark(2);
    L += launch_permute(c->vals, n, c->pos, c->mass, c->ids, c->halo_of, c->act,
                        c->bins, c->d_halos, c->so, c->act_list, c->dstats, s);
    L += launch_forest(c->so, F, s);
    mark(3);
    L += launch_search(c->so, F, n, c->act_list, c->cfg.box, c->cfg.n_ngb, c->cfg.ngb_tol,
                       c->cfg.fixed_h, c->cfg.kernel, c->cfg.precision == SIDM_FP32_SPLIT,
                       c->h_user,
                       c->nb_list, c->nb_count, c->nb_stride,
                       c->dstats, c->work, c->sms, c->tune,
                       c->cfg.estimator == SIDM_ESTIMATOR_OVERLAP, c->cfg.search_hint != 0, s);
    if (c->cfg.estimator == SIDM_ESTIMATOR_OVERLAP) L += launch_hmax(c->so, F, s);
    mark(4);
  }
  if (n > 0 && part == 1) {
    L += launch_permute_vel(n, c->vel, c->so, s);
    PairArgs pa;
    pa.kernel = c->cfg.kernel;
    pa.split = c->cfg.precision == SIDM_FP32_SPLIT;
    pa.c_sidm = c->cfg.c_sidm;
    pa.box = c->cfg.box;
    pa.pair_cap = c->pair_cap;
    pa.deferred = c->deferred;
    pa.lim_cand = c->lim_cand;
    pa.lim_cnt = c->lim_cnt;
    pa.lim_g = c->lim_g;
    pa.table = c->table;
    pa.ov = c->cfg.estimator == SIDM_ESTIMATOR_OVERLAP ? c->ov : OverlapTable{};
    L += launch_pairs(c->so, F, n, c->act_list, c->nb_list, c->nb_count, c->nb_stride, pa,
                      c->pairs, c->dtlim, c->dstats, c->work + 1, c->sms, c->tune, s);
    mark(5);
    const int nr = launch_resolve(c->pairs, c->pair_cap, c->cfg.max_resolver_passes, c->vel,
                                  c->mass, c->halo_of, c->d_halos, c->mirror, c->rb, c->dstats,
                                  c->sms, s);
    if (nr < 0) return SIDM_ERR_CUDA;
    L += nr;
    mark(6);
  }
  if (part == 1) {
    latch_kernel<<<1, 32, 0, s>>>(c->dstats, c->latched);
    L += 1;
  }
  *launches = L;
  return SIDM_OK;
}

// Captures launch_core into a graph; a capture the driver refuses leaves the
// context on direct launches (graph_state -1).
void capture_core(sidm_ctx* c, int rebuild) {
  int64_t total = 0;
  for (int part = 0; part < 2; ++part) {
    cudaGraphExec_t& x = c->graph_exec[rebuild][part];
    if (x) cudaGraphExecDestroy(x);
    x = nullptr;
  }
  for (int part = 0; part < 2; ++part) {
    cudaGraphExec_t& x = c->graph_exec[rebuild][part];
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      c->graph_state = -1;
      return;
    }
    int64_t k = 0;
    const int r = launch_core(c, false, rebuild != 0, &k, part);
    const cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (r != SIDM_OK || e != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      c->graph_state = -1;
      return;
    }
    const cudaError_t ei = cudaGraphInstantiate(&x, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      x = nullptr;
      cudaGetLastError();
      c->graph_state = -1;
      return;
    }
    total += k;
  }
  c->graph_version[rebuild] = c->layout_version;
  c->graph_launches[rebuild] = total;
  c->graph_state = 1;
}

int run_step(sidm_ctx* c, const uint8_t* active_mask, const int8_t* dt_bins,
             sidm_step_stats* stats) {
  if (c->cfg.estimator == SIDM_ESTIMATOR_OVERLAP && c->ov.na <= 0) return SIDM_ERR_NOT_READY;
  if (c->mirror && c->n > c->mirror_n) return SIDM_ERR_INVALID_ARG;   // the copy is too short
  const int64_t n = c->n;
  cudaStream_t s = c->stream;
  if (n > 0) {
    if (active_mask)
      CK(cudaMemcpyAsync(c->act, active_mask, n, is_device_ptr(active_mask)
                                                      ? cudaMemcpyDeviceToDevice
                                                      : cudaMemcpyHostToDevice, s));
    else
      CK(cudaMemsetAsync(c->act, 1, n, s));
    if (dt_bins)
      CK(cudaMemcpyAsync(c->bins, dt_bins, n, is_device_ptr(dt_bins) ? cudaMemcpyDeviceToDevice
                                                                     : cudaMemcpyHostToDevice, s));
    else
      CK(cudaMemsetAsync(c->bins, 0, n, s));
  }
  const int r0 = upload_haloes(c);
  if (r0 != SIDM_OK) return r0;
  int64_t& L = c->launches;
  if (stats) {
    CK(join_velocities(c));
    L += launch_conserved(c->vel, c->mass, n, c->cons_partial, c->cons, s);
  }
  const bool prof = c->have_events && n > 0;
  c->timed_step = prof;
  // full rebuild (keys + sort) or a refit in the key order of the last one
  const int rebuild = (c->cfg.rebuild_every <= 1 || c->order_version != c->layout_version ||
                       c->since_rebuild >= c->cfg.rebuild_every) ? 1 : 0;
  bool done = false;
  if (c->cfg.use_graph && !prof && n > 0 && c->graph_state >= 0) {
    if (!c->graph_exec[rebuild][0] || !c->graph_exec[rebuild][1] ||
        c->graph_version[rebuild] != c->layout_version)
      capture_core(c, rebuild);
    if (c->graph_exec[rebuild][0] && c->graph_exec[rebuild][1]) {
      CK(cudaGraphLaunch(c->graph_exec[rebuild][0], s));
      CK(join_velocities(c));
      CK(cudaGraphLaunch(c->graph_exec[rebuild][1], s));
      L += c->graph_launches[rebuild];
      done = true;
    }
  }
  if (!done) {
    for (int part = 0; part < 2; ++part) {
      if (part == 1) CK(join_velocities(c));
      int64_t k = 0;
      const int r = launch_core(c, prof, rebuild != 0, &k, part);
      L += k;
      if (r != SIDM_OK) return r;
    }
  }
  if (rebuild) {
    c->order_version = c->layout_version;
    c->since_rebuild = 1;
  } else {
    ++c->since_rebuild;
  }
  CK(cudaGetLastError());
  c->step += 1;
  c->stepped = true;
  if (!stats) return SIDM_OK;
  L += launch_conserved(c->vel, c->mass, n, c->cons_partial, c->cons + 4, s);
  CK(cudaMemcpyAsync(c->h_stats, c->dstats, sizeof(DevStats), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(c->h_cons, c->cons, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
  const int st = wait_and_collect(c);
  const DevStats& d = *c->h_stats;
  std::memset(stats, 0, sizeof(*stats));
  stats->n_active = (int64_t)d.n_active;
  stats->n_candidate_pairs = (int64_t)d.n_cand;
  stats->n_accepted = (int64_t)d.n_acc;
  stats->n_rounds = (int64_t)d.n_rounds;
  stats->n_p_ge_1 = (int64_t)d.n_pge1;
  stats->n_h_nonconv = (int64_t)d.n_nonconv;
  stats->n_dir_fail = (int64_t)d.n_dirfail;
  stats->max_multiplicity = (int64_t)d.max_mult;
  stats->sum_p = d.sum_p;
  stats->e_before = c->h_cons[0];
  stats->p_before[0] = c->h_cons[1];
  stats->p_before[1] = c->h_cons[2];
  stats->p_before[2] = c->h_cons[3];
  stats->e_after = c->h_cons[4];
  stats->p_after[0] = c->h_cons[5];
  stats->p_after[1] = c->h_cons[6];
  stats->p_after[2] = c->h_cons[7];
  stats->status = st;
  return st;
}

}  // namespace

extern "C" {

void sidm_default_config(sidm_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->n_ngb = 32;
  cfg->ngb_tol = 5;
  cfg->c_sidm = 0.1;
  cfg->box = 0.0;
  cfg->kernel = SIDM_KERNEL_CUBIC;
  cfg->precision = SIDM_FP64_PLAIN;
  cfg->fixed_h = 0.0;
  cfg->n_max = 0;
  cfg->pair_capacity = 0;
  cfg->stream = nullptr;
  cfg->device = -1;
}

int sidm_create(const sidm_config* cfg, sidm_ctx** out) {
  if (!cfg || !out) return SIDM_ERR_INVALID_ARG;
  *out = nullptr;
  if (cfg->n_ngb < 1 || cfg->ngb_tol < 0 || cfg->ngb_tol >= cfg->n_ngb ||
      cfg->n_ngb + cfg->ngb_tol + 2 > 256 || !(cfg->c_sidm > 0.0) || !(cfg->box >= 0.0) ||
      !std::isfinite(cfg->box) || (cfg->kernel != SIDM_KERNEL_CUBIC && cfg->kernel != SIDM_KERNEL_TOPHAT) ||
      (cfg->precision != SIDM_FP64_PLAIN && cfg->precision != SIDM_FP32_SPLIT) ||
      !(cfg->fixed_h >= 0.0) || cfg->n_max < 0 ||
      cfg->pair_capacity < 0 || cfg->rebuild_every < 0 || cfg->max_resolver_passes < 0 ||
      (cfg->estimator != SIDM_ESTIMATOR_ONE_SIDED && cfg->estimator != SIDM_ESTIMATOR_OVERLAP) ||
      (!cfg->alloc) != (!cfg->free))
    return SIDM_ERR_INVALID_ARG;
  sidm_ctx* c = new (std::nothrow) sidm_ctx();
  if (!c) return SIDM_ERR_OOM;
  c->cfg = *cfg;
  int dev = cfg->device;
  if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) { delete c; return SIDM_ERR_CUDA; }
  c->device = dev;
  DeviceGuard g(dev);
  if (cudaFree(nullptr) != cudaSuccess) { delete c; return SIDM_ERR_CUDA; }
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev);
  if (cfg->stream) {
    c->stream = (cudaStream_t)cfg->stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return SIDM_ERR_CUDA;
    }
    c->own_stream = true;
  }
  if (cudaStreamCreateWithFlags(&c->vstream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_vfree, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_vdone, cudaEventDisableTiming) != cudaSuccess) {
    sidm_destroy(c);
    return SIDM_ERR_CUDA;
  }
  if (cudaMallocHost(&c->h_stats, sizeof(DevStats)) != cudaSuccess ||
      cudaMallocHost(&c->h_cons, 8 * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&c->h_latched, sizeof(unsigned)) != cudaSuccess ||
      cudaMallocHost(&c->h_chg_count, sizeof(unsigned long long)) != cudaSuccess) {
    sidm_destroy(c);
    return SIDM_ERR_OOM;
  }
  if (cfg->profile) {
    for (int k = 0; k <= SIDM_N_PHASES; ++k)
      if (cudaEventCreate(&c->ev[k]) != cudaSuccess) { sidm_destroy(c); return SIDM_ERR_CUDA; }
    c->have_events = true;
  }
  if (cfg->n_max > 0) {
    const int r = ensure_capacity(c, cfg->n_max);
    if (r != SIDM_OK) { sidm_destroy(c); return r; }
  }
  *out = c;
  return SIDM_OK;
}

int sidm_phase_times(sidm_ctx* c, float* ms, int n) {
  if (!c || !ms || n < 0 || !c->have_events || !c->timed_step) return SIDM_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  CK(cudaEventSynchronize(c->ev[SIDM_N_PHASES]));
  for (int k = 0; k < n && k < SIDM_N_PHASES; ++k) CK(cudaEventElapsedTime(&ms[k], c->ev[k], c->ev[k + 1]));
  return SIDM_OK;
}

int64_t sidm_kernel_launches(const sidm_ctx* c) { return c ? c->launches : -1; }

// Periodic box: checks that every loaded coordinate lies in [0, box) (one
// bounding-box pass over all haloes together; waits for the stream).
int check_in_box(sidm_ctx* c) {
  const int64_t n = c->n;
  const int nh = (int)c->halos.size();
  int r = upload_haloes(c);
  if (r != SIDM_OK) return r;
  launch_bbox(c->pos, c->halo_of, n, c->d_halos, nh, c->stream);
  std::vector<unsigned long long> hm(6 * (size_t)nh);
  for (int k = 0; k < nh; ++k)
    CK(cudaMemcpyAsync(hm.data() + 6 * k, (const char*)(c->d_halos + k) + offsetof(Halo, mm),
                       6 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  for (int k = 0; k < nh; ++k)
    for (int a = 0; a < 3; ++a) {
      const double lo = ordered_to_dbl(hm[6 * k + a]), hi = ordered_to_dbl(hm[6 * k + 3 + a]);
      if (c->halos[k].n > 0 && (!(lo >= 0.0) || !(hi < c->cfg.box))) return SIDM_ERR_INVALID_ARG;
    }
  return SIDM_OK;
}

int sidm_set_particles(sidm_ctx* c, int64_t n, const double* pos, const double* vel,
                       const double* mass, double mass_scalar, const uint32_t* ids, int ptr_kind) {
  if (!c || n < 0 || n >= (int64_t)1 << 30 || (n > 0 && (!pos || !vel || !ids)) ||
      (ptr_kind != SIDM_HOST && ptr_kind != SIDM_DEVICE) || (!mass && !(mass_scalar > 0.0)))
    return SIDM_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  CK(join_velocities(c));
  int r = ensure_capacity(c, n);
  if (r != SIDM_OK) return r;
  const cudaMemcpyKind k = copy_kind_in(ptr_kind);
  if (n > 0) {
    CK(cudaMemcpyAsync(c->pos, pos, 3 * n * sizeof(double), k, c->stream));
    CK(cudaMemcpyAsync(c->vel, vel, 3 * n * sizeof(double), k, c->stream));
    CK(cudaMemcpyAsync(c->ids, ids, n * sizeof(uint32_t), k, c->stream));
    if (mass) CK(cudaMemcpyAsync(c->mass, mass, n * sizeof(double), k, c->stream));
    else fill(c->mass, n, mass_scalar, c->stream);
    fill(c->h_user, n, 0.0, c->stream);
    fill(c->dtlim, n, INFINITY, c->stream);
  }
  c->loaded = false;
  c->stepped = false;
  const int64_t off[2] = {0, n};
  r = layout_haloes(c, 1, off);
  if (r != SIDM_OK) return r;
  c->n = n;
  // periodic box: every coordinate in [0, box)
  if (c->cfg.box > 0.0 && n > 0) {
    r = check_in_box(c);
    if (r != SIDM_OK) {
      c->n = 0;
      return r;
    }
  }
  CK(cudaGetLastError());
  c->loaded = true;
  return SIDM_OK;
}

int sidm_set_haloes(sidm_ctx* c, int32_t n_halos, const int64_t* offsets) {
  if (!c || !c->loaded || n_halos < 1 || n_halos > (1 << 12) || !offsets) return SIDM_ERR_INVALID_ARG;
  if (offsets[0] != 0 || offsets[n_halos] != c->n) return SIDM_ERR_INVALID_ARG;
  for (int k = 0; k < n_halos; ++k)
    if (offsets[k + 1] < offsets[k]) return SIDM_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  CK(join_velocities(c));
  return layout_haloes(c, n_halos, offsets);
}

int sidm_set_positions(sidm_ctx* c, const double* pos, int ptr_kind) {
  if (!c || !c->loaded || !pos || (ptr_kind != SIDM_HOST && ptr_kind != SIDM_DEVICE))
    return SIDM_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  const int64_t n = c->n;
  if (n > 0)
    CK(cudaMemcpyAsync(c->pos, pos, 3 * n * sizeof(double), copy_kind_in(ptr_kind), c->stream));
  if (c->cfg.box > 0.0 && n > 0) return check_in_box(c);
  return SIDM_OK;
}

int sidm_set_velocities(sidm_ctx* c, const double* vel, int ptr_kind) {
  if (!c || !c->loaded || !vel || (ptr_kind != SIDM_HOST && ptr_kind != SIDM_DEVICE))
    return SIDM_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  if (c->n > 0) {
    // after the stream's earlier work on the velocities, beside its next work
    CK(cudaEventRecord(c->ev_vfree, c->stream));
    CK(cudaStreamWaitEvent(c->vstream, c->ev_vfree, 0));
    CK(cudaMemcpyAsync(c->vel, vel, 3 * c->n * sizeof(double), copy_kind_in(ptr_kind),
                       c->vstream));
    CK(cudaEventRecord(c->ev_vdone, c->vstream));
    c->vel_pending = true;
  }
  return SIDM_OK;
}

int sidm_write_particles(sidm_ctx* c, int64_t offset, int64_t count, const double* pos,
                         const double* vel, const double* mass, double mass_scalar,
                         const uint32_t* ids, int ptr_kind) {
  if (!c || !c->loaded || offset < 0 || count < 0 || offset > c->n ||
      offset + count > c->cap || (count > 0 && (!pos || !vel || !ids)) ||
      (ptr_kind != SIDM_HOST && ptr_kind != SIDM_DEVICE) || (!mass && !(mass_scalar > 0.0)))
    return SIDM_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  CK(join_velocities(c));
  if (count == 0) return SIDM_OK;
  const cudaMemcpyKind k = copy_kind_in(ptr_kind);
  cudaStream_t s = c->stream;
  CK(cudaMemcpyAsync(c->pos + 3 * offset, pos, 3 * count * sizeof(double), k, s));
  CK(cudaMemcpyAsync(c->vel + 3 * offset, vel, 3 * count * sizeof(double), k, s));
  CK(cudaMemcpyAsync(c->ids + offset, ids, count * sizeof(uint32_t), k, s));
  if (mass) CK(cudaMemcpyAsync(c->mass + offset, mass, count * sizeof(double), k, s));
  else fill(c->mass + offset, count, mass_scalar, s);
  fill(c->h_user + offset, count, 0.0, s);
  fill(c->dtlim + offset, count, INFINITY, s);
  c->stepped = false;
  if (offset + count > c->n) {
    // the loaded set grows: one halo over all particles until sidm_set_haloes
    const int64_t n = offset + count;
    const int64_t off[2] = {0, n};
    c->n = n;
    const int r = layout_haloes(c, 1, off);
    if (r != SIDM_OK) return r;
  }
  if (c->cfg.box > 0.0) {
    const int r = check_in_box(c);
    if (r != SIDM_OK) return r;
  }
  CK(cudaGetLastError());
  return SIDM_OK;
}

int sidm_set_count(sidm_ctx* c, int64_t n) {
  if (!c || !c->loaded || n < 0 || n > c->n) return SIDM_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  CK(join_velocities(c));
  if (n == c->n) return SIDM_OK;
  c->n = n;
  c->stepped = false;
  const int64_t off[2] = {0, n};
  return layout_haloes(c, 1, off);
}

}  // extern "C"

namespace {
// Copies `count` elements of `width` doubles (or words) from [from, ...) to
// [to, ...) within one device array; overlapping ranges are copied in
// chunks of |from - to| in the safe direction (stream-ordered).
template <class T>
cudaError_t move_range(T* base, int64_t width, int64_t from, int64_t to, int64_t count,
                       cudaStream_t s) {
  if (count <= 0 || from == to) return cudaSuccess;
  const int64_t d = from > to ? from - to : to - from;
  const int64_t step = d < count ? d : count;
  for (int64_t k = 0; k < count; k += step) {
    const int64_t len = std::min(step, count - k);
    const int64_t o = from > to ? k : count - k - len;   // front first when moving down
    const cudaError_t e = cudaMemcpyAsync(base + width * (to + o), base + width * (from + o),
                                          (size_t)(width * len) * sizeof(T),
                                          cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
}  // namespace

extern "C" {

int sidm_move_particles(sidm_ctx* c, int64_t from, int64_t to, int64_t count) {
  if (!c || !c->loaded || from < 0 || to < 0 || count < 0 || from + count > c->n ||
      to + count > c->n)
    return SIDM_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  CK(join_velocities(c));
  cudaStream_t s = c->stream;
  CK(move_range(c->pos, 3, from, to, count, s));
  CK(move_range(c->vel, 3, from, to, count, s));
  CK(move_range(c->mass, 1, from, to, count, s));
  CK(move_range(c->ids, 1, from, to, count, s));
  CK(move_range(c->h_user, 1, from, to, count, s));
  CK(move_range(c->dtlim, 1, from, to, count, s));
  if (count > 0 && from != to) c->stepped = false;
  return SIDM_OK;
}

int sidm_read_particles(sidm_ctx* c, int64_t offset, int64_t count, double* vel_out,
                        double* h_out, int ptr_kind) {
  if (!c || !c->loaded || offset < 0 || count < 0 || offset + count > c->n ||
      (count > 0 && !vel_out && !h_out) || (ptr_kind != SIDM_HOST && ptr_kind != SIDM_DEVICE))
    return SIDM_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  CK(join_velocities(c));
  const cudaMemcpyKind k = copy_kind_out(ptr_kind);
  if (count > 0) {
    if (vel_out)
      CK(cudaMemcpyAsync(vel_out, c->vel + 3 * offset, 3 * count * sizeof(double), k, c->stream));
    if (h_out)
      CK(cudaMemcpyAsync(h_out, c->h_user + offset, count * sizeof(double), k, c->stream));
  }
  return wait_and_collect(c);
}

int sidm_context_bytes(const sidm_config* cfg, int64_t n, int64_t* bytes) {
  if (!cfg || !bytes || n < 0 || n >= (int64_t)1 << 30 || cfg->n_ngb < 1 || cfg->ngb_tol < 0)
    return SIDM_ERR_INVALID_ARG;
  sidm_ctx d;
  d.cfg = *cfg;
  d.dry_run = true;
  d.nb_stride = cfg->n_ngb + cfg->ngb_tol;
  const int64_t want = std::max<int64_t>(n, 64);
  alloc_capacity(&d, want);
  // the box tree of one halo of n particles (float4 lower and upper corners)
  int64_t cnt[MAX_LEVELS] = {};
  const int levels = tree_levels_for(want, cnt);
  int64_t nodes = 0;
  for (int l = 0; l < levels; ++l) nodes += cnt[l];
  d.dry_bytes += 2 * (((std::max<int64_t>(nodes, 1) * (int64_t)sizeof(float4)) + 255) & ~255ll);
  *bytes = d.dry_bytes;
  return SIDM_OK;
}

int sidm_step(sidm_ctx* c, const uint8_t* active_mask, const int8_t* dt_bins, double dt_max,
              const sidm_sigma_model* sigma, uint64_t seed, sidm_step_stats* stats) {
  if (!c || !sigma) return SIDM_ERR_INVALID_ARG;
  if (!c->loaded) return SIDM_ERR_NOT_READY;
  if (!(dt_max > 0.0) || !std::isfinite(dt_max) || !valid_sigma(c, *sigma)) return SIDM_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  for (Halo& h : c->halos) set_step_params(h, dt_max, *sigma, seed, c->step);
  return run_step(c, active_mask, dt_bins, stats);
}

int sidm_step_haloes(sidm_ctx* c, const uint8_t* active_mask, const int8_t* dt_bins,
                     const sidm_halo_params* params, sidm_step_stats* stats) {
  if (!c || !params) return SIDM_ERR_INVALID_ARG;
  if (!c->loaded) return SIDM_ERR_NOT_READY;
  for (size_t k = 0; k < c->halos.size(); ++k) {
    const sidm_halo_params& p = params[k];
    if (!(p.dt_max > 0.0) || !std::isfinite(p.dt_max) || !valid_sigma(c, p.sigma))
      return SIDM_ERR_INVALID_ARG;
  }
  DeviceGuard g(c->device);
  for (size_t k = 0; k < c->halos.size(); ++k)
    set_step_params(c->halos[k], params[k].dt_max, params[k].sigma, params[k].seed,
                    params[k].step);
  return run_step(c, active_mask, dt_bins, stats);
}

namespace {

bool valid_tuning(const LaunchTuning& t) {
  return (t.search_window == 128 || t.search_window == 256 || t.search_window == 384 ||
          t.search_window == 512 || t.search_window == 768 || t.search_window == 1024) &&
         t.search_chunk >= 1 && t.search_chunk <= 64 && t.search_blocks_per_sm >= 1 &&
         t.search_blocks_per_sm <= 8 && t.pairs_chunk >= 1 && t.pairs_chunk <= 64 &&
         t.pairs_blocks_per_sm >= 1 && t.pairs_blocks_per_sm <= PAIRS_BLOCKS_MAX &&
         t.search_run >= 1 && t.search_run <= 16;
}

LaunchTuning from_public(const sidm_tuning& p) {
  LaunchTuning t;
  if (p.search_window) t.search_window = p.search_window;
  if (p.search_chunk) t.search_chunk = p.search_chunk;
  if (p.search_blocks_per_sm) t.search_blocks_per_sm = p.search_blocks_per_sm;
  if (p.pairs_chunk) t.pairs_chunk = p.pairs_chunk;
  if (p.pairs_blocks_per_sm) t.pairs_blocks_per_sm = p.pairs_blocks_per_sm;
  if (p.search_run) t.search_run = p.search_run;
  return t;
}

void to_public(const LaunchTuning& t, sidm_tuning* p) {
  p->search_window = t.search_window;
  p->search_chunk = t.search_chunk;
  p->search_blocks_per_sm = t.search_blocks_per_sm;
  p->pairs_chunk = t.pairs_chunk;
  p->pairs_blocks_per_sm = t.pairs_blocks_per_sm;
  p->search_run = t.search_run;
}

// Median time (ms) of `reps` steps, each from the saved state.
int time_candidate(sidm_ctx* c, const uint8_t* act, const int8_t* bins, int reps,
                   const double* v0, const double* h0, const double* d0, uint64_t step0,
                   float* ms) {
  const int64_t n = c->n;
  cudaEvent_t a = nullptr, b = nullptr;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  std::vector<float> t;
  int rc = SIDM_OK;
  for (int r = 0; r < reps && rc == SIDM_OK; ++r) {
    if (cudaMemcpyAsync(c->vel, v0, 3 * n * sizeof(double), cudaMemcpyDeviceToDevice,
                        c->stream) != cudaSuccess ||
        cudaMemcpyAsync(c->h_user, h0, n * sizeof(double), cudaMemcpyDeviceToDevice,
                        c->stream) != cudaSuccess ||
        cudaMemcpyAsync(c->dtlim, d0, n * sizeof(double), cudaMemcpyDeviceToDevice,
                        c->stream) != cudaSuccess) {
      rc = SIDM_ERR_CUDA;
      break;
    }
    c->step = step0;
    cudaEventRecord(a, c->stream);
    rc = run_step(c, act, bins, nullptr);
    cudaEventRecord(b, c->stream);
    if (rc != SIDM_OK) break;
    const int st = wait_and_collect(c);
    if (st < 0) rc = st;
    float x = 0.f;
    cudaEventElapsedTime(&x, a, b);
    t.push_back(x);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc != SIDM_OK) return rc;
  // the fastest repetition: interference only ever adds time
  *ms = *std::min_element(t.begin(), t.end());
  return SIDM_OK;
}

}  // namespace

namespace {

// ---- table of the kernel-overlap estimator (host) --------------------------
// ghat(a, s) = int_0^a 2 pi r^2 W(r, a) I(r) dr, where I(r) is the integral
// of W(., b), b = 1 - a, over the sphere of radius r around a point at
// distance s: with rho^2 = r^2 + s^2 - 2 r s mu it is
// (K / (b r s)) [F(min(r + s, b) / b) - F(min(|r - s|, b) / b)], F(t) the
// antiderivative of t f(t) of the kernel shape f (W = K f(r / h) / h^3).
// Between the kinks of f the integrand is a polynomial in r, so an 8-point
// Gauss-Legendre rule per piece is exact up to rounding.
double ov_shape(int kernel, double q) {
  if (!(q < 1.0)) return 0.0;
  if (kernel == SIDM_KERNEL_TOPHAT) return 1.0;
  if (q <= 0.5) return 1.0 - 6.0 * q * q + 6.0 * q * q * q;
  const double u = 1.0 - q;
  return 2.0 * u * u * u;
}
double ov_norm(int kernel) {
  return kernel == SIDM_KERNEL_TOPHAT ? 3.0 / (4.0 * M_PI) : 8.0 / M_PI;
}
double ov_F(int kernel, double t) {
  if (!(t > 0.0)) return 0.0;
  if (t > 1.0) t = 1.0;
  if (kernel == SIDM_KERNEL_TOPHAT) return 0.5 * t * t;
  if (t <= 0.5) return 0.5 * t * t - 1.5 * t * t * t * t + 1.2 * t * t * t * t * t;
  auto G = [](double x) {
    const double u = 1.0 - x;
    return -0.5 * u * u * u * u + 0.4 * u * u * u * u * u;
  };
  return 0.06875 + G(t) - G(0.5);  // 0.06875 = F(1/2)
}
double ov_ghat(int kernel, double a, double s) {
  const double b = 1.0 - a, K = ov_norm(kernel);
  if (!(s < 1.0)) return 0.0;
  if (a <= 0.0) return K * ov_shape(kernel, s);
  auto I = [&](double r) {
    if (s <= 0.0) return 2.0 * K * ov_shape(kernel, r / b) / (b * b * b);
    return K / (b * r * s) *
           (ov_F(kernel, std::min(r + s, b) / b) - ov_F(kernel, std::fabs(r - s) / b));
  };
  double cut[12];
  int nc = 0;
  cut[nc++] = 0.0;
  const double cand[9] = {0.5 * a, s, 0.5 * b - s, b - s, s - 0.5 * b, s - b, s + 0.5 * b, s + b,
                          a};
  for (double x : cand)
    if (x > 0.0 && x <= a) cut[nc++] = x;
  std::sort(cut, cut + nc);
  static const double gx[8] = {-0.9602898564975363, -0.7966664774136267, -0.5255324099163290,
                               -0.1834346424956498, 0.1834346424956498, 0.5255324099163290,
                               0.7966664774136267, 0.9602898564975363};
  static const double gw[8] = {0.1012285362903763, 0.2223810344533745, 0.3137066458778873,
                               0.3626837833783620, 0.3626837833783620, 0.3137066458778873,
                               0.2223810344533745, 0.1012285362903763};
  double total = 0.0;
  for (int k = 0; k + 1 < nc; ++k) {
    const double lo = cut[k], hi = cut[k + 1];
    if (!(hi > lo)) continue;
    for (int q = 0; q < 8; ++q) {
      const double r = 0.5 * (lo + hi) + 0.5 * (hi - lo) * gx[q];
      const double wa = K * ov_shape(kernel, r / a) / (a * a * a);
      total += 0.5 * (hi - lo) * gw[q] * 2.0 * M_PI * r * r * wa * I(r);
    }
  }
  return total;
}

}  // namespace

int sidm_overlap_table(int kernel, int32_t na, int32_t ns, double* out) {
  if (!out || na < 1 || na > 4096 || ns < 1 || ns > 65536 ||
      (kernel != SIDM_KERNEL_CUBIC && kernel != SIDM_KERNEL_TOPHAT))
    return SIDM_ERR_INVALID_ARG;
  for (int k = 0; k <= na; ++k)
    for (int l = 0; l <= ns; ++l)
      out[(int64_t)k * (ns + 1) + l] =
          ov_ghat(kernel, 0.5 * (double)k / (double)na, (double)l / (double)ns);
  return SIDM_OK;
}

int sidm_set_overlap_table(sidm_ctx* c, int32_t na, int32_t ns, const double* t) {
  if (!c || !t || na < 1 || na > 4096 || ns < 1 || ns > 65536) return SIDM_ERR_INVALID_ARG;
  const int64_t m = (int64_t)(na + 1) * (ns + 1);
  for (int64_t k = 0; k < m; ++k)
    if (!std::isfinite(t[k]) || !(t[k] >= 0.0)) return SIDM_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  std::vector<char> host(m * (sizeof(double) + sizeof(float)));
  double* hg = (double*)host.data();
  float* hf = (float*)(hg + m);
  for (int64_t k = 0; k < m; ++k) {
    hg[k] = t[k];
    float y = (float)t[k];
    if ((double)y < t[k]) y = std::nextafter(y, INFINITY);
    hf[k] = y;
  }
  CK(cudaStreamSynchronize(c->stream));
  if (c->ov_mem) raw_free(c, c->ov_mem);
  c->ov_mem = nullptr;
  c->ov = OverlapTable{};
  void* d = nullptr;
  CK(raw_alloc(c, &d, host.size()));
  c->ov_mem = d;
  CK(cudaMemcpy(d, host.data(), host.size(), cudaMemcpyHostToDevice));
  c->ov.na = na;
  c->ov.ns = ns;
  c->ov.g = (const double*)d;
  c->ov.g_ru = (const float*)((const double*)d + m);
  ++c->layout_version;  // the captured step holds the old table address
  return SIDM_OK;
}

int sidm_set_sigma_table(sidm_ctx* c, int32_t n, const double* v, const double* sg) {
  if (!c || !v || !sg || n < 2 || n > SIDM_SIGMA_TABLE_MAX) return SIDM_ERR_INVALID_ARG;
  for (int k = 0; k < n; ++k) {
    if (!std::isfinite(v[k]) || !(v[k] > 0.0) || !std::isfinite(sg[k]) || !(sg[k] >= 0.0))
      return SIDM_ERR_INVALID_ARG;
    // nodes must stay distinct after rounding to FP32 (the bounds of the FP32
    // pass compare them there)
    if (k > 0 && !(v[k] > v[k - 1] * (1.0 + 0x1p-20))) return SIDM_ERR_INVALID_ARG;
  }
  DeviceGuard g(c->device);
  // layout: v, s, ln v (FP64), then v rounded down / up, s down / up (FP32)
  std::vector<char> host(n * (3 * sizeof(double) + 4 * sizeof(float)));
  double* hv = (double*)host.data();
  double* hs = hv + n;
  double* hl = hs + n;
  float* f = (float*)(hl + n);
  auto rd = [](double x) {
    float y = (float)x;
    if ((double)y > x) y = std::nextafter(y, -INFINITY);
    return y;
  };
  auto ru = [](double x) {
    float y = (float)x;
    if ((double)y < x) y = std::nextafter(y, INFINITY);
    return y;
  };
  for (int k = 0; k < n; ++k) {
    hv[k] = v[k];
    hs[k] = sg[k];
    hl[k] = std::log(v[k]);
    f[k] = rd(v[k]);
    f[n + k] = ru(v[k]);
    f[2 * n + k] = rd(sg[k]);
    f[3 * n + k] = ru(sg[k]);
  }
  CK(cudaStreamSynchronize(c->stream));
  if (c->table_mem) raw_free(c, c->table_mem);
  c->table_mem = nullptr;
  c->table = SigmaTable{};
  void* d = nullptr;
  CK(raw_alloc(c, &d, host.size()));
  c->table_mem = d;
  CK(cudaMemcpy(d, host.data(), host.size(), cudaMemcpyHostToDevice));
  SigmaTable& T = c->table;
  T.n = n;
  T.v = (const double*)d;
  T.s = T.v + n;
  T.lnv = T.s + n;
  T.v_rd = (const float*)(T.lnv + n);
  T.v_ru = T.v_rd + n;
  T.s_rd = T.v_ru + n;
  T.s_ru = T.s_rd + n;
  ++c->layout_version;  // the captured step holds the old table address
  return SIDM_OK;
}

int sidm_set_tuning(sidm_ctx* c, const sidm_tuning* p) {
  if (!c || !p) return SIDM_ERR_INVALID_ARG;
  const LaunchTuning t = from_public(*p);
  if (!valid_tuning(t)) return SIDM_ERR_INVALID_ARG;
  c->tune = t;
  ++c->layout_version;
  return SIDM_OK;
}

int sidm_get_tuning(const sidm_ctx* c, sidm_tuning* p) {
  if (!c || !p) return SIDM_ERR_INVALID_ARG;
  to_public(c->tune, p);
  return SIDM_OK;
}

int sidm_graph_state(const sidm_ctx* c) {
  if (!c) return SIDM_ERR_INVALID_ARG;
  if (!c->cfg.use_graph) return 0;
  return c->graph_state;
}

int sidm_autotune(sidm_ctx* c, const uint8_t* active_mask, const int8_t* dt_bins,
                  const sidm_halo_params* params, int reps, sidm_tuning* best) {
  if (!c || !params || reps < 1 || reps > 16) return SIDM_ERR_INVALID_ARG;
  if (!c->loaded) return SIDM_ERR_NOT_READY;
  for (size_t k = 0; k < c->halos.size(); ++k)
    if (!(params[k].dt_max > 0.0) || !std::isfinite(params[k].dt_max) ||
        !valid_sigma(c, params[k].sigma))
      return SIDM_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  CK(join_velocities(c));
  const int64_t n = c->n;
  if (n <= 0) {
    if (best) to_public(c->tune, best);
    return SIDM_OK;
  }
  for (size_t k = 0; k < c->halos.size(); ++k)
    set_step_params(c->halos[k], params[k].dt_max, params[k].sigma, params[k].seed,
                    params[k].step);
  // the state the candidates start from, and restore at the end
  double* save = nullptr;
  CK(raw_alloc(c, (void**)&save, 5 * n * sizeof(double)));
  double *v0 = save, *h0 = save + 3 * n, *d0 = save + 4 * n;
  const uint64_t step0 = c->step;
  const int64_t since0 = c->since_rebuild;
  const uint64_t order0 = c->order_version;
  const int use_graph = c->cfg.use_graph, rebuild_every = c->cfg.rebuild_every;
  double* const mirror = c->mirror;
  c->cfg.use_graph = 0;      // candidates launch directly
  c->cfg.rebuild_every = 0;  // and rebuild fully, like the steps they stand for
  c->mirror = nullptr;       // and leave the host copy of the velocities alone
  int rc = SIDM_OK;
  if (cudaMemcpyAsync(v0, c->vel, 3 * n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(h0, c->h_user, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(d0, c->dtlim, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream) !=
          cudaSuccess)
    rc = SIDM_ERR_CUDA;
  LaunchTuning cur = c->tune;
  float cur_ms = 0.f;
  if (rc == SIDM_OK) rc = time_candidate(c, active_mask, dt_bins, reps, v0, h0, d0, step0, &cur_ms);
  // coordinate search over the launch shapes
  const int windows[] = {128, 256, 384, 512, 768, 1024};
  const int chunks[] = {1, 2, 4, 8, 16};
  const int sranges[] = {1, 2};   // ranges of 32 and 64 runs per search block
  const int sruns[] = {1, 2, 4};
  const int pblocks[] = {4, 6, 7};
  auto try_field = [&](int LaunchTuning::*field, const int* vals, int nv) {
    for (int k = 0; k < nv && rc == SIDM_OK; ++k) {
      if (cur.*field == vals[k]) continue;
      LaunchTuning t = cur;
      t.*field = vals[k];
      c->tune = t;
      float ms = 0.f;
      rc = time_candidate(c, active_mask, dt_bins, reps, v0, h0, d0, step0, &ms);
      // a new shape must win clearly: step times jitter by ~1 %
      if (rc == SIDM_OK && ms < 0.98f * cur_ms) {
        cur = t;
        cur_ms = ms;
      }
    }
  };
  try_field(&LaunchTuning::search_window, windows, (int)(sizeof(windows) / sizeof(windows[0])));
  try_field(&LaunchTuning::search_run, sruns, 3);
  try_field(&LaunchTuning::search_chunk, sranges, 2);
  try_field(&LaunchTuning::pairs_chunk, chunks, 5);
  try_field(&LaunchTuning::pairs_blocks_per_sm, pblocks, 3);
  // leave the simulation where it was
  c->tune = cur;
  ++c->layout_version;
  c->cfg.use_graph = use_graph;
  c->cfg.rebuild_every = rebuild_every;
  c->mirror = mirror;
  cudaMemcpyAsync(c->vel, v0, 3 * n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
  cudaMemcpyAsync(c->h_user, h0, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
  cudaMemcpyAsync(c->dtlim, d0, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
  c->step = step0;
  c->since_rebuild = since0;
  c->order_version = order0;
  c->stepped = false;   // the pair buffer holds a trial step's pairs
  const int st = wait_and_collect(c);
  raw_free(c, save);
  if (rc != SIDM_OK) return rc;
  if (st < 0) return st;
  if (best) to_public(cur, best);
  return SIDM_OK;
}

int sidm_sync(sidm_ctx* c) {
  if (!c) return SIDM_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  CK(join_velocities(c));
  return wait_and_collect(c);
}

int sidm_get_particles(sidm_ctx* c, double* vel_out, double* h_out, int ptr_kind) {
  if (!c || !c->loaded || (!vel_out && !h_out) || (ptr_kind != SIDM_HOST && ptr_kind != SIDM_DEVICE))
    return SIDM_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  CK(join_velocities(c));
  const cudaMemcpyKind k = copy_kind_out(ptr_kind);
  if (c->n > 0) {
    if (vel_out) CK(cudaMemcpyAsync(vel_out, c->vel, 3 * c->n * sizeof(double), k, c->stream));
    if (h_out) CK(cudaMemcpyAsync(h_out, c->h_user, c->n * sizeof(double), k, c->stream));
  }
  return wait_and_collect(c);
}

int sidm_get_changed(sidm_ctx* c, int32_t* idx_out, double* vel_out, int64_t cap,
                     int64_t* n_out, int ptr_kind) {
  if (!c || !n_out || cap < 0 || (cap > 0 && (!idx_out || !vel_out)) ||
      (ptr_kind != SIDM_HOST && ptr_kind != SIDM_DEVICE))
    return SIDM_ERR_INVALID_ARG;
  *n_out = 0;
  if (!c->loaded || c->n <= 0 || !c->stepped) return SIDM_OK;
  DeviceGuard g(c->device);
  CK(join_velocities(c));
  cudaStream_t s = c->stream;
  if (++c->chg_call == 0) c->chg_call = 1;   // stamps start at 0
  CK(cudaMemsetAsync(c->chg_count, 0, sizeof(unsigned long long), s));
  c->launches += launch_changed(c->pairs, c->pair_cap, c->dstats, c->chg_call, c->chg_stamps,
                                c->vel, c->chg_idx, c->chg_vel, c->chg_count, c->sms, s);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(c->h_chg_count, c->chg_count, sizeof(unsigned long long),
                     cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const int64_t cnt = (int64_t)*c->h_chg_count;
  const int64_t m = std::min(cnt, cap);
  if (m > 0) {
    const cudaMemcpyKind k = copy_kind_out(ptr_kind);
    CK(cudaMemcpyAsync(idx_out, c->chg_idx, m * sizeof(int32_t), k, s));
    CK(cudaMemcpyAsync(vel_out, c->chg_vel, 3 * m * sizeof(double), k, s));
  }
  *n_out = cnt;
  return wait_and_collect(c);
}

int sidm_set_velocity_mirror(sidm_ctx* c, double* host_vel, int64_t n) {
  if (!c || (host_vel && n < 0)) return SIDM_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  double* dev = nullptr;
  if (host_vel) {
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, host_vel) != cudaSuccess || pa.type != cudaMemoryTypeHost ||
        !pa.devicePointer || (reinterpret_cast<uintptr_t>(pa.devicePointer) & 7) != 0) {
      cudaGetLastError();
      return SIDM_ERR_INVALID_ARG;
    }
    dev = static_cast<double*>(pa.devicePointer);
  }
  CK(cudaStreamSynchronize(c->stream));   // no earlier step still writes the old copy
  c->mirror = dev;
  c->mirror_n = host_vel ? n : 0;
  ++c->layout_version;                     // a captured step holds the old address
  return SIDM_OK;
}

int sidm_update_velocities(sidm_ctx* c, double* vel_inout) {
  if (!c || !vel_inout) return SIDM_ERR_INVALID_ARG;
  if (!c->loaded || c->n <= 0 || !c->stepped) return SIDM_OK;
  DeviceGuard g(c->device);
  const int64_t n = c->n;
  // pinned host memory that the device addresses: the changed particles are
  // written into it from the device, with no staging and no host loop
  cudaPointerAttributes pa{};
  if (cudaPointerGetAttributes(&pa, vel_inout) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
      pa.devicePointer && (reinterpret_cast<uintptr_t>(pa.devicePointer) & 7) == 0) {
    CK(join_velocities(c));
    if (++c->chg_call == 0) c->chg_call = 1;   // stamps start at 0
    c->launches += launch_changed_to_host(c->pairs, c->pair_cap, c->dstats, c->chg_call,
                                          c->chg_stamps, c->vel,
                                          static_cast<double*>(pa.devicePointer), c->sms,
                                          c->stream);
    CK(cudaGetLastError());
    return wait_and_collect(c);
  }
  cudaGetLastError();   // a pointer the runtime does not know is not an error here
  if (c->h_chg_cap < n) {
    if (c->h_chg_idx) cudaFreeHost(c->h_chg_idx);
    if (c->h_chg_vel) cudaFreeHost(c->h_chg_vel);
    c->h_chg_idx = nullptr;
    c->h_chg_vel = nullptr;
    c->h_chg_cap = 0;
    CK(cudaMallocHost(&c->h_chg_idx, n * sizeof(int32_t)));
    CK(cudaMallocHost(&c->h_chg_vel, 3 * n * sizeof(double)));
    c->h_chg_cap = n;
  }
  int64_t cnt = 0;
  const int r = sidm_get_changed(c, c->h_chg_idx, c->h_chg_vel, n, &cnt, SIDM_HOST);
  if (r < 0) return r;
  for (int64_t k = 0; k < cnt; ++k) {
    double* d = vel_inout + 3 * (int64_t)c->h_chg_idx[k];
    const double* v = c->h_chg_vel + 3 * k;
    d[0] = v[0];
    d[1] = v[1];
    d[2] = v[2];
  }
  return r;
}

int sidm_timestep_limits(sidm_ctx* c, double* out, int ptr_kind) {
  if (!c || !c->loaded || !out || (ptr_kind != SIDM_HOST && ptr_kind != SIDM_DEVICE))
    return SIDM_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  if (c->n > 0)
    CK(cudaMemcpyAsync(out, c->dtlim, c->n * sizeof(double), copy_kind_out(ptr_kind), c->stream));
  return wait_and_collect(c);
}

int sidm_get_pairs(sidm_ctx* c, uint32_t* ab, uint64_t* ord, int64_t cap, int64_t* n_out) {
  if (!c || !c->loaded || cap < 0 || (cap > 0 && (!ab || !ord))) return SIDM_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  CK(cudaMemcpyAsync(c->h_stats, c->dstats, sizeof(DevStats), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  const int64_t total = (int64_t)c->h_stats->n_acc;
  const int64_t stored = std::min<int64_t>(total, c->pair_cap);
  std::vector<PairRec> h(stored);
  if (stored > 0)
    CK(cudaMemcpy(h.data(), c->pairs, stored * sizeof(PairRec), cudaMemcpyDeviceToHost));
  std::sort(h.begin(), h.end(), [](const PairRec& x, const PairRec& y) {
    if (x.ord != y.ord) return x.ord < y.ord;
    if (x.a != y.a) return x.a < y.a;
    return x.b < y.b;
  });
  for (int64_t k = 0; k < stored && k < cap; ++k) {
    ab[2 * k] = h[k].a;
    ab[2 * k + 1] = h[k].b;
    ord[k] = h[k].ord;
  }
  if (n_out) *n_out = total;
  return total > c->pair_cap ? SIDM_ERR_DEVICE_LIMIT : wait_and_collect(c);
}

int sidm_get_step(const sidm_ctx* c, uint64_t* step) {
  if (!c || !step) return SIDM_ERR_INVALID_ARG;
  *step = c->step;
  return SIDM_OK;
}

int sidm_set_step(sidm_ctx* c, uint64_t step) {
  if (!c) return SIDM_ERR_INVALID_ARG;
  c->step = step;
  return SIDM_OK;
}

const char* sidm_error_string(int status) {
  switch (status) {
    case SIDM_OK: return "ok";
    case SIDM_WARN_H_NOT_CONVERGED: return "warning: h bisection hit its evaluation cap";
    case SIDM_WARN_P_GE_1: return "warning: a pair probability reached 1 (timestep above the Eq. 18 limit)";
    case SIDM_WARN_DIRECTION: return "warning: a direction draw exhausted its tries";
    case SIDM_ERR_INVALID_ARG: return "invalid argument";
    case SIDM_ERR_OOM: return "out of device memory";
    case SIDM_ERR_CUDA: return "CUDA error";
    case SIDM_ERR_DEVICE_LIMIT: return "a bounded device loop or buffer gave up (search capacity, traversal stack, pair buffer or resolver rounds); the step is not valid";
    case SIDM_ERR_NOT_READY: return "no particles loaded";
    case SIDM_ERR_TOO_LARGE:
      return "input exceeds the fixed scratch of the no-allocation entry point "
             "(at most SIDM_NOALLOC_MAX_PARTICLES particles and SIDM_NOALLOC_MAX_PAIRS pairs)";
    default:
      if (status > 0) return "several warnings";
      return "unknown status";
  }
}

void sidm_destroy(sidm_ctx* c) {
  if (!c) return;
  {
    DeviceGuard g(c->device);
    if (c->vstream) cudaStreamSynchronize(c->vstream);
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_buffers(c);
    if (c->h_stats) cudaFreeHost(c->h_stats);
    if (c->h_cons) cudaFreeHost(c->h_cons);
    if (c->h_latched) cudaFreeHost(c->h_latched);
    if (c->h_chg_count) cudaFreeHost(c->h_chg_count);
    if (c->h_chg_idx) cudaFreeHost(c->h_chg_idx);
    if (c->h_chg_vel) cudaFreeHost(c->h_chg_vel);
    if (c->table_mem) raw_free(c, c->table_mem);
    if (c->ov_mem) raw_free(c, c->ov_mem);
    for (int k = 0; k <= SIDM_N_PHASES; ++k)
      if (c->ev[k]) cudaEventDestroy(c->ev[k]);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    if (c->vstream) cudaStreamDestroy(c->vstream);
    if (c->ev_vfree) cudaEventDestroy(c->ev_vfree);
    if (c->ev_vdone) cudaEventDestroy(c->ev_vdone);
  }
  delete c;
}

}  // extern "C"
