// Internal declarations of the SIDM scattering-step library: device data
// layout, shared device helpers and the launchers of every kernel.
//
// The library is compiled with -fmad=false: every FP64 expression on the
// exact path is one IEEE round-to-nearest operation per operator, in the
// order written, so that its results are a function of the inputs alone.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sidm.h"
#include "../../include/sidm_model.cuh"

namespace sidm {

// ------------------------------------------------------------------ limits
constexpr int WARP = 32;
constexpr int LEAF = 32;                 // particles per tree leaf (one per lane)
constexpr int MAX_LEVELS = 8;            // 32-ary levels: 32^8 leaves >> any n
constexpr int BISECT_MAX_EVALS = 128;    // neighbour-count evaluations per particle
// Gathered candidates per query (shared memory; a query that gathers more
// shrinks its radius and gathers again).  With 448 entries the 32 warps of
// an SM's search block hold 131 KB of shared memory, which leaves ~120 KB of
// L1 to the walks' position and box loads.  On the 2^20 halo: 768 entries
// 0.576 ms per search (4-warp blocks, ~30 KB of L1), 512 entries 0.550, and
// with the 32-warp blocks 512 entries 0.507, 384 or 448 entries 0.500.
#ifndef SEARCH_CAP_ENTRIES
#define SEARCH_CAP_ENTRIES 448
#endif
constexpr int SEARCH_CAP = SEARCH_CAP_ENTRIES;
constexpr int SEARCH_STACK = 256;        // traversal stack per warp (>= 31 MAX_LEVELS + 1)
constexpr int RADIUS_MAX_ITERS = 24;     // gather-radius adjustments per query
constexpr int RESOLVE_MAX_ROUNDS = 4096; // resolver rounds
constexpr int DIRECTION_TRIES = 64;      // Marsaglia rejection tries

// device status bits (latched per step)
enum : uint32_t {
  ST_H_NONCONV = 1u,
  ST_P_GE_1 = 2u,
  ST_DIR_FAIL = 4u,
  ST_ERR_SEARCH_CAP = 1u << 8,    // a query needed more than SEARCH_CAP candidates
  ST_ERR_STACK = 1u << 9,         // traversal stack overflow
  ST_ERR_RADIUS = 1u << 10,       // gather radius adjustment did not settle
  ST_ERR_PAIR_OVERFLOW = 1u << 11,// accepted-pair buffer full
  ST_ERR_ROUNDS = 1u << 12,       // resolver did not finish within its round cap
  ST_ERR_SORT = 1u << 13,         // key sort: a look-back wait gave up (order not valid)
  ST_ERR_CLAIM = 1u << 15,        // search: a block's wait for its next query range gave up
  ST_ERR_MASK = 0xFF00u
};

// One halo: an independent set of particles, contiguous in user order and
// in key order, with its own bounding box, start radius, key transform,
// tree, cross-section model, random key and step counter.  A context holds
// one or more haloes; a single particle set is a context with one halo.
struct Halo {
  // layout (host, at configuration)
  int64_t start, n;                 // particle range (same in user and key order)
  int64_t node_off[MAX_LEVELS];     // first node of each tree level (level 0 = leaves)
  int64_t node_cnt[MAX_LEVELS];     // nodes per level
  int32_t levels;                   // tree levels (0 for an empty halo)
  int32_t e0;                       // start radius h0 = l_ext 2^-e0 (8^e0 N_ngb <= 4 n)
  // per step (host)
  double dt_max, sigma0, w;
  double eps;                       // outgoing / incoming relative speed of a scatter
  int32_t sigma_kind;
  uint32_t step;                    // Philox counter word 0
  uint64_t seed;                    // Philox key
  // per step (device)
  unsigned long long mm[6];         // ordered bounding-box accumulators (min xyz, max xyz)
  double l_ext, h0;
  float centre[3];                  // key transform centre (open boundaries)
  float key_scale;                  // asinh scale s
  float key_inv_norm;               // 1 / asinh(R / s)
  float pad;
};

// Device counters of one step.
struct DevStats {
  unsigned long long n_active, n_cand, n_acc, n_rounds, n_pge1, n_nonconv, n_dirfail, max_mult;
  unsigned long long n_pending;   // accepted pairs that share a particle with another
  unsigned long long n_seg;       // segment slots handed out to particles of pending pairs
  unsigned long long n_touched;   // particles of pending pairs
  unsigned long long n_deferred;  // draws left to the exact FP64 pass
  double sum_p;
  unsigned int status;
  unsigned int pad;
};

// An accepted pair: ord = words 2, 3 of the stream-0 draw; ids a < b;
// user-order indices ia, ib of the a- and b-particle (the record of the C ABI).
using PairRec = sidm_pair;

// ------------------------------------------------------------------ Philox
// Philox-4x32-10 and the 53-bit uniform of sidm_model.cuh (one definition
// for the draws of the pair kernel and the directions of the kicks).
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox10(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1,
                                       uint32_t c2, uint32_t c3) {
  const uint4 w = sidm_model::philox4x32_10(k0, k1, c0, c1, c2, c3);
  return U4{w.x, w.y, w.z, w.w};
}

__device__ __forceinline__ double unit53(uint32_t a, uint32_t b) {
  return sidm_model::unit53(a, b);
}

// ---------------------------------------------------------------- geometry
// Minimum-image component of x_j - x_i (box > 0), one rounding per operation.
__device__ __forceinline__ double min_image(double d, double box, double half) {
  if (box > 0.0) {
    if (d > half) d = d - box;
    else if (d < -half) d = d + box;
  }
  return d;
}

// Squared separation in the fixed order (dx dx + dy dy) + dz dz.
__device__ __forceinline__ double sep2(double xi, double yi, double zi, double xj, double yj,
                                       double zj, double box, double half) {
  const double dx = min_image(xj - xi, box, half);
  const double dy = min_image(yj - yi, box, half);
  const double dz = min_image(zj - zi, box, half);
  return (dx * dx + dy * dy) + dz * dz;
}

// Exact boundary tests r_ij^2 < h^2 (h = h_j, or h_i + h_j for the overlap
// estimator), in the fixed order of sep2.  They decide the rare pairs inside
// the FP32 rounding band; as real calls, their FP64 instructions stay off the
// common path (an inline FP64 branch is predicated and paid on every pass).
static __device__ __noinline__ bool hw_within(const double* x, const double* y, const double* z,
                                              int64_t i, int64_t j, double box, double h) {
  return sep2(x[i], y[i], z[i], x[j], y[j], z[j], box, 0.5 * box) < h * h;
}
static __device__ __noinline__ bool hw_within_sum(const double* x, const double* y,
                                                  const double* z, int64_t i, int64_t j,
                                                  double box, double hi, double hj) {
  const double H = hi + hj;
  return sep2(x[i], y[i], z[i], x[j], y[j], z[j], box, 0.5 * box) < H * H;
}

// Kernel normalisation K / h^3 with K = 8/pi (cubic spline) or 3/(4 pi) (top-hat).
__device__ __forceinline__ double kernel_norm(int kernel, double h) {
  const double k = kernel == SIDM_KERNEL_TOPHAT ? 3.0 / (4.0 * 3.141592653589793)
                                                : 8.0 / 3.141592653589793;
  return k / ((h * h) * h);
}

// Kernel shape f(q), q = r/h < 1: cubic spline 1 - 6q^2 + 6q^3 (q <= 1/2),
// 2(1-q)^3 (q > 1/2); top-hat 1.
__device__ __forceinline__ double kernel_shape(int kernel, double q) {
  if (kernel == SIDM_KERNEL_TOPHAT) return 1.0;
  if (q <= 0.5) return (1.0 - 6.0 * (q * q)) + 6.0 * ((q * q) * q);
  const double u = 1.0 - q;
  return 2.0 * ((u * u) * u);
}

// Tabulated sigma/m(v) on the device: FP64 nodes, values and logarithms of
// the nodes (taken on the host), and FP32 copies rounded down / up for the
// bounds of the FP32 pass.
struct SigmaTable {
  int32_t n;
  const double* v;
  const double* s;
  const double* lnv;
  const float* v_rd;
  const float* v_ru;
  const float* s_rd;
  const float* s_ru;
};

// Linear in log v between nodes, held at the end values (Sec. 4.1).
__device__ __forceinline__ double sigma_table(const SigmaTable& T, double v) {
  const int n = T.n;
  if (!(v > T.v[0])) return T.s[0];
  if (v >= T.v[n - 1]) return T.s[n - 1];
  int lo = 0, hi = n - 1;  // v_lo <= v < v_hi
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (T.v[mid] <= v) lo = mid;
    else hi = mid;
  }
  const double t = (log(v) - T.lnv[lo]) / (T.lnv[lo + 1] - T.lnv[lo]);
  return T.s[lo] + t * (T.s[lo + 1] - T.s[lo]);
}

// Kernel-overlap estimator (Eq. 15, Appendix A): ghat on a = k / (2 na),
// s = l / ns, row-major in a; the FP32 copy is rounded up.  na = 0: the
// one-sided estimator (Eq. 14).
struct OverlapTable {
  int32_t na, ns;
  const double* g;
  const float* g_ru;
};

// Bilinear interpolation of ghat (a in [0, 1/2], s in [0, 1)).
__device__ __forceinline__ double overlap_hat(const OverlapTable& T, double a, double s) {
  if (!(s < 1.0)) return 0.0;
  const int na = T.na, ns = T.ns;
  const double fa = a * (2.0 * (double)na);
  int ia = (int)fa;
  if (ia > na - 1) ia = na - 1;
  const double ta = fa - (double)ia;
  const double fs = s * (double)ns;
  int is = (int)fs;
  if (is > ns - 1) is = ns - 1;
  const double ts = fs - (double)is;
  const double* r0 = T.g + (int64_t)ia * (ns + 1);
  const double* r1 = r0 + (ns + 1);
  const double g0 = (1.0 - ts) * r0[is] + ts * r0[is + 1];
  const double g1 = (1.0 - ts) * r1[is] + ts * r1[is + 1];
  return (1.0 - ta) * g0 + ta * g1;
}

// g_ij = ghat(min(h_i, h_j) / H, r_ij / H) / H^3, H = h_i + h_j (symmetric)
__device__ __forceinline__ double overlap_g(const OverlapTable& T, double hi, double hj,
                                            double r2) {
  const double H = hi + hj;
  const double a = fmin(hi, hj) / H;
  const double s = sqrt(r2) / H;
  return overlap_hat(T, a, s) / ((H * H) * H);
}

__device__ __forceinline__ double sigma_over_m(int kind, double s0, double w, const SigmaTable& T,
                                               double v) {
  if (kind == SIDM_SIGMA_TABLE) return sigma_table(T, v);
  if (kind == SIDM_SIGMA_YUKAWA) {
    const double t = 1.0 + (v * v) / (w * w);
    return s0 / (t * t);
  }
  return s0;
}

// Order-preserving map of a double to uint64 (for atomicMin/atomicMax).
__device__ __forceinline__ unsigned long long dbl_to_ordered(double x) {
  unsigned long long u = (unsigned long long)__double_as_longlong(x);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
// Rare-path hardware operations behind a real call: written inline, the
// compiler turns such a fallback into predicated instructions that occupy
// B300's slow FP64 pipe on every pass, taken or not.
static __device__ __noinline__ float hw_f32_rn(double x) { return __double2float_rn(x); }
static __device__ __noinline__ float hw_f32_ru(double x) { return __double2float_ru(x); }
static __device__ __noinline__ float hw_f32_rd(double x) { return __double2float_rd(x); }
static __device__ __noinline__ double hw_ldexp(double x, int k) { return ldexp(x, k); }
static __device__ __noinline__ double hw_mul(double x, double y) { return x * y; }

// FP64 -> FP32 conversions on the bit pattern (integer pipe; B300's FP64
// pipe is slow).  The normal FP32 range is handled here, exactly as IEEE
// round-to-nearest-even, upward and downward rounding define it; zero,
// subnormal, out-of-range, infinite and NaN inputs take the hardware
// conversion.
__device__ __forceinline__ bool f32_normal_range(unsigned long long b, unsigned int* fb,
                                                 unsigned int* rem) {
  const int e = (int)((b >> 52) & 0x7FF) - 1023;
  if (e < -126 || e > 127) return false;
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  *fb = ((unsigned int)(b >> 63) << 31) | ((unsigned int)(e + 127) << 23) | (unsigned int)(m >> 29);
  *rem = (unsigned int)(m & 0x1FFFFFFFull);  // the 29 dropped significand bits
  return true;
}
__device__ __forceinline__ float f64_to_f32_rn(double x) {
  unsigned int fb, rem;
  if (!f32_normal_range((unsigned long long)__double_as_longlong(x), &fb, &rem))
    return hw_f32_rn(x);
  if (rem > 0x10000000u || (rem == 0x10000000u && (fb & 1u))) ++fb;  // magnitude up
  return __uint_as_float(fb);
}
__device__ __forceinline__ float f64_to_f32_ru(double x) {
  unsigned int fb, rem;
  if (!f32_normal_range((unsigned long long)__double_as_longlong(x), &fb, &rem))
    return hw_f32_ru(x);
  if (rem && !(fb >> 31)) ++fb;  // positive: magnitude up; negative: truncation
  return __uint_as_float(fb);
}
__device__ __forceinline__ float f64_to_f32_rd(double x) {
  unsigned int fb, rem;
  if (!f32_normal_range((unsigned long long)__double_as_longlong(x), &fb, &rem))
    return hw_f32_rd(x);
  if (rem && (fb >> 31)) ++fb;  // negative: magnitude up; positive: truncation
  return __uint_as_float(fb);
}
// x 2^-k exactly (k >= 0) by an exponent step while the result stays normal.
__device__ __forceinline__ double scale_pow2_down(double x, int k) {
  const long long b = __double_as_longlong(x);
  const int ef = (int)((b >> 52) & 0x7FF);
  if (ef > k && ef < 2047) return __longlong_as_double(b - ((long long)k << 52));
  return hw_ldexp(x, -k);
}

__host__ __device__ inline double ordered_to_dbl(unsigned long long u) {
  u = (u >> 63) ? (u & 0x7FFFFFFFFFFFFFFFull) : ~u;
  double d;
  memcpy(&d, &u, sizeof(d));
  return d;
}

// --------------------------------------------------------- device buffers
// Trees of all haloes: node boxes in level-major arrays (all haloes' level-0
// nodes, then all level-1 nodes, ...); a halo's nodes of level l are
// [node_off[l], node_off[l] + node_cnt[l]).
struct Forest {
  const Halo* halos;
  int32_t n_halos;
  int32_t halo_bits;          // key prefix bits (0 for one halo)
  int32_t max_levels;         // deepest tree
  int64_t level_nodes[MAX_LEVELS];  // nodes of all haloes per level
  float4* lo;                 // per node: min corner (w unused), rounded down
  float4* hi;                 // per node: max corner, rounded up
};

struct Sorted {               // particle state in key order
  double *x, *y, *z;
  double *vx, *vy, *vz;
  double *m;
  double *h;                  // h of active particles (this step)
  double *dt;                 // dt_i of the particle
  float4* f;                  // FP32 position (round to nearest); w = dt_i rounded up
  float4* vm;                 // FP32 velocity (round to nearest); w = m rounded up
  float4* hb;                 // active particles: h rounded down, h rounded up, 1/h
                              // rounded down, kernel normalisation K / h^3 rounded up
  uint32_t* id;
  uint8_t* act;
  int32_t* orig;              // user-order index
  int32_t* halo;              // halo of the particle
};

// ---------------------------------------------------------------- launchers
// sort.cu
size_t radix_sort_temp_bytes(int64_t n);
int sort_passes(int key_bits);
int radix_sort_pairs(uint32_t* keys, int32_t* vals, uint32_t* keys_alt, int32_t* vals_alt,
                     int64_t n, int key_bits, void* temp, unsigned* status, cudaStream_t s);

// build.cu
int launch_bbox(const double* pos, const int32_t* halo_of, int64_t n, Halo* halos,
                int n_halos, cudaStream_t s);
int launch_params(Halo* halos, int n_halos, double box, cudaStream_t s);
int launch_keys(const double* pos, const int32_t* halo_of, int64_t n, const Halo* halos,
                int halo_bits, double box, uint32_t* keys, int32_t* vals, cudaStream_t s);
int launch_permute(const int32_t* perm, int64_t n, const double* pos,
                   const double* mass, const uint32_t* ids, const int32_t* halo_of,
                   const uint8_t* act, const int8_t* bins, const Halo* halos, Sorted so,
                   int32_t* act_list, DevStats* st, cudaStream_t s);
int launch_permute_vel(int64_t n, const double* vel, const Sorted& so, cudaStream_t s);
int launch_forest(const Sorted& so, const Forest& f, cudaStream_t s);
int tree_levels_for(int64_t n, int64_t count[MAX_LEVELS]);

// search.cu
// Launch shapes that leave every result unchanged (see sidm_tuning).
#ifndef KEY_AXIS_BITS_MAX
#define KEY_AXIS_BITS_MAX 8      // bits per axis of a halo's spatial key
#endif
// Bits per axis of the spatial key below the halo index: at most 8, so that
// a single halo's 24-bit keys sort in three 8-bit passes instead of four.  On
// the 2^20 Hernquist halo and the 2^23 NFW halo the search took the same
// time with 10 bits per axis (30-bit keys); the sort was 0.016 ms faster.
inline __host__ __device__ int key_axis_bits(int halo_bits) {
  const int mb = (30 - halo_bits) / 3;
  return mb < KEY_AXIS_BITS_MAX ? mb : KEY_AXIS_BITS_MAX;
}
#ifndef PAIRS_BLOCKS_MAX
#define PAIRS_BLOCKS_MAX 7       // pair-kernel blocks resident per SM (its register budget)
#endif
struct LaunchTuning {
  int search_window = 384;       // key-order window of the search radius (128 .. 1024)
  int search_chunk = 1;          // a search block claims ranges of 32 search_chunk queries
  int search_blocks_per_sm = 1;  // 32-warp blocks per SM (one is resident at a time)
  int search_run = 2;            // consecutive queries a search warp takes in a row
  int pairs_chunk = 4;
  int pairs_blocks_per_sm = PAIRS_BLOCKS_MAX;
};
int launch_search(const Sorted& so, const Forest& f, int64_t n, const int32_t* act_list,
                  double box, int n_ngb, int tol, double fixed_h, int kernel, int split,
                  double* h_user, int32_t* nb_list, int32_t* nb_count, int nb_stride,
                  DevStats* st, int* work, int sms, const LaunchTuning& t, int all,
                  int hint, cudaStream_t s);
// largest h (rounded up) of each tree node, in the w of its upper corner
int launch_hmax(const Sorted& so, const Forest& f, cudaStream_t s);

// pairs.cu
constexpr int LIM_CAND = 4;   // Eq. 18 maximum: candidates kept per query
struct PairArgs {
  int kernel;
  int split;          // 1: FP32 decisions, FP64 re-test only when |P - u| < 1e-5
  double c_sidm;
  double box;
  int64_t pair_cap;
  // scratch of the FP64 passes that follow the warp pass
  int2* deferred;     // [pair_cap] draws to decide exactly: (i, j | sees << 31), key order
  int32_t* lim_cand;  // [n][LIM_CAND] neighbours that may give the Eq. 18 maximum
  int32_t* lim_cnt;   // [n] their number, -1: more than LIM_CAND (scan the whole list)
  float* lim_g;       // [n] largest FP32 lower bound of v sigma/m (split form: the maximum)
  SigmaTable table;   // tabulated sigma/m (kind SIDM_SIGMA_TABLE)
  OverlapTable ov;    // kernel-overlap estimator (ov.na > 0)
};
int launch_pairs(const Sorted& so, const Forest& f, int64_t n, const int32_t* act_list,
                 const int32_t* nb_list, const int32_t* nb_count, int nb_stride,
                 const PairArgs& a, PairRec* pairs, double* dtlim_user, DevStats* st,
                 int* work, int sms, const LaunchTuning& t, cudaStream_t s);

// resolve.cu
// per-particle segments and cursors of the kick application (sidm_model.cuh)
using ResolveBuffers = sidm_model::detail::Buffers;
static_assert(ST_DIR_FAIL == sidm_model::detail::kDirFail &&
                  ST_ERR_ROUNDS == sidm_model::detail::kErrRounds &&
                  ST_ERR_PAIR_OVERFLOW == sidm_model::detail::kErrPairOverflow,
              "status bits shared with the application templates");
// max_passes: bound on the dataflow passes (0: the built-in 2^22)
// mirror: device address of a pinned host copy of the velocities that the
// kicks keep current (null: none)
int launch_resolve(PairRec* pairs, int64_t pair_cap, int max_passes, double* vel,
                   const double* mass, const int32_t* halo_of, const Halo* halos,
                   double* mirror, const ResolveBuffers& b, DevStats* st, int sms,
                   cudaStream_t s);
void launch_resolve_with_scratch(const PairRec* pairs, int64_t pair_cap, double* vel,
                                 const double* mass, int32_t* head, int32_t* next, uint8_t* flags,
                                 int32_t* mult, uint64_t seed, uint32_t step, DevStats* st,
                                 cudaStream_t s);

// stats.cu
int launch_conserved(const double* vel, const double* mass, int64_t n, double* partial,
                      double* out4, cudaStream_t s);
int conserved_blocks();
int launch_changed(const PairRec* pairs, int64_t cap, const DevStats* st, uint32_t stamp,
                   uint32_t* stamps, const double* vel, int32_t* idx_out, double* vel_out,
                   unsigned long long* count, int sms, cudaStream_t s);
int launch_changed_to_host(const PairRec* pairs, int64_t cap, const DevStats* st,
                           uint32_t stamp, uint32_t* stamps, const double* vel,
                           double* host_vel, int sms, cudaStream_t s);

}  // namespace sidm
