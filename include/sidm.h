/*
 * sidm.h -- C ABI of the B300 SIDM scattering-step library (libsidm.so).
 *
 * The library runs, on one CUDA device, the per-timestep Monte-Carlo
 * scattering step for self-interacting dark matter of Zier et al., "A Novel
 * Implementation of Self-Interacting Dark Matter in AREPO-2":
 *
 *   - for every active particle i, the search radius h_i that encloses
 *     N_ngb +- tol other particles, active or inactive (Sec. 4.2, Sec. 4.5);
 *   - the pair probability P(i|j) = 1/2 m_j (sigma/m)(v_ij) |v_i - v_j|
 *     W(|x_j - x_i|, h_i) dt_i (Eqs. 10, 11, 14, cubic spline or top-hat W, Sec. 4.2;
 *     constant or Yukawa-like sigma/m, Sec. 5.2);
 *   - one Philox-4x32-10 draw per unordered candidate pair against
 *     P_pair = P(i|j)[i active, j in N(i)] + P(j|i)[j active, i in N(j)];
 *   - elastic isotropic centre-of-momentum kicks (Sec. 4.1), several per
 *     particle per step, applied in ascending (ord, min id, max id) order so
 *     that each kick sees the velocities left by the earlier ones (Sec. 4.4);
 *   - the per-pair timestep limit of Eq. 18.
 *
 * Conventions shared by every entry point
 *   - Return value: SIDM_OK (0), a positive warning (the call took effect),
 *     or a negative error (see sidm_status).  sidm_error_string() names it.
 *   - ptr_kind: SIDM_HOST (0) for host memory, SIDM_DEVICE (1) for device
 *     memory of the context's device.  Inputs are copied; the caller keeps
 *     ownership of every pointer it passes and may reuse it after the call
 *     returns (host inputs) or after the context's stream has passed the
 *     call (device inputs).
 *   - Layouts: positions and velocities are n x 3 row-major FP64 arrays
 *     (x0 y0 z0 x1 y1 z1 ...); masses FP64; ids uint32, unique.
 *   - All device work is issued on the context's stream.  sidm_step() does
 *     not wait for the device unless `stats` is non-NULL; errors detected on
 *     the device (a bounded loop that gave up, a full pair buffer) are
 *     latched in the context and returned by the next call that waits:
 *     sidm_step() with stats, sidm_sync(), sidm_get_particles(),
 *     sidm_timestep_limits(), sidm_get_pairs().
 *   - One context is used by one host thread at a time.
 */
#ifndef SIDM_H
#define SIDM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SIDM_API __attribute__((visibility("default")))
#else
#define SIDM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sidm_ctx sidm_ctx;

typedef enum {
  SIDM_OK = 0,
  SIDM_WARN_H_NOT_CONVERGED = 1, /* a bisection hit its evaluation cap (the last h is kept) */
  SIDM_WARN_P_GE_1 = 2,          /* some P_pair >= 1 (accepted; dt too large for Eq. 18)    */
  SIDM_WARN_DIRECTION = 4,       /* a direction draw exhausted its 64 tries (e = +z used)   */
  SIDM_ERR_INVALID_ARG = -1,
  SIDM_ERR_OOM = -2,
  SIDM_ERR_CUDA = -3,
  SIDM_ERR_DEVICE_LIMIT = -4,    /* a bounded device loop or buffer gave up; step not valid:
                                    a full pair buffer is found before any kick (velocities
                                    untouched); after a bounded wait gave up (resolver passes,
                                    key-sort look-back) some kicks may have been applied */
  SIDM_ERR_NOT_READY = -5,       /* sidm_step before sidm_set_particles                     */
  SIDM_ERR_TOO_LARGE = -6        /* input beyond the fixed scratch of a no-allocation call  */
} sidm_status;

enum { SIDM_HOST = 0, SIDM_DEVICE = 1 };
enum { SIDM_KERNEL_CUBIC = 0, SIDM_KERNEL_TOPHAT = 1 };
enum { SIDM_SIGMA_CONST = 0, SIDM_SIGMA_YUKAWA = 1, SIDM_SIGMA_TABLE = 2 };
#define SIDM_SIGMA_TABLE_MAX 256
/* SIDM_FP64_PLAIN: every decision and value equals an FP64 evaluation in a
 * fixed operation order (FP32 is used only where it is provably decisive).
 * SIDM_FP32_SPLIT: separations, neighbour counts, kernel weights and
 * probabilities in FP32; FP64 kicks and accumulators; a draw is decided in
 * FP32 unless u (to its top 24 bits) lies within 1e-5 of the FP32 P, and
 * then exactly in FP64.  Its accepted pairs may differ from the FP64 form in
 * rare near-boundary cases; energy and momentum stay conserved to FP64
 * round-off. */
enum { SIDM_FP64_PLAIN = 0, SIDM_FP32_SPLIT = 1 };
enum { SIDM_ESTIMATOR_ONE_SIDED = 0, SIDM_ESTIMATOR_OVERLAP = 1 };

typedef struct {
  int n_ngb;            /* target neighbour number N_ngb (paper: 32)                     */
  int ngb_tol;          /* accepted band N_ngb +- ngb_tol (paper: 5)                      */
  double c_sidm;        /* C_SIDM of Eq. 18 (paper: 0.1)                                   */
  double box;           /* > 0: periodic cube [0, box)^3; 0: open boundaries              */
  int kernel;           /* SIDM_KERNEL_CUBIC (fiducial) or SIDM_KERNEL_TOPHAT              */
  int precision;        /* SIDM_FP64_PLAIN or SIDM_FP32_SPLIT                              */
  double fixed_h;       /* > 0: every active particle uses this h (no bisection); 0: adaptive */
  int64_t n_max;        /* capacity in particles (0: sized by the first sidm_set_particles) */
  int64_t pair_capacity;/* accepted-pair buffer (0: 2 n_max + 4096)                        */
  void* stream;         /* cudaStream_t for all work; NULL: a stream owned by the context */
  int device;           /* CUDA device ordinal (-1: the current device)                   */
  int profile;          /* 1: time the phases of every step with CUDA events              */
  int use_graph;        /* 1: capture the kernels of a step into a CUDA graph on first use
                           and replay it while the particle count, the halo layout and the
                           launch shapes stay the same (results are unchanged); 0: direct
                           launches.  Ignored while `profile` is set.                      */
  int estimator;        /* g_ij of the pair rate: SIDM_ESTIMATOR_ONE_SIDED, W(r_ij, h_i)
                           (Eq. 14, the paper's fiducial choice), or SIDM_ESTIMATOR_OVERLAP,
                           the overlap of both kernels (Eq. 15, Appendix A; needs
                           sidm_set_overlap_table; h is then found for every particle, and
                           the neighbours of i are all j with r_ij < h_i + h_j)           */
  int rebuild_every;    /* k > 1: the spatial keys are recomputed and sorted only every k
                           steps (and after any change of particle count or halo layout);
                           the steps in between keep that key order and refit the tree's
                           boxes to the current positions (the paper rebuilds its tree only
                           at domain decompositions, Sec. 4.3).  Results are unchanged; the
                           search slows as particles drift from their key order.  0 or 1:
                           every step (the default).                                        */
  int max_resolver_passes;  /* bound on the passes of the resolver's bounded wait (0: 2^22,
                           far above any step's needs).  A step that needs more returns
                           SIDM_ERR_DEVICE_LIMIT with some kicks applied; a small value
                           lets a test make that wait run out on purpose.             */
  /* Device memory of the context (the module keeps its particle and tree
   * arrays itself, Sec. 4.6; a host code may want them in its own pool).
   * alloc(bytes, stream, alloc_user) returns `bytes` (a multiple of 256) of
   * device memory of the context's device, 256-byte aligned, usable on
   * `stream` (the context's cudaStream_t), or NULL when it cannot (the
   * calling entry point then returns SIDM_ERR_OOM).  free(ptr, stream,
   * alloc_user) gives back a pointer alloc returned; the library calls it only
   * after the stream has finished all work on that memory.  Both NULL (the
   * default): cudaMalloc / cudaFree.  Set both or neither (else sidm_create
   * returns SIDM_ERR_INVALID_ARG).  Every device buffer of the context goes
   * through them: the capacity-sized arrays, the tree, the sigma and
   * overlap tables and sidm_autotune's saved state.  Pinned host staging
   * (a few bytes, and the changed-particle staging of sidm_update_velocities)
   * stays with cudaMallocHost. */
  void* (*alloc)(size_t bytes, void* stream, void* alloc_user);
  void (*free)(void* ptr, void* stream, void* alloc_user);
  void* alloc_user;
  int search_hint;      /* 1: a particle's neighbour search starts its candidate gather at
                           9/8 of the h it had at its last search (the h output), and keeps
                           that radius only when the gathered list surely holds N_ngb + tol
                           + 1 particles; otherwise, and at a first search, the radius comes
                           from the key order as in the plain form.  The usual SPH start from
                           the previous smoothing length (Sec. 4.5); h, the neighbour lists
                           and every result are unchanged, only the search's work shrinks
                           while particles move little between steps.  0 (the default): the
                           plain form, which carries no h from one step to the next.   */
} sidm_config;

/* Fills `cfg` with the paper's fiducial values (N_ngb 32 +- 5, C_SIDM 0.1,
 * cubic spline, open boundaries, FP64, adaptive h, current device). */
SIDM_API void sidm_default_config(sidm_config* cfg);

typedef struct {
  int kind;             /* SIDM_SIGMA_CONST or SIDM_SIGMA_YUKAWA                           */
  double sigma0;        /* sigma/m, or sigma0/m of sigma0/m / (1 + (v/w)^2)^2 (Sec. 5.2)    */
  double w;             /* velocity scale w of the Yukawa-like law                         */
  double inelastic;     /* 1 - eps (Sec. 4.1): each scatter leaves the pair's relative speed
                           at eps times its incoming value and keeps its centre-of-momentum
                           velocity; 0 = elastic (the paper's runs).  Must be finite and
                           <= 1 (eps >= 0); eps > 1 adds energy.                            */
} sidm_sigma_model;

typedef struct {
  int64_t n_active;            /* particles active in the step                              */
  int64_t n_candidate_pairs;   /* unordered candidate pairs drawn                            */
  int64_t n_accepted;          /* accepted pairs (kicks applied)                             */
  int64_t n_rounds;            /* resolver rounds of vertex-disjoint pairs                   */
  int64_t n_p_ge_1;            /* candidate pairs with P_pair >= 1                           */
  int64_t n_h_nonconv;         /* bisections that hit the evaluation cap                     */
  int64_t n_dir_fail;          /* direction draws that exhausted their tries                 */
  int64_t max_multiplicity;    /* most kicks received by one particle in the step            */
  double sum_p;                /* sum of P_pair over candidate pairs                         */
  double e_before, e_after;    /* total kinetic energy, compensated sums                     */
  double p_before[3], p_after[3]; /* total momentum                                         */
  int32_t status;              /* bitwise OR of warnings / latched error of this step        */
  int32_t reserved;
} sidm_step_stats;

/* Creates a context on cfg->device.  Returns SIDM_ERR_INVALID_ARG for
 * n_ngb < 1, ngb_tol < 0, ngb_tol >= n_ngb, c_sidm <= 0, box < 0, unknown
 * kernel or precision; SIDM_ERR_CUDA if the device cannot be used. */
SIDM_API int sidm_create(const sidm_config* cfg, sidm_ctx** out);

/* Loads n particles, 0 <= n < 2^30 (replaces any previous set; larger n:
 * SIDM_ERR_INVALID_ARG).  pos, vel: n x 3; mass:
 * n values, or NULL to give every particle `mass_scalar`; ids: n unique
 * uint32 (they key the random draws, Philox counter words 2-3).  With a
 * periodic box every coordinate must lie in [0, box).  The buffers grow if
 * n exceeds the capacity.  Resets h to 0 and the dt limits to +inf. */
SIDM_API int sidm_set_particles(sidm_ctx* ctx, int64_t n, const double* pos, const double* vel,
                       const double* mass, double mass_scalar, const uint32_t* ids,
                       int ptr_kind);

/* Replaces the velocities only (n x 3, the loaded count).  The copy runs on
 * a stream of the context's own, after the work already queued on
 * config.stream that uses the velocities, so that it overlaps the first part
 * of the next step (keys, sort, tree and search read positions only); every
 * later call that uses the velocities is ordered after it.  The source
 * buffer must stay unchanged until the copy is done: after the next
 * sidm_step, sidm_get_particles or sidm_sync has returned on the host
 * (sidm_step returns before it is done). */
SIDM_API int sidm_set_velocities(sidm_ctx* ctx, const double* vel, int ptr_kind);

/* Replaces the positions only (n x 3, the loaded count), as between two
 * scattering steps of a simulation whose particles drift (Fig. 1: the step
 * reads the current positions).  Masses, ids, h, the dt limits and the halo
 * layout are kept.  With a periodic box every coordinate must lie in
 * [0, box); the check waits for the stream and returns
 * SIDM_ERR_INVALID_ARG (positions are then already replaced). */
SIDM_API int sidm_set_positions(sidm_ctx* ctx, const double* pos, int ptr_kind);

/* ---- Sub-ranges of the loaded particles ----------------------------------
 * A serving loop keeps many independent haloes resident in one context
 * (each a segment, see sidm_set_haloes) and admits or retires one without
 * touching the others.
 *
 * sidm_write_particles: replaces particles [offset, offset + count) with
 * `count` new ones (layouts as sidm_set_particles; mass NULL: mass_scalar
 * for each).  0 <= offset <= n (no gap) and offset + count <= the capacity
 * (config.n_max, or the n of the sidm_set_particles that sized the
 * buffers); beyond it SIDM_ERR_INVALID_ARG (the buffers never move).  Their
 * h resets to 0 and their dt limits to +inf; every other particle, its
 * velocity, h and limit stay as they are.  If offset + count > n the loaded
 * count grows to offset + count and the context becomes one halo over all
 * particles (call sidm_set_haloes next).  Needs a context loaded once by
 * sidm_set_particles (n = 0 is allowed). */
SIDM_API int sidm_write_particles(sidm_ctx* ctx, int64_t offset, int64_t count, const double* pos,
                                  const double* vel, const double* mass, double mass_scalar,
                                  const uint32_t* ids, int ptr_kind);

/* Drops the particles from n on (0 <= n <= the loaded count); the context
 * becomes one halo over the remaining ones (call sidm_set_haloes next). */
SIDM_API int sidm_set_count(sidm_ctx* ctx, int64_t n);

/* Moves particles [from, from + count) to [to, to + count) with their
 * positions, velocities, masses, ids, h and dt limits, on the device and in
 * their order (overlapping ranges are fine); both ranges lie within the
 * loaded count.  What was at the destination is overwritten; the source
 * range keeps its old contents.  A serving loop uses it to close a hole left
 * by a retired halo.  A halo moved as a whole steps exactly as before: its
 * results depend on its particles and their order, not on where they sit.
 * The halo layout is not changed (call sidm_set_haloes next). */
SIDM_API int sidm_move_particles(sidm_ctx* ctx, int64_t from, int64_t to, int64_t count);

/* Copies the velocities (n x 3, if vel_out is non-NULL) and h (if h_out is
 * non-NULL) of particles [offset, offset + count); waits for the stream and
 * returns the latched status, as sidm_get_particles. */
SIDM_API int sidm_read_particles(sidm_ctx* ctx, int64_t offset, int64_t count, double* vel_out,
                                 double* h_out, int ptr_kind);

/* Device bytes a context created with `cfg` takes for a capacity of n
 * particles in one halo (the capacity-sized buffers and that halo's tree;
 * not the sigma and overlap tables): what an admission policy under a
 * memory budget needs.  No device work. */
SIDM_API int sidm_context_bytes(const sidm_config* cfg, int64_t n, int64_t* bytes);

/* One scattering step (the whole path above).
 *   active_mask: n bytes, nonzero = active; NULL = all particles active.
 *   dt_bins:     n int8 bins, dt_i = dt_max * 2^-bin_i (power-of-two
 *                individual timesteps); NULL = bin 0 for every particle.
 *   Either pointer may be host or device memory (detected per call).
 *   sigma:       cross-section model.
 *   seed:        Philox key; the context's step counter (starts at 0, +1 per
 *                successful call), modulo 2^32, is Philox counter word 0.
 *   stats:       NULL, or receives the step statistics (waits for the step).
 * The step reads start-of-step velocities for every probability and
 * applies the accepted kicks in (ord, min id, max id) order. */
SIDM_API int sidm_step(sidm_ctx* ctx, const uint8_t* active_mask, const int8_t* dt_bins, double dt_max,
              const sidm_sigma_model* sigma, uint64_t seed, sidm_step_stats* stats);

/* ---- Many independent haloes in one context ------------------------------
 * The particle arrays of sidm_set_particles may hold several independent
 * haloes (e.g. a batch of requests of different sizes), each a contiguous
 * segment: halo k is particles [offsets[k], offsets[k+1]).  Every halo gets
 * its own neighbour structure, start radius, cross-section model, random
 * key and step counter, so a halo's results are bit-identical to a context
 * that holds that halo alone with the same parameters; no pair ever joins
 * particles of two haloes.  One sidm_step_haloes() call steps all haloes
 * with one sequence of kernel launches.
 *
 * sidm_set_haloes: n_halos in [1, 4096]; offsets[0] = 0, offsets[n_halos] =
 * the loaded particle count, non-decreasing (empty haloes are allowed).
 * Must follow sidm_set_particles (which resets the context to one halo). */
typedef struct {
  double dt_max;              /* dt_i = dt_max 2^-bin_i for the halo's particles        */
  sidm_sigma_model sigma;     /* cross-section model of the halo                       */
  uint64_t seed;              /* Philox key of the halo                                */
  uint64_t step;              /* step counter of the halo (Philox counter word 0)      */
} sidm_halo_params;

SIDM_API int sidm_set_haloes(sidm_ctx* ctx, int32_t n_halos, const int64_t* offsets);

/* One scattering step of every halo; params[k] (host array of n_halos)
 * holds halo k's parameters.  active_mask, dt_bins and stats as for
 * sidm_step.  (sidm_step applies one parameter set, with the context's step
 * counter, to every halo.) */
SIDM_API int sidm_step_haloes(sidm_ctx* ctx, const uint8_t* active_mask, const int8_t* dt_bins,
                              const sidm_halo_params* params, sidm_step_stats* stats);

/* Waits for the context's stream; returns the latched device status. */
SIDM_API int sidm_sync(sidm_ctx* ctx);

/* Copies the current velocities (n x 3) and, if h_out is non-NULL, the
 * last h of every particle (0 for particles never active). */
SIDM_API int sidm_get_particles(sidm_ctx* ctx, double* vel_out, double* h_out, int ptr_kind);

/* The particles whose velocities the last step (sidm_step or
 * sidm_step_haloes) changed: the two particles of every accepted pair, each
 * once, in no fixed order.  idx_out[k] is a user-order index, vel_out[3k ..
 * 3k+2] its velocity now.  At most cap entries are written; *n_out is the
 * full count (at most twice the accepted pairs, and at most n).  Waits for
 * the stream.  A host code that keeps its own copy of the velocities moves
 * far fewer bytes this way than with sidm_get_particles, since a step kicks
 * a small fraction of the particles (Sec. 4.1: each particle scatters with
 * probability ~ its rate times dt).  Before the first step, and after
 * sidm_set_particles or sidm_autotune, *n_out = 0. */
SIDM_API int sidm_get_changed(sidm_ctx* ctx, int32_t* idx_out, double* vel_out, int64_t cap,
                              int64_t* n_out, int ptr_kind);

/* Keeps a host copy of the velocities current from the device: from the
 * next step on, each step writes the velocity of every particle it changes
 * into host_vel (user order, n x 3 doubles) as soon as that particle's last
 * kick of the step is applied, so the copy is complete when the step's work
 * on the stream is (sidm_sync, or any call that waits for the stream).
 * Entries of particles a step does not change are not touched: host_vel
 * must already hold the velocities the step starts from (those set or
 * loaded, as uploaded from this same array by sidm_set_velocities).
 * host_vel must be pinned host memory the device can address (cudaHostAlloc
 * or cudaHostRegister memory on a system with unified addressing, such as
 * PyTorch's pinned tensors) and hold n particles; a step of a context with
 * more particles than n returns SIDM_ERR_INVALID_ARG.  NULL stops the
 * writes.  Waits for the stream; sidm_autotune's trial steps do not write
 * the copy.  SIDM_ERR_INVALID_ARG if host_vel is not such memory. */
SIDM_API int sidm_set_velocity_mirror(sidm_ctx* ctx, double* host_vel, int64_t n);

/* Brings a host copy of the velocities up to date after a step: vel_inout
 * (host memory, n x 3) holds the velocities before the last step; the
 * velocities the step changed are written into it, and nothing else is
 * touched.  Only the changed particles cross the bus.  If vel_inout is
 * pinned host memory that the device can address (cudaHostAlloc or
 * cudaHostRegister memory on a system with unified addressing, such as
 * PyTorch's pinned tensors), a kernel writes each changed particle's
 * velocity straight into it; the pinned range must then cover all n x 3
 * doubles.  Otherwise they go, as with sidm_get_changed, into pinned staging
 * of the context's own (allocated on the first such call), and a host loop
 * scatters them.  Waits for the stream; returns the latched status of the
 * last step. */
SIDM_API int sidm_update_velocities(sidm_ctx* ctx, double* vel_inout);

/* Copies the Eq. 18 limit of every particle from its last active step
 * (+inf before its first active step, and when no neighbour moves
 * relative to it). */
SIDM_API int sidm_timestep_limits(sidm_ctx* ctx, double* dt_limit_out, int ptr_kind);

/* Accepted pairs of the last step in application order: ab[2k] = min id,
 * ab[2k+1] = max id, ord[k] = the 64-bit order key; up to `cap` entries,
 * *n_out = the total.  Host pointers. */
SIDM_API int sidm_get_pairs(sidm_ctx* ctx, uint32_t* ab, uint64_t* ord, int64_t cap, int64_t* n_out);

/* Step counter (resume support: the random stream is a pure function of
 * (seed, step counter, ids), so restoring the particles and the counter
 * reproduces a run bit for bit).  The draws use the counter modulo 2^32:
 * steps 2^32 apart share their random streams. */
SIDM_API int sidm_get_step(const sidm_ctx* ctx, uint64_t* step);
SIDM_API int sidm_set_step(sidm_ctx* ctx, uint64_t step);

/* Phase times (milliseconds, CUDA events on the context's stream) of the
 * last step of a context created with profile = 1; waits for the stream.
 * ms[k] for k < min(n, SIDM_N_PHASES): 0 keys (bounding box, start radius,
 * spatial keys), 1 sort, 2 structure (key-order copy, active list, box
 * tree), 3 search (h_SI), 4 pairs (probabilities, draws, Eq. 18),
 * 5 resolve (kicks).  Returns SIDM_ERR_INVALID_ARG without profiling. */
#define SIDM_N_PHASES 6
SIDM_API int sidm_phase_times(sidm_ctx* ctx, float* ms, int n);

/* Kernels launched by the context so far (all of them are this library's). */
SIDM_API int64_t sidm_kernel_launches(const sidm_ctx* ctx);

/* Tabulated sigma/m(v) (Sec. 4.1: an arbitrary tabulated function of the
 * pair's relative velocity, interpolated linearly in log v).  Host arrays of
 * n nodes (2 <= n <= SIDM_SIGMA_TABLE_MAX): v strictly increasing and > 0,
 * sigma/m >= 0, all finite; copied.  sigma/m(v) = sigma_0 for v <= v_0,
 * sigma_{n-1} for v >= v_{n-1}, else sigma_k + t (sigma_{k+1} - sigma_k) with
 * t = (ln v - ln v_k) / (ln v_{k+1} - ln v_k) on the segment v_k <= v < v_{k+1}.
 * Used by every halo whose model has kind SIDM_SIGMA_TABLE (sigma0 and w are
 * then ignored); a step with that kind before a table is set returns
 * SIDM_ERR_INVALID_ARG.  The logarithm of v in the FP64 evaluation is the
 * device's; results agree with a host evaluation to the last bits of
 * sigma/m (draws differ only if u falls within that distance of P). */
SIDM_API int sidm_set_sigma_table(sidm_ctx* ctx, int32_t n, const double* v,
                                  const double* sigma_over_m);

/* Table of the kernel-overlap estimator (Eq. 15, Appendix A): ghat(a, s) =
 * int W(|y|, a) W(|y - s z|, 1 - a) d^3y on a = k / (2 na), k = 0..na, and
 * s = l / ns, l = 0..ns, as (na + 1) x (ns + 1) host doubles, row-major in a
 * (copied).  A pair uses g_ij = ghat(min(h_i, h_j)/H, r_ij/H) / H^3 with
 * H = h_i + h_j, ghat interpolated bilinearly (0 for s >= 1).  1 <= na <= 4096,
 * 1 <= ns <= 65536, values finite and >= 0.  Required before a step of a
 * context with estimator SIDM_ESTIMATOR_OVERLAP (else SIDM_ERR_NOT_READY). */
SIDM_API int sidm_set_overlap_table(sidm_ctx* ctx, int32_t na, int32_t ns, const double* table);

/* Computes that table for kernel SIDM_KERNEL_CUBIC or SIDM_KERNEL_TOPHAT into
 * `out` ((na + 1) x (ns + 1) host doubles): spherical shells around one
 * particle, the angular integral of the other kernel in closed form, the
 * radial integral by Gauss-Legendre between the kernels' breakpoints (about
 * 1e-12 relative).  Host only; no context needed. */
SIDM_API int sidm_overlap_table(int kernel, int32_t na, int32_t ns, double* out);

/* ---- launch shapes (no counterpart in the paper) ------------------------
 * How the step's kernels are launched.  Every choice gives bit-identical
 * results; only the time changes.  Zero fields take the defaults. */
typedef struct {
  int search_window;        /* key-order window that bounds each search radius:
                               128, 256, 384 (default), 512, 768 or 1024 particles; a window
                               of fewer than n_ngb + ngb_tol + 2 particles runs as
                               256                                                   */
  int search_chunk;         /* a search block (32 warps, one run of search_run queries
                               per warp at a time) claims ranges of 32 x search_chunk
                               consecutive runs, 1..64 (1)                           */
  int search_blocks_per_sm; /* search blocks launched per SM, 1..8 (1); one is resident
                               at a time, the others start as blocks finish          */
  int pairs_chunk;          /* queries a pair warp claims at a time, 1..64 (4)        */
  int pairs_blocks_per_sm;  /* pair blocks of 4 warps per SM, 1..7 (7)                */
  int search_run;           /* consecutive active queries a search warp takes in a row,
                               1..16 (2); each query of a run after the first sizes
                               its first gather from the previous one's h            */
} sidm_tuning;

/* Sets / reads the launch shapes of the context.  SIDM_ERR_INVALID_ARG for a
 * value out of range (the context keeps its shapes).  Setting them drops a
 * captured step graph (it is captured again on the next step). */
SIDM_API int sidm_set_tuning(sidm_ctx* ctx, const sidm_tuning* t);
SIDM_API int sidm_get_tuning(const sidm_ctx* ctx, sidm_tuning* t);

/* Times candidate launch shapes on the next step (active mask, bins and one
 * sidm_halo_params per halo as for sidm_step_haloes; a single-halo context
 * takes one) and keeps the fastest.  Each candidate runs `reps` (1..16)
 * times from the same state and counts with its fastest run; a shape
 * replaces the current one only if it is at least 2 % faster.  Afterwards
 * the velocities, h, timestep limits
 * and the step counter are restored, so the call leaves the simulation
 * where it was.  Coordinate search: window, then search run, chunk and blocks,
 * then pair chunk and blocks.  Writes the chosen shapes to `best` (nullable).
 * Synchronises the stream; allocates one temporary copy of the state. */
SIDM_API int sidm_autotune(sidm_ctx* ctx, const uint8_t* active_mask, const int8_t* dt_bins,
                           const sidm_halo_params* params, int reps, sidm_tuning* best);

/* 1: the step runs as a captured CUDA graph; 0: direct launches (use_graph
 * off, profiling, or nothing stepped yet); -1: the driver refused the
 * capture and the context launches directly. */
SIDM_API int sidm_graph_state(const sidm_ctx* ctx);

/* ---- Kick application without any device allocation ----------------------
 * The paper has no counterpart to this entry point: it exists for callers
 * that cannot let a library allocate device memory -- simulation codes that
 * reserve all GPU memory in their own pool at start-up, or that call in from
 * a place where a cudaMalloc would synchronise the whole device or is not
 * allowed.  It applies a given list of accepted pairs to velocities exactly
 * as the kick phase of sidm_step() does (each particle meets its pairs in
 * ascending (ord, a, b) order; direction from Philox (seed, step, 1 + t, a,
 * b); elastic kick), so its result equals sidm_step()'s velocities for the
 * pairs sidm_get_pairs() reports.
 *
 * Memory: all scratch lives in one fixed array inside the library (a
 * file-scope __device__ array of 10.25 MiB), which every GPU that loads
 * the library holds until the process exits.  Hence the fixed maxima below;
 * larger inputs are rejected with SIDM_ERR_TOO_LARGE before any GPU work.
 * Nothing is allocated: no cudaMalloc, cudaFree or allocating library call.
 *
 * Arguments (all device pointers of the current device):
 *   pairs   n_pairs records; ia, ib are indices into vel / mass, a, b the
 *           ids used in the random counter (as sidm_get_pairs() reports them
 *           for ids equal to the indices), ord the order key;
 *   vel     n x 3 FP64 velocities, updated in place; mass: n FP64 masses;
 *   seed, step: the Philox key and the step counter of the draw;
 *   stream: cudaStream_t (NULL: the legacy default stream).
 * Records with equal (ord, a, b) keys are applied one after the other, in
 * the order given.  The step counter enters the random counter modulo 2^32
 * (as in sidm_step).
 * Returns SIDM_OK (or SIDM_WARN_DIRECTION); SIDM_ERR_TOO_LARGE for
 * n > SIDM_NOALLOC_MAX_PARTICLES or n_pairs > SIDM_NOALLOC_MAX_PAIRS;
 * SIDM_ERR_INVALID_ARG for NULL pointers, negative sizes, or a pair whose
 * index lies outside [0, n) or names one particle twice (checked on the
 * device; then no velocity is changed); SIDM_ERR_DEVICE_LIMIT when the
 * pairs form a dependency chain longer than the 4096 rounds of the kick
 * kernel (for instance one particle in more than 4096 pairs): the kicks of
 * the completed rounds are then already in vel; SIDM_ERR_CUDA on a CUDA
 * failure.  The call waits for the stream before it returns.
 *
 * Set-up: the first call on each device looks up the device address of the
 * scratch array (with that device current); make that first call before
 * any stream capture.  Every call shares the one array per device and
 * clears the parts it uses at the start; calls that overlap on the GPU
 * (different streams or host threads, same device) race on it and must not
 * be issued. */
#define SIDM_NOALLOC_MAX_PARTICLES (1 << 20)
#define SIDM_NOALLOC_MAX_PAIRS (1 << 18)
typedef struct {
  uint64_t ord;   /* order key of the pair                 */
  uint32_t a, b;  /* ids of the two particles, a < b         */
  int32_t ia, ib; /* indices of the a- and b-particle         */
} sidm_pair;
SIDM_API int sidm_apply_pairs_noalloc(const sidm_pair* pairs, int64_t n_pairs, double* vel,
                                      const double* mass, int64_t n, uint64_t seed,
                                      uint64_t step, void* stream);

SIDM_API const char* sidm_error_string(int status);

/* Frees every device buffer of the context (waits for its stream). */
SIDM_API void sidm_destroy(sidm_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* SIDM_H */
