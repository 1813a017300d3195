// Kick application without device allocation (sidm_apply_pairs_noalloc).
//
// For callers that cannot let a library allocate device memory (codes that
// reserve all GPU memory in their own pool at start-up, or that call in from
// a place where cudaMalloc would synchronise the device or is not allowed).
// The kick kernel of the scattering step needs scratch -- per-particle list
// heads and multiplicities, per-pair links and flags, a status block -- and
// here that scratch is one fixed file-scope __device__ array instead of
// context buffers.  The array is resident on every GPU that loads the
// library until the process exits; its fixed size bounds the inputs.
#include <cstddef>
#include <mutex>

#include "sidm_internal.cuh"

namespace sidm {
namespace {

constexpr int64_t NA_MAX = SIDM_NOALLOC_MAX_PARTICLES;
constexpr int64_t NP_MAX = SIDM_NOALLOC_MAX_PAIRS;

// byte layout of the scratch array (every part 256-byte aligned)
constexpr size_t OFF_HEAD = 0;
constexpr size_t OFF_MULT = OFF_HEAD + NA_MAX * sizeof(int32_t);
constexpr size_t OFF_NEXT = OFF_MULT + NA_MAX * sizeof(int32_t);
constexpr size_t OFF_FLAGS = OFF_NEXT + 2 * NP_MAX * sizeof(int32_t);
constexpr size_t OFF_STATS = OFF_FLAGS + ((NP_MAX + 255) / 256) * 256;
constexpr size_t SCRATCH_BYTES = OFF_STATS + 256;

static_assert(sizeof(sidm_pair) == sizeof(PairRec), "sidm_pair must match the pair record");
static_assert(OFF_STATS % 256 == 0 && sizeof(DevStats) <= 256, "scratch layout");

static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[MAX_DEVICES] = {};

// Device address of the scratch array for the current device (looked up
// once per device, with that device current).
cudaError_t scratch_for_current_device(unsigned char** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = (unsigned char*)g_scratch_addr[dev];
  return cudaSuccess;
}

// Clears what must start cleared (list heads -1, multiplicities and flags 0,
// the status block), sets the pair count and checks every pair's indices.
// pad = 1 marks an invalid index; the count is then set to 0 so that the
// kick kernel changes nothing.
__global__ void noalloc_prepare_kernel(const PairRec* pairs, int64_t n_pairs, int64_t n,
                                       unsigned char* scratch) {
  int32_t* head = (int32_t*)(scratch + OFF_HEAD);
  int32_t* mult = (int32_t*)(scratch + OFF_MULT);
  uint8_t* flags = scratch + OFF_FLAGS;
  DevStats* st = (DevStats*)(scratch + OFF_STATS);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int64_t i = t0; i < n; i += stride) {
    head[i] = -1;
    mult[i] = 0;
  }
  bool bad = false;
  for (int64_t p = t0; p < n_pairs; p += stride) {
    flags[p] = 0;
    const int64_t ia = pairs[p].ia, ib = pairs[p].ib;
    if (ia < 0 || ia >= n || ib < 0 || ib >= n || ia == ib) bad = true;
  }
  if (t0 == 0) {
    st->n_active = st->n_cand = st->n_rounds = st->n_pge1 = 0;
    st->n_nonconv = st->n_dirfail = st->max_mult = 0;
    st->sum_p = 0.0;
    st->status = 0;
  }
  if (bad) atomicOr(&st->pad, 1u);
}

__global__ void noalloc_count_kernel(int64_t n_pairs, unsigned char* scratch) {
  DevStats* st = (DevStats*)(scratch + OFF_STATS);
  st->n_acc = st->pad ? 0ull : (unsigned long long)n_pairs;
}

__global__ void noalloc_clear_pad_kernel(unsigned char* scratch) {
  ((DevStats*)(scratch + OFF_STATS))->pad = 0;
}

}  // namespace
}  // namespace sidm

using namespace sidm;

extern "C" int sidm_apply_pairs_noalloc(const sidm_pair* pairs, int64_t n_pairs, double* vel,
                                        const double* mass, int64_t n, uint64_t seed,
                                        uint64_t step, void* stream) {
  if (n < 0 || n_pairs < 0) return SIDM_ERR_INVALID_ARG;
  if (n > NA_MAX || n_pairs > NP_MAX) return SIDM_ERR_TOO_LARGE;
  if (n_pairs > 0 && (!pairs || !vel || !mass)) return SIDM_ERR_INVALID_ARG;
  if (n_pairs == 0) return SIDM_OK;
  unsigned char* scratch = nullptr;
  if (scratch_for_current_device(&scratch) != cudaSuccess) return SIDM_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  const PairRec* pr = (const PairRec*)pairs;
  const int64_t work = n > n_pairs ? n : n_pairs;
  int64_t blocks = (work + 255) / 256;
  if (blocks > 148 * 8) blocks = 148 * 8;
  noalloc_clear_pad_kernel<<<1, 1, 0, s>>>(scratch);
  noalloc_prepare_kernel<<<(unsigned)blocks, 256, 0, s>>>(pr, n_pairs, n, scratch);
  noalloc_count_kernel<<<1, 1, 0, s>>>(n_pairs, scratch);
  launch_resolve_with_scratch(pr, NP_MAX, vel, mass, (int32_t*)(scratch + OFF_HEAD),
                              (int32_t*)(scratch + OFF_NEXT), scratch + OFF_FLAGS,
                              (int32_t*)(scratch + OFF_MULT), seed, (uint32_t)step,
                              (DevStats*)(scratch + OFF_STATS), s);
  if (cudaGetLastError() != cudaSuccess) return SIDM_ERR_CUDA;
  unsigned st_word[2] = {0u, 0u};  // status, pad
  if (cudaMemcpyAsync(st_word, scratch + OFF_STATS + offsetof(DevStats, status), sizeof(st_word),
                      cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return SIDM_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return SIDM_ERR_CUDA;
  if (st_word[1]) return SIDM_ERR_INVALID_ARG;
  if (st_word[0] & ST_ERR_MASK) return SIDM_ERR_DEVICE_LIMIT;
  return (st_word[0] & ST_DIR_FAIL) ? SIDM_WARN_DIRECTION : SIDM_OK;
}
