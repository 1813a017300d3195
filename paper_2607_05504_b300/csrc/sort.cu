// Least-significant-digit radix sort of (uint32 key, int32 value) pairs and a
// device-wide exclusive scan.  The sort orders particles by their spatial key
// so that tree leaves are compact; it is stable, hence deterministic.
//
// Each 8-bit pass: (1) every block histograms the digit of its 4096-key tile,
// (2) one exclusive scan over the digit-major [digit][block] table gives every
// (digit, block) its output offset, (3) every block re-reads its tile in
// order, ranks each key among the earlier keys of the same digit (warp
// match + per-warp counters in shared memory) and scatters it.
#include "sidm_internal.cuh"

namespace sidm {

namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int RS_RADIX = 256;
constexpr int RS_WARPS = RS_THREADS / WARP;

constexpr int SC_THREADS = 1024;
constexpr int SC_ITEMS = 4;
constexpr int SC_TILE = SC_THREADS * SC_ITEMS;

__global__ void __launch_bounds__(RS_THREADS) rs_hist_kernel(const uint32_t* __restrict__ keys,
                                                             int64_t n, int shift,
                                                             uint32_t* __restrict__ hist,
                                                             int nblocks) {
  __shared__ uint32_t h[RS_RADIX];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int r = 0; r < RS_ITEMS; ++r) {
    const int64_t i = base + (int64_t)r * RS_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(RS_THREADS) rs_scatter_kernel(
    const uint32_t* __restrict__ keys_in, const int32_t* __restrict__ vals_in,
    uint32_t* __restrict__ keys_out, int32_t* __restrict__ vals_out, int64_t n, int shift,
    const uint32_t* __restrict__ offs, int nblocks) {
  __shared__ uint32_t s_run[RS_RADIX];
  __shared__ uint32_t s_cnt[RS_WARPS][RS_RADIX];
  __shared__ uint32_t s_base[RS_WARPS][RS_RADIX];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  s_run[t] = offs[(int64_t)t * nblocks + blockIdx.x];
  for (int w = 0; w < RS_WARPS; ++w) s_cnt[w][t] = 0;
  __syncthreads();
  const uint32_t lt = (1u << lane) - 1u;
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int r = 0; r < RS_ITEMS; ++r) {
    const int64_t i = base + (int64_t)r * RS_THREADS + t;
    const bool valid = i < n;
    uint32_t key = 0, d = RS_RADIX;
    int32_t val = 0;
    if (valid) {
      key = keys_in[i];
      val = vals_in[i];
      d = (key >> shift) & 255u;
    }
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t rank = __popc(peers & lt);
    if (valid && rank == 0) s_cnt[warp][d] = __popc(peers);
    __syncthreads();
    {
      uint32_t run = s_run[t];
      for (int w = 0; w < RS_WARPS; ++w) {
        const uint32_t c = s_cnt[w][t];
        s_base[w][t] = run;
        run += c;
        s_cnt[w][t] = 0;
      }
      s_run[t] = run;
    }
    __syncthreads();
    if (valid) {
      const uint32_t pos = s_base[warp][d] + rank;
      keys_out[pos] = key;
      vals_out[pos] = val;
    }
  }
}

// Block-wide exclusive scan of SC_TILE items; returns the tile total.
__device__ uint32_t block_scan_tile(uint32_t (&v)[SC_ITEMS], uint32_t* s_warp) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  uint32_t sum = 0;
#pragma unroll
  for (int k = 0; k < SC_ITEMS; ++k) { const uint32_t x = v[k]; v[k] = sum; sum += x; }
  uint32_t inc = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_warp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = (lane < SC_THREADS / 32) ? s_warp[lane] : 0u;
    uint32_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    s_warp[lane] = wi - w;         // exclusive prefix of warp totals
    if (lane == 31) s_warp[32] = wi;
  }
  __syncthreads();
  const uint32_t off = s_warp[warp] + (inc - sum);
#pragma unroll
  for (int k = 0; k < SC_ITEMS; ++k) v[k] += off;
  const uint32_t total = s_warp[32];
  __syncthreads();
  return total;
}

__global__ void __launch_bounds__(SC_THREADS) scan_tiles_kernel(const uint32_t* in, uint32_t* out,
                                                               int64_t n, uint32_t* sums) {
  __shared__ uint32_t s_warp[33];
  const int64_t base = (int64_t)blockIdx.x * SC_TILE + (int64_t)threadIdx.x * SC_ITEMS;
  uint32_t v[SC_ITEMS];
#pragma unroll
  for (int k = 0; k < SC_ITEMS; ++k) v[k] = (base + k < n) ? in[base + k] : 0u;
  const uint32_t total = block_scan_tile(v, s_warp);
#pragma unroll
  for (int k = 0; k < SC_ITEMS; ++k)
    if (base + k < n) out[base + k] = v[k];
  if (threadIdx.x == 0 && sums) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(SC_THREADS) scan_add_kernel(uint32_t* out, int64_t n,
                                                             const uint32_t* sums) {
  const uint32_t add = sums[blockIdx.x];
  const int64_t base = (int64_t)blockIdx.x * SC_TILE;
  for (int k = threadIdx.x; k < SC_TILE; k += SC_THREADS)
    if (base + k < n) out[base + k] += add;
}

}  // namespace

size_t exclusive_scan_temp_bytes(int64_t n) {
  const int64_t tiles = (n + SC_TILE - 1) / SC_TILE;
  return (size_t)(tiles + 1) * sizeof(uint32_t);
}

// Exclusive scan of n uint32 (in may equal out); n <= SC_TILE^2 (16.7 M).
int exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* tmp,
                       cudaStream_t s) {
  if (n <= 0) return 0;
  const int64_t tiles = (n + SC_TILE - 1) / SC_TILE;
  if (tiles == 1) {
    scan_tiles_kernel<<<1, SC_THREADS, 0, s>>>(in, out, n, nullptr);
    return 1;
  }
  scan_tiles_kernel<<<(unsigned)tiles, SC_THREADS, 0, s>>>(in, out, n, tmp);
  scan_tiles_kernel<<<1, SC_THREADS, 0, s>>>(tmp, tmp, tiles, nullptr);
  scan_add_kernel<<<(unsigned)tiles, SC_THREADS, 0, s>>>(out, n, tmp);
  return 3;
}

size_t radix_sort_temp_bytes(int64_t n) {
  const int64_t nblocks = (n + RS_TILE - 1) / RS_TILE;
  const int64_t entries = nblocks * RS_RADIX;
  return (size_t)entries * sizeof(uint32_t) + exclusive_scan_temp_bytes(entries) + 256;
}

// Sorts (keys, vals) by the low `key_bits` bits of the keys; the result is
// left in (keys, vals).  keys_alt / vals_alt are scratch of n entries.
int radix_sort_pairs(uint32_t* keys, int32_t* vals, uint32_t* keys_alt, int32_t* vals_alt,
                     int64_t n, int key_bits, void* temp, cudaStream_t s) {
  if (n <= 1) return 0;
  int launches = 0;
  const int nblocks = (int)((n + RS_TILE - 1) / RS_TILE);
  const int64_t entries = (int64_t)nblocks * RS_RADIX;
  uint32_t* hist = (uint32_t*)temp;
  uint32_t* scan_tmp = hist + entries;
  int passes = (key_bits + 7) / 8;
  if (passes & 1) ++passes;  // even number of passes: the result lands back in keys/vals
  uint32_t* kin = keys;
  int32_t* vin = vals;
  uint32_t* kout = keys_alt;
  int32_t* vout = vals_alt;
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    rs_hist_kernel<<<nblocks, RS_THREADS, 0, s>>>(kin, n, shift, hist, nblocks);
    launches += 2 + exclusive_scan_u32(hist, hist, entries, scan_tmp, s);
    rs_scatter_kernel<<<nblocks, RS_THREADS, 0, s>>>(kin, vin, kout, vout, n, shift, hist, nblocks);
    uint32_t* tk = kin; kin = kout; kout = tk;
    int32_t* tv = vin; vin = vout; vout = tv;
  }
  return launches;
}

}  // namespace sidm
