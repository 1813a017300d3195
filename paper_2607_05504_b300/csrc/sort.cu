// Least-significant-digit radix sort of (uint32 key, int32 value) pairs.  The
// sort orders particles by their spatial key so that tree leaves are compact;
// it is stable, hence deterministic.
//
// Single-pass digit placement ("onesweep" form, Merrill & Garland's
// decoupled look-back applied per digit):
//   1. one kernel histograms every 8-bit digit of every pass at once (the
//      digit counts do not depend on the order of the keys) and clears the
//      look-back slots;
//   2. per pass, one kernel: every block claims the next 4096-key tile in
//      order, publishes its digit counts, adds up the counts of the earlier
//      tiles from their published slots (stopping at the first slot that
//      already holds an inclusive prefix) and publishes its own inclusive
//      prefix.  Each of the 16 warps ranks the keys of its own 256-key part
//      of the tile among the earlier keys of the same digit (peers found by
//      one vote per digit bit, warp-private counters, no block barrier),
//      the tile is put in digit order in shared memory, and runs of equal
//      digits are written out by consecutive threads.
// A slot is one 32-bit word holding a 2-bit state and a 30-bit count, so a
// reader sees the state and the count together without a fence.  Six
// launches per sort at most (a memset, the histogram, up to four passes) instead of a
// histogram, scan and scatter per pass.
#include "sidm_internal.cuh"

namespace sidm {

namespace {

constexpr int OS_THREADS = 256;
constexpr int OS_ITEMS = 16;
constexpr int OS_TILE = OS_THREADS * OS_ITEMS;
constexpr int RADIX = 256;
constexpr int MAX_PASSES = 4;
constexpr uint32_t SLOT_AGG = 1u << 30;    // the tile's own count
constexpr uint32_t SLOT_PRE = 2u << 30;    // the count of this and every earlier tile
constexpr uint32_t SLOT_STATE = 3u << 30;
constexpr uint32_t SLOT_VALUE = (1u << 30) - 1u;
constexpr int LOOKBACK_MAX_SPINS = 1 << 20;
constexpr int LOOKBACK_BATCH = 8;            // earlier slots loaded per round trip
// temp layout (32-bit words): digit counts [MAX_PASSES][RADIX], tile
// counters [MAX_PASSES] (padded to 64 words), then the slots
// [passes][tiles][RADIX]
constexpr int HEAD_WORDS = MAX_PASSES * RADIX + 64;

__device__ __forceinline__ void st_relaxed_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__global__ void __launch_bounds__(OS_THREADS) os_hist_kernel(const uint32_t* __restrict__ keys,
                                                             int64_t n, int passes,
                                                             uint32_t* __restrict__ counts,
                                                             uint32_t* __restrict__ slots,
                                                             int tiles) {
  __shared__ uint32_t h[MAX_PASSES][RADIX];
  const int t = threadIdx.x;
#pragma unroll
  for (int p = 0; p < MAX_PASSES; ++p) h[p][t] = 0;
  for (int p = 0; p < passes; ++p)
    slots[((int64_t)p * tiles + blockIdx.x) * RADIX + t] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * OS_TILE;
  for (int r = 0; r < OS_ITEMS; ++r) {
    const int64_t i = base + (int64_t)r * OS_THREADS + t;
    if (i < n) {
      const uint32_t k = keys[i];
      for (int p = 0; p < passes; ++p) atomicAdd(&h[p][(k >> (8 * p)) & 255u], 1u);
    }
  }
  __syncthreads();
  for (int p = 0; p < passes; ++p)
    if (h[p][t]) atomicAdd(&counts[p * RADIX + t], h[p][t]);
}

// A pass runs PASS_THREADS threads on each 4096-key tile: warp w ranks keys
// [w 32 PASS_ITEMS, (w + 1) 32 PASS_ITEMS) of the tile; the per-digit work
// (tile counts, scans, look-back) is done by the first RADIX threads.  The
// tile is put in digit order in shared memory before the look-back (which
// then runs with the keys out of registers), and written out in runs of
// equal digits, so that neighbouring threads write neighbouring places.
constexpr int PASS_THREADS = 512;
constexpr int PASS_ITEMS = OS_TILE / PASS_THREADS;
constexpr int PASS_WARPS = PASS_THREADS / WARP;
constexpr int DIGIT_WARPS = RADIX / WARP;
static_assert(PASS_THREADS >= RADIX && PASS_ITEMS * PASS_THREADS == OS_TILE, "pass tiling");
static_assert(PASS_WARPS * RADIX == OS_TILE, "the warp counters and the tile's keys share memory");

__global__ void __launch_bounds__(PASS_THREADS, 2) os_pass_kernel(
    const uint32_t* __restrict__ keys_in, const int32_t* __restrict__ vals_in,
    uint32_t* __restrict__ keys_out, int32_t* __restrict__ vals_out, int64_t n, int pass,
    const uint32_t* __restrict__ counts, uint32_t* tile_ctr, uint32_t* slots, unsigned* status) {
  __shared__ uint32_t s_tile;
  // per warp: keys of each digit, then the warp's start within the digit;
  // afterwards the tile's keys in digit order
  __shared__ uint32_t s_cnt_key[PASS_WARPS * RADIX];
  __shared__ int32_t s_val[OS_TILE];
  __shared__ uint32_t s_wsum[2][DIGIT_WARPS];
  __shared__ uint32_t s_tstart[RADIX];   // start of each digit within the tile
  __shared__ int32_t s_off[RADIX];       // output place minus tile place, per digit
  uint32_t(*s_cnt)[RADIX] = reinterpret_cast<uint32_t(*)[RADIX]>(s_cnt_key);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const bool digit_thread = t < RADIX;               // thread t owns digit t
  const int shift = 8 * pass;
  if (t == 0) s_tile = atomicAdd(&tile_ctr[pass], 1u);
  for (int i = t; i < PASS_WARPS * RADIX; i += PASS_THREADS) s_cnt_key[i] = 0;
  __syncthreads();
  const int64_t tile = s_tile;
  const int64_t tbase = tile * OS_TILE;
  const int64_t base = tbase + (int64_t)warp * (PASS_ITEMS * WARP);
  const int tn = (int)(n - tbase < OS_TILE ? n - tbase : OS_TILE);   // keys in the tile

  // 1. rank every key among the earlier keys of its digit in the warp's
  //    part of the tile (warp-private counters, no block barrier)
  uint32_t key[PASS_ITEMS], rank[PASS_ITEMS];
  int32_t val[PASS_ITEMS];
  const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < PASS_ITEMS; ++r) {
    const int64_t i = base + (int64_t)r * WARP + lane;
    const bool valid = i < n;
    key[r] = valid ? keys_in[i] : 0u;
    val[r] = valid ? vals_in[i] : 0;
    const uint32_t d = valid ? (key[r] >> shift) & 255u : (uint32_t)RADIX;
    // lanes with the same digit: one vote per digit bit (and one for validity)
    uint32_t peers = __ballot_sync(0xffffffffu, valid);
    if (!valid) peers = ~peers;
#pragma unroll
    for (int bit = 0; bit < 8; ++bit) {
      const bool set = (d >> bit) & 1u;
      const uint32_t vb = __ballot_sync(0xffffffffu, set);
      peers &= set ? vb : ~vb;
    }
    const int leader = __ffs(peers) - 1;
    uint32_t before = 0;
    if (valid && lane == leader) {
      before = s_cnt[warp][d];
      s_cnt[warp][d] = before + __popc(peers);
    }
    rank[r] = __shfl_sync(0xffffffffu, before, leader) + __popc(peers & lt);
    __syncwarp();
  }
  __syncthreads();

  // 2. the tile's count of digit t, published at once; each warp's start
  //    within the digit; scans over the digits of the tile's counts and of
  //    the global counts
  uint32_t cnt = 0, g = 0, ic = 0, ig = 0;
  if (digit_thread) {
#pragma unroll
    for (int w = 0; w < PASS_WARPS; ++w) {
      const uint32_t c = s_cnt[w][t];
      s_cnt[w][t] = cnt;
      cnt += c;
    }
    st_relaxed_u32(slots + tile * RADIX + t, (tile == 0 ? SLOT_PRE : SLOT_AGG) | cnt);
    g = counts[pass * RADIX + t];
    ic = cnt;
    ig = g;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t yc = __shfl_up_sync(0xffffffffu, ic, o);
      const uint32_t yg = __shfl_up_sync(0xffffffffu, ig, o);
      if (lane >= o) {
        ic += yc;
        ig += yg;
      }
    }
    if (lane == 31) {
      s_wsum[0][warp] = ic;
      s_wsum[1][warp] = ig;
    }
  }
  __syncthreads();
  if (digit_thread) {
    uint32_t tc = ic - cnt, tg = ig - g;
    for (int w = 0; w < warp; ++w) {
      tc += s_wsum[0][w];
      tg += s_wsum[1][w];
    }
    s_tstart[t] = tc;
    ig = tg;   // keys of smaller digits, over all tiles
  }
  __syncthreads();

  // 3. each key's place in the tile's digit order, then the tile in that
  //    order (the keys over the counters, which are no longer needed)
#pragma unroll
  for (int r = 0; r < PASS_ITEMS; ++r) {
    const uint32_t d = (key[r] >> shift) & 255u;
    rank[r] += s_tstart[d] + s_cnt[warp][d];
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < PASS_ITEMS; ++r) {
    if (base + (int64_t)r * WARP + lane < n) {
      s_cnt_key[rank[r]] = key[r];
      s_val[rank[r]] = val[r];
    }
  }

  // 4. look back over the earlier tiles: slots j, j-1, ... are loaded
  //    LOOKBACK_BATCH at a time and consumed in order until an inclusive
  //    prefix; a slot not yet published is reloaded (the earlier tile's
  //    block is resident and publishes before it waits on anything; the
  //    wait is bounded nonetheless)
  uint32_t excl = 0;
  if (digit_thread && tile > 0) {
    int64_t j = tile - 1;
    int spins = 0;
    bool done = false;
    while (!done) {
      uint32_t v[LOOKBACK_BATCH];
#pragma unroll
      for (int k = 0; k < LOOKBACK_BATCH; ++k)
        v[k] = j - k >= 0 ? ld_relaxed_u32(slots + (j - k) * RADIX + t) : 0u;
      bool stall = false;
#pragma unroll
      for (int k = 0; k < LOOKBACK_BATCH; ++k) {
        if (done || stall) continue;
        const uint32_t state = v[k] & SLOT_STATE;
        if (state == 0u) {
          stall = true;
          continue;
        }
        excl += v[k] & SLOT_VALUE;
        if (state == SLOT_PRE || j == 0) done = true;
        else --j;
      }
      if (stall && ++spins > LOOKBACK_MAX_SPINS) {
        atomicOr(status, (unsigned)ST_ERR_SORT);
        break;
      }
    }
    st_relaxed_u32(slots + tile * RADIX + t, SLOT_PRE | (excl + cnt));
  }
  // output place of tile place i with digit t: keys of smaller digits, the
  // earlier tiles' keys of digit t, then i's place within the digit's run
  if (digit_thread) s_off[t] = (int32_t)(ig + excl) - (int32_t)s_tstart[t];
  __syncthreads();

  // 5. scatter (stable: warp, then round, then lane is the input order);
  //    consecutive threads write consecutive places of a digit's run
  for (int i = t; i < tn; i += PASS_THREADS) {
    const uint32_t k = s_cnt_key[i];
    const int64_t pos = (int64_t)s_off[(k >> shift) & 255u] + i;
    if (pos >= 0 && pos < n) {
      keys_out[pos] = k;
      vals_out[pos] = s_val[i];
    }
  }
}

}  // namespace

// 8-bit digit passes for a key width: an odd count leaves the result in the
// alternate buffers (the caller then starts from them, see sort_passes' users)
int sort_passes(int key_bits) {
  int passes = (key_bits + 7) / 8;
  if (passes > MAX_PASSES) passes = MAX_PASSES;
  return passes;
}

size_t radix_sort_temp_bytes(int64_t n) {
  const int64_t tiles = (n + OS_TILE - 1) / OS_TILE;
  return (size_t)(HEAD_WORDS + (int64_t)MAX_PASSES * tiles * RADIX) * sizeof(uint32_t);
}

// Sorts (keys, vals) by the low `key_bits` bits of the keys in
// sort_passes(key_bits) passes; the result is left in (keys, vals) after an
// even number of passes and in (keys_alt, vals_alt) after an odd number.
// keys_alt / vals_alt are scratch of n entries;
// n < 2^30.  A look-back that gives up sets ST_ERR_SORT in *status (the
// order is then not valid; every index written stays below n).
int radix_sort_pairs(uint32_t* keys, int32_t* vals, uint32_t* keys_alt, int32_t* vals_alt,
                     int64_t n, int key_bits, void* temp, unsigned* status, cudaStream_t s) {
  if (n <= 1) return 0;
  const int tiles = (int)((n + OS_TILE - 1) / OS_TILE);
  int passes = sort_passes(key_bits);
  uint32_t* counts = (uint32_t*)temp;
  uint32_t* tile_ctr = counts + MAX_PASSES * RADIX;
  uint32_t* slots = counts + HEAD_WORDS;
  if (cudaMemsetAsync(counts, 0, HEAD_WORDS * sizeof(uint32_t), s) != cudaSuccess) return -1;
  os_hist_kernel<<<tiles, OS_THREADS, 0, s>>>(keys, n, passes, counts, slots, tiles);
  uint32_t* kin = keys;
  int32_t* vin = vals;
  uint32_t* kout = keys_alt;
  int32_t* vout = vals_alt;
  for (int p = 0; p < passes; ++p) {
    os_pass_kernel<<<tiles, PASS_THREADS, 0, s>>>(kin, vin, kout, vout, n, p, counts, tile_ctr,
                                                slots + (int64_t)p * tiles * RADIX, status);
    uint32_t* tk = kin; kin = kout; kout = tk;
    int32_t* tv = vin; vin = vout; vout = tv;
  }
  return 1 + passes;
}

}  // namespace sidm
