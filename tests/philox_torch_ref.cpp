// Reads (key0 key1 c0 c1 c2 c3) lines on stdin and prints the four output
// words of PyTorch's header-only at::philox_engine for the same key and
// counter: an implementation of Philox-4x32-10 independent of the oracle's.
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
#include <cinttypes>

int main() {
  unsigned long long k0, k1, c0, c1, c2, c3;
  while (std::scanf("%llu %llu %llu %llu %llu %llu", &k0, &k1, &c0, &c1, &c2, &c3) == 6) {
    const uint64_t seed = (uint64_t)k0 | ((uint64_t)k1 << 32);
    const uint64_t subseq = (uint64_t)c2 | ((uint64_t)c3 << 32);
    const uint64_t offset = (uint64_t)c0 | ((uint64_t)c1 << 32);
    at::philox_engine eng(seed, subseq, offset);
    const uint32_t w0 = eng(), w1 = eng(), w2 = eng(), w3 = eng();
    std::printf("%u %u %u %u\n", w0, w1, w2, w3);
  }
  return 0;
}
