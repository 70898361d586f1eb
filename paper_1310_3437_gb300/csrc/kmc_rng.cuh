// kmc_rng.cuh -- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and the map of a
// 32-bit word to a uniform in [-1, 1), shared by the collision update and the
// device-side initial states.
#pragma once
#include <cstdint>

namespace kmc {

// ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) ---------------------- //
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
    uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
    uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// u = w 2^-31 - 1 for a 32-bit word w, built with integer operations: the value is
// (w - 2^31) 2^-31 exactly (32 significant bits at most), so the bits equal those of
// the binary64 expression, without its conversion, product and difference on the
// binary64 pipe.
__device__ __forceinline__ double word_uniform(uint32_t w) {
  const long long m = (long long)w - 2147483648ll;
  if (m == 0) return 0.0;
  const unsigned long long neg = m < 0 ? 1ull : 0ull;
  const unsigned long long a = (unsigned long long)(m < 0 ? -m : m);  // 1 .. 2^31
  const int e = 63 - __clzll((long long)a);
  const unsigned long long mant = (a << (52 - e)) & 0xFFFFFFFFFFFFFull;
  return __longlong_as_double((long long)((neg << 63) | ((unsigned long long)(1023 + e - 31) << 52) | mant));
}

}  // namespace kmc
