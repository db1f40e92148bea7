// Counter-based random numbers for the trajectory draws: Philox4x32-10
// (J. Salmon, M. Moraes, R. Dror, D. Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC'11).  Shared by the host controller and the device kernels
// so that a draw depends only on (seed, trajectory, stream, index).
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define QT_HD __host__ __device__ __forceinline__
#else
#define QT_HD inline
#endif

namespace qt {

struct U32x4 { uint32_t v[4]; };

QT_HD U32x4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                          uint32_t k0, uint32_t k1) {
  // ten rounds; each round multiplies lanes 0 and 2 by the Philox constants,
  // swaps the high halves across, xors in the round key and bumps the key by
  // the Weyl increments (golden ratio, sqrt(3) - 1)
#if defined(__CUDACC__)
#pragma unroll
#endif
  for (int r = 0; r < 10; ++r) {
    const uint64_t m0 = static_cast<uint64_t>(c0) * 0xD2511F53ull;
    const uint64_t m1 = static_cast<uint64_t>(c2) * 0xCD9E8D57ull;
    const uint32_t n0 = static_cast<uint32_t>(m1 >> 32) ^ c1 ^ k0;
    const uint32_t n2 = static_cast<uint32_t>(m0 >> 32) ^ c3 ^ k1;
    c1 = static_cast<uint32_t>(m1);
    c3 = static_cast<uint32_t>(m0);
    c0 = n0;
    c2 = n2;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  U32x4 o;
  o.v[0] = c0; o.v[1] = c1; o.v[2] = c2; o.v[3] = c3;
  return o;
}

// Uniform double in [0, 1) with 53 random bits: the top 27 bits of word 0
// and the top 26 bits of word 1.
QT_HD double uniform01(uint64_t seed, uint64_t traj, uint32_t stream, uint32_t index) {
  const U32x4 w = philox4x32_10(static_cast<uint32_t>(traj), static_cast<uint32_t>(traj >> 32),
                                stream, index, static_cast<uint32_t>(seed),
                                static_cast<uint32_t>(seed >> 32));
  const uint64_t bits = (static_cast<uint64_t>(w.v[0] >> 5) << 26) | (w.v[1] >> 6);
  return static_cast<double>(bits) * 0x1.0p-53;
}

enum : uint32_t { kStreamChannel = 0, kStreamSample = 1, kStreamReadout = 2 };

}  // namespace qt
