// Fused-gate application (Alg. 1, Sec. III.A) on a complex64 state.
//
// The state is 2^n interleaved (re, im) float pairs.  A k-qubit fused gate
// splits it into 2^(n-k) gather sets of 2^k amplitudes (the set's base
// index with every combination of the target bits).  One thread owns one
// set -- or, when qubit 0 is not a target, the two neighbouring sets that
// differ only in bit 0, so that each member is one 128-bit load of two
// adjacent amplitudes.  Consecutive threads own consecutive bases, so every
// warp-wide load or store covers whole 128-byte lines however high the
// target qubits are; low target qubits spread a warp's accesses over a few
// more lines that the same warp reads or writes in its other members, so
// DRAM still sees every byte once.
//
// The matrix is a __grid_constant__ kernel parameter: with the loops over
// rows and columns fully unrolled every matrix element is a constant-bank
// operand of the FMA that uses it, so the inner product costs 4 FFMA per
// complex multiply-add and no load instructions.  Each output row is stored
// as soon as it is complete (all inputs are already in registers).
//
// Bytes per launch: 16 * 2^n (every amplitude read once and written once).
// FLOPs per launch: 2^(k+2) * 2^(n+1) (the paper's count); at k <= 4 the
// FMA rate needed at full HBM bandwidth stays below the CUDA-core peak.
#include <cuda_runtime.h>

#include <mutex>

#include "kernels.h"

namespace qt {

template <int K>
struct ApplyArgs {
  float2 u[1 << K][1 << K];     // row-major gate matrix
  uint64_t offs[1 << K];        // amplitude offset of member m within a set
  uint32_t ins[K + 1];          // ascending bit positions to insert zeros at
  uint64_t num_sets;            // sets (or set pairs) to process
};

template <int K, bool PAIR>
__global__ void __launch_bounds__(256) k_apply(float2* __restrict__ psi,
                                               const __grid_constant__ ApplyArgs<K> a) {
  constexpr int M = 1 << K;
  constexpr int NI = PAIR ? K + 1 : K;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < a.num_sets;
       i += stride) {
    uint64_t base = i;
#pragma unroll
    for (int b = 0; b < NI; ++b) {
      const uint32_t s = a.ins[b];
      base = ((base >> s) << (s + 1)) | (base & ((1ull << s) - 1ull));
    }
    if constexpr (PAIR) {
      float4 v[M];
#pragma unroll
      for (int m = 0; m < M; ++m) v[m] = __ldcs(reinterpret_cast<const float4*>(psi + base + a.offs[m]));
#pragma unroll
      for (int j = 0; j < M; ++j) {
        float xr = 0.f, xi = 0.f, yr = 0.f, yi = 0.f;
#pragma unroll
        for (int m = 0; m < M; ++m) {
          const float ur = a.u[j][m].x, ui = a.u[j][m].y;
          xr = fmaf(ur, v[m].x, xr);
          xr = fmaf(-ui, v[m].y, xr);
          xi = fmaf(ur, v[m].y, xi);
          xi = fmaf(ui, v[m].x, xi);
          yr = fmaf(ur, v[m].z, yr);
          yr = fmaf(-ui, v[m].w, yr);
          yi = fmaf(ur, v[m].w, yi);
          yi = fmaf(ui, v[m].z, yi);
        }
        __stcs(reinterpret_cast<float4*>(psi + base + a.offs[j]), make_float4(xr, xi, yr, yi));
      }
    } else {
      float2 v[M];
#pragma unroll
      for (int m = 0; m < M; ++m) v[m] = __ldcs(psi + base + a.offs[m]);
#pragma unroll
      for (int j = 0; j < M; ++j) {
        float xr = 0.f, xi = 0.f;
#pragma unroll
        for (int m = 0; m < M; ++m) {
          const float ur = a.u[j][m].x, ui = a.u[j][m].y;
          xr = fmaf(ur, v[m].x, xr);
          xr = fmaf(-ui, v[m].y, xr);
          xi = fmaf(ur, v[m].y, xi);
          xi = fmaf(ui, v[m].x, xi);
        }
        __stcs(psi + base + a.offs[j], make_float2(xr, xi));
      }
    }
  }
}

static int g_sms = 0;
int sm_count() {
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_sms <= 0) g_sms = 1;
  });
  return g_sms;
}

template <int K, bool PAIR>
static cudaError_t launch_k(float2* psi, int n, const uint32_t* targets, const float2* U,
                            cudaStream_t st) {
  static int occ = 0;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_apply<K, PAIR>, 256, 0);
    if (occ <= 0) occ = 1;
  });
  ApplyArgs<K> a;
  constexpr int M = 1 << K;
  for (int j = 0; j < M; ++j)
    for (int m = 0; m < M; ++m) a.u[j][m] = U[j * M + m];
  for (int m = 0; m < M; ++m) {
    uint64_t o = 0;
    for (int b = 0; b < K; ++b)
      if ((m >> b) & 1) o |= 1ull << targets[b];
    a.offs[m] = o;
  }
  int ni = 0;
  if (PAIR) a.ins[ni++] = 0;
  for (int b = 0; b < K; ++b) a.ins[ni++] = targets[b];
  a.num_sets = 1ull << (n - K - (PAIR ? 1 : 0));
  const uint64_t want = (a.num_sets + 255) / 256;
  const uint64_t cap = static_cast<uint64_t>(sm_count()) * occ;
  const unsigned grid = static_cast<unsigned>(want < cap ? want : cap);
  k_apply<K, PAIR><<<grid, 256, 0, st>>>(psi, a);
  return cudaGetLastError();
}

cudaError_t launch_apply(float2* psi, int n, int k, const uint32_t* targets, const float2* U,
                         cudaStream_t st) {
  // targets ascending; pair mode needs qubit 0 free and at least one spare bit
  const bool pair = (targets[0] != 0) && (n >= k + 1);
  switch (k) {
    case 1: return pair ? launch_k<1, true>(psi, n, targets, U, st) : launch_k<1, false>(psi, n, targets, U, st);
    case 2: return pair ? launch_k<2, true>(psi, n, targets, U, st) : launch_k<2, false>(psi, n, targets, U, st);
    case 3: return pair ? launch_k<3, true>(psi, n, targets, U, st) : launch_k<3, false>(psi, n, targets, U, st);
    case 4: return pair ? launch_k<4, true>(psi, n, targets, U, st) : launch_k<4, false>(psi, n, targets, U, st);
    case 5: return launch_k<5, false>(psi, n, targets, U, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace qt
