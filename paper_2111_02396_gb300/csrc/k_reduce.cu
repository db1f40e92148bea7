// Read-only passes over the state: branch probabilities (Alg. 2 step 14),
// Z-string expectations and bitstring sampling, plus state init / scale.
//
// Precision: products are formed in FP32 from the complex64 state; partial
// sums over a short run of terms stay in FP32 and are then carried in FP64
// (FP64 throughput on this part is low, so it is used only at that coarse
// grain).  Every reduction has a fixed grid and a fixed combination order,
// so results are bitwise reproducible run to run.
#include <cuda_runtime.h>

#include <mutex>

#include "kernels.h"
#include "qt_philox.h"

namespace qt {

size_t scratch_partial_bytes() { return sizeof(double) * kMaxRedBlocks * 64; }

// ---------------------------------------------------------------------------
// block-wide FP64 reduction of W per-thread values into partial[block][W]
// ---------------------------------------------------------------------------
template <int W>
__device__ __forceinline__ void block_reduce_store(double (&acc)[W], double* __restrict__ partial) {
  __shared__ double sm[kRedThreads / 32][W];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < W; ++c) {
    double v = acc[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sm[warp][c] = v;
  }
  __syncthreads();
  const int nw = static_cast<int>(blockDim.x >> 5);   // blocks of at most kRedThreads threads
  for (int c = threadIdx.x; c < W; c += blockDim.x) {
    double v = 0.0;
    for (int w = 0; w < nw; ++w) v += sm[w][c];
    partial[static_cast<size_t>(blockIdx.x) * W + c] = v;
  }
}

__global__ void k_finalize(const double* __restrict__ partial, int nblocks, int W,
                           double* __restrict__ out) {
  for (int c = threadIdx.x; c < W; c += blockDim.x) {
    double v = 0.0;
    for (int b = 0; b < nblocks; ++b) v += partial[static_cast<size_t>(b) * W + c];
    out[c] = v;
  }
}

template <typename Kern>
static int red_grid(Kern kern, uint64_t work_items) {
  // one full wave of resident blocks, capped by the work and by the scratch
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kRedThreads, 0);
  if (occ <= 0) occ = 1;
  uint64_t g = static_cast<uint64_t>(sm_count()) * occ;
  const uint64_t need = (work_items + kRedThreads - 1) / kRedThreads;
  if (g > need) g = need;
  if (g > static_cast<uint64_t>(kMaxRedBlocks)) g = kMaxRedBlocks;
  if (g < 1) g = 1;
  return static_cast<int>(g);
}

// ---------------------------------------------------------------------------
// Reduced density block of qubits Q: rho[b][a] = sum_rest psi[rest,b] conj(psi[rest,a]).
// W = 4^q reals: the 2^q diagonal entries, then (re, im) of each b < a.
// ---------------------------------------------------------------------------
template <int Q>
struct RdmArgs {
  uint64_t offs[1 << Q];
  uint32_t ins[Q];
  uint64_t num_sets;
};

constexpr int kRdmChunk = 16;   // sets summed in FP32 before the FP64 carry

template <int Q>
__global__ void __launch_bounds__(kRedThreads) k_rdm(const float2* __restrict__ psi,
                                                     const __grid_constant__ RdmArgs<Q> a,
                                                     double* __restrict__ partial) {
  constexpr int D = 1 << Q, W = D * D;
  double acc[W];
  float f[W];
#pragma unroll
  for (int c = 0; c < W; ++c) { acc[c] = 0.0; f[c] = 0.f; }
  int cnt = 0;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < a.num_sets;
       i += stride) {
    uint64_t base = i;
#pragma unroll
    for (int b = 0; b < Q; ++b) {
      const uint32_t s = a.ins[b];
      base = ((base >> s) << (s + 1)) | (base & ((1ull << s) - 1ull));
    }
    float2 v[D];
#pragma unroll
    for (int m = 0; m < D; ++m) v[m] = __ldg(psi + base + a.offs[m]);
    int c = 0;
#pragma unroll
    for (int b = 0; b < D; ++b) { f[c] = fmaf(v[b].x, v[b].x, fmaf(v[b].y, v[b].y, f[c])); ++c; }
#pragma unroll
    for (int b = 0; b < D; ++b)
#pragma unroll
      for (int aa = b + 1; aa < D; ++aa) {
        // v_b conj(v_a)
        f[c] = fmaf(v[b].x, v[aa].x, fmaf(v[b].y, v[aa].y, f[c])); ++c;
        f[c] = fmaf(v[b].y, v[aa].x, fmaf(-v[b].x, v[aa].y, f[c])); ++c;
      }
    if (++cnt == kRdmChunk) {
#pragma unroll
      for (int k = 0; k < W; ++k) { acc[k] += static_cast<double>(f[k]); f[k] = 0.f; }
      cnt = 0;
    }
  }
#pragma unroll
  for (int k = 0; k < W; ++k) acc[k] += static_cast<double>(f[k]);
  block_reduce_store<W>(acc, partial);
}

template <int Q>
static cudaError_t rdm_q(const float2* psi, int n, const uint32_t* qubits, const Scratch& scr,
                         cudaStream_t st) {
  RdmArgs<Q> a;
  uint32_t s[Q];
  for (int b = 0; b < Q; ++b) s[b] = qubits[b];
  for (int i = 1; i < Q; ++i)
    for (int j = i; j > 0 && s[j - 1] > s[j]; --j) { const uint32_t t = s[j]; s[j] = s[j - 1]; s[j - 1] = t; }
  for (int b = 0; b < Q; ++b) a.ins[b] = s[b];
  for (int m = 0; m < (1 << Q); ++m) {
    uint64_t o = 0;
    for (int b = 0; b < Q; ++b)
      if ((m >> b) & 1) o |= 1ull << qubits[b];
    a.offs[m] = o;
  }
  a.num_sets = 1ull << (n - Q);
  static PerDevice grid_dev;
  const int grid = grid_dev.get([] { return red_grid(k_rdm<Q>, ~0ull >> 1); });
  const uint64_t need = (a.num_sets + kRedThreads - 1) / kRedThreads;
  const int g = static_cast<int>(need < static_cast<uint64_t>(grid) ? need : grid);
  k_rdm<Q><<<g, kRedThreads, 0, st>>>(psi, a, scr.partial);
  k_finalize<<<1, 64, 0, st>>>(scr.partial, g, 1 << (2 * Q), scr.result);
  return cudaGetLastError();
}

cudaError_t launch_rdm(const float2* psi, int n, int q, const uint32_t* qubits, const Scratch& scr,
                       cudaStream_t st) {
  if (q > n) return cudaErrorInvalidValue;
  switch (q) {
    case 1: return rdm_q<1>(psi, n, qubits, scr, st);
    case 2: return rdm_q<2>(psi, n, qubits, scr, st);
    case 3: return rdm_q<3>(psi, n, qubits, scr, st);
    default: return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------------------
// Branch probabilities of a channel on 4..6 qubits (Alg. 2 step 14): for G
// Kraus operators at a time, P_i = <psi|K_i^dag K_i|psi> = sum over gather
// sets of |K_i v|^2, plus N = <psi|psi> (the 4^q-entry reduced density of
// these widths would not fit in registers).  Each thread takes whole gather
// sets; its set is staged column-wise in shared memory (member m of thread t
// at v[m * blockDim + t], conflict-free) and the G operators sit in shared
// memory.  Products and row sums in FP32; runs of kKrausChunk sets in FP32,
// carried in FP64; fixed grid and reduction order.
// result[0] = N, result[1 + i] = P_i.
// ---------------------------------------------------------------------------
constexpr int kKrausThreads = 128;
constexpr int kKrausChunk = 16;

template <int Q>
struct KrausArgs {
  uint64_t offs[1 << Q];
  uint32_t ins[Q];
  uint64_t num_sets;
  const float2* ops;            // G matrices 2^Q x 2^Q, row-major (basis bit b <-> qubits[b])
};

template <int Q, int G>
__global__ void __launch_bounds__(kKrausThreads) k_kraus_norms(const float2* __restrict__ psi,
                                                               const __grid_constant__ KrausArgs<Q> a,
                                                               double* __restrict__ partial) {
  constexpr int D = 1 << Q, W = G + 1;
  extern __shared__ __align__(16) float2 s_dyn[];
  float2* sK = s_dyn;                          // G * D * D
  float2* sv = s_dyn + G * D * D;              // D * blockDim
  for (int i = threadIdx.x; i < G * D * D; i += blockDim.x) sK[i] = a.ops[i];
  __syncthreads();
  double acc[W];
  float f[W];
#pragma unroll
  for (int c = 0; c < W; ++c) { acc[c] = 0.0; f[c] = 0.f; }
  int cnt = 0;
  const int t = threadIdx.x, bd = blockDim.x;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < a.num_sets;
       i += stride) {
    uint64_t base = i;
#pragma unroll
    for (int b = 0; b < Q; ++b) {
      const uint32_t s = a.ins[b];
      base = ((base >> s) << (s + 1)) | (base & ((1ull << s) - 1ull));
    }
    for (int m = 0; m < D; ++m) {
      const float2 v = __ldg(psi + base + a.offs[m]);
      sv[m * bd + t] = v;
      f[0] = fmaf(v.x, v.x, fmaf(v.y, v.y, f[0]));
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const float2* K = sK + g * D * D;
      float row = 0.f;
      for (int j = 0; j < D; ++j) {
        float wr = 0.f, wi = 0.f;
#pragma unroll 8
        for (int m = 0; m < D; ++m) {
          const float2 k = K[j * D + m];
          const float2 v = sv[m * bd + t];
          wr = fmaf(k.x, v.x, fmaf(-k.y, v.y, wr));
          wi = fmaf(k.x, v.y, fmaf(k.y, v.x, wi));
        }
        row = fmaf(wr, wr, fmaf(wi, wi, row));
      }
      f[1 + g] += row;
    }
    if (++cnt == kKrausChunk) {
#pragma unroll
      for (int k = 0; k < W; ++k) { acc[k] += static_cast<double>(f[k]); f[k] = 0.f; }
      cnt = 0;
    }
  }
#pragma unroll
  for (int k = 0; k < W; ++k) acc[k] += static_cast<double>(f[k]);
  block_reduce_store<W>(acc, partial);
}

template <int Q, int G>
static cudaError_t kraus_norms_q(const float2* psi, int n, const uint32_t* qubits, const float2* ops_dev,
                                 const Scratch& scr, cudaStream_t st) {
  constexpr int D = 1 << Q;
  KrausArgs<Q> a;
  uint32_t s[Q];
  for (int b = 0; b < Q; ++b) s[b] = qubits[b];
  for (int i = 1; i < Q; ++i)
    for (int j = i; j > 0 && s[j - 1] > s[j]; --j) { const uint32_t t = s[j]; s[j] = s[j - 1]; s[j - 1] = t; }
  for (int b = 0; b < Q; ++b) a.ins[b] = s[b];
  for (int m = 0; m < D; ++m) {
    uint64_t o = 0;
    for (int b = 0; b < Q; ++b)
      if ((m >> b) & 1) o |= 1ull << qubits[b];
    a.offs[m] = o;
  }
  a.num_sets = 1ull << (n - Q);
  a.ops = ops_dev;
  const size_t smem = sizeof(float2) * (static_cast<size_t>(G) * D * D + static_cast<size_t>(D) * kKrausThreads);
  static PerDevice setup;
  const int grid = setup.get([smem] {
    if (cudaFuncSetAttribute(k_kraus_norms<Q, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem)) != cudaSuccess)
      return 0;
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_kraus_norms<Q, G>, kKrausThreads, smem);
    const int g = sm_count() * (occ > 0 ? occ : 1);
    return g < kMaxRedBlocks ? g : kMaxRedBlocks;
  });
  if (grid <= 0) return cudaErrorInvalidConfiguration;
  const uint64_t need = (a.num_sets + kKrausThreads - 1) / kKrausThreads;
  const int g = static_cast<int>(need < static_cast<uint64_t>(grid) ? need : grid);
  k_kraus_norms<Q, G><<<g, kKrausThreads, smem, st>>>(psi, a, scr.partial);
  k_finalize<<<1, 64, 0, st>>>(scr.partial, g, G + 1, scr.result);
  return cudaGetLastError();
}

int kraus_group(int q) { return q <= 4 ? 16 : (q == 5 ? 4 : 1); }

cudaError_t launch_kraus_norms(const float2* psi, int n, int q, const uint32_t* qubits, int nops,
                               const float2* ops_dev, const Scratch& scr, cudaStream_t st) {
  if (q > n || nops != kraus_group(q)) return cudaErrorInvalidValue;
  switch (q) {
    case 4: return kraus_norms_q<4, 16>(psi, n, qubits, ops_dev, scr, st);
    case 5: return kraus_norms_q<5, 4>(psi, n, qubits, ops_dev, scr, st);
    case 6: return kraus_norms_q<6, 1>(psi, n, qubits, ops_dev, scr, st);
    default: return cudaErrorInvalidValue;
  }
}

void rdm_unpack(int q, const double* r, double* rho) {
  const int D = 1 << q;
  int c = 0;
  for (int b = 0; b < D; ++b) {
    rho[2 * (b * D + b)] = r[c++];
    rho[2 * (b * D + b) + 1] = 0.0;
  }
  for (int b = 0; b < D; ++b)
    for (int a = b + 1; a < D; ++a) {
      const double re = r[c++], im = r[c++];
      rho[2 * (b * D + a)] = re;        // rho[b][a] = sum psi_b conj(psi_a)
      rho[2 * (b * D + a) + 1] = im;
      rho[2 * (a * D + b)] = re;        // Hermitian
      rho[2 * (a * D + b) + 1] = -im;
    }
}

// ---------------------------------------------------------------------------
// Z-string expectations: result[0] = N, result[1+m] = sum_x |psi_x|^2 (-1)^popc(x & mask_m)
// ---------------------------------------------------------------------------
struct ExpArgs {
  uint64_t masks[kExpGroup];
  int nm;
  uint64_t num_pairs;
};

constexpr int kExpChunk = 64;

__global__ void __launch_bounds__(kRedThreads) k_expect(const float2* __restrict__ psi,
                                                        const __grid_constant__ ExpArgs a,
                                                        double* __restrict__ partial) {
  constexpr int W = kExpGroup + 1;
  double acc[W];
  float f[W];
#pragma unroll
  for (int c = 0; c < W; ++c) { acc[c] = 0.0; f[c] = 0.f; }
  int cnt = 0;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < a.num_pairs;
       i += stride) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(psi) + i);
    const float w0 = fmaf(v.x, v.x, v.y * v.y), w1 = fmaf(v.z, v.z, v.w * v.w);
    const uint64_t x0 = 2 * i;
    f[0] += w0 + w1;
#pragma unroll
    for (int m = 0; m < kExpGroup; ++m) {
      if (m < a.nm) {
        const uint64_t mk = a.masks[m];
        const int s0 = __popcll(x0 & mk) & 1;
        const int s1 = s0 ^ static_cast<int>(mk & 1ull);
        f[1 + m] += (s0 ? -w0 : w0) + (s1 ? -w1 : w1);
      }
    }
    if (++cnt == kExpChunk) {
#pragma unroll
      for (int k = 0; k < W; ++k) { acc[k] += static_cast<double>(f[k]); f[k] = 0.f; }
      cnt = 0;
    }
  }
#pragma unroll
  for (int k = 0; k < W; ++k) acc[k] += static_cast<double>(f[k]);
  block_reduce_store<W>(acc, partial);
}

// n >= 9: a warp takes blocks of 512 amplitudes and lane l holds the 16
// amplitudes x = (blk << 9) | (j << 6) | (l << 1) | e, j = 0..7, e = 0..1,
// read with eight coalesced 128-bit loads.  Over the bits that vary inside
// the thread (0, 6, 7, 8) its 16 weights are Walsh-Hadamard transformed,
//   W[u] = sum_v (-1)^popc(u & v) w[v],   v = e | (j << 1),
// so that the block's share of sum_x |psi_x|^2 (-1)^popc(x & m) is
// (-1)^(parity of m on the fixed bits) * W[u_m], u_m being m's bits 0, 6, 7,
// 8.  The parity over the lane bits (1..5) is fixed per thread and the one
// over the block bits (>= 9) is one popc, so a mask costs a few instructions
// per 16 amplitudes.  FP32 runs cover 8 blocks (128 amplitudes per thread),
// then FP64.
struct ExpWArgs {
  uint32_t mblk[kExpGroup];     // mask bits >= 9, shifted down by 9
  uint32_t mlane[kExpGroup];    // mask bits 1..5, shifted down by 1
  uint32_t u[kExpGroup];        // mask bits (0, 6, 7, 8) as a 4-bit index
  int nm;
  uint64_t num_blocks;          // 2^(n - 9)
};

constexpr int kExpWChunk = 8;

__global__ void __launch_bounds__(kRedThreads) k_expect_wht(const float2* __restrict__ psi,
                                                            const __grid_constant__ ExpWArgs a,
                                                            double* __restrict__ partial) {
  constexpr int W = kExpGroup + 1;
  __shared__ float s_w[kRedThreads][17];        // each thread's transformed weights (padded row)
  double acc[W];
  float f[W];
#pragma unroll
  for (int c = 0; c < W; ++c) { acc[c] = 0.0; f[c] = 0.f; }
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t warp = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
  uint32_t slane = 0;                           // bit m: parity of mask m on the lane bits
  for (int m = 0; m < a.nm; ++m) slane |= (static_cast<uint32_t>(__popc(lane & a.mlane[m])) & 1u) << m;
  const float4* p4 = reinterpret_cast<const float4*>(psi);
  float* row = s_w[threadIdx.x];
  int cnt = 0;
  for (uint64_t blk = warp; blk < a.num_blocks; blk += nwarps) {
    float w[16];
    float4 q[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) q[j] = __ldg(p4 + (blk << 8) + j * 32 + lane);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      w[2 * j] = fmaf(q[j].x, q[j].x, q[j].y * q[j].y);
      w[2 * j + 1] = fmaf(q[j].z, q[j].z, q[j].w * q[j].w);
    }
    if (a.nm > 0) {
#pragma unroll
      for (int h = 1; h < 16; h <<= 1)
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if ((i & h) == 0) {
            const float x = w[i], y = w[i | h];
            w[i] = x + y;
            w[i | h] = x - y;
          }
      f[0] += w[0];
#pragma unroll
      for (int u = 0; u < 16; ++u) row[u] = w[u];
      const uint32_t b32 = static_cast<uint32_t>(blk);
#pragma unroll
      for (int m = 0; m < kExpGroup; ++m) {
        if (m < a.nm) {
          const float val = row[a.u[m]];
          const uint32_t sgn = (static_cast<uint32_t>(__popc(b32 & a.mblk[m])) ^ (slane >> m)) & 1u;
          f[1 + m] += sgn ? -val : val;
        }
      }
    } else {
      float t = 0.f;
#pragma unroll
      for (int v = 0; v < 16; ++v) t += w[v];
      f[0] += t;
    }
    if (++cnt == kExpWChunk) {
#pragma unroll
      for (int k = 0; k < W; ++k) { acc[k] += static_cast<double>(f[k]); f[k] = 0.f; }
      cnt = 0;
    }
  }
#pragma unroll
  for (int k = 0; k < W; ++k) acc[k] += static_cast<double>(f[k]);
  block_reduce_store<W>(acc, partial);
}

cudaError_t launch_expect(const float2* psi, int n, int nm, const uint64_t* masks,
                          const Scratch& scr, cudaStream_t st) {
  if (nm > kExpGroup || n < 1) return cudaErrorInvalidValue;
  if (n >= 9) {
    ExpWArgs a;
    for (int m = 0; m < kExpGroup; ++m) {
      const uint64_t mk = m < nm ? masks[m] : 0;
      a.mblk[m] = static_cast<uint32_t>(mk >> 9);
      a.mlane[m] = static_cast<uint32_t>((mk >> 1) & 31u);
      a.u[m] = static_cast<uint32_t>((mk & 1u) | (((mk >> 6) & 7u) << 1));
    }
    a.nm = nm;
    a.num_blocks = 1ull << (n - 9);
    static PerDevice gridw_dev;
    const int gridw = gridw_dev.get([] { return red_grid(k_expect_wht, ~0ull >> 1); });
    const uint64_t need = (a.num_blocks * 32 + kRedThreads - 1) / kRedThreads;
    const int g = static_cast<int>(need < static_cast<uint64_t>(gridw) ? need : gridw);
    k_expect_wht<<<g, kRedThreads, 0, st>>>(psi, a, scr.partial);
    k_finalize<<<1, 64, 0, st>>>(scr.partial, g, kExpGroup + 1, scr.result);
    return cudaGetLastError();
  }
  ExpArgs a;
  for (int m = 0; m < kExpGroup; ++m) a.masks[m] = m < nm ? masks[m] : 0;
  a.nm = nm;
  a.num_pairs = 1ull << (n - 1);
  static PerDevice grid_dev;
  const int grid = grid_dev.get([] { return red_grid(k_expect, ~0ull >> 1); });
  const uint64_t need = (a.num_pairs + kRedThreads - 1) / kRedThreads;
  const int g = static_cast<int>(need < static_cast<uint64_t>(grid) ? need : grid);
  k_expect<<<g, kRedThreads, 0, st>>>(psi, a, scr.partial);
  k_finalize<<<1, 64, 0, st>>>(scr.partial, g, kExpGroup + 1, scr.result);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Sampling.  C(x) is built in three levels with one fixed arithmetic, used
// both to build the block table and to search inside a block, so that the
// search sees the same cumulative values the table was built from:
//   chunk      64 amplitudes, warp inclusive scan in FP32 of (|a0|^2+|a1|^2)
//   sub-block  16 chunks, running FP32 sum of chunk totals  -> cdf_sub
//   block      64 sub-blocks, warp inclusive scan in FP64   -> block totals
//   table      inclusive FP64 scan of the block totals      -> cdf_cum
// A sample with uniform u targets t = u * C(2^n - 1) and returns the
// smallest x with t < C(x).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_incl_scan_f(float v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  return v;
}

__device__ __forceinline__ double warp_incl_scan_d(double v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  return v;
}

// weights of the two amplitudes a lane owns in a chunk (0 past the end)
__device__ __forceinline__ void chunk_weights(const float2* __restrict__ psi, uint64_t namps,
                                              uint64_t x0, float& w0, float& w1) {
  w0 = 0.f;
  w1 = 0.f;
  if (x0 < namps) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(psi + x0));
    w0 = fmaf(v.x, v.x, v.y * v.y);
    w1 = fmaf(v.z, v.z, v.w * v.w);
  }
}

__global__ void k_cdf_sub(const float2* __restrict__ psi, uint64_t namps, uint64_t nsub,
                          float* __restrict__ sub) {
  const int lane = threadIdx.x & 31;
  const uint64_t warp = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
  for (uint64_t s = warp; s < nsub; s += nwarps) {
    float run = 0.f;
    for (int c = 0; c < (1 << (kCdfSubLog - kCdfChunkLog)); ++c) {
      const uint64_t x0 = (s << kCdfSubLog) + (static_cast<uint64_t>(c) << kCdfChunkLog) + 2 * lane;
      float w0, w1;
      chunk_weights(psi, namps, x0, w0, w1);
      const float incl = warp_incl_scan_f(w0 + w1, lane);
      run += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) sub[s] = run;
  }
}

// lane values of block b: (double)sub[2L] + (double)sub[2L+1]
__device__ __forceinline__ void block_lane_values(const float* __restrict__ sub, uint64_t nsub,
                                                  uint64_t b, int lane, double& s0, double& s1) {
  const uint64_t i0 = (b << 6) + 2 * lane;
  s0 = i0 < nsub ? static_cast<double>(sub[i0]) : 0.0;
  s1 = i0 + 1 < nsub ? static_cast<double>(sub[i0 + 1]) : 0.0;
}

__global__ void k_cdf_blk(const float* __restrict__ sub, uint64_t nsub, uint64_t nblk,
                          double* __restrict__ cum) {
  const int lane = threadIdx.x & 31;
  const uint64_t warp = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
  for (uint64_t b = warp; b < nblk; b += nwarps) {
    double s0, s1;
    block_lane_values(sub, nsub, b, lane, s0, s1);
    const double incl = warp_incl_scan_d(s0 + s1, lane);
    if (lane == 31) cum[b] = incl;
  }
}

// in-place inclusive scan of nblk doubles by one block of 1024 threads
__global__ void __launch_bounds__(1024) k_cdf_scan(double* __restrict__ cum, uint64_t nblk) {
  __shared__ double tot[1024];
  const uint64_t per = (nblk + 1023) / 1024;
  const uint64_t lo = threadIdx.x * per;
  const uint64_t hi = lo + per < nblk ? lo + per : nblk;
  double s = 0.0;
  for (uint64_t i = lo; i < hi; ++i) s += cum[i];
  tot[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int t = 0; t < 1024; ++t) { const double v = tot[t]; tot[t] = r; r += v; }
  }
  __syncthreads();
  double r = tot[threadIdx.x];
  for (uint64_t i = lo; i < hi; ++i) { r += cum[i]; cum[i] = r; }
}

// ro (optional): readout errors (Sec. V.A), 2 per qubit: qubit q of value b
// is reported as 1 - b when u01(seed, traj, 2, (j << 6) | q) < ro[2q + b];
// lane l decides qubits l and l + 32, and the flips are OR-combined.
__global__ void k_sample(const float2* __restrict__ psi, uint64_t namps, const float* __restrict__ sub,
                         uint64_t nsub, const double* __restrict__ cum, uint64_t nblk, uint64_t seed,
                         uint64_t traj, uint32_t S, uint64_t* __restrict__ out, int n,
                         const double* __restrict__ ro) {
  const int lane = threadIdx.x & 31;
  const uint64_t warp = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
  for (uint64_t j = warp; j < S; j += nwarps) {
    const double total = cum[nblk - 1];
    const double t = uniform01(seed, traj, kStreamSample, static_cast<uint32_t>(j)) * total;
    // block: first b with t < cum[b]
    uint64_t lo = 0, hi = nblk - 1;
    while (lo < hi) {
      const uint64_t mid = (lo + hi) >> 1;
      if (t < cum[mid]) hi = mid; else lo = mid + 1;
    }
    const uint64_t b = lo;
    double trel = t - (b ? cum[b - 1] : 0.0);
    // sub-block inside the block (same lane values and scan as k_cdf_blk)
    double s0, s1;
    block_lane_values(sub, nsub, b, lane, s0, s1);
    const double incl = warp_incl_scan_d(s0 + s1, lane);
    double excl = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane == 0) excl = 0.0;
    unsigned hit = __ballot_sync(0xffffffffu, trel < incl);
    int L = hit ? __ffs(hit) - 1 : 31;
    const double eL = __shfl_sync(0xffffffffu, excl, L);
    const double s0L = __shfl_sync(0xffffffffu, s0, L);
    uint64_t sidx = (b << 6) + 2 * L;
    double base = eL;
    if (!(trel < eL + s0L)) { base = eL + s0L; sidx += 1; }
    if (sidx >= nsub) sidx = nsub - 1;
    trel -= base;
    // chunks inside the sub-block (same chunk arithmetic as k_cdf_sub)
    float run = 0.f;
    uint64_t x = ~0ull, last_nz = sidx << kCdfSubLog;
    for (int c = 0; c < (1 << (kCdfSubLog - kCdfChunkLog)); ++c) {
      const uint64_t x0 = (sidx << kCdfSubLog) + (static_cast<uint64_t>(c) << kCdfChunkLog) + 2 * lane;
      float w0, w1;
      chunk_weights(psi, namps, x0, w0, w1);
      const float inc = warp_incl_scan_f(w0 + w1, lane);
      const float tot = __shfl_sync(0xffffffffu, inc, 31);
      const float cend = run + inc;
      const float cstart = cend - (w0 + w1);
      const unsigned h = __ballot_sync(0xffffffffu, trel < static_cast<double>(cend));
      const unsigned nz = __ballot_sync(0xffffffffu, (w0 + w1) > 0.f);
      if (nz) {
        const int ln = 31 - __clz(nz);
        const float w1n = __shfl_sync(0xffffffffu, w1, ln);
        last_nz = (sidx << kCdfSubLog) + (static_cast<uint64_t>(c) << kCdfChunkLog) + 2 * ln + (w1n > 0.f ? 1 : 0);
      }
      if (h) {
        const int l2 = __ffs(h) - 1;
        const float cs = __shfl_sync(0xffffffffu, cstart, l2);
        const float a0 = __shfl_sync(0xffffffffu, w0, l2);
        x = (sidx << kCdfSubLog) + (static_cast<uint64_t>(c) << kCdfChunkLog) + 2 * l2 +
            (trel < static_cast<double>(cs + a0) ? 0 : 1);
        break;
      }
      run += tot;
    }
    if (x == ~0ull) x = last_nz;     // rounding put t past the sub-block end
    if (ro) {
      unsigned long long flips = 0ull;
      for (int q = lane; q < n; q += 32) {
        const uint32_t b = static_cast<uint32_t>((x >> q) & 1ull);
        const double u = uniform01(seed, traj, kStreamReadout, (static_cast<uint32_t>(j) << 6) | static_cast<uint32_t>(q));
        if (u < ro[2 * q + b]) flips |= 1ull << q;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) flips |= __shfl_xor_sync(0xffffffffu, flips, o);
      x ^= flips;
    }
    if (lane == 0) out[j] = x;
  }
}

// C(x) for every x, exactly as k_sample compares against it: the FP64 table
// up to the block, the FP64 lane scan up to the sub-block, and the FP32 run
// inside the sub-block up to x (one warp per sub-block, same chunk arithmetic)
__global__ void k_cdf_values(const float2* __restrict__ psi, uint64_t namps, const float* __restrict__ sub,
                             uint64_t nsub, const double* __restrict__ cum, double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const uint64_t warp = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
  for (uint64_t s = warp; s < nsub; s += nwarps) {
    const uint64_t b = s >> 6;
    double s0, s1;
    block_lane_values(sub, nsub, b, lane, s0, s1);
    const double incl = warp_incl_scan_d(s0 + s1, lane);
    double excl = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane == 0) excl = 0.0;
    const int L = static_cast<int>((s & 63) >> 1);
    const double eL = __shfl_sync(0xffffffffu, excl, L);
    const double s0L = __shfl_sync(0xffffffffu, s0, L);
    const double base = (b ? cum[b - 1] : 0.0) + ((s & 1) ? eL + s0L : eL);
    float run = 0.f;
    for (int c = 0; c < (1 << (kCdfSubLog - kCdfChunkLog)); ++c) {
      const uint64_t x0 = (s << kCdfSubLog) + (static_cast<uint64_t>(c) << kCdfChunkLog) + 2 * lane;
      float w0, w1;
      chunk_weights(psi, namps, x0, w0, w1);
      const float inc = warp_incl_scan_f(w0 + w1, lane);
      const float tot = __shfl_sync(0xffffffffu, inc, 31);
      const float cend = run + inc;
      const float cstart = cend - (w0 + w1);
      if (x0 < namps) {
        out[x0] = base + static_cast<double>(cstart + w0);
        out[x0 + 1] = base + static_cast<double>(cend);
      }
      run += tot;
    }
  }
}

// the three table levels of the sampling CDF (sub-block runs, block scans,
// FP64 table) into scr.cdf_sub / scr.cdf_cum
static void build_cdf_tables(const float2* psi, int n, const Scratch& scr, cudaStream_t st) {
  const uint64_t namps = 1ull << n;
  const uint64_t nsub = cdf_num_sub(n), nblk = cdf_num_blk(n);
  const int threads = 256, wpb = threads / 32;
  uint64_t g = (nsub + wpb - 1) / wpb;
  const uint64_t cap = static_cast<uint64_t>(sm_count()) * 8;
  if (g > cap) g = cap;
  k_cdf_sub<<<static_cast<unsigned>(g), threads, 0, st>>>(psi, namps, nsub, scr.cdf_sub);
  uint64_t gb = (nblk + wpb - 1) / wpb;
  if (gb > cap) gb = cap;
  k_cdf_blk<<<static_cast<unsigned>(gb), threads, 0, st>>>(scr.cdf_sub, nsub, nblk, scr.cdf_cum);
  k_cdf_scan<<<1, 1024, 0, st>>>(scr.cdf_cum, nblk);
}

cudaError_t launch_cdf_values(const float2* psi, int n, const Scratch& scr, double* out, cudaStream_t st) {
  if (n < 1) return cudaErrorInvalidValue;
  build_cdf_tables(psi, n, scr, st);
  const uint64_t nsub = cdf_num_sub(n);
  const int threads = 256, wpb = threads / 32;
  uint64_t g = (nsub + wpb - 1) / wpb;
  const uint64_t cap = static_cast<uint64_t>(sm_count()) * 8;
  if (g > cap) g = cap;
  k_cdf_values<<<static_cast<unsigned>(g), threads, 0, st>>>(psi, 1ull << n, scr.cdf_sub, nsub, scr.cdf_cum, out);
  return cudaGetLastError();
}

cudaError_t launch_sample(const float2* psi, int n, uint64_t seed, uint64_t traj, uint32_t S,
                          uint64_t* out, const Scratch& scr, cudaStream_t st, const double* readout) {
  if (n < 1) return cudaErrorInvalidValue;
  const uint64_t namps = 1ull << n;
  const uint64_t nsub = cdf_num_sub(n), nblk = cdf_num_blk(n);
  const int threads = 256, wpb = threads / 32;
  const uint64_t cap = static_cast<uint64_t>(sm_count()) * 8;
  build_cdf_tables(psi, n, scr, st);
  if (S > 0) {
    uint64_t gs = (S + wpb - 1) / wpb;
    if (gs > cap) gs = cap;
    k_sample<<<static_cast<unsigned>(gs), threads, 0, st>>>(psi, namps, scr.cdf_sub, nsub, scr.cdf_cum,
                                                           nblk, seed, traj, S, out, n, readout);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
__global__ void k_init(float4* __restrict__ psi, uint64_t npairs) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < npairs; i += stride)
    psi[i] = make_float4(i == 0 ? 1.f : 0.f, 0.f, 0.f, 0.f);
}

cudaError_t kernel_arch(int* binary_version, int* ptx_version) {
  cudaFuncAttributes a{};
  const cudaError_t e = cudaFuncGetAttributes(&a, k_init);
  if (e != cudaSuccess) return e;
  *binary_version = a.binaryVersion;
  *ptx_version = a.ptxVersion;
  return cudaSuccess;
}

__global__ void k_scale(float4* __restrict__ psi, uint64_t npairs, float f) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < npairs; i += stride) {
    float4 v = psi[i];
    v.x *= f; v.y *= f; v.z *= f; v.w *= f;
    psi[i] = v;
  }
}

static unsigned stream_grid(uint64_t items) {
  uint64_t g = (items + 255) / 256;
  const uint64_t cap = static_cast<uint64_t>(sm_count()) * 8;
  return static_cast<unsigned>(g < cap ? (g ? g : 1) : cap);
}

// ---------------------------------------------------------------------------
// Product-state preparation.  Fused gates that are the first to act on each
// of their qubits, on disjoint qubits, take |0...0> to the tensor product of
// their first columns (U |0> = U[:, 0]) with |0> on every other qubit.  With
// the qubits split at m, each factor on the low or on the high side, the
// amplitude is psi[x] = H[x >> m] * L[x mod 2^m]: the two tables are built
// first (FP64 products of the factors, rounded once), then one write pass
// fills the state, in place of the |0...0> pass and one pass per factor.
// ---------------------------------------------------------------------------
__global__ void k_fold_table(float2* __restrict__ out, uint32_t size, const __grid_constant__ FoldSpec s) {
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < size; e += stride) {
    double re = 0.0, im = 0.0;
    if (!(e & s.zmask)) {
      re = 1.0;
      for (int f = 0; f < s.nf; ++f) {
        uint32_t j = 0;
        for (int b = 0; b < s.w[f]; ++b) j |= ((e >> s.q[f][b]) & 1u) << b;
        const float2 v = s.v[s.off[f] + j];
        const double a = re * v.x - im * v.y;
        im = re * v.y + im * v.x;
        re = a;
      }
    }
    out[e] = make_float2(static_cast<float>(re), static_cast<float>(im));
  }
}

__global__ void __launch_bounds__(256) k_init_outer(float4* __restrict__ psi, const float2* __restrict__ tl,
                                                    const float2* __restrict__ th, int m, uint64_t npairs) {
  const uint64_t lmask = (1ull << m) - 1ull;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < npairs; i += stride) {
    const uint64_t x = 2ull * i;                  // even: both amplitudes share H[x >> m] (m >= 1)
    const float4 l = *reinterpret_cast<const float4*>(tl + (x & lmask));
    const float2 h = th[x >> m];
    __stcs(psi + i, make_float4(h.x * l.x - h.y * l.y, h.x * l.y + h.y * l.x,
                                h.x * l.z - h.y * l.w, h.x * l.w + h.y * l.z));
  }
}

cudaError_t launch_init_product(float2* psi, int n, int m, const FoldSpec& lo, const FoldSpec& hi,
                                float2* tables, cudaStream_t st) {
  if (n < 2 || m < 1 || m >= n || m > kFoldTableBits || n - m > kFoldTableBits) return cudaErrorInvalidValue;
  const uint32_t nl = 1u << m, nhi = 1u << (n - m);
  float2* tl = tables;
  float2* th = tables + nl;                      // nl even: th stays 16-byte aligned
  k_fold_table<<<stream_grid(nl), 256, 0, st>>>(tl, nl, lo);
  k_fold_table<<<stream_grid(nhi), 256, 0, st>>>(th, nhi, hi);
  const uint64_t np = 1ull << (n - 1);
  k_init_outer<<<stream_grid(np), 256, 0, st>>>(reinterpret_cast<float4*>(psi), tl, th, m, np);
  return cudaGetLastError();
}

cudaError_t launch_init_state(float2* psi, int n, cudaStream_t st) {
  if (n < 1) return cudaErrorInvalidValue;
  const uint64_t np = 1ull << (n - 1);
  k_init<<<stream_grid(np), 256, 0, st>>>(reinterpret_cast<float4*>(psi), np);
  return cudaGetLastError();
}

cudaError_t launch_scale(float2* psi, int n, float f, cudaStream_t st) {
  if (n < 1) return cudaErrorInvalidValue;
  const uint64_t np = 1ull << (n - 1);
  k_scale<<<stream_grid(np), 256, 0, st>>>(reinterpret_cast<float4*>(psi), np, f);
  return cudaGetLastError();
}

}  // namespace qt
