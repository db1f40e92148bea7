// Fused-gate application (Alg. 1, Sec. III.A) on a complex64 state.
//
// The state is 2^n interleaved (re, im) float pairs.  A k-qubit fused gate
// splits it into 2^(n-k) gather sets of 2^k amplitudes (the set's base
// index with every combination of the target bits); each set is one
// 2^k x 2^k matrix-vector product.
//
// k_apply_tile (the main kernel): a CTA of 128 threads owns one tile of
// 128 gather sets = 2^(7+k) amplitudes.  The tile is 2^h rows (h = number
// of "high" targets) of 2^C contiguous amplitudes, where C is the smallest
// width such that the row holds every "low" target plus 7 free bits; so a
// row is at least 1 KB and every warp-wide 128-bit load or store of the
// tile is fully coalesced whatever the target pattern.  The tile is staged
// in shared memory with an XOR swizzle (8-byte slot ^= a per-launch linear
// image of index bits 4..7) chosen so that the strided gathers of every
// target pattern are free of bank conflicts.  Each thread then gathers one
// set, multiplies, and scatters it back; the tile is stored with the same
// coalesced pattern.
//
// The matrix is a __grid_constant__ kernel parameter: its entries reach the
// FMAs through uniform registers loaded from the constant bank.  The complex
// products use the three-multiply form: with U = c + i d and v = a + i b,
// precomputing e = c + d and f = d - c per entry and s = a + b per amplitude,
//   Re(U v) = sum c s - sum b e,   Im(U v) = sum c s + sum a f,
// i.e. 3 FMA per complex multiply-add instead of 4.  The two sums that
// share an entry pair, (sum c s, sum e b), run as one packed FP32x2 FMA on
// the (c, e) pair, so a complex multiply-add issues 2 instructions.
//
// k_apply (direct, for states smaller than one tile): one thread per
// gather set (or per pair of sets that differ in bit 0), members loaded
// straight into registers.
//
// Bytes per launch: 16 * 2^n (every amplitude read once and written once).
// FLOPs per launch: 2^(k+2) * 2^(n+1) (the paper's count).
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
#pragma unroll 2
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
#pragma unroll 2
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

int sm_count() {
  static PerDevice sms;
  return sms.get([] {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
  });
}


// ---------------------------------------------------------------------------
// tiled kernel
// ---------------------------------------------------------------------------
constexpr int kTileThreads = 128;       // = gather sets per tile

// 16-byte aligned so that the matrix pairs sit on aligned constant-bank words
template <int K>
struct alignas(16) TileArgs {
  float2 ce[1 << K][1 << K];  // (Re U, Re U + Im U)
  float f[1 << K][1 << K];    // Im U - Re U
  uint64_t roff[1 << K];      // memory offset of tile row r
  uint64_t poff[1 << K];      // memory offset of tile index 256 c (chunk c of every thread)
  uint32_t smoff[1 << K];     // swizzled tile-local offset of member m
  uint32_t tins[K];           // tile-local target positions, ascending
  uint32_t hins[K];           // memory positions of the high targets, ascending
  uint8_t swzt[16];           // swizzle table: slot = l ^ swzt[(l >> 4) & 15]
  int nh;                     // number of high targets
  int C;                      // contiguous low bits per row
  uint64_t num_tiles;
};

__device__ __forceinline__ uint32_t swz(uint32_t l) { return l ^ ((l >> 4) & 15u); }

// The swizzle of the tile kernel is chosen per launch.  It XORs a linear
// (GF(2)) image of index bits 4..7 into bits 0..3, slot = l ^ G(l >> 4 & 15).
// A half-warp's 16 lanes differ in the 4 lowest non-target tile positions;
// those below 4 stay put, and G maps those in 4..7 onto the target positions
// below 4, so every 8-byte gather and scatter of a half-warp hits 16
// distinct bank pairs, whatever the targets.  (No fixed map does this for
// every pattern: the single-target cases force every entry of G to 1.)  The
// image of bit 4 also sets bit 0, which keeps the coalesced staging stores
// (lane t writes index 2t) conflict-free.
__device__ __forceinline__ uint32_t swz_t(uint32_t l, const uint8_t* t) { return l ^ t[(l >> 4) & 15u]; }

static void swizzle_table(const uint32_t* tpos, int K, uint8_t* tab) {
  uint32_t tmask = 0;
  for (int b = 0; b < K; ++b) tmask |= 1u << tpos[b];
  int lane[4], nl = 0;
  for (uint32_t p = 0; nl < 4; ++p)
    if (!((tmask >> p) & 1u)) lane[nl++] = static_cast<int>(p);
  uint32_t g[4] = {1u, 2u, 4u, 8u};    // image of bit 4 + i (the fixed map)
  if (lane[3] < 8) {
    int low = 0;                       // target positions below 4, ascending
    for (int i = 0; i < 4; ++i)
      if (lane[i] >= 4) {
        while (!((tmask >> low) & 1u)) ++low;
        g[lane[i] - 4] = 1u << low++;
      }
  }
  g[0] |= 1u;
  for (int x = 0; x < 16; ++x) {
    uint32_t v = 0;
    for (int i = 0; i < 4; ++i)
      if ((x >> i) & 1) v ^= g[i];
    tab[x] = static_cast<uint8_t>(v);
  }
}

// RU: unroll factor of the row loop; MINB: CTAs per SM that the register
// allocation must allow.  At K = 4 the kernel is issue-bound: rows go four
// at a time under an 8-CTA bound (64 registers), which gives the scheduler
// the most warps to choose from; a full row unroll keeps more values live
// than even 255 registers hold.
//
// Index arithmetic is hoisted out of the per-amplitude work with two
// identities.  The swizzle distributes over an OR of disjoint bit sets,
// swz(x | y) = swz(x) ^ swz(y), so member m of the thread's set sits at
// swz(sbase) ^ smoff[m] with smoff[m] = swz(moff[m]) precomputed.  The map
// from a tile index to its memory offset deposits bits (the row bits go to
// the high-target positions), so it too distributes over disjoint bits:
// thread t's chunk c (tile index 2t + 256c) is at offset(2t) | poff[c].
template <int K, int RU = 2, int MINB = 1>
__global__ void __launch_bounds__(kTileThreads, MINB) k_apply_tile(float2* __restrict__ psi,
                                                             const __grid_constant__ TileArgs<K> a) {
  constexpr int M = 1 << K;
  constexpr int TILE = kTileThreads * M;       // amplitudes per tile
  constexpr int NCH = TILE / 2 / kTileThreads; // float4 chunks per thread
  __shared__ __align__(16) float2 sm[TILE];
  const uint32_t tid = threadIdx.x;
  // this thread's gather set inside the tile (same for every tile)
  uint32_t sbase = tid;
#pragma unroll
  for (int b = 0; b < K; ++b) {
    const uint32_t t = a.tins[b];
    sbase = ((sbase >> t) << (t + 1)) | (sbase & ((1u << t) - 1u));
  }
  const uint32_t ss = swz_t(sbase, a.swzt);
  // one tile per CTA: a loop over tiles would make the matrix entries
  // loop-invariant, and the compiler would then hold them in registers
  {
    const uint64_t tile = blockIdx.x;
    uint64_t base = tile << a.C;
    for (int j = 0; j < a.nh; ++j) {
      const uint32_t h = a.hins[j];
      base = ((base >> h) << (h + 1)) | (base & ((1ull << h) - 1ull));
    }
    const uint32_t l0 = 2u * tid;
    float2* const pt = psi + (base | a.roff[l0 >> a.C] | (l0 & ((1u << a.C) - 1u)));
    // bits 4..7 of the tile index 2t + 256c are bits 3..6 of t, so the
    // swizzle of both amplitudes of a chunk is the same for every c
    const uint32_t fl = a.swzt[(tid >> 3) & 15u];
    const uint32_t s0 = l0 ^ fl, s1 = (l0 + 1u) ^ fl;
    // load rows -> shared (coalesced 128-bit)
    float4 buf[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) buf[c] = __ldcs(reinterpret_cast<const float4*>(pt + a.poff[c]));
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
      sm[s0 + 256u * c] = make_float2(buf[c].x, buf[c].y);
      sm[s1 + 256u * c] = make_float2(buf[c].z, buf[c].w);
    }
    __syncthreads();
    // one gather set per thread
    float va[M];
    float2 sb[M];    // (a + b, b) of member m
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const float2 v = sm[ss ^ a.smoff[m]];
      va[m] = v.x;
      sb[m] = make_float2(v.x + v.y, v.y);
    }
    // rows RU at a time: the matrix entries come in through uniform
    // constant loads (warp-uniform row index)
#pragma unroll RU
    for (int j = 0; j < M; ++j) {
      float2 tr = make_float2(0.f, 0.f);    // (sum c s, sum e b)
      float im = 0.f;
#pragma unroll
      for (int m = 0; m < M; ++m) {
        tr = __ffma2_rn(a.ce[j][m], sb[m], tr);
        im = fmaf(a.f[j][m], va[m], im);
      }
      sm[ss ^ a.smoff[j]] = make_float2(tr.x - tr.y, tr.x + im);
    }
    __syncthreads();
    // shared -> rows (coalesced 128-bit)
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
      const float2 x = sm[s0 + 256u * c], y = sm[s1 + 256u * c];
      __stcs(reinterpret_cast<float4*>(pt + a.poff[c]), make_float4(x.x, x.y, y.x, y.y));
    }
    __syncthreads();
  }
}

template <int K>
static cudaError_t launch_tile(float2* psi, int n, const uint32_t* targets, const float2* U,
                               cudaStream_t st) {
  constexpr int M = 1 << K;
  TileArgs<K> a;
  for (int j = 0; j < M; ++j)
    for (int m = 0; m < M; ++m) {
      const float re = U[j * M + m].x, im = U[j * M + m].y;
      a.ce[j][m] = make_float2(re, re + im);
      a.f[j][m] = im - re;
    }
  // C = 7 + number of targets below C
  int C = 7;
  for (;;) {
    int low = 0;
    for (int b = 0; b < K; ++b) low += targets[b] < static_cast<uint32_t>(C);
    if (C - low >= 7) break;
    ++C;
  }
  a.C = C;
  int nh = 0;
  uint32_t tpos[K];
  for (int b = 0; b < K; ++b) {
    if (targets[b] < static_cast<uint32_t>(C)) {
      tpos[b] = targets[b];
    } else {
      tpos[b] = static_cast<uint32_t>(C + nh);
      a.hins[nh++] = targets[b];
    }
  }
  a.nh = nh;
  for (int b = 0; b < K; ++b) a.tins[b] = tpos[b];   // ascending: low targets, then C, C+1, ...
  swizzle_table(tpos, K, a.swzt);
  for (int m = 0; m < M; ++m) {
    uint32_t o = 0;
    for (int b = 0; b < K; ++b)
      if ((m >> b) & 1) o |= 1u << tpos[b];
    a.smoff[m] = o ^ a.swzt[(o >> 4) & 15u];
  }
  for (int r = 0; r < M; ++r) {
    uint64_t o = 0;
    for (int j = 0; j < nh; ++j)
      if ((r >> j) & 1) o |= 1ull << a.hins[j];
    a.roff[r] = r < (1 << nh) ? o : 0;
  }
  // chunk c of every thread starts at tile index 256 c (< 2^(7+K))
  for (int c = 0; c < M; ++c) {
    const uint32_t l = 256u * static_cast<uint32_t>(c);
    a.poff[c] = c < M / 2 ? (a.roff[l >> C] | (l & ((1u << C) - 1u))) : 0;
  }
  a.num_tiles = 1ull << (n - C - nh);
  if constexpr (K == 4)
    k_apply_tile<4, 4, 8><<<static_cast<unsigned>(a.num_tiles), kTileThreads, 0, st>>>(psi, a);
  else if constexpr (K == 5)
    k_apply_tile<5, 2, 3><<<static_cast<unsigned>(a.num_tiles), kTileThreads, 0, st>>>(psi, a);
  else
    k_apply_tile<K><<<static_cast<unsigned>(a.num_tiles), kTileThreads, 0, st>>>(psi, a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// 6-qubit fused gates on CUDA cores (FP32 reference path for the split-TF32
// tensor-core kernel).  A 64 x 64 complex matrix (32 KB) does not fit in the
// kernel parameters, so it is staged in shared memory with the tile; each
// thread computes its set's 64 outputs in blocks of 16 rows, reading the
// inputs and the (warp-uniform, broadcast) matrix entries from shared memory
// and writing into a separate output tile.
// ---------------------------------------------------------------------------
struct Tile6Args {
  const float2* u;            // 64 x 64 row-major matrix (device)
  uint64_t roff[64];
  uint32_t moff[64];
  uint32_t tins[6];
  uint32_t hins[6];
  int nh, C;
  uint64_t num_tiles;
};

constexpr int kTile6Amps = kTileThreads * 64;                      // 8192 amplitudes
constexpr size_t kTile6Smem = sizeof(float2) * (2 * kTile6Amps + 64 * 64);   // 160 KB

__global__ void __launch_bounds__(kTileThreads, 1) k_apply_tile6(float2* __restrict__ psi,
                                                                 const __grid_constant__ Tile6Args a) {
  extern __shared__ __align__(16) float2 sm6[];
  float2* tin = sm6;
  float2* tout = sm6 + kTile6Amps;
  float2* U = sm6 + 2 * kTile6Amps;
  const uint32_t tid = threadIdx.x;
  for (int i = tid; i < 64 * 64; i += kTileThreads) U[i] = a.u[i];
  const uint32_t rowmask = (1u << a.C) - 1u;
  uint32_t sbase = tid;
#pragma unroll
  for (int b = 0; b < 6; ++b) {
    const uint32_t t = a.tins[b];
    sbase = ((sbase >> t) << (t + 1)) | (sbase & ((1u << t) - 1u));
  }
  const uint64_t tile = blockIdx.x;
  uint64_t base = tile << a.C;
  for (int j = 0; j < a.nh; ++j) {
    const uint32_t h = a.hins[j];
    base = ((base >> h) << (h + 1)) | (base & ((1ull << h) - 1ull));
  }
  for (int i = 0; i < kTile6Amps / 2 / kTileThreads; ++i) {
    const uint32_t l = 2u * (tid + i * kTileThreads);
    const uint32_t fl = (l >> 4) & 15u;
    float4 v = __ldcs(reinterpret_cast<const float4*>(psi + (base | a.roff[l >> a.C] | (l & rowmask))));
    if (fl & 1u) v = make_float4(v.z, v.w, v.x, v.y);
    *reinterpret_cast<float4*>(&tin[(l ^ fl) & ~1u]) = v;
  }
  __syncthreads();
  for (int rb = 0; rb < 64; rb += 16) {
    float xr[16], xi[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) { xr[j] = 0.f; xi[j] = 0.f; }
    for (int m = 0; m < 64; ++m) {
      const float2 v = tin[swz(sbase | a.moff[m])];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float2 u = U[(rb + j) * 64 + m];
        xr[j] = fmaf(u.x, v.x, fmaf(-u.y, v.y, xr[j]));
        xi[j] = fmaf(u.x, v.y, fmaf(u.y, v.x, xi[j]));
      }
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) tout[swz(sbase | a.moff[rb + j])] = make_float2(xr[j], xi[j]);
  }
  __syncthreads();
  for (int i = 0; i < kTile6Amps / 2 / kTileThreads; ++i) {
    const uint32_t l = 2u * (tid + i * kTileThreads);
    const uint32_t fl = (l >> 4) & 15u;
    float4 v = *reinterpret_cast<const float4*>(&tout[(l ^ fl) & ~1u]);
    if (fl & 1u) v = make_float4(v.z, v.w, v.x, v.y);
    __stcs(reinterpret_cast<float4*>(psi + (base | a.roff[l >> a.C] | (l & rowmask))), v);
  }
}

cudaError_t launch_apply6_fp32(float2* psi, int n, const uint32_t* targets, const float2* udev, cudaStream_t st) {
  if (n < 13) return cudaErrorInvalidValue;
  static PerDevice attr_set;
  const cudaError_t attr = static_cast<cudaError_t>(attr_set.get([] {
    return static_cast<int>(cudaFuncSetAttribute(k_apply_tile6, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 static_cast<int>(kTile6Smem)));
  }));
  if (attr != cudaSuccess) return attr;
  Tile6Args a;
  a.u = udev;
  int C = 7;
  for (;;) {
    int low = 0;
    for (int b = 0; b < 6; ++b) low += targets[b] < static_cast<uint32_t>(C);
    if (C - low >= 7) break;
    ++C;
  }
  a.C = C;
  int nh = 0;
  uint32_t tpos[6];
  for (int b = 0; b < 6; ++b) {
    if (targets[b] < static_cast<uint32_t>(C)) {
      tpos[b] = targets[b];
    } else {
      tpos[b] = static_cast<uint32_t>(C + nh);
      a.hins[nh++] = targets[b];
    }
  }
  a.nh = nh;
  for (int b = 0; b < 6; ++b) a.tins[b] = tpos[b];
  for (int m = 0; m < 64; ++m) {
    uint32_t o = 0;
    for (int b = 0; b < 6; ++b)
      if ((m >> b) & 1) o |= 1u << tpos[b];
    a.moff[m] = o;
    uint64_t r = 0;
    for (int j = 0; j < nh; ++j)
      if ((m >> j) & 1) r |= 1ull << a.hins[j];
    a.roff[m] = m < (1 << nh) ? r : 0;
  }
  a.num_tiles = 1ull << (n - C - nh);
  k_apply_tile6<<<static_cast<unsigned>(a.num_tiles), kTileThreads, kTile6Smem, st>>>(psi, a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Multi-gate pass: several fused gates applied to one tile in shared memory
// per HBM pass.  The tile holds qubits 0..6 (rows of 128 contiguous
// amplitudes) and up to 6 higher qubits; every gate of the group acts
// inside these qubits, so the state is read and written once for the whole
// group.  Gates are applied in order with a barrier between them; each
// thread applies its share of the gate's gather sets.
// ---------------------------------------------------------------------------
constexpr int kGroupThreads = 256;

struct GroupGate {
  uint8_t k;                  // width (1..4)
  uint8_t tins[4];            // tile-local target positions, ascending
  uint8_t pad[3];
  uint16_t moff[16];          // tile-local offset of member m
  uint32_t mat;               // float offset of (c, e, f) in GroupArgs::m
};

struct GroupArgs {
  GroupGate g[kGroupMaxGates];
  float m[kGroupMaxGates * 3 * 256];   // per gate: D*D (e, f) pairs, then D*D c values
  uint64_t roff[64];                   // memory offset of tile row r
  uint32_t hins[6];                    // memory positions of the high qubits, ascending
  int nh, ng;
  uint32_t nmat;                       // floats of m in use
  uint64_t num_tiles;
};

// one gate of a multi-gate pass; its matrix is in shared memory as (e, f)
// pairs followed by c values (the three-multiply form of k_apply_tile).  A
// thread applies two gather sets at a time; the (Sum b e, Sum a f) pair is
// one __ffma2_rn on the swapped member (b, a), and each 128-bit broadcast
// load (two pairs, or four c values) feeds both sets.
template <int K, int SPT>
__device__ __forceinline__ void group_gate(float2* sm, uint32_t tile_amps, const GroupGate G,
                                           const float* __restrict__ m) {
  constexpr int M = 1 << K;
  const uint32_t sets = tile_amps >> K;
  const float2* ef = reinterpret_cast<const float2*>(m);
  const float* c = m + 2 * M * M;
  for (uint32_t s0 = threadIdx.x * SPT; s0 < sets; s0 += kGroupThreads * SPT) {
    uint32_t bb[SPT];
    float2 x[SPT][M];
    float vs[SPT][M];
#pragma unroll
    for (int p = 0; p < SPT; ++p) {
      uint32_t b = s0 + p < sets ? s0 + p : s0;          // sets is even: never clamps in practice
#pragma unroll
      for (int i = 0; i < K; ++i) {
        const uint32_t t = G.tins[i];
        b = ((b >> t) << (t + 1)) | (b & ((1u << t) - 1u));
      }
      bb[p] = b;
#pragma unroll
      for (int j = 0; j < M; ++j) {
        const float2 v = sm[swz(b | G.moff[j])];
        x[p][j] = make_float2(v.y, v.x);
        vs[p][j] = v.x + v.y;
      }
    }
#pragma unroll 2
    for (int j = 0; j < M; ++j) {
      float2 pp[SPT];
      float t[SPT];
#pragma unroll
      for (int p = 0; p < SPT; ++p) { pp[p] = make_float2(0.f, 0.f); t[p] = 0.f; }
      if constexpr (M >= 4) {
#pragma unroll
        for (int q = 0; q < M; q += 4) {
          const float4 e01 = *reinterpret_cast<const float4*>(ef + j * M + q);
          const float4 e23 = *reinterpret_cast<const float4*>(ef + j * M + q + 2);
          const float4 cc = *reinterpret_cast<const float4*>(c + j * M + q);
          const float2 ev[4] = {make_float2(e01.x, e01.y), make_float2(e01.z, e01.w), make_float2(e23.x, e23.y),
                                make_float2(e23.z, e23.w)};
          const float cv[4] = {cc.x, cc.y, cc.z, cc.w};
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int p = 0; p < SPT; ++p) {
              pp[p] = __ffma2_rn(ev[u], x[p][q + u], pp[p]);
              t[p] = fmaf(cv[u], vs[p][q + u], t[p]);
            }
        }
      } else {
#pragma unroll
        for (int q = 0; q < M; ++q)
#pragma unroll
          for (int p = 0; p < SPT; ++p) {
            pp[p] = __ffma2_rn(ef[j * M + q], x[p][q], pp[p]);
            t[p] = fmaf(c[j * M + q], vs[p][q], t[p]);
          }
      }
#pragma unroll
      for (int p = 0; p < SPT; ++p)
        if (s0 + p < sets) sm[swz(bb[p] | G.moff[j])] = make_float2(t[p] - pp[p].x, t[p] + pp[p].y);
    }
  }
}

__global__ void __launch_bounds__(kGroupThreads, 2) k_apply_group(float2* __restrict__ psi,
                                                               const __grid_constant__ GroupArgs a) {
  extern __shared__ __align__(16) float2 smg[];
  const uint32_t tid = threadIdx.x;
  const uint32_t tile_amps = 128u << a.nh;
  float* smat = reinterpret_cast<float*>(smg + tile_amps);     // the group's matrices
  const uint64_t tile = blockIdx.x;
  uint64_t base = tile << 7;
  for (int j = 0; j < a.nh; ++j) {
    const uint32_t h = a.hins[j];
    base = ((base >> h) << (h + 1)) | (base & ((1ull << h) - 1ull));
  }
  for (uint32_t i = tid; i < a.nmat; i += kGroupThreads) smat[i] = a.m[i];
  for (uint32_t c = tid; c < tile_amps / 2; c += kGroupThreads) {
    const uint32_t l = 2u * c;
    const uint32_t fl = (l >> 4) & 15u;
    float4 v = __ldcs(reinterpret_cast<const float4*>(psi + (base | a.roff[l >> 7] | (l & 127u))));
    if (fl & 1u) v = make_float4(v.z, v.w, v.x, v.y);
    *reinterpret_cast<float4*>(&smg[(l ^ fl) & ~1u]) = v;
  }
  for (int gi = 0; gi < a.ng; ++gi) {
    __syncthreads();
    const GroupGate G = a.g[gi];            // descriptor in registers
    const float* m = smat + G.mat;
    switch (G.k) {
      case 1: group_gate<1, 2>(smg, tile_amps, G, m); break;
      case 2: group_gate<2, 2>(smg, tile_amps, G, m); break;
      case 3: group_gate<3, 2>(smg, tile_amps, G, m); break;
      default: group_gate<4, 2>(smg, tile_amps, G, m); break;
    }
  }
  __syncthreads();
  for (uint32_t c = tid; c < tile_amps / 2; c += kGroupThreads) {
    const uint32_t l = 2u * c;
    const uint32_t fl = (l >> 4) & 15u;
    float4 v = *reinterpret_cast<const float4*>(&smg[(l ^ fl) & ~1u]);
    if (fl & 1u) v = make_float4(v.z, v.w, v.x, v.y);
    __stcs(reinterpret_cast<float4*>(psi + (base | a.roff[l >> 7] | (l & 127u))), v);
  }
}

cudaError_t launch_apply_group(float2* psi, int n, int ng, const GroupPiece* pieces, cudaStream_t st) {
  if (ng < 1 || ng > kGroupMaxGates) return cudaErrorInvalidValue;
  static PerDevice attr_set;
  const cudaError_t attr = static_cast<cudaError_t>(attr_set.get([] {
    return static_cast<int>(cudaFuncSetAttribute(
        k_apply_group, cudaFuncAttributeMaxDynamicSharedMemorySize,
        static_cast<int>((sizeof(float2) << 13) + sizeof(float) * kGroupMaxGates * 3 * 256)));
  }));
  if (attr != cudaSuccess) return attr;
  GroupArgs a;
  // high qubits of the group (>= 7), ascending
  uint32_t hmask = 0;
  for (int gi = 0; gi < ng; ++gi)
    for (int b = 0; b < pieces[gi].k; ++b)
      if (pieces[gi].targets[b] >= 7) hmask |= 1u << (pieces[gi].targets[b] - 7);
  int nh = 0;
  for (int q = 0; q < 32; ++q)
    if (hmask & (1u << q)) {
      if (nh == 6) return cudaErrorInvalidValue;
      a.hins[nh++] = static_cast<uint32_t>(q + 7);
    }
  if (n < 7 + nh) return cudaErrorInvalidValue;
  a.nh = nh;
  a.ng = ng;
  auto tpos = [&](uint32_t q) -> uint32_t {
    if (q < 7) return q;
    for (int j = 0; j < nh; ++j)
      if (a.hins[j] == q) return static_cast<uint32_t>(7 + j);
    return 0;
  };
  uint32_t off = 0;
  for (int gi = 0; gi < ng; ++gi) {
    const GroupPiece& P = pieces[gi];
    GroupGate& G = a.g[gi];
    const int K = P.k, M = 1 << K;
    G.k = static_cast<uint8_t>(K);
    uint32_t pos[4];
    for (int b = 0; b < K; ++b) pos[b] = tpos(P.targets[b]);
    for (int b = 0; b < K; ++b) G.tins[b] = static_cast<uint8_t>(pos[b]);   // targets ascending -> positions ascending
    for (int j = 0; j < 16; ++j) {
      uint32_t o = 0;
      for (int b = 0; b < K; ++b)
        if ((j >> b) & 1) o |= 1u << pos[b];
      G.moff[j] = static_cast<uint16_t>(j < M ? o : 0);
    }
    G.mat = off;
    for (int j = 0; j < M * M; ++j) {          // (e, f) pairs, then c
      const float re = P.u[j].x, im = P.u[j].y;
      a.m[off + 2 * j] = re + im;
      a.m[off + 2 * j + 1] = im - re;
      a.m[off + 2 * M * M + j] = re;
    }
    off += 3 * M * M;
  }
  for (int r = 0; r < 64; ++r) {
    uint64_t o = 0;
    for (int j = 0; j < nh; ++j)
      if ((r >> j) & 1) o |= 1ull << a.hins[j];
    a.roff[r] = r < (1 << nh) ? o : 0;
  }
  a.nmat = off;
  a.num_tiles = 1ull << (n - 7 - nh);
  const size_t smem = (sizeof(float2) << (7 + nh)) + sizeof(float) * off;
  k_apply_group<<<static_cast<unsigned>(a.num_tiles), kGroupThreads, smem, st>>>(psi, a);
  return cudaGetLastError();
}

// smallest n for which one tile fits: 7 free bits + k targets
static inline bool tile_fits(int n, int k) { return n >= 7 + k; }

template <int K, bool PAIR>
static cudaError_t launch_k(float2* psi, int n, const uint32_t* targets, const float2* U,
                            cudaStream_t st) {
  static PerDevice occ_dev;
  const int occ = occ_dev.get([] {
    int v = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_apply<K, PAIR>, 256, 0);
    return v > 0 ? v : 1;
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
  if (tile_fits(n, k)) {
    switch (k) {
      case 1: return launch_tile<1>(psi, n, targets, U, st);
      case 2: return launch_tile<2>(psi, n, targets, U, st);
      case 3: return launch_tile<3>(psi, n, targets, U, st);
      case 4: return launch_tile<4>(psi, n, targets, U, st);
      case 5: return launch_tile<5>(psi, n, targets, U, st);
      default: return cudaErrorInvalidValue;
    }
  }
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
