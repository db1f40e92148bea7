// Batched form: thousands of small trajectories in one persistent launch.
//
// The plain loop (runtime.cu) spends one kernel launch per fused gate and a
// host round trip per stage-2 channel; for states of 2^8..2^18 amplitudes
// that is launch- and latency-bound (the paper notes qsim is not tuned for
// small circuits and its translation overhead dominates below 20 qubits,
// Sec. IV.A).  Here every trajectory of the batch, each with its own
// circuit, runs inside one persistent kernel:
//   - one CTA per SM takes trajectories from an atomic counter, largest
//     state first;
//   - a state of up to 2^14 amplitudes lives in the CTA's shared memory;
//     larger states live in a per-CTA slot of global memory (up to 2^20
//     amplitudes, so they stream from DRAM, and each thread keeps 16
//     amplitude loads in flight to cover the latency);
//   - stage 1 of Alg. 2 for every channel is decided on the device with the
//     same Philox4x32-10 draws as the plain loop; stage-2 flush points cut
//     the circuit into segments exactly as in the plain loop, and within a
//     segment a fused gate whose slots all hold their default operator uses
//     its precomputed matrix while any other piece has its members in the
//     segment composed into one matrix in shared memory;
//   - on global-memory states the first segment starts from a product
//     state: every piece that is first on its qubits is folded into the
//     initial state instead of making a pass of its own;
//   - the probability pass, stage 2, and bitstring sampling run in the CTA.
// Host side: circuits are fused on a thread pool (qt_fuse_many) and packed
// once into device tables with every distinct operator set stored once;
// qt_batch_run replays the launch sequence as a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "kernels.h"
#include "qt_internal.h"
#include "qt_philox.h"

namespace qt {
namespace bt {

constexpr int kMaxW = 6;            // widest fused gate in the batched form
constexpr int kSmemNMax = 14;       // states up to 2^14 amplitudes in shared memory
constexpr int kMaxN = 20;           // widest state of the batched form
// product-state start: sum of 2^w over the folded pieces (disjoint qubits,
// w <= 6, n <= 20 give at most 3 * 64 + 4)
constexpr int kFoldCols = 256;

struct Traj {
  uint32_t n, gate0, ngates, op0, nops, ch0, nch, chop0;   // ch0: output offset; chop0: ch_op table offset
  uint64_t arena_off;               // amplitude offset of the kept state (keep_states)
  uint32_t gf0, S;                  // offset of this trajectory's per-gate flags (per trajectory, like ch0);
                                    // with per-trajectory parameters: its sample count
  uint64_t seed, tid, soff;         // with per-trajectory parameters: Philox key, trajectory id, first
                                    // sample slot (a merged launch over several requests)
};
struct Op {
  uint8_t kind, q, q0, q1;
  uint32_t set;
  int32_t channel;                  // relative channel ordinal, -1 for gates
  uint32_t pad;
};
struct Set {
  uint32_t nk, q, def, pad;
  uint32_t mat, kraus, mtm, pbar;   // offsets: float2, float2, double, double
};
struct Gate {
  uint8_t w, t[kMaxW];
  uint8_t pad[1];
  uint32_t mat, mem0, nmem, minpos, maxpos;
};
struct Dev {
  const Traj* traj;
  const Op* ops;
  const Set* sets;
  const Gate* gates;
  const uint32_t* members;
  const uint32_t* ch_op;
  const float2* fmat;
  const double* dmat;
  const uint32_t* order;
  float2* arena;                    // per-CTA slots, or per-trajectory when keeping states
  uint64_t slot_amps;               // amplitudes per CTA slot (0: use traj.arena_off)
  int32_t* kraus;
  int32_t* stage;
  uint8_t* gflag;                   // per fused gate of the run: a member channel holds a non-default stage-1 choice
  uint64_t* samples;
  uint32_t* flushes;
  uint32_t* folds;                  // pieces folded into the product-state start, per trajectory (or null)
  unsigned int* counter;
  int* err;
  const uint64_t* run;              // {seed, first_traj} of the current run (device copy)
  uint32_t num, S, keep;
  uint32_t per_traj;                // 1: seed, id and samples from each Traj (merged launches)
};

// ---------------------------------------------------------------------------
// device helpers (all threads of the CTA call them together)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t insert_zeros(uint64_t x, int w, const int* sorted) {
  for (int b = 0; b < w; ++b) {
    const int s = sorted[b];
    x = ((x >> s) << (s + 1)) | (x & ((1ull << s) - 1ull));
  }
  return x;
}

// psi <- A psi on qubits order[0..W) (basis bit b <-> order[b]); A (row-major) in smem
template <int W, bool GLOBAL>
__device__ void cta_apply_w(float2* psi, int n, const int* order, const float2* A) {
  constexpr int D = 1 << W;
  int sorted[W];
  uint64_t off[D];
#pragma unroll
  for (int b = 0; b < W; ++b) sorted[b] = order[b];
#pragma unroll
  for (int i = 1; i < W; ++i)
#pragma unroll
    for (int j = i; j > 0; --j)
      if (sorted[j - 1] > sorted[j]) { const int t = sorted[j]; sorted[j] = sorted[j - 1]; sorted[j - 1] = t; }
#pragma unroll
  for (int m = 0; m < D; ++m) {
    uint64_t o = 0;
#pragma unroll
    for (int b = 0; b < W; ++b)
      if ((m >> b) & 1) o |= 1ull << order[b];
    off[m] = o;
  }
  // B sets per thread per round, all of their 16 amplitudes loaded before
  // any arithmetic: a state in global memory needs that many loads in
  // flight per thread to cover the memory latency (a shared-memory state
  // does not, and there the extra registers cost more than they save)
  constexpr int B = (!GLOBAL || D >= 16) ? 1 : 16 / D;
  const uint64_t sets = 1ull << (n - W);
  const uint64_t stride = static_cast<uint64_t>(blockDim.x);
  for (uint64_t s0 = threadIdx.x; s0 < sets; s0 += B * stride) {
    uint64_t base[B];
    float2 v[B][D];
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const uint64_t s = s0 + b * stride;
      base[b] = insert_zeros(s < sets ? s : s0, W, sorted);
#pragma unroll
      for (int m = 0; m < D; ++m) v[b][m] = psi[base[b] | off[m]];
    }
#pragma unroll
    for (int b = 0; b < B; ++b) {
      if (s0 + b * stride >= sets) break;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        float xr = 0.f, xi = 0.f;
#pragma unroll
        for (int m = 0; m < D; ++m) {
          const float2 a = A[j * D + m];
          xr = fmaf(a.x, v[b][m].x, fmaf(-a.y, v[b][m].y, xr));
          xi = fmaf(a.x, v[b][m].y, fmaf(a.y, v[b][m].x, xi));
        }
        psi[base[b] | off[j]] = make_float2(xr, xi);
      }
    }
  }
}

// widths 5 and 6: one gather set per thread, its 2^w members in a local
// array (registers or, at w = 6, local memory); kept out of line so that its
// register demand does not raise that of the rest of the kernel
template <int W>
__device__ __noinline__ void cta_apply_wide(float2* psi, int n, const int* order, const float2* A) {
  constexpr int D = 1 << W;
  int sorted[W];
  for (int b = 0; b < W; ++b) sorted[b] = order[b];
  for (int i = 1; i < W; ++i)
    for (int j = i; j > 0; --j)
      if (sorted[j - 1] > sorted[j]) { const int t = sorted[j]; sorted[j] = sorted[j - 1]; sorted[j - 1] = t; }
  const uint64_t sets = 1ull << (n - W);
  for (uint64_t s = threadIdx.x; s < sets; s += blockDim.x) {
    const uint64_t base = insert_zeros(s, W, sorted);
    float2 v[D];
    for (int m = 0; m < D; ++m) {
      uint64_t o = 0;
      for (int b = 0; b < W; ++b)
        if ((m >> b) & 1) o |= 1ull << order[b];
      v[m] = psi[base | o];
    }
    for (int j = 0; j < D; ++j) {
      float xr = 0.f, xi = 0.f;
      for (int m = 0; m < D; ++m) {
        const float2 a = A[j * D + m];
        xr = fmaf(a.x, v[m].x, fmaf(-a.y, v[m].y, xr));
        xi = fmaf(a.x, v[m].y, fmaf(a.y, v[m].x, xi));
      }
      uint64_t o = 0;
      for (int b = 0; b < W; ++b)
        if ((j >> b) & 1) o |= 1ull << order[b];
      psi[base | o] = make_float2(xr, xi);
    }
  }
}

__device__ __forceinline__ uint32_t insert_zeros32(uint32_t x, int w, const int* sorted) {
  for (int b = 0; b < w; ++b) {
    const int s = sorted[b];
    x = ((x >> s) << (s + 1)) | (x & ((1u << s) - 1u));
  }
  return x;
}

// psi <- A psi for a state in global memory (n <= 20, so 32-bit indices):
// each thread gathers NL = 16 amplitudes (B = 16 / 2^W sets, 64 KB per SM of
// 512 threads) before any arithmetic, so that enough loads are in flight
// to cover DRAM latency; each matrix entry is one broadcast 128-bit shared load,
// (a.x, a.x, a.y, a.y), reused by the thread's B sets; a complex
// multiply-add is two packed FP32x2 FMAs into P = sum a.x (v.x, v.y) and
// Q = sum a.y (v.x, v.y), and the output is (P.x - Q.y, P.y + Q.x).
template <int W>
__device__ __noinline__ void cta_apply_glob(float2* __restrict__ psi, int n, const int* order,
                                            const float4* __restrict__ A4) {
  constexpr int D = 1 << W;
  constexpr int NL = 16;
  constexpr int B = NL / D;
  int sorted[W];
  uint32_t off[D];
#pragma unroll
  for (int b = 0; b < W; ++b) sorted[b] = order[b];
#pragma unroll
  for (int i = 1; i < W; ++i)
#pragma unroll
    for (int j = i; j > 0; --j)
      if (sorted[j - 1] > sorted[j]) { const int t = sorted[j]; sorted[j] = sorted[j - 1]; sorted[j - 1] = t; }
#pragma unroll
  for (int m = 0; m < D; ++m) {
    uint32_t o = 0;
#pragma unroll
    for (int b = 0; b < W; ++b)
      if ((m >> b) & 1) o |= 1u << order[b];
    off[m] = o;
  }
  const uint32_t sets = 1u << (n - W);
  const uint32_t stride = blockDim.x;
  for (uint32_t s0 = threadIdx.x; s0 < sets; s0 += B * stride) {
    uint32_t base[B];
    float2 v[B][D];
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const uint32_t sb = s0 + b * stride;
      base[b] = insert_zeros32(sb < sets ? sb : s0, W, sorted);
#pragma unroll
      for (int m = 0; m < D; ++m) v[b][m] = psi[base[b] | off[m]];
    }
    // rows one at a time: unrolling them lets the compiler hoist every
    // matrix load of the pass into registers, which spills
#pragma unroll 1
    for (int j = 0; j < D; ++j) {
      float2 P[B], Q[B];
#pragma unroll
      for (int b = 0; b < B; ++b) { P[b] = make_float2(0.f, 0.f); Q[b] = make_float2(0.f, 0.f); }
#pragma unroll
      for (int m = 0; m < D; ++m) {
        const float4 a = A4[j * D + m];
        const float2 ax = make_float2(a.x, a.y), ay = make_float2(a.z, a.w);
#pragma unroll
        for (int b = 0; b < B; ++b) {
          P[b] = __ffma2_rn(ax, v[b][m], P[b]);
          Q[b] = __ffma2_rn(ay, v[b][m], Q[b]);
        }
      }
#pragma unroll
      for (int b = 0; b < B; ++b)
        if (s0 + b * stride < sets) psi[base[b] | off[j]] = make_float2(P[b].x - Q[b].y, P[b].y + Q[b].x);
    }
  }
}

// Aglob: the matrix in global memory (scaled by `scale` while staged), or
// smat itself when the matrix was composed in shared memory (scale unused).
template <bool GLOBAL>
__device__ void cta_apply(float2* psi, int n, int w, const int* order, const float2* Aglob, float scale,
                          float2* smat) {
  const int D = 1 << w;
  const bool staged = Aglob == smat;
  __syncthreads();                     // previous users of smat / psi are done
  if (GLOBAL && w <= 4) {
    float4* A4 = reinterpret_cast<float4*>(smat + (1u << (2 * kMaxW)));
    for (int i = threadIdx.x; i < D * D; i += blockDim.x) {
      const float2 a = Aglob[i];
      const float x = staged ? a.x : a.x * scale, y = staged ? a.y : a.y * scale;
      A4[i] = make_float4(x, x, y, y);
    }
    __syncthreads();
    switch (w) {
      case 1: cta_apply_glob<1>(psi, n, order, A4); break;
      case 2: cta_apply_glob<2>(psi, n, order, A4); break;
      case 3: cta_apply_glob<3>(psi, n, order, A4); break;
      default: cta_apply_glob<4>(psi, n, order, A4); break;
    }
    return;
  }
  if (!staged) {
    for (int i = threadIdx.x; i < D * D; i += blockDim.x) {
      const float2 a = Aglob[i];
      smat[i] = make_float2(a.x * scale, a.y * scale);
    }
    __syncthreads();
  }
  if (!GLOBAL) {
    switch (w) {
      case 1: cta_apply_w<1, false>(psi, n, order, smat); return;
      case 2: cta_apply_w<2, false>(psi, n, order, smat); return;
      case 3: cta_apply_w<3, false>(psi, n, order, smat); return;
      case 4: cta_apply_w<4, false>(psi, n, order, smat); return;
      default: break;
    }
  }
  if (w == 5) cta_apply_wide<5>(psi, n, order, smat);
  else cta_apply_wide<6>(psi, n, order, smat);
}

__device__ __forceinline__ float2 cmul_add(float2 a, float2 x, float2 acc) {
  acc.x = fmaf(a.x, x.x, fmaf(-a.y, x.y, acc.x));
  acc.y = fmaf(a.x, x.y, fmaf(a.y, x.x, acc.y));
  return acc;
}

// M <- A M for the 2^q x 2^q operator A (q = 1, 2; index bit b <-> pos[b]
// among the w basis bits of M), scaled by sc: every column of M is a vector
// that A acts on, as in Alg. 1.  M is D x D row-major in shared memory.
__device__ void cta_left_apply(float2* M, int w, int q, const int* pos, const float2* A, float sc) {
  const int D = 1 << w;
  if (q == 1) {
    const float2 a00 = make_float2(A[0].x * sc, A[0].y * sc), a01 = make_float2(A[1].x * sc, A[1].y * sc);
    const float2 a10 = make_float2(A[2].x * sc, A[2].y * sc), a11 = make_float2(A[3].x * sc, A[3].y * sc);
    const int p = pos[0];
    for (int u = threadIdx.x; u < (D >> 1) * D; u += blockDim.x) {
      const int c = u & (D - 1), rr = u >> w;
      const int r0 = ((rr >> p) << (p + 1)) | (rr & ((1 << p) - 1)), r1 = r0 | (1 << p);
      const float2 x0 = M[r0 * D + c], x1 = M[r1 * D + c];
      M[r0 * D + c] = cmul_add(a01, x1, cmul_add(a00, x0, make_float2(0.f, 0.f)));
      M[r1 * D + c] = cmul_add(a11, x1, cmul_add(a10, x0, make_float2(0.f, 0.f)));
    }
    return;
  }
  const int lo = pos[0] < pos[1] ? pos[0] : pos[1], hi = pos[0] < pos[1] ? pos[1] : pos[0];
  for (int u = threadIdx.x; u < (D >> 2) * D; u += blockDim.x) {
    const int c = u & (D - 1);
    int r = u >> w;
    r = ((r >> lo) << (lo + 1)) | (r & ((1 << lo) - 1));
    r = ((r >> hi) << (hi + 1)) | (r & ((1 << hi) - 1));
    int rows[4];
    float2 x[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      rows[m] = r | ((m & 1) << pos[0]) | (((m >> 1) & 1) << pos[1]);
      x[m] = M[rows[m] * D + c];
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const float2 a = A[j * 4 + m];
        acc = cmul_add(make_float2(a.x * sc, a.y * sc), x[m], acc);
      }
      M[rows[j] * D + c] = acc;
    }
  }
}

// reduced density of (q0[, q1]) -> out[0..W) (layout of rdm_unpack); thread 0 holds the result
__device__ void cta_rdm(const float2* psi, int n, int q, const int* order, double* out, double (*red)[17]) {
  const int D = 1 << q, W = D * D;
  double acc[16];
  float f[16];
  for (int c = 0; c < 16; ++c) { acc[c] = 0.0; f[c] = 0.f; }
  int sorted[2] = {order[0], q > 1 ? order[1] : 0};
  if (q > 1 && sorted[0] > sorted[1]) { const int t = sorted[0]; sorted[0] = sorted[1]; sorted[1] = t; }
  uint64_t off[4];
  for (int m = 0; m < D; ++m) {
    uint64_t o = 0;
    for (int b = 0; b < q; ++b)
      if ((m >> b) & 1) o |= 1ull << order[b];
    off[m] = o;
  }
  const uint64_t sets = 1ull << (n - q);
  int cnt = 0;
  for (uint64_t s = threadIdx.x; s < sets; s += blockDim.x) {
    const uint64_t base = insert_zeros(s, q, sorted);
    float2 v[4];
    for (int m = 0; m < D; ++m) v[m] = psi[base | off[m]];
    int c = 0;
    for (int b = 0; b < D; ++b) { f[c] = fmaf(v[b].x, v[b].x, fmaf(v[b].y, v[b].y, f[c])); ++c; }
    for (int b = 0; b < D; ++b)
      for (int a = b + 1; a < D; ++a) {
        f[c] = fmaf(v[b].x, v[a].x, fmaf(v[b].y, v[a].y, f[c])); ++c;
        f[c] = fmaf(v[b].y, v[a].x, fmaf(-v[b].x, v[a].y, f[c])); ++c;
      }
    if (++cnt == 16) {
      for (int k = 0; k < W; ++k) { acc[k] += static_cast<double>(f[k]); f[k] = 0.f; }
      cnt = 0;
    }
  }
  for (int k = 0; k < W; ++k) acc[k] += static_cast<double>(f[k]);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int k = 0; k < W; ++k) {
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int k = 0; k < W; ++k) {
      double v = 0.0;
      for (int w2 = 0; w2 < nw; ++w2) v += red[w2][k];
      out[k] = v;
    }
  __syncthreads();
}

__device__ __forceinline__ float warp_scan_f(float v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  return v;
}

// S samples: warp w owns a contiguous range of amplitudes; C(x) inside a
// range is the running FP32 sum of 32-amplitude chunk totals plus the
// chunk's warp scan; ranges are chained by an FP64 scan of their totals
__device__ void cta_sample(const float2* psi, int n, uint64_t seed, uint64_t traj, uint32_t S, uint64_t* out,
                           double* wcum) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint64_t amps = 1ull << n;
  uint64_t per = (amps + nw - 1) / nw;
  per = (per + 31) & ~31ull;
  __syncthreads();
  {
    const uint64_t lo = warp * per;
    float run = 0.f;
    for (uint64_t c = lo; c < lo + per; c += 32) {
      const uint64_t x = c + lane;
      float w = 0.f;
      if (x < amps) { const float2 a = psi[x]; w = fmaf(a.x, a.x, a.y * a.y); }
      const float inc = warp_scan_f(w, lane);
      run += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane == 0) wcum[warp] = static_cast<double>(run);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < nw; ++w) { r += wcum[w]; wcum[w] = r; }
  }
  __syncthreads();
  const double total = wcum[nw - 1];
  for (uint32_t j = warp; j < S; j += nw) {
    const double t = uniform01(seed, traj, kStreamSample, j) * total;
    int r = 0;
    while (r < nw - 1 && !(t < wcum[r])) ++r;
    const double trel = t - (r ? wcum[r - 1] : 0.0);
    const uint64_t lo = r * per;
    float run = 0.f;
    uint64_t x = ~0ull, last_nz = lo < amps ? lo : amps - 1;
    for (uint64_t c = lo; c < lo + per; c += 32) {
      const uint64_t xx = c + lane;
      float w = 0.f;
      if (xx < amps) { const float2 a = psi[xx]; w = fmaf(a.x, a.x, a.y * a.y); }
      const float inc = warp_scan_f(w, lane);
      const float tot = __shfl_sync(0xffffffffu, inc, 31);
      const unsigned nz = __ballot_sync(0xffffffffu, w > 0.f);
      if (nz) last_nz = c + 31 - __clz(nz);
      const unsigned h = __ballot_sync(0xffffffffu, trel < static_cast<double>(run + inc));
      if (h) { x = c + __ffs(h) - 1; break; }
      run += tot;
    }
    if (x == ~0ull || x >= amps) x = last_nz;
    if (lane == 0) out[j] = x;
  }
}

// The piece of fused gate G over ops [lo, hi): its members there composed in
// FP32 into one matrix over the gate's qubits, left in s_mat (D x D
// row-major; identity on qubits none of them touches).  The channel decided
// in stage 2 at the segment's start (op pend_pos) enters as its Kraus
// operator pend_choice scaled by pend_scale; any other channel as its
// stage-1 choice.
__device__ __forceinline__ void cta_compose_piece(const Dev& d, const Traj& T, const Gate& G, uint32_t lo, uint32_t hi,
                                  int pend_pos, int pend_choice, float pend_scale, float2* s_mat) {
  const int D = 1 << G.w;
  __syncthreads();                 // previous users of s_mat are done
  for (int i = threadIdx.x; i < D * D; i += blockDim.x)
    s_mat[i] = make_float2((i >> G.w) == (i & (D - 1)) ? 1.f : 0.f, 0.f);
  for (uint32_t mi = 0; mi < G.nmem; ++mi) {
    const uint32_t pos = d.members[G.mem0 + mi];
    if (pos < lo || pos >= hi) continue;
    const Op op = d.ops[T.op0 + pos];
    const Set st = d.sets[op.set];
    const uint32_t dd = 1u << (2 * op.q);
    const float2* A;
    float sc = 1.f;
    if (op.channel < 0) {
      A = d.fmat + st.mat;
    } else if (static_cast<int>(pos) == pend_pos) {
      A = d.fmat + st.kraus + pend_choice * dd;
      sc = pend_scale;
    } else {
      A = d.fmat + st.mat + d.kraus[T.ch0 + op.channel] * dd;
    }
    int p[2] = {0, 0};
    for (int b = 0; b < G.w; ++b) {
      if (G.t[b] == op.q0) p[0] = b;
      if (op.q > 1 && G.t[b] == op.q1) p[1] = b;
    }
    __syncthreads();               // the previous member's update is complete
    cta_left_apply(s_mat, G.w, op.q, p, A, sc);
  }
}

__device__ __forceinline__ uint32_t gate_mask(const Gate& G) {
  uint32_t m = 0;
  for (int b = 0; b < G.w; ++b) m |= 1u << G.t[b];
  return m;
}

// Product-state start (the first segment, ops [0, hi)).  A piece none of
// whose qubits an earlier piece of the segment touches acts on |0> of its
// own qubits and commutes with every piece before it, so it moves to the
// front: its column U[:, 0] becomes a factor of the initial state
//   psi[x] = prod_f U_f[x restricted to the qubits of f, 0],
// zero where x has a 1 on a qubit that no folded piece holds.  The qubits
// are split at m: the factors of the pieces wholly below m form a table of
// 2^m entries, those wholly from m up one of 2^(n-m) (both in s_mat), so an
// amplitude is one product of two table entries, times the factors of the
// few pieces that straddle m (m is chosen to have the fewest).  Writes the
// whole state, marks the folded gates (gate flag 2: the pass loop of the
// first segment skips them; a later segment treats such a gate, which the
// flush point cut, as a composed piece) and returns their number.
struct FoldPiece {
  uint32_t mask;                   // its qubits
  uint32_t gate;                   // its fused gate
  uint16_t off;                    // its column in s_col
  uint8_t w, q[kMaxW];             // its qubits, basis bit b <-> q[b]
};
constexpr uint32_t kTableAmps = 1u << (2 * kMaxW);   // s_mat holds both tables

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// factor U_f[x restricted to the qubits of f, 0]
__device__ __forceinline__ float2 fold_factor(const FoldPiece& F, const float2* s_col, uint32_t x) {
  uint32_t idx = 0;
  for (int b = 0; b < F.w; ++b) idx |= ((x >> F.q[b]) & 1u) << b;
  return s_col[F.off + idx];
}

__device__ __noinline__ int cta_product_start(const Dev& d, const Traj& T, float2* psi, uint32_t hi,
                                              float2* s_mat, float2* s_col, FoldPiece* s_fold) {
  __shared__ int s_split, s_nstr;
  __shared__ uint8_t s_str[kMaxN];
  const int tid = threadIdx.x;
  const int n = static_cast<int>(T.n);
  const uint32_t all = (1u << n) - 1u;
  uint32_t touched = 0, held = 0;
  int nf = 0, off = 0;
  // once every qubit is touched no later piece can fold
  for (uint32_t g = 0; g < T.ngates && touched != all; ++g) {
    const Gate G = d.gates[T.gate0 + g];
    if (G.minpos >= hi) continue;
    const uint32_t gm = gate_mask(G);
    const bool fold = !(gm & touched);
    touched |= gm;
    if (!fold) continue;
    const int D = 1 << G.w;
    const float2* col = d.fmat + G.mat;          // column 0 of the precomputed matrix, stride D
    if (G.maxpos >= hi || d.gflag[T.gf0 + g]) {
      cta_compose_piece(d, T, G, 0, hi, -1, 0, 1.f, s_mat);
      __syncthreads();
      col = s_mat;
    }
    for (int i = tid; i < D; i += blockDim.x) s_col[off + i] = col[i * D];
    if (tid == 0) {
      FoldPiece& F = s_fold[nf];
      F.mask = gm;
      F.gate = g;
      F.off = static_cast<uint16_t>(off);
      F.w = G.w;
      for (int b = 0; b < G.w; ++b) F.q[b] = G.t[b];
    }
    held |= gm;
    off += D;
    ++nf;
  }
  __syncthreads();                 // every thread has read the gate flags; s_fold is complete
  if (tid < 32) {
    // lane c scores the split at m = c: fewest straddling pieces, then the
    // most even tables, among the splits whose tables fit s_mat
    const int c = tid;
    uint32_t key = 0xffffffffu;
    if (c <= n && (1u << c) + (1u << (n - c)) <= kTableAmps) {
      int str = 0;
      for (int f = 0; f < nf; ++f) str += (s_fold[f].mask & ((1u << c) - 1u)) && (s_fold[f].mask >> c);
      key = (static_cast<uint32_t>(str) << 16) | (static_cast<uint32_t>(abs(2 * c - n)) << 5) |
            static_cast<uint32_t>(c);
    }
    for (int o = 16; o > 0; o >>= 1) key = min(key, __shfl_xor_sync(0xffffffffu, key, o));
    if (tid == 0) {
      const int m = static_cast<int>(key & 31u);
      s_split = m;
      int ns = 0;
      for (int f = 0; f < nf; ++f)
        if ((s_fold[f].mask & ((1u << m) - 1u)) && (s_fold[f].mask >> m)) s_str[ns++] = static_cast<uint8_t>(f);
      s_nstr = ns;
    }
    // mark the folded gates for the pass loop
    for (int f = tid; f < nf; f += 32) d.gflag[T.gf0 + s_fold[f].gate] = 2;
  }
  __syncthreads();
  const int m = s_split, ns = s_nstr;
  const uint32_t lmask = (1u << m) - 1u, nlo = 1u << m, nhi = 1u << (n - m);
  const uint32_t zero = all & ~held;                 // qubits no folded piece holds stay |0>
  float2* t_lo = s_mat;
  float2* t_hi = s_mat + nlo;
  for (uint32_t y = tid; y < nlo + nhi; y += blockDim.x) {
    const bool upper = y >= nlo;
    const uint32_t x = upper ? (y - nlo) << m : y;   // the index bits this entry stands for
    const uint32_t half = upper ? ~lmask : lmask;
    float2 v = make_float2(0.f, 0.f);
    if (!(x & zero)) {
      v.x = 1.f;
      for (int f = 0; f < nf; ++f)
        if (!(s_fold[f].mask & ~half)) v = cmul(v, fold_factor(s_fold[f], s_col, x));
    }
    if (upper) t_hi[y - nlo] = v;
    else t_lo[y] = v;
  }
  __syncthreads();
  const uint64_t amps = 1ull << n;
  for (uint64_t x = tid; x < amps; x += blockDim.x) {
    const uint32_t xi = static_cast<uint32_t>(x);
    float2 v = cmul(t_lo[xi & lmask], t_hi[xi >> m]);
    for (int j = 0; j < ns; ++j) v = cmul(v, fold_factor(s_fold[s_str[j]], s_col, xi));
    psi[x] = v;
  }
  __syncthreads();                 // the marks and the state are visible to the CTA
  return nf;
}

__device__ __forceinline__ int decide_stage1(const Set& st, const double* pbar, double r) {
  double rr = r;
  for (uint32_t i = 0; i < st.nk; ++i) {
    if (rr < pbar[i]) return static_cast<int>(i);
    rr -= pbar[i];
  }
  return -1;
}

// ---------------------------------------------------------------------------
// the persistent kernel
// ---------------------------------------------------------------------------
// GLOBAL = false: the launch's trajectories have states of <= 2^14 amplitudes,
// held in the CTA's shared memory; GLOBAL = true: larger states, held in a
// per-CTA slot of global memory (shared memory then holds only the matrix)
template <bool GLOBAL>
__global__ void __launch_bounds__(512) k_batch(const __grid_constant__ Dev d) {
  extern __shared__ __align__(16) float2 s_dyn[];
  float2* s_state = s_dyn;
  float2* s_mat = GLOBAL ? s_dyn : s_dyn + (1u << kSmemNMax);   // the pass's matrix, up to 64 x 64
  __shared__ double s_red[32][17];
  __shared__ double s_rho[16];
  __shared__ double s_wcum[32];
  __shared__ unsigned s_idx;
  __shared__ int s_next;
  __shared__ float s_scale;
  __shared__ int s_pend_pos, s_pend_choice;
  __shared__ float2 s_col[kFoldCols];               // columns U[:, 0] of the folded pieces
  __shared__ FoldPiece s_fold[kMaxN];
  const int tid = threadIdx.x;

  for (;;) {
    __syncthreads();
    if (tid == 0) s_idx = atomicAdd(d.counter, 1u);
    __syncthreads();
    const unsigned k = s_idx;
    if (k >= d.num) break;
    const uint32_t ti = d.order[k];
    const Traj T = d.traj[ti];
    const int n = static_cast<int>(T.n);
    const uint64_t amps = 1ull << n;
    const uint64_t seed = d.per_traj ? T.seed : d.run[0];
    const uint64_t traj_id = d.per_traj ? T.tid : d.run[1] + ti;
    const uint32_t S = d.per_traj ? T.S : d.S;
    uint64_t* samples = d.samples + (d.per_traj ? T.soff : static_cast<uint64_t>(ti) * d.S);
    float2* psi;
    if (!GLOBAL) psi = s_state;
    else psi = d.keep ? d.arena + T.arena_off : d.arena + static_cast<uint64_t>(blockIdx.x) * d.slot_amps;
    // shared-memory states start from |0...0>; global-memory states from the
    // product state that the first segment writes (cta_product_start)
    if (!GLOBAL)
      for (uint64_t x = tid; x < amps; x += blockDim.x) psi[x] = make_float2(x == 0 ? 1.f : 0.f, 0.f);
    // stage 1 of every channel from its draw and the lower bounds
    for (uint32_t c = tid; c < T.nch; c += blockDim.x) {
      const Op op = d.ops[T.op0 + d.ch_op[T.chop0 + c]];
      const Set st = d.sets[op.set];
      const double r = uniform01(seed, traj_id, kStreamChannel, c);
      const int ch = decide_stage1(st, d.dmat + st.pbar, r);
      d.kraus[T.ch0 + c] = ch;
      d.stage[T.ch0 + c] = ch >= 0 ? 1 : 0;
    }
    if (tid == 0) { s_pend_pos = -1; s_pend_choice = 0; s_scale = 1.f; }
    __syncthreads();
    // which fused gates cannot use their precomputed matrix because a member
    // channel took a non-default stage-1 choice (or none): decided once per
    // trajectory, one gate per thread, so that the pass loop below reads one
    // flag per gate instead of chasing each member's tables
    for (uint32_t g = tid; g < T.ngates; g += blockDim.x) {
      const Gate G = d.gates[T.gate0 + g];
      uint8_t fl = 0;
      for (uint32_t mi = 0; mi < G.nmem && !fl; ++mi) {
        const Op op = d.ops[T.op0 + d.members[G.mem0 + mi]];
        if (op.channel >= 0 && d.kraus[T.ch0 + op.channel] != static_cast<int>(d.sets[op.set].def)) fl = 1;
      }
      d.gflag[T.gf0 + g] = fl;
    }
    __syncthreads();
    uint32_t lo = 0, cur_ch = 0, nflush = 0;
    for (;;) {
      // next flush point
      if (tid == 0) {
        int nx = -1;
        for (uint32_t c = cur_ch; c < T.nch; ++c)
          if (d.stage[T.ch0 + c] == 0) { nx = static_cast<int>(c); break; }
        s_next = nx;
      }
      __syncthreads();
      const int fch = s_next;
      const uint32_t hi = fch >= 0 ? d.ch_op[T.chop0 + fch] : T.nops;
      const int pend_pos = s_pend_pos, pend_choice = s_pend_choice;
      const float pend_scale = s_scale;
      // the product-state start pays on global-memory states, where a pass
      // streams the state from DRAM; on shared-memory states (passes of a few
      // microseconds) it measured slower than the passes it saves
      const bool first = GLOBAL && lo == 0 && nflush == 0;
      if constexpr (GLOBAL) {
        if (first) {
          const int nf = cta_product_start(d, T, psi, hi, s_mat, s_col, s_fold);
          if (tid == 0 && d.folds) d.folds[ti] = static_cast<uint32_t>(nf);
        }
      }
      // apply ops [lo, hi): fused gates restricted to the segment (in the
      // first segment, those not folded into the initial state)
      for (uint32_t g = 0; g < T.ngates; ++g) {
        const Gate G = d.gates[T.gate0 + g];
        if (G.maxpos < lo || G.minpos >= hi) continue;
        if (first && d.gflag[T.gf0 + g] == 2) continue;
        bool dflt = G.minpos >= lo && G.maxpos < hi && !d.gflag[T.gf0 + g];
        // the channel decided in stage 2 at this segment's start is applied as
        // its normalized Kraus operator, so the gate holding it is never default
        if (dflt && pend_pos >= 0 && static_cast<uint32_t>(pend_pos) >= G.minpos &&
            static_cast<uint32_t>(pend_pos) <= G.maxpos)
          for (uint32_t mi = 0; dflt && mi < G.nmem; ++mi)
            if (static_cast<int>(d.members[G.mem0 + mi]) == pend_pos) dflt = false;
        if (dflt) {
          int order[kMaxW];
          for (int b = 0; b < G.w; ++b) order[b] = G.t[b];
          cta_apply<GLOBAL>(psi, n, G.w, order, d.fmat + G.mat, 1.f, s_mat);
          continue;
        }
        // a piece that is cut by the segment or holds a non-default operator:
        // its members in [lo, hi) are composed in FP32 in shared memory into
        // one matrix over the gate's qubits (identity on qubits none of them
        // touches), then applied in one pass
        cta_compose_piece(d, T, G, lo, hi, pend_pos, pend_choice, pend_scale, s_mat);
        int order[kMaxW];
        for (int b = 0; b < G.w; ++b) order[b] = G.t[b];
        cta_apply<GLOBAL>(psi, n, G.w, order, s_mat, 1.f, s_mat);
      }
      if (fch < 0) break;
      // stage 2 at the flush point (Alg. 2 steps 12-20)
      {
        const Op op = d.ops[T.op0 + hi];
        const Set st = d.sets[op.set];
        int order[2] = {op.q0, op.q1};
        __syncthreads();
        cta_rdm(psi, n, op.q, order, s_rho, s_red);
        if (tid == 0) {
          const int D = 1 << op.q;
          double rho[2 * 16];
          int c = 0;
          for (int b = 0; b < D; ++b) { rho[2 * (b * D + b)] = s_rho[c++]; rho[2 * (b * D + b) + 1] = 0.0; }
          for (int b = 0; b < D; ++b)
            for (int a = b + 1; a < D; ++a) {
              const double re = s_rho[c++], im = s_rho[c++];
              rho[2 * (b * D + a)] = re; rho[2 * (b * D + a) + 1] = im;
              rho[2 * (a * D + b)] = re; rho[2 * (a * D + b) + 1] = -im;
            }
          double N = 0.0;
          for (int b = 0; b < D; ++b) N += rho[2 * (b * D + b)];
          const double* pbar = d.dmat + st.pbar;
          double rr = uniform01(seed, traj_id, kStreamChannel, static_cast<uint32_t>(fch));
          for (uint32_t i = 0; i < st.nk; ++i) rr -= pbar[i];
          int chosen = -1, last = -1, last_pos = -1;
          double Pc = 1.0;
          for (uint32_t i = 0; i < st.nk; ++i) {
            const double* M = d.dmat + st.mtm + static_cast<size_t>(i) * D * D * 2;
            double P = 0.0;                                  // tr(M rho)
            for (int a = 0; a < D; ++a)
              for (int b = 0; b < D; ++b) {
                const double mr = M[2 * (a * D + b)], mi2 = M[2 * (a * D + b) + 1];
                const double rr2 = rho[2 * (b * D + a)], ri = rho[2 * (b * D + a) + 1];
                P += mr * rr2 - mi2 * ri;
              }
            double dlt = P / N - pbar[i];
            if (dlt < 0.0) dlt = 0.0;
            if (dlt > 0.0) last = static_cast<int>(i);
            if (P > 0.0) last_pos = static_cast<int>(i);
            if (chosen < 0 && rr < dlt) { chosen = static_cast<int>(i); Pc = P; }
            if (chosen < 0) rr -= dlt;
          }
          if (chosen < 0) {
            chosen = last >= 0 ? last : (last_pos >= 0 ? last_pos : static_cast<int>(st.def));
            const double* M = d.dmat + st.mtm + static_cast<size_t>(chosen) * D * D * 2;
            Pc = 0.0;
            for (int a = 0; a < D; ++a)
              for (int b = 0; b < D; ++b)
                Pc += M[2 * (a * D + b)] * rho[2 * (b * D + a)] - M[2 * (a * D + b) + 1] * rho[2 * (b * D + a) + 1];
          }
          d.kraus[T.ch0 + fch] = chosen;
          d.stage[T.ch0 + fch] = 2;
          s_pend_pos = static_cast<int>(hi);
          s_pend_choice = chosen;
          s_scale = static_cast<float>(1.0 / sqrt(Pc > 0.0 ? Pc : 1.0));
        }
        __syncthreads();
        ++nflush;
        lo = hi;
        cur_ch = static_cast<uint32_t>(fch) + 1;
      }
    }
    __syncthreads();
    if (S) cta_sample(psi, n, seed, traj_id, S, samples, s_wcum);
    if (d.keep && !GLOBAL) {
      __syncthreads();
      for (uint64_t x = tid; x < amps; x += blockDim.x) d.arena[T.arena_off + x] = psi[x];
    }
    if (tid == 0) {
      d.flushes[ti] = nflush;
      if (!GLOBAL && d.folds) d.folds[ti] = 0;
    }
  }
}

}  // namespace bt

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

uint64_t fnv1a(const void* p, size_t n, uint64_t h = 1469598103934665603ull) {
  const uint8_t* b = static_cast<const uint8_t*>(p);
  for (size_t i = 0; i < n; ++i) { h ^= b[i]; h *= 1099511628211ull; }
  return h;
}

// a distinct operator set (gate or channel)
struct SetKey {
  uint64_t h;
  const Op* op;
};

bool same_set(const Op& a, const Op& b) {
  if (a.kind != b.kind || a.q != b.q || a.num_ops != b.num_ops) return false;
  if (a.mats.size() != b.mats.size() || std::memcmp(a.mats.data(), b.mats.data(), sizeof(cd) * a.mats.size()) != 0)
    return false;
  if (a.probs.size() != b.probs.size()) return false;
  return a.probs.empty() || std::memcmp(a.probs.data(), b.probs.data(), sizeof(double) * a.probs.size()) == 0;
}

uint64_t set_hash(const Op& op) {
  uint64_t h = fnv1a(&op.kind, sizeof(op.kind));
  h = fnv1a(&op.q, sizeof(op.q), h);
  h = fnv1a(op.mats.data(), sizeof(cd) * op.mats.size(), h);
  if (!op.probs.empty()) h = fnv1a(op.probs.data(), sizeof(double) * op.probs.size(), h);
  return h;
}

}  // namespace

struct DevMem {
  void* p = nullptr;
  size_t bytes = 0;
  ~DevMem() { if (p) cudaFree(p); }
  bool alloc(size_t b) {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = b;
    if (b == 0) return true;
    if (cudaMalloc(&p, b) != cudaSuccess) { cudaGetLastError(); p = nullptr; return false; }
    return true;
  }
};

}  // namespace qt

using namespace qt;

struct qt_batch {
  uint32_t num = 0;
  uint32_t total_ch = 0;
  uint64_t total_amps = 0;
  uint32_t max_n = 0;
  std::vector<bt::Traj> traj;
  std::vector<uint32_t> order;
  DevMem tables, arena, outs, counter;
  uint64_t* hrun = nullptr;         // pinned {seed, first_traj}; the graph copies it to counter+16
  bt::Dev dev{};
  size_t off_kraus = 0, off_stage = 0, off_samples = 0, off_flushes = 0, off_folds = 0, off_err = 0, off_gflag = 0;
  uint64_t total_gates = 0;         // sum of the trajectories' fused-gate counts (one flag each per run)
  uint32_t S = 0, keep = 0;
  std::vector<uint8_t> host;        // host image of the device tables
  uint64_t lane_samples = 0;        // merged launches: total sample slots
  qt_batch_params last{};
  // results on the host
  std::vector<int32_t> kraus, stage;
  std::vector<uint64_t> samples;
  std::vector<uint32_t> flushes, folds;
  double device_ms = 0.0;
  uint64_t gate_ops = 0, fused_gates = 0;
  // trajectories with states in global memory (n > 14) come first in `order`;
  // the two classes run as two persistent launches, the second on a side
  // stream so that its CTAs take SMs as the first launch's CTAs retire
  uint32_t nglob = 0;
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // CUDA graph of the launch sequence
  cudaGraphExec_t gexec = nullptr;
  cudaGraph_t graph = nullptr;
  uint32_t g_threads = 0, g_threads_glob = 0, g_S = 0, g_keep = 0;
  ~qt_batch() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    if (hrun) cudaFreeHost(hrun);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (side) cudaStreamDestroy(side);
  }
};

// Pack num fused circuits (trajectory i runs fused[i]) into B's host fields
// and device tables: B->tables grows when the image does not fit, and the
// image is copied with cudaMemcpyAsync on st (the call returns once the
// pageable source has been staged).  per (optional): per-trajectory seed,
// trajectory id and sample count of a merged launch.
static qt_status pack_batch(qt_batch* B, uint32_t num, const qt_fused* const* fused, const LaneTraj* per,
                            const char* who, cudaStream_t st) {
  B->num = num;
  B->total_ch = 0;
  B->total_amps = 0;
  B->max_n = 0;
  B->nglob = 0;
  B->total_gates = 0;
  B->gate_ops = 0;
  B->fused_gates = 0;
  B->traj.assign(num, bt::Traj{});
  // ---- per-circuit checks and distinct operator sets ----
  std::unordered_map<uint64_t, std::vector<uint32_t>> set_index;
  std::vector<const Op*> sets;
  std::vector<bt::Op> ops;
  std::vector<bt::Gate> gates;
  std::vector<uint32_t> members, ch_op;
  std::vector<float2> fmat;
  std::vector<double> dmat;
  std::vector<uint32_t> set_fmat, set_kraus, set_mtm, set_pbar;
  // a fused circuit that appears several times (e.g. many trajectories of one
  // request) is packed once; its trajectories share the tables
  std::unordered_map<const qt_fused*, uint32_t> first_use;
  for (uint32_t i = 0; i < num; ++i) {
    const qt_fused* f = fused[i];
    if (!f) return set_error(QT_ERR_INVALID_ARG, "%s: fused %u is NULL", who, i);
    auto seen = first_use.find(f);
    if (seen != first_use.end()) {
      const bt::Traj& P = B->traj[seen->second];
      bt::Traj& T = B->traj[i];
      T = P;
      T.ch0 = B->total_ch;                 // outputs and per-run flags are per trajectory
      B->total_ch += T.nch;
      T.gf0 = static_cast<uint32_t>(B->total_gates);
      B->total_gates += T.ngates;
      B->gate_ops += f->gate_ops;
      continue;
    }
    first_use.emplace(f, i);
    const Circuit& c = *f->c;
    if (c.n > static_cast<uint32_t>(bt::kMaxN) || c.n < 1)
      return set_error(QT_ERR_UNSUPPORTED, "%s: circuit %u has %u qubits (batched form: 1..%d)", who, i, c.n,
                       bt::kMaxN);
    bt::Traj& T = B->traj[i];
    T.n = c.n;
    T.op0 = static_cast<uint32_t>(ops.size());
    T.nops = static_cast<uint32_t>(c.ops.size());
    T.ch0 = B->total_ch;
    T.chop0 = static_cast<uint32_t>(ch_op.size());
    T.nch = static_cast<uint32_t>(c.channel_op.size());
    T.gate0 = static_cast<uint32_t>(gates.size());
    T.ngates = static_cast<uint32_t>(f->gates.size());
    T.gf0 = static_cast<uint32_t>(B->total_gates);
    B->total_gates += T.ngates;
    B->total_ch += T.nch;
    B->max_n = std::max(B->max_n, c.n);
    std::vector<uint32_t> local_sets;   // set ids by op
    // within-circuit cache: consecutive ops mostly repeat a handful of sets
    std::vector<std::pair<const Op*, uint32_t>> recent;
    for (uint32_t oi = 0; oi < c.ops.size(); ++oi) {
      const Op& op = c.ops[oi];
      if (op.q > 2) return set_error(QT_ERR_UNSUPPORTED, "%s: circuit %u op %u has %u qubits (batched form: <= 2)", who, i, oi, op.q);
      uint32_t sid = UINT32_MAX;
      for (auto& r : recent)
        if (same_set(*r.first, op)) { sid = r.second; break; }
      if (sid == UINT32_MAX) {
        const uint64_t h = set_hash(op);
        auto& bucket = set_index[h];
        for (uint32_t cand : bucket)
          if (same_set(*sets[cand], op)) { sid = cand; break; }
        if (sid == UINT32_MAX) {
          sid = static_cast<uint32_t>(sets.size());
          sets.push_back(&op);
          bucket.push_back(sid);
        }
        recent.emplace_back(&op, sid);
        if (recent.size() > 16) recent.erase(recent.begin());
      }
      bt::Op o{};
      o.kind = static_cast<uint8_t>(op.kind);
      o.q = static_cast<uint8_t>(op.q);
      o.q0 = static_cast<uint8_t>(op.qubits[0]);
      o.q1 = static_cast<uint8_t>(op.q > 1 ? op.qubits[1] : 0);
      o.set = sid;
      o.channel = op.channel;
      ops.push_back(o);
      if (op.channel >= 0) ch_op.push_back(oi);
      if (op.kind == QT_OP_GATE) B->gate_ops++;
    }
    for (const FusedGate& fg : f->gates) {
      if (fg.targets.size() > static_cast<size_t>(bt::kMaxW))
        return set_error(QT_ERR_UNSUPPORTED, "%s: fused width %zu > %d in circuit %u", who, fg.targets.size(),
                         bt::kMaxW, i);
      bt::Gate g{};
      g.w = static_cast<uint8_t>(fg.targets.size());
      for (size_t b = 0; b < fg.targets.size(); ++b) g.t[b] = static_cast<uint8_t>(fg.targets[b]);
      g.mat = static_cast<uint32_t>(fmat.size());
      for (const cd& x : fg.def) fmat.push_back(make_float2(static_cast<float>(x.real()), static_cast<float>(x.imag())));
      g.mem0 = static_cast<uint32_t>(members.size());
      g.nmem = static_cast<uint32_t>(fg.members.size());
      g.minpos = UINT32_MAX;
      g.maxpos = 0;
      for (uint32_t m : fg.members) {
        members.push_back(m);
        g.minpos = std::min(g.minpos, m);
        g.maxpos = std::max(g.maxpos, m);
      }
      gates.push_back(g);
      B->fused_gates++;
    }
    if (fmat.size() > 0x7fffffffu) return set_error(QT_ERR_UNSUPPORTED, "%s: matrix table too large", who);
  }
  // operator-set tables
  std::vector<bt::Set> dsets(sets.size());
  for (size_t s = 0; s < sets.size(); ++s) {
    const Op& op = *sets[s];
    bt::Set& S = dsets[s];
    S.nk = op.num_ops;
    S.q = op.q;
    S.def = static_cast<uint32_t>(op.def);
    S.mat = static_cast<uint32_t>(fmat.size());
    for (const cd& x : op.mats) fmat.push_back(make_float2(static_cast<float>(x.real()), static_cast<float>(x.imag())));
    S.kraus = static_cast<uint32_t>(fmat.size());
    const std::vector<cd>& kr = op.kind == QT_OP_GATE ? op.mats : op.kraus;
    for (const cd& x : kr) fmat.push_back(make_float2(static_cast<float>(x.real()), static_cast<float>(x.imag())));
    S.mtm = static_cast<uint32_t>(dmat.size());
    for (const cd& x : op.mtm) { dmat.push_back(x.real()); dmat.push_back(x.imag()); }
    S.pbar = static_cast<uint32_t>(dmat.size());
    for (double p : op.pbar) dmat.push_back(p);
    if (op.pbar.empty()) dmat.push_back(0.0);
  }
  // processing order: largest states first
  B->order.resize(num);
  for (uint32_t i = 0; i < num; ++i) B->order[i] = i;
  std::stable_sort(B->order.begin(), B->order.end(),
                   [&](uint32_t a, uint32_t b) { return B->traj[a].n > B->traj[b].n; });
  uint64_t soff = 0;
  for (uint32_t i = 0; i < num; ++i) {
    bt::Traj& T = B->traj[i];
    T.arena_off = B->total_amps;
    B->total_amps += 1ull << T.n;
    if (T.n > static_cast<uint32_t>(bt::kSmemNMax)) B->nglob++;
    T.seed = per ? per[i].seed : 0;
    T.tid = per ? per[i].traj : 0;
    T.S = per ? per[i].S : 0;
    T.soff = soff;
    soff += T.S;
  }
  B->lane_samples = soff;
  // ---- one device buffer for all tables ----
  auto align = [](size_t x) { return (x + 255) & ~size_t(255); };
  size_t off = 0;
  const size_t o_traj = off; off = align(off + sizeof(bt::Traj) * num);
  const size_t o_ops = off; off = align(off + sizeof(bt::Op) * ops.size());
  const size_t o_sets = off; off = align(off + sizeof(bt::Set) * dsets.size());
  const size_t o_gates = off; off = align(off + sizeof(bt::Gate) * std::max<size_t>(gates.size(), 1));
  const size_t o_mem = off; off = align(off + sizeof(uint32_t) * std::max<size_t>(members.size(), 1));
  const size_t o_chop = off; off = align(off + sizeof(uint32_t) * std::max<size_t>(ch_op.size(), 1));
  const size_t o_fmat = off; off = align(off + sizeof(float2) * fmat.size());
  const size_t o_dmat = off; off = align(off + sizeof(double) * std::max<size_t>(dmat.size(), 1));
  const size_t o_order = off; off = align(off + sizeof(uint32_t) * num);
  if (B->tables.bytes < off && !B->tables.alloc(off))
    return set_error(QT_ERR_OUT_OF_MEMORY, "%s: device tables (%zu bytes)", who, off);
  std::vector<uint8_t>& host = B->host;
  host.assign(off, 0);
  auto put = [&](size_t o, const void* src, size_t n) { if (n) std::memcpy(host.data() + o, src, n); };
  put(o_traj, B->traj.data(), sizeof(bt::Traj) * num);
  put(o_ops, ops.data(), sizeof(bt::Op) * ops.size());
  put(o_sets, dsets.data(), sizeof(bt::Set) * dsets.size());
  put(o_gates, gates.data(), sizeof(bt::Gate) * gates.size());
  put(o_mem, members.data(), sizeof(uint32_t) * members.size());
  put(o_chop, ch_op.data(), sizeof(uint32_t) * ch_op.size());
  put(o_fmat, fmat.data(), sizeof(float2) * fmat.size());
  put(o_dmat, dmat.data(), sizeof(double) * dmat.size());
  put(o_order, B->order.data(), sizeof(uint32_t) * num);
  cudaError_t e = cudaMemcpyAsync(B->tables.p, host.data(), off, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return set_error(QT_ERR_CUDA, "%s: cudaMemcpyAsync: %s", who, cudaGetErrorString(e));
  uint8_t* base = static_cast<uint8_t*>(B->tables.p);
  bt::Dev& d = B->dev;
  d.traj = reinterpret_cast<const bt::Traj*>(base + o_traj);
  d.ops = reinterpret_cast<const bt::Op*>(base + o_ops);
  d.sets = reinterpret_cast<const bt::Set*>(base + o_sets);
  d.gates = reinterpret_cast<const bt::Gate*>(base + o_gates);
  d.members = reinterpret_cast<const uint32_t*>(base + o_mem);
  d.ch_op = reinterpret_cast<const uint32_t*>(base + o_chop);
  d.fmat = reinterpret_cast<const float2*>(base + o_fmat);
  d.dmat = reinterpret_cast<const double*>(base + o_dmat);
  d.order = reinterpret_cast<const uint32_t*>(base + o_order);
  d.num = num;
  return QT_OK;
}

// counters, pinned run parameters, and the side stream of the second launch
static qt_status init_batch_runtime(qt_batch* B, const char* who) {
  bt::Dev& d = B->dev;
  // work counters of the two launches (2 x 4 B), error flag (4 B), run parameters at +16 (2 x 8 B)
  if (!B->counter.alloc(32)) return set_error(QT_ERR_OUT_OF_MEMORY, "%s: counter", who);
  d.counter = static_cast<unsigned int*>(B->counter.p);
  d.err = reinterpret_cast<int*>(static_cast<unsigned int*>(B->counter.p) + 2);
  d.run = reinterpret_cast<const uint64_t*>(static_cast<uint8_t*>(B->counter.p) + 16);
  if (cudaMallocHost(&B->hrun, 2 * sizeof(uint64_t)) != cudaSuccess)
    return set_error(QT_ERR_OUT_OF_MEMORY, "%s: pinned parameters", who);
  if (cudaStreamCreateWithFlags(&B->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&B->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&B->ev_join, cudaEventDisableTiming) != cudaSuccess)
    return set_error(QT_ERR_CUDA, "%s: side stream", who);
  return QT_OK;
}

// dynamic shared memory of the two launches: the matrix area (64 x 64
// complex64) and, for global states, its 16 x 16 (x, x, y, y) expansion
// behind it; the shared-memory class adds the 2^14-amplitude state
constexpr size_t kSmemMat = sizeof(float2) * (1u << (2 * bt::kMaxW)) + sizeof(float4) * 256;
constexpr size_t kSmemState = (sizeof(float2) << bt::kSmemNMax) + kSmemMat;

static cudaError_t batch_kernel_attrs() {
  static PerDevice attr_set;
  return static_cast<cudaError_t>(attr_set.get([] {
    cudaError_t e1 = cudaFuncSetAttribute(bt::k_batch<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          static_cast<int>(kSmemState));
    if (e1 == cudaSuccess)
      e1 = cudaFuncSetAttribute(bt::k_batch<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(kSmemMat));
    return static_cast<int>(e1);
  }));
}

// One run's two persistent launches on stream s, with tables, outputs and
// arena as d holds them: the work counters are zeroed, the global-memory
// class launches on s and the shared-memory class on the side stream (forked
// from and joined back into s), so that its CTAs take SMs as the first
// launch's CTAs retire.
static cudaError_t launch_classes(qt_batch* b, const bt::Dev& d, uint32_t threads, uint32_t threads_glob,
                                  cudaStream_t s) {
  const uint32_t nglob = b->nglob, nsh = b->num - b->nglob;
  const unsigned grid_g = static_cast<unsigned>(std::min<uint64_t>(sm_count(), nglob));
  const unsigned grid_s = static_cast<unsigned>(std::min<uint64_t>(sm_count(), nsh));
  bt::Dev dg = d, ds = d;
  dg.num = nglob;
  ds.order = d.order + nglob;
  ds.num = nsh;
  ds.counter = d.counter + 1;
  cudaError_t r = cudaMemsetAsync(b->counter.p, 0, 2 * sizeof(unsigned int) + sizeof(int), s);
  if (r != cudaSuccess) return r;
  const bool both = nglob && nsh;
  if (both) {
    r = cudaEventRecord(b->ev_fork, s);
    if (r == cudaSuccess) r = cudaStreamWaitEvent(b->side, b->ev_fork, 0);
    if (r != cudaSuccess) return r;
  }
  if (nglob) bt::k_batch<true><<<grid_g, threads_glob, kSmemMat, s>>>(dg);
  if (nsh) bt::k_batch<false><<<grid_s, threads, kSmemState, both ? b->side : s>>>(ds);
  r = cudaGetLastError();
  if (r == cudaSuccess && both) {
    r = cudaEventRecord(b->ev_join, b->side);
    if (r == cudaSuccess) r = cudaStreamWaitEvent(s, b->ev_join, 0);
  }
  return r;
}

extern "C" {

qt_status qt_fuse_many(uint32_t num, const qt_circuit* const* circuits, uint32_t max_fused_qubits,
                       uint32_t threads, qt_fused** out) {
  clear_error();
  if (!circuits || !out) return set_error(QT_ERR_INVALID_ARG, "qt_fuse_many: NULL argument");
  for (uint32_t i = 0; i < num; ++i) {
    out[i] = nullptr;
    if (!circuits[i]) return set_error(QT_ERR_INVALID_ARG, "qt_fuse_many: circuit %u is NULL", i);
  }
  if (max_fused_qubits > QT_MAX_FUSED_QUBITS)
    return set_error(QT_ERR_INVALID_ARG, "qt_fuse_many: max_fused_qubits %u > 6", max_fused_qubits);
  unsigned nt = threads ? threads : std::max(1u, std::thread::hardware_concurrency());
  nt = std::min<unsigned>(nt, std::max<uint32_t>(num, 1));
  std::atomic<uint32_t> next{0};
  std::atomic<int> failed{0};
  auto work = [&] {
    for (;;) {
      const uint32_t i = next.fetch_add(1);
      if (i >= num) return;
      const qt_circuit* c = circuits[i];
      uint32_t k = max_fused_qubits ? max_fused_qubits : (c->n >= 20 ? 4 : (c->n >= 12 ? 3 : 2));
      k = std::min<uint32_t>(k, c->n);
      qt_fused* f = new (std::nothrow) qt_fused();
      if (!f || fuse_circuit(*c, k, *f) != QT_OK) {
        delete f;
        failed = 1;
        continue;
      }
      out[i] = f;
    }
  };
  std::vector<std::thread> pool;
  for (unsigned t = 1; t < nt; ++t) pool.emplace_back(work);
  work();
  for (auto& t : pool) t.join();
  if (failed) {
    for (uint32_t i = 0; i < num; ++i) { delete out[i]; out[i] = nullptr; }
    return set_error(QT_ERR_INTERNAL, "qt_fuse_many: fusion failed");
  }
  return QT_OK;
}

qt_status qt_batch_create(uint32_t num, const qt_fused* const* fused, qt_batch** out) {
  clear_error();
  if (!fused || !out || num == 0) return set_error(QT_ERR_INVALID_ARG, "qt_batch_create: NULL argument or empty batch");
  *out = nullptr;
  std::unique_ptr<qt_batch> B(new (std::nothrow) qt_batch());
  if (!B) return set_error(QT_ERR_OUT_OF_MEMORY, "qt_batch_create: host allocation");
  qt_status s = pack_batch(B.get(), num, fused, nullptr, "qt_batch_create", nullptr);
  if (s == QT_OK) s = init_batch_runtime(B.get(), "qt_batch_create");
  if (s != QT_OK) return s;
  const cudaError_t e = cudaStreamSynchronize(nullptr);   // the tables are on the device
  if (e != cudaSuccess) return set_error(QT_ERR_CUDA, "qt_batch_create: %s", cudaGetErrorString(e));
  *out = B.release();
  return QT_OK;
}

qt_status qt_batch_run(qt_batch* b, const qt_batch_params* p) {
  clear_error();
  TraceRange tr("qt batched run");
  if (!b || !p) return set_error(QT_ERR_INVALID_ARG, "qt_batch_run: NULL argument");
  if (p->samples_per_traj > 1u << 20) return set_error(QT_ERR_INVALID_ARG, "qt_batch_run: samples_per_traj too large");
  const uint32_t threads = p->threads ? p->threads : 512;
  const uint32_t threads_glob = p->threads_global ? p->threads_global : threads;
  for (uint32_t t : {threads, threads_glob})
    if (t != 128 && t != 256 && t != 512)
      return set_error(QT_ERR_INVALID_ARG, "qt_batch_run: threads %u (128, 256 or 512)", t);
  cudaStream_t st = static_cast<cudaStream_t>(p->stream);
  bt::Dev& d = b->dev;
  const bool relayout = !b->outs.p || p->samples_per_traj != b->S || (p->keep_states != 0) != (b->keep != 0);
  if (relayout) {
    if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    b->S = p->samples_per_traj;
    b->keep = p->keep_states ? 1u : 0u;
    auto align = [](size_t x) { return (x + 255) & ~size_t(255); };
    size_t off = 0;
    b->off_kraus = off; off = align(off + sizeof(int32_t) * std::max<uint32_t>(b->total_ch, 1));
    b->off_stage = off; off = align(off + sizeof(int32_t) * std::max<uint32_t>(b->total_ch, 1));
    b->off_samples = off; off = align(off + sizeof(uint64_t) * std::max<uint64_t>(uint64_t(b->num) * b->S, 1));
    b->off_flushes = off; off = align(off + sizeof(uint32_t) * b->num);
    b->off_folds = off; off = align(off + sizeof(uint32_t) * b->num);
    b->off_gflag = off; off = align(off + std::max<uint64_t>(b->total_gates, 1));
    if (!b->outs.alloc(off)) return set_error(QT_ERR_OUT_OF_MEMORY, "qt_batch_run: outputs");
    uint8_t* o = static_cast<uint8_t*>(b->outs.p);
    d.kraus = reinterpret_cast<int32_t*>(o + b->off_kraus);
    d.stage = reinterpret_cast<int32_t*>(o + b->off_stage);
    d.samples = reinterpret_cast<uint64_t*>(o + b->off_samples);
    d.flushes = reinterpret_cast<uint32_t*>(o + b->off_flushes);
    d.folds = reinterpret_cast<uint32_t*>(o + b->off_folds);
    d.gflag = o + b->off_gflag;
    int sms = sm_count();
    const uint64_t slot = b->max_n > static_cast<uint32_t>(bt::kSmemNMax) ? (1ull << b->max_n) : 0;
    const uint64_t arena_amps = b->keep ? b->total_amps : slot * sms;
    if (!b->arena.alloc(sizeof(float2) * arena_amps))
      return set_error(QT_ERR_OUT_OF_MEMORY, "qt_batch_run: state arena (%llu amplitudes)",
                       static_cast<unsigned long long>(arena_amps));
    d.arena = static_cast<float2*>(b->arena.p);
    d.slot_amps = slot;
    d.keep = b->keep;
    d.S = b->S;
    b->kraus.assign(b->total_ch, 0);
    b->stage.assign(b->total_ch, 0);
    b->samples.assign(static_cast<size_t>(b->num) * b->S, 0);
    b->flushes.assign(b->num, 0);
    b->folds.assign(b->num, 0);
  }
  b->hrun[0] = p->seed;
  b->hrun[1] = p->first_traj;
  const cudaError_t attr = batch_kernel_attrs();
  if (attr != cudaSuccess) return set_error(QT_ERR_CUDA, "qt_batch_run: smem attribute: %s", cudaGetErrorString(attr));
  struct Events {                   // the run's timing events, destroyed on every return
    cudaEvent_t a = nullptr, b = nullptr;
    ~Events() {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
  } ev;
  cudaError_t e = cudaEventCreate(&ev.a);
  if (e == cudaSuccess) e = cudaEventCreate(&ev.b);
  if (e != cudaSuccess) return set_error(QT_ERR_CUDA, "qt_batch_run: cudaEventCreate: %s", cudaGetErrorString(e));
  cudaEvent_t e0 = ev.a, e1 = ev.b;
  auto enqueue = [&](cudaStream_t s) -> cudaError_t {
    cudaError_t r = cudaMemcpyAsync(static_cast<uint8_t*>(b->counter.p) + 16, b->hrun, 2 * sizeof(uint64_t),
                                    cudaMemcpyHostToDevice, s);
    if (r != cudaSuccess) return r;
    return launch_classes(b, d, threads, threads_glob, s);
  };
  e = cudaEventRecord(e0, st);
  if (e == cudaSuccess && p->use_graph && st) {
    // the graph copies the run parameters from pinned memory when it runs, so
    // it is rebuilt only when the launch shape changes
    if (b->gexec && (b->g_threads != threads || b->g_threads_glob != threads_glob)) {
      cudaGraphExecDestroy(b->gexec); b->gexec = nullptr;
      cudaGraphDestroy(b->graph); b->graph = nullptr;
    }
    if (!b->gexec) {
      e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaError_t r = enqueue(st);
        e = cudaStreamEndCapture(st, &b->graph);
        if (r != cudaSuccess) e = r;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec, b->graph, 0);
      b->g_threads = threads;
      b->g_threads_glob = threads_glob;
    }
    if (e == cudaSuccess) e = cudaGraphLaunch(b->gexec, st);
  } else if (e == cudaSuccess) {
    e = enqueue(st);
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  b->last = *p;
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->kraus.data(), d.kraus, sizeof(int32_t) * b->total_ch, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->stage.data(), d.stage, sizeof(int32_t) * b->total_ch, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && b->S)
    e = cudaMemcpyAsync(b->samples.data(), d.samples, sizeof(uint64_t) * b->samples.size(), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->flushes.data(), d.flushes, sizeof(uint32_t) * b->num, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->folds.data(), d.folds, sizeof(uint32_t) * b->num, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e != cudaSuccess) return set_error(QT_ERR_CUDA, "qt_batch_run: %s", cudaGetErrorString(e));
  b->device_ms = ms;
  return QT_OK;
}

qt_status qt_batch_samples(const qt_batch* b, uint64_t* out, size_t cap) {
  clear_error();
  if (!b || (!out && !b->samples.empty())) return set_error(QT_ERR_INVALID_ARG, "qt_batch_samples: NULL argument");
  if (cap < b->samples.size()) return set_error(QT_ERR_INVALID_ARG, "qt_batch_samples: cap %zu < %zu", cap, b->samples.size());
  if (!b->samples.empty()) std::memcpy(out, b->samples.data(), sizeof(uint64_t) * b->samples.size());
  return QT_OK;
}

qt_status qt_batch_kraus_indices(const qt_batch* b, uint32_t i, int32_t* kraus, int32_t* stage, size_t cap,
                                 uint32_t* num_channels) {
  clear_error();
  if (!b) return set_error(QT_ERR_INVALID_ARG, "qt_batch_kraus_indices: NULL batch");
  if (i >= b->num) return set_error(QT_ERR_INVALID_ARG, "qt_batch_kraus_indices: index %u out of range", i);
  const bt::Traj& T = b->traj[i];
  if (num_channels) *num_channels = T.nch;
  if ((kraus || stage) && cap < T.nch) return set_error(QT_ERR_INVALID_ARG, "qt_batch_kraus_indices: cap %zu < %u", cap, T.nch);
  if (kraus && T.nch) std::memcpy(kraus, b->kraus.data() + T.ch0, sizeof(int32_t) * T.nch);
  if (stage && T.nch) std::memcpy(stage, b->stage.data() + T.ch0, sizeof(int32_t) * T.nch);
  return QT_OK;
}

qt_status qt_batch_state(const qt_batch* b, uint32_t i, void* dst, size_t bytes) {
  clear_error();
  if (!b || !dst) return set_error(QT_ERR_INVALID_ARG, "qt_batch_state: NULL argument");
  if (!b->keep) return set_error(QT_ERR_INVALID_ARG, "qt_batch_state: the last run did not keep its states");
  if (i >= b->num) return set_error(QT_ERR_INVALID_ARG, "qt_batch_state: index %u out of range", i);
  const bt::Traj& T = b->traj[i];
  const size_t sb = sizeof(float2) << T.n;
  if (bytes < sb) return set_error(QT_ERR_INVALID_ARG, "qt_batch_state: %zu bytes < %zu", bytes, sb);
  // the kept state is un-normalized (deferred operators): normalize a device copy
  DevMem tmp, part;
  if (!tmp.alloc(sb) || !part.alloc(scratch_partial_bytes() + sizeof(double) * 64))
    return set_error(QT_ERR_OUT_OF_MEMORY, "qt_batch_state: buffers");
  Scratch scr;
  scr.partial = static_cast<double*>(part.p);
  scr.result = scr.partial + scratch_partial_bytes() / sizeof(double);
  double N = 0.0;
  cudaError_t e = cudaMemcpy(tmp.p, static_cast<float2*>(b->arena.p) + T.arena_off, sb, cudaMemcpyDeviceToDevice);
  if (e == cudaSuccess) e = launch_expect(static_cast<const float2*>(tmp.p), static_cast<int>(T.n), 0, nullptr, scr, 0);
  if (e == cudaSuccess) e = cudaMemcpy(&N, scr.result, sizeof(double), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess)
    e = launch_scale(static_cast<float2*>(tmp.p), static_cast<int>(T.n), static_cast<float>(1.0 / std::sqrt(N)), 0);
  if (e == cudaSuccess) e = cudaMemcpy(dst, tmp.p, sb, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return set_error(QT_ERR_CUDA, "qt_batch_state: %s", cudaGetErrorString(e));
  return QT_OK;
}

qt_status qt_batch_stats(const qt_batch* b, qt_batch_stats_t* out) {
  clear_error();
  if (!b || !out) return set_error(QT_ERR_INVALID_ARG, "qt_batch_stats: NULL argument");
  out->num_traj = b->num;
  out->num_channels = b->total_ch;
  out->total_amps = b->total_amps;
  out->fused_gates = b->fused_gates;
  out->gate_ops = b->gate_ops;
  uint64_t f = 0;
  for (uint32_t x : b->flushes) f += x;
  out->flushes = f;
  out->device_ms = b->device_ms;
  uint64_t fo = 0;
  for (uint32_t x : b->folds) fo += x;
  out->folded_pieces = fo;
  return QT_OK;
}

void qt_batch_destroy(qt_batch* b) { delete b; }

qt_status qt_batch_autotune(uint32_t num, const qt_circuit* const* circuits, uint32_t sample, uint32_t kmin,
                            uint32_t kmax, void* stream, qt_batch_tuning* best, double* table) {
  clear_error();
  if (!circuits || !best || num == 0)
    return set_error(QT_ERR_INVALID_ARG, "qt_batch_autotune: NULL argument or empty batch");
  kmin = std::max<uint32_t>(kmin, 1);
  kmax = std::min<uint32_t>(kmax, bt::kMaxW);
  if (kmin > kmax) return set_error(QT_ERR_INVALID_ARG, "qt_batch_autotune: empty k range");
  static const uint32_t kThreadOpts[3] = {128, 256, 512};
  const uint32_t nk = kmax - kmin + 1;
  best->k_shared = best->k_global = kmin;
  best->threads_shared = best->threads_global = 512;
  if (table)
    for (uint32_t i = 0; i < 2 * nk * 3; ++i) table[i] = 0.0;
  // the two classes of the batched kernel: states in shared memory (n <= 14)
  // and states in global memory, each tuned on a spread sample of its own
  for (int cls = 0; cls < 2; ++cls) {
    std::vector<const qt_circuit*> members;
    for (uint32_t i = 0; i < num; ++i) {
      if (!circuits[i]) return set_error(QT_ERR_INVALID_ARG, "qt_batch_autotune: circuit %u is NULL", i);
      if ((circuits[i]->n > static_cast<uint32_t>(bt::kSmemNMax)) == (cls == 1)) members.push_back(circuits[i]);
    }
    if (members.empty()) continue;
    const uint32_t nm = static_cast<uint32_t>(members.size());
    const uint32_t ns = std::max<uint32_t>(1, std::min(sample ? sample : 256u, nm));
    std::vector<const qt_circuit*> sub(ns);
    for (uint32_t i = 0; i < ns; ++i) sub[i] = members[static_cast<uint64_t>(i) * nm / ns];
    double best_ms = 1e300;
    for (uint32_t k = kmin; k <= kmax; ++k) {
      std::vector<qt_fused*> f(ns, nullptr);
      qt_status s = qt_fuse_many(ns, sub.data(), k, 0, f.data());
      if (s != QT_OK) return s;
      qt_batch* b = nullptr;
      s = qt_batch_create(ns, const_cast<const qt_fused* const*>(f.data()), &b);
      for (auto* x : f) qt_fused_destroy(x);
      if (s != QT_OK) return s;
      for (int ti = 0; ti < 3; ++ti) {
        qt_batch_params p{};
        p.seed = 0x5eed;
        p.samples_per_traj = 16;
        p.threads = kThreadOpts[ti];
        p.threads_global = kThreadOpts[ti];
        p.stream = stream;
        double ms = 0.0;
        for (int rep = 0; rep < 3 && s == QT_OK; ++rep) {
          p.first_traj = rep;
          s = qt_batch_run(b, &p);
          if (rep > 0) ms += b->device_ms;     // the first run is warm-up
        }
        if (s != QT_OK) { qt_batch_destroy(b); return s; }
        if (table) table[(cls * nk + (k - kmin)) * 3 + ti] = ms / 2.0;
        if (ms < best_ms) {
          best_ms = ms;
          if (cls == 0) { best->k_shared = k; best->threads_shared = kThreadOpts[ti]; }
          else { best->k_global = k; best->threads_global = kThreadOpts[ti]; }
        }
      }
      qt_batch_destroy(b);
    }
  }
  return QT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// merged launches of the serving form (the batch lane)
// ---------------------------------------------------------------------------
namespace qt {

struct BatchLane {
  qt_batch B;
  cudaStream_t st = nullptr;
  uint32_t max_n = 0;
  uint64_t slot = 0;                // amplitudes per global-memory state slot
  std::vector<const qt_fused*> fused;
};

qt_status lane_create(uint32_t max_n, void* stream, BatchLane** out) {
  if (!out) return set_error(QT_ERR_INVALID_ARG, "lane_create: NULL argument");
  *out = nullptr;
  if (max_n < 1 || max_n > static_cast<uint32_t>(bt::kMaxN))
    return set_error(QT_ERR_INVALID_ARG, "lane_create: max_n %u outside 1..%d", max_n, bt::kMaxN);
  std::unique_ptr<BatchLane> L(new (std::nothrow) BatchLane());
  if (!L) return set_error(QT_ERR_OUT_OF_MEMORY, "lane_create: host allocation");
  L->st = static_cast<cudaStream_t>(stream);
  L->max_n = max_n;
  qt_status s = init_batch_runtime(&L->B, "lane_create");
  if (s != QT_OK) return s;
  if (max_n > static_cast<uint32_t>(bt::kSmemNMax)) {
    L->slot = 1ull << max_n;
    if (!L->B.arena.alloc(sizeof(float2) * L->slot * sm_count()))
      return set_error(QT_ERR_OUT_OF_MEMORY, "lane_create: state slots (%u qubits)", max_n);
  }
  *out = L.release();
  return QT_OK;
}

void lane_destroy(BatchLane* l) { delete l; }

qt_status lane_run(BatchLane* L, uint32_t num, const LaneTraj* tr, uint64_t* samples, uint32_t* flushes) {
  TraceRange range("qt merged batched launch");
  if (!L || !tr || num == 0) return set_error(QT_ERR_INVALID_ARG, "lane_run: NULL argument or no trajectories");
  qt_batch* b = &L->B;
  L->fused.resize(num);
  for (uint32_t i = 0; i < num; ++i) {
    if (!tr[i].f) return set_error(QT_ERR_INVALID_ARG, "lane_run: trajectory %u has no circuit", i);
    if (tr[i].f->c->n > L->max_n)
      return set_error(QT_ERR_UNSUPPORTED, "lane_run: %u qubits > the lane's %u", tr[i].f->c->n, L->max_n);
    L->fused[i] = tr[i].f;
  }
  qt_status s = pack_batch(b, num, L->fused.data(), tr, "lane_run", L->st);
  if (s != QT_OK) return s;
  auto align = [](size_t x) { return (x + 255) & ~size_t(255); };
  size_t off = 0;
  const size_t o_kraus = off; off = align(off + sizeof(int32_t) * std::max<uint32_t>(b->total_ch, 1));
  const size_t o_stage = off; off = align(off + sizeof(int32_t) * std::max<uint32_t>(b->total_ch, 1));
  const size_t o_samp = off; off = align(off + sizeof(uint64_t) * std::max<uint64_t>(b->lane_samples, 1));
  const size_t o_flush = off; off = align(off + sizeof(uint32_t) * num);
  const size_t o_gflag = off; off = align(off + std::max<uint64_t>(b->total_gates, 1));
  if (b->outs.bytes < off && !b->outs.alloc(off)) return set_error(QT_ERR_OUT_OF_MEMORY, "lane_run: outputs");
  uint8_t* o = static_cast<uint8_t*>(b->outs.p);
  bt::Dev d = b->dev;
  d.kraus = reinterpret_cast<int32_t*>(o + o_kraus);
  d.stage = reinterpret_cast<int32_t*>(o + o_stage);
  d.samples = reinterpret_cast<uint64_t*>(o + o_samp);
  d.flushes = reinterpret_cast<uint32_t*>(o + o_flush);
  d.folds = nullptr;
  d.gflag = o + o_gflag;
  d.arena = static_cast<float2*>(b->arena.p);
  d.slot_amps = L->slot;
  d.keep = 0;
  d.S = 0;
  d.per_traj = 1;
  cudaError_t e = batch_kernel_attrs();
  if (e == cudaSuccess) e = launch_classes(b, d, 512, 512, L->st);
  if (e == cudaSuccess && b->lane_samples)
    e = cudaMemcpyAsync(samples, d.samples, sizeof(uint64_t) * b->lane_samples, cudaMemcpyDeviceToHost, L->st);
  if (e == cudaSuccess && flushes)
    e = cudaMemcpyAsync(flushes, d.flushes, sizeof(uint32_t) * num, cudaMemcpyDeviceToHost, L->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(L->st);
  if (e != cudaSuccess) return set_error(QT_ERR_CUDA, "lane_run: %s", cudaGetErrorString(e));
  return QT_OK;
}

}  // namespace qt
