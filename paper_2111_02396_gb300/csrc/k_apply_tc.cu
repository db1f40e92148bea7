// Fused-gate application on the 5th-generation tensor cores (tcgen05) for
// wide fused gates (k = 5, 6), in split-TF32 with FP32 accumulation.
//
// Alg. 1 over a batch of gather sets is a dense contraction: with the 2^k
// amplitudes of a set interleaved as 2^(k+1) reals a, the output set is
// W a, W the real embedding of U (entry (j, m) of U = c + i d becomes the
// 2x2 block [[c, -d], [d, c]]).  A tile of 128 sets is the matrix
// A [128 x K] (K = 2^(k+1)), and D = A B with B = W^T [K x N], N = K.
// Sec. III.A counts 2^(q-1) flop per byte: 32 at q = 6, well above what
// CUDA cores sustain at HBM speed, so the contraction goes to tcgen05.mma.
//
// Precision: each FP32 operand x is split into x_hi = tf32(x) and
// x_lo = tf32(x - x_hi); D = A_hi B_hi + A_hi B_lo + A_lo B_hi accumulates
// in FP32 (the three-pass split-TF32 scheme, Ootomo & Yokota 2022), which
// leaves only the A_lo B_lo term (~2^-22 relative) out.
//
// Data flow (one persistent CTA per SM, 10 warps):
//   warp 9     producer: stages each tile of 128 gather sets in shared memory
//              with bulk asynchronous copies (cp.async.bulk, one per row of
//              2^C >= 128 contiguous amplitudes; the row holds every low
//              target), completing on a transaction-count mbarrier; 8 tile
//              buffers for k = 4, 4 for k = 5, and for k = 6 (B takes 128 KB)
//              one buffer staged as two chunk halves;
//   warps 0-3  converters: thread t owns set t of the tile (TMEM lane t); it
//              reads a chunk of its members from the staged tile into
//              registers, hands the staged bytes back to the producer, waits
//              for its TMEM slot, splits hi/lo, and writes A to TMEM with
//              tcgen05.st (A operand taken from TMEM);
//   warp 8     MMA issuer: one elected thread issues tcgen05.mma (M=128,
//              N=2^(k+1), K=8 per instruction) with A in TMEM and B in
//              shared memory, and commits to mbarriers;
//   warps 4-7  epilogue: tcgen05.ld of the accumulator rows, stores of the
//              output sets (consecutive threads, consecutive sets).
// How the converters and the epilogue address amplitudes (single 8-byte
// members, 16-byte member pairs, or 16-byte set pairs exchanged by shuffles)
// is a template parameter chosen per target pattern (see MODE below).
// TMEM (512 columns): two A slots of 128 columns (hi at +0, lo at +64; one
// chunk of up to 32 members) and two accumulators of N columns (at 256 and
// 256 + N), so conversion, MMA and draining overlap while the next tile's
// bytes are in flight.
//
// B (hi and lo) is staged once per CTA in shared memory in the K-major
// no-swizzle layout: core matrices of 8 rows x 16 bytes; adjacent core
// matrices along K are LBO = 128 bytes apart, along N SBO = 128 * K/4 bytes.
//
// Every mbarrier wait is bounded: on timeout the kernel sets *err, waits
// (bounded) for its own MMAs to drain, frees its TMEM and returns.
#include <cuda_runtime.h>

#include <mutex>

#include "kernels.h"

namespace qt {

namespace tc {

constexpr int kThreads = 320;           // 10 warps
constexpr int kTileSets = 128;          // M
constexpr int kMaxChunkReals = 64;      // K per A slot (up to 32 members)
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kSpinLimit = 1u << 21;   // x <= 1 us suspend per try -> ~2 s bound
constexpr uint32_t kSuspendNs = 1000;       // suspend-time hint of one try_wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// one bounded try: the thread is suspended until the phase completes or the
// hint (ns) runs out, so a waiter wakes when its data lands instead of after
// a fixed sleep
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.b32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendNs)
      : "memory");
  return ok != 0;
}

// teardown wait: keeps waiting even after another role has set *err (the
// operations it waits for are this CTA's own), bounded by the spin limit
__device__ __forceinline__ bool mbar_drain(uint64_t* bar, uint32_t parity, int* err, int code) {
  for (uint32_t it = 0; it < kSpinLimit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
  }
  atomicOr(err, code);
  return false;
}

// bounded wait; false on timeout (and *err is set) or when another role has
// already reported an error
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err, int code) {
  for (uint32_t it = 0; it < kSpinLimit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*reinterpret_cast<volatile int*>(err)) return false;
  }
  atomicOr(err, code);
  return false;
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// global -> shared bulk copy of `bytes` (16-byte aligned, multiple of 16),
// completing on `bar`
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// a wait's outcome, made the same for the whole warp when the warp then
// exchanges values with shuffles (every lane must reach them)
template <bool UNIFORM>
__device__ __forceinline__ bool warp_ok(bool ok) {
  if constexpr (UNIFORM) return __all_sync(0xffffffffu, ok);
  else return ok;
}

// x = hi + lo, both TF32 (the split of the three-pass scheme)
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - __uint_as_float(hi));
}

// 32 consecutive 32-bit columns of this thread's lane
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
      "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
      "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]),
      "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]),
      "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
      : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr)
      : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// D[tmem] (+)= A[tmem] * B[smem desc]
__device__ __forceinline__ void mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// shared-memory matrix descriptor, K-major, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((addr >> 4) & 0x3FFFu);
  d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
  d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
  d |= 1ull << 46;          // descriptor version for tcgen05
  return d;                 // base offset 0, layout type 0 (no swizzle)
}

// instruction descriptor: D f32, A/B tf32, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

}  // namespace tc

template <int K>
struct TcArgs {
  uint64_t roff[1 << K];     // memory offset of tile row r (high-target bits)
  uint32_t moff[1 << K];     // tile-local offset of member m
  uint32_t tins[K];          // tile-local target positions, ascending
  uint32_t hins[K];          // memory positions of the high targets, ascending
  int nh, C;                 // high targets; contiguous low bits per row
  uint64_t num_tiles;        // tiles of 128 sets
  const float* bmat;         // W row-major [N x N] FP32 (N = 2^(K+1)), device
  int* err;                  // device error flag
  uint32_t lbo, sbo;         // B descriptor offsets (bytes)
};

// MODE selects how the converters and the epilogue move amplitudes between
// the staged tile, TMEM and the state (a template parameter, so that each
// target pattern runs code without the others' branches):
//   kMemberPairs: qubit 0 is a target (member bit 0 sits at offset 0), so
//     members 2j and 2j + 1 of a set are adjacent, 16-byte aligned
//     amplitudes (the set's own offset has bit 0 clear): one 16-byte access
//     each;
//   kSetPairs: qubit 0 is not a target, so the sets of threads 2i and 2i + 1
//     (TMEM lanes 2i, 2i + 1) differ only in amplitude bit 0: member m of both
//     is one 16-byte chunk.  The even thread takes the chunk of member m, the
//     odd one that of member m + 1, and one shuffle swaps the halves each
//     needs; the epilogue writes the same chunks after the reverse swap.
//     Half the shared-memory wavefronts and global store instructions of
//     single 8-byte accesses where low targets make them conflict;
//   kSingle: 8-byte accesses, one member at a time.
constexpr int kSingle = 0, kMemberPairs = 1, kSetPairs = 2;

template <int K, int MODE>
__global__ void __launch_bounds__(tc::kThreads, 1) k_apply_tc(float2* __restrict__ psi, const __grid_constant__ TcArgs<K> a) {
  using namespace tc;
  constexpr int NM = 1 << K;                 // members per set
  constexpr int N = 2 * NM;                  // reals per set = K dim = N dim
  constexpr int CR = N < kMaxChunkReals ? N : kMaxChunkReals;   // reals per A chunk
  constexpr int NCHUNK = N / CR;             // A chunks per tile (1 or 2)
  constexpr int MPC = CR / 2;                // members per chunk (16 or 32)
  constexpr int TILE_AMPS = kTileSets * NM;
  constexpr int NBUF = K >= 6 ? 1 : (K == 5 ? 4 : 8);   // staged tiles (bytes in flight)
  constexpr int RING = 3;                    // split mode: chunk-half buffers in a ring
  constexpr int TBUF_AMPS = (NBUF * TILE_AMPS > RING * TILE_AMPS / 2) ? NBUF * TILE_AMPS : RING * TILE_AMPS / 2;
  constexpr uint32_t IDESC = idesc_tf32(kTileSets, N);
  extern __shared__ __align__(1024) uint8_t smem[];
  float* bhi = reinterpret_cast<float*>(smem);
  float* blo = bhi + N * N;
  float2* tbuf = reinterpret_cast<float2*>(blo + N * N);          // NBUF tiles, or RING chunk halves
  uint64_t* bars = reinterpret_cast<uint64_t*>(tbuf + TBUF_AMPS);
  uint64_t* a_full = bars;         // [2]
  uint64_t* a_empty = bars + 2;    // [2]
  uint64_t* d_full = bars + 4;     // [2]
  uint64_t* d_empty = bars + 6;    // [2]
  uint64_t* t_full = bars + 8;     // [8] tile staged (transaction bytes)
  uint64_t* t_empty = bars + 16;   // [8] tile read by the converters
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 24);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rowmask = (1u << a.C) - 1u;
  const uint32_t rowbytes = static_cast<uint32_t>(sizeof(float2)) << a.C;
  const int nrows = 1 << a.nh;

  // stage B = W^T (hi, lo) in the K-major core-matrix layout: element
  // (n, k) of row n of W at (n/8)*SBO + (k/4)*LBO + (n%8)*16 + (k%4)*4
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) {
    const int n = i / N, k = i % N;
    const float w = a.bmat[i];
    const float hi = __uint_as_float(to_tf32(w));
    const float lo = __uint_as_float(to_tf32(w - hi));
    const uint32_t off = (n >> 3) * a.sbo + (k >> 2) * a.lbo + (n & 7) * 16 + (k & 3) * 4;
    *reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(bhi) + off) = hi;
    *reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(blo) + off) = lo;
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&a_full[i], 128);
      mbar_init(&a_empty[i], 1);
      mbar_init(&d_full[i], 1);
      mbar_init(&d_empty[i], 128);
    }
    for (int i = 0; i < 8; ++i) {
      mbar_init(&t_full[i], 1);
      mbar_init(&t_empty[i], 128);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // make the generic-proxy B stores visible to the tensor core (async proxy)
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 8) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t a_col0 = 0, d_col0 = 256;

  // k = 6: when the top target is a high qubit, chunk c of a tile is exactly
  // the half of its rows whose top row bit is c, so the two halves of the
  // single tile buffer are staged and released independently
  const bool split = NCHUNK == 2 && a.nh >= 1 && a.tins[K - 1] == static_cast<uint32_t>(a.C + a.nh - 1);
  if (warp == 9) {
    // ---------------- producer: bulk copies of the tile rows ----------------
    // lane 0 waits for a free buffer and sets its transaction count; then the
    // warp's 32 lanes issue the unit's row copies together (up to 64 rows)
    {
      uint32_t lastuse[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      int issued[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      // stage units: whole tiles (several buffers), or for k = 6 with a high
      // top target the two chunk halves of one tile buffer
      uint32_t it = 0;
      const int nunits = split ? 2 : 1;
      const int urows = nrows / nunits;
      const uint32_t ubytes = static_cast<uint32_t>(sizeof(float2) * TILE_AMPS) / nunits;
      bool stop = false;
      for (uint64_t tile = blockIdx.x; tile < a.num_tiles && !stop; tile += gridDim.x, ++it) {
        uint64_t base = tile << a.C;
        for (int j = 0; j < a.nh; ++j) {
          const uint32_t h = a.hins[j];
          base = ((base >> h) << (h + 1)) | (base & ((1ull << h) - 1ull));
        }
        for (int u = 0; u < nunits; ++u) {
          // split: chunk half g = 2 it + u goes to ring slot g % RING
          const uint32_t g = 2u * it + static_cast<uint32_t>(u);
          const uint32_t b = split ? g % RING : it % NBUF;
          const uint32_t use = split ? g / RING : it / NBUF;
          int go = 1;
          if (lane == 0) {
            if (use > 0 && !mbar_wait(&t_empty[b], (use - 1) & 1, a.err, 32)) go = 0;
            else mbar_expect_tx(&t_full[b], ubytes);
          }
          go = __shfl_sync(0xffffffffu, go, 0);      // also orders the copies after expect_tx
          if (!go) { stop = true; break; }
          float2* dst = split ? tbuf + b * (TILE_AMPS / 2) : tbuf + b * TILE_AMPS;
          for (int r = lane; r < urows; r += 32)
            bulk_g2s(dst + (static_cast<uint32_t>(r) << a.C), psi + (base | a.roff[u * urows + r]), rowbytes,
                     &t_full[b]);
          lastuse[b] = use;
          issued[b] = 1;
        }
      }
      // no copy may outlive the CTA: wait (bounded) for the last staged units
      if (lane == 0)
        for (int b = 0; b < 8; ++b)
          if (issued[b]) mbar_drain(&t_full[b], lastuse[b] & 1, a.err, 128);
    }
    __syncwarp();
  } else if (warp < 4) {
    // ---------------- converters ----------------
    const uint32_t lane_base = static_cast<uint32_t>(warp * 32) << 16;
    const bool odd = lane & 1;
    uint32_t sbase = threadIdx.x;
#pragma unroll
    for (int b = 0; b < K; ++b) {
      const uint32_t t = a.tins[b];
      sbase = ((sbase >> t) << (t + 1)) | (sbase & ((1u << t) - 1u));
    }
    uint32_t chunk_iter = 0, it = 0;
    bool ok = true;
    for (uint64_t tile = blockIdx.x; tile < a.num_tiles && ok; tile += gridDim.x, ++it) {
      const uint32_t b = split ? 0u : it % NBUF;
      if (!split && !warp_ok<MODE == kSetPairs>(mbar_wait(&t_full[b], (it / NBUF) & 1, a.err, 64))) break;
      const float2* tb = tbuf + b * TILE_AMPS;
      // chunk and column-block loops stay rolled: four roles of one CTA run
      // different code, and the smaller kernel measured faster
#pragma unroll 1
      for (int c = 0; c < NCHUNK; ++c, ++chunk_iter) {
        // split: this chunk half sits in ring slot chunk_iter % RING; its members'
        // tile offsets carry the top target bit (TILE_AMPS / 2) when c = 1
        const uint32_t rs = chunk_iter % RING;
        uint32_t tsub = 0;                   // tile offset of the staged unit's first amplitude
        if (split) {
          if (!warp_ok<MODE == kSetPairs>(mbar_wait(&t_full[rs], (chunk_iter / RING) & 1, a.err, 64))) {
            ok = false;
            break;
          }
          tb = tbuf + rs * (TILE_AMPS / 2);
          tsub = static_cast<uint32_t>(c) * (TILE_AMPS / 2);
        }
        // this chunk's members of the thread's set, read from the staged tile
        // before waiting for the TMEM slot (the reads do not depend on it)
        float2 val[MPC];
        if constexpr (MODE == kSetPairs) {
#pragma unroll
          for (int m = 0; m < MPC; m += 2) {
            const int i = c * MPC + m;
            const uint32_t mo = odd ? a.moff[i + 1] : a.moff[i];
            const float4 v = *reinterpret_cast<const float4*>(tb + (((sbase & ~1u) | mo) - tsub));
            // even: (x, y) is its member m, (z, w) the odd thread's member m;
            // odd: (z, w) is its member m + 1, (x, y) the even thread's
            const float rx = __shfl_xor_sync(0xffffffffu, odd ? v.x : v.z, 1);
            const float ry = __shfl_xor_sync(0xffffffffu, odd ? v.y : v.w, 1);
            val[m] = odd ? make_float2(rx, ry) : make_float2(v.x, v.y);
            val[m + 1] = odd ? make_float2(v.z, v.w) : make_float2(rx, ry);
          }
        } else if constexpr (MODE == kMemberPairs) {
          // members 2j and 2j + 1 are adjacent amplitudes: one 16-byte load
#pragma unroll
          for (int m = 0; m < MPC; m += 2) {
            const float4 v = *reinterpret_cast<const float4*>(tb + ((sbase | a.moff[c * MPC + m]) - tsub));
            val[m] = make_float2(v.x, v.y);
            val[m + 1] = make_float2(v.z, v.w);
          }
        } else {
#pragma unroll
          for (int m = 0; m < MPC; ++m) val[m] = tb[(sbase | a.moff[c * MPC + m]) - tsub];
        }
        // the staged bytes are in registers: hand the buffer back to the producer
        if (split) mbar_arrive(&t_empty[rs]);                       // this chunk half
        else if (c == NCHUNK - 1) mbar_arrive(&t_empty[b]);         // the tile's last chunk
        const uint32_t slot = chunk_iter & 1;
        const uint32_t use = chunk_iter >> 1;
        if (use > 0 && !warp_ok<MODE == kSetPairs>(mbar_wait(&a_empty[slot], (use - 1) & 1, a.err, 1))) {
          ok = false;
          break;
        }
#pragma unroll
        for (int half = 0; half < MPC / 16; ++half) {
          uint32_t hi[32], lo[32];
#pragma unroll
          for (int m = 0; m < 16; ++m) {
            split_tf32(val[half * 16 + m].x, hi[2 * m], lo[2 * m]);
            split_tf32(val[half * 16 + m].y, hi[2 * m + 1], lo[2 * m + 1]);
          }
          const uint32_t col = a_col0 + slot * 128 + half * 32;
          tmem_st32(tmem + lane_base + col, hi);
          tmem_st32(tmem + lane_base + col + 64, lo);
        }
        tmem_wait_st();
        fence_before();
        mbar_arrive(&a_full[slot]);
      }
    }
  } else if (warp < 8) {
    // ---------------- epilogue ----------------
    const int w4 = warp - 4;
    const uint32_t lane_base = static_cast<uint32_t>(w4 * 32) << 16;
    const bool odd = lane & 1;
    uint32_t sbase = static_cast<uint32_t>(w4 * 32 + lane);
#pragma unroll
    for (int b = 0; b < K; ++b) {
      const uint32_t t = a.tins[b];
      sbase = ((sbase >> t) << (t + 1)) | (sbase & ((1u << t) - 1u));
    }
    uint32_t iter = 0;
    for (uint64_t tile = blockIdx.x; tile < a.num_tiles; tile += gridDim.x, ++iter) {
      const uint32_t db = iter & 1;
      if (!warp_ok<MODE == kSetPairs>(mbar_wait(&d_full[db], (iter >> 1) & 1, a.err, 2))) break;
      fence_after();
      uint64_t base = tile << a.C;
      for (int j = 0; j < a.nh; ++j) {
        const uint32_t h = a.hins[j];
        base = ((base >> h) << (h + 1)) | (base & ((1ull << h) - 1ull));
      }
      // accumulator columns in blocks of 32, two loads in flight per wait
#pragma unroll 1
      for (int cb = 0; cb < N / 32; cb += 2) {
        uint32_t v[2][32];
        tmem_ld32(tmem + lane_base + d_col0 + db * N + cb * 32, v[0]);
        if (cb + 1 < N / 32) tmem_ld32(tmem + lane_base + d_col0 + db * N + (cb + 1) * 32, v[1]);
        tmem_wait_ld();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (cb + h >= N / 32) break;
          if constexpr (MODE == kSetPairs) {
#pragma unroll
            for (int j = 0; j < 16; j += 2) {
              const int i = (cb + h) * 16 + j;
              const float2 mj = make_float2(__uint_as_float(v[h][2 * j]), __uint_as_float(v[h][2 * j + 1]));
              const float2 mj1 = make_float2(__uint_as_float(v[h][2 * j + 2]), __uint_as_float(v[h][2 * j + 3]));
              // the even thread writes member j of both sets, the odd one member j + 1
              const float rx = __shfl_xor_sync(0xffffffffu, odd ? mj.x : mj1.x, 1);
              const float ry = __shfl_xor_sync(0xffffffffu, odd ? mj.y : mj1.y, 1);
              const uint32_t l = (sbase & ~1u) | (odd ? a.moff[i + 1] : a.moff[i]);
              __stcs(reinterpret_cast<float4*>(psi + (base | a.roff[l >> a.C] | (l & rowmask))),
                     odd ? make_float4(rx, ry, mj1.x, mj1.y) : make_float4(mj.x, mj.y, rx, ry));
            }
          } else if constexpr (MODE == kMemberPairs) {
#pragma unroll
            for (int j = 0; j < 16; j += 2) {
              const uint32_t l = sbase | a.moff[(cb + h) * 16 + j];
              __stcs(reinterpret_cast<float4*>(psi + (base | a.roff[l >> a.C] | (l & rowmask))),
                     make_float4(__uint_as_float(v[h][2 * j]), __uint_as_float(v[h][2 * j + 1]),
                                 __uint_as_float(v[h][2 * j + 2]), __uint_as_float(v[h][2 * j + 3])));
            }
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const uint32_t l = sbase | a.moff[(cb + h) * 16 + j];
              __stcs(psi + (base | a.roff[l >> a.C] | (l & rowmask)),
                     make_float2(__uint_as_float(v[h][2 * j]), __uint_as_float(v[h][2 * j + 1])));
            }
          }
        }
      }
      fence_before();
      mbar_arrive(&d_empty[db]);
    }
  } else {
    // ---------------- MMA issuer (warp 8) ----------------
    uint32_t chunk_iter = 0, iter = 0;
    const uint32_t bhi_addr = smem_u32(bhi), blo_addr = smem_u32(blo);
    bool ok = true;
    for (uint64_t tile = blockIdx.x; tile < a.num_tiles && ok; tile += gridDim.x, ++iter) {
      const uint32_t db = iter & 1;
      if (iter >= 2 && !mbar_wait(&d_empty[db], ((iter >> 1) - 1) & 1, a.err, 4)) { ok = false; break; }
      const uint32_t d_tmem = tmem + d_col0 + db * N;
      for (int c = 0; c < NCHUNK; ++c, ++chunk_iter) {
        const uint32_t slot = chunk_iter & 1;
        if (!mbar_wait(&a_full[slot], (chunk_iter >> 1) & 1, a.err, 8)) { ok = false; break; }
        fence_after();
        if (lane == 0) {
#pragma unroll
          for (int kk = 0; kk < CR / 8; ++kk) {
            const int kglob = c * CR + kk * 8;                           // K offset in B
            const uint32_t a_hi = tmem + a_col0 + slot * 128 + kk * 8;
            const uint32_t a_lo = a_hi + 64;
            const uint64_t dhi = smem_desc(bhi_addr + (kglob >> 2) * a.lbo, a.lbo, a.sbo);
            const uint64_t dlo = smem_desc(blo_addr + (kglob >> 2) * a.lbo, a.lbo, a.sbo);
            mma_ts(d_tmem, a_hi, dhi, IDESC, (c > 0 || kk > 0) ? 1u : 0u);
            mma_ts(d_tmem, a_hi, dlo, IDESC, 1u);
            mma_ts(d_tmem, a_lo, dhi, IDESC, 1u);
          }
          mma_commit(&a_empty[slot]);
        }
        __syncwarp();
      }
      if (!ok) break;
      if (lane == 0) mma_commit(&d_full[db]);
      __syncwarp();
    }
  }
  // teardown: a last commit on a private barrier covers every MMA this CTA
  // issued; wait for it (bounded) before freeing TMEM.  The producer's copies
  // have all completed: every staged tile was waited for by the converters,
  // or the kernel is on its error path after a bounded wait.
  __syncthreads();
  if (warp == 8) {
    __shared__ uint64_t drain;
    if (lane == 0) {
      mbar_init(&drain, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      mma_commit(&drain);
    }
    __syncwarp();
    if (lane == 0) mbar_drain(&drain, 0, a.err, 16);
    __syncwarp();
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// Set pairs pay where a warp's 8-byte accesses conflict 8-way or worse: a
// 128-byte line of banks holds 16 amplitudes, so a half-warp's sets spread
// over 2^(non-targets among amplitude bits 0..3) bank offsets, which is 2
// when bits 1, 2 and 3 are all targets.  With 4-way conflicts or fewer the
// extra shuffles cost more than the wavefronts they save (measured).
template <int K>
static bool set_pairs_pay(const uint32_t* targets) {
  int low = 0;
  for (int b = 0; b < K; ++b) low += targets[b] >= 1u && targets[b] <= 3u;
  return low == 3;
}

template <int K>
static cudaError_t launch_tc_k(float2* psi, int n, const uint32_t* targets, const float* wdev, int* err,
                               cudaStream_t st, uint32_t lbo_override, uint32_t sbo_override) {
  constexpr int NM = 1 << K;
  constexpr int N = 2 * NM;
  constexpr int NBUF = K >= 6 ? 1 : (K == 5 ? 4 : 8);
  constexpr int TILE_AMPS = tc::kTileSets * NM;
  constexpr int TBUF_AMPS = (NBUF * TILE_AMPS > 3 * TILE_AMPS / 2) ? NBUF * TILE_AMPS : 3 * TILE_AMPS / 2;
  const size_t smem = 2 * sizeof(float) * N * N + TBUF_AMPS * sizeof(float2) + 24 * sizeof(uint64_t) + 16;
  static PerDevice attr_set;
  const cudaError_t attr_err = static_cast<cudaError_t>(attr_set.get([&] {
    cudaError_t e = cudaFuncSetAttribute(k_apply_tc<K, kSingle>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_apply_tc<K, kMemberPairs>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               static_cast<int>(smem));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_apply_tc<K, kSetPairs>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               static_cast<int>(smem));
    return static_cast<int>(e);
  }));
  if (attr_err != cudaSuccess) return attr_err;
  TcArgs<K> a;
  // tile: 2^nh rows of 2^C contiguous amplitudes, C = 7 + targets below C
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
  for (int b = 0; b < K; ++b) a.tins[b] = tpos[b];
  for (int m = 0; m < NM; ++m) {
    uint32_t o = 0;
    for (int b = 0; b < K; ++b)
      if ((m >> b) & 1) o |= 1u << tpos[b];
    a.moff[m] = o;
    uint64_t r = 0;
    for (int j = 0; j < nh; ++j)
      if ((m >> j) & 1) r |= 1ull << a.hins[j];
    a.roff[m] = m < (1 << nh) ? r : 0;
  }
  a.num_tiles = 1ull << (n - C - nh);
  a.bmat = wdev;
  a.err = err;
  a.lbo = lbo_override ? lbo_override : 128;
  a.sbo = sbo_override ? sbo_override : 128 * (N / 4);
  uint64_t grid = static_cast<uint64_t>(sm_count());
  if (grid > a.num_tiles) grid = a.num_tiles;
  if (a.moff[1] == 1u)            // qubit 0 is a target (targets ascending)
    k_apply_tc<K, kMemberPairs><<<static_cast<unsigned>(grid), tc::kThreads, smem, st>>>(psi, a);
  else if (set_pairs_pay<K>(targets))
    k_apply_tc<K, kSetPairs><<<static_cast<unsigned>(grid), tc::kThreads, smem, st>>>(psi, a);
  else
    k_apply_tc<K, kSingle><<<static_cast<unsigned>(grid), tc::kThreads, smem, st>>>(psi, a);
  return cudaGetLastError();
}

bool tc_supported(int n, int k) { return k >= 4 && k <= 6 && n >= k + 7; }

cudaError_t launch_apply_tc(float2* psi, int n, int k, const uint32_t* targets, const float* wdev, int* err,
                            cudaStream_t st, uint32_t lbo, uint32_t sbo) {
  if (!tc_supported(n, k)) return cudaErrorInvalidValue;
  if (k == 4) return launch_tc_k<4>(psi, n, targets, wdev, err, st, lbo, sbo);
  if (k == 5) return launch_tc_k<5>(psi, n, targets, wdev, err, st, lbo, sbo);
  return launch_tc_k<6>(psi, n, targets, wdev, err, st, lbo, sbo);
}

void real_embedding(int k, const float2* U, float* W) {
  const int NM = 1 << k, N = 2 * NM;
  for (int j = 0; j < NM; ++j)
    for (int m = 0; m < NM; ++m) {
      const float c = U[j * NM + m].x, d = U[j * NM + m].y;
      W[(2 * j) * N + 2 * m] = c;
      W[(2 * j) * N + 2 * m + 1] = -d;
      W[(2 * j + 1) * N + 2 * m] = d;
      W[(2 * j + 1) * N + 2 * m + 1] = c;
    }
}

}  // namespace qt
