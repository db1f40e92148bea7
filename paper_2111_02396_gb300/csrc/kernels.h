// Launchers of the sm_103a kernels (host-callable, C++ linkage).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include <nvtx3/nvToolsExt.h>

#include "qt.h"

namespace qt {

// NVTX range for profilers (ncu --nvtx, nsys): a named span of host work and the
// launches it makes; costs a few ns when no tool is attached.
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

// A launch parameter that depends on the device (SM count, occupancy, a
// kernel attribute set once): computed by f() the first time it is asked for
// with a given device current, then reused for that device.  f() must be
// idempotent (two threads may both compute it the first time).
class PerDevice {
 public:
  template <typename F>
  int get(F&& f) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return f();
    const int v = vals_[dev].load(std::memory_order_acquire);
    if (v != 0) return v - 1;
    const int r = f();
    vals_[dev].store(r + 1, std::memory_order_release);
    return r;
  }

 private:
  static constexpr int kMaxDevices = 64;
  std::atomic<int> vals_[kMaxDevices] = {};
};

// ---- device scratch sizes -------------------------------------------------
constexpr int kRedThreads = 256;          // threads of the reduction kernels
constexpr int kMaxRedBlocks = 152 * 8;    // upper bound of their grid
constexpr int kRdmMaxQ = 3;               // reduced density matrix: q <= 3
constexpr int kExpGroup = 16;             // Z masks per expectation pass
// CDF for sampling: chunk = 64 amplitudes (one warp, 128-bit loads),
// sub-block = 16 chunks, block = 64 sub-blocks
constexpr int kCdfChunkLog = 6, kCdfSubLog = 10, kCdfBlkLog = 16;

inline uint64_t cdf_num_sub(int n) { return ((1ull << n) + (1ull << kCdfSubLog) - 1) >> kCdfSubLog; }
inline uint64_t cdf_num_blk(int n) { return (cdf_num_sub(n) + 63) >> 6; }

struct Scratch {
  double* partial = nullptr;   // kMaxRedBlocks * 64 doubles
  double* result = nullptr;    // 64 doubles
  float* cdf_sub = nullptr;    // cdf_num_sub(n) floats
  double* cdf_cum = nullptr;   // cdf_num_blk(n) doubles
};
size_t scratch_partial_bytes();

// ---- kernels ---------------------------------------------------------------
// state <- U (2^k x 2^k row-major complex64, basis `targets` sorted ascending)
cudaError_t launch_apply(float2* psi, int n, int k, const uint32_t* targets, const float2* U,
                         cudaStream_t st);
// rho (4^q doubles, layout of rdm_unpack) of qubits Q into scr.result
cudaError_t launch_rdm(const float2* psi, int n, int q, const uint32_t* qubits, const Scratch& scr,
                       cudaStream_t st);
// Channels on 4..6 qubits: N and P_i = |K_i psi|^2 for kraus_group(q)
// operators (16, 4, 1 for q = 4, 5, 6; pad with zero matrices) into
// scr.result[0] (N) and scr.result[1..]; ops_dev: the operators, 2^q x 2^q
// row-major complex64 in device memory, basis bit b <-> qubits[b]
int kraus_group(int q);
cudaError_t launch_kraus_norms(const float2* psi, int n, int q, const uint32_t* qubits, int nops,
                               const float2* ops_dev, const Scratch& scr, cudaStream_t st);
// N = <psi|psi> and sum |psi_x|^2 (-1)^popc(x&mask) for nm <= 16 masks into scr.result[0..nm]
cudaError_t launch_expect(const float2* psi, int n, int nm, const uint64_t* masks,
                          const Scratch& scr, cudaStream_t st);
// S samples of trajectory traj into out (device)
cudaError_t launch_sample(const float2* psi, int n, uint64_t seed, uint64_t traj, uint32_t S,
                          uint64_t* out, const Scratch& scr, cudaStream_t st, const double* readout = nullptr);
// C(x) of every x as the sampler forms it (2^n doubles into out, device)
cudaError_t launch_cdf_values(const float2* psi, int n, const Scratch& scr, double* out, cudaStream_t st);
// 6-qubit fused gate on CUDA cores (FP32), matrix 64x64 row-major in device memory, n >= 13
cudaError_t launch_apply6_fp32(float2* psi, int n, const uint32_t* targets, const float2* udev, cudaStream_t st);
// multi-gate pass: up to kGroupMaxGates fused gates (width <= 4, targets
// ascending, matrix row-major) whose qubits lie in {0..6} plus at most 6
// higher qubits, applied in one pass over the state (n >= 7 + #high qubits)
constexpr int kGroupMaxGates = 8;
constexpr int kGroupMaxHigh = 6;
struct GroupPiece {
  int k;
  uint32_t targets[4];
  const float2* u;
};
cudaError_t launch_apply_group(float2* psi, int n, int ng, const GroupPiece* pieces, cudaStream_t st);
// tensor-core path (split-TF32, k = 4..6, n >= k + 7): W is the real
// embedding of U, row-major [2^(k+1) x 2^(k+1)] FP32 in device memory; *err
// is set (nonzero) if a bounded wait in the kernel ran out
bool tc_supported(int n, int k);
cudaError_t launch_apply_tc(float2* psi, int n, int k, const uint32_t* targets, const float* wdev, int* err,
                            cudaStream_t st, uint32_t lbo = 0, uint32_t sbo = 0);
void real_embedding(int k, const float2* U, float* W);
// |0...0>
cudaError_t launch_init_state(float2* psi, int n, cudaStream_t st);
// Product-state preparation: psi[x] = H[x >> m] * L[x mod 2^m], each table the
// product of factor columns (U |0> of a fused gate on its own qubits) on the
// qubits below m (L) or from m up (H); qubits no factor holds are |0>.
constexpr int kFoldMax = 32;          // factors per table
constexpr int kFoldVals = 1024;       // factor values per table
constexpr int kFoldTableBits = 20;    // largest table: 2^20 entries
struct FoldSpec {
  float2 v[kFoldVals];                // factor columns, concatenated
  uint16_t off[kFoldMax];             // offset of factor f's 2^w values in v
  uint8_t w[kFoldMax];                // factor width (1..6)
  uint8_t q[kFoldMax][6];             // qubit of index bit b of factor f, relative to the table
  uint64_t zmask;                     // table bits that no factor holds (must be 0)
  int nf;                             // factors
};
// tables: 2^m + 2^(n-m) complex64 of device scratch; 1 <= m, n - m <= 20
cudaError_t launch_init_product(float2* psi, int n, int m, const FoldSpec& lo, const FoldSpec& hi,
                                float2* tables, cudaStream_t st);
// psi *= f
cudaError_t launch_scale(float2* psi, int n, float f, cudaStream_t st);

// unpack the 4^q reals of an rdm result into a row-major complex matrix
// rho[b][a] = sum psi_b conj(psi_a)
void rdm_unpack(int q, const double* r, double* rho_interleaved);

int sm_count();
// binaryVersion / ptxVersion of the library's kernels on the current device
cudaError_t kernel_arch(int* binary_version, int* ptx_version);

}  // namespace qt
