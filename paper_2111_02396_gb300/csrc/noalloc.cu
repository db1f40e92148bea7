// Allocation-free variant of the branch-probability pass.
//
// Some callers cannot let a library call cudaMalloc / cudaFree (or any
// allocator) on their behalf: a host application that reserves all of the
// GPU's memory for its own pool at start-up, or a latency-critical loop
// where an allocation or free could stall the device.  For them,
// qt_state_reduced_density_noalloc runs the same reduction kernels as
// qt_state_reduced_density, but its FP64 scratch (per-block partial sums
// and the final row) lives in one file-scope __device__ array of fixed size
// instead of being allocated per call.
//
// Properties of that array:
//   - it is kMaxRedBlocks * 64 + 64 doubles (608.5 KiB), enough for the
//     largest reduction the kernels launch (q <= 3, i.e. 64 FP64 values per
//     block); every GPU that loads the library holds it until the process
//     exits;
//   - every call on a device shares it and it keeps the last call's
//     contents.  Nothing in it has to start at zero: every partial and the
//     result row are overwritten before they are read;
//   - two calls whose kernels overlap on the GPU (different streams, or
//     different host threads) race on it; callers must order them.
//
// The host-side name of a __device__ variable is not a device address, so
// the array's address is looked up with cudaGetSymbolAddress, with the
// calling device current.  The lookup is repeated on every call rather than
// cached: the address belongs to the context that loaded the module, and a
// device reset (or a caller switching contexts) would leave a cached pointer
// stale.  The lookup neither allocates nor enqueues work; the first call on a
// device may load the library's module there, so that first call should come
// before any stream capture.
#include <cuda_runtime.h>

#include "kernels.h"
#include "qt_internal.h"

namespace qt {

constexpr size_t kNoAllocDoubles = static_cast<size_t>(kMaxRedBlocks) * 64 + 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

static qt_status noalloc_scratch(double** out) {
  double* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_noalloc_scratch);
  if (e != cudaSuccess || !p)
    return set_error(QT_ERR_CUDA, "qt_state_reduced_density_noalloc: cudaGetSymbolAddress: %s",
                     cudaGetErrorString(e));
  *out = p;
  return QT_OK;
}

}  // namespace qt

using namespace qt;

extern "C" qt_status qt_state_reduced_density_noalloc(const void* state, uint32_t n, uint32_t q,
                                                      const uint32_t* qubits, double* out, void* stream) {
  clear_error();
  if (!state || !qubits || !out)
    return set_error(QT_ERR_INVALID_ARG, "qt_state_reduced_density_noalloc: NULL argument");
  if (reinterpret_cast<uintptr_t>(state) & 15u)
    return set_error(QT_ERR_INVALID_ARG, "qt_state_reduced_density_noalloc: state not 16-byte aligned");
  if (n < 1 || n > QT_MAX_QUBITS)
    return set_error(QT_ERR_INVALID_ARG, "qt_state_reduced_density_noalloc: n=%u outside 1..%d", n, QT_MAX_QUBITS);
  // the fixed scratch holds 64 FP64 values per block: q <= 3
  if (q < 1 || q > static_cast<uint32_t>(kRdmMaxQ) || q > n)
    return set_error(QT_ERR_UNSUPPORTED,
                     "qt_state_reduced_density_noalloc: q=%u exceeds the fixed scratch (q <= 3 and q <= n)", q);
  uint64_t mask = 0;
  for (uint32_t b = 0; b < q; ++b) {
    if (qubits[b] >= n)
      return set_error(QT_ERR_INVALID_ARG, "qt_state_reduced_density_noalloc: qubit %u >= n", qubits[b]);
    if (mask & (1ull << qubits[b]))
      return set_error(QT_ERR_INVALID_ARG, "qt_state_reduced_density_noalloc: repeated qubit");
    mask |= 1ull << qubits[b];
  }
  double* scratch = nullptr;
  qt_status s = noalloc_scratch(&scratch);
  if (s != QT_OK) return s;
  Scratch scr;
  scr.partial = scratch;                                   // kMaxRedBlocks * 64 doubles
  scr.result = scratch + static_cast<size_t>(kMaxRedBlocks) * 64;   // 64 doubles
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = launch_rdm(static_cast<const float2*>(state), static_cast<int>(n), static_cast<int>(q), qubits,
                             scr, st);
  double r[64];
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(r, scr.result, sizeof(double) << (2 * q), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess)
    return set_error(QT_ERR_CUDA, "qt_state_reduced_density_noalloc: %s", cudaGetErrorString(e));
  rdm_unpack(static_cast<int>(q), r, out);
  return QT_OK;
}
