// Trajectory controller and C ABI (Sec. III.E, Alg. 2).
//
// Delayed inner products, as run here: stage 1 of every channel depends
// only on its draw r and the lower bounds pbar, so all stage-1 decisions of
// a trajectory are taken on the host before any kernel runs.  Channels that
// stage 1 cannot decide ("flush points") cut the circuit into segments.
// Each segment is applied as the fused gates restricted to the segment's
// operations (a fused gate whose slots all hold their default operator and
// that lies wholly inside the segment uses its precomputed matrix; any
// other piece is recomposed on the host in FP64).  At a flush point one
// read pass evaluates the reduced density block rho_Q of the channel's
// qubits in FP64, which gives N = tr rho_Q and P_i = tr(K_i^dag K_i rho_Q)
// for every branch at once; stage 2 then picks the branch and the operator
// K_i / sqrt(P_i) becomes the first member of the next segment.  The
// conventional (eager) algorithm is the same loop with every channel a
// flush point.
#include <cuda_runtime.h>

#include <algorithm>
#include <bit>
#include <cmath>
#include <cstdlib>
#include <deque>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <vector>

#include "kernels.h"
#include "qt_internal.h"
#include "qt_philox.h"

namespace qt {

// ---------------------------------------------------------------------------
// device memory
// ---------------------------------------------------------------------------
struct Allocator {
  qt_alloc_fn alloc = nullptr;
  qt_free_fn free = nullptr;
  void* ctx = nullptr;
};
static Allocator g_alloc;
static std::mutex g_alloc_mu;

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  Allocator a;
  cudaStream_t st = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept { *this = std::move(o); }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) {
      release();
      p = o.p; bytes = o.bytes; a = o.a; st = o.st;
      o.p = nullptr; o.bytes = 0;
    }
    return *this;
  }
  ~DevBuf() { release(); }
  bool alloc(size_t b, cudaStream_t s) {
    release();
    {
      std::lock_guard<std::mutex> lk(g_alloc_mu);
      a = g_alloc;
    }
    st = s;
    bytes = b;
    if (a.alloc) {
      p = a.alloc(b, s, a.ctx);
    } else if (cudaMallocAsync(&p, b, s) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    return p != nullptr;
  }
  void release() {
    if (!p) return;
    if (a.alloc) {
      if (a.free) a.free(p, bytes, st, a.ctx);
    } else {
      cudaFreeAsync(p, st);
    }
    p = nullptr;
  }
  template <typename T> T* as() const { return static_cast<T*>(p); }
};

static qt_status cuda_fail(cudaError_t e, const char* where) {
  return set_error(QT_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}
#define QT_CUDA(call, where)                         \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return cuda_fail(e_, where); \
  } while (0)

struct ScratchBufs {
  DevBuf partial, result, sub, cum;
  Scratch s;
  bool alloc(int n, cudaStream_t st) {
    if (!partial.alloc(scratch_partial_bytes(), st)) return false;
    if (!result.alloc(sizeof(double) * 64, st)) return false;
    if (!sub.alloc(sizeof(float) * cdf_num_sub(n), st)) return false;
    if (!cum.alloc(sizeof(double) * cdf_num_blk(n), st)) return false;
    s.partial = partial.as<double>();
    s.result = result.as<double>();
    s.cdf_sub = sub.as<float>();
    s.cdf_cum = cum.as<double>();
    return true;
  }
};

static void to_f32(const std::vector<cd>& m, std::vector<float2>& out) {
  out.resize(m.size());
  for (size_t i = 0; i < m.size(); ++i)
    out[i] = make_float2(static_cast<float>(m[i].real()), static_cast<float>(m[i].imag()));
}

}  // namespace qt

using namespace qt;

struct qt_run {
  const qt_fused* f = nullptr;
  qt_run_params p{};
  std::vector<uint64_t> masks;
  uint32_t n = 0, T = 0, nch = 0;
  std::vector<int32_t> kraus, stage;
  std::vector<uint64_t> samples;
  std::vector<double> expect, norms;
  std::vector<DevBuf> states;
  DevBuf readout;                  // 2n readout error probabilities (device), or empty
  ScratchBufs scr;
  qt_run_stats_t stats{};
  cudaStream_t st = nullptr;
};

namespace qt {

// stage 1 / stage 2 of Alg. 2 on one draw.  P == nullptr: stage 1 only,
// returns -1 when it does not decide.  Otherwise the two-stage partition of
// [0,1): lower-bound intervals first, then intervals of width P_i/N - pbar_i.
static int decide(const Op& op, double r, const double* P, double N, int* stage_out) {
  double rr = r;
  for (uint32_t i = 0; i < op.num_ops; ++i) {
    if (rr < op.pbar[i]) { *stage_out = 1; return static_cast<int>(i); }
    rr -= op.pbar[i];
  }
  if (!P) return -1;
  *stage_out = 2;
  int last = -1, last_pos = -1;
  for (uint32_t i = 0; i < op.num_ops; ++i) {
    double d = P[i] / N - op.pbar[i];
    if (d < 0.0) d = 0.0;                    // rounding
    if (d > 0.0) last = static_cast<int>(i);
    if (P[i] > 0.0) last_pos = static_cast<int>(i);
    if (rr < d) return static_cast<int>(i);
    rr -= d;
  }
  return last >= 0 ? last : (last_pos >= 0 ? last_pos : op.def);
}

struct Controller {
  qt_run& R;
  const Circuit& c;
  const Fused& f;
  std::vector<std::vector<float2>> def32;   // default fused matrices in FP32
  std::vector<cd> tmp;
  std::vector<float2> tmp32;
  double* pinned = nullptr;
  std::vector<cudaEvent_t> ev;              // timing events (pairs)
  std::vector<int> ev_width;                // gate width of each timed pass (0: multi-gate)
  size_t ev_used = 0;

  explicit Controller(qt_run& r) : R(r), c(*r.f->c), f(*r.f) {
    def32.resize(f.gates.size());
    for (size_t g = 0; g < f.gates.size(); ++g) to_f32(f.gates[g].def, def32[g]);
  }
  ~Controller() {
    if (pinned) cudaFreeHost(pinned);
    for (auto e : ev) cudaEventDestroy(e);
  }

  // tensor-core path buffers (split-TF32, widths 4..6)
  DevBuf wbuf, errbuf;
  std::vector<float> wtmp;

  // QT_TF32X3 sends 5- and 6-qubit pieces to the tensor cores; narrower
  // pieces stay on the CUDA-core kernel, which is faster for them
  bool use_tc(int k) const {
    return R.p.precision == QT_TF32X3 && k >= 5 && tc_supported(static_cast<int>(R.n), k);
  }

  qt_status launch_one(float2* psi, const std::vector<uint32_t>& targets, const float2* U) {
    const int k = static_cast<int>(targets.size());
    if (use_tc(k)) {
      if (!wbuf.p && !wbuf.alloc(sizeof(float) * 128 * 128, R.st))
        return set_error(QT_ERR_OUT_OF_MEMORY, "tensor-core matrix buffer");
      if (!errbuf.p) {                      // device error flag of the tensor-core kernel, cleared once
        if (!errbuf.alloc(sizeof(int), R.st)) return set_error(QT_ERR_OUT_OF_MEMORY, "error flag");
        QT_CUDA(cudaMemsetAsync(errbuf.p, 0, sizeof(int), R.st), "cudaMemsetAsync");
      }
      const int N = 2 << k;
      wtmp.resize(static_cast<size_t>(N) * N);
      real_embedding(k, U, wtmp.data());
      QT_CUDA(cudaMemcpyAsync(wbuf.p, wtmp.data(), sizeof(float) * N * N, cudaMemcpyHostToDevice, R.st),
              "cudaMemcpyAsync(W)");
      R.stats.h2d_bytes += sizeof(float) * N * N;
      QT_CUDA(launch_apply_tc(psi, static_cast<int>(R.n), k, targets.data(), wbuf.as<float>(), errbuf.as<int>(), R.st),
              "tensor-core apply kernel launch");
      return QT_OK;
    }
    if (k == 6 && R.n >= 13) {
      if (!wbuf.p && !wbuf.alloc(sizeof(float) * 128 * 128, R.st))
        return set_error(QT_ERR_OUT_OF_MEMORY, "matrix buffer");
      QT_CUDA(cudaMemcpyAsync(wbuf.p, U, sizeof(float2) * 64 * 64, cudaMemcpyHostToDevice, R.st), "cudaMemcpyAsync(U)");
      R.stats.h2d_bytes += sizeof(float2) * 64 * 64;
      QT_CUDA(launch_apply6_fp32(psi, static_cast<int>(R.n), targets.data(), wbuf.as<float2>(), R.st),
              "6-qubit apply kernel launch");
      return QT_OK;
    }
    if (k > 5) return set_error(QT_ERR_UNSUPPORTED, "fused width %d needs n >= 13", k);
    QT_CUDA(launch_apply(psi, static_cast<int>(R.n), k, targets.data(), U, R.st), "apply kernel launch");
    const size_t d = 1ull << k;
    R.stats.h2d_bytes += sizeof(float2) * d * d;
    return QT_OK;
  }

  qt_status check_device_error() {
    if (!errbuf.p) return QT_OK;
    int e = 0;
    QT_CUDA(cudaMemcpyAsync(&e, errbuf.p, sizeof(int), cudaMemcpyDeviceToHost, R.st), "cudaMemcpyAsync(err)");
    QT_CUDA(cudaStreamSynchronize(R.st), "cudaStreamSynchronize(err)");
    if (e) return set_error(QT_ERR_TIMEOUT, "tensor-core kernel: a bounded wait ran out (code %d)", e);
    return QT_OK;
  }

  // one pass over the state, optionally bracketed by timing events
  template <typename F>
  qt_status timed_launch(F&& launch, const char* what, int width) {
    const bool timed = (R.p.flags & QT_FLAG_TIME_KERNELS) != 0;
    if (timed) {
      if (ev_used + 2 > ev.size()) {
        for (int k = 0; k < 2; ++k) {
          cudaEvent_t e;
          QT_CUDA(cudaEventCreate(&e), "cudaEventCreate");
          ev.push_back(e);
        }
      }
      QT_CUDA(cudaEventRecord(ev[ev_used], R.st), "cudaEventRecord");
    }
    cudaError_t e = cudaSuccess;
    qt_status ls = launch(e);
    if (ls != QT_OK) return ls;
    if (e != cudaSuccess) return cuda_fail(e, what);
    if (timed) {
      QT_CUDA(cudaEventRecord(ev[ev_used + 1], R.st), "cudaEventRecord");
      if (ev_width.size() < ev.size() / 2) ev_width.resize(ev.size() / 2);
      ev_width[ev_used / 2] = width;
      ev_used += 2;
    }
    R.stats.passes_by_width[width < 8 ? width : 0]++;
    R.stats.fused_passes++;
    R.stats.kernel_launches++;
    R.stats.apply_bytes += 16ull << R.n;
    return QT_OK;
  }

  qt_status apply(float2* psi, const std::vector<uint32_t>& targets, const float2* U) {
    return timed_launch([&](cudaError_t&) { return launch_one(psi, targets, U); }, "apply kernel launch",
                        static_cast<int>(targets.size()));
  }

  qt_status collect_timing() {
    if (!ev_used) return QT_OK;
    QT_CUDA(cudaEventSynchronize(ev[ev_used - 1]), "cudaEventSynchronize");
    double ms = 0.0;
    for (size_t i = 0; i < ev_used; i += 2) {
      float t = 0.f;
      QT_CUDA(cudaEventElapsedTime(&t, ev[i], ev[i + 1]), "cudaEventElapsedTime");
      ms += t;
      const int w = ev_width[i / 2];
      R.stats.apply_ms_by_width[w < 8 ? w : 0] += t;
    }
    R.stats.apply_ms += ms;
    ev_used = 0;
    return QT_OK;
  }

  // one piece of a segment: a fused gate restricted to the segment's ops
  struct Piece {
    std::vector<uint32_t> targets;
    const float2* u;
    uint64_t full;                    // qubit mask
  };
  std::deque<std::vector<float2>> owned;

  // The pieces of ops [lo, hi) of the circuit, in launch order.  choice[ch]
  // is the operator of each channel; norm_scale[ch] > 0 marks a stage-2
  // choice applied as K_i * norm_scale (the Kraus form, normalized).
  // Composed pieces keep their matrices in `owned` until the next call.
  void collect_pieces(uint32_t lo, uint32_t hi, const std::vector<int>& choice,
                      const std::vector<double>& norm_scale, std::vector<Piece>& pieces) {
    std::vector<std::pair<uint32_t, const cd*>> seq;
    std::vector<std::vector<cd>> scaled;
    pieces.clear();
    owned.clear();
    for (size_t g = 0; g < f.gates.size(); ++g) {
      const FusedGate& fg = f.gates[g];
      seq.clear();
      scaled.clear();
      bool whole = true, dflt = true;
      uint64_t mask = 0;
      for (uint32_t m : fg.members) {
        if (m < lo || m >= hi) { whole = false; continue; }
        const Op& op = c.ops[m];
        for (uint32_t b = 0; b < op.q; ++b) mask |= 1ull << op.qubits[b];
        if (op.kind == QT_OP_GATE) {
          seq.emplace_back(m, op.mat(0));
          continue;
        }
        const int ch = op.channel;
        const int ci = choice[ch];
        if (norm_scale[ch] > 0.0) {
          dflt = false;
          const size_t dd = static_cast<size_t>(op.dim()) * op.dim();
          scaled.emplace_back(op.kraus_op(static_cast<uint32_t>(ci)), op.kraus_op(static_cast<uint32_t>(ci)) + dd);
          for (auto& x : scaled.back()) x *= norm_scale[ch];
          seq.emplace_back(m, nullptr);      // patched below
        } else {
          if (ci != op.def) dflt = false;
          seq.emplace_back(m, op.mat(static_cast<uint32_t>(ci)));
        }
      }
      if (seq.empty()) continue;
      size_t si = 0;
      for (auto& e : seq)
        if (!e.second) e.second = scaled[si++].data();
      if (whole && dflt) {
        uint64_t fm = 0;
        for (uint32_t q : fg.targets) fm |= 1ull << q;
        pieces.push_back(Piece{fg.targets, def32[g].data(), fm});
        continue;
      }
      std::vector<uint32_t> targets;
      for (uint32_t q = 0; q < 64; ++q)
        if (mask & (1ull << q)) targets.push_back(q);
      compose(c, targets, seq, tmp);
      owned.emplace_back();
      to_f32(tmp, owned.back());
      pieces.push_back(Piece{targets, owned.back().data(), mask});
    }
  }

  // Apply ops [lo, hi) of the circuit.
  qt_status run_segment(float2* psi, uint32_t lo, uint32_t hi, const std::vector<int>& choice,
                        const std::vector<double>& norm_scale) {
    std::vector<Piece> pieces;
    collect_pieces(lo, hi, choice, norm_scale, pieces);
    return launch_pieces(psi, pieces);
  }

  // Product-state folding of the first segment.  A piece none of whose
  // qubits an earlier piece of the segment touches acts on |0> of its own
  // qubits and commutes with every piece before it, so it can move to the
  // front and its output U[:, 0] becomes a factor of the initial product
  // state.  The qubits are split at m; a factor must lie wholly below or
  // wholly from m up.  m is chosen (tables of at most 2^20 entries) to fold
  // the most pieces.  Returns m, or 0 when nothing folds.
  static constexpr uint32_t kFoldMinQubits = 12;
  DevBuf foldbuf;

  int plan_fold(const std::vector<Piece>& pieces, std::vector<char>& fold) const {
    const int n = static_cast<int>(R.n);
    std::vector<size_t> first;
    uint64_t touched = 0;
    for (size_t i = 0; i < pieces.size(); ++i) {
      if (!(pieces[i].full & touched)) first.push_back(i);
      touched |= pieces[i].full;
    }
    if (first.empty()) return 0;
    auto pick = [&](int m, std::vector<char>* mark) {
      const uint64_t low = (1ull << m) - 1ull;
      int side_n[2] = {0, 0}, side_v[2] = {0, 0}, cnt = 0;
      for (size_t i : first) {
        const uint64_t f = pieces[i].full;
        const int side = (f & ~low) == 0 ? 0 : ((f & low) == 0 ? 1 : -1);
        if (side < 0) continue;
        const int d = 1 << pieces[i].targets.size();
        if (side_n[side] >= kFoldMax || side_v[side] + d > kFoldVals) continue;
        side_n[side]++;
        side_v[side] += d;
        cnt++;
        if (mark) (*mark)[i] = 1;
      }
      return cnt;
    };
    const int mlo = std::max(1, n - kFoldTableBits), mhi = std::min(kFoldTableBits, n - 1);
    int best_m = 0, best = 0;
    for (int m = mlo; m <= mhi; ++m) {
      const int cnt = pick(m, nullptr);
      if (cnt > best || (cnt == best && cnt > 0 && std::abs(2 * m - n) < std::abs(2 * best_m - n))) {
        best = cnt;
        best_m = m;
      }
    }
    if (best == 0) return 0;
    fold.assign(pieces.size(), 0);
    pick(best_m, &fold);
    return best_m;
  }

  // Apply ops [0, hi) starting from |0...0>.
  qt_status run_first_segment(float2* psi, uint32_t hi, const std::vector<int>& choice,
                              const std::vector<double>& norm_scale) {
    std::vector<Piece> pieces;
    collect_pieces(0, hi, choice, norm_scale, pieces);
    const int n = static_cast<int>(R.n);
    std::vector<char> fold;
    const int m = R.n >= kFoldMinQubits ? plan_fold(pieces, fold) : 0;
    if (m == 0) {
      QT_CUDA(launch_init_state(psi, n, R.st), "init kernel launch");
      R.stats.kernel_launches++;
      return launch_pieces(psi, pieces);
    }
    FoldSpec side[2];
    uint64_t held[2] = {0, 0};
    for (int k = 0; k < 2; ++k) {
      std::memset(&side[k], 0, sizeof(FoldSpec));
    }
    std::vector<Piece> rest;
    uint64_t folded = 0;
    for (size_t i = 0; i < pieces.size(); ++i) {
      if (!fold[i]) {
        rest.push_back(pieces[i]);
        continue;
      }
      const Piece& P = pieces[i];
      const int k = (P.full >> m) == 0 ? 0 : 1;
      const int base = k ? m : 0;
      FoldSpec& S = side[k];
      const int w = static_cast<int>(P.targets.size());
      const int d = 1 << w;
      const int f = S.nf++;
      S.w[f] = static_cast<uint8_t>(w);
      S.off[f] = static_cast<uint16_t>(f ? S.off[f - 1] + (1 << S.w[f - 1]) : 0);
      for (int b = 0; b < w; ++b) {
        S.q[f][b] = static_cast<uint8_t>(static_cast<int>(P.targets[b]) - base);
        held[k] |= 1ull << S.q[f][b];
      }
      for (int j = 0; j < d; ++j) S.v[S.off[f] + j] = P.u[static_cast<size_t>(j) * d];   // column 0
      folded++;
    }
    side[0].zmask = ((1ull << m) - 1ull) & ~held[0];
    side[1].zmask = ((1ull << (n - m)) - 1ull) & ~held[1];
    const size_t need = sizeof(float2) * ((1ull << m) + (1ull << (n - m)));
    if (foldbuf.bytes < need && !foldbuf.alloc(need, R.st))
      return set_error(QT_ERR_OUT_OF_MEMORY, "product-state tables");
    QT_CUDA(launch_init_product(psi, n, m, side[0], side[1], foldbuf.as<float2>(), R.st),
            "product-state kernel launch");
    R.stats.kernel_launches += 3;
    R.stats.folded_pieces += folded;
    R.stats.fold_split = static_cast<uint32_t>(m);
    return launch_pieces(psi, rest);
  }

  // Launch the pieces of a segment in order.  With QT_FLAG_MULTI_GATE, consecutive
  // pieces (moved earlier past pieces they share no qubit with) whose qubits
  // lie in {0..6} plus at most kGroupMaxHigh higher qubits share one
  // multi-gate pass over the state.
  // Peephole merge of a segment's pieces, extending the fusion of Sec. III.B
  // across the cuts that flush points make: a piece moves forward to the
  // first later piece that shares a qubit with it (every piece in between
  // acts on other qubits, so the two commute) and the two become one piece
  // when their qubits number at most the run's fusion width.  A flush point
  // cuts the fused gates in flight into before- and after-pieces; merged with
  // a neighbour, such a remainder costs no pass of its own.  The product is
  // formed in FP64 from the pieces' FP32 matrices and rounded once.
  std::vector<cd> mtmp, mcol;
  void merge_pieces(std::vector<Piece>& pieces) {
    // 6-qubit passes need n >= 13 (the run checks its fused gates for that up front)
    const int kmax = std::min(static_cast<int>(f.kmax), R.n >= 13 ? 6 : 5);
    std::vector<char> gone(pieces.size(), 0);
    size_t merged = 0;
    for (size_t a = 0; a < pieces.size(); ++a) {
      if (gone[a]) continue;
      size_t b = a + 1;
      while (b < pieces.size() && (gone[b] || !(pieces[b].full & pieces[a].full))) ++b;
      if (b == pieces.size()) continue;
      const uint64_t u = pieces[a].full | pieces[b].full;
      if (std::popcount(u) > kmax) continue;
      std::vector<uint32_t> targets;
      for (uint32_t q = 0; q < 64; ++q)
        if (u & (1ull << q)) targets.push_back(q);
      const int w = static_cast<int>(targets.size()), D = 1 << w;
      // columns of the identity, then piece a, then piece b (column-major)
      mcol.assign(static_cast<size_t>(D) * D, cd(0.0));
      for (int j = 0; j < D; ++j) mcol[static_cast<size_t>(j) * D + j] = 1.0;
      for (const Piece* P : {&pieces[a], &pieces[b]}) {
        const int q = static_cast<int>(P->targets.size()), d = 1 << q;
        int pos[QT_MAX_OP_QUBITS];
        for (int i = 0; i < q; ++i)
          pos[i] = static_cast<int>(std::lower_bound(targets.begin(), targets.end(), P->targets[i]) - targets.begin());
        mtmp.resize(static_cast<size_t>(d) * d);
        for (int i = 0; i < d * d; ++i) mtmp[i] = cd(P->u[i].x, P->u[i].y);
        for (int j = 0; j < D; ++j) apply_small(&mcol[static_cast<size_t>(j) * D], w, q, pos, mtmp.data());
      }
      owned.emplace_back(static_cast<size_t>(D) * D);
      std::vector<float2>& M = owned.back();
      for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
          const cd x = mcol[static_cast<size_t>(j) * D + i];
          M[static_cast<size_t>(i) * D + j] = make_float2(static_cast<float>(x.real()), static_cast<float>(x.imag()));
        }
      pieces[b] = Piece{std::move(targets), M.data(), u};
      gone[a] = 1;
      ++merged;
    }
    if (!merged) return;
    size_t o = 0;
    for (size_t i = 0; i < pieces.size(); ++i) {
      if (gone[i]) continue;
      if (o != i) pieces[o] = std::move(pieces[i]);   // never onto itself (that empties a vector)
      ++o;
    }
    pieces.resize(o);
    R.stats.merged_pieces += merged;
  }

  qt_status launch_pieces(float2* psi, std::vector<Piece>& pieces) {
    merge_pieces(pieces);
    const bool group = (R.p.flags & QT_FLAG_MULTI_GATE) && R.n >= 8;
    const int hmax = std::min<int>(kGroupMaxHigh, static_cast<int>(R.n) - 7);
    const uint64_t low = (1ull << 7) - 1ull;
    std::vector<char> done(pieces.size(), 0);
    std::vector<size_t> members;
    for (size_t a = 0; a < pieces.size(); ++a) {
      if (done[a]) continue;
      done[a] = 1;
      members.assign(1, a);
      const int wa = static_cast<int>(pieces[a].targets.size());
      const bool groupable_a = group && wa <= 4 && !use_tc(wa) &&
                               std::popcount(pieces[a].full & ~low) <= hmax;
      if (groupable_a) {
        uint64_t hm = pieces[a].full & ~low, blocked = 0;
        for (size_t b = a + 1; b < pieces.size() && b < a + 64 &&
                               members.size() < static_cast<size_t>(kGroupMaxGates); ++b) {
          if (done[b]) continue;
          const Piece& P = pieces[b];
          const int wb = static_cast<int>(P.targets.size());
          if ((P.full & blocked) == 0 && wb <= 4 && std::popcount(hm | (P.full & ~low)) <= hmax) {
            hm |= P.full & ~low;
            members.push_back(b);
            done[b] = 1;
            continue;
          }
          blocked |= P.full;
        }
      }
      if (members.size() == 1) {
        qt_status s = apply(psi, pieces[a].targets, pieces[a].u);
        if (s != QT_OK) return s;
        R.stats.fused_pieces++;
        continue;
      }
      GroupPiece gp[kGroupMaxGates];
      for (size_t i = 0; i < members.size(); ++i) {
        const Piece& P = pieces[members[i]];
        gp[i].k = static_cast<int>(P.targets.size());
        for (size_t b = 0; b < P.targets.size(); ++b) gp[i].targets[b] = P.targets[b];
        gp[i].u = P.u;
        const size_t d = 1ull << P.targets.size();
        R.stats.h2d_bytes += sizeof(float2) * d * d;
      }
      qt_status s = timed_launch([&](cudaError_t& e) {
        e = launch_apply_group(psi, static_cast<int>(R.n), static_cast<int>(members.size()), gp, R.st);
        return QT_OK;
      }, "multi-gate pass launch", 0);
      if (s != QT_OK) return s;
      R.stats.fused_pieces += members.size();
    }
    return QT_OK;
  }

  // Channels on 4..6 qubits: P_i = |K_i psi|^2 on the device, kraus_group(q)
  // operators per pass (zero matrices pad the last group); N from the same pass.
  DevBuf kbuf;
  std::vector<float2> ktmp;
  qt_status kraus_probabilities(const float2* psi, const Op& op, double& N, double* P) {
    TraceRange tr("qt probability pass (wide channel)");
    const int q = static_cast<int>(op.q), D = 1 << q, G = kraus_group(q);
    const size_t mat = static_cast<size_t>(D) * D;
    if (kbuf.bytes < sizeof(float2) * G * mat && !kbuf.alloc(sizeof(float2) * G * mat, R.st))
      return set_error(QT_ERR_OUT_OF_MEMORY, "Kraus operator buffer");
    for (uint32_t g0 = 0; g0 < op.num_ops; g0 += static_cast<uint32_t>(G)) {
      ktmp.assign(G * mat, make_float2(0.f, 0.f));
      for (uint32_t j = 0; j < static_cast<uint32_t>(G) && g0 + j < op.num_ops; ++j) {
        const cd* K = op.kraus_op(g0 + j);
        for (size_t e = 0; e < mat; ++e)
          ktmp[j * mat + e] = make_float2(static_cast<float>(K[e].real()), static_cast<float>(K[e].imag()));
      }
      QT_CUDA(cudaMemcpyAsync(kbuf.p, ktmp.data(), sizeof(float2) * G * mat, cudaMemcpyHostToDevice, R.st),
              "cudaMemcpyAsync(Kraus operators)");
      QT_CUDA(launch_kraus_norms(psi, static_cast<int>(R.n), q, op.qubits, G, kbuf.as<float2>(), R.scr.s, R.st),
              "Kraus probability kernel launch");
      QT_CUDA(cudaMemcpyAsync(pinned, R.scr.s.result, sizeof(double) * (G + 1), cudaMemcpyDeviceToHost, R.st),
              "cudaMemcpyAsync(probabilities)");
      QT_CUDA(cudaStreamSynchronize(R.st), "cudaStreamSynchronize(probabilities)");
      R.stats.h2d_bytes += sizeof(float2) * G * mat;
      R.stats.d2h_bytes += sizeof(double) * (G + 1);
      R.stats.kernel_launches += 2;
      N = pinned[0];
      for (uint32_t j = 0; j < static_cast<uint32_t>(G) && g0 + j < op.num_ops; ++j) P[g0 + j] = pinned[1 + j];
    }
    R.stats.prob_passes++;
    return QT_OK;
  }

  // probability pass of channel op `oi`: returns N and P[0..num_ops)
  qt_status probabilities(const float2* psi, uint32_t oi, double& N, double* P) {
    TraceRange tr("qt probability pass");
    const Op& op = c.ops[oi];
    if (op.q > static_cast<uint32_t>(kRdmMaxQ)) {
      if (op.q > R.n) return set_error(QT_ERR_INVALID_ARG, "channel on %u qubits of a %u-qubit state", op.q, R.n);
      return kraus_probabilities(psi, op, N, P);
    }
    QT_CUDA(launch_rdm(psi, static_cast<int>(R.n), static_cast<int>(op.q), op.qubits, R.scr.s, R.st),
            "probability kernel launch");
    const int W = 1 << (2 * op.q);
    QT_CUDA(cudaMemcpyAsync(pinned, R.scr.s.result, sizeof(double) * W, cudaMemcpyDeviceToHost, R.st),
            "cudaMemcpyAsync(probabilities)");
    QT_CUDA(cudaStreamSynchronize(R.st), "cudaStreamSynchronize(probabilities)");
    R.stats.prob_passes++;
    R.stats.kernel_launches += 2;
    R.stats.d2h_bytes += sizeof(double) * W;
    const int D = static_cast<int>(op.dim());
    double rho[2 * 64];
    rdm_unpack(static_cast<int>(op.q), pinned, rho);
    N = 0.0;
    for (int b = 0; b < D; ++b) N += rho[2 * (b * D + b)];
    for (uint32_t i = 0; i < op.num_ops; ++i) {
      const cd* M = op.mtm_op(i);
      double acc = 0.0;                     // tr(M rho) = sum_ab M[a][b] rho[b][a]
      for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b) {
          const cd r(rho[2 * (b * D + a)], rho[2 * (b * D + a) + 1]);
          acc += (M[a * D + b] * r).real();
        }
      P[i] = acc;
    }
    return QT_OK;
  }

  // Stage 1 of every channel of a trajectory (Alg. 2): the operator each
  // channel's draw selects from the lower bounds alone, or a flush point where
  // it does not; `diverge` is the first channel whose draw does not keep the
  // channel's default operator in stage 1 (nch if every channel does).
  struct Stage1 {
    std::vector<int> choice;
    std::vector<double> rdraw;
    std::vector<uint32_t> flush_ops;
    uint32_t diverge = 0;
  };

  void stage1(uint32_t t, Stage1& s1) {
    const uint64_t traj = R.p.first_traj + t;
    const uint32_t nch = R.nch;
    s1.choice.assign(nch, 0);
    s1.rdraw.resize(nch);
    s1.flush_ops.clear();
    s1.diverge = nch;
    int32_t* kr = R.kraus.data() + static_cast<size_t>(t) * nch;
    int32_t* sg = R.stage.data() + static_cast<size_t>(t) * nch;
    for (uint32_t ch = 0; ch < nch; ++ch) {
      const Op& op = c.ops[c.channel_op[ch]];
      s1.rdraw[ch] = uniform01(R.p.seed, traj, kStreamChannel, ch);
      int st = 0;
      const int ci = (R.p.mode == QT_DELAYED) ? decide(op, s1.rdraw[ch], nullptr, 1.0, &st) : -1;
      if (ci >= 0) {
        s1.choice[ch] = ci;
        kr[ch] = ci;
        sg[ch] = 1;
      } else {
        s1.choice[ch] = op.def;
        s1.flush_ops.push_back(c.channel_op[ch]);
      }
      if (ci != op.def && s1.diverge == nch) s1.diverge = ch;
    }
  }

  // Ops [start, end) of trajectory t on psi, which already holds ops [0, start)
  // with every channel among them on its default operator (start = 0: psi is
  // prepared from |0...0>).  Every flush point of the trajectory is at or
  // after start.
  qt_status run_from(uint32_t t, float2* psi, const Stage1& s1, uint32_t start) {
    const uint32_t nch = R.nch;
    std::vector<int> choice = s1.choice;
    std::vector<double> scale(nch, 0.0);
    int32_t* kr = R.kraus.data() + static_cast<size_t>(t) * nch;
    int32_t* sg = R.stage.data() + static_cast<size_t>(t) * nch;
    const std::vector<uint32_t>& flush_ops = s1.flush_ops;
    uint32_t lo = start;
    const uint32_t nops = static_cast<uint32_t>(c.ops.size());
    for (size_t k = 0; k <= flush_ops.size(); ++k) {
      const uint32_t hi = k < flush_ops.size() ? flush_ops[k] : nops;
      qt_status s = (k == 0 && start == 0) ? run_first_segment(psi, hi, choice, scale)
                                           : run_segment(psi, lo, hi, choice, scale);
      if (s != QT_OK) return s;
      if (k == flush_ops.size()) break;
      const uint32_t oi = flush_ops[k];
      const Op& op = c.ops[oi];
      double N = 0.0, P[64];
      s = probabilities(psi, oi, N, P);
      if (s != QT_OK) return s;
      int st = 2;
      const int ci = decide(op, s1.rdraw[op.channel], P, N, &st);
      choice[op.channel] = ci;
      scale[op.channel] = 1.0 / std::sqrt(P[ci] > 0.0 ? P[ci] : 1.0);
      kr[op.channel] = ci;
      sg[op.channel] = st;
      R.stats.flushes += (st == 2);
      lo = oi;
    }
    return QT_OK;
  }

  qt_status trajectory(uint32_t t, float2* psi) {
    TraceRange tr("qt trajectory");
    Stage1 s1;
    stage1(t, s1);
    return run_from(t, psi, s1, 0);
  }

  qt_status finish_trajectory(uint32_t t, const float2* psi, uint64_t* d_samples) {
    qt_status s = measure(t, psi, d_samples);
    if (s == QT_OK) s = collect_timing();
    if (s == QT_OK) s = check_device_error();
    return s;
  }

  // Shared default-choice prefix (QT_FLAG_SHARE_PREFIX).  Every trajectory
  // of the run applies the same operators up to its first channel whose draw
  // leaves the default operator (stage 1 fixes that point before any kernel
  // runs), so the trajectories are taken in order of that point and one
  // shared state advances along the default path: each trajectory copies the
  // shared state at its divergence point and runs only its own suffix, and
  // trajectories that never diverge are measured on the shared final state.
  // The operations are those of the per-trajectory loop in the same order;
  // only the boundaries of the fused pieces differ (the piece that straddles
  // a divergence point is split, as at a flush point).
  qt_status run_shared(float2* shared, float2* work, uint64_t* d_samples) {
    TraceRange tr("qt trajectories sharing their prefix");
    const uint32_t T = R.T, nch = R.nch;
    const uint32_t nops = static_cast<uint32_t>(c.ops.size());
    std::vector<Stage1> plan(T);
    std::vector<uint32_t> order(T);
    for (uint32_t t = 0; t < T; ++t) {
      stage1(t, plan[t]);
      order[t] = t;
    }
    std::stable_sort(order.begin(), order.end(),
                     [&](uint32_t a, uint32_t b) { return plan[a].diverge < plan[b].diverge; });
    const std::vector<int> defaults = [&] {
      std::vector<int> d(nch);
      for (uint32_t ch = 0; ch < nch; ++ch) d[ch] = c.ops[c.channel_op[ch]].def;
      return d;
    }();
    const std::vector<double> noscale(nch, 0.0);
    const size_t sbytes = sizeof(float2) << R.n;
    bool started = false;
    uint32_t at = 0;                       // ops [0, at) applied to the shared state
    for (uint32_t t : order) {
      const Stage1& s1 = plan[t];
      const uint32_t D = s1.diverge < nch ? c.channel_op[s1.diverge] : nops;
      qt_status s = QT_OK;
      if (!started) {
        s = run_first_segment(shared, D, defaults, noscale);
        started = true;
      } else if (D > at) {
        s = run_segment(shared, at, D, defaults, noscale);
      }
      if (s != QT_OK) return s;
      at = std::max(at, D);
      R.stats.prefix_ops += D;
      float2* dst = R.p.keep_states ? R.states[t].as<float2>() : work;
      if (s1.diverge == nch && !R.p.keep_states) {
        s = finish_trajectory(t, shared, d_samples);   // the default path to the end
        if (s != QT_OK) return s;
        continue;
      }
      QT_CUDA(cudaMemcpyAsync(dst, shared, sbytes, cudaMemcpyDeviceToDevice, R.st), "cudaMemcpyAsync(prefix)");
      R.stats.prefix_copies++;
      if (s1.diverge < nch) {
        s = run_from(t, dst, s1, D);
        if (s != QT_OK) return s;
      }
      s = finish_trajectory(t, dst, d_samples);
      if (s != QT_OK) return s;
    }
    return QT_OK;
  }

  qt_status measure(uint32_t t, const float2* psi, uint64_t* d_samples) {
    TraceRange tr("qt measure");
    const uint64_t traj = R.p.first_traj + t;
    const uint32_t M = static_cast<uint32_t>(R.masks.size());
    double N = 0.0;
    for (uint32_t g0 = 0; g0 < std::max<uint32_t>(M, 1); g0 += kExpGroup) {
      const int nm = static_cast<int>(std::min<uint32_t>(kExpGroup, M - std::min(M, g0)));
      QT_CUDA(launch_expect(psi, static_cast<int>(R.n), nm, R.masks.data() + std::min(M, g0), R.scr.s, R.st),
              "expectation kernel launch");
      QT_CUDA(cudaMemcpyAsync(pinned, R.scr.s.result, sizeof(double) * (kExpGroup + 1),
                              cudaMemcpyDeviceToHost, R.st), "cudaMemcpyAsync(expectation)");
      QT_CUDA(cudaStreamSynchronize(R.st), "cudaStreamSynchronize(expectation)");
      R.stats.d2h_bytes += sizeof(double) * (kExpGroup + 1);
      R.stats.kernel_launches += 2;
      N = pinned[0];
      for (int m = 0; m < nm; ++m) R.expect[static_cast<size_t>(t) * M + g0 + m] = pinned[1 + m] / N;
    }
    R.norms[t] = N;
    if (R.p.samples_per_traj) {
      QT_CUDA(launch_sample(psi, static_cast<int>(R.n), R.p.seed, traj, R.p.samples_per_traj,
                            d_samples + static_cast<size_t>(t) * R.p.samples_per_traj, R.scr.s, R.st,
                            R.readout.as<const double>()),
              "sampling kernel launch");
      R.stats.kernel_launches += 4;
    }
    return QT_OK;
  }
};

}  // namespace qt

extern "C" {

qt_status qt_kernel_arch(int32_t* binary_version, int32_t* ptx_version) {
  clear_error();
  if (!binary_version || !ptx_version) return set_error(QT_ERR_INVALID_ARG, "qt_kernel_arch: NULL argument");
  int b = 0, p = 0;
  QT_CUDA(kernel_arch(&b, &p), "qt_kernel_arch: cudaFuncGetAttributes");
  *binary_version = b;
  *ptx_version = p;
  return QT_OK;
}

qt_status qt_set_allocator(qt_alloc_fn alloc, qt_free_fn free_fn, void* ctx) {
  clear_error();
  if ((alloc == nullptr) != (free_fn == nullptr))
    return set_error(QT_ERR_INVALID_ARG, "qt_set_allocator: give both functions or neither");
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_alloc.alloc = alloc;
  g_alloc.free = free_fn;
  g_alloc.ctx = ctx;
  return QT_OK;
}

// readout errors: 2n probabilities in [0, 1]; the sample index must fit the
// Philox counter layout (j << 6) | q
static qt_status check_readout(const double* ro, uint32_t n, uint64_t S, const char* who) {
  if (!ro) return QT_OK;
  if (S >= (1ull << 26)) return set_error(QT_ERR_INVALID_ARG, "%s: readout errors need fewer than 2^26 samples", who);
  for (uint32_t i = 0; i < 2 * n; ++i)
    if (!(ro[i] >= 0.0 && ro[i] <= 1.0))
      return set_error(QT_ERR_INVALID_ARG, "%s: readout error %u is %g (must be in [0, 1])", who, i, ro[i]);
  return QT_OK;
}

qt_status qt_run_trajectories(const qt_fused* f, const qt_run_params* p, qt_run** out) {
  clear_error();
  if (!f || !p || !out) return set_error(QT_ERR_INVALID_ARG, "qt_run_trajectories: NULL argument");
  *out = nullptr;
  if (p->mode != QT_DELAYED && p->mode != QT_EAGER)
    return set_error(QT_ERR_INVALID_ARG, "qt_run_trajectories: unknown mode %u", p->mode);
  if (p->precision != QT_FP32 && p->precision != QT_TF32X3)
    return set_error(QT_ERR_INVALID_ARG, "qt_run_trajectories: unknown precision %u", p->precision);
  if (p->num_z_masks && !p->z_masks)
    return set_error(QT_ERR_INVALID_ARG, "qt_run_trajectories: z_masks is NULL");
  const Circuit& c = *f->c;
  if (c.n < 1) return set_error(QT_ERR_INVALID_ARG, "qt_run_trajectories: empty circuit");
  {
    const qt_status rs = check_readout(p->readout_error, c.n, p->samples_per_traj, "qt_run_trajectories");
    if (rs != QT_OK) return rs;
  }
  for (const auto& g : f->gates)
    if (g.targets.size() > 5 && c.n < 13)
      return set_error(QT_ERR_UNSUPPORTED, "qt_run_trajectories: fused width %zu needs n >= 13", g.targets.size());
  std::unique_ptr<qt_run> R(new (std::nothrow) qt_run());
  if (!R) return set_error(QT_ERR_OUT_OF_MEMORY, "qt_run_trajectories: host allocation");
  R->f = f;
  R->p = *p;
  R->p.z_masks = nullptr;
  R->p.readout_error = nullptr;
  R->masks.assign(p->z_masks, p->z_masks + p->num_z_masks);
  R->n = c.n;
  R->T = p->num_traj;
  R->nch = static_cast<uint32_t>(c.channel_op.size());
  R->st = static_cast<cudaStream_t>(p->stream);
  R->kraus.assign(static_cast<size_t>(R->T) * R->nch, -1);
  R->stage.assign(static_cast<size_t>(R->T) * R->nch, 0);
  R->samples.assign(static_cast<size_t>(R->T) * p->samples_per_traj, 0);
  R->expect.assign(static_cast<size_t>(R->T) * R->masks.size(), 0.0);
  R->norms.assign(R->T, 0.0);
  R->stats.num_traj = R->T;
  R->stats.num_channels = R->nch;
  if (!R->scr.alloc(static_cast<int>(c.n), R->st))
    return set_error(QT_ERR_OUT_OF_MEMORY, "qt_run_trajectories: scratch allocation");
  if (p->readout_error) {
    if (!R->readout.alloc(sizeof(double) * 2 * c.n, R->st))
      return set_error(QT_ERR_OUT_OF_MEMORY, "qt_run_trajectories: readout errors");
    QT_CUDA(cudaMemcpyAsync(R->readout.p, p->readout_error, sizeof(double) * 2 * c.n, cudaMemcpyHostToDevice, R->st),
            "cudaMemcpyAsync(readout)");
    R->stats.h2d_bytes += sizeof(double) * 2 * c.n;
  }
  const size_t sbytes = sizeof(float2) << c.n;
  // shared default-choice prefix: delayed mode only (the conventional
  // algorithm evaluates every channel, so no two trajectories share a prefix)
  const bool share = (p->flags & QT_FLAG_SHARE_PREFIX) && p->mode == QT_DELAYED && p->num_traj > 1;
  DevBuf work, dsamp, shared;
  if (!p->keep_states && !work.alloc(sbytes, R->st))
    return set_error(QT_ERR_OUT_OF_MEMORY, "qt_run_trajectories: state allocation (%zu bytes)", sbytes);
  if (share && !shared.alloc(sbytes, R->st))
    return set_error(QT_ERR_OUT_OF_MEMORY, "qt_run_trajectories: shared-prefix state allocation (%zu bytes)", sbytes);
  if (p->keep_states) {
    R->states.resize(R->T);
    for (uint32_t t = 0; t < R->T; ++t)
      if (!R->states[t].alloc(sbytes, R->st))
        return set_error(QT_ERR_OUT_OF_MEMORY, "qt_run_trajectories: state %u allocation (%zu bytes)", t, sbytes);
  }
  const size_t nsamp = static_cast<size_t>(R->T) * p->samples_per_traj;
  if (nsamp && !dsamp.alloc(sizeof(uint64_t) * nsamp, R->st))
    return set_error(QT_ERR_OUT_OF_MEMORY, "qt_run_trajectories: sample buffer");
  Controller ctl(*R);
  QT_CUDA(cudaMallocHost(&ctl.pinned, sizeof(double) * 128), "cudaMallocHost");
  cudaEvent_t e0, e1;
  QT_CUDA(cudaEventCreate(&e0), "cudaEventCreate");
  QT_CUDA(cudaEventCreate(&e1), "cudaEventCreate");
  struct EvGuard { cudaEvent_t a, b; ~EvGuard() { cudaEventDestroy(a); cudaEventDestroy(b); } } eg{e0, e1};
  QT_CUDA(cudaEventRecord(e0, R->st), "cudaEventRecord");
  if (share) {
    qt_status s = ctl.run_shared(shared.as<float2>(), work.as<float2>(), dsamp.as<uint64_t>());
    if (s != QT_OK) return s;
  } else {
    for (uint32_t t = 0; t < R->T; ++t) {
      float2* psi = p->keep_states ? R->states[t].as<float2>() : work.as<float2>();
      qt_status s = ctl.trajectory(t, psi);
      if (s != QT_OK) return s;
      s = ctl.finish_trajectory(t, psi, dsamp.as<uint64_t>());
      if (s != QT_OK) return s;
    }
  }
  QT_CUDA(cudaEventRecord(e1, R->st), "cudaEventRecord");
  if (nsamp) {
    QT_CUDA(cudaMemcpyAsync(R->samples.data(), dsamp.p, sizeof(uint64_t) * nsamp, cudaMemcpyDeviceToHost, R->st),
            "cudaMemcpyAsync(samples)");
    R->stats.d2h_bytes += sizeof(uint64_t) * nsamp;
  }
  QT_CUDA(cudaStreamSynchronize(R->st), "cudaStreamSynchronize(run)");
  float ms = 0.f;
  QT_CUDA(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
  R->stats.device_ms = ms;
  R->stats.gate_ops = f->gate_ops * R->T;
  *out = R.release();
  return QT_OK;
}

void qt_run_destroy(qt_run* r) { delete r; }

qt_status qt_run_stats(const qt_run* r, qt_run_stats_t* out) {
  clear_error();
  if (!r || !out) return set_error(QT_ERR_INVALID_ARG, "qt_run_stats: NULL argument");
  *out = r->stats;
  return QT_OK;
}

qt_status qt_run_kraus_indices(const qt_run* r, int32_t* kraus, int32_t* stage, size_t cap) {
  clear_error();
  if (!r) return set_error(QT_ERR_INVALID_ARG, "qt_run_kraus_indices: NULL run");
  const size_t need = r->kraus.size();
  if ((kraus || stage) && cap < need)
    return set_error(QT_ERR_INVALID_ARG, "qt_run_kraus_indices: cap %zu < %zu", cap, need);
  if (kraus) std::memcpy(kraus, r->kraus.data(), sizeof(int32_t) * need);
  if (stage) std::memcpy(stage, r->stage.data(), sizeof(int32_t) * need);
  return QT_OK;
}

qt_status qt_sample(qt_run* r, uint32_t S, uint64_t* out) {
  clear_error();
  if (!r || (!out && S)) return set_error(QT_ERR_INVALID_ARG, "qt_sample: NULL argument");
  if (S == r->p.samples_per_traj) {
    std::memcpy(out, r->samples.data(), sizeof(uint64_t) * r->samples.size());
    return QT_OK;
  }
  if (r->states.empty())
    return set_error(QT_ERR_INVALID_ARG, "qt_sample: S=%u differs from the run's samples_per_traj=%u and states were not kept",
                     S, r->p.samples_per_traj);
  DevBuf d;
  if (!d.alloc(sizeof(uint64_t) * S * r->T, r->st)) return set_error(QT_ERR_OUT_OF_MEMORY, "qt_sample: buffer");
  for (uint32_t t = 0; t < r->T; ++t)
    QT_CUDA(launch_sample(r->states[t].as<float2>(), static_cast<int>(r->n), r->p.seed, r->p.first_traj + t, S,
                          d.as<uint64_t>() + static_cast<size_t>(t) * S, r->scr.s, r->st, r->readout.as<const double>()),
            "sampling kernel launch");
  QT_CUDA(cudaMemcpyAsync(out, d.p, sizeof(uint64_t) * S * r->T, cudaMemcpyDeviceToHost, r->st), "cudaMemcpyAsync");
  QT_CUDA(cudaStreamSynchronize(r->st), "cudaStreamSynchronize");
  return QT_OK;
}

qt_status qt_expectation(qt_run* r, uint32_t M, const uint64_t* masks, double* out) {
  clear_error();
  if (!r || (M && (!masks || !out))) return set_error(QT_ERR_INVALID_ARG, "qt_expectation: NULL argument");
  if (M == r->masks.size() && std::equal(r->masks.begin(), r->masks.end(), masks)) {
    std::memcpy(out, r->expect.data(), sizeof(double) * r->expect.size());
    return QT_OK;
  }
  if (r->states.empty())
    return set_error(QT_ERR_INVALID_ARG, "qt_expectation: masks differ from the run's and states were not kept");
  double* pinned = nullptr;
  QT_CUDA(cudaMallocHost(&pinned, sizeof(double) * (kExpGroup + 1)), "cudaMallocHost");
  for (uint32_t t = 0; t < r->T; ++t)
    for (uint32_t g0 = 0; g0 < M; g0 += kExpGroup) {
      const int nm = static_cast<int>(std::min<uint32_t>(kExpGroup, M - g0));
      cudaError_t e = launch_expect(r->states[t].as<float2>(), static_cast<int>(r->n), nm, masks + g0, r->scr.s, r->st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(pinned, r->scr.s.result, sizeof(double) * (kExpGroup + 1), cudaMemcpyDeviceToHost, r->st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(r->st);
      if (e != cudaSuccess) {
        cudaFreeHost(pinned);
        return cuda_fail(e, "qt_expectation");
      }
      for (int m = 0; m < nm; ++m) out[static_cast<size_t>(t) * M + g0 + m] = pinned[1 + m] / pinned[0];
    }
  cudaFreeHost(pinned);
  return QT_OK;
}

qt_status qt_run_norms(const qt_run* r, double* out) {
  clear_error();
  if (!r || !out) return set_error(QT_ERR_INVALID_ARG, "qt_run_norms: NULL argument");
  std::memcpy(out, r->norms.data(), sizeof(double) * r->norms.size());
  return QT_OK;
}

qt_status qt_run_state(const qt_run* r, uint32_t t, void* dst, size_t bytes) {
  clear_error();
  if (!r || !dst) return set_error(QT_ERR_INVALID_ARG, "qt_run_state: NULL argument");
  if (r->states.empty()) return set_error(QT_ERR_INVALID_ARG, "qt_run_state: run did not keep its states");
  if (t >= r->T) return set_error(QT_ERR_INVALID_ARG, "qt_run_state: trajectory %u out of range", t);
  const size_t sb = sizeof(float2) << r->n;
  if (bytes < sb) return set_error(QT_ERR_INVALID_ARG, "qt_run_state: %zu bytes < %zu", bytes, sb);
  DevBuf tmp;
  if (!tmp.alloc(sb, r->st)) return set_error(QT_ERR_OUT_OF_MEMORY, "qt_run_state: buffer");
  QT_CUDA(cudaMemcpyAsync(tmp.p, r->states[t].p, sb, cudaMemcpyDeviceToDevice, r->st), "cudaMemcpyAsync");
  const double N = r->norms[t];
  QT_CUDA(launch_scale(tmp.as<float2>(), static_cast<int>(r->n), static_cast<float>(1.0 / std::sqrt(N)), r->st),
          "scale kernel launch");
  QT_CUDA(cudaMemcpyAsync(dst, tmp.p, sb, cudaMemcpyDeviceToHost, r->st), "cudaMemcpyAsync");
  QT_CUDA(cudaStreamSynchronize(r->st), "cudaStreamSynchronize");
  return QT_OK;
}

// ---------------------------------------------------------------------------
// state-level calls
// ---------------------------------------------------------------------------
static qt_status check_state(const void* state, uint32_t n, const char* who) {
  if (!state) return set_error(QT_ERR_INVALID_ARG, "%s: state is NULL", who);
  if (reinterpret_cast<uintptr_t>(state) & 15u) return set_error(QT_ERR_INVALID_ARG, "%s: state not 16-byte aligned", who);
  if (n < 1 || n > QT_MAX_QUBITS) return set_error(QT_ERR_INVALID_ARG, "%s: n=%u outside 1..%d", who, n, QT_MAX_QUBITS);
  return QT_OK;
}

static qt_status check_qubits(uint32_t n, uint32_t q, const uint32_t* qubits, const char* who) {
  if (!qubits) return set_error(QT_ERR_INVALID_ARG, "%s: qubits is NULL", who);
  uint64_t m = 0;
  for (uint32_t b = 0; b < q; ++b) {
    if (qubits[b] >= n) return set_error(QT_ERR_INVALID_ARG, "%s: qubit %u >= n", who, qubits[b]);
    if (m & (1ull << qubits[b])) return set_error(QT_ERR_INVALID_ARG, "%s: repeated qubit", who);
    m |= 1ull << qubits[b];
  }
  return QT_OK;
}

qt_status qt_state_apply(void* state, uint32_t n, uint32_t q, const uint32_t* qubits, const double* U,
                         uint32_t precision, void* stream) {
  clear_error();
  qt_status s = check_state(state, n, "qt_state_apply");
  if (s != QT_OK) return s;
  const bool tc = precision == QT_TF32X3 && q >= 5 && tc_supported(static_cast<int>(n), static_cast<int>(q));
  if (q < 1 || q > n || q > 6 || (q == 6 && n < 13))
    return set_error(QT_ERR_UNSUPPORTED, "qt_state_apply: q=%u (1..min(n,5); 6 needs n >= 13)", q);
  if (precision != QT_FP32 && precision != QT_TF32X3) return set_error(QT_ERR_INVALID_ARG, "qt_state_apply: precision");
  if (!U) return set_error(QT_ERR_INVALID_ARG, "qt_state_apply: U is NULL");
  s = check_qubits(n, q, qubits, "qt_state_apply");
  if (s != QT_OK) return s;
  // reorder the matrix basis to ascending qubits
  std::vector<uint32_t> sorted(qubits, qubits + q);
  std::sort(sorted.begin(), sorted.end());
  int pos[QT_MAX_OP_QUBITS];
  for (uint32_t b = 0; b < q; ++b)
    pos[b] = static_cast<int>(std::lower_bound(sorted.begin(), sorted.end(), qubits[b]) - sorted.begin());
  const int D = 1 << q;
  auto perm = [&](int i) {   // user-basis index of sorted-basis index i
    int u = 0;
    for (uint32_t b = 0; b < q; ++b)
      if ((i >> pos[b]) & 1) u |= 1 << b;
    return u;
  };
  std::vector<float2> M(static_cast<size_t>(D) * D);
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) {
      const size_t e = static_cast<size_t>(perm(i)) * D + perm(j);
      M[static_cast<size_t>(i) * D + j] = make_float2(static_cast<float>(U[2 * e]), static_cast<float>(U[2 * e + 1]));
    }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (tc) {
    const int N = 2 << q;
    std::vector<float> W(static_cast<size_t>(N) * N);
    real_embedding(static_cast<int>(q), M.data(), W.data());
    DevBuf wd, ed;
    if (!wd.alloc(sizeof(float) * N * N, st) || !ed.alloc(sizeof(int), st))
      return set_error(QT_ERR_OUT_OF_MEMORY, "qt_state_apply: matrix buffer");
    QT_CUDA(cudaMemsetAsync(ed.p, 0, sizeof(int), st), "cudaMemsetAsync");
    QT_CUDA(cudaMemcpyAsync(wd.p, W.data(), sizeof(float) * N * N, cudaMemcpyHostToDevice, st), "cudaMemcpyAsync");
    QT_CUDA(launch_apply_tc(static_cast<float2*>(state), static_cast<int>(n), static_cast<int>(q), sorted.data(),
                            wd.as<float>(), ed.as<int>(), st),
            "qt_state_apply (tensor cores)");
    int e = 0;
    QT_CUDA(cudaMemcpyAsync(&e, ed.p, sizeof(int), cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync");
    QT_CUDA(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    if (e) return set_error(QT_ERR_TIMEOUT, "qt_state_apply: tensor-core kernel wait ran out (code %d)", e);
    return QT_OK;
  }
  if (q == 6) {
    DevBuf ud;
    if (!ud.alloc(sizeof(float2) * 64 * 64, st)) return set_error(QT_ERR_OUT_OF_MEMORY, "qt_state_apply: matrix buffer");
    QT_CUDA(cudaMemcpyAsync(ud.p, M.data(), sizeof(float2) * 64 * 64, cudaMemcpyHostToDevice, st), "cudaMemcpyAsync");
    QT_CUDA(launch_apply6_fp32(static_cast<float2*>(state), static_cast<int>(n), sorted.data(), ud.as<float2>(), st),
            "qt_state_apply (6 qubits)");
    QT_CUDA(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    return QT_OK;
  }
  QT_CUDA(launch_apply(static_cast<float2*>(state), static_cast<int>(n), static_cast<int>(q), sorted.data(), M.data(), st),
          "qt_state_apply");
  return QT_OK;
}

qt_status qt_state_reduced_density(const void* state, uint32_t n, uint32_t q, const uint32_t* qubits, double* out,
                                   void* stream) {
  clear_error();
  qt_status s = check_state(state, n, "qt_state_reduced_density");
  if (s != QT_OK) return s;
  if (q < 1 || q > n || q > static_cast<uint32_t>(kRdmMaxQ))
    return set_error(QT_ERR_UNSUPPORTED, "qt_state_reduced_density: q=%u (1..min(n,3))", q);
  if (!out) return set_error(QT_ERR_INVALID_ARG, "qt_state_reduced_density: out is NULL");
  s = check_qubits(n, q, qubits, "qt_state_reduced_density");
  if (s != QT_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ScratchBufs scr;
  if (!scr.alloc(1, st)) return set_error(QT_ERR_OUT_OF_MEMORY, "qt_state_reduced_density: scratch");
  QT_CUDA(launch_rdm(static_cast<const float2*>(state), static_cast<int>(n), static_cast<int>(q), qubits, scr.s, st),
          "qt_state_reduced_density");
  double r[64];
  QT_CUDA(cudaMemcpyAsync(r, scr.s.result, sizeof(double) << (2 * q), cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync");
  QT_CUDA(cudaStreamSynchronize(st), "cudaStreamSynchronize");
  rdm_unpack(static_cast<int>(q), r, out);
  return QT_OK;
}

qt_status qt_state_kraus_probabilities(const void* state, uint32_t n, uint32_t q, const uint32_t* qubits,
                                       uint32_t num_ops, const double* ops, double* P, double* N, void* stream) {
  clear_error();
  qt_status s = check_state(state, n, "qt_state_kraus_probabilities");
  if (s != QT_OK) return s;
  if (q < 1 || q > n || q > QT_MAX_OP_QUBITS)
    return set_error(QT_ERR_UNSUPPORTED, "qt_state_kraus_probabilities: q=%u (1..min(n,6))", q);
  if (num_ops < 1 || num_ops > 64 || !ops || !P || !N)
    return set_error(QT_ERR_INVALID_ARG, "qt_state_kraus_probabilities: NULL argument or num_ops outside 1..64");
  s = check_qubits(n, q, qubits, "qt_state_kraus_probabilities");
  if (s != QT_OK) return s;
  const int D = 1 << q;
  const size_t mat = static_cast<size_t>(D) * D;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ScratchBufs scr;
  if (!scr.alloc(1, st)) return set_error(QT_ERR_OUT_OF_MEMORY, "qt_state_kraus_probabilities: scratch");
  if (q <= kRdmMaxQ) {                     // P_i = tr(K_i^dag K_i rho) from the reduced density
    QT_CUDA(launch_rdm(static_cast<const float2*>(state), static_cast<int>(n), static_cast<int>(q), qubits, scr.s, st),
            "qt_state_kraus_probabilities");
    double r[64], rho[2 * 64];
    QT_CUDA(cudaMemcpyAsync(r, scr.s.result, sizeof(double) << (2 * q), cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync");
    QT_CUDA(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    rdm_unpack(static_cast<int>(q), r, rho);
    *N = 0.0;
    for (int b = 0; b < D; ++b) *N += rho[2 * (b * D + b)];
    for (uint32_t i = 0; i < num_ops; ++i) {
      const double* K = ops + 2 * mat * i;
      double acc = 0.0;                    // sum_{a,b} (K^dag K)[a][b] rho[b][a]
      for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b) {
          cd m(0.0, 0.0);
          for (int j = 0; j < D; ++j)
            m += std::conj(cd(K[2 * (j * D + a)], K[2 * (j * D + a) + 1])) * cd(K[2 * (j * D + b)], K[2 * (j * D + b) + 1]);
          acc += (m * cd(rho[2 * (b * D + a)], rho[2 * (b * D + a) + 1])).real();
        }
      P[i] = acc;
    }
    return QT_OK;
  }
  const int G = kraus_group(static_cast<int>(q));
  DevBuf kd;
  if (!kd.alloc(sizeof(float2) * G * mat, st)) return set_error(QT_ERR_OUT_OF_MEMORY, "qt_state_kraus_probabilities: operators");
  std::vector<float2> tmp;
  for (uint32_t g0 = 0; g0 < num_ops; g0 += static_cast<uint32_t>(G)) {
    tmp.assign(G * mat, make_float2(0.f, 0.f));
    for (uint32_t j = 0; j < static_cast<uint32_t>(G) && g0 + j < num_ops; ++j)
      for (size_t e = 0; e < mat; ++e) {
        const double* K = ops + 2 * (mat * (g0 + j) + e);
        tmp[j * mat + e] = make_float2(static_cast<float>(K[0]), static_cast<float>(K[1]));
      }
    QT_CUDA(cudaMemcpyAsync(kd.p, tmp.data(), sizeof(float2) * G * mat, cudaMemcpyHostToDevice, st), "cudaMemcpyAsync");
    QT_CUDA(launch_kraus_norms(static_cast<const float2*>(state), static_cast<int>(n), static_cast<int>(q), qubits, G,
                               kd.as<float2>(), scr.s, st),
            "qt_state_kraus_probabilities");
    double r[17];
    QT_CUDA(cudaMemcpyAsync(r, scr.s.result, sizeof(double) * (G + 1), cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync");
    QT_CUDA(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    *N = r[0];
    for (uint32_t j = 0; j < static_cast<uint32_t>(G) && g0 + j < num_ops; ++j) P[g0 + j] = r[1 + j];
  }
  return QT_OK;
}

qt_status qt_state_sample(const void* state, uint32_t n, uint64_t seed, uint64_t traj, uint32_t S, uint64_t* out,
                          const double* readout_error, void* stream) {
  clear_error();
  qt_status s = check_state(state, n, "qt_state_sample");
  if (s != QT_OK) return s;
  if (S && !out) return set_error(QT_ERR_INVALID_ARG, "qt_state_sample: out is NULL");
  s = check_readout(readout_error, n, S, "qt_state_sample");
  if (s != QT_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ScratchBufs scr;
  DevBuf d, ro;
  if (!scr.alloc(static_cast<int>(n), st) || (S && !d.alloc(sizeof(uint64_t) * S, st)) ||
      (readout_error && !ro.alloc(sizeof(double) * 2 * n, st)))
    return set_error(QT_ERR_OUT_OF_MEMORY, "qt_state_sample: scratch");
  if (readout_error)
    QT_CUDA(cudaMemcpyAsync(ro.p, readout_error, sizeof(double) * 2 * n, cudaMemcpyHostToDevice, st),
            "cudaMemcpyAsync(readout)");
  QT_CUDA(launch_sample(static_cast<const float2*>(state), static_cast<int>(n), seed, traj, S, d.as<uint64_t>(), scr.s, st,
                        ro.as<const double>()),
          "qt_state_sample");
  if (S) QT_CUDA(cudaMemcpyAsync(out, d.p, sizeof(uint64_t) * S, cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync");
  QT_CUDA(cudaStreamSynchronize(st), "cudaStreamSynchronize");
  return QT_OK;
}

qt_status qt_state_cdf(const void* state, uint32_t n, double* out, void* stream) {
  clear_error();
  qt_status s = check_state(state, n, "qt_state_cdf");
  if (s != QT_OK) return s;
  if (n > 28) return set_error(QT_ERR_UNSUPPORTED, "qt_state_cdf: n=%u (at most 28: 2^n doubles go to the host)", n);
  if (!out) return set_error(QT_ERR_INVALID_ARG, "qt_state_cdf: out is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ScratchBufs scr;
  DevBuf d;
  const size_t bytes = sizeof(double) << n;
  if (!scr.alloc(static_cast<int>(n), st) || !d.alloc(bytes, st))
    return set_error(QT_ERR_OUT_OF_MEMORY, "qt_state_cdf: scratch");
  QT_CUDA(launch_cdf_values(static_cast<const float2*>(state), static_cast<int>(n), scr.s, d.as<double>(), st),
          "qt_state_cdf");
  QT_CUDA(cudaMemcpyAsync(out, d.p, bytes, cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync");
  QT_CUDA(cudaStreamSynchronize(st), "cudaStreamSynchronize");
  return QT_OK;
}

qt_status qt_state_expect_z(const void* state, uint32_t n, uint32_t M, const uint64_t* masks, double* out,
                            void* stream) {
  clear_error();
  qt_status s = check_state(state, n, "qt_state_expect_z");
  if (s != QT_OK) return s;
  if (M && (!masks || !out)) return set_error(QT_ERR_INVALID_ARG, "qt_state_expect_z: NULL argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ScratchBufs scr;
  if (!scr.alloc(1, st)) return set_error(QT_ERR_OUT_OF_MEMORY, "qt_state_expect_z: scratch");
  double r[kExpGroup + 1];
  for (uint32_t g0 = 0; g0 < M; g0 += kExpGroup) {
    const int nm = static_cast<int>(std::min<uint32_t>(kExpGroup, M - g0));
    QT_CUDA(launch_expect(static_cast<const float2*>(state), static_cast<int>(n), nm, masks + g0, scr.s, st),
            "qt_state_expect_z");
    QT_CUDA(cudaMemcpyAsync(r, scr.s.result, sizeof(r), cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync");
    QT_CUDA(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    for (int m = 0; m < nm; ++m) out[g0 + m] = r[1 + m] / r[0];
  }
  return QT_OK;
}

}  // extern "C"
