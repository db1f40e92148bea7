// Internal types of the quantum-trajectory library (host side).
#pragma once
#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include "qt.h"

namespace qt {

using cd = std::complex<double>;

// One operation of the circuit (Sec. II).
struct Op {
  int kind = QT_OP_GATE;
  uint32_t moment = 0;
  uint32_t q = 0;                 // number of qubits
  uint32_t qubits[QT_MAX_OP_QUBITS] = {0};
  uint32_t num_ops = 1;           // 1 for gates
  std::vector<cd> mats;           // num_ops x d x d: gate U, Kraus K_i, or mixture U_i
  std::vector<double> probs;      // mixture p_i (renormalized)
  std::vector<double> pbar;       // channel lower bounds (Sec. III.E)
  std::vector<cd> kraus;          // Kraus form: K_i, or sqrt(p_i) U_i for mixtures
  std::vector<cd> mtm;            // K_i^dag K_i (Kraus form)
  bool diag_mtm = false;          // every K_i^dag K_i is diagonal
  int channel = -1;               // channel ordinal (circuit order), -1 for gates
  int def = 0;                    // default operator: largest pbar (lowest index on ties)
  double s = 0.0;                 // sum of the lower bounds
  uint32_t dim() const { return 1u << q; }
  const cd* mat(uint32_t i) const { return mats.data() + static_cast<size_t>(i) * dim() * dim(); }
  const cd* kraus_op(uint32_t i) const {
    return kraus.data() + static_cast<size_t>(i) * dim() * dim();
  }
  const cd* mtm_op(uint32_t i) const {
    return mtm.data() + static_cast<size_t>(i) * dim() * dim();
  }
};

struct Circuit {
  uint32_t n = 0;
  std::vector<Op> ops;
  std::vector<uint32_t> channel_op;   // op index of channel c
};

struct FusedGate {
  std::vector<uint32_t> targets;      // sorted qubits, width = targets.size()
  std::vector<uint32_t> members;      // op indices in execution order
  std::vector<cd> def;                // row-major default matrix (slots on their default op)
  bool has_channel = false;
};

struct Fused {
  const Circuit* c = nullptr;
  uint32_t kmax = 4;
  std::vector<FusedGate> gates;
  std::vector<uint32_t> gate_of_op;   // fused gate containing op i
  uint64_t gate_ops = 0;              // unfused gates
};

// ---- status / error message (thread local) --------------------------------
qt_status set_error(qt_status s, const char* fmt, ...);
void clear_error();

// ---- host linear algebra (host_circuit.cpp) --------------------------------
// smallest eigenvalue of a Hermitian d x d matrix (row-major)
double hermitian_min_eig(int d, const cd* A);
// v (2^w) <- A v where A acts on `q` qubits at positions pos[0..q-1] of the
// w-qubit index (bit b of A's index <-> position pos[b])
void apply_small(cd* v, int w, int q, const int* pos, const cd* A);
// matrix (row-major, 2^w x 2^w, basis `targets`) of the product of ops, in
// order, each given by (op index, operator matrix)
void compose(const Circuit& c, const std::vector<uint32_t>& targets,
             const std::vector<std::pair<uint32_t, const cd*>>& seq, std::vector<cd>& out);

// ---- fusion (host_fuse.cpp) -------------------------------------------------
qt_status fuse_circuit(const Circuit& c, uint32_t kmax, Fused& f);

}  // namespace qt

struct qt_circuit : qt::Circuit {};
struct qt_fused : qt::Fused {};

namespace qt {

// ---- merged batched launches (batch.cu), the serving form's batch lane -----
// One trajectory of a merged launch: its fused circuit, Philox key,
// trajectory id and sample count.  Trajectories of different requests share
// one persistent launch; each one's results depend only on these fields.
struct LaneTraj {
  const qt_fused* f;
  uint64_t seed, traj;
  uint32_t S;
};
struct BatchLane;
// A lane owns its stream-ordered device buffers (tables and outputs grow as
// needed; the global-memory state slots are sized once for states of up to
// max_n qubits) and reuses them across launches.
qt_status lane_create(uint32_t max_n, void* stream, BatchLane** out);
void lane_destroy(BatchLane* l);
// Run every trajectory (n <= max_n) in one launch of each state class on the
// lane's stream; samples: sum of S entries in trajectory order; flushes: one
// count per trajectory.  Blocks until the results are on the host.
qt_status lane_run(BatchLane* l, uint32_t num, const LaneTraj* tr, uint64_t* samples, uint32_t* flushes);


}  // namespace qt
