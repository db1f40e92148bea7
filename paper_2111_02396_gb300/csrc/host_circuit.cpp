// Circuit IR, validation and the Kraus lower bounds of Sec. III.E.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>

#include "qt_internal.h"

namespace qt {

static thread_local std::string g_err;

qt_status set_error(qt_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

void clear_error() { g_err.clear(); }

// Smallest eigenvalue of a Hermitian matrix by cyclic Jacobi sweeps with
// complex rotations: each (p,q) step first removes the phase of a_pq with a
// diagonal unitary, then zeroes it with a real plane rotation.
double hermitian_min_eig(int d, const cd* Ain) {
  if (d == 1) return Ain[0].real();
  if (d == 2) {  // closed form of the 2x2 Hermitian eigenproblem
    const double a = Ain[0].real(), b = Ain[3].real();
    const double h = 0.5 * (a - b);
    return 0.5 * (a + b) - std::sqrt(h * h + std::norm(Ain[1]));
  }
  std::vector<cd> A(Ain, Ain + static_cast<size_t>(d) * d);
  auto at = [&](int i, int j) -> cd& { return A[static_cast<size_t>(i) * d + j]; };
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, dia = 0.0;
    for (int i = 0; i < d; ++i) {
      dia += std::norm(at(i, i));
      for (int j = i + 1; j < d; ++j) off += std::norm(at(i, j));
    }
    if (off == 0.0 || off < 1e-32 * dia) break;
    for (int p = 0; p < d; ++p)
      for (int q = p + 1; q < d; ++q) {
        const double r = std::abs(at(p, q));
        if (r == 0.0) continue;
        const cd ph = at(p, q) / r;             // e^{i phi}
        const double a = at(p, p).real(), b = at(q, q).real();
        const double theta = (b - a) / (2.0 * r);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        const cd e = std::conj(ph);              // e^{-i phi}
        for (int k = 0; k < d; ++k) {            // A <- A J,  J = diag(1, e) R
          const cd xp = at(k, p), xq = at(k, q);
          at(k, p) = c * xp - s * e * xq;
          at(k, q) = s * xp + c * e * xq;
        }
        for (int k = 0; k < d; ++k) {            // A <- J^dag A
          const cd xp = at(p, k), xq = at(q, k);
          at(p, k) = c * xp - s * ph * xq;
          at(q, k) = s * xp + c * ph * xq;
        }
      }
  }
  double m = at(0, 0).real();
  for (int i = 1; i < d; ++i) m = std::min(m, at(i, i).real());
  return m;
}

void apply_small(cd* v, int w, int q, const int* pos, const cd* A) {
  const int D = 1 << w, M = 1 << q;
  int mask = 0;
  for (int b = 0; b < q; ++b) mask |= 1 << pos[b];
  cd in[64], out[64];
  int idx[64];
  for (int base = 0; base < D; ++base) {
    if (base & mask) continue;
    for (int k = 0; k < M; ++k) {
      int x = base;
      for (int b = 0; b < q; ++b)
        if ((k >> b) & 1) x |= 1 << pos[b];
      idx[k] = x;
      in[k] = v[x];
    }
    for (int j = 0; j < M; ++j) {
      cd acc = 0.0;
      for (int k = 0; k < M; ++k) acc += A[j * M + k] * in[k];
      out[j] = acc;
    }
    for (int j = 0; j < M; ++j) v[idx[j]] = out[j];
  }
}

void compose(const Circuit& c, const std::vector<uint32_t>& targets,
             const std::vector<std::pair<uint32_t, const cd*>>& seq, std::vector<cd>& out) {
  const int w = static_cast<int>(targets.size());
  const int D = 1 << w;
  std::vector<cd> colmaj(static_cast<size_t>(D) * D, cd(0.0));
  for (int j = 0; j < D; ++j) colmaj[static_cast<size_t>(j) * D + j] = 1.0;
  for (const auto& st : seq) {
    const Op& op = c.ops[st.first];
    int pos[QT_MAX_OP_QUBITS];
    for (uint32_t b = 0; b < op.q; ++b) {
      pos[b] = static_cast<int>(std::lower_bound(targets.begin(), targets.end(), op.qubits[b]) -
                                targets.begin());
    }
    for (int j = 0; j < D; ++j)
      apply_small(&colmaj[static_cast<size_t>(j) * D], w, static_cast<int>(op.q), pos, st.second);
  }
  out.assign(static_cast<size_t>(D) * D, cd(0.0));
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) out[static_cast<size_t>(i) * D + j] = colmaj[static_cast<size_t>(j) * D + i];
}

static void matmul_dagger_a(int d, const cd* A, cd* out) {  // out = A^dag A
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      cd acc = 0.0;
      for (int k = 0; k < d; ++k) acc += std::conj(A[k * d + i]) * A[k * d + j];
      out[i * d + j] = acc;
    }
}

static double max_dev_from_identity(int d, const cd* S) {
  double m = 0.0;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) m = std::max(m, std::abs(S[i * d + j] - (i == j ? 1.0 : 0.0)));
  return m;
}

}  // namespace qt

using namespace qt;

extern "C" {

const char* qt_last_error(void) { return g_err.c_str(); }

qt_status qt_circuit_create(uint32_t num_qubits, uint32_t num_ops, const qt_op* ops,
                            qt_circuit** out) {
  clear_error();
  if (!out) return set_error(QT_ERR_INVALID_ARG, "qt_circuit_create: out is NULL");
  *out = nullptr;
  if (num_qubits < 1 || num_qubits > QT_MAX_QUBITS)
    return set_error(QT_ERR_INVALID_ARG, "qt_circuit_create: num_qubits %u outside 1..%d",
                     num_qubits, QT_MAX_QUBITS);
  if (num_ops > 0 && !ops) return set_error(QT_ERR_INVALID_ARG, "qt_circuit_create: ops is NULL");
  qt_circuit* c = new (std::nothrow) qt_circuit();
  if (!c) return set_error(QT_ERR_OUT_OF_MEMORY, "qt_circuit_create: host allocation");
  c->n = num_qubits;
  c->ops.resize(num_ops);
  std::map<uint32_t, uint64_t> moment_mask;
  uint32_t last_moment = 0;
  int channels = 0;
  for (uint32_t i = 0; i < num_ops; ++i) {
    const qt_op& in = ops[i];
    Op& op = c->ops[i];
    auto fail = [&](qt_status s, const char* what) {
      delete c;
      return set_error(s, "qt_circuit_create: op %u: %s", i, what);
    };
    if (in.kind != QT_OP_GATE && in.kind != QT_OP_KRAUS && in.kind != QT_OP_MIXTURE)
      return fail(QT_ERR_INVALID_ARG, "unknown kind");
    if (in.num_qubits < 1 || in.num_qubits > QT_MAX_OP_QUBITS)
      return fail(QT_ERR_INVALID_ARG, "num_qubits outside 1..6");
    if (!in.mats) return fail(QT_ERR_INVALID_ARG, "mats is NULL");
    if (in.num_ops < 1 || in.num_ops > 64) return fail(QT_ERR_INVALID_ARG, "num_ops outside 1..64");
    if (in.kind == QT_OP_GATE && in.num_ops != 1) return fail(QT_ERR_INVALID_ARG, "a gate has num_ops 1");
    if (i > 0 && in.moment < last_moment) return fail(QT_ERR_INVALID_ARG, "moments must not decrease");
    last_moment = in.moment;
    uint64_t mask = 0;
    for (uint32_t b = 0; b < in.num_qubits; ++b) {
      if (in.qubits[b] >= num_qubits) return fail(QT_ERR_INVALID_ARG, "qubit out of range");
      if (mask & (1ull << in.qubits[b])) return fail(QT_ERR_INVALID_ARG, "repeated qubit");
      mask |= 1ull << in.qubits[b];
      op.qubits[b] = in.qubits[b];
    }
    uint64_t& mm = moment_mask[in.moment];
    if (mm & mask) return fail(QT_ERR_INVALID_ARG, "overlaps another op of its moment");
    mm |= mask;
    op.kind = in.kind;
    op.moment = in.moment;
    op.q = in.num_qubits;
    op.num_ops = in.num_ops;
    const uint32_t d = op.dim();
    const size_t dd = static_cast<size_t>(d) * d;
    op.mats.resize(dd * op.num_ops);
    for (size_t e = 0; e < dd * op.num_ops; ++e) op.mats[e] = cd(in.mats[2 * e], in.mats[2 * e + 1]);
    std::vector<cd> tmp(dd), sum(dd);
    if (op.kind == QT_OP_GATE || op.kind == QT_OP_MIXTURE) {
      for (uint32_t k = 0; k < op.num_ops; ++k) {
        matmul_dagger_a(static_cast<int>(d), op.mat(k), tmp.data());
        if (!(max_dev_from_identity(static_cast<int>(d), tmp.data()) <= 1e-8))
          return fail(QT_ERR_INVALID_ARG, "gate / mixture operator is not unitary (1e-8)");
      }
    }
    if (op.kind == QT_OP_GATE) continue;
    op.channel = channels++;
    c->channel_op.push_back(i);
    op.kraus.resize(dd * op.num_ops);
    op.mtm.resize(dd * op.num_ops);
    op.pbar.resize(op.num_ops);
    if (op.kind == QT_OP_MIXTURE) {
      if (!in.probs) return fail(QT_ERR_INVALID_ARG, "mixture probs is NULL");
      double ps = 0.0;
      for (uint32_t k = 0; k < op.num_ops; ++k) {
        if (!(in.probs[k] >= 0.0)) return fail(QT_ERR_INVALID_ARG, "negative mixture probability");
        ps += in.probs[k];
      }
      if (!(std::fabs(ps - 1.0) <= 1e-12)) return fail(QT_ERR_INVALID_ARG, "mixture probabilities do not sum to 1 (1e-12)");
      op.probs.resize(op.num_ops);
      for (uint32_t k = 0; k < op.num_ops; ++k) {
        op.probs[k] = in.probs[k] / ps;
        op.pbar[k] = op.probs[k];                  // K_i = sqrt(p_i) U_i: sigma_min^2 = p_i
        const double sp = std::sqrt(op.probs[k]);
        for (size_t e = 0; e < dd; ++e) op.kraus[k * dd + e] = sp * op.mats[k * dd + e];
      }
    } else {
      for (size_t e = 0; e < dd * op.num_ops; ++e) op.kraus[e] = op.mats[e];
    }
    std::fill(sum.begin(), sum.end(), cd(0.0));
    op.diag_mtm = true;
    for (uint32_t k = 0; k < op.num_ops; ++k) {
      cd* M = op.mtm.data() + k * dd;
      matmul_dagger_a(static_cast<int>(d), op.kraus_op(k), M);
      for (size_t e = 0; e < dd; ++e) sum[e] += M[e];
      for (uint32_t r = 0; r < d; ++r)
        for (uint32_t cc = 0; cc < d; ++cc)
          if (r != cc && std::abs(M[r * d + cc]) > 1e-15) op.diag_mtm = false;
      if (op.kind == QT_OP_KRAUS)
        op.pbar[k] = std::max(0.0, hermitian_min_eig(static_cast<int>(d), M));
    }
    if (op.kind == QT_OP_KRAUS && !(max_dev_from_identity(static_cast<int>(d), sum.data()) <= 1e-10))
      return fail(QT_ERR_NOT_CPTP, "sum_i K_i^dag K_i differs from I by more than 1e-10");
    op.s = 0.0;
    op.def = 0;
    for (uint32_t k = 0; k < op.num_ops; ++k) {
      op.s += op.pbar[k];
      if (op.pbar[k] > op.pbar[op.def]) op.def = static_cast<int>(k);
    }
  }
  *out = c;
  return QT_OK;
}

void qt_circuit_destroy(qt_circuit* c) { delete c; }

qt_status qt_channel_lower_bounds(const qt_circuit* c, uint32_t channel, double* pbar,
                                  size_t cap, uint32_t* num_ops) {
  clear_error();
  if (!c) return set_error(QT_ERR_INVALID_ARG, "qt_channel_lower_bounds: circuit is NULL");
  if (channel >= c->channel_op.size())
    return set_error(QT_ERR_INVALID_ARG, "qt_channel_lower_bounds: channel %u out of range", channel);
  const Op& op = c->ops[c->channel_op[channel]];
  if (num_ops) *num_ops = op.num_ops;
  if (pbar)
    for (uint32_t k = 0; k < op.num_ops && k < cap; ++k) pbar[k] = op.pbar[k];
  return QT_OK;
}

}  // extern "C"
