/*
 * oracle.h -- plain FP64 CPU reference for the quantum-trajectory method of
 * "Simulations of Quantum Circuits with Approximate Noise using qsim and
 * Cirq" (arXiv 2111.02396).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline / reference arm call this code.  It shares no
 * source with the CUDA library and is deliberately slow and unfused: every
 * operation is applied one at a time, exactly as the paper's algorithms
 * state them.
 *
 * Conventions: amplitude index bit j is qubit j; an operator on qubits
 * Q[0..q-1] is a 2^q x 2^q row-major complex matrix whose index bit b is
 * qubit Q[b].
 */
#ifndef QT_ORACLE_H
#define QT_ORACLE_H
#include <stdint.h>
#include <complex.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef double _Complex orc_cplx;

enum { ORC_GATE = 0, ORC_KRAUS = 1, ORC_MIXTURE = 2 };
enum { ORC_DELAYED = 0, ORC_EAGER = 1, ORC_CUMULATIVE = 2 };

/* A circuit as flat arrays (op i uses qubits[qoff[i] .. qoff[i]+nq[i]) and
 * matrices mats[moff[i] ..] of nmat[i] operators, each 4^nq[i] entries). */
typedef struct {
  int32_t num_qubits;
  int32_t num_ops;
  const int32_t* kind;
  const int32_t* nq;
  const int32_t* qoff;
  const int32_t* qubits;
  const int32_t* nmat;
  const int64_t* moff;     /* offset in complex elements */
  const orc_cplx* mats;
  const int64_t* poff;     /* offset of op i's probabilities in probs (mixtures) */
  const double* probs;
} orc_circuit;

/* Philox4x32-10 block function (Salmon et al., SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* Uniform double in [0,1) from counter (traj, stream, index), key = seed. */
double orc_u01(uint64_t seed, uint64_t traj, uint32_t stream, uint32_t index);

/* Alg. 1: apply a 2^q x 2^q matrix to every gather set of the state. */
void orc_apply(orc_cplx* psi, int n, int q, const int32_t* qubits, const orc_cplx* U);
/* <psi|psi> with a fixed summation order. */
double orc_norm2(const orc_cplx* psi, int n);
/* P_i = <psi|K_i^dag K_i|psi> for i < nk, evaluated in place (Alg. 2, step 14). */
void orc_kraus_norms(const orc_cplx* psi, int n, int q, const int32_t* qubits,
                     int nk, const orc_cplx* K, double* P);
/* Smallest eigenvalue of K^dag K (= smallest singular value of K, squared). */
double orc_lower_bound(int q, const orc_cplx* K);

/* One trajectory of Alg. 2 (DELAYED), of the conventional algorithm (EAGER,
 * same two-stage partition of [0,1)), or of textbook cumulative sampling
 * (CUMULATIVE).  psi (2^n) receives the final normalized state.  Per
 * channel c (circuit order): kraus_idx[c], stage[c] (1 or 2) and margin[c]
 * = distance of the draw to the nearest partition boundary.  max_ops < 0
 * runs the whole circuit; otherwise it stops after max_ops ops (timing
 * samples).  Returns the number of stage-2 evaluations (flushes). */
int orc_run_trajectory(const orc_circuit* c, int mode, uint64_t seed, uint64_t traj,
                       int64_t max_ops, orc_cplx* psi, int32_t* kraus_idx,
                       int32_t* stage, double* margin);

/* T trajectories traj0..traj0+T-1, parallel over trajectories (small n). */
void orc_run_trajectories(const orc_circuit* c, int mode, uint64_t seed, uint64_t traj0,
                          int T, orc_cplx* psis, int32_t* kraus_idx, int32_t* stage,
                          double* margin, int32_t* flushes);

/* S samples: smallest x with u_j * C(2^n-1) < C(x), C the cumulative sum of
 * |psi_x|^2 in index order, u_j from Philox stream 1.  margin_j = distance
 * of u_j*C(2^n-1) to the nearest of C(x-1), C(x), relative to C(2^n-1). */
void orc_sample(const orc_cplx* psi, int n, uint64_t seed, uint64_t traj, int S,
                uint64_t* out, double* margin);
/* <Z_mask> = sum_x |psi_x|^2 (-1)^popcount(x & mask) / <psi|psi>. */
void orc_expect_z(const orc_cplx* psi, int n, int M, const uint64_t* masks, double* out);

/* Readout errors (Sec. V.A, parallel readout errors): qubit q of sample j,
 * whose true value is b, is read as 1 - b with probability err[2q + b]
 * (err[2q] = P(read 1 | 0), err[2q + 1] = P(read 0 | 1)).  The decision
 * draws u = u01 from Philox stream 2 at index (j << 6) | q and flips when
 * u < err[2q + b].  bits[0..S) is modified in place. */
void orc_readout(uint64_t* bits, int S, int n, const double* err, uint64_t seed, uint64_t traj);

/* Exact density-matrix evolution of the whole circuit from |0..0><0..0|:
 * rho <- U rho U^dag for gates, rho <- sum_i K_i rho K_i^dag for channels.
 * rho is 4^n complex, element (r, c) at index r + c * 2^n. */
void orc_density_evolve(const orc_circuit* c, orc_cplx* rho);

#ifdef __cplusplus
}
#endif
#endif
