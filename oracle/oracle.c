/*
 * oracle.c -- plain FP64 CPU reference for the quantum-trajectory method of
 * arXiv 2111.02396 (qsim + Cirq noise simulation).
 *
 * TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU baseline).
 * Nothing here is fused, blocked or reordered beyond what the paper's
 * algorithms state; summations run in a fixed order so results do not
 * depend on the OpenMP thread count.
 *
 *   orc_apply           Alg. 1 (Sec. III.A): 2^(n-q) gather / matvec / scatter
 *   orc_kraus_norms     Alg. 2 step 14: p_i = <psi|K_i^dag K_i|psi>, in place
 *   orc_lower_bound     Sec. III.E: pbar_i = smallest singular value of K_i, squared
 *   orc_run_trajectory  Alg. 2 (delayed inner products) and the conventional
 *                       algorithm it is compared with (Sec. III.E)
 *   orc_sample          bitstring measurement of all qubits (Sec. V.C)
 *   orc_expect_z        Z-string expectations (densities, Sec. V.C)
 *   orc_readout         readout bit flips of sampled bitstrings (Sec. V.A)
 *   orc_density_evolve  exact channel evolution rho -> sum_i K_i rho K_i^dag
 */
#include "oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_CHUNK 4096  /* fixed summation chunk (elements or gather sets) */

/* ------------------------------------------------------------------------ */
/* Philox4x32-10: Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC'11.  Ten rounds of the Philox S-box with the       */
/* published multipliers and Weyl key increments.                          */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; round++) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

double orc_u01(uint64_t seed, uint64_t traj, uint32_t stream, uint32_t index) {
  uint32_t ctr[4] = {(uint32_t)traj, (uint32_t)(traj >> 32), stream, index};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t w[4];
  orc_philox4x32_10(ctr, key, w);
  /* 53 random bits: 27 from w0, 26 from w1 */
  double hi = (double)(w[0] >> 5);
  double lo = (double)(w[1] >> 6);
  return (hi * 67108864.0 + lo) * (1.0 / 9007199254740992.0);
}

/* ------------------------------------------------------------------------ */
/* Alg. 1                                                                   */
/* ------------------------------------------------------------------------ */
static void sorted_copy(int q, const int32_t* qubits, int32_t* s) {
  for (int i = 0; i < q; i++) s[i] = qubits[i];
  for (int i = 1; i < q; i++)
    for (int j = i; j > 0 && s[j - 1] > s[j]; j--) {
      int32_t t = s[j]; s[j] = s[j - 1]; s[j - 1] = t;
    }
}

/* base index of gather set i: i with a zero bit inserted at every gate qubit */
static uint64_t insert_zeros(uint64_t i, int q, const int32_t* sorted) {
  uint64_t x = i;
  for (int b = 0; b < q; b++) {
    uint64_t p = (uint64_t)sorted[b];
    uint64_t low = x & ((1ull << p) - 1ull);
    x = ((x >> p) << (p + 1)) | low;
  }
  return x;
}

/* member k of the gather set with base `base`: bit b of k goes to qubit Q[b] */
static uint64_t member(uint64_t base, int k, int q, const int32_t* qubits) {
  uint64_t x = base;
  for (int b = 0; b < q; b++)
    if ((k >> b) & 1) x |= 1ull << qubits[b];
  return x;
}

void orc_apply(orc_cplx* psi, int n, int q, const int32_t* qubits, const orc_cplx* U) {
  int32_t s[8];
  sorted_copy(q, qubits, s);
  const int M = 1 << q;
  const int64_t sets = (int64_t)1 << (n - q);
#pragma omp parallel for schedule(static) if (n >= 17)
  for (int64_t i = 0; i < sets; i++) {
    orc_cplx v[64], w[64];
    uint64_t idx[64];
    uint64_t base = insert_zeros((uint64_t)i, q, s);
    for (int k = 0; k < M; k++) {
      idx[k] = member(base, k, q, qubits);
      v[k] = psi[idx[k]];
    }
    for (int j = 0; j < M; j++) {
      orc_cplx acc = 0.0;
      for (int k = 0; k < M; k++) acc += U[j * M + k] * v[k];
      w[j] = acc;
    }
    for (int j = 0; j < M; j++) psi[idx[j]] = w[j];
  }
}

static double abs2(orc_cplx z) { return creal(z) * creal(z) + cimag(z) * cimag(z); }

double orc_norm2(const orc_cplx* psi, int n) {
  const int64_t N = (int64_t)1 << n;
  const int64_t nch = (N + ORC_CHUNK - 1) / ORC_CHUNK;
  double* part = (double*)malloc(sizeof(double) * nch);
#pragma omp parallel for schedule(static) if (n >= 17)
  for (int64_t c = 0; c < nch; c++) {
    double s = 0.0;
    int64_t end = (c + 1) * ORC_CHUNK < N ? (c + 1) * ORC_CHUNK : N;
    for (int64_t x = c * ORC_CHUNK; x < end; x++) s += abs2(psi[x]);
    part[c] = s;
  }
  double t = 0.0;
  for (int64_t c = 0; c < nch; c++) t += part[c];
  free(part);
  return t;
}

void orc_kraus_norms(const orc_cplx* psi, int n, int q, const int32_t* qubits,
                     int nk, const orc_cplx* K, double* P) {
  int32_t s[8];
  sorted_copy(q, qubits, s);
  const int M = 1 << q;
  const int64_t sets = (int64_t)1 << (n - q);
  const int64_t nch = (sets + ORC_CHUNK - 1) / ORC_CHUNK;
  double* part = (double*)calloc((size_t)(nch * nk), sizeof(double));
#pragma omp parallel for schedule(static) if (n >= 17)
  for (int64_t c = 0; c < nch; c++) {
    int64_t end = (c + 1) * ORC_CHUNK < sets ? (c + 1) * ORC_CHUNK : sets;
    for (int64_t i = c * ORC_CHUNK; i < end; i++) {
      orc_cplx v[64];
      uint64_t base = insert_zeros((uint64_t)i, q, s);
      for (int k = 0; k < M; k++) v[k] = psi[member(base, k, q, qubits)];
      for (int op = 0; op < nk; op++) {
        const orc_cplx* Ki = K + (int64_t)op * M * M;
        double sq = 0.0;
        for (int j = 0; j < M; j++) {
          orc_cplx acc = 0.0;
          for (int k = 0; k < M; k++) acc += Ki[j * M + k] * v[k];
          sq += abs2(acc);                       /* |(K_i psi)_j|^2 */
        }
        part[c * nk + op] += sq;
      }
    }
  }
  for (int op = 0; op < nk; op++) {
    double t = 0.0;
    for (int64_t c = 0; c < nch; c++) t += part[c * nk + op];
    P[op] = t;
  }
  free(part);
}

/* ------------------------------------------------------------------------ */
/* Lower bound: smallest eigenvalue of the Hermitian K^dag K, found with    */
/* the cyclic Jacobi method on its real symmetric embedding                 */
/* [[Re, -Im], [Im, Re]] (every eigenvalue appears twice).                  */
/* ------------------------------------------------------------------------ */
static double jacobi_min_eig(int m, double* S) {
  for (int sweep = 0; sweep < 200; sweep++) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < m; i++) {
      diag += S[i * m + i] * S[i * m + i];
      for (int j = i + 1; j < m; j++) off += S[i * m + j] * S[i * m + j];
    }
    if (off == 0.0 || off <= 1e-32 * diag) break;
    for (int p = 0; p < m; p++)
      for (int q = p + 1; q < m; q++) {
        double apq = S[p * m + q];
        if (apq == 0.0) continue;
        double theta = (S[q * m + q] - S[p * m + p]) / (2.0 * apq);
        double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < m; k++) {
          double a = S[k * m + p], b = S[k * m + q];
          S[k * m + p] = c * a - s * b;
          S[k * m + q] = s * a + c * b;
        }
        for (int k = 0; k < m; k++) {
          double a = S[p * m + k], b = S[q * m + k];
          S[p * m + k] = c * a - s * b;
          S[q * m + k] = s * a + c * b;
        }
      }
  }
  double mn = S[0];
  for (int i = 1; i < m; i++) mn = S[i * m + i] < mn ? S[i * m + i] : mn;
  return mn;
}

double orc_lower_bound(int q, const orc_cplx* K) {
  const int d = 1 << q, m = 2 * d;
  orc_cplx* A = (orc_cplx*)malloc(sizeof(orc_cplx) * d * d);
  double* S = (double*)malloc(sizeof(double) * m * m);
  for (int i = 0; i < d; i++)                 /* A = K^dag K */
    for (int j = 0; j < d; j++) {
      orc_cplx acc = 0.0;
      for (int k = 0; k < d; k++) acc += conj(K[k * d + i]) * K[k * d + j];
      A[i * d + j] = acc;
    }
  for (int i = 0; i < d; i++)
    for (int j = 0; j < d; j++) {
      double re = creal(A[i * d + j]), im = cimag(A[i * d + j]);
      S[i * m + j] = re;
      S[i * m + (j + d)] = -im;
      S[(i + d) * m + j] = im;
      S[(i + d) * m + (j + d)] = re;
    }
  double lam = jacobi_min_eig(m, S);
  free(A);
  free(S);
  return lam < 0.0 ? 0.0 : lam;   /* K^dag K is positive semidefinite */
}

/* ------------------------------------------------------------------------ */
/* Trajectories (Sec. III.E, Alg. 2)                                        */
/* ------------------------------------------------------------------------ */
/* Kraus operators of op i; for a mixture K_j = sqrt(p_j) U_j (Sec. II). */
static const orc_cplx* op_kraus(const orc_circuit* c, int i, orc_cplx* buf) {
  const orc_cplx* m = c->mats + c->moff[i];
  if (c->kind[i] != ORC_MIXTURE) return m;
  const int64_t dd = (int64_t)1 << (2 * c->nq[i]);
  for (int j = 0; j < c->nmat[i]; j++) {
    double sp = sqrt(c->probs[c->poff[i] + j]);
    for (int64_t e = 0; e < dd; e++) buf[j * dd + e] = sp * m[j * dd + e];
  }
  return buf;
}

static void scale_op(int q, const orc_cplx* K, double f, orc_cplx* out) {
  const int64_t dd = (int64_t)1 << (2 * q);
  for (int64_t e = 0; e < dd; e++) out[e] = f * K[e];
}

static double min_dist(double r, double b, double cur) {
  double d = fabs(r - b);
  return d < cur ? d : cur;
}

int orc_run_trajectory(const orc_circuit* c, int mode, uint64_t seed, uint64_t traj,
                       int64_t max_ops, orc_cplx* psi, int32_t* kraus_idx,
                       int32_t* stage, double* margin) {
  const int n = c->num_qubits;
  const int64_t N = (int64_t)1 << n;
  memset(psi, 0, sizeof(orc_cplx) * N);
  psi[0] = 1.0;                                     /* |0...0> */
  orc_cplx* kbuf = (orc_cplx*)malloc(sizeof(orc_cplx) * 16 * 4096);
  orc_cplx* tmp = (orc_cplx*)malloc(sizeof(orc_cplx) * 4096);
  double lb[64], P[64], d[64];
  int ch = 0, flushes = 0;
  const int64_t nops = (max_ops >= 0 && max_ops < c->num_ops) ? max_ops : c->num_ops;
  for (int64_t i = 0; i < nops; i++) {
    const int q = c->nq[i];
    const int32_t* Q = c->qubits + c->qoff[i];
    if (c->kind[i] == ORC_GATE) {
      orc_apply(psi, n, q, Q, c->mats + c->moff[i]);
      continue;
    }
    const int k = c->nmat[i];
    const int64_t dd = (int64_t)1 << (2 * q);
    const orc_cplx* K = op_kraus(c, (int)i, kbuf);
    for (int j = 0; j < k; j++)
      lb[j] = (c->kind[i] == ORC_MIXTURE) ? c->probs[c->poff[i] + j]
                                          : orc_lower_bound(q, K + j * dd);
    const double r = orc_u01(seed, traj, 0, (uint32_t)ch);
    int chosen = -1, st = 1;
    double mg = INFINITY;

    if (mode == ORC_CUMULATIVE) {
      /* textbook: first i with r < p_1 + ... + p_i */
      double Nrm = orc_norm2(psi, n);
      orc_kraus_norms(psi, n, q, Q, k, K, P);
      double acc = 0.0;
      for (int j = 0; j < k; j++) {
        acc += P[j] / Nrm;
        mg = min_dist(r, acc, mg);
        if (chosen < 0 && r < acc) chosen = j;
      }
      if (chosen < 0)
        for (int j = 0; j < k; j++) if (P[j] > 0.0) chosen = j;
      scale_op(q, K + chosen * dd, 1.0 / sqrt(P[chosen]), tmp);
      orc_apply(psi, n, q, Q, tmp);
      st = 2;
      flushes++;
    } else {
      /* stage 1 (Alg. 2 steps 4-11): partition [0, s) by the lower bounds */
      double rr = r, acc = 0.0;
      for (int j = 0; j < k; j++) {
        acc += lb[j];
        mg = min_dist(r, acc, mg);
      }
      for (int j = 0; j < k; j++) {
        if (rr < lb[j]) { chosen = j; break; }
        rr -= lb[j];
      }
      if (mode == ORC_DELAYED && chosen >= 0) {
        /* deferred: applied now, unnormalized -- the oracle applies every
         * deferred operator in order as it goes */
        orc_apply(psi, n, q, Q, K + chosen * dd);
      } else {
        /* stage 2 (steps 12-21): all earlier operators are applied; evaluate
         * p_i = P_i / <psi|psi> in place */
        double Nrm = orc_norm2(psi, n);
        orc_kraus_norms(psi, n, q, Q, k, K, P);
        double s = acc, acc2 = s;
        for (int j = 0; j < k; j++) {
          d[j] = P[j] / Nrm - lb[j];
          if (d[j] < 0.0) d[j] = 0.0;            /* rounding */
          acc2 += d[j];
          mg = min_dist(r, acc2, mg);
        }
        if (chosen < 0) {
          st = 2;
          for (int j = 0; j < k; j++) {
            if (rr < d[j]) { chosen = j; break; }
            rr -= d[j];
          }
          if (chosen < 0)                        /* rounding past the end */
            for (int j = 0; j < k; j++) if (d[j] > 0.0) chosen = j;
          if (chosen < 0)
            for (int j = 0; j < k; j++) if (P[j] > 0.0) chosen = j;
        }
        scale_op(q, K + chosen * dd, 1.0 / sqrt(P[chosen]), tmp);
        orc_apply(psi, n, q, Q, tmp);            /* (1/sqrt(p_i)) K_i, normalized */
        flushes++;
      }
    }
    if (kraus_idx) kraus_idx[ch] = chosen;
    if (stage) stage[ch] = st;
    if (margin) margin[ch] = mg;
    ch++;
  }
  double Nrm = orc_norm2(psi, n);
  double f = 1.0 / sqrt(Nrm);
#pragma omp parallel for schedule(static) if (n >= 17)
  for (int64_t x = 0; x < N; x++) psi[x] *= f;
  free(kbuf);
  free(tmp);
  return flushes;
}

void orc_run_trajectories(const orc_circuit* c, int mode, uint64_t seed, uint64_t traj0,
                          int T, orc_cplx* psis, int32_t* kraus_idx, int32_t* stage,
                          double* margin, int32_t* flushes) {
  const int n = c->num_qubits;
  const int64_t N = (int64_t)1 << n;
  int nch = 0;
  for (int i = 0; i < c->num_ops; i++) nch += (c->kind[i] != ORC_GATE);
#pragma omp parallel for schedule(dynamic, 1) if (n < 17)
  for (int t = 0; t < T; t++) {
    orc_cplx* psi = psis ? psis + (int64_t)t * N : (orc_cplx*)malloc(sizeof(orc_cplx) * N);
    int f = orc_run_trajectory(c, mode, seed, traj0 + (uint64_t)t, -1, psi,
                               kraus_idx ? kraus_idx + (int64_t)t * nch : NULL,
                               stage ? stage + (int64_t)t * nch : NULL,
                               margin ? margin + (int64_t)t * nch : NULL);
    if (flushes) flushes[t] = f;
    if (!psis) free(psi);
  }
}

/* ------------------------------------------------------------------------ */
/* Measurement                                                              */
/* ------------------------------------------------------------------------ */
static const double* g_sort_key;
static int cmp_idx(const void* a, const void* b) {
  double x = g_sort_key[*(const int*)a], y = g_sort_key[*(const int*)b];
  return (x > y) - (x < y);
}

void orc_sample(const orc_cplx* psi, int n, uint64_t seed, uint64_t traj, int S,
                uint64_t* out, double* margin) {
  const int64_t N = (int64_t)1 << n;
  double total = 0.0;
  for (int64_t x = 0; x < N; x++) total += abs2(psi[x]);   /* C(2^n - 1) */
  double* t = (double*)malloc(sizeof(double) * (S > 0 ? S : 1));
  int* order = (int*)malloc(sizeof(int) * (S > 0 ? S : 1));
  for (int j = 0; j < S; j++) {
    t[j] = orc_u01(seed, traj, 1, (uint32_t)j) * total;
    order[j] = j;
  }
  g_sort_key = t;
  qsort(order, (size_t)S, sizeof(int), cmp_idx);
  int jp = 0;
  int64_t last_nz = 0;
  double C = 0.0;
  for (int64_t x = 0; x < N && jp < S; x++) {
    double Cprev = C;
    double w = abs2(psi[x]);
    C += w;
    if (w > 0.0) last_nz = x;
    while (jp < S && t[order[jp]] < C) {        /* smallest x with target < C(x) */
      int j = order[jp++];
      out[j] = (uint64_t)x;
      if (margin) {
        double a = t[j] - Cprev, b = C - t[j];
        margin[j] = (a < b ? a : b) / total;
      }
    }
  }
  for (; jp < S; jp++) {                        /* target >= C(2^n-1) by rounding */
    int j = order[jp];
    out[j] = (uint64_t)last_nz;
    if (margin) margin[j] = 0.0;
  }
  free(t);
  free(order);
}

/* Readout errors (Sec. V.A): a qubit in |b> is reported as the other value
 * with the error probability measured for b (p00 error for b = 0, p11 error
 * for b = 1).  One draw per qubit per sample, on its own Philox stream. */
void orc_readout(uint64_t* bits, int S, int n, const double* err, uint64_t seed, uint64_t traj) {
  for (int j = 0; j < S; j++) {
    uint64_t x = bits[j];
    for (int q = 0; q < n; q++) {
      const int b = (int)((x >> q) & 1u);
      const double u = orc_u01(seed, traj, 2, ((uint32_t)j << 6) | (uint32_t)q);
      if (u < err[2 * q + b]) x ^= (uint64_t)1 << q;
    }
    bits[j] = x;
  }
}

void orc_expect_z(const orc_cplx* psi, int n, int M, const uint64_t* masks, double* out) {
  const int64_t N = (int64_t)1 << n;
  const int64_t nch = (N + ORC_CHUNK - 1) / ORC_CHUNK;
  double* part = (double*)calloc((size_t)(nch * (M + 1)), sizeof(double));
#pragma omp parallel for schedule(static) if (n >= 17)
  for (int64_t c = 0; c < nch; c++) {
    int64_t end = (c + 1) * ORC_CHUNK < N ? (c + 1) * ORC_CHUNK : N;
    for (int64_t x = c * ORC_CHUNK; x < end; x++) {
      double w = abs2(psi[x]);
      part[c * (M + 1)] += w;
      for (int m = 0; m < M; m++) {
        int odd = __builtin_popcountll((uint64_t)x & masks[m]) & 1;
        part[c * (M + 1) + 1 + m] += odd ? -w : w;
      }
    }
  }
  double tot[65];
  double* T = (M + 1 <= 65) ? tot : (double*)malloc(sizeof(double) * (M + 1));
  for (int m = 0; m <= M; m++) {
    double s = 0.0;
    for (int64_t c = 0; c < nch; c++) s += part[c * (M + 1) + m];
    T[m] = s;
  }
  for (int m = 0; m < M; m++) out[m] = T[1 + m] / T[0];
  if (T != tot) free(T);
  free(part);
}

/* ------------------------------------------------------------------------ */
/* Exact density-matrix evolution (n <= 7).  rho is stored as a 2n-qubit    */
/* vector (row bits 0..n-1, column bits n..2n-1), so rho -> A rho B^dag is  */
/* A applied to the row qubits and conj(B) applied to the column qubits.    */
/* ------------------------------------------------------------------------ */
static void conj_op(int q, const orc_cplx* A, orc_cplx* out) {
  const int64_t dd = (int64_t)1 << (2 * q);
  for (int64_t e = 0; e < dd; e++) out[e] = conj(A[e]);
}

void orc_density_evolve(const orc_circuit* c, orc_cplx* rho) {
  const int n = c->num_qubits;
  const int64_t D2 = (int64_t)1 << (2 * n);
  memset(rho, 0, sizeof(orc_cplx) * D2);
  rho[0] = 1.0;
  orc_cplx* acc = (orc_cplx*)malloc(sizeof(orc_cplx) * D2);
  orc_cplx* t = (orc_cplx*)malloc(sizeof(orc_cplx) * D2);
  orc_cplx* kbuf = (orc_cplx*)malloc(sizeof(orc_cplx) * 16 * 4096);
  orc_cplx* cj = (orc_cplx*)malloc(sizeof(orc_cplx) * 4096);
  for (int i = 0; i < c->num_ops; i++) {
    const int q = c->nq[i];
    const int32_t* Q = c->qubits + c->qoff[i];
    int32_t Qc[8];
    for (int b = 0; b < q; b++) Qc[b] = Q[b] + n;
    const int64_t dd = (int64_t)1 << (2 * q);
    if (c->kind[i] == ORC_GATE) {
      const orc_cplx* U = c->mats + c->moff[i];
      orc_apply(rho, 2 * n, q, Q, U);
      conj_op(q, U, cj);
      orc_apply(rho, 2 * n, q, Qc, cj);
      continue;
    }
    const orc_cplx* K = op_kraus(c, i, kbuf);
    memset(acc, 0, sizeof(orc_cplx) * D2);
    for (int j = 0; j < c->nmat[i]; j++) {
      memcpy(t, rho, sizeof(orc_cplx) * D2);
      orc_apply(t, 2 * n, q, Q, K + j * dd);
      conj_op(q, K + j * dd, cj);
      orc_apply(t, 2 * n, q, Qc, cj);
      for (int64_t e = 0; e < D2; e++) acc[e] += t[e];
    }
    memcpy(rho, acc, sizeof(orc_cplx) * D2);
  }
  free(acc);
  free(t);
  free(kbuf);
  free(cj);
}
