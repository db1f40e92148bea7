/*
 * qt.h -- C ABI of the GB300 (sm_103a) quantum-trajectory library.
 *
 * Method: "Simulations of Quantum Circuits with Approximate Noise using qsim
 * and Cirq" (arXiv 2111.02396).  A noisy circuit (gates and noise channels,
 * Sec. II) is simulated by quantum trajectories (Sec. III.E): one Kraus
 * operator is sampled per channel and applied to a 2^n-amplitude complex64
 * state vector; gates are fused (Sec. III.B) and applied as 2^q x 2^q
 * matrix-vector products over the state (Alg. 1); branch probabilities are
 * evaluated only when the lower bounds do not decide (delayed inner products,
 * Alg. 2).
 *
 * Conventions
 *   - amplitude index bit j is qubit j; an operator on qubits Q[0..q-1] is a
 *     2^q x 2^q row-major matrix whose index bit b is qubit Q[b];
 *   - matrices cross the ABI as interleaved (re, im) FP64;
 *   - every trajectory starts in |0...0>;
 *   - random numbers: Philox4x32-10 (Salmon et al., SC'11), key = seed,
 *     counter = (traj_lo, traj_hi, stream, index); stream 0 index c draws
 *     the uniform of channel c (circuit order), stream 1 index j draws the
 *     uniform of sample j; u01 = ((w0 >> 5) * 2^26 + (w1 >> 6)) * 2^-53.
 *
 * Errors: every call returns a qt_status; 0 is success, negative values are
 * errors and leave outputs unspecified.  No call aborts the process.  The
 * message of the last error on the calling thread is qt_last_error().
 *
 * Ownership: handles (qt_circuit, qt_fused, qt_run, qt_server) are owned by
 * the library and freed by their *_destroy call; arrays passed in are read
 * during the call only (copied where kept); output arrays are owned by the
 * caller and sized as each call states.  Device memory comes from the
 * allocator installed with qt_set_allocator (stream-ordered cudaMallocAsync
 * by default).  qt_circuit and qt_fused handles are immutable after
 * creation and may be shared between threads; a qt_run is used by one
 * thread at a time.
 */
#ifndef QT_H
#define QT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QT_OK = 0,
  QT_ERR_INVALID_ARG = -1,   /* malformed input (range, moment overlap, sizes) */
  QT_ERR_NOT_CPTP = -2,      /* Kraus list with sum K^dag K != I (tolerance 1e-10) */
  QT_ERR_OUT_OF_MEMORY = -3, /* allocator or budget refused */
  QT_ERR_CUDA = -4,          /* CUDA runtime error (message names the call) */
  QT_ERR_TIMEOUT = -5,       /* a bounded device wait ran out */
  QT_ERR_UNSUPPORTED = -6,   /* valid request outside the library's limits */
  QT_ERR_INTERNAL = -7       /* device-side consistency check failed */
} qt_status;

typedef enum { QT_OP_GATE = 0, QT_OP_KRAUS = 1, QT_OP_MIXTURE = 2 } qt_op_kind;
typedef enum { QT_DELAYED = 0, QT_EAGER = 1 } qt_mode;
typedef enum { QT_FP32 = 0, QT_TF32X3 = 1 } qt_precision;
#define QT_FLAG_TIME_KERNELS 1u
#define QT_FLAG_MULTI_GATE 2u    /* group fused gates into multi-gate passes (opt-in) */
#define QT_FLAG_SHARE_PREFIX 4u  /* share the default-choice prefix between trajectories (opt-in) */

#define QT_MAX_QUBITS 34      /* largest state: 2^34 complex64 = 128 GiB */
#define QT_MAX_OP_QUBITS 6    /* widest gate or channel */
#define QT_MAX_FUSED_QUBITS 6 /* widest fused gate */

/* One operation of a moment (Sec. II): a gate, a Kraus channel
 * (KrausChannel) or a mixed-unitary channel (MixedUnitaryChannel). */
typedef struct {
  int32_t kind;            /* qt_op_kind */
  uint32_t moment;         /* ops of one moment act on disjoint qubits */
  uint32_t num_qubits;     /* 1..QT_MAX_OP_QUBITS */
  uint32_t qubits[QT_MAX_OP_QUBITS];
  uint32_t num_ops;        /* 1 for a gate; Kraus operators / mixture terms */
  const double* probs;     /* MIXTURE: num_ops probabilities summing to 1 (+-1e-12) */
  const double* mats;      /* num_ops matrices, 2^q x 2^q, row-major, (re,im) FP64 */
} qt_op;

typedef struct qt_circuit qt_circuit;
typedef struct qt_fused qt_fused;
typedef struct qt_run qt_run;
typedef struct qt_server qt_server;

/* Build and validate a noisy circuit (Sec. II; channel terms Sec. III.E).
 * Checks qubit ranges, disjointness within each moment, sum K^dag K = I for
 * Kraus channels (1e-10) and sum p = 1 for mixtures (1e-12, then
 * renormalized).  Computes the lower bounds pbar_i = sigma_min(K_i)^2 of
 * Sec. III.E (mixtures: pbar_i = p_i, so s = 1).  All input arrays are
 * copied.  Errors: QT_ERR_INVALID_ARG, QT_ERR_NOT_CPTP. */
qt_status qt_circuit_create(uint32_t num_qubits, uint32_t num_ops, const qt_op* ops,
                            qt_circuit** out);

/* Gate fusion (Sec. III.B): greedily merge operations that are close in
 * space and time into fused gates of at most max_fused_qubits qubits
 * (1..6; 0 = automatic choice).  Channels become slots of the fused gates;
 * the matrix of each fused gate with every slot on its most likely
 * (largest pbar) operator is precomputed.  The circuit must outlive the
 * fused handle.  Errors: QT_ERR_INVALID_ARG. */
qt_status qt_fuse(const qt_circuit* c, uint32_t max_fused_qubits, qt_fused** out);

/* Parameters of a trajectory run. */
typedef struct {
  uint64_t seed;               /* Philox key */
  uint64_t first_traj;         /* trajectory ids first_traj .. first_traj+num_traj-1 */
  uint32_t num_traj;
  uint32_t mode;               /* QT_DELAYED (Alg. 2) or QT_EAGER (conventional) */
  uint32_t precision;          /* QT_FP32, or QT_TF32X3 for 5-6 qubit fused gates */
  uint32_t samples_per_traj;   /* bitstrings drawn from each final state */
  uint32_t num_z_masks;        /* Z-string expectations on each final state */
  const uint64_t* z_masks;     /* num_z_masks masks (copied) */
  uint32_t keep_states;        /* 1: keep every final state on the device */
  uint32_t flags;              /* QT_FLAG_TIME_KERNELS: time each fused-gate pass;
                                  QT_FLAG_MULTI_GATE: several fused gates per pass;
                                  QT_FLAG_SHARE_PREFIX: delayed mode only -- stage 1 fixes, before
                                  any kernel runs, each trajectory's first channel whose draw
                                  leaves the default operator; the operators before it are the
                                  same for every trajectory, so one shared state advances along
                                  that default path and each trajectory copies it at its own
                                  point (16 * 2^n bytes) and runs only the rest.  Same draws,
                                  branch records and samples; states equal up to FP32 rounding
                                  (fused pieces are split at the copy points).  Needs one more
                                  state buffer. */
  void* stream;                /* cudaStream_t (0 = legacy default stream) */
  uint64_t timeout_ns;         /* bound on any device wait (0 = 10 s) */
  const double* readout_error; /* NULL, or readout errors of the samples (Sec. V.A, parallel
                                  readout errors), 2 per qubit, copied: qubit q of true value b is
                                  reported as 1 - b with probability readout_error[2q + b]
                                  (the p00 error for b = 0, the p11 error for b = 1), decided
                                  by u01(seed, traj, 2, (j << 6) | q) < readout_error[2q + b]
                                  for sample j; needs samples_per_traj < 2^26 */
} qt_run_params;

/* Run num_traj trajectories of Alg. 2 (QT_DELAYED) or of the conventional
 * algorithm (QT_EAGER, every channel evaluated immediately; branch choice
 * from the same two-stage partition of [0,1)).  Per channel c the draw is
 * r = u01(seed, traj, stream 0, index c); stage 1 picks the first i with
 * r < pbar_i after subtracting the earlier pbar's and defers K_i; otherwise
 * the deferred operators are applied, N = <psi|psi> and
 * P_i = <psi|K_i^dag K_i|psi> are evaluated in one in-place pass, and
 * K_i / sqrt(P_i) is applied for the first i with r < P_i/N - pbar_i.
 * Requested samples and expectations are evaluated on each final state.
 * Blocks until the results are on the host.  Errors: QT_ERR_INVALID_ARG,
 * QT_ERR_OUT_OF_MEMORY, QT_ERR_CUDA, QT_ERR_UNSUPPORTED. */
qt_status qt_run_trajectories(const qt_fused* f, const qt_run_params* p, qt_run** out);

/* Bitstrings of the run (Sec. V.C: after each computation every qubit is
 * measured, and the measured bitstrings are compared with the device's;
 * Sec. II: measurement results of a Cirq circuit).  Each final state is
 * measured in the computational basis, i.e. x is drawn with probability
 * |psi_x|^2 / <psi|psi>: out[t * S + j] is sample j of trajectory t, bit k
 * = qubit k; the smallest x with u_j * C(2^n - 1) < C(x), C the cumulative
 * sum of |psi_x|^2 in index order (FP64), u_j = u01(seed, traj, 1, j).
 * S must equal the run's samples_per_traj, or, if the run kept its states,
 * any S (drawn now).  out holds num_traj * S entries. */
qt_status qt_sample(qt_run* r, uint32_t samples_per_traj, uint64_t* out);

/* Z-string expectations <psi| Z^{mask} |psi> / <psi|psi> of each final
 * state: out[t * num_terms + m].  These are the observables of Sec. V.C: the
 * site densities P(q_j = 1) = (1 - <Z_j>) / 2 of the Fermi-Hubbard and
 * non-interacting-fermion comparisons, and the Z-basis cost <C> of QAOA (a
 * sum of Z-strings); averaged over r trajectories their Monte Carlo error
 * falls as 1/sqrt(r) (Sec. III.E).  The masks must equal the run's z_masks,
 * or, if the run kept its states, be any masks (evaluated now). */
qt_status qt_expectation(qt_run* r, uint32_t num_terms, const uint64_t* z_masks,
                         double* out);

/* Per-trajectory records of a run (Sec. II "measurement key": the index of
 * the selected Kraus operator).  kraus: num_traj * num_channels int32
 * (channel order = circuit order); stage: same shape, 1 = decided by the
 * lower bounds, 2 = decided by evaluated probabilities; cap = entries
 * available in each array (either may be NULL). */
qt_status qt_run_kraus_indices(const qt_run* r, int32_t* kraus, int32_t* stage, size_t cap);

/* Statistics of a run. */
typedef struct {
  uint32_t num_traj, num_channels;
  uint64_t fused_passes;      /* fused-gate kernel launches (state passes) */
  uint64_t prob_passes;       /* probability-evaluation passes (Alg. 2 step 14) */
  uint64_t gate_ops;          /* unfused gates applied (gate-equivalents) */
  uint64_t flushes;           /* channels decided in stage 2 */
  double device_ms;           /* device time of the trajectory loop (events) */
  double apply_ms;            /* device time inside fused-gate kernels
                                 (QT_FLAG_TIME_KERNELS, else 0) */
  uint64_t apply_bytes;       /* algorithmic bytes of those kernels: 16 per
                                 amplitude per pass (read + write, complex64) */
  uint64_t h2d_bytes;         /* host->device bytes (copies + matrix parameters) */
  uint64_t d2h_bytes;         /* device->host bytes */
  uint64_t kernel_launches;   /* kernels of this library launched by the run */
  uint64_t fused_pieces;      /* fused gates (or segment pieces of them) applied; several
                                 share one pass when a multi-gate pass groups them */
  uint64_t passes_by_width[8];  /* fused-gate passes by gate width 1..7; [0] = multi-gate passes */
  double apply_ms_by_width[8];  /* their device time (QT_FLAG_TIME_KERNELS, else 0) */
  uint64_t folded_pieces;     /* leading fused gates folded into the initial product state
                                 (each the first on its qubits; one write pass makes
                                 U[:, 0] of all of them, for n >= 12); not in fused_passes */
  uint32_t fold_split;        /* qubit split m of the last product-state start (tables of
                                 2^m and 2^(n-m) entries, each at most 2^20), 0 if none */
  uint32_t pad;
  uint64_t prefix_copies;     /* QT_FLAG_SHARE_PREFIX: copies of the shared state */
  uint64_t prefix_ops;        /* QT_FLAG_SHARE_PREFIX: operations the trajectories took from the
                                 shared state (summed over trajectories) */
  uint64_t merged_pieces;     /* segment pieces merged into a later piece on the same qubits
                                 (at most the fusion width together); not in fused_passes */
} qt_run_stats_t;
qt_status qt_run_stats(const qt_run* r, qt_run_stats_t* out);

/* <psi|psi> of every final state before normalization (num_traj doubles):
 * 1 for unitary circuits up to rounding, so |N - 1| is the norm drift of
 * the arithmetic. */
qt_status qt_run_norms(const qt_run* r, double* out);

/* Normalized final state of trajectory `traj` (index within the run) as
 * complex64 (re, im float pairs); needs keep_states; dst is host memory of
 * bytes >= 8 * 2^n. */
qt_status qt_run_state(const qt_run* r, uint32_t traj, void* dst, size_t bytes);

/* Device allocator (e.g. a framework's caching allocator).  alloc returns
 * device memory of at least `bytes` usable on `stream`, or NULL; free
 * releases it.  Passing NULLs restores the default (cudaMallocAsync). */
typedef void* (*qt_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*qt_free_fn)(void* ptr, size_t bytes, void* stream, void* ctx);
qt_status qt_set_allocator(qt_alloc_fn alloc, qt_free_fn free_fn, void* ctx);

void qt_circuit_destroy(qt_circuit* c);
void qt_fused_destroy(qt_fused* f);
void qt_run_destroy(qt_run* r);
const char* qt_last_error(void);

/* Architecture the library's kernels were compiled for, as the CUDA runtime
 * reports it for the current device (cudaFuncGetAttributes): binary_version
 * 103 is sm_103a code (GB300); ptx_version 0 when no PTX is embedded. */
qt_status qt_kernel_arch(int32_t* binary_version, int32_t* ptx_version);

/* Introspection of the fused plan (host only, no GPU needed). */
typedef struct {
  uint32_t num_fused, max_width, num_ops, num_channels;
} qt_fused_info_t;
qt_status qt_fused_info(const qt_fused* f, qt_fused_info_t* out);
/* Fused gate g: its target qubits (sorted, <= 6), the op indices it contains
 * (circuit order positions, members[] of length cap) and its default matrix
 * (2^w x 2^w row-major (re,im) FP64, NULL to skip). */
qt_status qt_fused_gate(const qt_fused* f, uint32_t g, uint32_t* width, uint32_t* targets,
                        uint32_t* num_members, uint32_t* members, size_t cap, double* matrix);
/* Lower bounds pbar_i of channel c (circuit order), cap entries. */
qt_status qt_channel_lower_bounds(const qt_circuit* c, uint32_t channel, double* pbar,
                                  size_t cap, uint32_t* num_ops);

/* ---------------------------------------------------------------------- */
/* State-level calls: the hot kernels on a caller-owned device state      */
/* (complex64, 2^n amplitudes, 16-byte aligned).                           */
/* ---------------------------------------------------------------------- */

/* Alg. 1: state <- U on qubits[0..q-1] (q <= 6); U host FP64 (re,im). */
qt_status qt_state_apply(void* state, uint32_t n, uint32_t q, const uint32_t* qubits,
                         const double* U, uint32_t precision, void* stream);
/* Reduced density block of qubits Q (q <= 3): rho[b][a] = sum_rest
 * psi[rest,b] conj(psi[rest,a]), FP64 accumulation; out host (re,im) FP64
 * 4^q complex, row-major.  P_i = tr(K_i^dag K_i rho) (Alg. 2 step 14). */
qt_status qt_state_reduced_density(const void* state, uint32_t n, uint32_t q,
                                   const uint32_t* qubits, double* out, void* stream);
/* Branch probabilities of a Kraus channel on a caller-owned state (Alg. 2
 * step 14): P_i = <psi|K_i^dag K_i|psi> for the num_ops (<= 64) operators of
 * a channel on qubits[0..q-1] (q <= 6; ops host, num_ops matrices 2^q x 2^q
 * row-major (re, im) FP64, basis bit b <-> qubits[b]) and N = <psi|psi>;
 * P and N host.  q <= 3 goes through the reduced density block; q = 4..6
 * evaluates |K_i psi|^2 per operator on the device (FP32 products, FP64
 * carry, fixed reduction order), 16, 4 or 1 operators per pass. */
qt_status qt_state_kraus_probabilities(const void* state, uint32_t n, uint32_t q, const uint32_t* qubits,
                                       uint32_t num_ops, const double* ops, double* P, double* N, void* stream);
/* Measurement of every qubit (Sec. V.C) on a caller-owned state: S
 * bitstrings x drawn with probability |psi_x|^2 / <psi|psi> (the cumulative
 * rule of qt_sample) with uniforms u01(seed, traj, 1, j); out host, S
 * entries.  readout_error: NULL, or 2 per qubit as in qt_run_params (the
 * parallel readout errors of Sec. V.A; host, copied). */
qt_status qt_state_sample(const void* state, uint32_t n, uint64_t seed, uint64_t traj,
                          uint32_t S, uint64_t* out, const double* readout_error, void* stream);
/* The cumulative distribution C(x) = sum_{y <= x} |psi_y|^2 that the
 * measurement of Sec. V.C samples from (qt_state_sample, qt_sample), as the
 * sampler itself forms it: FP32 squares and FP32 running sums inside runs of
 * 1024 amplitudes, FP64 across runs.  out host, 2^n doubles (out[2^n - 1] is
 * the total); n <= 28.  A sample x is the smallest x with u * C(2^n - 1) <
 * C(x), so these values bound where a sample can land when u falls within
 * rounding of a boundary. */
qt_status qt_state_cdf(const void* state, uint32_t n, double* out, void* stream);
/* Z-string expectations <psi| Z^{mask} |psi> / <psi|psi> of a caller-owned
 * state (the Sec. V.C observables: site densities (1 - <Z_j>) / 2, QAOA
 * Z-string costs); out host, num_terms doubles. */
qt_status qt_state_expect_z(const void* state, uint32_t n, uint32_t num_terms,
                            const uint64_t* z_masks, double* out, void* stream);

/* ---------------------------------------------------------------------- */
/* Batched form: many small trajectories in one persistent launch          */
/* ---------------------------------------------------------------------- */
typedef struct qt_batch qt_batch;

/* Gate fusion (Sec. III.B) of many circuits on host threads (0 = one per
 * core); out[i] receives the fused handle of circuits[i]. */
qt_status qt_fuse_many(uint32_t num, const qt_circuit* const* circuits, uint32_t max_fused_qubits,
                       uint32_t threads, qt_fused** out);

/* Pack num fused circuits (1..20 qubits, ops on <= 2 qubits, fused width
 * <= 6) into device tables for the batched kernel; trajectory i of the batch
 * runs fused[i].  Distinct operator sets are stored once.  The fused handles
 * may be destroyed afterwards.  Errors: QT_ERR_INVALID_ARG,
 * QT_ERR_UNSUPPORTED, QT_ERR_OUT_OF_MEMORY, QT_ERR_CUDA. */
qt_status qt_batch_create(uint32_t num, const qt_fused* const* fused, qt_batch** out);

typedef struct {
  uint64_t seed;               /* Philox key */
  uint64_t first_traj;         /* trajectory i of the batch uses id first_traj + i */
  uint32_t samples_per_traj;   /* bitstrings per final state */
  uint32_t keep_states;        /* 1: keep final states for qt_batch_state */
  uint32_t use_graph;          /* replay the launch sequence as a CUDA graph (needs a stream) */
  uint32_t threads;            /* CTA size of trajectories whose states fit in shared memory
                                  (n <= 14): 128, 256 or 512 (0 = 512) */
  void* stream;                /* cudaStream_t */
  uint32_t threads_global;     /* CTA size of trajectories whose states live in global memory
                                  (n > 14): 128, 256 or 512 (0 = threads) */
} qt_batch_params;

/* Run one trajectory of every circuit of the batch (Alg. 2, the same draws
 * and decisions as qt_run_trajectories with the same seed and trajectory id)
 * in one persistent kernel; blocks until the results are on the host. */
qt_status qt_batch_run(qt_batch* b, const qt_batch_params* p);
/* Samples of the last run: out[i * S + j], cap entries available. */
qt_status qt_batch_samples(const qt_batch* b, uint64_t* out, size_t cap);
/* Branch records of trajectory i of the last run (as qt_run_kraus_indices). */
qt_status qt_batch_kraus_indices(const qt_batch* b, uint32_t i, int32_t* kraus, int32_t* stage, size_t cap,
                                 uint32_t* num_channels);
/* Normalized final state of trajectory i (needs keep_states), complex64 on the host. */
qt_status qt_batch_state(const qt_batch* b, uint32_t i, void* dst, size_t bytes);
typedef struct {
  uint32_t num_traj, num_channels;
  uint64_t total_amps, fused_gates, gate_ops, flushes;
  double device_ms;            /* device time of the last run (events) */
  uint64_t folded_pieces;      /* pieces folded into the product-state start (last run) */
} qt_batch_stats_t;
qt_status qt_batch_stats(const qt_batch* b, qt_batch_stats_t* out);
void qt_batch_destroy(qt_batch* b);
/* Autotuner of the batched form.  The batched kernel runs two classes of
 * trajectories: states of <= 2^14 amplitudes held in a CTA's shared memory,
 * and larger states streamed from a per-CTA slot of global memory.  Their
 * costs differ (the first is bound by latency and arithmetic, the second by
 * memory traffic), so each class is tuned on its own spread sample of at
 * most `sample` circuits (0 = 256): every fusion width kmin..kmax (<= 6) at
 * 128, 256 and 512 threads per CTA (warm-up + 2 timed runs).  best receives
 * the fastest width and CTA size of each class (a class absent from the
 * batch keeps kmin and 512); table (optional, 2 * (kmax - kmin + 1) * 3
 * doubles) the mean ms per run, [(class * (kmax - kmin + 1) + k - kmin) * 3
 * + {128, 256, 512}], class 0 = shared memory, 1 = global memory. */
typedef struct {
  uint32_t k_shared, threads_shared;   /* n <= 14 */
  uint32_t k_global, threads_global;   /* n > 14 */
} qt_batch_tuning;
qt_status qt_batch_autotune(uint32_t num, const qt_circuit* const* circuits, uint32_t sample, uint32_t kmin,
                            uint32_t kmax, void* stream, qt_batch_tuning* best, double* table);

/* ---------------------------------------------------------------------- */
/* Serving form: a request loop with continuous batching                  */
/* ---------------------------------------------------------------------- */
typedef struct {
  uint64_t budget_bytes;       /* device-memory budget for resident states */
  uint32_t max_slots;          /* concurrent plain-loop requests (one stream each), 1..64 */
  uint32_t small_n_max;        /* the batch lane takes requests of n <= 14, and of n <= this
                                  (<= 20) when a request has >= 64 trajectories; 0: no lane */
  uint32_t flags;              /* QT_SERVER_DRY_RUN: no GPU work (scheduling only);
                                  QT_SERVER_NO_SHARED_PREFIX: plain workers run every
                                  trajectory on its own (the per-trajectory loop) */
} qt_server_config;
#define QT_SERVER_DRY_RUN 1u
#define QT_SERVER_NO_SHARED_PREFIX 2u

typedef struct {
  uint64_t seed;               /* Philox key */
  uint64_t first_traj;         /* trajectory ids first_traj .. first_traj + num_traj - 1 */
  uint32_t num_traj;
  uint32_t samples_per_traj;
} qt_server_request;

typedef struct {
  int32_t state;               /* 0 queued, 1 running, 2 done, 3 failed, 4 cancelled */
  int32_t status;              /* qt_status of a finished request */
  uint32_t attempts;           /* > 1 after a deferral or a requeue */
  int32_t worker;
  uint32_t batched;            /* ran in the batched form */
  uint32_t num_traj, samples_per_traj, pad;
  uint64_t bytes;              /* admitted footprint */
  uint64_t flushes;            /* stage-2 channels over its trajectories */
  double queued_s;             /* submit -> first start */
  double latency_s;            /* submit -> done (-1 while active) */
} qt_server_req_info;

typedef struct {
  uint64_t budget, inflight_bytes, peak_inflight_bytes;   /* in-flight bytes include the lane's */
  uint32_t queued, running, done, failed, workers_alive, requeued, deferred, pad;
  uint64_t lane_bytes;         /* reserved for the batch lane's global-memory state slots */
  uint64_t lane_launches;      /* merged launches of the batch lane */
  uint64_t lane_trajectories;  /* trajectories they ran */
} qt_server_stats_t;

enum { QT_FAULT_WORKER_EXIT = 1, QT_FAULT_ALLOC = 2 };

/* Start the server on the current device: max_slots plain-loop workers,
 * each with its own CUDA stream, and (small_n_max > 0) a batch lane with a
 * stream of its own.
 *   - Batch lane: small requests (see small_n_max; ops on <= 2 qubits) wait in
 *     their own queue; whenever the lane is free it takes all of them at once
 *     and runs their trajectories -- each with its own circuit, seed and
 *     trajectory id -- in one merged launch of the batched kernel (the
 *     trajectories-as-independent-jobs workload of Sec. IV); requests arriving
 *     meanwhile join the next launch.  Its global-memory state slots (one per
 *     SM, 8 * 2^small_n_max bytes each, for n > 14) are reserved against the
 *     budget at creation (the lane keeps to n <= 14 if they would take more
 *     than half the budget).
 *   - Plain workers: the other requests are admitted in arrival order as soon
 *     as a worker is free and the footprint of the requests in flight plus
 *     its own fits budget_bytes: 8 * 2^n bytes per resident state (Sec. IV.A),
 *     two states when the request has more than one trajectory (they share
 *     the default-choice prefix, QT_FLAG_SHARE_PREFIX, unless the server was
 *     created with QT_SERVER_NO_SHARED_PREFIX), plus scratch.
 * A request's results depend only on its own circuit, seed and trajectory
 * ids, so they are the same alone and in any mix. */
qt_status qt_server_create(const qt_server_config* cfg, qt_server** out);
/* Queue a request; the fused circuit must outlive it.  A request whose
 * footprint alone exceeds the budget is refused (QT_ERR_OUT_OF_MEMORY). */
qt_status qt_server_submit(qt_server* s, const qt_fused* f, const qt_server_request* r, uint64_t* id);
qt_status qt_server_poll(qt_server* s, uint64_t id, int32_t* state);
/* Block until the request is finished (timeout_ns 0 = no limit). */
qt_status qt_server_wait(qt_server* s, uint64_t id, uint64_t timeout_ns);
/* Cancel a request that has not started. */
qt_status qt_server_cancel(qt_server* s, uint64_t id);
/* Samples (num_traj * samples_per_traj, trajectory-major) and info of a
 * request; samples may be NULL to read the info only. */
qt_status qt_server_result(qt_server* s, uint64_t id, uint64_t* samples, size_t cap, qt_server_req_info* info);
/* Forget a finished request. */
qt_status qt_server_release(qt_server* s, uint64_t id);
qt_status qt_server_stats(qt_server* s, qt_server_stats_t* out);
/* Host-side fault injection: the next `count` dequeues (by a worker or the
 * lane) kill their thread (QT_FAULT_WORKER_EXIT; the watchdog requeues the
 * request -- every request of the lane's launch -- and starts a replacement)
 * or fail with an allocation error (QT_FAULT_ALLOC; the requests are deferred
 * and retried). */
qt_status qt_server_inject(qt_server* s, uint32_t fault, uint32_t count);
/* Finish running requests, stop the workers and free the server. */
void qt_server_destroy(qt_server* s);

/* Allocation-free variant of qt_state_reduced_density (no counterpart in the
 * paper: it exists for callers that cannot let a library allocate device
 * memory -- e.g. an application that reserves all GPU memory for its own pool
 * at start-up, or a latency-critical loop that must not stall on cudaMalloc /
 * cudaFree).  Same arguments, result and precision as
 * qt_state_reduced_density; it calls no allocator of any kind.  Its FP64
 * scratch is one fixed array inside libqt.so: 1216 * 64 + 64 doubles
 * (608.5 KiB), which every GPU that loads the library holds until the process
 * exits; q must be <= 3 (larger requests are rejected with
 * QT_ERR_UNSUPPORTED and a message naming the limit).  Every call looks up
 * that array's device address in the current context (so a device reset does
 * not leave a stale address behind); the first call on a device may load the
 * library's module there, so make that first call before any stream
 * capture.  All calls share the array and it keeps the last call's contents
 * (nothing in it needs to start at zero), so calls whose kernels overlap on
 * the GPU -- different streams or host threads -- race: order them. */
qt_status qt_state_reduced_density_noalloc(const void* state, uint32_t n, uint32_t q,
                                           const uint32_t* qubits, double* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* QT_H */
