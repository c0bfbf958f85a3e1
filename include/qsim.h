/*
 * qsim.h -- C ABI of the GB300 quantum-circuit hot path.
 *
 * What it computes (the thesis "Supercomputer simulations of transmon quantum
 * computers", D. Willsch, 2020):
 *   - an n-qubit state vector of 2^n complex amplitudes a_J
 *     (Eq. (multiqubitstate), section "Multiple qubits");
 *   - circuits as ordered products of one- and two-qubit gates
 *     (section "Quantum circuits": time runs left to right, so the matrices
 *     multiply in reversed order), gates from Tab. (elementarygateset) plus
 *     the rotations of Eqs. (singlequbitrotationx)-(singlequbitrotationz),
 *     CNOT of Eq. (cnotgate), CZ = diag(1,1,1,-1), controlled phase, SWAP
 *     and explicit 2x2 / 4x4 matrices;
 *   - outcome probabilities p_J = |a_J|^2 (Born rule);
 *   - batches of small density matrices evolved by gates and noise channels
 *     written as Pauli transfer matrices (Eq. (paulitransfermatrix)), with
 *     probabilities p_J = <<E_J|G|rho>> (Eq. (GSTBornRuleVectorized)), the
 *     multinomial log-likelihood and its gradient.
 *
 * Conventions
 *   - A qubit is named by its BIT POSITION b in the amplitude index J
 *     (b = 0 is the least significant bit).  The thesis's qubit i (i-th tensor
 *     factor, j_0 most significant) is bit n-1-i.
 *   - Gate matrices act as U[out][in].  For a two-qubit gate q[0] is the most
 *     significant bit of the gate's local index (the control of CNOT/CZ/CP),
 *     matching the 4x4 CNOT layout of Eq. (cnotgate).
 *   - Amplitudes are stored interleaved (re, im); complex64 = 2 x float,
 *     complex128 = 2 x double.
 *   - Every call is asynchronous on the state's CUDA stream unless it returns
 *     a value through a HOST pointer (then it synchronises that stream).
 *
 * Errors: every entry point returns a qs_status and never throws.  On an error
 * the state is left unchanged (QS_EINVAL, QS_ENOMEM are detected before any
 * kernel is launched); qs_last_error() returns a thread-local message.
 * Ownership: a qs_state_t owns its device memory (obtained from the caller's
 * allocator, or cudaMalloc when none is given) until sv_destroy.  Output
 * buffers are always caller-owned.
 */
#ifndef QSIM_H
#define QSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QS_OK = 0,
  QS_EINVAL = 1,        /* invalid argument: bad qubit, duplicate qubits, n out of range, NaN angle */
  QS_ENOMEM = 2,        /* device allocation failed; nothing was changed */
  QS_ECUDA = 3,         /* a CUDA runtime call failed (message has the CUDA error string) */
  QS_ETIMEOUT = 4,      /* a bounded device-side wait gave up (status word set by a kernel) */
  QS_EUNSUPPORTED = 5   /* valid request this build does not implement */
} qs_status;

typedef enum { QS_C64 = 0, QS_C128 = 1 } qs_prec;

/* Gate kinds.  One-qubit kinds use q[0] only. */
typedef enum {
  QS_I = 0, QS_X = 1, QS_Y = 2, QS_Z = 3, QS_H = 4, QS_S = 5, QS_SDG = 6, QS_T = 7, QS_TDG = 8,
  QS_PX = 9,   /* +X = R^x(-pi/2) */
  QS_MX = 10,  /* -X = R^x(+pi/2) */
  QS_PY = 11,  /* +Y = R^y(-pi/2) */
  QS_MY = 12,  /* -Y = R^y(+pi/2) */
  QS_RX = 13, QS_RY = 14, QS_RZ = 15,     /* param[0] = theta, Eqs. (singlequbitrotationx-z) */
  QS_U1 = 16,                             /* param[0] = lambda */
  QS_U2 = 17,                             /* param = (phi, lambda) */
  QS_U3 = 18,                             /* param = (theta, phi, lambda) */
  QS_RK = 19,                             /* param[0] = k, R(k) = U1(2 pi / 2^k) */
  QS_MAT1 = 20,                           /* explicit 2x2 in m[0..7] */
  QS_CNOT = 32,                           /* q[0] control, q[1] target */
  QS_CZ = 33,
  QS_CP = 34,                             /* diag(1,1,1,e^{i param[0]}) */
  QS_SWAP = 35,
  QS_MAT2 = 36                            /* explicit 4x4 in m[0..31] */
} qs_gate_kind;

/* One gate (296 bytes, 8-byte aligned).  m: explicit matrix, complex128
 * row-major U[out][in], (re, im) interleaved; only read for QS_MAT1/QS_MAT2. */
typedef struct {
  int32_t kind;
  int32_t q[2];
  int32_t reserved;
  double param[3];
  double m[32];
} qs_gate;

/* Device allocator supplied by the caller (e.g. PyTorch's caching allocator).
 * alloc returns NULL on failure.  stream is the state's cudaStream_t. */
typedef struct {
  void* (*alloc)(size_t bytes, void* stream, void* ctx);
  void (*free)(void* ptr, size_t bytes, void* stream, void* ctx);
  void* ctx;
} qs_allocator;

typedef struct qs_state_s* qs_state_t;

typedef enum {
  QS_METHOD_TILED = 0,       /* fused shared-memory tile passes */
  QS_METHOD_PLAIN = 1,       /* one kernel launch per gate (comparison baseline) */
  /* gates fused into dense 5-qubit blocks (32x32 unitaries, products of the
   * circuit's gates), each applied as a real [2^(n-5) x 64] x [64 x 64] GEMM
   * on the tensor cores (tcgen05) in split precision: each operand is the sum
   * of its parts, the products of the parts whose order of magnitude matters
   * are accumulated in FP32, and for a unitary block every 32-amplitude row is
   * rescaled to its input norm.  complex64 states with n >= 12 only
   * (QS_EUNSUPPORTED otherwise); synchronous (the call checks the kernels'
   * bounded-wait status word). */
  QS_METHOD_BLOCKS_TF32 = 2, /* two TF32 parts, 4 products (~1e-6 relative over 100 blocks) */
  QS_METHOD_BLOCKS_BF16 = 3, /* three BF16 parts, 6 products (~6e-7 relative over 100 blocks) */
  /* the default (also when opts is NULL): for complex64 states with n >= 12
   * the circuit is cut into 5-qubit blocks; a block with more than half of its
   * 1024 entries nonzero is a dense contraction and runs as a BF16-split GEMM on
   * the tensor cores, and each maximal run of sparser blocks (diagonal or nearly
   * diagonal stretches, permutations) is replayed gate by gate through the tile
   * passes.  With only one or two dense blocks, the whole circuit runs on tile
   * passes when that takes no more tile passes and remaps than the sparse runs
   * alone (the blocks' sweeps are saved).  Other states use QS_METHOD_TILED.
   * Synchronous like the block methods. */
  QS_METHOD_AUTO = 4
} qs_method;

typedef struct {
  int32_t method;       /* qs_method */
  int32_t flags;        /* QS_OPT_* */
  int32_t reserved[6];
} qs_opts;

/* Record CUDA events around every launch of the call (on the state's stream)
 * and report per-kind device times in qs_stats.kernel_ms; makes the call
 * synchronous. */
#define QS_OPT_TIME_KERNELS 1

/* Per-call statistics (filled when a non-NULL pointer is given). */
typedef struct {
  int64_t gates_in;        /* gates given */
  int64_t ops_fused;       /* device ops after fusion / folding */
  int64_t passes;          /* full-state read+write sweeps */
  int64_t launches;        /* kernel launches */
  double bytes_moved;      /* algorithmic bytes: passes * 2 * 2^n * sizeof(amplitude) */
  double flops;            /* algorithmic flops: 2 per real FMA of the complex MACs;
                              16 per amplitude per dense or controlled one-qubit op,
                              8 per diagonal op, 32 per two-qubit dense op */
  int64_t upload_bytes;    /* op descriptors copied host -> device */
  int64_t tile_launches;   /* launches of the tile-pass kernel */
  double kernel_ms[5];     /* with QS_OPT_TIME_KERNELS: tile, plain, remap, small-state, block GEMM */
  double tile_flops;       /* algorithmic flops of the tile-pass launches */
} qs_stats;

/* ---- state vector ------------------------------------------------------ */

/* Allocate an n-qubit state (1 <= n <= 36) of precision prec on the current
 * device and set it to |0...0>.  alloc may be NULL (cudaMalloc).  stream is a
 * cudaStream_t (NULL = legacy default stream). */
qs_status sv_create(int n, int prec, const qs_allocator* alloc, void* stream, qs_state_t* out);
/* A state over a caller-owned device buffer of 2^n interleaved amplitudes of
 * precision prec (16-byte aligned), used in place and left as it is (no
 * |0...0>): every state-vector entry point then reads and updates that buffer.
 * The library allocates only its own scratch and op buffers (alloc may be
 * NULL: cudaMalloc); sv_destroy frees those and never the buffer, which must
 * outlive the state.  Used by the sharded executor, whose shards stay in their
 * own memory across the exchange steps.  Errors: QS_EINVAL, QS_ENOMEM. */
qs_status sv_wrap(int n, int prec, void* device_buf, const qs_allocator* alloc, void* stream,
                  qs_state_t* out);
qs_status sv_destroy(qs_state_t st);
qs_status sv_set_stream(qs_state_t st, void* stream);
qs_status sv_info(qs_state_t st, int* n, int* prec, void** device_ptr);

/* |J> (basis state, Eq. (multiqubitstate)). */
qs_status sv_set_basis(qs_state_t st, uint64_t J);
/* Copy 2^n interleaved amplitudes in/out; buf is a device pointer when
 * on_device != 0 (no synchronisation), else a host pointer (synchronises). */
qs_status sv_copy_in(qs_state_t st, const void* buf, int on_device);
qs_status sv_copy_out(qs_state_t st, void* buf, int on_device);

/* psi <- U_L ... U_1 psi for gates[0..ngates) in time order (section "Quantum
 * circuits", Eq. (twoqubitqft) shows the reversal).  opts may be NULL. */
qs_status sv_apply_circuit(qs_state_t st, const qs_gate* gates, size_t ngates,
                           const qs_opts* opts, qs_stats* stats);

/* Born rule p_J = |a_J|^2.  out: device buffer of float (out_fp64 = 0) or
 * double; with marg_mask == 0 or all n bits set, 2^n values in index order;
 * otherwise the marginal over the bits in marg_mask, 2^popcount(mask) values
 * indexed by those bits packed in increasing bit order.  out may be NULL.
 * norm_out (HOST, may be NULL) receives sum_J p_J accumulated in fp64 and
 * makes the call synchronous. */
qs_status sv_probs(qs_state_t st, void* out, int out_fp64, uint64_t marg_mask, double* norm_out);

/* sv_probs into a HOST buffer: the same values (2^n, or 2^popcount(mask) for a
 * marginal; float or double as out_fp64).  Into page-locked host memory that the
 * device can address (cudaHostAlloc / pinned), the kernel writes the full
 * distribution directly; into any other host memory it is formed in 64 MiB
 * chunks in a device staging buffer (obtained from the state's allocator at the
 * first call and kept until sv_destroy) and each chunk copied to host_out.
 * Copies queued by sv_probs_host_async on this state are waited for first.
 * norm_out as in sv_probs.  Synchronises.  Errors: QS_EINVAL, QS_ENOMEM,
 * QS_EUNSUPPORTED (marginal over more than 16 qubits), QS_ECUDA. */
qs_status sv_probs_host(qs_state_t st, void* host_out, int out_fp64, uint64_t marg_mask, double* norm_out);

/* The full distribution p_J = |a_J|^2 (Born rule, as sv_probs) into a HOST
 * buffer without waiting for the copy, so that it overlaps whatever the caller
 * queues next on the state.  The probabilities are formed on the state's stream
 * into one of two device buffers that the state keeps (2 x 2^n floats or
 * doubles, from the state's allocator at the first call, released by
 * sv_destroy), then copied to host_out on a copy stream of the state's own.  The
 * call returns once both steps are queued: the state may be changed at once (the
 * copy reads the buffer, not the amplitudes), but host_out (2^n floats when
 * out_fp64 = 0, else doubles; page-locked for the copy to run asynchronously)
 * must stay allocated and unread until sv_probs_wait returns.  The two buffers
 * are used in turn; a call whose buffer still feeds an earlier copy makes the
 * state's stream wait for that copy on the device.  The copy runs on a copy
 * engine, which shares HBM with the kernels queued after the call: beside kernels
 * that keep HBM busy (the 5-qubit block passes) it runs far slower than alone,
 * and the synchronous sv_probs_host, whose kernel writes into the host buffer
 * itself, is the faster choice there.  Errors: QS_EINVAL (NULL state or
 * host_out), QS_ENOMEM (the buffers), QS_ECUDA. */
qs_status sv_probs_host_async(qs_state_t st, void* host_out, int out_fp64);
/* Waits for every copy that sv_probs_host_async queued on this state; returns
 * QS_ECUDA with the message if one of them failed.  sv_destroy waits too. */
qs_status sv_probs_wait(qs_state_t st);

/* Multinomial log-likelihood l = sum_J n_J log p_J (terms with n_J = 0 are 0;
 * p_J <= 0 with n_J > 0 is clamped to 1e-300 and counted).  counts: DEVICE,
 * 2^n uint32.  out (HOST) receives l; clamped (HOST, may be NULL) the count
 * of clamped terms.  Synchronises. */
qs_status sv_loglik(qs_state_t st, const uint32_t* counts, double* out, int64_t* clamped);

/* Adjoint gradient of L(p(psi)) with respect to every gate angle, where
 * psi = U_L...U_1 psi_0 and psi_0 is the current content of st:
 *   mode 0: L = sum_J w_J p_J, w = weights (DEVICE, 2^n doubles);
 *   mode 1: L = sum_J n_J log p_J, weights = counts as DEVICE 2^n doubles.
 * dtheta (HOST, ngates*3 doubles): dL/dparam[k] of gate g at [3g+k], 0 for
 * unparameterised gates.  loss (HOST, may be NULL) receives L.  On return st
 * holds the final state U psi_0.  checkpoint_every = 0 uncomputes states with
 * U^dagger; k > 0 stores a device copy every k gates and recomputes forward
 * from it (deep circuits).  Synchronises. */
qs_status sv_grad(qs_state_t st, const qs_gate* gates, size_t ngates, const double* weights,
                  int mode, int checkpoint_every, double* dtheta, double* loss);

/* ---- batched density matrices / Pauli transfer matrices ---------------- */

/* Op codes of a batched noisy circuit (rows of 4 int32: code, q0, q1, aux).
 * After X90/Y90/CZ/IDLE the circuit's noise channel acts on every qubit the op
 * touches (IDLE: all): symmetric depolarizing (p_x = p_y = p_z = p/3, Eq.
 * (singletDepolarizingChannel)) and then amplitude damping with decay
 * parameter 1 and rate gamma (Eqs. (singletAmplitudeDampingChannel1-2)). */
enum {
  QS_DM_X90 = 0,   /* R^x(theta_x) on q0 */
  QS_DM_Y90 = 1,   /* R^y(theta_y) on q0 */
  QS_DM_CZ = 2,    /* CZ on (q0, q1) */
  QS_DM_IDLE = 3,  /* identity on the register */
  QS_DM_PTM1 = 4,  /* user 4x4 PTM ptm1[aux] on q0, no channel */
  QS_DM_PTM2 = 5   /* user 16x16 PTM ptm2[aux] on (q0 most significant digit, q1), no channel */
};

/* A batch of small noisy circuits; every pointer is DEVICE memory.
 * State of circuit c: Pauli vector r_i = Tr(P^_i rho) of its nq[c] qubits
 * (Eqs. (paulibasis), (GSTVectorizedRho); base-4 digit b of i belongs to
 * bit b), initial rho = |0...0><0...0|, measurement E_J = |J><J|. */
typedef struct {
  int32_t n_circuits;
  int32_t max_qubits;      /* >= every nq[c], <= 6 (sizes shared memory and scratch) */
  int32_t max_ops;         /* >= every op_off[c+1]-op_off[c] (sizes gradient checkpoints) */
  int32_t n_ptm1;          /* entries in ptm1 (aux of QS_DM_PTM1 must be below) */
  int32_t n_ptm2;          /* entries in ptm2 */
  int32_t flags;           /* QS_DM_VALIDATE, or 0 */
  const int32_t* nq;       /* [C] 1..6 */
  const int64_t* op_off;   /* [C+1] rows of ops for circuit c: op_off[c]..op_off[c+1] */
  const int32_t* ops;      /* [rows*4] (code, q0, q1, aux) */
  const double* params;    /* [C*4] theta_x, theta_y, p, gamma */
  const int64_t* out_off;  /* [C+1] offsets of circuit c's 2^nq outcomes in probs/counts */
  const int32_t* counts;   /* [out_off[C]] or NULL (no likelihood / gradient) */
  const double* ptm1;      /* user 4x4 PTMs, row-major, or NULL */
  const double* ptm2;      /* user 16x16 PTMs, row-major, or NULL */
} qs_dm_batch;

/* Opt-in check of the channels a batch describes (section "Quantum operations"):
 * before anything is launched, every user PTM (ptm1, ptm2; gst ptms) is copied to
 * the host and must be trace preserving -- first row (1, 0, ..., 0), the
 * property stated after Eq. (paulitransfermatrix) -- and completely positive --
 * its Choi matrix (Eq. (choimatrix)) positive semidefinite -- each within
 * 1e-8; the built-in channels' parameters must have p and gamma in [0, 1] and
 * finite angles.  A failure returns QS_EINVAL, launches nothing, and
 * qs_last_error() names the first failing matrix (or circuit) by its index.
 * Without the flag the inputs are used as given.  The check synchronises the
 * stream (it reads the device arrays). */
#define QS_DM_VALIDATE 1

/* Forward (and optionally adjoint) pass of a batch.  probs (DEVICE, float,
 * out_off[C] values, may be NULL); loglik (DEVICE, double [C], may be NULL;
 * needs counts); grad (DEVICE, double [C*4] = d loglik / d(theta_x, theta_y,
 * p, gamma), may be NULL; needs counts).  Asynchronous on stream.
 * Probabilities p_J <= 0 met with n_J > 0 are clamped to 1e-300.
 * A circuit whose nq, length, op code, qubit or PTM index is out of range is
 * skipped and its outputs are set to NaN (checked on the device; the call
 * still returns QS_OK).  The gradient uses device scratch for checkpoints
 * (stream-ordered cudaMallocAsync/cudaFreeAsync inside the call). */
qs_status dm_apply_channels(const qs_dm_batch* batch, float* probs, double* loglik, double* grad,
                            void* stream);

/* ---- serving: continuous batching of circuits ----------------------------
 * A server owns a scheduler thread and max_inflight worker threads.  Submitted
 * circuits (each from |0...0>, result = marginal outcome probabilities over
 * marg_mask, the Born rule of section "Quantum circuits") are admitted as device
 * memory and slots free up, while earlier ones are still running:
 *   - circuits with n <= small_max_qubits go through one persistent packed
 *     kernel of persistent_ctas CTAs fed by a device-visible work queue in
 *     mapped host memory: each CTA takes the next published circuit, runs it on
 *     a state held in its shared memory and publishes the result; a CTA that
 *     finds no work waits at most idle_ms, then the kernel ends reporting
 *     QS_ETIMEOUT in its status word (counted in qs_server_stats.idle_timeouts)
 *     and is launched again when work arrives.  It also ends after 50 ms, and
 *     while it may run the tensor-core block passes of this library leave
 *     persistent_ctas SMs (at most half of them) free;
 *   - larger circuits get a resident state (stream-ordered allocation within
 *     mem_budget) on a worker's stream and run the default method
 *     (QS_METHOD_AUTO; QS_METHOD_TILED with large_tiled = 1), overlapping with
 *     each other and with the packed kernel.
 * Latency = completion seen by the server - submission time. */
typedef struct qs_server_s* qs_server_t;

typedef struct {
  int32_t prec;              /* QS_C64 or QS_C128 */
  int32_t small_max_qubits;  /* <= 14 (QS_C64) / 13 (QS_C128); 0 = largest allowed */
  int32_t max_inflight;      /* large circuits on the device at once; 0 = 4 */
  int32_t persistent_ctas;   /* CTAs of the persistent packed kernel; 0 = 16 */
  uint64_t mem_budget;       /* device bytes for resident states; 0 = 80% of free memory */
  int32_t idle_ms;           /* the packed kernel's bounded wait for work; 0 = 5 ms */
  int32_t large_tiled;       /* 1: large circuits on QS_METHOD_TILED instead of QS_METHOD_AUTO */
} qs_server_config;

typedef struct {
  int64_t submitted, completed, packed_launches, packed_circuits, large_circuits;
  double p50_ms, p99_ms, mean_ms, max_ms;
  double wall_s;             /* first submission to last completion */
  double circuits_per_s;
  uint64_t peak_bytes;       /* largest resident-state footprint */
  int64_t idle_timeouts;     /* launches of the packed kernel that ended by its idle limit */
} qs_server_stats;

qs_status qs_server_create(const qs_server_config* cfg, qs_server_t* out);
/* Copies the gates; returns at once with a ticket.  marg_mask: bits of the
 * marginal (popcount <= 12; 0 means all n bits, allowed for n <= 12).
 * n in [1, 30]. */
qs_status qs_server_submit(qs_server_t s, int n, const qs_gate* gates, size_t ngates,
                           uint64_t marg_mask, int64_t* ticket);
/* Blocks until the circuit is done; result (HOST, 2^popcount doubles, may be
 * NULL), latency_ms (HOST, may be NULL).  Each ticket can be waited once. */
qs_status qs_server_wait(qs_server_t s, int64_t ticket, double* result, double* latency_ms);
qs_status qs_server_stats_get(qs_server_t s, qs_server_stats* out);
/* Waits for all submitted circuits, stops the scheduler, frees everything. */
qs_status qs_server_destroy(qs_server_t s);
/* Testing hook for the scheduler's error path: the next completion query of the
 * running persistent packed kernel reports cuda_error (a cudaError_t value other
 * than cudaSuccess and cudaErrorNotReady) instead of asking the device.  A query
 * that reports an error completes the queued small circuits with it: their
 * qs_server_wait returns QS_ECUDA with the error's name, and the queue starts
 * over.  Errors: QS_EINVAL. */
qs_status qs_server_inject_query_error(qs_server_t s, int cuda_error);

/* The check of QS_DM_VALIDATE on HOST arrays: count n-qubit PTMs (n = 1 or 2,
 * 4^n x 4^n doubles each, row-major G[out][in], the Pauli basis order of
 * Eq. (paulibasis)).  QS_OK when every one is trace preserving and completely
 * positive within 1e-8; otherwise QS_EINVAL, *bad_index (may be NULL) = the first
 * failing matrix (-1 on success) and a message saying which property failed.
 * Host only: no CUDA call. */
qs_status qs_ptm_check(const double* ptms, int n, int count, int* bad_index);

/* ---- probabilities without allocation ------------------------------------
 * The thesis has no counterpart of this entry point; it exists for callers
 * that may not allocate device memory (their own allocator owns the device,
 * or an allocation is not allowed where they call it).  It computes what
 * sv_probs computes, but for caller-owned buffers and without any cudaMalloc /
 * cudaFree or other allocation: amps (DEVICE, 2^n interleaved amplitudes of
 * precision prec), out (DEVICE, float or double as out_fp64, 2^n values, or
 * 2^popcount(mask) marginal values, may be NULL), norm_out (HOST, may be
 * NULL; synchronises stream).  Its reduction scratch is one fixed array in
 * device global memory (about 41 KB per device, held until the process
 * exits): n <= 36 and marginals over at most 12 qubits, else QS_EINVAL.  Every
 * call looks up that array's device address on the current device.  With lazy
 * module loading (the CUDA default) the first call on each device loads the
 * library module that holds the array, which places it in device memory: make
 * one call per device before the regions where allocation is not allowed (and
 * before capturing the stream into a graph).  All calls share the array and
 * find the previous call's contents in it (the kernels clear what must start
 * at zero); calls that overlap on the GPU race on it. */
qs_status qs_probs_noalloc(const void* amps, int n, int prec, void* out, int out_fp64,
                           uint64_t marg_mask, double* norm_out, void* stream);

/* ---- GST predictions for repeated gates ---------------------------------- */

/* Eq. (GSTPrediction): p_J(r) = <<E_J| (G_s)^r G_(prep) |rho>> for batches of
 * 1- or 2-qubit sequences, with Pauli transfer matrices (Eq.
 * (paulitransfermatrix), normalised Pauli basis of Eq. (paulibasis): base-4
 * digit b of an index belongs to qubit b, qubit 0 the least significant) acting on
 * Pauli vectors (Eqs. (GSTVectorizedRho), (GSTVectorizedEJ)).  All arrays are
 * DEVICE memory, FP64: ptms n_ptm x 4^n x 4^n (G[out][in]); rho 4^n; effects
 * 2^n x 4^n (row J = <<E_J|, J = the outcome bit string); gate count int32 (PTM
 * index of G_s); prep count x 8 int32: the PTM indices of G_(prep) in time order
 * (the first listed acts first), -1 ends a list.  A sequence with an index out of
 * range (or, for the power, reps < 0) gets NaN outputs. */
typedef struct {
  int32_t n;              /* qubits: 1 or 2 */
  int32_t count;          /* sequences */
  int32_t r_max;          /* dm_gst_series: repetitions 1..r_max */
  int32_t n_ptm;          /* PTMs in the table */
  int32_t flags;          /* QS_DM_VALIDATE (checks every PTM of the table), or 0 */
  int32_t reserved;
  const double* ptms;
  const double* rho;
  const double* effects;
  const int32_t* gate;
  const int32_t* prep;
} qs_gst_batch;

/* Every r = 1..r_max: probs (DEVICE, count x r_max x 2^n float) gets
 * p_J(r) at [(i r_max + r - 1) 2^n + J].  One warp per sequence, one
 * matrix-vector product per repetition in FP32 (inputs converted once).
 * Asynchronous on stream.  Errors: QS_EINVAL (NULL, n, r_max), QS_ECUDA. */
qs_status dm_gst_series(const qs_gst_batch* b, float* probs, void* stream);

/* One repetition count per sequence, reps (DEVICE, count int64 >= 0), by
 * repeated squaring of G_s in FP64 (about 2 log2 r matrix products): probs
 * (DEVICE, count x 2^n double).  Asynchronous on stream.  Errors: as above. */
qs_status dm_gst_power(const qs_gst_batch* b, const int64_t* reps, double* probs, void* stream);

/* ---- [[4,2,2]] error detection ----------------------------------------- */

/* Evaluation of the error-detection experiment, simulation side (Eq.
 * (errordetectionDbareenc)).  Per circuit c (all arrays DEVICE float):
 *   enc[c*32 + J]  outcome probabilities of the encoded circuit on 5 qubits (bit b of
 *                  J = qubit q_b: q0 the ancilla, q1..q4 the data qubits), e.g.
 *                  from dm_apply_channels;
 *   bare[c*4 + J], ideal[c*4 + J]  bare and noiseless bare distributions,
 *                  J = 2 j0 + j1 (j0 = q3, j1 = q4).
 * Outputs: p_enc[c*4 + L] the postselected logical distribution (outcomes with
 * q0 = 1 or an odd number of 1's on q1..q4 discarded, the rest mapped onto the
 * logical basis of Eqs. (errordetection00L)-(errordetection11L) and renormalised;
 * zeros when nothing is kept), ratio[c] the kept fraction (postselection ratio),
 * d_bare[c], d_enc[c] = (1/2) sum_L |p_L - ideal_L|.  Asynchronous on stream.
 * Errors: QS_EINVAL (count < 0, NULL array), QS_ECUDA. */
qs_status dm_code422_eval(int count, const float* enc, const float* bare, const float* ideal,
                          float* p_enc, float* ratio, float* d_bare, float* d_enc, void* stream);

/* ---- checkpoint / resume ------------------------------------------------ */

/* Binary checkpoint of the state, for resuming an interrupted simulation (the
 * thesis's solver saves its state vector in binary form for that purpose).
 * File: a 48-byte little-endian header -- magic "QSIMSV1\0", uint32 n, uint32
 * prec, uint64 amplitude bytes, uint64 checksum, 16 zero bytes -- then the 2^n
 * interleaved (re, im) amplitudes in the state's precision.  The checksum is the
 * sum mod 2^64, over the amplitude bytes as 64-bit words w_i (i from 0), of
 * splitmix64_finaliser(w_i + (i + 1) * 0x9E3779B97F4A7C15), computed on the GPU.
 * sv_save writes path (replacing it); the state is unchanged.  sv_load reads a
 * checkpoint written for the same n and precision into the state.  Both stream
 * through 2 x 64 MiB of pinned host memory and synchronise the state's stream.
 * Errors: QS_EINVAL (NULL; file cannot be opened, written or read; not a
 * checkpoint; n or precision differ -- the state unchanged; truncated file or
 * checksum mismatch -- the state reset to |0...0>), QS_ENOMEM, QS_ECUDA. */
qs_status sv_save(qs_state_t st, const char* path);
qs_status sv_load(qs_state_t st, const char* path);

/* ---- readout transforms ------------------------------------------------ */

/* Bloch vectors of every qubit (Eq. (multiqubitblochvector)): for q = 0..n-1
 * (bit positions) r_out[3q], r_out[3q+1], r_out[3q+2] = <sigma^x_q>,
 * <sigma^y_q>, <sigma^z_q> = the sums over the amplitude pairs (a0, a1) that
 * differ only in bit q of 2 Re(a0* a1), 2 Im(a0* a1), |a0|^2 - |a1|^2 (no
 * normalisation).  r_out: HOST, 3n doubles.  Sums in the state's precision
 * within a tile of 4096 amplitudes, FP64 across tiles; one read of the state
 * per 12 (first) or 8 (further) qubits.  Uses the state's scratch; synchronises
 * its stream.  Errors: QS_EINVAL (NULL), QS_ECUDA. */
qs_status sv_bloch(qs_state_t st, double* r_out);

/* Measurement-error model (Eq. (errordetectionMeasurementError)), in place:
 * each bit of an outcome string is misread independently, so
 *   p_J <- sum_J' p_J' prod_q P_q(j_q | j'_q),
 * with P_q(1 | 0) = e01[q] (a 0 counted as a 1) and P_q(0 | 1) = e10[q]; the
 * thesis's model is e01[q] = e10[q] = eps, where the product is
 * eps^D (1 - eps)^(n - D), D the Hamming distance of J and J'.  probs: DEVICE,
 * 2^n floats (fp64 = 0) or doubles (fp64 = 1), bit q of the index = qubit q,
 * 16-byte aligned; e01 (HOST, n doubles in [0, 1]), e10 (HOST, n doubles, or
 * NULL for e10 = e01).  1 <= n <= 40.  One read+write of probs per 12 (first)
 * or 8 (further) qubits, asynchronous on stream.  Errors: QS_EINVAL (NULL,
 * misaligned, n or a rate out of range), QS_ECUDA. */
qs_status qs_meas_error(void* probs, int n, int fp64, const double* e01, const double* e10,
                        void* stream);

/* ---- profiling --------------------------------------------------------- */

/* Between qs_profile_begin and qs_profile_end every state-vector launch of
 * this library is bracketed by CUDA events recorded on its stream (no
 * synchronisation).  qs_profile_end synchronises those events and returns,
 * per kind (0 tile pass, 1 plain per-gate, 2 remap, 3 small state, 4 block GEMM), the
 * summed device milliseconds and launch counts (HOST arrays of 5, may be
 * NULL).  One session per process at a time. */
qs_status qs_profile_begin(void);
qs_status qs_profile_end(double* kernel_ms, int64_t* launches);

/* ---- measurement -------------------------------------------------------- */

/* Measured arithmetic peak of the current GPU (no thesis counterpart: the
 * denominator of the rooflines of kernels bound by plain arithmetic).  kind 0:
 * FP32 multiply-adds issued as packed FP32x2 instructions; kind 1: FP64
 * multiply-adds.  Every SM runs 2048 threads of 8 independent FMA chains; the
 * best of three timed launches (CUDA events on stream, after one warm-up) gives
 * flops_per_s (2 per FMA).  sm_count (may be NULL): the device's SM count;
 * ms (may be NULL): that launch's time.  Synchronises stream.  Errors:
 * QS_EINVAL, QS_ECUDA. */
qs_status qs_alu_peak(int kind, double* flops_per_s, int* sm_count, double* ms, void* stream);

/* ---- misc -------------------------------------------------------------- */

const char* qs_last_error(void);
const char* qs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* QSIM_H */
