/*
 * qs.h — C ABI of libqs, a GB300 (sm_103a) state-vector gate engine.
 *
 * The library applies quantum gates to a state of 2^n complex amplitudes
 * held in GPU memory.  arXiv 2506.09198 (Sec. I) names this multiplication
 * of gate matrices into the state vector as the central step of full
 * state-vector simulation.
 *
 * Layout (Sec. II-A, Fig. 1): amplitudes are stored array-of-structures,
 * (re, im) side by side: complex64 = two floats (8 bytes), complex128 = two
 * doubles (16 bytes) — the memory layout of torch.complex64/complex128.
 * Qubit q is bit q of the amplitude index, qubit 0 the least significant
 * (Algorithm 1: a gate on target t pairs index up, bit t = 0, with
 * lo = up + 2^t).
 *
 * Matrices are always passed in double precision, row-major, with each
 * complex entry as (re, im).  For a k-qubit matrix the row and column index
 * is s = sum_j bit(targets[j]) * 2^j: targets[0] is the least significant
 * (the paper fixes no basis order; this is the reading used throughout).
 * A control list means the gate acts only on amplitudes whose control bits
 * are all 1 (Fig. 4, Sec. III-A).  Controls on 0 are made by conjugating
 * with X.
 *
 * Errors: every function returns a qs_status.  QS_OK is 0.  On any other
 * value, qs_last_error() returns a message for the calling thread.  The
 * library never aborts and never throws across this boundary.  Gate calls
 * are asynchronous on the state's stream: an error raised on the device
 * (for example a bounded wait that ran out) is recorded in that state's own
 * device error word and reported by the state's next synchronous call
 * (qs_sync, qs_norm, qs_probs, qs_copy_out, qs_gather); other states are not
 * affected.  A batched launch records its errors in the first state's word.
 *
 * Threads: a qs_state handle is not thread-safe; distinct handles may be
 * used from distinct threads.
 */
#ifndef QS_H
#define QS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QS_OK = 0,
  QS_ERR_ARG = 1,          /* invalid argument (range, duplicate qubit, bad table) */
  QS_ERR_OOM = 2,          /* device memory could not be allocated */
  QS_ERR_CUDA = 3,         /* a CUDA runtime call failed (message has the CUDA error) */
  QS_ERR_TIMEOUT = 4,      /* a bounded wait (host or device) ran out */
  QS_ERR_UNSUPPORTED = 5,  /* valid request this build does not handle */
  QS_ERR_DEVICE = 6        /* a device-side check recorded an error */
} qs_status;

typedef enum { QS_C64 = 0, QS_C128 = 1 } qs_dtype;

/* Arithmetic used for complex128 states.
 * QS_MATH_DF: products and sums in float-float (pairs of FP32 values, about
 *   48 significant bits) on the FP32 pipes; every result is rounded back to
 *   IEEE double.  Default: GB300's FP64 pipe is about 70x slower than FP32.
 *   Amplitude components below 2^-74 in magnitude are flushed to zero and
 *   magnitudes must stay below 2^100.
 * QS_MATH_FP64: plain IEEE double arithmetic on the FP64 pipe.
 * complex64 states always compute in FP32. */
typedef enum { QS_MATH_DF = 0, QS_MATH_FP64 = 1 } qs_math;

typedef struct qs_state_s* qs_state;

enum {
  QS_MAX_QUBITS = 40,     /* index arithmetic limit; memory limits come first */
  QS_MAX_TARGETS = 8,     /* largest target set of a diagonal/permutation gate */
  QS_MAX_DENSE = 5        /* largest target set of a general (dense) matrix gate */
};

/* ---- state lifetime -------------------------------------------------- */

/* The first qs_create or qs_wrap on a device also fills the library's phase
 * tables there (static device arrays, 40 KiB, by a synchronous copy), so it
 * must not run inside a stream capture. */

/* Allocate a state of n qubits (1 <= n <= QS_MAX_QUBITS) with cudaMalloc on
 * the current device and set it to |0...0>.  The handle owns the memory and
 * uses the legacy default stream until qs_set_stream.  QS_ERR_OOM if the
 * allocation fails. */
qs_status qs_create(int n, qs_dtype dtype, qs_state* out);

/* Wrap caller-owned device memory (for example a torch tensor) of
 * 2^n amplitudes of dtype, 16-byte aligned.  The handle never frees it.
 * stream may be NULL (legacy default stream). */
qs_status qs_wrap(int n, qs_dtype dtype, void* device_ptr, void* stream, qs_state* out);

/* A state larger than HBM allows: the top g qubits (1 <= g <= 6) select one
 * of 2^g segments of 2^(n-g) amplitudes; segments 0 .. hbm_segments - 1 are
 * allocated in device memory (cudaMalloc), the others in pinned host memory
 * that the GPU reads and writes directly (cudaHostAlloc, mapped; over
 * NVLink-C2C on Grace).  The paper places a state that outgrows one memory
 * across two (Sec. II-B, NUMA V1/V2); this is that placement for HBM and host
 * memory.  n - g >= 10 (a gate's targets and controls must fit the local
 * qubits with room to spare).  The handle takes every call that takes a state
 * except qs_wrap, qs_device_ptr, qs_autotune and the batched calls
 * (QS_ERR_UNSUPPORTED).  A gate on local qubits runs on each segment; a
 * control on a global qubit selects segments; a diagonal gate's global
 * targets are fixed per segment; a gate that needs a global qubit as a target
 * first swaps it with a local qubit (half of every segment pair is
 * exchanged), and an internal qubit map keeps the logical order, which
 * qs_copy_out, qs_gather and qs_probs restore first.  Segments in host memory
 * run on the per-gate kernels only; segments in device memory also run fused
 * blocks.  State |0...0>.  QS_ERR_OOM if an allocation fails. */
qs_status qs_create_split(int n, qs_dtype dtype, int g, int hbm_segments, qs_state* out);

/* Release the handle (and its memory if it owns it).  NULL is accepted. */
qs_status qs_destroy(qs_state s);

qs_status qs_set_stream(qs_state s, void* cuda_stream);
qs_status qs_set_math(qs_state s, qs_math math);
/* Engine for complex64 dense gates on 3..5 targets (qs_apply_dense,
 * QS_GATE_UK).  On the tensor cores each group of 2^k amplitudes is a row of
 * a GEMM with the gate's real 2^(k+1) x 2^(k+1) form (3 or 4 targets: the
 * 5-target form I (x) U with the lowest free qubits); operands are split into TF32 head
 * and remainder and three products are summed in FP32, so the error stays at
 * FP32's level (per amplitude within (4 d + 8) 2^-24 sum_c |U_rc||x_c|).  On
 * the CUDA cores each output is one FP32 FMA chain.
 * mode 1 (default): the tensor cores at 5 targets, and at 3 or 4 targets when
 *   qubits 0 and 1 are both targets or controls (the CUDA-core kernel's
 *   accesses are strided then); the CUDA cores otherwise.
 * mode 2: the tensor cores wherever they apply (3 targets need 2 free qubits).
 * mode 0: the CUDA cores.
 * complex128 states ignore it: they run on the CUDA cores in their math mode
 * (float-float: one lane per output row, TwoSum accumulation; FP64: FMA
 * chains). */
qs_status qs_set_tensor_cores(qs_state s, int mode);
qs_status qs_num_qubits(qs_state s, int* n);
qs_status qs_device_ptr(qs_state s, void** device_ptr);

/* ---- data movement ---------------------------------------------------- */

/* |idx> (0 <= idx < 2^n), written on the state's stream. */
qs_status qs_init_basis(qs_state s, uint64_t idx);

/* Copy 2^n amplitudes of the state's dtype from host memory, interleaved
 * (re, im).  Asynchronous on the state's stream when host is pinned; the
 * caller keeps host valid until the stream reaches this point. */
qs_status qs_copy_in(qs_state s, const void* host);

/* Copy the whole state to host memory (same layout).  Synchronous. */
qs_status qs_copy_out(qs_state s, void* host);

/* Like qs_copy_out, but asynchronous on the state's stream: the copy is
 * complete when the stream reaches this point (qs_sync).  host should be
 * pinned (page-locked) so that the copy overlaps other streams' work. */
qs_status qs_copy_out_async(qs_state s, void* host);

/* host_out[j] = amplitude idx[j] (count entries, state's dtype), for
 * sampled checks of large states.  Synchronous.  Indices must be < 2^n. */
qs_status qs_gather(qs_state s, const uint64_t* idx, int64_t count, void* host_out);

/* ---- gates (asynchronous on the state's stream) ---------------------- */

/* Single-qubit gate U (2x2: u00 u01 u10 u11, each (re, im)) on target.
 * Pairs (up, lo = up + 2^target): up' = u00 up + u01 lo, lo' = u10 up + u11 lo
 * (Algorithm 1, generalised from the Hadamard to any U). */
qs_status qs_apply_1q(qs_state s, int target, const double U[8]);

/* Two-qubit gate U (4x4) on (t0, t1), t0 != t1.  On each quad
 * (a, a+2^t0, a+2^t1, a+2^t0+2^t1) with matrix index b_t0 + 2 b_t1 (Sec.
 * III-A names two-qubit gates; the basis order is this library's reading). */
qs_status qs_apply_2q(qs_state s, int t0, int t1, const double U[32]);

/* Controlled single-qubit gate: U on target where all nctrl controls are 1
 * (Fig. 4: only amplitudes with control bit 1 are updated).  nctrl may be 0.
 * CNOT is ctrl = {c}, U = X. */
qs_status qs_apply_ctrl(qs_state s, const int* ctrls, int nctrl, int target, const double U[8]);

/* General gate: the 2^k x 2^k matrix U (row-major, (re, im) pairs) on k
 * targets (1 <= k <= QS_MAX_DENSE) where all nctrl controls are 1.  Sub-
 * register value s = sum_j bit(i, targets[j]) 2^j indexes rows and columns;
 * each group of 2^k amplitudes sharing the other bits is multiplied by U
 * (the in-place matrix-vector product of Sec. II-C and Fig. 3, extended
 * from the paper's one and two targets to k).
 * Diagonal and permutation matrices run as qs_apply_diag / qs_apply_perm;
 * dense matrices on 3..5 targets run on the tensor cores or the FP32 CUDA
 * cores for complex64 states (qs_set_tensor_cores), on the CUDA cores in the
 * state's math mode for complex128 states. */
qs_status qs_apply_dense(qs_state s, const int* ctrls, int nctrl, const int* targets, int k, const double* U);

/* Diagonal gate on k targets (1 <= k <= QS_MAX_TARGETS):
 * psi_i <- d[s(i)] psi_i with s(i) = sum_j bit(i, targets[j]) 2^j; d holds
 * 2^k complex entries (re, im).  Controlled phase shifts (Sec. III-B) and
 * phase oracles are diagonal gates. */
qs_status qs_apply_diag(qs_state s, const int* targets, int k, const double* d);

/* Permutation gate: where all controls are 1, the basis state with target
 * sub-register value v moves to perm[v] (a bijection of 0..2^k-1,
 * 1 <= k <= QS_MAX_TARGETS).  Controlled modular multiplication of the
 * Shor-like workload (Sec. III-D) is such a gate.  Amplitudes are moved,
 * never rounded. */
qs_status qs_apply_perm(qs_state s, const int* ctrls, int nctrl, const int* targets, int k, const uint32_t* perm);

/* ---- circuits ---------------------------------------------------------- */

typedef enum {
  QS_GATE_U1 = 0,    /* 2x2 matrix on targets[0] */
  QS_GATE_UK = 1,    /* 2^k x 2^k matrix: any for k <= QS_MAX_DENSE (5; see
                        qs_apply_dense); for 6 <= k <= 8 only diagonal or
                        permutation matrices (QS_ERR_UNSUPPORTED otherwise) */
  QS_GATE_DIAG = 2,  /* 2^k diagonal entries */
  QS_GATE_PERM = 3   /* uint32 table of 2^k entries */
} qs_gate_kind;

typedef struct {
  int32_t kind;                     /* qs_gate_kind */
  int32_t k;                        /* number of targets */
  int32_t targets[QS_MAX_TARGETS];  /* distinct, < n */
  uint64_t ctrl_mask;               /* bit q set: qubit q is a control */
  int64_t offset;                   /* first double of the gate's data in
                                       qs_circuit.data (U1/UK/DIAG), or first
                                       entry in qs_circuit.perm (PERM) */
} qs_gate;

typedef struct {
  int64_t n_gates;
  const qs_gate* gates;
  const double* data;     /* matrices and diagonals, (re, im) interleaved */
  const uint32_t* perm;   /* permutation tables */
} qs_circuit;

typedef struct {
  int32_t max_fuse;   /* fusion: 1 = none (one kernel per gate); 2..6 = most
                         qubits above the resident low block that one fused
                         block may span (the block's tile holds 2^max_fuse
                         strided chunks); 0 = the qs_autotune choice for this
                         dtype, math mode and qubit count (4 if untuned) */
  int32_t use_graph;  /* qs_batch_run only (qs_fuse_run ignores it): 1
                         captures the call's launches as one CUDA graph and
                         launches that (fewer launch gaps); nothing is reused
                         across calls: qs_batch_compile does that */
  int32_t reserved[6];
} qs_run_opts;

/* Run a circuit on one state.  A dense gate on 3..5 targets is first
 * multiplied in FP64 with the gates after it that stay within 5 qubits (gates
 * on other qubits are stepped over where they commute with the block) into
 * one matrix applied in one pass.  Consecutive gates on the same one or two
 * qubits are multiplied into one 2x2 / 4x4 matrix in FP64 where that
 * saves arithmetic (never for permutations); then gates whose qubits fit
 * one block of at most max_fuse qubits are applied by one fused kernel that
 * keeps the block's amplitudes on chip for all of its gates (related work,
 * Sec. I: gate fusion and cache blocking).  Result equals applying the
 * gates one by one, up to rounding; permutations and SWAPs move amplitudes
 * exactly.  Between consecutive complex128 fused blocks the device memory
 * holds the state in an internal float-float form; it is back in (re, im)
 * doubles when the call's work completes on the stream.  If the call fails
 * after launching work (a device error or timeout at the next synchronous
 * call), the state's contents are unspecified.  opts may be NULL
 * (autotuned, no graph). */
qs_status qs_fuse_run(qs_state s, const qs_circuit* c, const qs_run_opts* opts);

/* Launch counts of the last qs_fuse_run on the state.  Every fused-block
 * launch reads and writes the whole state once (one HBM pass); a per-gate
 * launch reads and writes the amplitudes its gate changes. */
typedef struct {
  int64_t fused_launches;  /* fused-block kernels (one HBM pass each) */
  int64_t gate_launches;   /* gates run on the per-gate kernels */
  int64_t dense_blocks;    /* dense gates on 3..5 targets composed with the
                              gates after them on at most 5 qubits into one
                              matrix (one per-gate launch each) */
  int64_t dense_gates;     /* gates those blocks absorbed */
  int64_t reserved[4];
} qs_run_stats;
qs_status qs_last_run_stats(qs_state s, qs_run_stats* out);

/* Autotuner for fusion: run circuit c on s with every fusion setting
 * (max_fuse 1..6, which also sets the tile shape: 2^max_fuse strided chunks
 * of contiguous amplitudes), time each on the device (the fastest of three
 * runs after an untimed one), and remember the fastest fused setting for
 * states of s's dtype, math mode and qubit count, whatever circuit later
 * runs on them (tune on the circuit that matters; a width tuned on one
 * circuit family is a guess for another);
 * qs_fuse_run with max_fuse = 0 then uses it (default 4 before any tuning).
 * s is scratch: it is reset to |0...0> before each trial and holds the last
 * trial's result afterwards.  Synchronous.  best_max_fuse and best_ms may be
 * NULL. */
qs_status qs_autotune(qs_state s, const qs_circuit* c, int* best_max_fuse, double* best_ms);

/* Run circuits[i] on states[i] for i < count (distinct states, one dtype and
 * math mode, one device), asynchronously on the first state's stream.  Each
 * state's circuit is compiled into fused blocks (as qs_fuse_run does).
 * States that fit one tile (11 qubits complex128, 12 complex64) run in one
 * persistent launch: CTAs claim whole states, largest estimated cost first.
 * States of up to 20 qubits follow block by block: launch k applies block k
 * of every such state, its tiles spread over the GPU.  Wider states follow as
 * fused whole-GPU blocks (qs_fuse_run).  The first state's stream first waits
 * for the work already queued on every other member's stream, and every
 * other member's stream then waits for the batch (events; the host does not
 * block).  The circuits are read before the call returns.  Every gate must fit
 * a fused tile op (dense on at most 2 targets, diagonal or permutation on at
 * most 8): a dense gate on 3..5 targets gives QS_ERR_UNSUPPORTED here (run it
 * with qs_fuse_run or qs_apply_dense). */
qs_status qs_batch_run(qs_state* states, const qs_circuit* const* circuits, int count, const qs_run_opts* opts);

/* A compiled batch: the work of qs_batch_run compiled and captured as a CUDA
 * graph once, then launched any number of times (each launch applies the
 * circuits again to the states' current contents).  The handle owns its
 * device workspace (one cudaMalloc at compile time) and copies everything it
 * needs from the circuits, so they may be freed after qs_batch_compile.
 * Destroying a member state invalidates the handle: qs_batch_launch then
 * returns QS_ERR_ARG.  Not thread-safe per handle. */
typedef struct qs_batch_s* qs_batch;

/* Compile and capture (synchronous host work; device copies are queued on the
 * first state's stream).  count >= 1; the arguments are checked as in
 * qs_batch_run.  Must not run inside a stream capture. */
qs_status qs_batch_compile(qs_state* states, const qs_circuit* const* circuits, int count, qs_batch* out);

/* Launch the captured graph on the first state's current stream, with the
 * same stream ordering against the other members as qs_batch_run. */
qs_status qs_batch_launch(qs_batch b);

/* Wait for the handle's last launch, then release it.  NULL is accepted. */
qs_status qs_batch_destroy(qs_batch b);

/* ---- reductions (synchronous) ---------------------------------------- */

/* out = sum_i |psi_i|^2, accumulated with at least 48 significant bits and
 * combined in FP64. */
qs_status qs_norm(qs_state s, double* out);

/* out[v] = sum over i with sub-register value v on qubits[0..k-1] of
 * |psi_i|^2 (2^k doubles, 1 <= k <= 16). */
qs_status qs_probs(qs_state s, const int* qubits, int k, double* out);

/* Marginal probabilities like qs_probs, or the norm with k = 0, for callers
 * that cannot allocate memory.  The paper has no counterpart: this is a
 * deployment variant.  qs_probs grows a per-state scratch buffer with
 * cudaMalloc (and a pinned host buffer); callers whose device memory belongs
 * to another allocator, that must not pay an allocation or the device-wide
 * synchronisation of a later cudaFree inside a latency-critical loop, or that
 * hold only raw device pointers, call this instead.  It allocates nothing:
 * its scratch is a fixed array of 2^16 doubles (512 KiB) inside the library's
 * device image, held by every GPU that loads the library until exit.
 *   device_state  2^n amplitudes of dtype, device memory of the current GPU,
 *                 16-byte aligned (host memory or another GPU's memory is
 *                 rejected with QS_ERR_ARG)
 *   qubits, k     0 <= k <= min(16, n) distinct qubits (k = 0: out[0] = norm)
 *   device_out    2^k doubles of device memory of the current GPU (8-byte
 *                 aligned, checked like device_state), written
 *                 asynchronously on stream (NULL: legacy default stream)
 * Larger k is rejected with QS_ERR_ARG.  The first call on each device looks
 * up the scratch address on the current device; make it before any stream
 * capture.  All calls share the scratch: calls that overlap on the GPU race,
 * so serialise them.  The scratch keeps the last call's contents; every slot
 * a call reads is written by that call first. */
qs_status qs_probs_noalloc(const void* device_state, int n, qs_dtype dtype, const int* qubits, int k,
                           double* device_out, void* stream);

/* Limit of every bounded wait inside the fused and batched kernels (a wait
 * on a tile copy or on the warps that consume it), in seconds, 0 to 60;
 * default 2.  Applies to launches queued after the call, process-wide; with
 * 0 a wait gives up at once if its barrier is not complete when it first
 * checks.  A wait that runs out stops the kernel early: the kernel records
 * QS_ERR_TIMEOUT in the state's error word, lets its own copies land and
 * returns, so the context stays usable and the state's contents are
 * unspecified.  Production code keeps the default; a short limit is for
 * testing that path. */
qs_status qs_set_wait_limit(double seconds);

/* Wait for the state's stream with a host-side deadline: QS_ERR_TIMEOUT if
 * it has not drained after timeout_s seconds (the work is not cancelled).
 * Reports device-side errors recorded since the last synchronous call. */
qs_status qs_sync(qs_state s, double timeout_s);

const char* qs_last_error(void);
const char* qs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* QS_H */
