// Internal declarations shared by the translation units of libqs.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "qs.h"

struct qs_state_s {
  int n = 0;
  qs_dtype dtype = QS_C128;
  qs_math math = QS_MATH_DF;
  // complex64 dense gates on 3..5 targets: CUDA cores (0), tensor cores where
  // they are faster (1), tensor cores wherever they apply (2);
  // qs_set_tensor_cores.
  int tensor_cores = 1;
  void* psi = nullptr;  // device amplitudes
  bool owns = false;
  cudaStream_t stream = nullptr;
  int device = 0;
  // Per-state scratch for reductions, grown on demand (cudaMalloc).
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  void* host_scratch = nullptr;  // pinned host mirror for small results
  size_t host_scratch_bytes = 0;
  // Slot of this state's device-side error word (0: the shared overflow
  // slot, used once every other slot is taken).
  int err_slot = 0;
  // Launches of the last qs_fuse_run on this state (qs_last_run_stats).
  int64_t run_fused_launches = 0;
  int64_t run_gate_launches = 0;
  int64_t run_dense_blocks = 0;  // composed dense blocks (qs_densefuse.h)
  int64_t run_dense_gates = 0;   // gates they absorbed
  // Split state (qs_create_split): segments, placement and qubit map
  // (qs_split.cu); nullptr for a state in one allocation.
  void* split = nullptr;
};

namespace qs {

qs_status fail(qs_status st, const char* fmt, ...);
qs_status cuda_fail(cudaError_t e, const char* what);
#define QS_CUDA(call)                                  \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return ::qs::cuda_fail(e_, #call); \
  } while (0)

inline size_t amp_bytes(qs_dtype dt) { return dt == QS_C64 ? 8 : 16; }

// Device-side error words: kernels that run bounded waits record a nonzero
// code in the word of the state they work on; qs_sync and every synchronous
// call on that state read and clear it.
qs_status device_error_check(qs_state s);
uint32_t* error_word(qs_state s);
// Limit of every bounded device-side wait, in nanoseconds (qs_set_wait_limit).
uint64_t wait_limit_ns();

// Number of resident CTAs per SM for a kernel, cached per function pointer.
int sm_count(int device);

// ---------------------------------------------------------------------------
// Gate descriptors handed to the kernel launchers (already validated).
// ---------------------------------------------------------------------------
// Bits inserted into a compressed item index to form an amplitude index:
// positions ascending; fixed_mask holds the bits that are 1 (controls,
// matched pattern bits).
struct InsertSpec {
  int npos = 0;
  uint64_t high_mask[QS_MAX_QUBITS];  // ~((1 << pos_j) - 1), ascending pos_j
  uint64_t fixed_mask = 0;
};
InsertSpec make_insert(const std::vector<int>& positions, uint64_t fixed_mask);

// Dense single-qubit gate (optionally controlled).
qs_status launch_dense1(qs_state s, int target, uint64_t ctrl_mask, const double* U);
// Dense two-qubit gate (optionally controlled), matrix index b_t0 + 2 b_t1.
qs_status launch_dense2(qs_state s, int t0, int t1, uint64_t ctrl_mask, const double* U);
// Multiply every amplitude whose bits under `mask` equal `pattern` by c.
qs_status launch_phase(qs_state s, uint64_t mask, uint64_t pattern, double c_re, double c_im);
// Swap pair partners on target (X), times +-i for Y (kind 1), under ctrl_mask.
qs_status launch_xy(qs_state s, int target, uint64_t ctrl_mask, int y);
// General diagonal on k targets under ctrl_mask.
qs_status launch_diag(qs_state s, const int* targets, int k, uint64_t ctrl_mask, const double* d);
// Permutation on k targets under ctrl_mask.
qs_status launch_perm(qs_state s, const int* targets, int k, uint64_t ctrl_mask, const uint32_t* perm);

// Reductions / data movement (qs_reduce.cu).
qs_status launch_init_basis(qs_state s, uint64_t idx);
qs_status run_norm(qs_state s, double* out);
qs_status run_probs(qs_state s, const int* qubits, int k, double* out);
qs_status run_gather(qs_state s, const uint64_t* idx, int64_t count, void* host_out);

// Gate dispatch shared by the single-gate API and the circuit runner:
// classify the gate (identity, diagonal, phase on a pattern, X/Y move,
// permutation, dense) and launch the cheapest kernel for it.
qs_status dispatch_u1(qs_state s, int target, uint64_t ctrl_mask, const double* U);
// Dense gate on 3..5 targets (qs_densek.cu): tensor cores or FP32 CUDA
// cores for complex64 states (the state's tensor-core mode), FP64 CUDA cores
// for complex128.
qs_status launch_dense_k(qs_state s, const int* targets, int k, uint64_t ctrl_mask, const double* U);
qs_status dispatch_uk(qs_state s, const int* targets, int k, uint64_t ctrl_mask, const double* M);
qs_status dispatch_diag(qs_state s, const int* targets, int k, uint64_t ctrl_mask, const double* d);
qs_status dispatch_perm(qs_state s, const int* targets, int k, uint64_t ctrl_mask, const uint32_t* perm);

// Phase tables for runs of phase terms (qs_phase.cu): entry 256 b + v is
// exp(2 pi i (v 2^(8b)) / 2^32).  ensure_phase_tables fills them on the
// current device (once; synchronous copies, so not inside a stream
// capture); phase_table returns the device address of one format:
// 0 float2, 1 double2, 2 float4 (re head, im head, re tail, im tail).
void turn_cos_sin(uint32_t m, double* c, double* s);
qs_status ensure_phase_tables(int device);
const void* phase_table(int device, int format);

// Internal handles: a state record over memory the caller manages (psi may
// be nullptr), with its own error word; free_sub_state releases the record
// and its scratch buffers, never psi.
qs_state new_sub_state(int n, qs_dtype dtype, void* psi);
void free_sub_state(qs_state s);

// Split states (qs_split.cu).
qs_status split_run(qs_state s, const qs_circuit* c, int max_fuse);
// One gate given through the single-gate calls (arguments validated).
qs_status split_gate(qs_state s, int kind, const int* targets, int k, uint64_t ctrl_mask, const double* data,
                     size_t ndata, const uint32_t* perm);
qs_status split_init_basis(qs_state s, uint64_t idx);
qs_status split_copy_in(qs_state s, const void* host);
qs_status split_copy_out(qs_state s, void* host, bool sync);
qs_status split_gather(qs_state s, const uint64_t* idx, int64_t count, void* host_out);
qs_status split_norm(qs_state s, double* out);
qs_status split_probs(qs_state s, const int* qubits, int k, double* out);
qs_status split_check(qs_state s);
void split_set_stream(qs_state s, cudaStream_t stream);
void split_set_math(qs_state s, qs_math math);
void split_set_tensor_cores(qs_state s, int enable);
void split_destroy(qs_state s);
qs_status qs_fuse_run_gatewise(qs_state s, const qs_circuit* c);

qs_status ensure_scratch(qs_state s, size_t bytes);
qs_status ensure_host_scratch(qs_state s, size_t bytes);

}  // namespace qs
