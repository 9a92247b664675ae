// C ABI of libqs: handles, argument validation, error reporting, and the
// single-gate entry points.  Every function validates its arguments before it
// touches CUDA, returns a qs_status and never throws.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <chrono>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "qs_internal.h"

namespace qs {

static thread_local char g_last_error[512] = "";

qs_status fail(qs_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
  return st;
}

qs_status cuda_fail(cudaError_t e, const char* what) {
  const qs_status st = (e == cudaErrorMemoryAllocation) ? QS_ERR_OOM : QS_ERR_CUDA;
  return fail(st, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

// Device-side error words, one per live state (per device that loaded this
// module).  Slot 0 is shared by the states created once every other slot is
// taken; a nonzero word means that a bounded wait of a kernel working on the
// slot's state ran out.
constexpr int kErrSlots = 8192;
__device__ uint32_t g_err_words[kErrSlots];

namespace slots {
std::mutex g_slot_mu;
std::vector<int> g_free_slots;
bool g_slots_init = false;
std::atomic<uint64_t> g_wait_ns{2000000000ull};

int acquire_err_slot() {
  std::lock_guard<std::mutex> lk(g_slot_mu);
  if (!g_slots_init) {
    for (int i = kErrSlots - 1; i >= 1; --i) g_free_slots.push_back(i);
    g_slots_init = true;
  }
  if (g_free_slots.empty()) return 0;
  const int slot = g_free_slots.back();
  g_free_slots.pop_back();
  return slot;
}

void release_err_slot(int slot) {
  if (slot <= 0) return;
  std::lock_guard<std::mutex> lk(g_slot_mu);
  g_free_slots.push_back(slot);
}

}  // namespace slots
using namespace slots;

namespace {
uint32_t* err_words(int device) {
  static std::mutex mu;
  static void* addr[64] = {nullptr};
  std::lock_guard<std::mutex> lk(mu);
  if (device < 0 || device >= 64) return nullptr;
  if (!addr[device]) {
    if (cudaGetSymbolAddress(&addr[device], g_err_words) != cudaSuccess) addr[device] = nullptr;
  }
  return (uint32_t*)addr[device];
}
}  // namespace

uint32_t* error_word(qs_state s) {
  uint32_t* base = err_words(s->device);
  return base ? base + s->err_slot : nullptr;
}

uint64_t wait_limit_ns() { return g_wait_ns.load(std::memory_order_relaxed); }

qs_status device_error_check(qs_state s) {
  uint32_t v = 0;
  const size_t off = (size_t)s->err_slot * sizeof(uint32_t);
  cudaError_t e = cudaMemcpyFromSymbolAsync(&v, g_err_words, sizeof(v), off, cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "device error check");
  if (v != 0) {
    const uint32_t zero = 0;
    cudaMemcpyToSymbolAsync(g_err_words, &zero, sizeof(zero), off, cudaMemcpyHostToDevice, s->stream);
    cudaStreamSynchronize(s->stream);
    if (v == 1) return fail(QS_ERR_TIMEOUT, "a device-side bounded wait ran out (code %u)", v);
    return fail(QS_ERR_DEVICE, "device-side check failed (code %u)", v);
  }
  return QS_OK;
}

int sm_count(int device) {
  static std::mutex mu;
  static int cache[64] = {0};
  std::lock_guard<std::mutex> lk(mu);
  if (device < 0 || device >= 64) return 1;
  if (cache[device] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || v < 1) v = 1;
    cache[device] = v;
  }
  return cache[device];
}

qs_status ensure_scratch(qs_state s, size_t bytes) {
  if (s->scratch_bytes >= bytes) return QS_OK;
  if (s->scratch) {
    QS_CUDA(cudaStreamSynchronize(s->stream));
    cudaFree(s->scratch);
    s->scratch = nullptr;
    s->scratch_bytes = 0;
  }
  size_t want = 1 << 20;
  while (want < bytes) want <<= 1;
  QS_CUDA(cudaMalloc(&s->scratch, want));
  s->scratch_bytes = want;
  return QS_OK;
}

qs_status ensure_host_scratch(qs_state s, size_t bytes) {
  if (s->host_scratch_bytes >= bytes) return QS_OK;
  if (s->host_scratch) {
    QS_CUDA(cudaStreamSynchronize(s->stream));
    cudaFreeHost(s->host_scratch);
    s->host_scratch = nullptr;
    s->host_scratch_bytes = 0;
  }
  size_t want = 4096;
  while (want < bytes) want <<= 1;
  QS_CUDA(cudaMallocHost(&s->host_scratch, want));
  s->host_scratch_bytes = want;
  return QS_OK;
}

qs_state new_sub_state(int n, qs_dtype dtype, void* psi) {
  qs_state s = new (std::nothrow) qs_state_s();
  if (!s) return nullptr;
  s->n = n;
  s->dtype = dtype;
  s->psi = psi;
  s->owns = false;
  if (cudaGetDevice(&s->device) != cudaSuccess) s->device = 0;
  s->err_slot = acquire_err_slot();
  return s;
}

void free_sub_state(qs_state s) {
  if (!s) return;
  if (s->err_slot > 0) {
    uint32_t* w = error_word(s);
    if (w) {
      cudaMemsetAsync(w, 0, sizeof(uint32_t), s->stream);
      cudaStreamSynchronize(s->stream);
    }
    release_err_slot(s->err_slot);
  }
  if (s->scratch) cudaFree(s->scratch);
  if (s->host_scratch) cudaFreeHost(s->host_scratch);
  delete s;
}

void release_plan_cache(qs_state s);  // qs_circuit.cu

}  // namespace qs

using namespace qs;

namespace {

qs_status check_state(qs_state s) {
  if (!s) return fail(QS_ERR_ARG, "state handle is NULL");
  return QS_OK;
}

qs_status check_qubit(qs_state s, int q, const char* what) {
  if (q < 0 || q >= s->n) return fail(QS_ERR_ARG, "%s %d out of range [0, %d)", what, q, s->n);
  return QS_OK;
}

// Validates controls and targets (all distinct and in range) and builds the
// control mask.
qs_status check_qubits(qs_state s, const int* ctrls, int nctrl, const int* targets, int k, uint64_t* ctrl_mask) {
  if (nctrl < 0 || (nctrl > 0 && !ctrls)) return fail(QS_ERR_ARG, "bad control list");
  if (k < 1 || !targets) return fail(QS_ERR_ARG, "bad target list");
  uint64_t used = 0, cm = 0;
  for (int j = 0; j < k; ++j) {
    qs_status st = check_qubit(s, targets[j], "target");
    if (st != QS_OK) return st;
    if ((used >> targets[j]) & 1ull) return fail(QS_ERR_ARG, "qubit %d appears twice", targets[j]);
    used |= 1ull << targets[j];
  }
  for (int j = 0; j < nctrl; ++j) {
    qs_status st = check_qubit(s, ctrls[j], "control");
    if (st != QS_OK) return st;
    if ((used >> ctrls[j]) & 1ull) return fail(QS_ERR_ARG, "qubit %d appears twice", ctrls[j]);
    used |= 1ull << ctrls[j];
    cm |= 1ull << ctrls[j];
  }
  *ctrl_mask = cm;
  return QS_OK;
}

qs_status check_finite(const double* v, size_t count, const char* what) {
  if (!v) return fail(QS_ERR_ARG, "%s is NULL", what);
  for (size_t j = 0; j < count; ++j)
    if (!(v[j] == v[j]) || v[j] > 1.7e308 || v[j] < -1.7e308) return fail(QS_ERR_ARG, "%s has a non-finite entry", what);
  return QS_OK;
}

int max_qubits(qs_dtype dt) { return dt == QS_C64 ? 35 : 34; }

qs_status new_state(int n, qs_dtype dtype, qs_state* out) {
  if (!out) return fail(QS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (dtype != QS_C64 && dtype != QS_C128) return fail(QS_ERR_ARG, "unknown dtype %d", (int)dtype);
  if (n < 1 || n > max_qubits(dtype))
    return fail(QS_ERR_ARG, "n = %d outside [1, %d] for this dtype", n, max_qubits(dtype));
  qs_state s = new (std::nothrow) qs_state_s();
  if (!s) return fail(QS_ERR_OOM, "host allocation failed");
  s->n = n;
  s->dtype = dtype;
  *out = s;
  return QS_OK;
}

}  // namespace

extern "C" {

const char* qs_last_error(void) { return g_last_error; }
const char* qs_version(void) { return "libqs 0.1 (sm_103a)"; }

qs_status qs_create(int n, qs_dtype dtype, qs_state* out) {
  if (!out) return fail(QS_ERR_ARG, "out is NULL");
  *out = nullptr;
  qs_state s = nullptr;
  qs_status st = new_state(n, dtype, &s);
  if (st != QS_OK) return st;
  cudaError_t e = cudaGetDevice(&s->device);
  if (e != cudaSuccess) {
    delete s;
    return cuda_fail(e, "cudaGetDevice");
  }
  const size_t bytes = amp_bytes(dtype) << n;
  e = cudaMalloc(&s->psi, bytes);
  if (e != cudaSuccess) {
    delete s;
    return cuda_fail(e, "cudaMalloc(state)");
  }
  s->owns = true;
  s->err_slot = acquire_err_slot();
  st = ensure_phase_tables(s->device);
  if (st == QS_OK) st = launch_init_basis(s, 0);
  if (st == QS_OK) {
    e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) st = cuda_fail(e, "init");
  }
  if (st != QS_OK) {
    release_err_slot(s->err_slot);
    cudaFree(s->psi);
    delete s;
    return st;
  }
  *out = s;
  return QS_OK;
}

qs_status qs_wrap(int n, qs_dtype dtype, void* device_ptr, void* stream, qs_state* out) {
  if (!out) return fail(QS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!device_ptr) return fail(QS_ERR_ARG, "device_ptr is NULL");
  if (((uintptr_t)device_ptr) % 16 != 0) return fail(QS_ERR_ARG, "device_ptr must be 16-byte aligned");
  qs_state s = nullptr;
  qs_status st = new_state(n, dtype, &s);
  if (st != QS_OK) return st;
  cudaPointerAttributes attr;
  cudaError_t e = cudaPointerGetAttributes(&attr, device_ptr);
  if (e != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
    delete s;
    if (e != cudaSuccess) return cuda_fail(e, "cudaPointerGetAttributes");
    return fail(QS_ERR_ARG, "device_ptr is not device memory");
  }
  s->device = attr.device;
  s->psi = device_ptr;
  s->owns = false;
  s->stream = (cudaStream_t)stream;
  st = ensure_phase_tables(s->device);
  if (st != QS_OK) {
    delete s;
    return st;
  }
  s->err_slot = acquire_err_slot();
  *out = s;
  return QS_OK;
}

qs_status qs_destroy(qs_state s) {
  if (!s) return QS_OK;
  if (s->split) split_destroy(s);
  cudaStreamSynchronize(s->stream);
  release_plan_cache(s);
  if (s->err_slot > 0) {
    // The next owner of the slot starts from a clear word.
    uint32_t* w = error_word(s);
    if (w) {
      cudaMemsetAsync(w, 0, sizeof(uint32_t), s->stream);
      cudaStreamSynchronize(s->stream);
    }
    release_err_slot(s->err_slot);
  }
  if (s->owns && s->psi) cudaFree(s->psi);
  if (s->scratch) cudaFree(s->scratch);
  if (s->host_scratch) cudaFreeHost(s->host_scratch);
  delete s;
  return QS_OK;
}

qs_status qs_set_stream(qs_state s, void* cuda_stream) {
  qs_status st = check_state(s);
  if (st != QS_OK) return st;
  s->stream = (cudaStream_t)cuda_stream;
  if (s->split) split_set_stream(s, s->stream);
  return QS_OK;
}

qs_status qs_set_math(qs_state s, qs_math math) {
  qs_status st = check_state(s);
  if (st != QS_OK) return st;
  if (math != QS_MATH_DF && math != QS_MATH_FP64) return fail(QS_ERR_ARG, "unknown math mode %d", (int)math);
  s->math = math;
  if (s->split) split_set_math(s, math);
  return QS_OK;
}

qs_status qs_set_tensor_cores(qs_state s, int enable) {
  qs_status st = check_state(s);
  if (st != QS_OK) return st;
  if (enable < 0 || enable > 2) return fail(QS_ERR_ARG, "tensor-core mode %d outside [0, 2]", enable);
  s->tensor_cores = enable;
  if (s->split) split_set_tensor_cores(s, enable);
  return QS_OK;
}

qs_status qs_num_qubits(qs_state s, int* n) {
  qs_status st = check_state(s);
  if (st != QS_OK) return st;
  if (!n) return fail(QS_ERR_ARG, "n is NULL");
  *n = s->n;
  return QS_OK;
}

qs_status qs_device_ptr(qs_state s, void** p) {
  qs_status st = check_state(s);
  if (st != QS_OK) return st;
  if (!p) return fail(QS_ERR_ARG, "output pointer is NULL");
  if (s->split) return fail(QS_ERR_UNSUPPORTED, "a split state has no single device pointer");
  *p = s->psi;
  return QS_OK;
}

qs_status qs_init_basis(qs_state s, uint64_t idx) {
  qs_status st = check_state(s);
  if (st != QS_OK) return st;
  if (idx >= (1ull << s->n)) return fail(QS_ERR_ARG, "basis index out of range");
  if (s->split) return split_init_basis(s, idx);
  return launch_init_basis(s, idx);
}

qs_status qs_copy_in(qs_state s, const void* host) {
  qs_status st = check_state(s);
  if (st != QS_OK) return st;
  if (!host) return fail(QS_ERR_ARG, "host is NULL");
  if (s->split) return split_copy_in(s, host);
  QS_CUDA(cudaMemcpyAsync(s->psi, host, amp_bytes(s->dtype) << s->n, cudaMemcpyHostToDevice, s->stream));
  return QS_OK;
}

qs_status qs_copy_out(qs_state s, void* host) {
  qs_status st = check_state(s);
  if (st != QS_OK) return st;
  if (!host) return fail(QS_ERR_ARG, "host is NULL");
  if (s->split) return split_copy_out(s, host, true);
  QS_CUDA(cudaMemcpyAsync(host, s->psi, amp_bytes(s->dtype) << s->n, cudaMemcpyDeviceToHost, s->stream));
  QS_CUDA(cudaStreamSynchronize(s->stream));
  return device_error_check(s);
}

qs_status qs_copy_out_async(qs_state s, void* host) {
  qs_status st = check_state(s);
  if (st != QS_OK) return st;
  if (!host) return fail(QS_ERR_ARG, "host is NULL");
  if (s->split) return split_copy_out(s, host, false);
  QS_CUDA(cudaMemcpyAsync(host, s->psi, amp_bytes(s->dtype) << s->n, cudaMemcpyDeviceToHost, s->stream));
  return QS_OK;
}

qs_status qs_gather(qs_state s, const uint64_t* idx, int64_t count, void* host_out) {
  qs_status st = check_state(s);
  if (st != QS_OK) return st;
  if (count < 0 || (count > 0 && (!idx || !host_out))) return fail(QS_ERR_ARG, "bad gather arguments");
  for (int64_t j = 0; j < count; ++j)
    if (idx[j] >= (1ull << s->n)) return fail(QS_ERR_ARG, "gather index %lld out of range", (long long)j);
  if (s->split) return split_gather(s, idx, count, host_out);
  return run_gather(s, idx, count, host_out);
}

qs_status qs_apply_1q(qs_state s, int target, const double U[8]) {
  qs_status st = check_state(s);
  if (st != QS_OK) return st;
  uint64_t cm = 0;
  if ((st = check_qubits(s, nullptr, 0, &target, 1, &cm)) != QS_OK) return st;
  if ((st = check_finite(U, 8, "U")) != QS_OK) return st;
  if (s->split) return split_gate(s, QS_GATE_U1, &target, 1, 0, U, 8, nullptr);
  return dispatch_u1(s, target, 0, U);
}

qs_status qs_apply_2q(qs_state s, int t0, int t1, const double U[32]) {
  qs_status st = check_state(s);
  if (st != QS_OK) return st;
  const int tg[2] = {t0, t1};
  uint64_t cm = 0;
  if ((st = check_qubits(s, nullptr, 0, tg, 2, &cm)) != QS_OK) return st;
  if ((st = check_finite(U, 32, "U")) != QS_OK) return st;
  if (s->split) return split_gate(s, QS_GATE_UK, tg, 2, 0, U, 32, nullptr);
  return dispatch_uk(s, tg, 2, 0, U);
}

qs_status qs_apply_ctrl(qs_state s, const int* ctrls, int nctrl, int target, const double U[8]) {
  qs_status st = check_state(s);
  if (st != QS_OK) return st;
  uint64_t cm = 0;
  if ((st = check_qubits(s, ctrls, nctrl, &target, 1, &cm)) != QS_OK) return st;
  if ((st = check_finite(U, 8, "U")) != QS_OK) return st;
  if (s->split) return split_gate(s, QS_GATE_U1, &target, 1, cm, U, 8, nullptr);
  return dispatch_u1(s, target, cm, U);
}

qs_status qs_apply_dense(qs_state s, const int* ctrls, int nctrl, const int* targets, int k, const double* U) {
  qs_status st = check_state(s);
  if (st != QS_OK) return st;
  if (k < 1 || k > QS_MAX_DENSE) return fail(QS_ERR_ARG, "k = %d outside [1, %d]", k, (int)QS_MAX_DENSE);
  uint64_t cm = 0;
  if ((st = check_qubits(s, ctrls, nctrl, targets, k, &cm)) != QS_OK) return st;
  const size_t nd = (size_t)2 << (2 * k);
  if ((st = check_finite(U, nd, "U")) != QS_OK) return st;
  if (s->split) return split_gate(s, k == 1 ? QS_GATE_U1 : QS_GATE_UK, targets, k, cm, U, nd, nullptr);
  if (k == 1) return dispatch_u1(s, targets[0], cm, U);
  return dispatch_uk(s, targets, k, cm, U);
}

qs_status qs_apply_diag(qs_state s, const int* targets, int k, const double* d) {
  qs_status st = check_state(s);
  if (st != QS_OK) return st;
  if (k < 1 || k > QS_MAX_TARGETS) return fail(QS_ERR_ARG, "k = %d outside [1, %d]", k, (int)QS_MAX_TARGETS);
  uint64_t cm = 0;
  if ((st = check_qubits(s, nullptr, 0, targets, k, &cm)) != QS_OK) return st;
  if ((st = check_finite(d, (size_t)2 << k, "d")) != QS_OK) return st;
  if (s->split) return split_gate(s, QS_GATE_DIAG, targets, k, 0, d, (size_t)2 << k, nullptr);
  return dispatch_diag(s, targets, k, 0, d);
}

qs_status qs_apply_perm(qs_state s, const int* ctrls, int nctrl, const int* targets, int k, const uint32_t* perm) {
  qs_status st = check_state(s);
  if (st != QS_OK) return st;
  if (k < 1 || k > QS_MAX_TARGETS) return fail(QS_ERR_ARG, "k = %d outside [1, %d]", k, (int)QS_MAX_TARGETS);
  uint64_t cm = 0;
  if ((st = check_qubits(s, ctrls, nctrl, targets, k, &cm)) != QS_OK) return st;
  if (!perm) return fail(QS_ERR_ARG, "perm is NULL");
  std::vector<char> seen((size_t)1 << k, 0);
  for (int v = 0; v < (1 << k); ++v) {
    if (perm[v] >= (1u << k) || seen[perm[v]]) return fail(QS_ERR_ARG, "perm is not a bijection of 0..2^k-1");
    seen[perm[v]] = 1;
  }
  if (s->split) return split_gate(s, QS_GATE_PERM, targets, k, cm, nullptr, 0, perm);
  return dispatch_perm(s, targets, k, cm, perm);
}

qs_status qs_norm(qs_state s, double* out) {
  qs_status st = check_state(s);
  if (st != QS_OK) return st;
  if (!out) return fail(QS_ERR_ARG, "out is NULL");
  if (s->split) return split_norm(s, out);
  return run_norm(s, out);
}

qs_status qs_probs(qs_state s, const int* qubits, int k, double* out) {
  qs_status st = check_state(s);
  if (st != QS_OK) return st;
  if (k < 1 || k > 16 || k > s->n) return fail(QS_ERR_ARG, "k = %d outside [1, min(16, n)]", k);
  if (!out) return fail(QS_ERR_ARG, "out is NULL");
  uint64_t cm = 0;
  if ((st = check_qubits(s, nullptr, 0, qubits, k, &cm)) != QS_OK) return st;
  if (s->split) return split_probs(s, qubits, k, out);
  return run_probs(s, qubits, k, out);
}

qs_status qs_set_wait_limit(double seconds) {
  if (!(seconds >= 0.0) || seconds > 60.0) return fail(QS_ERR_ARG, "wait limit %g s outside [0, 60]", seconds);
  g_wait_ns.store((uint64_t)(seconds * 1e9), std::memory_order_relaxed);
  return QS_OK;
}

qs_status qs_sync(qs_state s, double timeout_s) {
  qs_status st = check_state(s);
  if (st != QS_OK) return st;
  if (!(timeout_s >= 0)) return fail(QS_ERR_ARG, "timeout must be >= 0");
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t e = cudaStreamQuery(s->stream);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) return cuda_fail(e, "stream");
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (el > timeout_s) return fail(QS_ERR_TIMEOUT, "stream not drained after %.3f s", timeout_s);
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  if (s->split) return split_check(s);
  return device_error_check(s);
}

}  // extern "C"
