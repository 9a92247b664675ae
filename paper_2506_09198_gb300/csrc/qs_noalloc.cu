// qs_probs_noalloc: marginal probabilities (or the norm) of a state held in
// caller-owned device memory, without allocating anything.
//
// Who needs this: callers that cannot call cudaMalloc.  qs_probs keeps a
// per-state scratch buffer that it grows with cudaMalloc (and a pinned host
// buffer from cudaMallocHost).  That fails or is unwelcome when the device
// memory belongs to another allocator (a framework's caching pool that has
// reserved the free memory, so a raw cudaMalloc runs out of memory), when the
// caller runs in a latency-critical loop where an allocation — and the
// device-wide synchronisation of a later cudaFree — is not acceptable, or when
// the caller only holds device pointers and owns no qs_state at all.  This
// entry point uses a fixed scratch array that lives in the library's own
// device image instead.
//
// The scratch is a file-scope static __device__ array of
// QS_NOALLOC_MAX_PARTIALS doubles (512 KiB).  Every GPU that loads the
// library holds it until the process exits.  Host code must not use the
// array's name as an address: on the host it is only a stand-in symbol.  The
// first call on each device, with that device current, looks up the device
// address with cudaGetSymbolAddress, checks the result and caches it; make
// that first call before any stream capture.
//
// All calls share the one array, which keeps the last call's contents.  The
// partial-sum kernel writes every slot it later reads, so nothing has to be
// cleared first.  Calls whose work overlaps on the GPU (two streams, or two
// threads) race on the array: serialise them.
#include <mutex>

#include "qs_internal.h"

#define QS_NOALLOC_MAX_PARTIALS (1u << 16)

static __device__ __align__(256) double g_noalloc_partials[QS_NOALLOC_MAX_PARTIALS];

namespace qs {
qs_status launch_probs_into(const void* psi, int n, qs_dtype dtype, const int* qubits, int k, double* partial,
                            uint64_t partial_cap, double* dout, cudaStream_t stream, int device);
}

using namespace qs;

namespace {

std::mutex g_setup_mu;
double* g_scratch_addr[64] = {nullptr};

// Device address of the scratch array on `device` (the current device).
qs_status scratch_for_device(int device, double** out) {
  if (device < 0 || device >= 64) return fail(QS_ERR_UNSUPPORTED, "device ordinal %d not supported", device);
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
    if (!p) return fail(QS_ERR_CUDA, "cudaGetSymbolAddress returned NULL for the no-alloc scratch");
    g_scratch_addr[device] = (double*)p;
  }
  *out = g_scratch_addr[device];
  return QS_OK;
}

}  // namespace

extern "C" qs_status qs_probs_noalloc(const void* device_state, int n, qs_dtype dtype, const int* qubits, int k,
                                      double* device_out, void* stream) {
  if (!device_state) return fail(QS_ERR_ARG, "device_state is NULL");
  if (((uintptr_t)device_state) % 16 != 0) return fail(QS_ERR_ARG, "device_state must be 16-byte aligned");
  if (dtype != QS_C64 && dtype != QS_C128) return fail(QS_ERR_ARG, "unknown dtype %d", (int)dtype);
  const int nmax = dtype == QS_C64 ? 35 : 34;
  if (n < 1 || n > nmax) return fail(QS_ERR_ARG, "n = %d outside [1, %d]", n, nmax);
  if (k < 0 || k > 16 || k > n)
    return fail(QS_ERR_ARG, "k = %d outside [0, min(16, n)]: the %u-entry scratch holds at most 2^16 outcomes", k,
                QS_NOALLOC_MAX_PARTIALS);
  if (k > 0 && !qubits) return fail(QS_ERR_ARG, "qubits is NULL");
  uint64_t used = 0;
  for (int j = 0; j < k; ++j) {
    if (qubits[j] < 0 || qubits[j] >= n) return fail(QS_ERR_ARG, "qubit %d out of range [0, %d)", qubits[j], n);
    if ((used >> qubits[j]) & 1ull) return fail(QS_ERR_ARG, "qubit %d appears twice", qubits[j]);
    used |= 1ull << qubits[j];
  }
  if (!device_out) return fail(QS_ERR_ARG, "device_out is NULL");
  if (((uintptr_t)device_out) % 8 != 0) return fail(QS_ERR_ARG, "device_out must be 8-byte aligned");
  int device = 0;
  QS_CUDA(cudaGetDevice(&device));
  // Both buffers must be device memory of the current GPU: a host pointer or
  // another GPU's memory is an argument error, not a kernel fault.  (Looking
  // up pointer attributes allocates nothing.)
  const void* ptrs[2] = {device_state, device_out};
  const char* names[2] = {"device_state", "device_out"};
  for (int j = 0; j < 2; ++j) {
    cudaPointerAttributes attr;
    const cudaError_t e = cudaPointerGetAttributes(&attr, ptrs[j]);
    if (e != cudaSuccess) return cuda_fail(e, "cudaPointerGetAttributes");
    if (attr.type != cudaMemoryTypeDevice)
      return fail(QS_ERR_ARG, "%s is not device memory (memory type %d)", names[j], (int)attr.type);
    if (attr.device != device)
      return fail(QS_ERR_ARG, "%s is on device %d, but device %d is current", names[j], attr.device, device);
  }
  double* scratch = nullptr;
  qs_status st = scratch_for_device(device, &scratch);
  if (st != QS_OK) return st;
  return launch_probs_into(device_state, n, dtype, qubits, k, scratch, QS_NOALLOC_MAX_PARTIALS, device_out,
                           (cudaStream_t)stream, device);
}
