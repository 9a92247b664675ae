// Reductions (norm, marginal probabilities), basis-state initialisation and
// sampled gathers.
//
// Sums of |psi_i|^2 are formed exactly in short runs on the FP32 pipes (each
// square as TwoProduct head + tail, run heads chained with TwoSum), and each
// run is added into a per-thread FP64 accumulator; per-thread and per-block
// partials are combined in FP64 in a fixed tree order, so results are
// deterministic for a given state size.  Marginals over k qubits run one
// reduction per outcome over the amplitudes whose measured bits equal it.
#include <cstring>

#include "qs_internal.h"
#include "qs_math.cuh"

namespace qs {

namespace {

constexpr int kRThreads = 256;

struct RunSum {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add_sq(float x) {
    const float p = x * x;
    const float e = __fmaf_rn(x, x, -p);
    const float t = s + p;
    const float bb = t - s;
    c += ((s - (t - bb)) + (p - bb)) + e;
    s = t;
  }
  // (h + l)^2 = h^2 + 2hl + l^2; the l^2 term is below 2^-96 h^2.
  __device__ __forceinline__ void add_sq(float h, float l) {
    const float p = h * h;
    const float e = __fmaf_rn(2.0f * h, l, __fmaf_rn(h, h, -p));
    const float t = s + p;
    const float bb = t - s;
    c += ((s - (t - bb)) + (p - bb)) + e;
    s = t;
  }
  __device__ __forceinline__ double flush() {
    const double r = f2d_exact(s) + f2d_exact(c);
    s = 0.f;
    c = 0.f;
    return r;
  }
};

__device__ __forceinline__ void accumulate(RunSum& r, const float2& a) {
  r.add_sq(a.x);
  r.add_sq(a.y);
}
__device__ __forceinline__ void accumulate(RunSum& r, const double2& a) {
  float h, l;
  d2ff(a.x, h, l);
  r.add_sq(h, l);
  d2ff(a.y, h, l);
  r.add_sq(h, l);
}

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[kRThreads / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < kRThreads / 32 ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;  // valid in thread 0
}

// Block (chunk c, outcome v) sums |psi_i|^2 over i = deposit(f) | bits(v),
// f in [c*per_chunk, (c+1)*per_chunk).  deposit spreads the free index over
// the unmeasured qubits (insert zeros at the measured positions).
struct MeasSpec {
  int npos;
  uint64_t high_mask[QS_MAX_QUBITS];
  int k;
  int qubits[16];
};

__device__ __forceinline__ uint64_t deposit(uint64_t f, const MeasSpec& m) {
  for (int j = 0; j < m.npos; ++j) f += f & m.high_mask[j];
  return f;
}

template <class Amp, int RUN>
__global__ void __launch_bounds__(kRThreads) k_sq_partial(const Amp* __restrict__ psi, uint64_t per_chunk,
                                                          int log_nchunks, MeasSpec m, double* __restrict__ partial) {
  const uint32_t v = blockIdx.x >> log_nchunks;
  const uint64_t chunk = blockIdx.x & ((1u << log_nchunks) - 1u);
  uint64_t vbits = 0;
  for (int j = 0; j < m.k; ++j)
    if ((v >> j) & 1u) vbits |= 1ull << m.qubits[j];
  const uint64_t f0 = chunk * per_chunk;
  double acc = 0.0;
  RunSum r;
  // RUN consecutive strided items per thread before one FP64 add.
  for (uint64_t f = threadIdx.x; f < per_chunk; f += (uint64_t)kRThreads * RUN) {
    Amp a[RUN];
#pragma unroll
    for (int u = 0; u < RUN; ++u) {
      const uint64_t ff = f + (uint64_t)u * kRThreads;
      if (ff < per_chunk) a[u] = psi[deposit(f0 + ff, m) | vbits];
    }
#pragma unroll
    for (int u = 0; u < RUN; ++u)
      if (f + (uint64_t)u * kRThreads < per_chunk) accumulate(r, a[u]);
    acc += r.flush();
  }
  const double t = block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// out[v] = sum over c of partial[v * nchunks + c], pairwise in a fixed order.
__global__ void __launch_bounds__(kRThreads) k_sum_rows(const double* __restrict__ partial, int nchunks,
                                                        double* __restrict__ out) {
  const double* row = partial + (uint64_t)blockIdx.x * nchunks;
  double acc = 0.0;
  for (int c = threadIdx.x; c < nchunks; c += kRThreads) acc += row[c];
  const double t = block_sum(acc);
  if (threadIdx.x == 0) out[blockIdx.x] = t;
}

template <class Amp>
__global__ void k_set_amp(Amp* psi, uint64_t idx, Amp value) {
  psi[idx] = value;
}

template <class Amp>
__global__ void k_gather(const Amp* __restrict__ psi, const uint64_t* __restrict__ idx, int64_t count,
                         Amp* __restrict__ out) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < count; j += (int64_t)gridDim.x * blockDim.x)
    out[j] = psi[idx[j]];
}

template <class Amp>
qs_status probs_impl(qs_state s, const int* qubits, int k, double* out) {
  MeasSpec m;
  std::memset(&m, 0, sizeof(m));
  std::vector<int> pos(qubits, qubits + k);
  InsertSpec ins = make_insert(pos, 0);
  m.npos = ins.npos;
  for (int j = 0; j < QS_MAX_QUBITS; ++j) m.high_mask[j] = ins.high_mask[j];
  m.k = k;
  for (int j = 0; j < k; ++j) m.qubits[j] = qubits[j];
  const int nfree = s->n - k;
  const uint64_t nout = 1ull << k;
  // About 8 CTAs per SM in total; chunks are powers of two dividing 2^nfree.
  const uint64_t want = (uint64_t)sm_count(s->device) * 8;
  uint64_t nchunks = 1;
  int log_nchunks = 0;
  while (nchunks * nout < want && nchunks * 2 <= (1ull << nfree) && nchunks < 65536) {
    nchunks *= 2;
    ++log_nchunks;
  }
  const uint64_t per_chunk = (1ull << nfree) / nchunks;
  const size_t need = (nout * nchunks + nout) * sizeof(double);
  qs_status st = ensure_scratch(s, need);
  if (st != QS_OK) return st;
  st = ensure_host_scratch(s, nout * sizeof(double));
  if (st != QS_OK) return st;
  double* partial = (double*)s->scratch;
  double* dout = partial + nout * nchunks;
  constexpr int RUN = sizeof(Amp) == 16 ? 4 : 8;
  const unsigned grid = (unsigned)(nchunks * nout);
  k_sq_partial<Amp, RUN><<<grid, kRThreads, 0, s->stream>>>((const Amp*)s->psi, per_chunk, log_nchunks, m, partial);
  QS_CUDA(cudaGetLastError());
  k_sum_rows<<<(unsigned)nout, kRThreads, 0, s->stream>>>(partial, (int)nchunks, dout);
  QS_CUDA(cudaGetLastError());
  QS_CUDA(cudaMemcpyAsync(s->host_scratch, dout, nout * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  QS_CUDA(cudaStreamSynchronize(s->stream));
  std::memcpy(out, s->host_scratch, nout * sizeof(double));
  return device_error_check(s);
}

}  // namespace

qs_status run_probs(qs_state s, const int* qubits, int k, double* out) {
  if (s->dtype == QS_C64) return probs_impl<float2>(s, qubits, k, out);
  return probs_impl<double2>(s, qubits, k, out);
}

qs_status run_norm(qs_state s, double* out) { return run_probs(s, nullptr, 0, out); }

// Same partial-sum and row-sum kernels as run_probs, writing into buffers the
// caller provides: partial (partial_cap doubles) and dout (2^k doubles, device
// memory).  Allocates nothing on host or device and does not synchronise.
qs_status launch_probs_into(const void* psi, int n, qs_dtype dtype, const int* qubits, int k, double* partial,
                            uint64_t partial_cap, double* dout, cudaStream_t stream, int device) {
  MeasSpec m;
  std::memset(&m, 0, sizeof(m));
  int pos[16];
  for (int j = 0; j < k; ++j) pos[j] = qubits[j];
  for (int a = 1; a < k; ++a)  // insertion sort, ascending
    for (int b = a; b > 0 && pos[b - 1] > pos[b]; --b) {
      const int t = pos[b];
      pos[b] = pos[b - 1];
      pos[b - 1] = t;
    }
  m.npos = k;
  for (int j = 0; j < k; ++j) m.high_mask[j] = ~((1ull << pos[j]) - 1ull);
  m.k = k;
  for (int j = 0; j < k; ++j) m.qubits[j] = qubits[j];
  const int nfree = n - k;
  const uint64_t nout = 1ull << k;
  if (partial_cap < nout) return fail(QS_ERR_ARG, "scratch holds %llu partials, %llu outcomes requested",
                                      (unsigned long long)partial_cap, (unsigned long long)nout);
  const uint64_t want = (uint64_t)sm_count(device) * 8;
  uint64_t nchunks = 1;
  int log_nchunks = 0;
  while (nchunks * nout < want && nchunks * 2 <= (1ull << nfree) && nchunks < 65536 &&
         nchunks * 2 * nout <= partial_cap) {
    nchunks *= 2;
    ++log_nchunks;
  }
  const uint64_t per_chunk = (1ull << nfree) / nchunks;
  const unsigned grid = (unsigned)(nchunks * nout);
  if (dtype == QS_C64) {
    k_sq_partial<float2, 8><<<grid, kRThreads, 0, stream>>>((const float2*)psi, per_chunk, log_nchunks, m, partial);
  } else {
    k_sq_partial<double2, 4><<<grid, kRThreads, 0, stream>>>((const double2*)psi, per_chunk, log_nchunks, m,
                                                               partial);
  }
  QS_CUDA(cudaGetLastError());
  k_sum_rows<<<(unsigned)nout, kRThreads, 0, stream>>>(partial, (int)nchunks, dout);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

qs_status launch_init_basis(qs_state s, uint64_t idx) {
  const size_t bytes = amp_bytes(s->dtype) << s->n;
  QS_CUDA(cudaMemsetAsync(s->psi, 0, bytes, s->stream));
  if (s->dtype == QS_C64)
    k_set_amp<float2><<<1, 1, 0, s->stream>>>((float2*)s->psi, idx, make_float2(1.f, 0.f));
  else
    k_set_amp<double2><<<1, 1, 0, s->stream>>>((double2*)s->psi, idx, make_double2(1.0, 0.0));
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

qs_status run_gather(qs_state s, const uint64_t* idx, int64_t count, void* host_out) {
  if (count == 0) return QS_OK;
  const size_t ab = amp_bytes(s->dtype);
  // Output block starts on a 256-byte boundary (16-byte amplitude stores).
  const size_t out_off = ((size_t)count * sizeof(uint64_t) + 255) & ~(size_t)255;
  const size_t need = out_off + (size_t)count * ab;
  qs_status st = ensure_scratch(s, need);
  if (st != QS_OK) return st;
  uint64_t* didx = (uint64_t*)s->scratch;
  void* dout = (char*)s->scratch + out_off;
  QS_CUDA(cudaMemcpyAsync(didx, idx, (size_t)count * sizeof(uint64_t), cudaMemcpyHostToDevice, s->stream));
  const unsigned grid = (unsigned)((count + 255) / 256 < 4096 ? (count + 255) / 256 : 4096);
  if (s->dtype == QS_C64)
    k_gather<float2><<<grid, 256, 0, s->stream>>>((const float2*)s->psi, didx, count, (float2*)dout);
  else
    k_gather<double2><<<grid, 256, 0, s->stream>>>((const double2*)s->psi, didx, count, (double2*)dout);
  QS_CUDA(cudaGetLastError());
  QS_CUDA(cudaMemcpyAsync(host_out, dout, (size_t)count * ab, cudaMemcpyDeviceToHost, s->stream));
  QS_CUDA(cudaStreamSynchronize(s->stream));
  return device_error_check(s);
}

}  // namespace qs
