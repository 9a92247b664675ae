// Per-gate kernels: dense 1q/2q, phase on a bit pattern, X/Y moves, k-target
// diagonal and permutation gates, for complex64 (FP32), complex128 with
// float-float arithmetic (default) and complex128 with FP64 arithmetic.
//
// Every kernel walks a compressed "item" index and forms amplitude indices by
// inserting fixed bits (the target's 0, controls' 1s), so a controlled gate
// reads and writes only the 2^(n-c) amplitudes it changes (the paper's Fig. 4
// access pattern, without the skipped branches).  Loops are grid-stride with
// the grid sized to the resident CTAs of all 152 SMs; each thread keeps ILP
// independent items in flight with 128-bit (c128) or 64-bit (c64) accesses,
// consecutive threads on consecutive items so every access is coalesced once
// the target is above the lowest qubits.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <type_traits>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <unordered_map>

#include "qs_internal.h"
#include "qs_math.cuh"

namespace qs {

struct DevInsert {
  int npos;
  uint64_t high_mask[QS_MAX_QUBITS];
  uint64_t fixed_mask;
};

static_assert(sizeof(DevInsert) == sizeof(InsertSpec), "layout");

InsertSpec make_insert(const std::vector<int>& positions, uint64_t fixed_mask) {
  std::vector<int> p = positions;
  std::sort(p.begin(), p.end());
  InsertSpec s;
  s.npos = (int)p.size();
  for (int j = 0; j < s.npos; ++j) s.high_mask[j] = ~((1ull << p[j]) - 1ull);
  for (int j = s.npos; j < QS_MAX_QUBITS; ++j) s.high_mask[j] = 0;
  s.fixed_mask = fixed_mask;
  return s;
}

static DevInsert to_dev(const InsertSpec& s) {
  DevInsert d;
  std::memcpy(&d, &s, sizeof(d));
  return d;
}

// Insert a zero at each position (ascending): adding the bits at and above
// the position doubles them, i.e. shifts them up by one.
__device__ __forceinline__ uint64_t expand_index(uint64_t p, const DevInsert& ins) {
  for (int j = 0; j < ins.npos; ++j) p += p & ins.high_mask[j];
  return p | ins.fixed_mask;
}

// Sign flips and moves without arithmetic (exact in every precision).
__device__ __forceinline__ float2 neg_amp(float2 a) {
  return make_float2(__uint_as_float(__float_as_uint(a.x) ^ 0x80000000u),
                     __uint_as_float(__float_as_uint(a.y) ^ 0x80000000u));
}
__device__ __forceinline__ double neg_d(double x) {
  return __hiloint2double(__double2hiint(x) ^ (int)0x80000000u, __double2loint(x));
}
__device__ __forceinline__ double2 neg_amp(double2 a) { return make_double2(neg_d(a.x), neg_d(a.y)); }
__device__ __forceinline__ float neg_s(float x) { return __uint_as_float(__float_as_uint(x) ^ 0x80000000u); }
__device__ __forceinline__ double neg_s(double x) { return neg_d(x); }

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------
template <class P>
struct Mat2 {
  typename P::Coef m[4];
};
template <class P>
struct Mat4 {
  typename P::Coef m[16];
  int row_exp[4];  // float-float path: sum_k (|re| + |im|) of row r < 2^row_exp[r]
};

// Smallest e with sum_k (|re u_rk| + |im u_rk|) (as floats) < 2^e.
static int row_exponent(const double* U, int row, int dim) {
  double sum = 0.0;
  for (int c = 0; c < dim; ++c) {
    const double* z = U + 2 * (row * dim + c);
    sum += std::fabs((double)(float)z[0]) + std::fabs((double)(float)z[1]);
  }
  if (sum == 0.0) return -126;
  int e = 0;
  std::frexp(sum, &e);  // sum = f 2^e, 0.5 <= f < 1, so sum < 2^e
  return e;
}

constexpr int kThreads = 256;

#ifdef QS_DENSE1_MIN_BLOCKS
#define QS_DENSE1_BOUNDS __launch_bounds__(kThreads, QS_DENSE1_MIN_BLOCKS)
#else
#define QS_DENSE1_BOUNDS __launch_bounds__(kThreads)
#endif

template <class P, int ILP>
__global__ void QS_DENSE1_BOUNDS k_dense1(typename P::Amp* __restrict__ psi, uint64_t n_items,
                                                     uint64_t tbit, DevInsert ins, Mat2<P> g) {
  using Amp = typename P::Amp;
  using Val = typename P::Val;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; base < n_items; base += stride * ILP) {
    uint64_t iu[ILP];
    Amp a[ILP], b[ILP];
#pragma unroll
    for (int u = 0; u < ILP; ++u) {
      const uint64_t item = base + u * stride;
      if (item < n_items) {
        iu[u] = expand_index(item, ins);
        a[u] = psi[iu[u]];
        b[u] = psi[iu[u] ^ tbit];
      }
    }
#pragma unroll
    for (int u = 0; u < ILP; ++u) {
      const uint64_t item = base + u * stride;
      if (item < n_items) {
        Val v[2] = {P::load(a[u]), P::load(b[u])};
        psi[iu[u]] = P::template mac_round<2>(&g.m[0], v);
        psi[iu[u] | tbit] = P::template mac_round<2>(&g.m[2], v);
      }
    }
  }
}

#ifndef QS_DENSE2_ILP
#define QS_DENSE2_ILP 1
#endif
// Six resident CTAs per SM (40 registers): the float-float 4x4 kernel waits on
// memory, and the extra warps keep more loads in flight.
#ifndef QS_DENSE2_MIN_BLOCKS
#define QS_DENSE2_MIN_BLOCKS 6
#endif
#define QS_DENSE2_BOUNDS __launch_bounds__(kThreads, QS_DENSE2_MIN_BLOCKS)

template <class P, int ILP>
__global__ void QS_DENSE2_BOUNDS k_dense2(typename P::Amp* __restrict__ psi, uint64_t n_items,
                                                     uint64_t b0, uint64_t b1, DevInsert ins, Mat4<P> g) {
  using Amp = typename P::Amp;
  using Val = typename P::Val;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; base < n_items; base += stride * ILP) {
    uint64_t i0[ILP];
    Amp a[ILP][4];
#pragma unroll
    for (int u = 0; u < ILP; ++u) {
      const uint64_t item = base + u * stride;
      if (item < n_items) {
        i0[u] = expand_index(item, ins);
        a[u][0] = psi[i0[u]];
        a[u][1] = psi[i0[u] | b0];
        a[u][2] = psi[i0[u] | b1];
        a[u][3] = psi[i0[u] | b0 | b1];
      }
    }
#pragma unroll
    for (int u = 0; u < ILP; ++u) {
      const uint64_t item = base + u * stride;
      if (item < n_items) {
        Val v[4] = {P::load(a[u][0]), P::load(a[u][1]), P::load(a[u][2]), P::load(a[u][3])};
        // Dense 4x4 rows (16 products) use the anchored accumulation; 2x2
        // rows keep TwoSum, which stays exact when heads cancel (structured
        // states such as Grover's, where every pair computes the same values
        // and rounding errors would add coherently).
        if constexpr (std::is_same<P, MathDFGate>::value) {
          const int mexp = P::template max_exp_field<4>(v);
          psi[i0[u]] = P::template mac_anchor_round<4>(&g.m[0], v, g.row_exp[0], mexp);
          psi[i0[u] | b0] = P::template mac_anchor_round<4>(&g.m[4], v, g.row_exp[1], mexp);
          psi[i0[u] | b1] = P::template mac_anchor_round<4>(&g.m[8], v, g.row_exp[2], mexp);
          psi[i0[u] | b0 | b1] = P::template mac_anchor_round<4>(&g.m[12], v, g.row_exp[3], mexp);
        } else {
          psi[i0[u]] = P::template mac_round<4>(&g.m[0], v);
          psi[i0[u] | b0] = P::template mac_round<4>(&g.m[4], v);
          psi[i0[u] | b1] = P::template mac_round<4>(&g.m[8], v);
          psi[i0[u] | b0 | b1] = P::template mac_round<4>(&g.m[12], v);
        }
      }
    }
  }
}

// psi_i *= c for every i whose bits under the inserted positions match the
// fixed pattern; NEG: c = -1, done as a sign flip.
template <class P, bool NEG, int ILP>
__global__ void __launch_bounds__(kThreads) k_phase(typename P::Amp* __restrict__ psi, uint64_t n_items,
                                                    DevInsert ins, typename P::Coef c) {
  using Amp = typename P::Amp;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; base < n_items; base += stride * ILP) {
    uint64_t ii[ILP];
    Amp a[ILP];
#pragma unroll
    for (int u = 0; u < ILP; ++u) {
      const uint64_t item = base + u * stride;
      if (item < n_items) {
        ii[u] = expand_index(item, ins);
        a[u] = psi[ii[u]];
      }
    }
#pragma unroll
    for (int u = 0; u < ILP; ++u) {
      const uint64_t item = base + u * stride;
      if (item < n_items) {
        if constexpr (NEG) {
          psi[ii[u]] = neg_amp(a[u]);
        } else {
          typename P::Val v = P::load(a[u]);
          psi[ii[u]] = P::template mac_round<1>(&c, &v);
        }
      }
    }
  }
}

// X: swap partners.  Y: up' = -i lo, lo' = i up (moves and sign flips only).
// The partner of index i is i ^ tbit: for X and Y tbit is the target bit (0
// in i); a transposition of two sub-register values p <-> q (SWAP) has i on
// p and tbit = the index bits where p and q differ.
template <class Amp, bool Y, int ILP>
__global__ void __launch_bounds__(kThreads) k_xy(Amp* __restrict__ psi, uint64_t n_items, uint64_t tbit,
                                                 DevInsert ins) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; base < n_items; base += stride * ILP) {
    uint64_t iu[ILP];
    Amp a[ILP], b[ILP];
#pragma unroll
    for (int u = 0; u < ILP; ++u) {
      const uint64_t item = base + u * stride;
      if (item < n_items) {
        iu[u] = expand_index(item, ins);
        a[u] = psi[iu[u]];
        b[u] = psi[iu[u] ^ tbit];
      }
    }
#pragma unroll
    for (int u = 0; u < ILP; ++u) {
      const uint64_t item = base + u * stride;
      if (item < n_items) {
        if constexpr (Y) {
          Amp up = b[u], lo = a[u];
          up.x = b[u].y;            // -i (x + iy) = y - ix
          up.y = neg_s(b[u].x);
          lo.x = neg_s(a[u].y);     //  i (x + iy) = -y + ix
          lo.y = a[u].x;
          psi[iu[u]] = up;
          psi[iu[u] ^ tbit] = lo;
        } else {
          psi[iu[u]] = b[u];
          psi[iu[u] ^ tbit] = a[u];
        }
      }
    }
  }
}

constexpr int kMaxDiag = 1 << QS_MAX_TARGETS;

template <class P>
struct DiagTable {
  int k;
  int targets[QS_MAX_TARGETS];
  typename P::Coef d[kMaxDiag];
};

template <class P, int ILP>
__global__ void __launch_bounds__(kThreads) k_diag(typename P::Amp* __restrict__ psi, uint64_t n_items,
                                                   DevInsert ins, const __grid_constant__ DiagTable<P> tab) {
  using Amp = typename P::Amp;
  using Coef = typename P::Coef;
  // Lanes read different entries: gathered from the parameter bank they
  // would serialise, so the table is staged in shared memory first.
  __shared__ __align__(16) unsigned char s_raw[sizeof(Coef) * kMaxDiag];
  Coef* s_d = reinterpret_cast<Coef*>(s_raw);
  for (int i = threadIdx.x; i < (1 << tab.k); i += blockDim.x) s_d[i] = tab.d[i];
  __syncthreads();
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; base < n_items; base += stride * ILP) {
    uint64_t ii[ILP];
    Amp a[ILP];
#pragma unroll
    for (int u = 0; u < ILP; ++u) {
      const uint64_t item = base + u * stride;
      if (item < n_items) {
        ii[u] = expand_index(item, ins);
        a[u] = psi[ii[u]];
      }
    }
#pragma unroll
    for (int u = 0; u < ILP; ++u) {
      const uint64_t item = base + u * stride;
      if (item < n_items) {
        uint32_t sidx = 0;
        for (int j = 0; j < tab.k; ++j) sidx |= (uint32_t)((ii[u] >> tab.targets[j]) & 1u) << j;
        typename P::Val v = P::load(a[u]);
        psi[ii[u]] = P::template mac_round<1>(&s_d[sidx], &v);
      }
    }
  }
}

// Permutation on k targets.  A CTA stages tile_groups whole groups (the 2^k
// amplitudes that share every non-target bit) in shared memory, then writes
// element s of each group to sub-register position perm[s].  Groups are the
// compressed index with target and control bits inserted, so consecutive
// threads touch consecutive addresses along the lowest free qubits.
struct PermTable {
  int k;
  uint32_t perm[kMaxDiag];
  uint64_t offset[kMaxDiag];  // sub-register value -> index bits on targets
};

template <class Amp>
__global__ void __launch_bounds__(kThreads) k_perm(Amp* __restrict__ psi, uint64_t n_groups, int log_tile_groups,
                                                   DevInsert ins, const __grid_constant__ PermTable tab) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Amp* tile = reinterpret_cast<Amp*>(smem_raw);
  const int sub = 1 << tab.k;
  const int G = 1 << log_tile_groups;
  const int elems = G * sub;
  for (uint64_t g0 = (uint64_t)blockIdx.x * G; g0 < n_groups; g0 += (uint64_t)gridDim.x * G) {
    for (int e = threadIdx.x; e < elems; e += blockDim.x) {
      const int g = e & (G - 1);
      const int sidx = e >> log_tile_groups;
      if (g0 + g < n_groups) tile[e] = psi[expand_index(g0 + g, ins) | tab.offset[sidx]];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < elems; e += blockDim.x) {
      const int g = e & (G - 1);
      const int sidx = e >> log_tile_groups;
      if (g0 + g < n_groups) psi[expand_index(g0 + g, ins) | tab.offset[tab.perm[sidx]]] = tile[e];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Launch helpers
// ---------------------------------------------------------------------------
static std::mutex g_occ_mu;
static std::unordered_map<const void*, int> g_occ;

template <class F>
static int resident_ctas(F kernel, int threads, size_t smem) {
  std::lock_guard<std::mutex> lk(g_occ_mu);
  auto it = g_occ.find((const void*)kernel);
  if (it != g_occ.end()) return it->second;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem) != cudaSuccess || occ < 1) occ = 1;
  g_occ[(const void*)kernel] = occ;
  return occ;
}

template <class F>
static unsigned grid_for(F kernel, uint64_t items, int ilp, int device, size_t smem = 0) {
  const uint64_t per_cta = (uint64_t)kThreads * ilp;
  const uint64_t need = (items + per_cta - 1) / per_cta;
  const uint64_t full = (uint64_t)sm_count(device) * resident_ctas(kernel, kThreads, smem);
  uint64_t g = need < full ? need : full;
  return (unsigned)(g < 1 ? 1 : g);
}

static qs_status after_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, what);
  return QS_OK;
}

static std::vector<int> with_ctrls(std::vector<int> pos, uint64_t ctrl_mask) {
  for (int q = 0; q < 64; ++q)
    if ((ctrl_mask >> q) & 1ull) pos.push_back(q);
  return pos;
}

static int popcount64(uint64_t x) { return __builtin_popcountll(x); }

template <class P>
static Mat2<P> mat2(const double* U) {
  Mat2<P> g;
  for (int j = 0; j < 4; ++j) g.m[j] = P::make_coef(U[2 * j], U[2 * j + 1]);
  return g;
}

template <class P>
static qs_status dense1_impl(qs_state s, int t, uint64_t ctrl_mask, const double* U) {
  constexpr int ILP = 2;
  const uint64_t items = 1ull << (s->n - 1 - popcount64(ctrl_mask));
  DevInsert ins = to_dev(make_insert(with_ctrls({t}, ctrl_mask), ctrl_mask));
  auto kern = k_dense1<P, ILP>;
  unsigned grid = grid_for(kern, items, ILP, s->device);
  kern<<<grid, kThreads, 0, s->stream>>>((typename P::Amp*)s->psi, items, 1ull << t, ins, mat2<P>(U));
  return after_launch("k_dense1");
}

qs_status launch_dense1(qs_state s, int target, uint64_t ctrl_mask, const double* U) {
  if (s->dtype == QS_C64) return dense1_impl<MathF32>(s, target, ctrl_mask, U);
  if (s->math == QS_MATH_FP64) return dense1_impl<MathF64>(s, target, ctrl_mask, U);
  return dense1_impl<MathDFGate>(s, target, ctrl_mask, U);
}

template <class P>
static qs_status dense2_impl(qs_state s, int t0, int t1, uint64_t ctrl_mask, const double* U) {
  constexpr int ILP = QS_DENSE2_ILP;
  const uint64_t items = 1ull << (s->n - 2 - popcount64(ctrl_mask));
  DevInsert ins = to_dev(make_insert(with_ctrls({t0, t1}, ctrl_mask), ctrl_mask));
  Mat4<P> g;
  for (int j = 0; j < 16; ++j) g.m[j] = P::make_coef(U[2 * j], U[2 * j + 1]);
  for (int r = 0; r < 4; ++r) g.row_exp[r] = row_exponent(U, r, 4);
  auto kern = k_dense2<P, ILP>;
  unsigned grid = grid_for(kern, items, ILP, s->device);
  kern<<<grid, kThreads, 0, s->stream>>>((typename P::Amp*)s->psi, items, 1ull << t0, 1ull << t1, ins, g);
  return after_launch("k_dense2");
}

qs_status launch_dense2(qs_state s, int t0, int t1, uint64_t ctrl_mask, const double* U) {
  if (s->dtype == QS_C64) return dense2_impl<MathF32>(s, t0, t1, ctrl_mask, U);
  if (s->math == QS_MATH_FP64) return dense2_impl<MathF64>(s, t0, t1, ctrl_mask, U);
  return dense2_impl<MathDFGate>(s, t0, t1, ctrl_mask, U);
}

template <class P>
static qs_status phase_impl(qs_state s, uint64_t mask, uint64_t pattern, double cre, double cim) {
  constexpr int ILP = 4;
  const uint64_t items = 1ull << (s->n - popcount64(mask));
  std::vector<int> pos;
  for (int q = 0; q < s->n; ++q)
    if ((mask >> q) & 1ull) pos.push_back(q);
  DevInsert ins = to_dev(make_insert(pos, pattern & mask));
  if (cre == -1.0 && cim == 0.0) {
    auto kern = k_phase<P, true, ILP>;
    unsigned grid = grid_for(kern, items, ILP, s->device);
    kern<<<grid, kThreads, 0, s->stream>>>((typename P::Amp*)s->psi, items, ins, P::make_coef(cre, cim));
  } else {
    auto kern = k_phase<P, false, ILP>;
    unsigned grid = grid_for(kern, items, ILP, s->device);
    kern<<<grid, kThreads, 0, s->stream>>>((typename P::Amp*)s->psi, items, ins, P::make_coef(cre, cim));
  }
  return after_launch("k_phase");
}

qs_status launch_phase(qs_state s, uint64_t mask, uint64_t pattern, double c_re, double c_im) {
  if (s->dtype == QS_C64) return phase_impl<MathF32>(s, mask, pattern, c_re, c_im);
  if (s->math == QS_MATH_FP64) return phase_impl<MathF64>(s, mask, pattern, c_re, c_im);
  return phase_impl<MathDFGate>(s, mask, pattern, c_re, c_im);
}

template <class Amp>
static qs_status xy_impl(qs_state s, int t, uint64_t ctrl_mask, int y) {
  constexpr int ILP = 2;
  const uint64_t items = 1ull << (s->n - 1 - popcount64(ctrl_mask));
  DevInsert ins = to_dev(make_insert(with_ctrls({t}, ctrl_mask), ctrl_mask));
  if (y) {
    auto kern = k_xy<Amp, true, ILP>;
    unsigned grid = grid_for(kern, items, ILP, s->device);
    kern<<<grid, kThreads, 0, s->stream>>>((Amp*)s->psi, items, 1ull << t, ins);
  } else {
    auto kern = k_xy<Amp, false, ILP>;
    unsigned grid = grid_for(kern, items, ILP, s->device);
    kern<<<grid, kThreads, 0, s->stream>>>((Amp*)s->psi, items, 1ull << t, ins);
  }
  return after_launch("k_xy");
}

// Exchange of the amplitudes whose sub-register on targets is p with those
// where it is q (all other bits equal, controls 1): reads and writes only the
// 2^(n - k - c + 1) amplitudes that move.
template <class Amp>
static qs_status pairswap_impl(qs_state s, const int* targets, int k, uint64_t ctrl_mask, uint32_t p, uint32_t q) {
  constexpr int ILP = 2;
  const uint64_t items = 1ull << (s->n - k - popcount64(ctrl_mask));
  uint64_t pbits = 0, qbits = 0;
  for (int j = 0; j < k; ++j) {
    if ((p >> j) & 1u) pbits |= 1ull << targets[j];
    if ((q >> j) & 1u) qbits |= 1ull << targets[j];
  }
  std::vector<int> pos(targets, targets + k);
  DevInsert ins = to_dev(make_insert(with_ctrls(pos, ctrl_mask), ctrl_mask | pbits));
  auto kern = k_xy<Amp, false, ILP>;
  unsigned grid = grid_for(kern, items, ILP, s->device);
  kern<<<grid, kThreads, 0, s->stream>>>((Amp*)s->psi, items, pbits ^ qbits, ins);
  return after_launch("k_xy");
}

qs_status launch_pairswap(qs_state s, const int* targets, int k, uint64_t ctrl_mask, uint32_t p, uint32_t q) {
  if (s->dtype == QS_C64) return pairswap_impl<float2>(s, targets, k, ctrl_mask, p, q);
  return pairswap_impl<double2>(s, targets, k, ctrl_mask, p, q);
}

qs_status launch_xy(qs_state s, int target, uint64_t ctrl_mask, int y) {
  if (s->dtype == QS_C64) return xy_impl<float2>(s, target, ctrl_mask, y);
  return xy_impl<double2>(s, target, ctrl_mask, y);
}

template <class P>
static qs_status diag_impl(qs_state s, const int* targets, int k, uint64_t ctrl_mask, const double* d) {
  constexpr int ILP = 2;
  const uint64_t items = 1ull << (s->n - popcount64(ctrl_mask));
  std::vector<int> pos;
  for (int q = 0; q < s->n; ++q)
    if ((ctrl_mask >> q) & 1ull) pos.push_back(q);
  DevInsert ins = to_dev(make_insert(pos, ctrl_mask));
  DiagTable<P> tab;
  std::memset(&tab, 0, sizeof(tab));
  tab.k = k;
  for (int j = 0; j < k; ++j) tab.targets[j] = targets[j];
  for (int v = 0; v < (1 << k); ++v) tab.d[v] = P::make_coef(d[2 * v], d[2 * v + 1]);
  auto kern = k_diag<P, ILP>;
  unsigned grid = grid_for(kern, items, ILP, s->device);
  kern<<<grid, kThreads, 0, s->stream>>>((typename P::Amp*)s->psi, items, ins, tab);
  return after_launch("k_diag");
}

qs_status launch_diag(qs_state s, const int* targets, int k, uint64_t ctrl_mask, const double* d) {
  if (s->dtype == QS_C64) return diag_impl<MathF32>(s, targets, k, ctrl_mask, d);
  if (s->math == QS_MATH_FP64) return diag_impl<MathF64>(s, targets, k, ctrl_mask, d);
  return diag_impl<MathDFGate>(s, targets, k, ctrl_mask, d);
}

template <class Amp>
static qs_status perm_impl(qs_state s, const int* targets, int k, uint64_t ctrl_mask, const uint32_t* perm) {
  const int log_tile_elems = 11;  // 2048 amplitudes staged per CTA
  const int log_g = log_tile_elems - k;
  const int nfree = s->n - k - popcount64(ctrl_mask);
  const int log_tile_groups = log_g < nfree ? log_g : nfree;
  const uint64_t n_groups = 1ull << nfree;
  std::vector<int> pos(targets, targets + k);
  pos = with_ctrls(pos, ctrl_mask);
  DevInsert ins = to_dev(make_insert(pos, ctrl_mask));
  PermTable tab;
  std::memset(&tab, 0, sizeof(tab));
  tab.k = k;
  for (int v = 0; v < (1 << k); ++v) {
    tab.perm[v] = perm[v];
    uint64_t off = 0;
    for (int j = 0; j < k; ++j)
      if ((v >> j) & 1) off |= 1ull << targets[j];
    tab.offset[v] = off;
  }
  const size_t smem = sizeof(Amp) << (log_tile_groups + k);
  auto kern = k_perm<Amp>;
  const uint64_t tiles = n_groups >> log_tile_groups;
  const uint64_t full = (uint64_t)sm_count(s->device) * resident_ctas(kern, kThreads, 32768);
  const unsigned grid = (unsigned)(tiles < full ? tiles : full);
  kern<<<grid < 1 ? 1 : grid, kThreads, smem, s->stream>>>((Amp*)s->psi, n_groups, log_tile_groups, ins, tab);
  return after_launch("k_perm");
}

qs_status launch_perm(qs_state s, const int* targets, int k, uint64_t ctrl_mask, const uint32_t* perm) {
  if (s->dtype == QS_C64) return perm_impl<float2>(s, targets, k, ctrl_mask, perm);
  return perm_impl<double2>(s, targets, k, ctrl_mask, perm);
}

// ---------------------------------------------------------------------------
// Classification and dispatch
// ---------------------------------------------------------------------------
static bool is_c(const double* z, double re, double im) { return z[0] == re && z[1] == im; }

qs_status dispatch_u1(qs_state s, int t, uint64_t ctrl_mask, const double* U) {
  const double *u00 = U, *u01 = U + 2, *u10 = U + 4, *u11 = U + 6;
  const uint64_t tb = 1ull << t;
  if (is_c(u01, 0, 0) && is_c(u10, 0, 0)) {  // diagonal
    if (is_c(u00, 1, 0) && is_c(u11, 1, 0)) return QS_OK;  // identity
    if (is_c(u00, 1, 0)) return launch_phase(s, ctrl_mask | tb, ctrl_mask | tb, u11[0], u11[1]);
    if (is_c(u11, 1, 0)) return launch_phase(s, ctrl_mask | tb, ctrl_mask, u00[0], u00[1]);
    const int tg[1] = {t};
    const double d[4] = {u00[0], u00[1], u11[0], u11[1]};
    return launch_diag(s, tg, 1, ctrl_mask, d);
  }
  if (is_c(u00, 0, 0) && is_c(u11, 0, 0)) {  // anti-diagonal
    if (is_c(u01, 1, 0) && is_c(u10, 1, 0)) return launch_xy(s, t, ctrl_mask, 0);
    if (is_c(u01, 0, -1) && is_c(u10, 0, 1)) return launch_xy(s, t, ctrl_mask, 1);
  }
  return launch_dense1(s, t, ctrl_mask, U);
}

qs_status dispatch_diag(qs_state s, const int* targets, int k, uint64_t ctrl_mask, const double* d) {
  // Entries equal to 1 need no work: one entry != 1 is a phase on a pattern.
  int n_other = 0, v_other = -1;
  for (int v = 0; v < (1 << k); ++v)
    if (!is_c(d + 2 * v, 1, 0)) {
      ++n_other;
      v_other = v;
    }
  if (n_other == 0) return QS_OK;
  if (n_other == 1) {
    uint64_t mask = ctrl_mask, pattern = ctrl_mask;
    for (int j = 0; j < k; ++j) {
      mask |= 1ull << targets[j];
      if ((v_other >> j) & 1) pattern |= 1ull << targets[j];
    }
    return launch_phase(s, mask, pattern, d[2 * v_other], d[2 * v_other + 1]);
  }
  return launch_diag(s, targets, k, ctrl_mask, d);
}

qs_status dispatch_perm(qs_state s, const int* targets, int k, uint64_t ctrl_mask, const uint32_t* perm) {
  bool ident = true;
  for (int v = 0; v < (1 << k); ++v) ident = ident && perm[v] == (uint32_t)v;
  if (ident) return QS_OK;
  if (k == 1) return launch_xy(s, targets[0], ctrl_mask, 0);
  // A single transposition p <-> q (SWAP is 01 <-> 10) moves only its pairs.
  int moved = 0;
  uint32_t mp = 0, mq = 0;
  for (int v = 0; v < (1 << k); ++v)
    if (perm[v] != (uint32_t)v) {
      if (moved == 0) mp = (uint32_t)v;
      if (moved == 1) mq = (uint32_t)v;
      ++moved;
    }
  if (moved == 2 && perm[mp] == mq && perm[mq] == mp) return launch_pairswap(s, targets, k, ctrl_mask, mp, mq);
  return launch_perm(s, targets, k, ctrl_mask, perm);
}

qs_status dispatch_uk(qs_state s, const int* targets, int k, uint64_t ctrl_mask, const double* M) {
  const int dim = 1 << k;
  bool diag = true, permlike = true;
  std::vector<uint32_t> perm(dim, 0);
  for (int c = 0; c < dim; ++c) {
    int ones = 0;
    for (int r = 0; r < dim; ++r) {
      const double* z = M + 2 * (r * dim + c);
      if (r != c && !is_c(z, 0, 0)) diag = false;
      if (is_c(z, 1, 0)) {
        ++ones;
        perm[c] = (uint32_t)r;
      } else if (!is_c(z, 0, 0)) {
        permlike = false;
      }
    }
    if (ones != 1) permlike = false;
  }
  if (diag) {
    std::vector<double> d(2 * dim);
    for (int v = 0; v < dim; ++v) {
      d[2 * v] = M[2 * (v * dim + v)];
      d[2 * v + 1] = M[2 * (v * dim + v) + 1];
    }
    return dispatch_diag(s, targets, k, ctrl_mask, d.data());
  }
  if (permlike) {
    std::vector<bool> seen(dim, false);
    bool bij = true;
    for (int c = 0; c < dim; ++c) {
      bij = bij && !seen[perm[c]];
      seen[perm[c]] = true;
    }
    if (bij) return dispatch_perm(s, targets, k, ctrl_mask, perm.data());
  }
  if (k == 1) return launch_dense1(s, targets[0], ctrl_mask, M);
  if (k == 2) return launch_dense2(s, targets[0], targets[1], ctrl_mask, M);
  if (k <= 5) return launch_dense_k(s, targets, k, ctrl_mask, M);
  return fail(QS_ERR_UNSUPPORTED, "dense gates on %d targets (at most 5)", k);
}

}  // namespace qs
