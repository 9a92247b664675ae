// Dense gates on 3..5 targets: every group of d = 2^k amplitudes that share
// their non-target bits (and have all controls 1) is multiplied by the
// 2^k x 2^k matrix U (Sec. II-B: a k-qubit gate acts as a 2^k x 2^k
// unitary on the index bits it targets; Algorithm 1 is the k = 1 case).
//
// Two kernels:
//
// k_dense_tc (complex64 states, k = 4 and 5 unless disabled): the
// fifth-generation tensor cores.  Over reals with (re, im) interleaved, the action on one
// group is y = R x with the 2d x 2d real matrix
//   R[2r][2c] = Re U[r][c],   R[2r][2c+1] = -Im U[r][c],
//   R[2r+1][2c] = Im U[r][c], R[2r+1][2c+1] = Re U[r][c],
// so a tile of 128 groups is one GEMM: D[128 x 2d] = A[128 x 2d] R^T.  The
// gate costs 8d real flops per amplitude (256 at k = 5), more than the FP32
// pipes deliver per byte of HBM traffic at k = 5.  TF32 keeps 11 significant
// bits, so every operand is split X = X_hi + X_lo (both rounded to TF32) and
// D = A_lo R_hi + A_hi R_lo + A_hi R_hi; the dropped A_lo R_lo is about
// 2^-24 of the result, so the error stays at FP32's level.
//
// k_dense_k (complex64 at k = 3 or on request, complex128 always): one thread per group
// on the CUDA cores, U in shared memory (broadcast reads), the d outputs as
// d-term FMA chains in FP32 (complex64) or FP64 (complex128).
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "qs_internal.h"
#include "qs_tile_dev.cuh"

namespace qs {

namespace {

// ---------------------------------------------------------------------------
// Shared host description of a dense gate's groups
// ---------------------------------------------------------------------------
struct DenseGeom {
  int k = 0, d = 0;
  int targets[5] = {0};
  uint64_t n_groups = 0;
  InsertSpec ins;          // zeros at targets and controls; controls set
  uint64_t offs[32] = {0};  // index bits of target sub-register value s
  std::vector<int> free_pos;  // lowest non-target, non-control positions (up to 7)
};

DenseGeom dense_geom(const qs_state s, const int* targets, int k, uint64_t ctrl_mask) {
  DenseGeom g;
  g.k = k;
  g.d = 1 << k;
  for (int j = 0; j < k; ++j) g.targets[j] = targets[j];
  std::vector<int> pos(targets, targets + k);
  uint64_t used = ctrl_mask;
  for (int j = 0; j < k; ++j) used |= 1ull << targets[j];
  for (int q = 0; q < 64; ++q)
    if ((ctrl_mask >> q) & 1ull) pos.push_back(q);
  g.ins = make_insert(pos, ctrl_mask);
  g.n_groups = 1ull << (s->n - (int)pos.size());
  for (int v = 0; v < g.d; ++v) {
    uint64_t o = 0;
    for (int j = 0; j < k; ++j)
      if ((v >> j) & 1) o |= 1ull << targets[j];
    g.offs[v] = o;
  }
  for (int q = 0; q < s->n && (int)g.free_pos.size() < 7; ++q)
    if (!((used >> q) & 1ull)) g.free_pos.push_back(q);
  return g;
}

// Round a float to the nearest TF32 value (ties away from zero): keep the
// sign, the exponent and the top 10 mantissa bits.
float tf32_round_host(float x) {
  uint32_t b;
  std::memcpy(&b, &x, 4);
  b = (b + 0x1000u) & 0xFFFFE000u;
  float r;
  std::memcpy(&r, &b, 4);
  return r;
}

// ---------------------------------------------------------------------------
// Tensor-core kernel
// ---------------------------------------------------------------------------
constexpr int kTcRows = 128;     // groups per tile: the MMA's M
constexpr int kTcThreads = 256;  // 8 warps gather and scatter; warps 0-3 read the accumulator

// The host orders the targets by position (and permutes U to match), so bit
// 0 of the sub-register value s is the lowest target: the amplitudes s and
// s + 1 of a group are the columns 4j..4j+3 of its A row, one 16-byte chunk.
// Each thread moves such pairs.  A tile's pairs are numbered by a local index
// whose bits are the other target bits and up to 7 row bits, in ascending
// address order: thread tid takes pairs tid + 256 i, its bits 0-7 mapped by
// lam_addr / lam_sr, i by the step tables; each maps to address bits and to
// (row, s), packed as row << 8 | s.
struct TcParams {
  uint64_t n_tiles;
  int rb;      // row bits of a tile: 7, fewer when the state has fewer groups
  int npairs;  // pairs in a tile: 2^(k - 1 + rb)
  int npos;
  int pair_vec;       // the lowest target is qubit 0: a pair is 16 contiguous bytes
  uint64_t pair_bit;  // address bit of s bit 0
  uint64_t high_mask[QS_MAX_QUBITS];
  uint64_t fixed_mask;
  uint64_t lam_addr[8];
  uint32_t lam_sr[8];
  uint64_t step_addr[8];
  uint32_t step_sr[8];
  float u_hi[2 * 32 * 32];  // U (targets in position order) as (re, im), rounded to TF32
  float u_lo[2 * 32 * 32];  // U - u_hi, rounded to TF32
  uint64_t wait_ns;
};
static_assert(sizeof(TcParams) < 30000, "kernel parameter space");

// Operands in the K-major layout with the 128-byte swizzle: a row's K = 32
// TF32 values of one atom column are 128 bytes, 8 rows make a 1024-byte atom,
// and 16-byte chunk j of row r sits at chunk j ^ (r % 8).  K = 64 takes two
// atom columns, each all rows deep.
template <int KQ>
struct TcShape {
  static constexpr int D = 1 << KQ;
  static constexpr int K = 2 * D;  // reals per row; the MMA's N and K
  static_assert(K == 32 || K == 64, "whole 128-byte swizzle atoms along K");
  static constexpr int kAtomsK = K / 32;
  static constexpr uint32_t kABytes = kTcRows * K * 4;  // one A operand
  static constexpr uint32_t kBBytes = K * K * 4;        // one B operand
  static constexpr uint32_t kOffAlo = kABytes;
  static constexpr uint32_t kOffBhi = 2 * kABytes;
  static constexpr uint32_t kOffBlo = 2 * kABytes + kBBytes;
  static constexpr uint32_t kOffBar = 2 * kABytes + 2 * kBBytes;
  static constexpr uint32_t kSmem = kOffBar + 32;
  static constexpr uint32_t kCols = (uint32_t)K;           // TMEM columns (power of two >= 32)
  static constexpr int kStageStride = D + 2;               // float2 per staged row (16-byte rows, padded)
  static constexpr int kPairs = kTcRows * D / 2 / kTcThreads;  // pairs per thread per tile
  static_assert(kTcRows * kStageStride * 8 <= 2 * kABytes, "output stage fits the A operands");
  static_assert(kPairs <= 8, "step tables");
};

// Byte offset of element (row, col) of a swizzled K-major operand of `rows`
// rows.
__device__ __forceinline__ uint32_t sw128_off(int row, int col, int rows) {
  return (uint32_t)((col >> 5) * rows * 128 + row * 128 + ((((col & 31) >> 2) ^ (row & 7)) << 4) + (col & 3) * 4);
}

// Shared-memory matrix descriptor for the swizzled K-major layout: start
// address, leading byte offset 16 (unused with this swizzle), stride byte
// offset 1024 (between 8-row atoms), descriptor version 1, layout type 2
// (128-byte swizzle).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
         (2ull << 61);
}

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive accumulator columns of this thread's lane.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ uint64_t tile_base(uint64_t tile, const TcParams& p) {
  uint64_t g = tile << p.rb;
  for (int j = 0; j < p.npos; ++j) g += g & p.high_mask[j];
  return g | p.fixed_mask;
}

// One CTA per tile at a time (persistent over tiles): gather the tile's
// groups into the A operands (split into TF32 head and remainder), one
// thread issues the MMAs and commits them to an mbarrier, the next tile's
// amplitudes are loaded while they run, then warps 0-3 read the accumulator
// rows (lane = row) into a padded staging area and all threads scatter it.
template <int KQ>
__global__ void __launch_bounds__(kTcThreads, 2)
    k_dense_tc(float2* __restrict__ psi, const __grid_constant__ TcParams p, uint32_t* __restrict__ err) {
  using S = TcShape<KQ>;
  constexpr int D = S::D, K = S::K, E = S::kPairs;
  // The swizzle follows address bits 4-9, so the operands start on
  // 1024-byte boundaries.  The dynamic shared memory (no static shared
  // memory here) starts on one; were it not, the kernel records device
  // error code 3 and returns before touching memory.  No padding is
  // allocated for it: 64 more bytes per CTA would leave room for one CTA
  // per SM instead of two.
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5;
  if (smem_addr(smem) & 1023u) {
    if (tid == 0) atomicCAS(err, 0u, 3u);
    return;
  }
  const uint32_t base = smem_addr(smem);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + S::kOffBar);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + S::kOffBar + 16);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                 "n"(S::kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  // Zero the A operands (rows beyond a small state's groups stay zero) and
  // build R's TF32 parts (the B operand: N = K rows, K-major).
  for (uint32_t o = (uint32_t)tid * 16u; o < 2 * S::kABytes; o += kTcThreads * 16u)
    *reinterpret_cast<float4*>(smem + o) = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int e = tid; e < K * K; e += kTcThreads) {
    const int row = e / K, col = e % K;
    const int ui = 2 * ((row >> 1) * D + (col >> 1));
    float h, l;
    if ((row & 1) == (col & 1)) {  // Re U
      h = p.u_hi[ui];
      l = p.u_lo[ui];
    } else if ((row & 1) == 0) {  // -Im U
      h = -p.u_hi[ui + 1];
      l = -p.u_lo[ui + 1];
    } else {  // Im U
      h = p.u_hi[ui + 1];
      l = p.u_lo[ui + 1];
    }
    const uint32_t off = sw128_off(row, col, K);
    *reinterpret_cast<float*>(smem + S::kOffBhi + off) = h;
    *reinterpret_cast<float*>(smem + S::kOffBlo + off) = l;
  }
  // This thread's part of every tile-local pair index.
  uint64_t a_t = 0;
  uint32_t sr_t = 0;
#pragma unroll
  for (int b = 0; b < 8; ++b)
    if ((tid >> b) & 1) {
      a_t |= p.lam_addr[b];
      sr_t |= p.lam_sr[b];
    }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  // Instruction descriptor: FP32 accumulator (bits 4-5 = 1), TF32 A and B
  // (bits 7-9, 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at bit 17,
  // M >> 4 at bit 24.
  constexpr uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(K >> 3) << 17) |
                             ((uint32_t)(kTcRows >> 4) << 24);
  float4* stage = reinterpret_cast<float4*>(smem);  // row r: (D + 2) / 2 float4, pairs (s, s + 1)
  constexpr int kStage4 = S::kStageStride / 2;

  float4 x[E];
  auto load_tile = [&](uint64_t t) {
    const uint64_t tb = tile_base(t, p) | a_t;
#pragma unroll
    for (int i = 0; i < E; ++i)
      if (tid + i * kTcThreads < p.npairs) {
        const uint64_t a = tb | p.step_addr[i];
        if (p.pair_vec) {
          x[i] = *reinterpret_cast<const float4*>(psi + a);
        } else {
          const float2 u = psi[a], v = psi[a | p.pair_bit];
          x[i] = make_float4(u.x, u.y, v.x, v.y);
        }
      }
  };

  uint64_t tile = blockIdx.x;
  if (tile < p.n_tiles) load_tile(tile);
  uint32_t phase = 0;
  for (; tile < p.n_tiles; tile += gridDim.x) {
#pragma unroll
    for (int i = 0; i < E; ++i)
      if (tid + i * kTcThreads < p.npairs) {
        const uint32_t sr = sr_t | p.step_sr[i];
        const uint32_t off = sw128_off((int)(sr >> 8), 2 * (int)(sr & 0xFFu), kTcRows);
        const float4 h = make_float4(tf32_round(x[i].x), tf32_round(x[i].y), tf32_round(x[i].z), tf32_round(x[i].w));
        *reinterpret_cast<float4*>(smem + off) = h;
        *reinterpret_cast<float4*>(smem + S::kOffAlo + off) =
            make_float4(tf32_round(x[i].x - h.x), tf32_round(x[i].y - h.y), tf32_round(x[i].z - h.z),
                        tf32_round(x[i].w - h.w));
      }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
      // Three products, small ones first; K / 8 MMAs of K-depth 8 (32 bytes
      // of a 128-byte swizzled row) each.
      uint32_t acc = 0;
#pragma unroll
      for (int prod = 0; prod < 3; ++prod) {
        const uint32_t a = base + (prod == 0 ? S::kOffAlo : 0u);
        const uint32_t b = base + (prod == 1 ? S::kOffBlo : S::kOffBhi);
#pragma unroll
        for (int ks = 0; ks < K / 8; ++ks) {
          const uint32_t within = (uint32_t)(ks & 3) * 32u, atom = (uint32_t)(ks >> 2);
          tc_mma(tmem, smem_desc_sw128(a + atom * (kTcRows * 128u) + within),
                 smem_desc_sw128(b + atom * (uint32_t)(K * 128) + within), idesc, acc);
          acc = 1;
        }
      }
      tc_commit(smem_addr(bar));
    }
    const uint64_t next = tile + gridDim.x;
    if (next < p.n_tiles) load_tile(next);
    // Bounded wait for the MMAs by warp 0 (the others wait at the barrier
    // without taking issue slots); on expiry every thread agrees, and thread
    // 0 drains the MMAs still in flight (they read and write this CTA's own
    // memory and complete) before the accumulator is freed.
    bool done = true;
    if (warp == 0) {
      done = mbar_try(bar, phase);
      if (!done) {
        const uint64_t t0 = global_ns();
        while (!(done = mbar_try(bar, phase)))
          if (global_ns() - t0 > p.wait_ns) break;
      }
    }
    if (__syncthreads_or(!done)) {
      if (tid == 0) {
        atomicCAS(err, 0u, 1u);
        const uint64_t t0 = global_ns();
        while (!mbar_try(bar, phase) && global_ns() - t0 < kDrainNs) {
        }
      }
      break;
    }
    phase ^= 1u;
    tc_fence_after();
    if (warp < 4) {
      const int row = warp * 32 + (tid & 31);
      const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
      for (int c0 = 0; c0 < K; c0 += 16) {
        float v[16];
        tc_ld16(lane_addr + (uint32_t)c0, v);
#pragma unroll
        for (int j = 0; j < 4; ++j)
          stage[row * kStage4 + (c0 >> 2) + j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
      }
    }
    tc_fence_before();
    __syncthreads();
    {
      const uint64_t tb = tile_base(tile, p) | a_t;
#pragma unroll
      for (int i = 0; i < E; ++i)
        if (tid + i * kTcThreads < p.npairs) {
          const uint32_t sr = sr_t | p.step_sr[i];
          const float4 v = stage[(int)(sr >> 8) * kStage4 + (int)((sr & 0xFFu) >> 1)];
          const uint64_t a = tb | p.step_addr[i];
          if (p.pair_vec) {
            *reinterpret_cast<float4*>(psi + a) = v;
          } else {
            psi[a] = make_float2(v.x, v.y);
            psi[a | p.pair_bit] = make_float2(v.z, v.w);
          }
        }
    }
    __syncthreads();
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(S::kCols) : "memory");
  }
}

// ---------------------------------------------------------------------------
// CUDA-core kernel
// ---------------------------------------------------------------------------
template <typename T>
struct Cplx;
template <>
struct Cplx<float> {
  using V = float2;
};
template <>
struct Cplx<double> {
  using V = double2;
};

template <typename T, int KQ>
struct DenseKParams {
  uint64_t n_groups;
  int npos;
  uint64_t high_mask[QS_MAX_QUBITS];
  uint64_t fixed_mask;
  uint64_t offs[1 << KQ];
  T u[2 << (2 * KQ)];  // U row-major, (re, im) pairs
};

template <typename T, int KQ>
__global__ void __launch_bounds__(128)
    k_dense_k(typename Cplx<T>::V* __restrict__ psi, const __grid_constant__ DenseKParams<T, KQ> p) {
  using V = typename Cplx<T>::V;
  constexpr int D = 1 << KQ;
  // U in shared memory, read by every thread at the same address (a
  // broadcast): 16 bytes per load, two complex coefficients in FP32.
  __shared__ __align__(16) T us[2 * D * D];
  for (int i = threadIdx.x; i < 2 * D * D; i += blockDim.x) us[i] = p.u[i];
  __syncthreads();
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < p.n_groups; g += stride) {
    uint64_t b = g;
    for (int j = 0; j < p.npos; ++j) b += b & p.high_mask[j];
    b |= p.fixed_mask;
    V x[D];
#pragma unroll
    for (int c = 0; c < D; ++c) x[c] = psi[b | p.offs[c]];
#pragma unroll 1
    for (int r = 0; r < D; ++r) {
      T re = 0, im = 0;
      const T* ur = us + 2 * r * D;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const T u_re = ur[2 * c], u_im = ur[2 * c + 1];
        re = fma(u_re, x[c].x, re);
        re = fma(-u_im, x[c].y, re);
        im = fma(u_re, x[c].y, im);
        im = fma(u_im, x[c].x, im);
      }
      V y;
      y.x = re;
      y.y = im;
      psi[b | p.offs[r]] = y;
    }
  }
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
template <typename T, int KQ>
qs_status launch_cuda_core(qs_state s, const DenseGeom& g, const double* U) {
  using V = typename Cplx<T>::V;
  constexpr int D = 1 << KQ;
  static thread_local DenseKParams<T, KQ> p;
  std::memset(&p, 0, sizeof(p));
  p.n_groups = g.n_groups;
  p.npos = g.ins.npos;
  for (int j = 0; j < QS_MAX_QUBITS; ++j) p.high_mask[j] = g.ins.high_mask[j];
  p.fixed_mask = g.ins.fixed_mask;
  for (int v = 0; v < D; ++v) p.offs[v] = g.offs[v];
  for (int i = 0; i < 2 * D * D; ++i) p.u[i] = (T)U[i];
  const uint64_t blocks = (g.n_groups + 127) / 128;
  const uint64_t cap = (uint64_t)sm_count(s->device) * 16;
  const unsigned grid = (unsigned)(blocks < cap ? blocks : cap);
  k_dense_k<T, KQ><<<grid, 128, 0, s->stream>>>((V*)s->psi, p);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

template <int KQ>
qs_status launch_tensor_core(qs_state s, const DenseGeom& g, const double* U) {
  using S = TcShape<KQ>;
  constexpr int D = 1 << KQ;
  static thread_local TcParams p;
  std::memset(&p, 0, sizeof(p));
  const int rb = (int)g.free_pos.size();
  p.rb = rb;
  p.npairs = 1 << (KQ - 1 + rb);
  p.n_tiles = g.n_groups >> rb;
  p.npos = g.ins.npos;
  for (int j = 0; j < QS_MAX_QUBITS; ++j) p.high_mask[j] = g.ins.high_mask[j];
  p.fixed_mask = g.ins.fixed_mask;
  // Targets in position order: bit j of the kernel's sub-register value is
  // target order[j] of the caller's, and U is permuted to match.
  int order[5];
  for (int j = 0; j < KQ; ++j) order[j] = j;
  std::sort(order, order + KQ, [&](int a, int b) { return g.targets[a] < g.targets[b]; });
  auto user_index = [&](int v) {
    int u = 0;
    for (int j = 0; j < KQ; ++j)
      if ((v >> j) & 1) u |= 1 << order[j];
    return u;
  };
  p.pair_bit = 1ull << g.targets[order[0]];
  p.pair_vec = g.targets[order[0]] == 0 ? 1 : 0;
  // Pair-index bits in ascending address order: sorted targets 1..k-1 map
  // to s bits 1..k-1, the r-th lowest free position to row bit r.
  std::vector<std::pair<int, uint32_t>> bits;
  for (int j = 1; j < KQ; ++j) bits.push_back({g.targets[order[j]], 1u << j});
  for (int r = 0; r < rb; ++r) bits.push_back({g.free_pos[r], (1u << r) << 8});
  std::sort(bits.begin(), bits.end());
  for (int b = 0; b < (int)bits.size() && b < 8; ++b) {
    p.lam_addr[b] = 1ull << bits[b].first;
    p.lam_sr[b] = bits[b].second;
  }
  for (int i = 0; i < 8; ++i)
    for (int b = 8; b < (int)bits.size(); ++b)
      if ((i >> (b - 8)) & 1) {
        p.step_addr[i] |= 1ull << bits[b].first;
        p.step_sr[i] |= bits[b].second;
      }
  for (int r = 0; r < D; ++r)
    for (int c = 0; c < D; ++c)
      for (int part = 0; part < 2; ++part) {
        const double u = U[2 * (user_index(r) * D + user_index(c)) + part];
        const float h = tf32_round_host((float)u);
        p.u_hi[2 * (r * D + c) + part] = h;
        p.u_lo[2 * (r * D + c) + part] = tf32_round_host((float)(u - (double)h));
      }
  p.wait_ns = wait_limit_ns();
  uint32_t* err = error_word(s);
  if (!err) return fail(QS_ERR_CUDA, "device error word unavailable");
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [] {
    attr_err = cudaFuncSetAttribute(k_dense_tc<KQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::kSmem);
    // All of the unified L1 / shared array as shared memory: two CTAs per SM
    // at k = 5 (the default split leaves room for one).
    if (attr_err == cudaSuccess)
      attr_err = cudaFuncSetAttribute(k_dense_tc<KQ>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared);
  });
  if (attr_err != cudaSuccess) return cuda_fail(attr_err, "k_dense_tc set-up");
  // Two CTAs per SM: the launch bounds keep the registers within half the
  // file and two copies of the shared memory fit (the grid-stride loop over
  // tiles stays correct with fewer resident).
  const uint64_t cap = (uint64_t)sm_count(s->device) * 2;
  const unsigned grid = (unsigned)(p.n_tiles < cap ? p.n_tiles : cap);
  k_dense_tc<KQ><<<grid, kTcThreads, S::kSmem, s->stream>>>((float2*)s->psi, p, err);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

}  // namespace

// Dense (not diagonal, not a permutation) gate on 3..5 targets under
// ctrl_mask, already validated.
qs_status launch_dense_k(qs_state s, const int* targets, int k, uint64_t ctrl_mask, const double* U) {
  if (k < 3 || k > 5) return fail(QS_ERR_UNSUPPORTED, "dense gates on %d targets (at most 5)", k);
  const DenseGeom g = dense_geom(s, targets, k, ctrl_mask);
  // The tensor cores take k = 4, 5 (rows of whole 128-byte swizzle atoms);
  // at k = 3 the FP32 CUDA cores already keep up with HBM.
  if (s->dtype == QS_C64 && s->tensor_cores && k >= 4) {
    if (k == 4) return launch_tensor_core<4>(s, g, U);
    return launch_tensor_core<5>(s, g, U);
  }
  if (s->dtype == QS_C64) {
    if (k == 3) return launch_cuda_core<float, 3>(s, g, U);
    if (k == 4) return launch_cuda_core<float, 4>(s, g, U);
    return launch_cuda_core<float, 5>(s, g, U);
  }
  if (k == 3) return launch_cuda_core<double, 3>(s, g, U);
  if (k == 4) return launch_cuda_core<double, 4>(s, g, U);
  return launch_cuda_core<double, 5>(s, g, U);
}

}  // namespace qs
