// Dense gates on 3..5 targets: every group of d = 2^k amplitudes that share
// their non-target bits (and have all controls 1) is multiplied by the
// 2^k x 2^k matrix U.  The paper applies a gate as an in-place
// matrix-vector multiplication (Sec. II-C, Fig. 3) with kernels for one and
// two targets (Algorithm 1 is the one-target case); a gate on k targets is
// the same product with the 2^k x 2^k matrix on the index bits it targets.
//
// Two kernels:
//
// k_dense_tc (complex64 states, as the state's tensor-core mode selects; 3
// and 4 targets run as the 5-target gate I (x) U on free qubits): the
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
// k_dense_k (complex64 where the mode selects it, complex128 in FP64
// arithmetic): one thread per group on the CUDA cores, U in shared memory
// (broadcast reads), the d outputs as d-term FMA chains in FP32 or FP64.
//
// k_dense_df (complex128 in float-float arithmetic, the default): one lane
// per output row, inputs split to float-float once and shared through shared
// memory, each row an anchored float-float accumulation.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "qs_internal.h"
#include "qs_math.cuh"
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
constexpr int kTcRows = 128;  // groups per tile: the MMA's M
// Warp roles: 0-7 read the accumulator and store (warp w reads TMEM lane
// quarter w % 4, column half w / 4), 8-23 load and split amplitudes into the
// A stages, 24 issues the MMAs (one thread).  The register file is four 16K
// partitions (one per SM sub-partition); 25 warps leave 72 registers a
// thread, enough for a producer to hold two tiles of loads in flight.
constexpr int kTcEpiWarps = 8, kTcProdWarps = 16;
constexpr int kTcEpiThreads = 32 * kTcEpiWarps, kTcProdThreads = 32 * kTcProdWarps;
constexpr int kTcMmaWarp = kTcEpiWarps + kTcProdWarps;
constexpr int kTcThreads = 32 * (kTcMmaWarp + 1);

// The host orders the targets by position (and permutes U to match), so bit
// 0 of the sub-register value s is the lowest target: the amplitudes s and
// s + 1 of a group are the columns 4j..4j+3 of its A row, one 16-byte chunk.
// Threads move such pairs.  A tile's pairs are numbered by a local index whose
// bits are the other target bits and up to 7 row bits, in ascending address
// order.  Producer thread t takes pairs t + 512 i (t's bits 0-8 mapped by
// prod_*, i by prod_step_*), epilogue thread t pairs t + 256 i (bits 0-7 by
// lam_*, i by step_*); each maps to address bits and to (row, s), packed as
// row << 8 | s.
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
  uint64_t prod_addr[9];
  uint32_t prod_sr[9];
  uint64_t prod_step_addr[4];
  uint32_t prod_step_sr[4];
  float u_hi[2 * 32 * 32];  // U (targets in position order) as (re, im), rounded to TF32
  float u_lo[2 * 32 * 32];  // U - u_hi, rounded to TF32
  uint64_t wait_ns;
};
static_assert(sizeof(TcParams) < 30000, "kernel parameter space");

// Operands in the K-major layout with the 128-byte swizzle: a row's K = 32
// TF32 values of one atom column are 128 bytes, 8 rows make a 1024-byte atom,
// and 16-byte chunk j of row r sits at chunk j ^ (r % 8).  K = 64 takes two
// atom columns, each all rows deep.  Two A stages and two TMEM accumulators;
// the output stage is the epilogue's own.
template <int KQ>
struct TcShape {
  static constexpr int D = 1 << KQ;
  static constexpr int K = 2 * D;  // reals per row; the MMA's N and K
  static_assert(K == 32 || K == 64, "whole 128-byte swizzle atoms along K");
  static constexpr uint32_t kABytes = kTcRows * K * 4;  // one A operand
  static constexpr uint32_t kBBytes = K * K * 4;        // one B operand
  static constexpr uint32_t kStageA = 2 * kABytes;      // head + remainder of one stage
  static constexpr uint32_t kOffBhi = 2 * kStageA;
  static constexpr uint32_t kOffBlo = kOffBhi + kBBytes;
  static constexpr int kStageStride = D + 2;  // float2 per staged output row (16-byte rows, padded)
  static constexpr uint32_t kOffOut = kOffBlo + kBBytes;
  static constexpr uint32_t kOffBar = kOffOut + kTcRows * kStageStride * 8;  // 8 mbarriers
  static constexpr uint32_t kSmem = kOffBar + 80;                            // + TMEM address slot
  static constexpr uint32_t kCols = 2 * (uint32_t)K;  // TMEM: two accumulators (power of two >= 32)
  static constexpr int kProdPairs = kTcRows * D / 2 / kTcProdThreads;  // per producer thread per tile
  static constexpr int kEpiPairs = kTcRows * D / 2 / kTcEpiThreads;    // per epilogue thread per tile
  static_assert(kTcProdThreads == 512 && kTcEpiThreads == 256, "index tables");
  static_assert(kProdPairs >= 1 && kProdPairs <= 4 && kEpiPairs <= 8, "step tables");
  static_assert(kSmem <= 227 * 1024, "shared memory per CTA");
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

// Round to the nearest TF32 value (ties away from zero) with two integer
// operations: add half of the dropped 13 bits' range to the magnitude, then
// clear them (finite inputs far below FLT_MAX).
__device__ __forceinline__ float tf32_round(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
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

// Group-wide barrier and AND-reduction among the epilogue warps (named
// barrier 1, 256 threads).
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kTcEpiThreads) : "memory"); }
__device__ __forceinline__ bool epi_all(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(kTcEpiThreads)
      : "memory");
  return r != 0;
}

// Persistent over tiles (tile j of this CTA: blockIdx.x + j gridDim.x),
// warp-specialized, with mbarriers between the roles and no CTA-wide
// barrier in the loop:
//   producers  wait empty[s], split the amplitudes held in registers into A
//              stage s, arrive on full[s], then load tile j + 2 into
//              registers (tile j + 1's loads are in flight meanwhile);
//   MMA thread waits full[s] and acc_empty[s], issues the three TF32
//              products into accumulator s, commits to empty[s] and
//              acc_full[s];
//   epilogue   waits acc_full[s], reads its half rows (lane = row), arrives
//              on acc_empty[s], and stores the rows through the output
//              stage (in address order);
// with s = j % 2.  Every wait is bounded: on expiry (or once another thread
// recorded an error) a role leaves its loop and the others' waits then run
// out too; the MMA thread waits (bounded) for its last commit so that no MMA
// is in flight, and the accumulator is freed after the final barrier.
template <int KQ>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_dense_tc(float2* __restrict__ psi, const __grid_constant__ TcParams p, uint32_t* __restrict__ err) {
  using S = TcShape<KQ>;
  constexpr int D = S::D, K = S::K;
  // The swizzle follows address bits 4-9, so the operands start on
  // 1024-byte boundaries.  The dynamic shared memory (no static shared
  // memory here) starts on one; were it not, the kernel records device
  // error code 3 and returns before touching memory.
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (smem_addr(smem) & 1023u) {
    if (tid == 0) atomicCAS(err, 0u, 3u);
    return;
  }
  const uint32_t base = smem_addr(smem);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S::kOffBar);
  uint64_t* empty = full + 2;
  uint64_t* acc_full = full + 4;
  uint64_t* acc_empty = full + 6;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + S::kOffBar + 64);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                 "n"(S::kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int st = 0; st < 2; ++st) {
      mbar_init(full + st, kTcProdThreads);
      mbar_init(empty + st, 1);
      mbar_init(acc_full + st, 1);
      mbar_init(acc_empty + st, kTcEpiThreads);
    }
    mbar_fence_init();
  }
  // Zero both A stages (rows beyond a small state's groups stay zero) and
  // build R's TF32 parts (the B operand: N = K rows, K-major).
  for (uint32_t o = (uint32_t)tid * 16u; o < 2 * S::kStageA; o += kTcThreads * 16u)
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
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint64_t stride = gridDim.x;

  if (warp >= kTcEpiWarps && warp < kTcMmaWarp) {
    // ---- producers ----
    constexpr int E = S::kProdPairs;
    const int t = tid - kTcEpiThreads;
    uint64_t a_t = 0;
    uint32_t sr_t = 0;
#pragma unroll
    for (int b = 0; b < 9; ++b)
      if ((t >> b) & 1) {
        a_t |= p.prod_addr[b];
        sr_t |= p.prod_sr[b];
      }
    // Two tiles in registers: tile j is split into its stage while tile
    // j + 1's loads are in flight; then tile j + 2's loads are issued.
    float4 xa[E], xb[E];
    auto load_tile = [&](float4(&x)[E], uint64_t tl) {
      const uint64_t tb = tile_base(tl, p) | a_t;
#pragma unroll
      for (int i = 0; i < E; ++i)
        if (t + i * kTcProdThreads < p.npairs) {
          const uint64_t a = tb | p.prod_step_addr[i];
          if (p.pair_vec) {
            x[i] = *reinterpret_cast<const float4*>(psi + a);
          } else {
            const float2 u = psi[a], v = psi[a | p.pair_bit];
            x[i] = make_float4(u.x, u.y, v.x, v.y);
          }
        }
    };
    auto put = [&](const float4(&x)[E], uint32_t j) -> bool {
      const int st = (int)(j & 1u);
      if (!mbar_wait(empty + st, ((j >> 1) & 1u) ^ 1u, err, p.wait_ns)) return false;
      unsigned char* a_hi = smem + st * S::kStageA;
#pragma unroll
      for (int i = 0; i < E; ++i)
        if (t + i * kTcProdThreads < p.npairs) {
          const uint32_t sr = sr_t | p.prod_step_sr[i];
          const uint32_t off = sw128_off((int)(sr >> 8), 2 * (int)(sr & 0xFFu), kTcRows);
          const float4 h =
              make_float4(tf32_round(x[i].x), tf32_round(x[i].y), tf32_round(x[i].z), tf32_round(x[i].w));
          *reinterpret_cast<float4*>(a_hi + off) = h;
          *reinterpret_cast<float4*>(a_hi + S::kABytes + off) =
              make_float4(tf32_round(x[i].x - h.x), tf32_round(x[i].y - h.y), tf32_round(x[i].z - h.z),
                          tf32_round(x[i].w - h.w));
        }
      fence_async_smem();
      mbar_arrive(full + st);
      return true;
    };
    uint64_t tile = blockIdx.x;
    if (tile < p.n_tiles) load_tile(xa, tile);
    if (tile + stride < p.n_tiles) load_tile(xb, tile + stride);
    for (uint32_t j = 0; tile < p.n_tiles; j += 2, tile += 2 * stride) {
      if (!put(xa, j)) break;
      if (tile + 2 * stride < p.n_tiles) load_tile(xa, tile + 2 * stride);
      if (tile + stride >= p.n_tiles) break;
      if (!put(xb, j + 1)) break;
      if (tile + 3 * stride < p.n_tiles) load_tile(xb, tile + 3 * stride);
    }
    __syncwarp();
  } else if (warp == kTcMmaWarp) {
    // ---- MMA issue (one thread) ----
    if (lane == 0) {
      // Instruction descriptor: FP32 accumulator (bits 4-5 = 1), TF32 A and
      // B (bits 7-9, 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at
      // bit 17, M >> 4 at bit 24.
      constexpr uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(K >> 3) << 17) |
                                 ((uint32_t)(kTcRows >> 4) << 24);
      int last = -1;  // accumulator of the last commit
      uint32_t last_parity = 0;
      uint64_t tile = blockIdx.x;
      for (uint32_t j = 0; tile < p.n_tiles; ++j, tile += stride) {
        const int st = (int)(j & 1u);
        const uint32_t parity = (j >> 1) & 1u;
        if (!mbar_wait(full + st, parity, err, p.wait_ns)) break;
        if (!mbar_wait(acc_empty + st, parity ^ 1u, err, p.wait_ns)) break;
        tc_fence_after();
        // Three products, small ones first; K / 8 MMAs of K-depth 8 (32
        // bytes of a 128-byte swizzled row) each.
        uint32_t acc = 0;
        const uint32_t d_tmem = tmem + (uint32_t)(st * K);
#pragma unroll
        for (int prod = 0; prod < 3; ++prod) {
          const uint32_t a = base + (uint32_t)st * S::kStageA + (prod == 0 ? S::kABytes : 0u);
          const uint32_t b = base + (prod == 1 ? S::kOffBlo : S::kOffBhi);
#pragma unroll
          for (int ks = 0; ks < K / 8; ++ks) {
            const uint32_t within = (uint32_t)(ks & 3) * 32u, atom = (uint32_t)(ks >> 2);
            tc_mma(d_tmem, smem_desc_sw128(a + atom * (kTcRows * 128u) + within),
                   smem_desc_sw128(b + atom * (uint32_t)(K * 128) + within), idesc, acc);
            acc = 1;
          }
        }
        tc_commit(smem_addr(empty + st));
        tc_commit(smem_addr(acc_full + st));
        last = st;
        last_parity = parity;
      }
      // No MMA may be in flight when the accumulator is freed.
      if (last >= 0) {
        const uint64_t t0 = global_ns();
        while (!mbar_try(acc_full + last, last_parity) && global_ns() - t0 < kDrainNs) {
        }
      }
    }
    __syncwarp();
  } else {
    // ---- epilogue (warps 0-7; warp w reads lanes 32 (w % 4) + lane, column half w / 4) ----
    constexpr int E = S::kEpiPairs;
    constexpr int kOut4 = S::kStageStride / 2;
    constexpr int kHalf = K / 2;
    float4* out = reinterpret_cast<float4*>(smem + S::kOffOut);  // row r: pairs (s, s + 1)
    const int t = tid;
    uint64_t a_t = 0;
    uint32_t sr_t = 0;
#pragma unroll
    for (int b = 0; b < 8; ++b)
      if ((t >> b) & 1) {
        a_t |= p.lam_addr[b];
        sr_t |= p.lam_sr[b];
      }
    const int quarter = warp & 3, half = warp >> 2;
    const int row = quarter * 32 + lane;
    uint64_t tile = blockIdx.x;
    for (uint32_t j = 0; tile < p.n_tiles; ++j, tile += stride) {
      const int st = (int)(j & 1u);
      const bool ok = mbar_wait(acc_full + st, (j >> 1) & 1u, err, p.wait_ns);
      __syncwarp();  // the barrier reduction and TMEM loads below are warp-aligned
      if (!epi_all(ok)) break;
      tc_fence_after();
      float v[kHalf];
#pragma unroll
      for (int c0 = 0; c0 < kHalf; c0 += 16)
        tc_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(st * K + half * kHalf + c0), v + c0);
      tc_fence_before();
      mbar_arrive(acc_empty + st);
      // The previous tile's stores have read the output stage.
      epi_sync();
#pragma unroll
      for (int q = 0; q < kHalf / 4; ++q)
        out[row * kOut4 + half * (kHalf / 4) + q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      epi_sync();
      const uint64_t tb = tile_base(tile, p) | a_t;
#pragma unroll
      for (int i = 0; i < E; ++i)
        if (t + i * kTcEpiThreads < p.npairs) {
          const uint32_t sr = sr_t | p.step_sr[i];
          const float4 w = out[(int)(sr >> 8) * kOut4 + (int)((sr & 0xFFu) >> 1)];
          const uint64_t a = tb | p.step_addr[i];
          if (p.pair_vec) {
            *reinterpret_cast<float4*>(psi + a) = w;
          } else {
            psi[a] = make_float2(w.x, w.y);
            psi[a | p.pair_bit] = make_float2(w.z, w.w);
          }
        }
    }
    __syncwarp();
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
// Float-float kernel
// ---------------------------------------------------------------------------
// A warp holds G = 32 / d groups; lane = g d + r computes output r of group g.
// Each lane loads input r, splits it into float-float once and stages it in
// shared memory (padded per group); lane r then accumulates sum_c U[r][c] x_c
// over its group's staged inputs (TwoSum of the heads, exact product tails,
// the rest in the tail sum: its error stays near 2^-43 of the row's partial
// sums for 32 terms, where an anchored head sum, whose anchor must exceed the
// row's coefficient sum times the largest input, loses 2^-38 of it) and
// rounds to double.
template <int KQ>
struct DFDenseParams {
  uint64_t n_groups;
  int npos;
  uint64_t high_mask[QS_MAX_QUBITS];
  uint64_t fixed_mask;
  uint64_t offs[1 << KQ];
  // U[r][c] at [c][r] as (re_h, re_l, im_h, im_l); the kernel expands it
  // into the two terms of the packed (re, im) product in shared memory.
  float4 u[(1 << KQ) * (1 << KQ)];
};

template <int KQ>
__global__ void __launch_bounds__(256) k_dense_df(double2* __restrict__ psi, const __grid_constant__ DFDenseParams<KQ> p) {
  constexpr int D = 1 << KQ, G = 32 / D, kWarps = 256 / 32;
  // (re_h, re_h, re_l, re_l) and (-im_h, im_h, -im_l, im_l) per coefficient.
  __shared__ float4 ua[D * D], ub[D * D];
  __shared__ float4 xs[kWarps][G * (D + 1)];  // per warp: (re_h, im_h, re_l, im_l) of each group's inputs
  for (int i = threadIdx.x; i < D * D; i += blockDim.x) {
    const float4 u = p.u[i];
    ua[i] = make_float4(u.x, u.x, u.y, u.y);
    ub[i] = make_float4(-u.z, u.z, -u.w, u.w);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int gl = lane / D, r = lane % D;
  const uint64_t warps = (uint64_t)gridDim.x * kWarps;
  const uint64_t off_r = p.offs[r];
  for (uint64_t g0 = ((uint64_t)blockIdx.x * kWarps + w) * G; g0 < p.n_groups; g0 += warps * G) {
    const uint64_t g = g0 + gl;
    const bool ok = g < p.n_groups;
    uint64_t b = g;
    for (int j = 0; j < p.npos; ++j) b += b & p.high_mask[j];
    b |= p.fixed_mask;
    const double2 x = ok ? psi[b | off_r] : make_double2(0.0, 0.0);
    float rh, rl, ih, il;
    d2ff(x.x, rh, rl);
    d2ff(x.y, ih, il);
    xs[w][gl * (D + 1) + r] = make_float4(rh, ih, rl, il);
    __syncwarp();
    DF2Acc acc;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const float4 v = xs[w][gl * (D + 1) + c];
      const float4 a4 = ua[c * D + r], b4 = ub[c * D + r];
      DF2Term ta, tb;
      ta.h = make_float2(a4.x, a4.y);
      ta.hn = make_float2(-a4.x, -a4.y);
      ta.l = make_float2(a4.z, a4.w);
      tb.h = make_float2(b4.x, b4.y);
      tb.hn = make_float2(-b4.x, -b4.y);
      tb.l = make_float2(b4.z, b4.w);
      if (c == 0)
        acc.template first<false>(ta, make_float2(v.x, v.y), make_float2(v.z, v.w));
      else
        acc.template add<false>(ta, make_float2(v.x, v.y), make_float2(v.z, v.w));
      acc.template add<false>(tb, make_float2(v.y, v.x), make_float2(v.w, v.z));
    }
    __syncwarp();  // every lane has read the staged inputs
    if (ok)
      psi[b | off_r] = make_double2(f2d_exact(acc.S.x) + f2d_exact(acc.C.x), f2d_exact(acc.S.y) + f2d_exact(acc.C.y));
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
qs_status launch_float_float(qs_state s, const DenseGeom& g, const double* U) {
  constexpr int D = 1 << KQ;
  static thread_local DFDenseParams<KQ> p;
  std::memset(&p, 0, sizeof(p));
  p.n_groups = g.n_groups;
  p.npos = g.ins.npos;
  for (int j = 0; j < QS_MAX_QUBITS; ++j) p.high_mask[j] = g.ins.high_mask[j];
  p.fixed_mask = g.ins.fixed_mask;
  for (int v = 0; v < D; ++v) p.offs[v] = g.offs[v];
  for (int r = 0; r < D; ++r)
    for (int c = 0; c < D; ++c) {
      const double re = U[2 * (r * D + c)], im = U[2 * (r * D + c) + 1];
      const float rh = (float)re, ih = (float)im;
      const float rl = (float)(re - (double)rh), il = (float)(im - (double)ih);
      p.u[c * D + r] = make_float4(rh, rl, ih, il);
    }
  const uint64_t warps = (g.n_groups * D + 31) / 32;
  const uint64_t blocks = (warps + 7) / 8;
  const uint64_t cap = (uint64_t)sm_count(s->device) * 8;
  const unsigned grid = (unsigned)(blocks < cap ? blocks : cap);
  k_dense_df<KQ><<<grid, 256, 0, s->stream>>>((double2*)s->psi, p);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

template <int KQ>
qs_status launch_tensor_core(qs_state s, const DenseGeom& g, const double* U) {
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
  const int low_target = g.targets[order[0]];
  p.pair_bit = 1ull << low_target;
  p.pair_vec = low_target == 0 ? 1 : 0;
  // Pair-index bits in ascending address order: sorted targets 1..k-1 map
  // to s bits 1..k-1, the r-th lowest free position to row bit r.
  std::vector<std::pair<int, uint32_t>> bits;
  for (int j = 1; j < KQ; ++j) bits.push_back({g.targets[order[j]], 1u << j});
  for (int r = 0; r < rb; ++r) bits.push_back({g.free_pos[r], (1u << r) << 8});
  std::sort(bits.begin(), bits.end());
  // Epilogue: 8 thread bits, then up to 3 step bits; producers: 9 and 2.
  for (int b = 0; b < (int)bits.size(); ++b) {
    const uint64_t ab = 1ull << bits[b].first;
    const uint32_t sb = bits[b].second;
    if (b < 8) {
      p.lam_addr[b] = ab;
      p.lam_sr[b] = sb;
    } else {
      for (int i = 0; i < 8; ++i)
        if ((i >> (b - 8)) & 1) {
          p.step_addr[i] |= ab;
          p.step_sr[i] |= sb;
        }
    }
    if (b < 9) {
      p.prod_addr[b] = ab;
      p.prod_sr[b] = sb;
    } else {
      for (int i = 0; i < 4; ++i)
        if ((i >> (b - 9)) & 1) {
          p.prod_step_addr[i] |= ab;
          p.prod_step_sr[i] |= sb;
        }
    }
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
  using S = TcShape<KQ>;
  // Set on every launch (a host call of microseconds against a launch of
  // milliseconds), so the state's current device has them too.
  QS_CUDA(cudaFuncSetAttribute(k_dense_tc<KQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::kSmem));
  // All of the unified L1 / shared array as shared memory.
  QS_CUDA(cudaFuncSetAttribute(k_dense_tc<KQ>, cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared));
  // One CTA per SM (its pipeline holds up to four tiles).
  const uint64_t cap = (uint64_t)sm_count(s->device);
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
  if (s->dtype == QS_C64 && s->tensor_cores != 0) {
    // The CUDA-core kernel's loads are strided when its consecutive groups
    // are far apart, i.e. when qubits 0 and 1 are both targets or controls:
    // then the tensor cores win at k = 3, 4 too (measured at 30 qubits: 4.8
    // against 1.9-2.9 TB/s); otherwise the CUDA cores keep up with HBM there
    // (4.8-5.7 TB/s).  At k = 5 the tensor cores always win.  Mode 2 takes
    // the tensor cores wherever they apply.
    const int low_free = g.free_pos.empty() ? 64 : g.free_pos[0];
    const bool strided = low_free >= 2;
    if (k == 5) return launch_tensor_core<5>(s, g, U);
    if (strided || s->tensor_cores == 2) {
      // Fewer targets run as the 5-target gate I (x) U on the lowest free
      // qubits (new high bits of the index: block-diagonal, 2^(5-k) copies of
      // U), at the 5-target kernel's rate; k = 4 without a free qubit runs on
      // the 4-target kernel.
      const int pad = 5 - k;
      if ((int)g.free_pos.size() >= pad) {
        int t5[5];
        for (int j = 0; j < k; ++j) t5[j] = targets[j];
        for (int j = 0; j < pad; ++j) t5[k + j] = g.free_pos[j];
        const int d = 1 << k;
        static thread_local double V[2 * 32 * 32];
        std::memset(V, 0, sizeof(V));
        for (int r = 0; r < 32; ++r)
          for (int c = 0; c < 32; ++c)
            if ((r >> k) == (c >> k)) {
              V[2 * (r * 32 + c)] = U[2 * ((r & (d - 1)) * d + (c & (d - 1)))];
              V[2 * (r * 32 + c) + 1] = U[2 * ((r & (d - 1)) * d + (c & (d - 1))) + 1];
            }
        return launch_tensor_core<5>(s, dense_geom(s, t5, 5, ctrl_mask), V);
      }
      if (k == 4) return launch_tensor_core<4>(s, g, U);
    }
  }
  if (s->dtype == QS_C64) {
    if (k == 3) return launch_cuda_core<float, 3>(s, g, U);
    if (k == 4) return launch_cuda_core<float, 4>(s, g, U);
    return launch_cuda_core<float, 5>(s, g, U);
  }
  if (s->math == QS_MATH_DF) {
    if (k == 3) return launch_float_float<3>(s, g, U);
    if (k == 4) return launch_float_float<4>(s, g, U);
    return launch_float_float<5>(s, g, U);
  }
  if (k == 3) return launch_cuda_core<double, 3>(s, g, U);
  if (k == 4) return launch_cuda_core<double, 4>(s, g, U);
  return launch_cuda_core<double, 5>(s, g, U);
}

}  // namespace qs
