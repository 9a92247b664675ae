// Device building blocks of the fused-block engine shared by the per-circuit
// tile kernel (qs_tile.cu) and the batched kernel (qs_batch.cu): PTX wrappers
// for mbarriers, bulk asynchronous copies and named barriers; the tile
// precision policies; and the application of one gate op to a tile held in
// shared memory.
#pragma once
#include <cstdint>
#include <type_traits>

#include "qs_math.cuh"
#include "qs_tile.cuh"

namespace qs {

#ifndef QS_TILE_STAGES
#define QS_TILE_STAGES 3
#endif
#ifndef QS_TILE_MIN_CTAS
#define QS_TILE_MIN_CTAS 2
#endif
// Consumer threads per CTA (a power of two); a tile is kTileConsumers x 2^RB
// amplitudes, RB the policy's register bits.
#ifndef QS_TILE_CONSUMERS_LOG
#define QS_TILE_CONSUMERS_LOG 8
#endif
constexpr int kTileConsumersLog = QS_TILE_CONSUMERS_LOG;
constexpr int kTileConsumers = 1 << kTileConsumersLog;
constexpr int kTileThreads = kTileConsumers + 32;
// Threads of a CTA under policy TP: the consumers, plus a producer warp
// unless consumer thread 0 takes that role (TP::kFoldProducer).
template <class TP>
constexpr int tile_threads() {
  return TP::kFoldProducer ? kTileConsumers : kTileThreads;
}
constexpr int kStages = QS_TILE_STAGES;
constexpr int kTileMinCtas = QS_TILE_MIN_CTAS;
// Bound of the waits that let a CTA's own copies land before it exits after
// an error (the copies are in-range and always complete).
constexpr uint64_t kDrainNs = 2000000000ull;

// ---------------------------------------------------------------------------
// PTX helpers: mbarrier, bulk copies, proxy fence, named barriers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Non-blocking check of a phase (try_wait may suspend the thread for a
// while before it reports an incomplete phase; test_wait does not).
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait (limit_ns of %globaltimer): false when it gave up (timeout
// recorded, or another thread already recorded an error).  A limit of 0
// gives up at once if the phase is not complete when first checked.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t* err, uint64_t limit_ns) {
  if (limit_ns == 0) {
    if (mbar_test(bar, parity)) return true;
    atomicCAS(err, 0u, 1u);
    return false;
  }
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try(bar, parity)) {
    if (*(volatile uint32_t*)err != 0u) return false;
    if (global_ns() - t0 > limit_ns) {
      atomicCAS(err, 0u, 1u);
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ void bulk_load(void* dst_smem, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst_smem)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void bulk_store(void* dst, const void* src_smem, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src_smem)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// At most one committed bulk group of this thread may still be reading
// shared memory.
__device__ __forceinline__ void bulk_wait_read_one() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void consumers_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kTileConsumers) : "memory");
}
// Consumer-wide OR of a predicate (uniform result).
__device__ __forceinline__ bool consumers_any(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(kTileConsumers)
      : "memory");
  return r != 0;
}

// ---------------------------------------------------------------------------
// Tile precision policies
// ---------------------------------------------------------------------------
struct TileF32 {
  using M = MathF32;
  // A producer warp of its own beside the eight consumer warps.
  static constexpr bool kFoldProducer = false;
  // Copy a 2x2 op's four coefficients to registers before the pairs.
  static constexpr bool kHoistCoefs = true;
  // Uncontrolled 4x4 ops take the quads two at a time (one coefficient load
  // serves both); the batched kernel, with more live state, opts out.
  static constexpr bool kQuadPairs = true;
  // Stage the block's ops and coefficients in shared memory.
  static constexpr bool kStagePlan = true;
  using Glob = float2;
  using Sm = float2;
  static constexpr int kTileLog = kTileConsumersLog + 4;  // 4096 amplitudes, 32 KB (256 consumers)
  static constexpr int kRegBits = 4;  // 16 amplitudes per thread
  static constexpr int kBankBits = 4;  // 16 amplitudes per 128-byte shared-memory row
  static __device__ __forceinline__ Sm to_sm(Glob g) { return g; }
  static __device__ __forceinline__ Glob from_sm(Sm s) { return s; }
  static __device__ __forceinline__ M::Val val(Sm s) { return M::load(s); }
  // One 16-byte load per coefficient (a and b together).
  static __device__ __forceinline__ float4 ldc4(const M::Coef* c) { return *reinterpret_cast<const float4*>(c); }
  template <int K>
  static __device__ __forceinline__ Sm mac(const M::Coef* c, const M::Val* v) {
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const float4 q = ldc4(c + k);
      acc = k == 0 ? mul2(make_float2(q.x, q.y), v[0].v) : fma2(make_float2(q.x, q.y), v[k].v, acc);
      acc = fma2(make_float2(q.z, q.w), v[k].vs, acc);
    }
    return acc;
  }
  // A row of four coefficients already in registers ((a, b) per float4).
  static __device__ __forceinline__ Sm mac4(const float4* c, const M::Val* v) {
    float2 acc = mul2(make_float2(c[0].x, c[0].y), v[0].v);
    acc = fma2(make_float2(c[0].z, c[0].w), v[0].vs, acc);
#pragma unroll
    for (int k = 1; k < 4; ++k) {
      acc = fma2(make_float2(c[k].x, c[k].y), v[k].v, acc);
      acc = fma2(make_float2(c[k].z, c[k].w), v[k].vs, acc);
    }
    return acc;
  }
  // Real coefficients: the (-mi, mi) terms are zero and skipped.
  template <int K>
  static __device__ __forceinline__ Sm mac_real(const M::Coef* c, const M::Val* v) {
    float2 acc = mul2(c[0].a, v[0].v);
#pragma unroll
    for (int k = 1; k < K; ++k) acc = fma2(c[k].a, v[k].v, acc);
    return acc;
  }
  template <int K>
  static __device__ __forceinline__ int mexp(const M::Val*) { return 0; }
  template <int K>
  static __device__ __forceinline__ Sm mac_rows(const M::Coef* c, const M::Val* v, int, int) {
    return mac<K>(c, v);
  }
  static __device__ __forceinline__ Sm neg(Sm a) {
    return make_float2(__uint_as_float(__float_as_uint(a.x) ^ 0x80000000u),
                       __uint_as_float(__float_as_uint(a.y) ^ 0x80000000u));
  }
  // -i (x + iy) = y - ix
  static __device__ __forceinline__ Sm mul_minus_i(Sm a) { return make_float2(a.y, -a.x); }
  static __device__ __forceinline__ Sm mul_i(Sm a) { return make_float2(-a.y, a.x); }
  // Phase-table entries (cos, sin) and sign flips under bit 31 of s.
  using Phase = float2;
  static constexpr int kPhaseFormat = 0;
  static __device__ __forceinline__ M::Coef phase_coef(Phase p) {
    return M::Coef{make_float2(p.x, p.x), make_float2(-p.y, p.y)};
  }
  static __device__ __forceinline__ Sm neg_if(Sm a, uint32_t s) {
    return make_float2(__uint_as_float(__float_as_uint(a.x) ^ s), __uint_as_float(__float_as_uint(a.y) ^ s));
  }
};

// complex64 policy of the batched kernel: one quad at a time.
struct TileF32Batch : TileF32 {
  static constexpr bool kQuadPairs = false;
};

__device__ __forceinline__ double dneg(double x) {
  return __hiloint2double(__double2hiint(x) ^ (int)0x80000000u, __double2loint(x));
}

struct TileF64 {
  using M = MathF64;
  static constexpr bool kFoldProducer = false;
  static constexpr bool kHoistCoefs = true;
  static constexpr bool kQuadPairs = false;
  // Stage the block's ops and coefficients in shared memory.
  static constexpr bool kStagePlan = true;
  using Glob = double2;
  using Sm = double2;
  static constexpr int kTileLog = kTileConsumersLog + 3;  // 2048 amplitudes, 32 KB (256 consumers)
  static constexpr int kRegBits = 3;  // 8 amplitudes per thread
  static constexpr int kBankBits = 3;  // 8 amplitudes per 128-byte shared-memory row
  static __device__ __forceinline__ Sm to_sm(Glob g) { return g; }
  static __device__ __forceinline__ Glob from_sm(Sm s) { return s; }
  static __device__ __forceinline__ M::Val val(Sm s) { return M::load(s); }
  template <int K>
  static __device__ __forceinline__ Sm mac(const M::Coef* c, const M::Val* v) { return M::mac_round<K>(c, v); }
  template <int K>
  static __device__ __forceinline__ Sm mac_real(const M::Coef* c, const M::Val* v) {
    double re = 0.0, im = 0.0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      re = __fma_rn(c[k].re, v[k].re, re);
      im = __fma_rn(c[k].re, v[k].im, im);
    }
    return make_double2(re, im);
  }
  template <int K>
  static __device__ __forceinline__ int mexp(const M::Val*) { return 0; }
  template <int K>
  static __device__ __forceinline__ Sm mac_rows(const M::Coef* c, const M::Val* v, int, int) {
    return M::mac_round<K>(c, v);
  }
  static __device__ __forceinline__ Sm neg(Sm a) { return make_double2(dneg(a.x), dneg(a.y)); }
  static __device__ __forceinline__ Sm mul_minus_i(Sm a) { return make_double2(a.y, dneg(a.x)); }
  static __device__ __forceinline__ Sm mul_i(Sm a) { return make_double2(dneg(a.y), a.x); }
  using Phase = double2;
  static constexpr int kPhaseFormat = 1;
  static __device__ __forceinline__ M::Coef phase_coef(Phase p) { return M::Coef{p.x, p.y}; }
  static __device__ __forceinline__ double dneg_if(double x, uint32_t s) {
    return __hiloint2double(__double2hiint(x) ^ (int)s, __double2loint(x));
  }
  static __device__ __forceinline__ Sm neg_if(Sm a, uint32_t s) { return make_double2(dneg_if(a.x, s), dneg_if(a.y, s)); }
};

// Float-float tile element: (re_h, im_h, re_l, im_l), |l| <= ulp(h)/2.
struct TileDF {
  using M = MathDF;
  static constexpr bool kFoldProducer = false;
  static constexpr bool kQuadPairs = false;
  // Plans are staged in shared memory: the lanes of a diagonal op gather
  // different coefficients, which the parameter bank would serialise.
  static constexpr bool kStagePlan = true;
  // A float-float coefficient is 64 bytes: a 2x2 op reads its coefficients
  // from the staged plan where it uses them rather than holding all four.
  static constexpr bool kHoistCoefs = false;
  using Glob = double2;
  using Sm = float4;
  static constexpr int kTileLog = kTileConsumersLog + 3;
  static constexpr int kRegBits = 3;  // 8 amplitudes per thread
  static constexpr int kBankBits = 3;  // 8 amplitudes per 128-byte shared-memory row
  static __device__ __forceinline__ Sm to_sm(Glob g) {
    Sm s;
    d2ff(g.x, s.x, s.z);
    d2ff(g.y, s.y, s.w);
    return s;
  }
  // One FP64 add per component rounds h + l to double.
  static __device__ __forceinline__ Glob from_sm(Sm s) {
    return make_double2(f2d_exact(s.x) + f2d_exact(s.z), f2d_exact(s.y) + f2d_exact(s.w));
  }
  static __device__ __forceinline__ M::Val val(Sm s) {
    M::Val v;
    v.h = make_float2(s.x, s.y);
    v.l = make_float2(s.z, s.w);
    v.hs = make_float2(s.y, s.x);
    v.ls = make_float2(s.w, s.z);
    return v;
  }
  template <int K>
  static __device__ __forceinline__ Sm mac(const M::Coef* c, const M::Val* v) {
    const DF2Acc a = M::mac<K>(c, v);
    // Renormalise (S, C) to head and tail with Fast2Sum (Dekker 1971); C is
    // the lower-order part, so the head absorbs it and the tail keeps the
    // remainder.
    const float2 s = add2(a.S, a.C);
    const float2 e = sub2(a.C, sub2(s, a.S));
    return make_float4(s.x, s.y, e.x, e.y);
  }
  template <int K>
  static __device__ __forceinline__ Sm mac_real(const M::Coef* c, const M::Val* v) {
    DF2Acc a;
    a.first(c[0].a, v[0].h, v[0].l);
#pragma unroll
    for (int k = 1; k < K; ++k) a.add(c[k].a, v[k].h, v[k].l);
    const float2 s = add2(a.S, a.C);
    const float2 e = sub2(a.C, sub2(s, a.S));
    return make_float4(s.x, s.y, e.x, e.y);
  }
  template <int K>
  static __device__ __forceinline__ int mexp(const M::Val* v) { return M::max_exp_field<K>(v); }
  // Anchored accumulation for dense rows (row_exp from the host, mexp from
  // the inputs), renormalised like mac.
  template <int K>
  static __device__ __forceinline__ Sm mac_rows(const M::Coef* c, const M::Val* v, int row_exp, int mx) {
    const DF2Acc a = M::mac_anchor<K>(c, v, row_exp, mx);
    const float2 s = add2(a.S, a.C);
    const float2 e = sub2(a.C, sub2(s, a.S));
    return make_float4(s.x, s.y, e.x, e.y);
  }
  static __device__ __forceinline__ float fneg(float x) { return __uint_as_float(__float_as_uint(x) ^ 0x80000000u); }
  static __device__ __forceinline__ Sm neg(Sm a) { return make_float4(fneg(a.x), fneg(a.y), fneg(a.z), fneg(a.w)); }
  static __device__ __forceinline__ Sm mul_minus_i(Sm a) { return make_float4(a.y, fneg(a.x), a.w, fneg(a.z)); }
  static __device__ __forceinline__ Sm mul_i(Sm a) { return make_float4(fneg(a.y), a.x, fneg(a.w), a.z); }
  // Phase-table entries: (cos head, sin head, cos tail, sin tail).
  using Phase = float4;
  static constexpr int kPhaseFormat = 2;
  static __device__ __forceinline__ M::Coef phase_coef(Phase p) {
    M::Coef c;
    c.a.h = make_float2(p.x, p.x);
    c.a.hn = make_float2(-p.x, -p.x);
    c.a.l = make_float2(p.z, p.z);
    c.a.ll = make_float2(0.f, 0.f);
    c.b.h = make_float2(-p.y, p.y);
    c.b.hn = make_float2(p.y, -p.y);
    c.b.l = make_float2(-p.w, p.w);
    c.b.ll = make_float2(0.f, 0.f);
    return c;
  }
  static __device__ __forceinline__ float fxor(float x, uint32_t s) { return __uint_as_float(__float_as_uint(x) ^ s); }
  static __device__ __forceinline__ Sm neg_if(Sm a, uint32_t s) {
    return make_float4(fxor(a.x, s), fxor(a.y, s), fxor(a.z, s), fxor(a.w, s));
  }
};

// TileDF with consumer thread 0 issuing the copies between its tiles: two CTAs
// of eight warps (16 per SM, four on each register partition) leave 128
// registers a thread, where a ninth producer warp per CTA (five warps on
// some partitions) caps them at 96 and makes the float-float 4x4 ops spill.
// Thread 0 then waits for the slowest warp once per tile, which costs more
// than it saves on blocks without 4x4 ops.
struct TileDFFold : TileDF {
  static constexpr bool kFoldProducer = true;
};

// The batched kernel stages float-float plans like k_tile does.
using TileDFBatch = TileDF;

// ---------------------------------------------------------------------------
// Register-resident tile consumer
// ---------------------------------------------------------------------------
// Global index of a tile's first amplitude: the tile number spread over the
// free qubits (zeros inserted at the high tile qubits, ascending).
__device__ __forceinline__ uint64_t tile_base(uint64_t tau, int L, int m, const uint64_t* base_high) {
  uint64_t b = tau << L;
  for (int j = 0; j < m; ++j) b += b & base_high[j];
  return b;
}

template <class TP>
struct RegTile {
  static constexpr int RB = TP::kRegBits;
  static constexpr int R = 1 << RB;
  using Sm = typename TP::Sm;
  using Glob = typename TP::Glob;
  using Val = typename TP::M::Val;
  using Coef = typename TP::M::Coef;

  Sm v[R];
  uint32_t pbit[RB];  // local index bit of register bit j (0 when unused)
  uint32_t toff;      // local index bits of this thread
  uint32_t tsw;       // swizzled byte offset of toff
  uint32_t psw[RB];   // swizzled byte offset of pbit[j]
  int reff;           // registers in use (SMALL: tiles smaller than 2^RB)
  bool active;        // this thread holds amplitudes

  // Shared-memory position of local index lam for layout changes: within
  // each 128-byte row the column is XORed with the row number, so a warp
  // whose lanes differ only in high local bits still spreads over all banks.
  static constexpr int kSwB = sizeof(typename TP::Sm) == 16 ? 3 : 4;
  static __device__ __forceinline__ uint32_t swz(uint32_t lam) {
    return lam ^ ((lam >> kSwB) & ((1u << kSwB) - 1u));
  }
  // Registers beyond 2^tile_log (tiles smaller than 2^RB amplitudes) carry
  // no amplitude: ops may compute on them, reads and writes skip them.
  __device__ __forceinline__ bool live(int r) const { return r < reff; }

  // Local index bits of register r (r is a compile-time constant in the
  // unrolled loops, so this folds to a few ORs).
  __device__ __forceinline__ uint32_t roff(int r) const {
    uint32_t o = 0;
#pragma unroll
    for (int j = 0; j < RB; ++j)
      if ((r >> j) & 1) o |= pbit[j];
    return o;
  }

  // Set the layout: register bit j is local bit pos[j]; the other local
  // bits, ascending, take the thread index bits.
  __device__ __forceinline__ void set_layout(const uint8_t* pos, int rb, int tile_log, int tid) {
    uint32_t regmask = 0;
#pragma unroll
    for (int j = 0; j < RB; ++j) {
      pbit[j] = j < rb ? (1u << pos[j]) : 0u;
      regmask |= pbit[j];
    }
    uint32_t t = 0;
    int jt = 0;
    for (int b = 0; b < tile_log; ++b) {
      if ((regmask >> b) & 1u) continue;
      if ((tid >> jt) & 1) t |= 1u << b;
      ++jt;
    }
    toff = t;
    tsw = swz(t) * (uint32_t)sizeof(Sm);
#pragma unroll
    for (int j = 0; j < RB; ++j) psw[j] = swz(pbit[j]) * (uint32_t)sizeof(Sm);
    reff = 1 << rb;
    active = (tid >> (tile_log - rb)) == 0;
  }

  // Relabel for a swap of local bits a and b (no data moves).
  __device__ __forceinline__ void swap_bits(int a, int b) {
    auto sw = [a, b](uint32_t x) {
      const uint32_t d = ((x >> a) ^ (x >> b)) & 1u;
      return x ^ ((d << a) | (d << b));
    };
    toff = sw(toff);
    tsw = swz(toff) * (uint32_t)sizeof(Sm);
#pragma unroll
    for (int j = 0; j < RB; ++j) {
      pbit[j] = sw(pbit[j]);
      psw[j] = swz(pbit[j]) * (uint32_t)sizeof(Sm);
    }
  }

  // Byte offsets: swz is linear over XOR on disjoint bits, so the swizzled
  // offset of register r is the thread's offset XOR those of r's bits.
  __device__ __forceinline__ uint32_t sw_off(int r) const {
    uint32_t o = tsw;
#pragma unroll
    for (int j = 0; j < RB; ++j)
      if ((r >> j) & 1) o ^= psw[j];
    return o;
  }

  // raw: the staged tile already holds the working format.
  __device__ __forceinline__ void read_glob(const unsigned char* smem, bool raw) {
    const Glob* g = reinterpret_cast<const Glob*>(smem);
    const Sm* t = reinterpret_cast<const Sm*>(smem);
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (live(r) && active) v[r] = raw ? t[toff | roff(r)] : TP::to_sm(g[toff | roff(r)]);
  }
  __device__ __forceinline__ void read_sm(const unsigned char* smem) {
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (live(r) && active) v[r] = *reinterpret_cast<const Sm*>(smem + sw_off(r));
  }
  __device__ __forceinline__ void write_sm(unsigned char* smem) const {
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (live(r) && active) *reinterpret_cast<Sm*>(smem + sw_off(r)) = v[r];
  }
  __device__ __forceinline__ void write_glob(unsigned char* smem, bool raw) const {
    Glob* g = reinterpret_cast<Glob*>(smem);
    Sm* t = reinterpret_cast<Sm*>(smem);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (!live(r) || !active) continue;
      if (raw) t[toff | roff(r)] = v[r];
      else g[toff | roff(r)] = TP::from_sm(v[r]);
    }
  }

  template <int K, bool CTRL, bool REAL>
  __device__ __forceinline__ void dense1(const Coef* cf, uint32_t lmask) {
    Coef hc[TP::kHoistCoefs ? 4 : 1];
    if constexpr (TP::kHoistCoefs) {
#pragma unroll
      for (int j = 0; j < 4; ++j) hc[j] = cf[j];
    }
    const Coef* c = TP::kHoistCoefs ? hc : cf;
    // 2x2 rows keep TwoSum accumulation (exact under cancellation).
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (r & (1 << K)) continue;
      if (CTRL && ((toff | roff(r)) & lmask) != lmask) continue;
      const Val x[2] = {TP::val(v[r]), TP::val(v[r | (1 << K)])};
      if (REAL) {
        v[r] = TP::template mac_real<2>(c, x);
        v[r | (1 << K)] = TP::template mac_real<2>(c + 2, x);
      } else {
        v[r] = TP::template mac<2>(c, x);
        v[r | (1 << K)] = TP::template mac<2>(c + 2, x);
      }
    }
  }

  template <int K>
  __device__ __forceinline__ void xswap(bool y, uint32_t lmask) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (r & (1 << K)) continue;
      if (((toff | roff(r)) & lmask) != lmask) continue;
      const Sm a = v[r], b = v[r | (1 << K)];
      v[r] = y ? TP::mul_minus_i(b) : b;
      v[r | (1 << K)] = y ? TP::mul_i(a) : a;
    }
  }

  // The i-th register whose bits B0 and B1 are clear (a quad's base).
  static constexpr int quad_base(int i, int b01) {
    int c = 0;
    for (int r = 0; r < R; ++r) {
      if (r & b01) continue;
      if (c == i) return r;
      ++c;
    }
    return 0;
  }

  template <int K0, int K1>
  __device__ __forceinline__ void dense2(const Coef* cf, uint32_t lmask, const uint8_t* rexp) {
    constexpr int B0 = 1 << K0, B1 = 1 << K1;
    if constexpr (TP::kQuadPairs) {
      if (lmask == 0) {
        // complex64, no controls: two quads per pass over the matrix, so
        // each row of coefficients is loaded once for both.
#pragma unroll
        for (int p = 0; p < R / 4; p += 2) {
          constexpr int kB = B0 | B1;
          const int ra = quad_base(p, kB), rb = quad_base(p + 1, kB);
          const Val xa[4] = {TP::val(v[ra]), TP::val(v[ra | B0]), TP::val(v[ra | B1]), TP::val(v[ra | B0 | B1])};
          const Val xb[4] = {TP::val(v[rb]), TP::val(v[rb | B0]), TP::val(v[rb | B1]), TP::val(v[rb | B0 | B1])};
          Sm oa[4], ob[4];
#pragma unroll
          for (int row = 0; row < 4; ++row) {
            float4 c[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) c[k] = TP::ldc4(cf + 4 * row + k);
            oa[row] = TP::mac4(c, xa);
            ob[row] = TP::mac4(c, xb);
          }
          v[ra] = oa[0];
          v[ra | B0] = oa[1];
          v[ra | B1] = oa[2];
          v[ra | B0 | B1] = oa[3];
          v[rb] = ob[0];
          v[rb | B0] = ob[1];
          v[rb | B1] = ob[2];
          v[rb | B0 | B1] = ob[3];
        }
        return;
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (r & (B0 | B1)) continue;
      if (lmask && ((toff | roff(r)) & lmask) != lmask) continue;
      const Val x[4] = {TP::val(v[r]), TP::val(v[r | B0]), TP::val(v[r | B1]), TP::val(v[r | B0 | B1])};
      const int mx = TP::template mexp<4>(x);
      v[r] = TP::template mac_rows<4>(cf, x, (int)rexp[0] - 128, mx);
      v[r | B0] = TP::template mac_rows<4>(cf + 4, x, (int)rexp[1] - 128, mx);
      v[r | B1] = TP::template mac_rows<4>(cf + 8, x, (int)rexp[2] - 128, mx);
      v[r | B0 | B1] = TP::template mac_rows<4>(cf + 12, x, (int)rexp[3] - 128, mx);
    }
  }

  __device__ __forceinline__ void phase(const Coef* cf, uint32_t lmask, uint32_t lpat, bool neg) {
    const Coef c = cf[0];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (((toff | roff(r)) & lmask) != lpat) continue;
      if (neg) {
        v[r] = TP::neg(v[r]);
      } else {
        const Val x = TP::val(v[r]);
        v[r] = TP::template mac<1>(&c, &x);
      }
    }
  }

  __device__ __forceinline__ void diag(const TileOp& op, const Coef* cf, uint64_t base) {
    // Table index s = (tile bits) | (thread bits) | (register bits): the
    // first two are fixed for the thread, the register part is the OR of
    // the entries of the register's set bits, found once per op.
    uint32_t sg = 0;
    for (int j = 0; j < op.k; ++j)
      if (op.gq[j] != 0xFF) sg |= (uint32_t)((base >> op.gq[j]) & 1ull) << j;
    uint32_t rbit[RB];
#pragma unroll
    for (int b = 0; b < RB; ++b) rbit[b] = 0u;
    for (int j = 0; j < op.nloc; ++j) {
      const uint32_t lb = 1u << op.tpos[j], sb = 1u << op.tj[j];
      if (toff & lb) sg |= sb;
#pragma unroll
      for (int b = 0; b < RB; ++b) rbit[b] |= pbit[b] == lb ? sb : 0u;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const uint32_t lam = toff | roff(r);
      if ((lam & op.lmask) != op.lmask) continue;
      uint32_t sidx = sg;
#pragma unroll
      for (int b = 0; b < RB; ++b)
        if ((r >> b) & 1) sidx |= rbit[b];
      const Val x = TP::val(v[r]);
      v[r] = TP::template mac<1>(cf + sidx, &x);
    }
  }

  // A run of phase terms (t[0] is the TOP_POLY op): sum each amplitude's
  // phase on the 2^-32-turn grid in an integer, then multiply once by the
  // table entries of its bytes (or flip signs when only bit 31 can be set).
  // Terms with the same register condition are summed per thread first.
  __device__ __forceinline__ void add_group(uint32_t* acc, uint32_t rm, uint32_t rp, uint32_t g) const {
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] += ((uint32_t)r & rm) == rp ? g : 0u;
  }
  // exp(2 pi i g / 2^32) from the table bytes of g (byte `first` up), applied
  // to the registers r with (r & rm) == rp.
  __device__ __forceinline__ void apply_group_phase(uint32_t rm, uint32_t rp, uint32_t g, int first,
                                                    const typename TP::Phase* __restrict__ tab) {
    Sm z = __ldg(tab + 256 * first + ((g >> (8 * first)) & 255u));
    for (int b = first + 1; b < 4; ++b) {
      const Coef c = TP::phase_coef(__ldg(tab + 256 * b + ((g >> (8 * b)) & 255u)));
      const Val x = TP::val(z);
      z = TP::template mac<1>(&c, &x);
    }
    const Coef cz = TP::phase_coef(z);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (((uint32_t)r & rm) != rp) continue;
      const Val x = TP::val(v[r]);
      v[r] = TP::template mac<1>(&cz, &x);
    }
  }
  __device__ __forceinline__ void poly(const TileOp* __restrict__ t, uint64_t base,
                                       const typename TP::Phase* __restrict__ tab) {
    const int count = t[0].k;
    const int first = t[0].nloc;
    if (first > 4) return;
    if (t[0].tpos[0]) {
      // Factored: each group's phase is one table product per thread,
      // multiplied into the group's registers.
      uint32_t g = 0, gkey = t[0].coef;
      for (int i = 0;; ++i) {
        const bool end = i == count;
        uint4 a = make_uint4(0u, 0u, 0u, 0u);
        ulonglong2 pr = make_ulonglong2(0ull, 0ull);
        if (!end) {
          a = *reinterpret_cast<const uint4*>(t + i);  // lmask, lpat, group key, m
          pr = *reinterpret_cast<const ulonglong2*>(&t[i].gmask);
        }
        if (end || a.z != gkey) {
          if (g != 0u) apply_group_phase(gkey & 0xFFu, (gkey >> 8) & 0xFFu, g, (int)(gkey >> 16) & 0xFF, tab);
          if (end) break;
          g = 0;
          gkey = a.z;
        }
        if ((base & pr.x) != pr.y) continue;
        g += (toff & a.x) == a.y ? a.w : 0u;
      }
      return;
    }
    uint32_t acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0u;
    uint32_t g = 0, gkey = t[0].coef;
    for (int i = 0; i < count; ++i) {
      const uint4 a = *reinterpret_cast<const uint4*>(t + i);  // lmask, lpat, group key, m
      const ulonglong2 pr = *reinterpret_cast<const ulonglong2*>(&t[i].gmask);
      if (a.z != gkey) {  // uniform: the same plan for every thread
        add_group(acc, gkey & 0xFFu, (gkey >> 8) & 0xFFu, g);
        g = 0;
        gkey = a.z;
      }
      if ((base & pr.x) != pr.y) continue;
      g += (toff & a.x) == a.y ? a.w : 0u;
    }
    add_group(acc, gkey & 0xFFu, (gkey >> 8) & 0xFFu, g);
    if (first == 4) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = TP::neg_if(v[r], acc[r] & 0x80000000u);
      return;
    }
    for (int b = first; b < 4; ++b) {
      const typename TP::Phase* tb = tab + 256 * b;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const Coef c = TP::phase_coef(__ldg(tb + ((acc[r] >> (8 * b)) & 255u)));
        const Val xv = TP::val(v[r]);
        v[r] = TP::template mac<1>(&c, &xv);
      }
    }
  }

  // Permutation of local targets: through shared memory (write in place,
  // read each destination's source).
  __device__ __forceinline__ void perm(const TileOp& op, const uint8_t* inv, unsigned char* smem) {
    consumers_sync();
    write_sm(smem);
    consumers_sync();
    const Sm* t = reinterpret_cast<const Sm*>(smem);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (!live(r) || !active) continue;
      const uint32_t d = toff | roff(r);
      uint32_t src = d;
      if ((d & op.lmask) == op.lmask) {
        uint32_t sidx = 0;
        for (int j = 0; j < op.k; ++j) sidx |= ((d >> op.tpos[j]) & 1u) << j;
        const uint32_t sv = inv[sidx];
        for (int j = 0; j < op.k; ++j) src = (src & ~(1u << op.tpos[j])) | (((sv >> j) & 1u) << op.tpos[j]);
      }
      v[r] = t[swz(src)];
    }
  }
};

template <class RT, bool CTRL, bool REAL>
__device__ __forceinline__ void dense1_k(RT& rt, int k, const typename RT::Coef* cf, uint32_t lmask) {
  switch (k) {
    case 0: rt.template dense1<0, CTRL, REAL>(cf, lmask); break;
    case 1: rt.template dense1<1, CTRL, REAL>(cf, lmask); break;
    case 2: if constexpr (RT::RB > 2) rt.template dense1<(RT::RB > 2 ? 2 : 0), CTRL, REAL>(cf, lmask); break;
    default: if constexpr (RT::RB > 3) rt.template dense1<(RT::RB > 3 ? 3 : 0), CTRL, REAL>(cf, lmask); break;
  }
}

template <class RT, int K>
__device__ __forceinline__ void dense2_k1(RT& rt, int k1, const typename RT::Coef* cf, uint32_t lmask,
                                          const uint8_t* rexp) {
  switch (k1) {
    case 0: if constexpr (K != 0) rt.template dense2<K, 0>(cf, lmask, rexp); break;
    case 1: if constexpr (K != 1) rt.template dense2<K, 1>(cf, lmask, rexp); break;
    case 2: if constexpr (K != 2 && RT::RB > 2) rt.template dense2<K, (RT::RB > 2 ? 2 : 0)>(cf, lmask, rexp); break;
    default: if constexpr (K != 3 && RT::RB > 3) rt.template dense2<K, (RT::RB > 3 ? 3 : 0)>(cf, lmask, rexp); break;
  }
}

// Apply a block's ops to one tile.  ops[0] is a TOP_LAYOUT: the first read
// converts the staged global-format tile; the tile is written back in global
// format after the last op.
template <class TP>
__device__ __forceinline__ void consume_tile(unsigned char* smem, const TileOp* __restrict__ ops, int nops,
                                             const typename TP::M::Coef* __restrict__ coefs,
                                             const uint8_t* __restrict__ perm_tables, int fmt,
                                             const typename TP::Phase* __restrict__ phase_tab, int tile_log,
                                             uint64_t base, int tid) {
  using RT = RegTile<TP>;
  RT rt;
  const int rb = tile_log < RT::RB ? tile_log : RT::RB;
  bool first = true;
  for (int o = 0; o < nops; ++o) {
    const TileOp& op = ops[o];
    if (op.kind == TOP_POLY) {  // the run's own terms carry their tile predicates
      if (rt.active) rt.poly(ops + o, base, phase_tab);
      o += op.k > 0 ? op.k - 1 : 0;
      continue;
    }
    if ((base & op.gmask) != op.gpat) continue;
    if (!rt.active && op.kind != TOP_LAYOUT && op.kind != TOP_PERM) continue;
    const typename RT::Coef* cf = coefs + op.coef;
    switch (op.kind) {
      case TOP_LAYOUT:
        if (first) {
          rt.set_layout(op.tpos, rb, tile_log, tid);
          rt.read_glob(smem, (fmt & kTileInFF) != 0);
          first = false;
        } else {
          consumers_sync();
          rt.write_sm(smem);
          consumers_sync();
          rt.set_layout(op.tpos, rb, tile_log, tid);
          rt.read_sm(smem);
        }
        break;
      case TOP_DENSE1:
        if (op.lmask == 0) {
          if (op.nloc) dense1_k<RT, false, true>(rt, op.tpos[0], cf, 0);
          else dense1_k<RT, false, false>(rt, op.tpos[0], cf, 0);
        } else {
          if (op.nloc) dense1_k<RT, true, true>(rt, op.tpos[0], cf, op.lmask);
          else dense1_k<RT, true, false>(rt, op.tpos[0], cf, op.lmask);
        }
        break;
      case TOP_XSWAP:
      case TOP_Y: {
        const bool y = op.kind == TOP_Y;
        switch (op.tpos[0]) {
          case 0: rt.template xswap<0>(y, op.lmask); break;
          case 1: rt.template xswap<1>(y, op.lmask); break;
          case 2: if constexpr (RT::RB > 2) rt.template xswap<(RT::RB > 2 ? 2 : 0)>(y, op.lmask); break;
          default: if constexpr (RT::RB > 3) rt.template xswap<(RT::RB > 3 ? 3 : 0)>(y, op.lmask); break;
        }
        break;
      }
      case TOP_DENSE2:
        switch (op.tpos[0]) {
          case 0: dense2_k1<RT, 0>(rt, op.tpos[1], cf, op.lmask, op.tj); break;
          case 1: dense2_k1<RT, 1>(rt, op.tpos[1], cf, op.lmask, op.tj); break;
          case 2: if constexpr (RT::RB > 2) dense2_k1<RT, (RT::RB > 2 ? 2 : 0)>(rt, op.tpos[1], cf, op.lmask, op.tj); break;
          default: if constexpr (RT::RB > 3) dense2_k1<RT, (RT::RB > 3 ? 3 : 0)>(rt, op.tpos[1], cf, op.lmask, op.tj); break;
        }
        break;
      case TOP_PHASE:
        rt.phase(cf, op.lmask, op.lpat, false);
        break;
      case TOP_NEG:
        rt.phase(cf, op.lmask, op.lpat, true);
        break;
      case TOP_DIAG:
        rt.diag(op, cf, base);
        break;
      case TOP_PERM:
        rt.perm(op, perm_tables + op.ptab, smem);
        break;
      case TOP_SWAPBITS:
        rt.swap_bits(op.tpos[0], op.tpos[1]);
        break;
    }
  }
  consumers_sync();
  rt.write_glob(smem, (fmt & kTileOutFF) != 0);
}

}  // namespace qs
