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

constexpr int kTileConsumers = 256;
constexpr int kTileThreads = kTileConsumers + 32;
constexpr int kStages = 3;
constexpr uint64_t kWaitNs = 2000000000ull;

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
// Bounded wait: false when it gave up (timeout recorded, or another thread
// already recorded an error).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t* err) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try(bar, parity)) {
    if (*(volatile uint32_t*)err != 0u) return false;
    if (global_ns() - t0 > kWaitNs) {
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
  using Glob = float2;
  using Sm = float2;
  static constexpr int kTileLog = 12;  // 4096 amplitudes, 32 KB
  static constexpr int kIlp = 4;
  static __device__ __forceinline__ Sm to_sm(Glob g) { return g; }
  static __device__ __forceinline__ Glob from_sm(Sm s) { return s; }
  static __device__ __forceinline__ M::Val val(Sm s) { return M::load(s); }
  template <int K>
  static __device__ __forceinline__ Sm mac(const M::Coef* c, const M::Val* v) { return M::mac_round<K>(c, v); }
  static __device__ __forceinline__ Sm neg(Sm a) {
    return make_float2(__uint_as_float(__float_as_uint(a.x) ^ 0x80000000u),
                       __uint_as_float(__float_as_uint(a.y) ^ 0x80000000u));
  }
  // -i (x + iy) = y - ix
  static __device__ __forceinline__ Sm mul_minus_i(Sm a) { return make_float2(a.y, -a.x); }
  static __device__ __forceinline__ Sm mul_i(Sm a) { return make_float2(-a.y, a.x); }
};

__device__ __forceinline__ double dneg(double x) {
  return __hiloint2double(__double2hiint(x) ^ (int)0x80000000u, __double2loint(x));
}

struct TileF64 {
  using M = MathF64;
  using Glob = double2;
  using Sm = double2;
  static constexpr int kTileLog = 11;  // 2048 amplitudes, 32 KB
  static constexpr int kIlp = 2;
  static __device__ __forceinline__ Sm to_sm(Glob g) { return g; }
  static __device__ __forceinline__ Glob from_sm(Sm s) { return s; }
  static __device__ __forceinline__ M::Val val(Sm s) { return M::load(s); }
  template <int K>
  static __device__ __forceinline__ Sm mac(const M::Coef* c, const M::Val* v) { return M::mac_round<K>(c, v); }
  static __device__ __forceinline__ Sm neg(Sm a) { return make_double2(dneg(a.x), dneg(a.y)); }
  static __device__ __forceinline__ Sm mul_minus_i(Sm a) { return make_double2(a.y, dneg(a.x)); }
  static __device__ __forceinline__ Sm mul_i(Sm a) { return make_double2(dneg(a.y), a.x); }
};

// Float-float tile element: (re_h, im_h, re_l, im_l), |l| <= ulp(h)/2.
struct TileDF {
  using M = MathDF;
  using Glob = double2;
  using Sm = float4;
  static constexpr int kTileLog = 11;
  static constexpr int kIlp = 2;
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
    // TwoSum(S, C) -> normalised head and tail
    const float2 s = add2(a.S, a.C);
    const float2 bb = sub2(s, a.S);
    const float2 e = add2(sub2(a.S, sub2(s, bb)), sub2(a.C, bb));
    return make_float4(s.x, s.y, e.x, e.y);
  }
  static __device__ __forceinline__ float fneg(float x) { return __uint_as_float(__float_as_uint(x) ^ 0x80000000u); }
  static __device__ __forceinline__ Sm neg(Sm a) { return make_float4(fneg(a.x), fneg(a.y), fneg(a.z), fneg(a.w)); }
  static __device__ __forceinline__ Sm mul_minus_i(Sm a) { return make_float4(a.y, fneg(a.x), a.w, fneg(a.z)); }
  static __device__ __forceinline__ Sm mul_i(Sm a) { return make_float4(fneg(a.y), a.x, fneg(a.w), a.z); }
};

// ---------------------------------------------------------------------------
// Kernel
// ---------------------------------------------------------------------------
// Local item index -> local amplitude index: insert a zero at each listed
// position (adding the bits at and above a position shifts them up by one),
// then set the fixed bits.  The first four masks live in registers.
struct LocalExpand {
  int npos;
  uint32_t h0, h1, h2, h3, fixed;
  const TileOp* op;
  __device__ __forceinline__ explicit LocalExpand(const TileOp& o)
      : npos(o.npos), h0(o.himask[0]), h1(o.himask[1]), h2(o.himask[2]), h3(o.himask[3]), fixed(o.ifixed), op(&o) {}
  __device__ __forceinline__ uint32_t operator()(uint32_t i) const {
    if (npos > 0) i += i & h0;
    if (npos > 1) i += i & h1;
    if (npos > 2) i += i & h2;
    if (npos > 3) i += i & h3;
    for (int p = 4; p < npos; ++p) i += i & op->himask[p];
    return i | fixed;
  }
};

// Global index of a tile's first amplitude: the tile number spread over the
// free qubits (zeros inserted at the high tile qubits, ascending).
__device__ __forceinline__ uint64_t tile_base(uint64_t tau, int L, int m, const uint64_t* base_high) {
  uint64_t b = tau << L;
  for (int j = 0; j < m; ++j) b += b & base_high[j];
  return b;
}

template <class TP>
__device__ __forceinline__ void apply_op(typename TP::Sm* __restrict__ t, const TileOp& op,
                                         const typename TP::M::Coef* __restrict__ coefs,
                                         const uint8_t* __restrict__ perm_tables, uint32_t tile_amps, uint64_t base,
                                         int tid) {
  using Sm = typename TP::Sm;
  using Val = typename TP::M::Val;
  using Coef = typename TP::M::Coef;
  constexpr int U = TP::kIlp;  // independent items in flight per thread
  const Coef* cf = coefs + op.coef;
  const LocalExpand ex(op);
  const uint32_t items = tile_amps >> op.npos;
  const uint32_t step = (uint32_t)kTileConsumers * U;
  switch (op.kind) {
    case TOP_DENSE1: {
      const uint32_t tb = 1u << op.tpos[0];
      Coef c[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) c[j] = cf[j];
      for (uint32_t it0 = tid; it0 < items; it0 += step) {
        uint32_t ii[U];
        Sm a[U], b[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (it0 + u * kTileConsumers < items) {
            ii[u] = ex(it0 + u * kTileConsumers);
            a[u] = t[ii[u]];
            b[u] = t[ii[u] | tb];
          }
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (it0 + u * kTileConsumers < items) {
            const Val v[2] = {TP::val(a[u]), TP::val(b[u])};
            t[ii[u]] = TP::template mac<2>(c, v);
            t[ii[u] | tb] = TP::template mac<2>(c + 2, v);
          }
      }
      break;
    }
    case TOP_DENSE2: {
      const uint32_t b0 = 1u << op.tpos[0], b1 = 1u << op.tpos[1];
      for (uint32_t it = tid; it < items; it += kTileConsumers) {
        const uint32_t i = ex(it);
        const Val v[4] = {TP::val(t[i]), TP::val(t[i | b0]), TP::val(t[i | b1]), TP::val(t[i | b0 | b1])};
        t[i] = TP::template mac<4>(cf, v);
        t[i | b0] = TP::template mac<4>(cf + 4, v);
        t[i | b1] = TP::template mac<4>(cf + 8, v);
        t[i | b0 | b1] = TP::template mac<4>(cf + 12, v);
      }
      break;
    }
    case TOP_PHASE: {
      const Coef c = cf[0];
      for (uint32_t it0 = tid; it0 < items; it0 += step) {
        uint32_t ii[U];
        Sm a[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (it0 + u * kTileConsumers < items) {
            ii[u] = ex(it0 + u * kTileConsumers);
            a[u] = t[ii[u]];
          }
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (it0 + u * kTileConsumers < items) {
            const Val v = TP::val(a[u]);
            t[ii[u]] = TP::template mac<1>(&c, &v);
          }
      }
      break;
    }
    case TOP_NEG: {
      for (uint32_t it = tid; it < items; it += kTileConsumers) {
        const uint32_t i = ex(it);
        t[i] = TP::neg(t[i]);
      }
      break;
    }
    case TOP_DIAG: {
      uint32_t sg = 0;
      for (int j = 0; j < op.k; ++j)
        if (op.gq[j] != 0xFF) sg |= (uint32_t)((base >> op.gq[j]) & 1ull) << j;
      for (uint32_t it0 = tid; it0 < items; it0 += step) {
        uint32_t ii[U];
        Sm a[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (it0 + u * kTileConsumers < items) {
            ii[u] = ex(it0 + u * kTileConsumers);
            a[u] = t[ii[u]];
          }
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (it0 + u * kTileConsumers < items) {
            uint32_t sidx = sg;
            for (int j = 0; j < op.nloc; ++j) sidx |= ((ii[u] >> op.tpos[j]) & 1u) << op.tj[j];
            const Val v = TP::val(a[u]);
            t[ii[u]] = TP::template mac<1>(cf + sidx, &v);
          }
      }
      break;
    }
    case TOP_XSWAP:
    case TOP_Y: {
      const uint32_t tb = 1u << op.tpos[0];
      const bool y = op.kind == TOP_Y;
      for (uint32_t it = tid; it < items; it += kTileConsumers) {
        const uint32_t i = ex(it);
        const Sm a = t[i], b = t[i | tb];
        t[i] = y ? TP::mul_minus_i(b) : b;
        t[i | tb] = y ? TP::mul_i(a) : a;
      }
      break;
    }
    case TOP_PERM: {
      // Two phases through registers: gather every destination's source,
      // then write, so the permutation is applied in place.
      constexpr int kMaxPer = (1 << TP::kTileLog) / kTileConsumers;
      Sm buf[kMaxPer];
      const uint8_t* inv = perm_tables + op.ptab;
#pragma unroll
      for (int r = 0; r < kMaxPer; ++r) {
        const uint32_t d = (uint32_t)tid + (uint32_t)r * kTileConsumers;
        if (d < tile_amps) {
          uint32_t src = d;
          if ((d & op.lmask) == op.lmask) {
            uint32_t sidx = 0;
            for (int j = 0; j < op.k; ++j) sidx |= ((d >> op.tpos[j]) & 1u) << j;
            const uint32_t sv = inv[sidx];
            for (int j = 0; j < op.k; ++j) src = (src & ~(1u << op.tpos[j])) | (((sv >> j) & 1u) << op.tpos[j]);
          }
          buf[r] = t[src];
        }
      }
      consumers_sync();
#pragma unroll
      for (int r = 0; r < kMaxPer; ++r) {
        const uint32_t d = (uint32_t)tid + (uint32_t)r * kTileConsumers;
        if (d < tile_amps) t[d] = buf[r];
      }
      break;
    }
  }
}

}  // namespace qs
