// Fused-block kernel and host fuser.
//
// k_tile is persistent (one or two CTAs per SM).  A producer (a warp of its
// own, or consumer thread 0 between its tiles for float-float blocks with
// 4x4 ops) streams tiles between HBM and shared memory with bulk asynchronous
// copies (cp.async.bulk, the TMA engine) — one copy per contiguous chunk, completion
// tracked by mbarrier transaction counts — through a ring of kStages buffers.
// Eight consumer warps apply the block's gates to the tile in shared memory,
// one gate after another, and hand the buffer back; the producer writes it to
// HBM with bulk stores and refills it.  Loads, arithmetic and stores of
// different tiles overlap, and the state is read and written once per block
// however many gates the block holds (gate fusion / cache blocking, Sec. I).
//
// Complex128 tiles are converted once on arrival to float-float form (head
// and tail FP32 pairs, same 16 bytes) so every gate of the block runs on the
// FP32 pipes without re-splitting doubles; they are rounded back to IEEE
// double once before the store.
//
// Every wait is bounded (qs_set_wait_limit, 2 s of %globaltimer by default):
// on expiry the kernel records QS_ERR_TIMEOUT's code in the state's device
// error word, all warps agree to stop, the producer waits for the copies it
// issued, and the kernel returns.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <unordered_map>
#include <vector>

#include "qs_internal.h"
#include "qs_math.cuh"
#include "qs_tile.cuh"
#include "qs_tile_dev.cuh"
#include "qs_fuser.h"
#include "qs_densefuse.h"
#include "qs_matfuse.h"

namespace qs {

template <class TP>
__global__ void __launch_bounds__(tile_threads<TP>(), kTileMinCtas) k_tile(typename TP::Glob* __restrict__ psi,
                                                       const __grid_constant__ TilePlan<typename TP::M::Coef> plan,
                                                       uint32_t* __restrict__ err) {
  using Glob = typename TP::Glob;
  using Sm = typename TP::Sm;
  static_assert(sizeof(Glob) == sizeof(Sm), "in-place tile conversion");
  extern __shared__ __align__(128) unsigned char smem[];
  const uint32_t tile_amps = 1u << (plan.L + plan.m);
  const uint32_t tile_bytes = tile_amps * (uint32_t)sizeof(Glob);
  const uint32_t chunk_amps = 1u << plan.L;
  const uint32_t chunk_bytes = chunk_amps * (uint32_t)sizeof(Glob);
  const uint32_t n_chunks = 1u << plan.m;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * tile_bytes);
  uint64_t* done = full + kStages;
  // The block's ops and coefficients, staged once per CTA where the policy
  // asks for it: every thread reads them for every tile, and shared-memory
  // vector loads beat constant-bank loads with run-time indices.
  TileOp* s_ops = reinterpret_cast<TileOp*>(done + kStages);
  using Coef = typename TP::M::Coef;
  Coef* s_coefs = reinterpret_cast<Coef*>(s_ops + plan.nops);
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&done[s], kTileConsumers);
    }
    mbar_fence_init();
  }
  {
    static_assert(sizeof(TileOp) % 16 == 0 && sizeof(Coef) % 16 == 0, "16-byte staging");
    if (TP::kStagePlan) {
      const uint4* so = reinterpret_cast<const uint4*>(plan.ops);
      uint4* d = reinterpret_cast<uint4*>(s_ops);
      const int n_op16 = plan.nops * (int)(sizeof(TileOp) / 16);
      for (int i = tid; i < n_op16; i += blockDim.x) d[i] = so[i];
      const uint4* sc = reinterpret_cast<const uint4*>(plan.coefs);
      uint4* dc = reinterpret_cast<uint4*>(s_coefs);
      const int n_cf16 = plan.ncoefs * (int)(sizeof(Coef) / 16);
      for (int i = tid; i < n_cf16; i += blockDim.x) dc[i] = sc[i];
    }
  }
  __syncthreads();

  if constexpr (TP::kFoldProducer) {
    // ------------- consumers; thread 0 also moves the tiles -------------
    // This CTA's tiles are tau = blockIdx.x + j * gridDim.x, j < n_mine.
    // Tiles j + 1 .. j + kAhead are in flight while tile j is consumed;
    // after tile j, thread 0 waits until every consumer is done with it,
    // stores it, and loads tile j + kAhead into the stage that tile j - 1
    // left (whose store has read it by then: at most one store group, tile
    // j's, may still be reading).  Warp 0's other lanes wait at __syncwarp.
    constexpr uint32_t kAhead = kStages - 1;
    const uint32_t n_mine =
        plan.n_tiles > blockIdx.x ? (uint32_t)((plan.n_tiles - 1 - blockIdx.x) / gridDim.x + 1) : 0u;
    auto tile_at = [&](uint32_t j) {
      return tile_base(blockIdx.x + (uint64_t)j * gridDim.x, plan.L, plan.m, plan.base_high);
    };
    auto issue_load = [&](uint32_t j) {
      const int s = (int)(j % kStages);
      unsigned char* buf = smem + (size_t)s * tile_bytes;
      const uint64_t b = tile_at(j);
      mbar_expect_tx(&full[s], tile_bytes);
      for (uint32_t c = 0; c < n_chunks; ++c)
        bulk_load(buf + (size_t)c * chunk_bytes, psi + b + plan.chunk_off[c], chunk_bytes, &full[s]);
    };
    uint32_t loads_issued = 0;
    if (tid == 0)
      for (; loads_issued < n_mine && loads_issued < kAhead; ++loads_issued) issue_load(loads_issued);
    bool stop = false;  // thread 0: a wait of the copying role gave up
    uint32_t j = 0;
    for (; j < n_mine; ++j) {
      const int s = (int)(j % kStages);
      const bool ok = mbar_wait(&full[s], (j / kStages) & 1u, err, plan.wait_ns);
      if (consumers_any(!ok || stop)) break;
      Sm* t = reinterpret_cast<Sm*>(smem + (size_t)s * tile_bytes);
      consume_tile<TP>(reinterpret_cast<unsigned char*>(t), s_ops, plan.nops, s_coefs, plan.perm, plan.fmt,
                       static_cast<const typename TP::Phase*>(plan.phase_tab), plan.L + plan.m, tile_at(j), tid);
      fence_async_smem();
      mbar_arrive(&done[s]);
      if (tid == 0) {
        if (!mbar_wait(&done[s], (j / kStages) & 1u, err, plan.wait_ns)) {
          stop = true;
        } else {
          const uint64_t b = tile_at(j);
          unsigned char* buf = smem + (size_t)s * tile_bytes;
          for (uint32_t c = 0; c < n_chunks; ++c)
            bulk_store(psi + b + plan.chunk_off[c], buf + (size_t)c * chunk_bytes, chunk_bytes);
          bulk_commit();
          if (loads_issued < n_mine) {
            bulk_wait_read_one();
            issue_load(loads_issued++);
          }
        }
      }
      __syncwarp();
    }
    if (tid == 0) {
      // After an early stop, let the loads still in flight land (bounded;
      // they are plain in-range reads) before shared memory goes away.
      for (uint32_t jj = j; jj < loads_issued; ++jj) {
        const int s = (int)(jj % kStages);
        const uint64_t t0 = global_ns();
        while (!mbar_try(&full[s], (jj / kStages) & 1u) && global_ns() - t0 < kDrainNs) {
        }
      }
      bulk_wait_all();
    }
    return;
  }

  if (tid >= kTileConsumers) {
    // ---------------- producer ----------------
    if (tid != kTileConsumers) return;
    uint32_t j = 0;
    bool ok = true;
    uint32_t loads_issued = 0;
    for (;; ++j) {
      const uint64_t tau = blockIdx.x + (uint64_t)j * gridDim.x;
      if (tau >= plan.n_tiles) break;
      const int s = (int)(j % kStages);
      unsigned char* buf = smem + (size_t)s * tile_bytes;
      if (j >= (uint32_t)kStages) {
        const uint32_t jp = j - kStages;
        if (!mbar_wait(&done[s], (jp / kStages) & 1u, err, plan.wait_ns)) {
          ok = false;
          break;
        }
        const uint64_t bprev = tile_base(blockIdx.x + (uint64_t)jp * gridDim.x, plan.L, plan.m, plan.base_high);
        for (uint32_t c = 0; c < n_chunks; ++c)
          bulk_store(psi + bprev + plan.chunk_off[c], buf + (size_t)c * chunk_bytes, chunk_bytes);
        bulk_commit();
        bulk_wait_read_all();
      }
      const uint64_t b = tile_base(tau, plan.L, plan.m, plan.base_high);
      mbar_expect_tx(&full[s], tile_bytes);
      for (uint32_t c = 0; c < n_chunks; ++c)
        bulk_load(buf + (size_t)c * chunk_bytes, psi + b + plan.chunk_off[c], chunk_bytes, &full[s]);
      ++loads_issued;
    }
    const uint32_t count = j;  // tiles whose loads were issued
    if (ok) {
      const uint32_t first = count > (uint32_t)kStages ? count - kStages : 0u;
      for (uint32_t jj = first; jj < count; ++jj) {
        const int s = (int)(jj % kStages);
        if (!mbar_wait(&done[s], (jj / kStages) & 1u, err, plan.wait_ns)) {
          ok = false;
          break;
        }
        const uint64_t b = tile_base(blockIdx.x + (uint64_t)jj * gridDim.x, plan.L, plan.m, plan.base_high);
        unsigned char* buf = smem + (size_t)s * tile_bytes;
        for (uint32_t c = 0; c < n_chunks; ++c)
          bulk_store(psi + b + plan.chunk_off[c], buf + (size_t)c * chunk_bytes, chunk_bytes);
        bulk_commit();
      }
    }
    if (!ok) {
      // Let every load this CTA issued land before the CTA's shared memory
      // goes away (bounded; the copies are plain in-range reads).
      const uint32_t first = loads_issued > (uint32_t)kStages ? loads_issued - kStages : 0u;
      for (uint32_t jj = first; jj < loads_issued; ++jj) {
        const int s = (int)(jj % kStages);
        const uint64_t t0 = global_ns();
        while (!mbar_try(&full[s], (jj / kStages) & 1u) && global_ns() - t0 < kDrainNs) {
        }
      }
    }
    bulk_wait_all();
    return;
  }

  // ---------------- consumers ----------------
  for (uint32_t j = 0;; ++j) {
    const uint64_t tau = blockIdx.x + (uint64_t)j * gridDim.x;
    if (tau >= plan.n_tiles) break;
    const int s = (int)(j % kStages);
    const bool ok = mbar_wait(&full[s], (j / kStages) & 1u, err, plan.wait_ns);
    if (consumers_any(!ok)) break;
    Sm* t = reinterpret_cast<Sm*>(smem + (size_t)s * tile_bytes);
    const uint64_t base = tile_base(tau, plan.L, plan.m, plan.base_high);
    consume_tile<TP>(reinterpret_cast<unsigned char*>(t), TP::kStagePlan ? s_ops : plan.ops, plan.nops,
                     TP::kStagePlan ? s_coefs : plan.coefs, plan.perm, plan.fmt,
                     static_cast<const typename TP::Phase*>(plan.phase_tab), plan.L + plan.m, base, tid);
    fence_async_smem();
    mbar_arrive(&done[s]);
  }
}

// ---------------------------------------------------------------------------
// Host: blocks -> plans -> launches
// ---------------------------------------------------------------------------
namespace {

using namespace fuser;

#ifndef QS_PERM_MAX_HIGH
#define QS_PERM_MAX_HIGH 6
#endif
constexpr int kPermMaxHigh = QS_PERM_MAX_HIGH;  // high qubits of a permutation-only block
constexpr int kMinChunkLog128 = 3;  // chunks of at least 128 bytes
constexpr int kMinChunkLog64 = 4;

static_assert(sizeof(TilePlan<MathDF::Coef>) <= 32764 && sizeof(TilePlan<MathF64::Coef>) <= 32764 &&
                  sizeof(TilePlan<MathF32::Coef>) <= 32764,
              "a plan must fit the kernel parameter space");

template <class Coef>
void fill_plan(TilePlan<Coef>* plan, int n, const BlockOut<Coef>& bo) {
  const Geom& g = bo.geom;
  std::memset(plan, 0, sizeof(*plan));
  plan->n = n;
  plan->L = g.L;
  plan->m = g.m;
  plan->n_tiles = 1ull << (n - g.L - g.m);
  for (int j = 0; j < g.m; ++j) plan->base_high[j] = ~((1ull << g.hq[j]) - 1ull);
  for (int c = 0; c < (1 << g.m); ++c) {
    uint64_t off = 0;
    for (int j = 0; j < g.m; ++j)
      if ((c >> j) & 1) off |= 1ull << g.hq[j];
    plan->chunk_off[c] = off;
  }
  plan->nops = (int)bo.ops.size();
  plan->ncoefs = (int)bo.coefs.size();
  plan->fmt = 0;
  std::memcpy(plan->ops, bo.ops.data(), bo.ops.size() * sizeof(TileOp));
  std::memcpy(plan->coefs, bo.coefs.data(), bo.coefs.size() * sizeof(Coef));
  if (!bo.perm.empty()) std::memcpy(plan->perm, bo.perm.data(), bo.perm.size());
}

template <class TP>
qs_status launch_plan_as(qs_state s, const TilePlan<typename TP::M::Coef>& plan) {
  using Coef = typename TP::M::Coef;
  const size_t tile_bytes = sizeof(typename TP::Glob) << (plan.L + plan.m);
  const size_t smem = kStages * tile_bytes + 2 * kStages * sizeof(uint64_t) +
                      (TP::kStagePlan ? (size_t)plan.nops * sizeof(TileOp) + (size_t)plan.ncoefs * sizeof(Coef) : 0);
  auto kern = k_tile<TP>;
  // The dynamic shared-memory limit is a property of the function: set it
  // once to the largest tile so that launches with any tile size are valid.
  static std::mutex mu;
  static bool attr_set = false;
  static std::unordered_map<int, int> occ_cache;
  int occ = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!attr_set) {
      const size_t max_smem = kStages * ((size_t)sizeof(typename TP::Glob) << TP::kTileLog) +
                              2 * kStages * sizeof(uint64_t) + kTileMaxOps * sizeof(TileOp) + kTileMaxCoefBytes;
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_smem);
      if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_tile)");
      attr_set = true;
    }
    const int key = (int)smem;
    auto it = occ_cache.find(key);
    if (it == occ_cache.end()) {
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, tile_threads<TP>(), smem) != cudaSuccess || occ < 1)
        occ = 1;
      occ_cache[key] = occ;
    } else {
      occ = it->second;
    }
  }
  const uint64_t full = (uint64_t)sm_count(s->device) * occ;
  const unsigned grid = (unsigned)(plan.n_tiles < full ? plan.n_tiles : full);
  uint32_t* err = error_word(s);
  if (!err) return fail(QS_ERR_CUDA, "device error word unavailable");
  kern<<<grid, tile_threads<TP>(), smem, s->stream>>>((typename TP::Glob*)s->psi, plan, err);
  ++s->run_fused_launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(QS_ERR_CUDA, "k_tile launch (grid %u, smem %zu, plan %zu bytes, %d ops, L %d, m %d): %s", grid, smem,
                sizeof(plan), plan.nops, plan.L, plan.m, cudaGetErrorString(e));
  return QS_OK;
}

// Float-float blocks with 4x4 ops run with warp 0 as the producer (no
// spills in the 4x4 rows); the others keep the producer warp.
template <class TP>
qs_status launch_plan(qs_state s, const TilePlan<typename TP::M::Coef>& plan) {
  if constexpr (std::is_same<TP, TileDF>::value) {
    for (int i = 0; i < plan.nops; ++i)
      if (plan.ops[i].kind == TOP_DENSE2) return launch_plan_as<TileDFFold>(s, plan);
  }
  return launch_plan_as<TP>(s, plan);
}

qs_status dispatch_single(qs_state s, const FGate& g) {
  if (g.kind == kGatePattern) return launch_phase(s, g.pmask, g.ppat, g.data[0], g.data[1]);
  if (g.kind == QS_GATE_PERM) return dispatch_perm(s, g.targets, g.k, g.ctrl, g.perm);
  if (g.kind == QS_GATE_DIAG) return dispatch_diag(s, g.targets, g.k, g.ctrl, g.data);
  if (g.kind == QS_GATE_U1) return dispatch_u1(s, g.targets[0], g.ctrl, g.data);
  return dispatch_uk(s, g.targets, g.k, g.ctrl, g.data);
}

// Translate, schedule and launch one block under policy TP.
template <class TP>
qs_status launch_block(qs_state s, const std::vector<FGate>& gates, const std::vector<size_t>& members,
                       size_t count, const Geom& geom, Limits lim) {
  using Coef = typename TP::M::Coef;
  static thread_local BlockOut<Coef> bo;
  static thread_local std::vector<unsigned char> plan_mem;
  PlanBuilder<typename TP::M> pb(&bo, geom, lim);
  for (size_t i = 0; i < count; ++i)
    if (!pb.add(gates[members[i]])) return fail(QS_ERR_UNSUPPORTED, "block rebuild failed");
  if (bo.ops.empty()) return QS_OK;
  group_terms(bo.ops);
  bo.ops = schedule_layouts(bo.ops, geom.L + geom.m, TP::kRegBits, TP::kBankBits);
  if (bo.ops.size() > (size_t)kTileMaxOps)
    return fail(QS_ERR_UNSUPPORTED, "fused block of %zu ops exceeds %d", bo.ops.size(), kTileMaxOps);
  const void* ptab = phase_table(s->device, TP::kPhaseFormat);
  if (!ptab) return fail(QS_ERR_CUDA, "phase tables missing on device %d", s->device);
  plan_mem.resize(sizeof(TilePlan<Coef>));
  TilePlan<Coef>* plan = reinterpret_cast<TilePlan<Coef>*>(plan_mem.data());
  fill_plan(plan, s->n, bo);
  plan->phase_tab = ptab;
  plan->wait_ns = wait_limit_ns();
  return launch_plan<TP>(s, *plan);
}

template <class TP>
qs_status run_blocks(qs_state s, const std::vector<FGate>& gates, int max_high) {
  using Coef = typename TP::M::Coef;
  // Float-float blocks that follow one another keep the state in head +
  // tail float form in HBM between them (16 bytes per amplitude, like the
  // doubles): only the first reads doubles and only the last writes them.
  constexpr bool kChain = std::is_same<TP, TileDF>::value;
  const int n = s->n;
  const int min_chunk = sizeof(typename TP::Glob) == 16 ? kMinChunkLog128 : kMinChunkLog64;
  // Scheduling adds at most one layout change per non-diagonal gate (weight
  // 2 in the op budget; diagonal gates weigh 1), plus one bank-friendly
  // layout before the first op and one after the last.
  // Staged plans keep their coefficients within kTileMaxCoefBytes of shared
  // memory; plans read from the parameter bank take the whole pool.
  const int max_coefs = TP::kStagePlan ? std::min(kTileMaxCoefs, kTileMaxCoefBytes / (int)sizeof(Coef)) : kTileMaxCoefs;
  const Limits lim{kTileMaxOps - 2, max_coefs, kTileMaxPermBytes};
  const void* ptab = phase_table(s->device, TP::kPhaseFormat);
  if (!ptab) return fail(QS_ERR_CUDA, "phase tables missing on device %d", s->device);
  static thread_local std::vector<unsigned char> plan_mem[2];
  plan_mem[0].resize(sizeof(TilePlan<Coef>));
  plan_mem[1].resize(sizeof(TilePlan<Coef>));
  TilePlan<Coef>* plan = reinterpret_cast<TilePlan<Coef>*>(plan_mem[0].data());
  TilePlan<Coef>* pend = reinterpret_cast<TilePlan<Coef>*>(plan_mem[1].data());
  bool pend_valid = false;
  // Launch the held plan; its output stays in float-float form when the
  // next launch is a float-float plan too.
  auto flush = [&](bool next_chained) -> qs_status {
    if (!pend_valid) return QS_OK;
    pend_valid = false;
    if (next_chained) pend->fmt |= kTileOutFF;
    return launch_plan<TP>(s, *pend);
  };
  BlockOut<Coef> bo;
  std::vector<char> taken(gates.size(), 0);
  size_t next = 0;
  while (next < gates.size()) {
    if (taken[next]) {
      ++next;
      continue;
    }
    Geom geom;
    std::vector<size_t> members;
    if (gates[next].kind == QS_GATE_PERM && max_high < kPermMaxHigh) {
      // Runs of permutations (the swap networks of QFTs) move amplitudes
      // only: give them more high qubits than arithmetic blocks take.
      members = choose_block(gates, taken, next, n, TP::kTileLog, kPermMaxHigh, min_chunk, lim, 512, &geom, true);
      if (members.size() <= 1) members.clear();
    }
    if (members.empty())
      members = choose_block(gates, taken, next, n, TP::kTileLog, max_high, min_chunk, lim, 512, &geom);
    // A gate that fits no tile, or a block of one gate (staging gains
    // nothing), runs on the per-gate kernels.
    size_t emitted = 0;
    if (members.size() > 1) {
      PlanBuilder<typename TP::M> pb(&bo, geom, lim);
      for (size_t idx : members) {
        if (!pb.add(gates[idx])) break;
        taken[idx] = 1;
        ++emitted;
      }
    }
    if (emitted == 0) {
      qs_status st = flush(false);
      ++s->run_gate_launches;
      if (st == QS_OK) st = dispatch_single(s, gates[next]);
      if (st != QS_OK) return st;
      taken[next] = 1;
      continue;
    }
    if (bo.ops.empty()) continue;
    group_terms(bo.ops);
    bo.ops = schedule_layouts(bo.ops, geom.L + geom.m, TP::kRegBits, TP::kBankBits);
    if (bo.ops.size() > (size_t)kTileMaxOps)
      return fail(QS_ERR_UNSUPPORTED, "fused block of %zu ops exceeds %d", bo.ops.size(), kTileMaxOps);
    if (kChain && !pend_valid && moves_only(bo.ops)) {
      // Moves and sign flips are exact in any policy: outside a float-float
      // chain the FP64 tile skips the conversions (same tile size and
      // layouts).
      static_assert(TileF64::kTileLog == TileDF::kTileLog && TileF64::kRegBits == TileDF::kRegBits,
                    "move-only blocks reuse the float-float geometry");
      qs_status st = launch_block<TileF64>(s, gates, members, emitted, geom, lim);
      if (st != QS_OK) return st;
      continue;
    }
    fill_plan(plan, n, bo);
    plan->phase_tab = ptab;
    plan->wait_ns = wait_limit_ns();
    const bool chained = kChain && pend_valid;
    qs_status st = flush(kChain);
    if (st != QS_OK) return st;
    if (chained) plan->fmt |= kTileInFF;
    std::swap(plan, pend);
    pend_valid = true;
  }
  return flush(false);
}

}  // namespace

qs_status run_fused(qs_state s, const qs_circuit* c, int max_high) {
  std::vector<FGate> gates;
  gates.reserve((size_t)c->n_gates);
  for (int64_t i = 0; i < c->n_gates; ++i) gates.push_back(normalise(c, c->gates[i]));
  XPusher xp;   // owns conjugated tables until the blocks are launched
  gates = xp.run(gates);
  // Dense blocks first, on the circuit's own order (the 1q/2q fusion below
  // moves pending small gates next to the gates that close them).
  DenseFuser df;  // owns the composed dense blocks until they are launched
  gates = df.run(gates);
  s->run_dense_blocks += df.blocks();
  s->run_dense_gates += df.absorbed();
  MatFuser mf;  // owns the fused matrices until the blocks are launched
  gates = mf.run(gates);
  if (max_high > kTileMaxHigh) max_high = kTileMaxHigh;
  if (s->dtype == QS_C64) return run_blocks<TileF32>(s, gates, max_high);
  if (s->math == QS_MATH_FP64) return run_blocks<TileF64>(s, gates, max_high);
  return run_blocks<TileDF>(s, gates, max_high);
}

}  // namespace qs
