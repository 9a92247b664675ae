// Batched execution of many independent states in one persistent launch.
//
// Every state's circuit is compiled on the host into fused blocks (the same
// fuser and tile ops as qs_fuse_run, with no per-block size limits).  States
// are ordered by estimated cost, largest first, and CTAs claim them from a
// global counter, so uneven qubit counts balance across the 152 SMs.  A CTA
// owns a claimed state until its circuit is done: a state no larger than one
// tile is loaded into shared memory once, runs its whole circuit there and
// is written back once; larger states stream through the CTA's tile ring
// block after block (a block's stores complete before the next block's loads
// start, since blocks overlap in memory).
//
// Roles inside a CTA are those of k_tile: a producer thread claims states,
// issues the bulk copies and publishes a small descriptor per tile in shared
// memory; eight consumer warps apply the ops.  Waits are bounded as in k_tile.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <type_traits>
#include <vector>

#include "qs_fuser.h"
#include "qs_matfuse.h"
#include "qs_internal.h"
#include "qs_tile_dev.cuh"

namespace qs {

qs_status check_gate(const qs_state s, const qs_circuit* c, int64_t gi);  // qs_circuit.cu
qs_status run_fused(qs_state s, const qs_circuit* c, int max_high);          // qs_tile.cu
int fuse_width_for(qs_state s);                                              // qs_circuit.cu

// Widest state that the batched launches take (single-tile states whole on
// one CTA, wider ones block by block over the grid); wider states run as
// fused whole-GPU blocks.
constexpr int kBatchLocalMax = 20;

struct BatchBlock {
  int L, m, nops, fmt;  // fmt: kTileInFF / kTileOutFF (float-float state between a state's blocks)
  uint32_t op0, coef0, perm0, ncoefs;
  uint64_t n_tiles;
  uint64_t base_high[kTileMaxHigh];
  int8_t hq[kTileMaxHigh];
};

// A work item: blocks block0 .. block0 + nblocks - 1 of one state, in
// order; of each block only tiles tau0 .. tau1 - 1 (clamped to its count).
// resident: the state is one tile under every block: it is loaded once,
// all its blocks run on it in shared memory, and it is stored once.
struct BatchState {
  void* psi;
  uint32_t block0, nblocks;
  uint64_t tau0, tau1;
  uint32_t resident;
  uint32_t pad;
};

struct TileDesc {
  uint32_t block;   // 0xFFFFFFFF: no more work
  uint32_t nchain;  // blocks block .. block + nchain - 1 run on this tile
  uint64_t tau;
};

template <class TP>
struct BatchArgs {
  const BatchState* states;
  const BatchBlock* blocks;
  const TileOp* ops;
  const typename TP::M::Coef* coefs;
  const uint8_t* perm;
  const typename TP::Phase* phase_tab;
  uint32_t n_states;
  uint32_t* counter;  // next state to claim (zeroed before the launch)
  uint32_t* err;
  uint64_t wait_ns;   // limit of each bounded wait
};

// Shared memory for staging one block's plan (as in k_tile: keeps two CTAs
// per SM next to the tile ring).
constexpr size_t kStageBytes = kTileMaxOps * sizeof(TileOp) + kTileMaxCoefBytes;

__device__ __forceinline__ uint64_t chunk_offset(const BatchBlock& b, uint32_t c) {
  uint64_t off = 0;
  for (int j = 0; j < b.m; ++j)
    if ((c >> j) & 1u) off |= 1ull << b.hq[j];
  return off;
}

template <class TP>
__global__ void __launch_bounds__(kTileThreads, kTileMinCtas) k_batch(const BatchArgs<TP> a) {
  using Glob = typename TP::Glob;
  using Sm = typename TP::Sm;
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr uint32_t kMaxTileBytes = (uint32_t)sizeof(Glob) << TP::kTileLog;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kMaxTileBytes);
  uint64_t* done = full + kStages;
  TileDesc* desc = reinterpret_cast<TileDesc*>(done + kStages);
  // Staging area for the current block's ops and coefficients (policies
  // that stage, blocks that fit).
  using Coef = typename TP::M::Coef;
  TileOp* s_ops = reinterpret_cast<TileOp*>(desc + kStages);
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&done[s], kTileConsumers);
    }
    mbar_fence_init();
  }
  __syncthreads();

  if (tid >= kTileConsumers) {
    // ---------------- producer ----------------
    if (tid != kTileConsumers) return;
    bool pending[kStages] = {false, false, false};
    uint32_t pend_block[kStages], pend_j[kStages];
    uint64_t pend_tau[kStages];
    Glob* pend_psi[kStages];
    uint32_t j = 0;
    bool ok = true;
    // Make stage s free: store the tile it holds once the consumers are done.
    auto release = [&](int s) -> bool {
      if (!pending[s]) return true;
      if (!mbar_wait(&done[s], (pend_j[s] / kStages) & 1u, a.err, a.wait_ns)) return false;
      const BatchBlock& b = a.blocks[pend_block[s]];
      const uint32_t chunk_bytes = (uint32_t)sizeof(Glob) << b.L;
      const uint64_t base = tile_base(pend_tau[s], b.L, b.m, b.base_high);
      unsigned char* buf = smem + (size_t)s * kMaxTileBytes;
      for (uint32_t c = 0; c < (1u << b.m); ++c)
        bulk_store(pend_psi[s] + base + chunk_offset(b, c), buf + (size_t)c * chunk_bytes, chunk_bytes);
      bulk_commit();
      bulk_wait_read_all();
      pending[s] = false;
      return true;
    };
    auto drain = [&]() -> bool {
      for (uint32_t jj = (j > (uint32_t)kStages ? j - kStages : 0u); jj < j; ++jj)
        if (!release((int)(jj % kStages))) return false;
      bulk_wait_all();
      asm volatile("fence.proxy.async.global;" ::: "memory");
      return true;
    };
    for (;;) {
      const uint32_t si = atomicAdd(a.counter, 1u);
      if (si >= a.n_states) break;
      const BatchState st = a.states[si];
      if (st.resident) {
        // One tile under every block: one load, the whole chain of blocks on
        // the consumers' side, one store (release() stores with the last
        // block's geometry, which is the first's: L = n, m = 0).
        const BatchBlock& b = a.blocks[st.block0];
        const uint32_t tile_bytes = (uint32_t)sizeof(Glob) << b.L;
        const int s = (int)(j % kStages);
        if (!release(s)) {
          ok = false;
          break;
        }
        desc[s].block = st.block0;
        desc[s].nchain = st.nblocks;
        desc[s].tau = 0;
        pending[s] = true;
        pend_block[s] = st.block0 + st.nblocks - 1;
        pend_j[s] = j;
        pend_tau[s] = 0;
        pend_psi[s] = reinterpret_cast<Glob*>(st.psi);
        mbar_expect_tx(&full[s], tile_bytes);
        bulk_load(smem + (size_t)s * kMaxTileBytes, st.psi, tile_bytes, &full[s]);
        ++j;
        continue;
      }
      for (uint32_t bi = st.block0; bi < st.block0 + st.nblocks && ok; ++bi) {
        // Blocks of one state overlap in memory: finish the previous block.
        if (bi != st.block0 && !drain()) {
          ok = false;
          break;
        }
        const BatchBlock& b = a.blocks[bi];
        const uint32_t chunk_bytes = (uint32_t)sizeof(Glob) << b.L;
        const uint32_t tile_bytes = chunk_bytes << b.m;
        const uint64_t tau_end = st.tau1 < b.n_tiles ? st.tau1 : b.n_tiles;
        for (uint64_t tau = st.tau0; tau < tau_end; ++tau, ++j) {
          const int s = (int)(j % kStages);
          if (!release(s)) {
            ok = false;
            break;
          }
          desc[s].block = bi;
          desc[s].nchain = 1;
          desc[s].tau = tau;
          pending[s] = true;
          pend_block[s] = bi;
          pend_j[s] = j;
          pend_tau[s] = tau;
          pend_psi[s] = reinterpret_cast<Glob*>(st.psi);
          const uint64_t base = tile_base(tau, b.L, b.m, b.base_high);
          unsigned char* buf = smem + (size_t)s * kMaxTileBytes;
          mbar_expect_tx(&full[s], tile_bytes);
          for (uint32_t c = 0; c < (1u << b.m); ++c)
            bulk_load(buf + (size_t)c * chunk_bytes, reinterpret_cast<Glob*>(st.psi) + base + chunk_offset(b, c),
                      chunk_bytes, &full[s]);
        }
      }
      if (!ok) break;
    }
    if (ok) {
      // End marker for the consumers, then store what is still in flight.
      const int s = (int)(j % kStages);
      ok = release(s);
      if (ok) {
        desc[s].block = 0xFFFFFFFFu;
        mbar_arrive(&full[s]);
        ok = drain();
      }
    }
    if (!ok) {
      // Let issued loads land before the CTA exits (bounded).
      for (uint32_t jj = (j > (uint32_t)kStages ? j - kStages : 0u); jj < j; ++jj) {
        const int s = (int)(jj % kStages);
        const uint64_t t0 = global_ns();
        while (!mbar_try(&full[s], (jj / kStages) & 1u) && global_ns() - t0 < kDrainNs) {
        }
      }
      bulk_wait_all();
    }
    return;
  }

  // ---------------- consumers ----------------
  uint32_t staged = 0xFFFFFFFFu;
  for (uint32_t j = 0;; ++j) {
    const int s = (int)(j % kStages);
    const bool ok = mbar_wait(&full[s], (j / kStages) & 1u, a.err, a.wait_ns);
    if (consumers_any(!ok)) break;
    const TileDesc d = desc[s];
    if (d.block == 0xFFFFFFFFu) break;
    Sm* t = reinterpret_cast<Sm*>(smem + (size_t)s * kMaxTileBytes);
    for (uint32_t bi = d.block; bi < d.block + d.nchain; ++bi) {
      const BatchBlock& b = a.blocks[bi];
      const TileOp* ops = a.ops + b.op0;
      const Coef* coefs = a.coefs + b.coef0;
      if (TP::kStagePlan && b.nops * sizeof(TileOp) + b.ncoefs * sizeof(Coef) <= kStageBytes) {
        Coef* s_coefs = reinterpret_cast<Coef*>(s_ops + b.nops);
        if (bi != staged) {  // uniform: every consumer reads the same descriptor
          consumers_sync();  // the previous block's plan (and tile) are no longer read
          const uint4* so = reinterpret_cast<const uint4*>(ops);
          uint4* dst = reinterpret_cast<uint4*>(s_ops);
          const int n_op16 = b.nops * (int)(sizeof(TileOp) / 16);
          for (int i = tid; i < n_op16; i += kTileConsumers) dst[i] = so[i];
          const uint4* sc = reinterpret_cast<const uint4*>(coefs);
          uint4* dc = reinterpret_cast<uint4*>(s_coefs);
          const int n_cf16 = (int)(b.ncoefs * sizeof(Coef) / 16);
          for (int i = tid; i < n_cf16; i += kTileConsumers) dc[i] = sc[i];
          consumers_sync();
          staged = bi;
        } else if (bi != d.block) {
          consumers_sync();  // the previous block's writes to the tile are complete
        }
        ops = s_ops;
        coefs = s_coefs;
      } else if (bi != d.block) {
        consumers_sync();
      }
      const uint64_t base = tile_base(d.tau, b.L, b.m, b.base_high);
      consume_tile<TP>(reinterpret_cast<unsigned char*>(t), ops, b.nops, coefs, a.perm + b.perm0, b.fmt,
                       a.phase_tab, b.L + b.m, base, tid);
    }
    fence_async_smem();
    mbar_arrive(&done[s]);
  }
}

// ---------------------------------------------------------------------------
// Host
// ---------------------------------------------------------------------------
namespace {

using namespace fuser;

// Device image of one compiled batch: work items, blocks, ops, coefficients,
// permutation tables and the claim counters.
struct BatchWork {
  void* dev = nullptr;
  size_t dev_bytes = 0;
  size_t off_states = 0, off_blocks = 0, off_ops = 0, off_coefs = 0, off_perm = 0, off_counter = 0;
  uint32_t n_states = 0;  // work items of the persistent launch (single-tile states)
  // Multi-tile states run in steps: step k applies block k of each of them,
  // its tiles spread over the grid as separate work items (one launch each).
  std::vector<size_t> step_off;
  std::vector<uint32_t> step_n;
};

std::mutex g_batch_mu;
// One-shot batches (qs_batch_run) compile into one workspace per (device,
// stream): reuse is ordered by the stream, so no launch can see a workspace
// that a later call overwrites.
std::map<std::pair<int, cudaStream_t>, BatchWork*> g_oneshot_work;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

template <class TP>
qs_status compile_batch(qs_state* states, const qs_circuit* const* circuits, int count, BatchWork* bw,
                        cudaStream_t stream) {
  using Coef = typename TP::M::Coef;
  const int min_chunk = sizeof(typename TP::Glob) == 16 ? 3 : 4;
  // Every block's plan fits the shared-memory staging area, as in k_tile
  // (a state that is one tile runs its blocks back to back on the tile).
  const Limits lim{kTileMaxOps - 2, std::min(kTileMaxCoefs, kTileMaxCoefBytes / (int)sizeof(Coef)), kTileMaxPermBytes};
  std::vector<BatchState> bstates(count);
  std::memset(bstates.data(), 0, bstates.size() * sizeof(BatchState));
  std::vector<BatchBlock> blocks;
  std::vector<TileOp> ops;
  std::vector<Coef> coefs;
  std::vector<uint8_t> perm;
  std::vector<double> cost(count, 0.0);
  BlockOut<Coef> bo;
  for (int i = 0; i < count; ++i) {
    const qs_state s = states[i];
    const qs_circuit* c = circuits[i];
    std::vector<FGate> gates;
    gates.reserve((size_t)c->n_gates);
    for (int64_t g = 0; g < c->n_gates; ++g) gates.push_back(normalise(c, c->gates[g]));
    XPusher xp;   // conjugated tables and fused matrices live until this
    gates = xp.run(gates);
    MatFuser mf;  // state's blocks are copied out
    gates = mf.run(gates);
    const int max_high = std::max(2, std::min(kTileMaxHigh, fuse_width_for(s)));
    bstates[i].psi = s->psi;
    bstates[i].block0 = (uint32_t)blocks.size();
    bstates[i].tau0 = 0;
    bstates[i].tau1 = ~0ull;
    std::vector<char> taken(gates.size(), 0);
    size_t next = 0;
    while (next < gates.size()) {
      if (taken[next]) {
        ++next;
        continue;
      }
      Geom geom;
      // The fusion width qs_autotune chose for this qubit count (4 untuned):
      // wider blocks take more strided qubits, each halving the contiguous
      // chunk a bulk copy moves.
      std::vector<size_t> members =
          choose_block(gates, taken, next, s->n, TP::kTileLog, max_high, min_chunk, lim, 512, &geom);
      if (members.empty() && max_high < kTileMaxHigh)  // a gate wider than the tuned block
        members = choose_block(gates, taken, next, s->n, TP::kTileLog, kTileMaxHigh, min_chunk, lim, 512, &geom);
      if (members.empty()) return fail(QS_ERR_UNSUPPORTED, "batch state %d: gate %zu fits no tile", i, next);
      PlanBuilder<typename TP::M> pb(&bo, geom, lim);
      size_t emitted = 0;
      for (size_t idx : members) {
        if (!pb.add(gates[idx])) break;
        taken[idx] = 1;
        ++emitted;
      }
      if (emitted == 0) return fail(QS_ERR_UNSUPPORTED, "batch state %d: gate %zu could not be placed", i, next);
      if (bo.ops.empty()) continue;
      group_terms(bo.ops);
      bo.ops = schedule_layouts(bo.ops, geom.L + geom.m, TP::kRegBits, TP::kBankBits);
      if (bo.ops.size() > (size_t)kTileMaxOps)
        return fail(QS_ERR_UNSUPPORTED, "batch state %d: fused block of %zu ops exceeds %d", i, bo.ops.size(),
                    kTileMaxOps);
      BatchBlock b;
      std::memset(&b, 0, sizeof(b));
      b.L = geom.L;
      b.m = geom.m;
      b.nops = (int)bo.ops.size();
      b.op0 = (uint32_t)ops.size();
      b.coef0 = (uint32_t)coefs.size();
      b.ncoefs = (uint32_t)bo.coefs.size();
      b.perm0 = (uint32_t)perm.size();
      b.n_tiles = 1ull << (s->n - geom.L - geom.m);
      for (int jq = 0; jq < geom.m; ++jq) {
        b.base_high[jq] = ~((1ull << geom.hq[jq]) - 1ull);
        b.hq[jq] = (int8_t)geom.hq[jq];
      }
      blocks.push_back(b);
      ops.insert(ops.end(), bo.ops.begin(), bo.ops.end());
      coefs.insert(coefs.end(), bo.coefs.begin(), bo.coefs.end());
      perm.insert(perm.end(), bo.perm.begin(), bo.perm.end());
      cost[i] += (double)(1ull << s->n) * (2.0 + (double)b.nops);
    }
    bstates[i].nblocks = (uint32_t)blocks.size() - bstates[i].block0;
    // Float-float policies keep the state in (head, tail) form between its
    // blocks: the first block reads doubles, the last writes them.
    if (std::is_same<typename TP::M, MathDF>::value)
      for (uint32_t k = 0; k < bstates[i].nblocks; ++k)
        blocks[bstates[i].block0 + k].fmt =
            (k > 0 ? kTileInFF : 0) | (k + 1 < bstates[i].nblocks ? kTileOutFF : 0);
  }
  // States that fit one tile run whole, one CTA each, largest estimated cost
  // first.  A state of several tiles would serialise all its blocks on one
  // CTA; instead step k applies block k of every such state, with its tiles
  // spread over the grid (one launch per step; the launch boundary orders
  // the blocks of a state).
  std::vector<int> order;
  std::vector<int> multi;
  for (int i = 0; i < count; ++i) {
    bool one_tile = true;
    for (uint32_t k = 0; k < bstates[i].nblocks; ++k) one_tile = one_tile && blocks[bstates[i].block0 + k].n_tiles == 1;
    (one_tile ? order : multi).push_back(i);
  }
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  std::vector<BatchState> sorted;
  for (int i : order) {
    sorted.push_back(bstates[i]);
    sorted.back().resident = 1;
  }
  uint32_t nsteps = 0;
  for (int i : multi) nsteps = std::max(nsteps, bstates[i].nblocks);
  const uint64_t grid_est = (uint64_t)sm_count(states[0]->device) * kTileMinCtas;
  std::vector<BatchState> step_items;
  std::vector<size_t> step_first(nsteps), step_count(nsteps);
  for (uint32_t k = 0; k < nsteps; ++k) {
    std::vector<int> here;
    uint64_t total = 0;
    for (int i : multi)
      if (bstates[i].nblocks > k) {
        here.push_back(i);
        total += blocks[bstates[i].block0 + k].n_tiles;
      }
    std::stable_sort(here.begin(), here.end(), [&](int x, int y) {
      return blocks[bstates[x].block0 + k].n_tiles > blocks[bstates[y].block0 + k].n_tiles;
    });
    // Tiles per work item: about two items per CTA.
    const uint64_t per = std::max<uint64_t>(1, (total + 2 * grid_est - 1) / (2 * grid_est));
    step_first[k] = step_items.size();
    for (int i : here) {
      const uint64_t nt = blocks[bstates[i].block0 + k].n_tiles;
      for (uint64_t t0 = 0; t0 < nt; t0 += per) {
        BatchState w = bstates[i];
        w.resident = 0;
        w.block0 = bstates[i].block0 + k;
        w.nblocks = 1;
        w.tau0 = t0;
        w.tau1 = std::min(nt, t0 + per);
        step_items.push_back(w);
      }
    }
    step_count[k] = step_items.size() - step_first[k];
  }

  size_t off = 0;
  bw->off_states = off;
  off = align_up(off + sorted.size() * sizeof(BatchState), 256);
  const size_t off_steps = off;
  off = align_up(off + step_items.size() * sizeof(BatchState), 256);
  bw->off_blocks = off;
  off = align_up(off + blocks.size() * sizeof(BatchBlock), 256);
  bw->off_ops = off;
  off = align_up(off + ops.size() * sizeof(TileOp), 256);
  bw->off_coefs = off;
  off = align_up(off + coefs.size() * sizeof(Coef), 256);
  bw->off_perm = off;
  off = align_up(off + perm.size() + 1, 256);
  bw->off_counter = off;
  off = align_up(off + (1 + (size_t)nsteps) * sizeof(uint32_t), 256);
  if (bw->dev_bytes < off) {
    if (bw->dev) {
      cudaStreamSynchronize(stream);
      cudaFree(bw->dev);
      bw->dev = nullptr;
      bw->dev_bytes = 0;
    }
    QS_CUDA(cudaMalloc(&bw->dev, off));
    bw->dev_bytes = off;
  }
  std::vector<unsigned char> host(off, 0);
  std::memcpy(host.data() + bw->off_states, sorted.data(), sorted.size() * sizeof(BatchState));
  if (!step_items.empty())
    std::memcpy(host.data() + off_steps, step_items.data(), step_items.size() * sizeof(BatchState));
  std::memcpy(host.data() + bw->off_blocks, blocks.data(), blocks.size() * sizeof(BatchBlock));
  std::memcpy(host.data() + bw->off_ops, ops.data(), ops.size() * sizeof(TileOp));
  std::memcpy(host.data() + bw->off_coefs, coefs.data(), coefs.size() * sizeof(Coef));
  if (!perm.empty()) std::memcpy(host.data() + bw->off_perm, perm.data(), perm.size());
  // Stream-ordered after the previous batch that used this buffer.
  QS_CUDA(cudaMemcpyAsync(bw->dev, host.data(), off, cudaMemcpyHostToDevice, stream));
  bw->n_states = (uint32_t)sorted.size();
  bw->step_off.resize(nsteps);
  bw->step_n.resize(nsteps);
  for (uint32_t k = 0; k < nsteps; ++k) {
    bw->step_off[k] = off_steps + step_first[k] * sizeof(BatchState);
    bw->step_n[k] = (uint32_t)step_count[k];
  }
  return QS_OK;
}

template <class TP>
qs_status launch_batch(qs_state s0, const BatchWork* bw, cudaStream_t stream) {
  const size_t smem = kStages * ((size_t)sizeof(typename TP::Glob) << TP::kTileLog) + 2 * kStages * sizeof(uint64_t) +
                      kStages * sizeof(TileDesc) + (TP::kStagePlan ? kStageBytes : 0);
  auto kern = k_batch<TP>;
  QS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kTileThreads, smem) != cudaSuccess || occ < 1) occ = 1;
  const uint32_t full = (uint32_t)(sm_count(s0->device) * occ);
  BatchArgs<TP> args;
  unsigned char* base = (unsigned char*)bw->dev;
  args.blocks = (const BatchBlock*)(base + bw->off_blocks);
  args.ops = (const TileOp*)(base + bw->off_ops);
  args.coefs = (const typename TP::M::Coef*)(base + bw->off_coefs);
  args.perm = base + bw->off_perm;
  args.phase_tab = static_cast<const typename TP::Phase*>(phase_table(s0->device, TP::kPhaseFormat));
  if (!args.phase_tab) return fail(QS_ERR_CUDA, "phase tables missing on device %d", s0->device);
  uint32_t* counters = (uint32_t*)(base + bw->off_counter);
  args.err = error_word(s0);
  if (!args.err) return fail(QS_ERR_CUDA, "device error word unavailable");
  args.wait_ns = wait_limit_ns();
  QS_CUDA(cudaMemsetAsync(counters, 0, (1 + bw->step_n.size()) * sizeof(uint32_t), stream));
  auto go = [&](const BatchState* items, uint32_t n, uint32_t* counter) -> qs_status {
    if (n == 0) return QS_OK;
    args.states = items;
    args.n_states = n;
    args.counter = counter;
    kern<<<std::min(full, n), kTileThreads, smem, stream>>>(args);
    QS_CUDA(cudaGetLastError());
    return QS_OK;
  };
  qs_status st = go((const BatchState*)(base + bw->off_states), bw->n_states, counters);
  for (size_t k = 0; k < bw->step_n.size() && st == QS_OK; ++k)
    st = go((const BatchState*)(base + bw->step_off[k]), bw->step_n[k], counters + 1 + k);
  return st;
}

// States up to kBatchLocalMax qubits share the batched launches; wider states
// need the whole GPU per block and run as fused blocks after them, in the same
// stream order.
struct Split {
  std::vector<qs_state> local_states, wide_states;
  std::vector<const qs_circuit*> local_circuits, wide_circuits;
};

Split split_batch(qs_state* states, const qs_circuit* const* circuits, int count) {
  Split sp;
  for (int i = 0; i < count; ++i) {
    if (states[i]->n <= kBatchLocalMax) {
      sp.local_states.push_back(states[i]);
      sp.local_circuits.push_back(circuits[i]);
    } else {
      sp.wide_states.push_back(states[i]);
      sp.wide_circuits.push_back(circuits[i]);
    }
  }
  return sp;
}

template <class TP>
qs_status enqueue_batch(qs_state s0, const BatchWork* bw, const Split& sp, cudaStream_t stream) {
  if (bw->n_states > 0 || !bw->step_n.empty()) {
    qs_status r = launch_batch<TP>(s0, bw, stream);
    if (r != QS_OK) return r;
  }
  for (size_t i = 0; i < sp.wide_states.size(); ++i) {
    qs_state w = sp.wide_states[i];
    cudaStream_t saved = w->stream;
    w->stream = stream;
    qs_status r = run_fused(w, sp.wide_circuits[i], fuse_width_for(w));
    w->stream = saved;
    if (r != QS_OK) return r;
  }
  return QS_OK;
}

// Make `stream` wait for the work queued so far on every member state's own
// stream, without blocking the host.
qs_status streams_join(qs_state* states, int count, cudaStream_t stream, cudaEvent_t ev) {
  std::vector<cudaStream_t> seen;
  for (int i = 0; i < count; ++i) {
    cudaStream_t o = states[i]->stream;
    if (o == stream || std::find(seen.begin(), seen.end(), o) != seen.end()) continue;
    seen.push_back(o);
    QS_CUDA(cudaEventRecord(ev, o));
    QS_CUDA(cudaStreamWaitEvent(stream, ev, 0));
  }
  return QS_OK;
}

// Make every member state's own stream wait for the batch queued on `stream`.
qs_status streams_fork(qs_state* states, int count, cudaStream_t stream, cudaEvent_t ev) {
  QS_CUDA(cudaEventRecord(ev, stream));
  std::vector<cudaStream_t> seen;
  for (int i = 0; i < count; ++i) {
    cudaStream_t o = states[i]->stream;
    if (o == stream || std::find(seen.begin(), seen.end(), o) != seen.end()) continue;
    seen.push_back(o);
    QS_CUDA(cudaStreamWaitEvent(o, ev, 0));
  }
  return QS_OK;
}

cudaEvent_t order_event() {
  static thread_local cudaEvent_t ev = nullptr;
  if (!ev && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) ev = nullptr;
  return ev;
}

// Capture the batch's launches into an executable graph.
template <class TP>
qs_status capture_batch(qs_state s0, const BatchWork* bw, const Split& sp, cudaGraphExec_t* out) {
  cudaStream_t cap;
  QS_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  qs_status st = QS_OK;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    st = enqueue_batch<TP>(s0, bw, sp, cap);
    e = cudaStreamEndCapture(cap, &g);
  }
  cudaStreamDestroy(cap);
  if (st != QS_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(e, "batch graph capture");
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  return QS_OK;
}

template <class TP>
qs_status run_batch(qs_state* states, const qs_circuit* const* circuits, int count, const qs_run_opts* opts) {
  qs_state s0 = states[0];
  if (!error_word(s0)) return fail(QS_ERR_CUDA, "device error word unavailable");
  cudaEvent_t ev = order_event();
  if (!ev) return fail(QS_ERR_CUDA, "event creation failed");
  std::lock_guard<std::mutex> lk(g_batch_mu);
  BatchWork*& slot = g_oneshot_work[std::make_pair(s0->device, s0->stream)];
  if (!slot) slot = new BatchWork();
  BatchWork* bw = slot;
  const Split sp = split_batch(states, circuits, count);
  if (!sp.local_states.empty()) {
    qs_status st = compile_batch<TP>((qs_state*)sp.local_states.data(), sp.local_circuits.data(),
                                     (int)sp.local_states.size(), bw, s0->stream);
    if (st != QS_OK) return st;
  } else {
    bw->n_states = 0;
    bw->step_off.clear();
    bw->step_n.clear();
  }
  // Every state's pending work must finish before the batch touches it.
  qs_status st = streams_join(states, count, s0->stream, ev);
  if (st != QS_OK) return st;
  if (opts && opts->use_graph) {
    cudaGraphExec_t exec = nullptr;
    st = capture_batch<TP>(s0, bw, sp, &exec);
    if (st != QS_OK) return st;
    cudaError_t e = cudaGraphLaunch(exec, s0->stream);
    cudaGraphExecDestroy(exec);  // freed once the launch completes
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch(batch)");
  } else {
    st = enqueue_batch<TP>(s0, bw, sp, s0->stream);
    if (st != QS_OK) return st;
  }
  return streams_fork(states, count, s0->stream, ev);
}

}  // namespace

qs_status batch_check(qs_state* states, const qs_circuit* const* circuits, int count) {
  if (count < 0 || (count > 0 && (!states || !circuits))) return fail(QS_ERR_ARG, "bad batch");
  if (count == 0) return QS_OK;
  const qs_state s0 = states[0];
  for (int i = 0; i < count; ++i) {
    if (!states[i] || !circuits[i]) return fail(QS_ERR_ARG, "batch entry %d is NULL", i);
    if (states[i]->split) return fail(QS_ERR_UNSUPPORTED, "batch entry %d is a split state", i);
    if (states[i]->dtype != s0->dtype || states[i]->math != s0->math)
      return fail(QS_ERR_ARG, "batch entry %d: every state must have the dtype and math mode of the first", i);
    if (states[i]->device != s0->device) return fail(QS_ERR_ARG, "batch entry %d is on another device", i);
    const qs_circuit* c = circuits[i];
    if (c->n_gates < 0 || (c->n_gates > 0 && !c->gates)) return fail(QS_ERR_ARG, "batch circuit %d is malformed", i);
    for (int64_t g = 0; g < c->n_gates; ++g) {
      qs_status st = check_gate(states[i], c, g);
      if (st != QS_OK) return st;
    }
  }
  std::vector<const void*> seen;
  for (int i = 0; i < count; ++i) seen.push_back(states[i]->psi);
  std::sort(seen.begin(), seen.end());
  if (std::adjacent_find(seen.begin(), seen.end()) != seen.end())
    return fail(QS_ERR_ARG, "a state appears twice in the batch");
  return QS_OK;
}

qs_status batch_run(qs_state* states, const qs_circuit* const* circuits, int count, const qs_run_opts* opts) {
  qs_status st = batch_check(states, circuits, count);
  if (st != QS_OK || count == 0) return st;
  const qs_state s0 = states[0];
  if (s0->dtype == QS_C64) return run_batch<TileF32Batch>(states, circuits, count, opts);
  if (s0->math == QS_MATH_FP64) return run_batch<TileF64>(states, circuits, count, opts);
  return run_batch<TileDFBatch>(states, circuits, count, opts);
}

}  // namespace qs

// ---------------------------------------------------------------------------
// Compiled batches: compiled and captured once, launched many times
// ---------------------------------------------------------------------------
struct qs_batch_s {
  qs::BatchWork work;  // owned device image
  cudaGraphExec_t graph = nullptr;
  cudaEvent_t last = nullptr;  // recorded after each launch
  std::vector<qs_state> states;
  bool valid = true;   // false once a member state has been destroyed
};

namespace qs {
namespace {
std::mutex g_live_mu;
std::vector<qs_batch_s*> g_live_batches;
}  // namespace

// A destroyed state invalidates every compiled batch that holds it.
void release_batch_cache(qs_state s) {
  std::lock_guard<std::mutex> lk(g_live_mu);
  for (qs_batch_s* b : g_live_batches)
    if (b->valid && std::find(b->states.begin(), b->states.end(), s) != b->states.end()) b->valid = false;
}

template <class TP>
qs_status compile_handle(qs_batch_s* b, qs_state* states, const qs_circuit* const* circuits, int count) {
  qs_state s0 = states[0];
  const Split sp = split_batch(states, circuits, count);
  if (!sp.local_states.empty()) {
    qs_status st = compile_batch<TP>((qs_state*)sp.local_states.data(), sp.local_circuits.data(),
                                     (int)sp.local_states.size(), &b->work, s0->stream);
    if (st != QS_OK) return st;
  }
  return capture_batch<TP>(s0, &b->work, sp, &b->graph);
}

}  // namespace qs

using namespace qs;

extern "C" {

qs_status qs_batch_run(qs_state* states, const qs_circuit* const* circuits, int count, const qs_run_opts* opts) {
  return batch_run(states, circuits, count, opts);
}

qs_status qs_batch_compile(qs_state* states, const qs_circuit* const* circuits, int count, qs_batch* out) {
  if (!out) return fail(QS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (count < 1) return fail(QS_ERR_ARG, "a compiled batch needs at least one state");
  qs_status st = batch_check(states, circuits, count);
  if (st != QS_OK) return st;
  qs_batch_s* b = new (std::nothrow) qs_batch_s();
  if (!b) return fail(QS_ERR_OOM, "host allocation failed");
  b->states.assign(states, states + count);
  const qs_state s0 = states[0];
  if (cudaEventCreateWithFlags(&b->last, cudaEventDisableTiming) != cudaSuccess) {
    delete b;
    return fail(QS_ERR_CUDA, "event creation failed");
  }
  if (s0->dtype == QS_C64)
    st = compile_handle<TileF32Batch>(b, states, circuits, count);
  else if (s0->math == QS_MATH_FP64)
    st = compile_handle<TileF64>(b, states, circuits, count);
  else
    st = compile_handle<TileDFBatch>(b, states, circuits, count);
  if (st == QS_OK) {
    // The workspace copy is queued on the first state's stream; the graph
    // is launched there too, so it is ordered after the copy.
    std::lock_guard<std::mutex> lk(g_live_mu);
    g_live_batches.push_back(b);
    *out = b;
    return QS_OK;
  }
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->work.dev) {
    cudaStreamSynchronize(s0->stream);
    cudaFree(b->work.dev);
  }
  cudaEventDestroy(b->last);
  delete b;
  return st;
}

qs_status qs_batch_launch(qs_batch b) {
  if (!b) return fail(QS_ERR_ARG, "batch handle is NULL");
  {
    std::lock_guard<std::mutex> lk(g_live_mu);
    if (!b->valid) return fail(QS_ERR_ARG, "a state of this compiled batch has been destroyed");
  }
  cudaEvent_t ev = order_event();
  if (!ev) return fail(QS_ERR_CUDA, "event creation failed");
  qs_state s0 = b->states[0];
  qs_status st = streams_join(b->states.data(), (int)b->states.size(), s0->stream, ev);
  if (st != QS_OK) return st;
  QS_CUDA(cudaGraphLaunch(b->graph, s0->stream));
  QS_CUDA(cudaEventRecord(b->last, s0->stream));
  return streams_fork(b->states.data(), (int)b->states.size(), s0->stream, ev);
}

qs_status qs_batch_destroy(qs_batch b) {
  if (!b) return QS_OK;
  {
    std::lock_guard<std::mutex> lk(g_live_mu);
    g_live_batches.erase(std::remove(g_live_batches.begin(), g_live_batches.end(), b), g_live_batches.end());
  }
  // Launches in flight keep reading the workspace: wait for the last one.
  cudaEventSynchronize(b->last);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->work.dev) cudaFree(b->work.dev);
  cudaEventDestroy(b->last);
  delete b;
  return QS_OK;
}

}  // extern "C"
