// Test harness, not part of the library: runs the host-side rewrites that
// qs_fuse_run applies to a gate list before it forms blocks (X gates pushed
// through diagonals, dense gates on 3..5 targets composed with the gates
// after them, consecutive 1q/2q gates multiplied), and hands the rewritten
// list back so that a CPU test can apply it and the original with the
// oracle and compare the states; and the order in which the fused runner
// would then execute the gates, block by block, so that a test can check
// that the blocks only move gates past gates they commute with.  Built by
// tests/test_host_rewrites.py and linked against the in-tree libqs.so.
#include <cstring>
#include <vector>

#include "qs_densefuse.h"
#include "qs_fuser.h"
#include "qs_matfuse.h"
#include "qs_tile_dev.cuh"

using qs::fuser::DenseFuser;
using qs::fuser::FGate;
using qs::fuser::MatFuser;
using qs::fuser::XPusher;

// One rewritten gate.  kind: QS_GATE_* or 100 (a phase on a bit pattern:
// amplitudes whose index has the bits ppat under pmask are multiplied by one
// coefficient).  Its numbers are at data[data_off..] (a 2^k x 2^k matrix for
// U1/UK, 2^k entries for DIAG, one coefficient for a pattern, complex as
// re, im) or perm[perm_off..] (2^k entries).
struct RwGate {
  int32_t kind, k;
  int32_t targets[QS_MAX_TARGETS];
  uint64_t ctrl, pmask, ppat;
  int64_t data_off, perm_off;
};

// stages: 1 = XPusher, 2 = DenseFuser, 4 = MatFuser, in the order
// qs_fuse_run uses.  Returns the number of gates written, or -1 if a buffer
// is too small.
extern "C" int64_t rw_rewrite(const qs_circuit* c, int stages, RwGate* out, int64_t max_out, double* data,
                              int64_t max_data, uint32_t* perm, int64_t max_perm) {
  std::vector<FGate> gates;
  for (int64_t i = 0; i < c->n_gates; ++i) gates.push_back(qs::fuser::normalise(c, c->gates[i]));
  XPusher xp;
  DenseFuser df;
  MatFuser mf;
  if (stages & 1) gates = xp.run(gates);
  if (stages & 2) gates = df.run(gates);
  if (stages & 4) gates = mf.run(gates);
  if ((int64_t)gates.size() > max_out) return -1;
  int64_t nd = 0, np = 0;
  for (size_t i = 0; i < gates.size(); ++i) {
    const FGate& g = gates[i];
    RwGate& r = out[i];
    std::memset(&r, 0, sizeof(r));
    r.kind = g.kind;
    r.k = g.k;
    for (int j = 0; j < g.k && j < QS_MAX_TARGETS; ++j) r.targets[j] = g.targets[j];
    r.ctrl = g.ctrl;
    r.pmask = g.pmask;
    r.ppat = g.ppat;
    r.data_off = nd;
    r.perm_off = np;
    const int64_t dim = (int64_t)1 << g.k;
    if (g.kind == QS_GATE_PERM) {
      if (np + dim > max_perm) return -1;
      std::memcpy(perm + np, g.perm, (size_t)dim * sizeof(uint32_t));
      np += dim;
      continue;
    }
    const int64_t nums = g.kind == qs::fuser::kGatePattern ? 2 : g.kind == QS_GATE_DIAG ? 2 * dim : 2 * dim * dim;
    if (nd + nums > max_data) return -1;
    std::memcpy(data + nd, g.data, (size_t)nums * sizeof(double));
    nd += nums;
  }
  return (int64_t)gates.size();
}

namespace {

// The gate list after the three rewrites, as qs_fuse_run forms it.
std::vector<FGate> rewritten(const qs_circuit* c, XPusher& xp, DenseFuser& df, MatFuser& mf) {
  std::vector<FGate> gates;
  for (int64_t i = 0; i < c->n_gates; ++i) gates.push_back(qs::fuser::normalise(c, c->gates[i]));
  return mf.run(df.run(xp.run(gates)));
}

// The block selection of the fused runner under tile policy TP: blocks are
// chosen from the earliest gate not yet taken (permutation runs first with
// up to 6 high qubits), their members added in order until the plan is
// full; a gate that starts no block of two or more runs alone.  Writes, in
// execution order, each gate's index in the rewritten list and its block.
template <class TP>
int64_t block_order(const std::vector<FGate>& gates, int n, int max_high, int64_t* order, int32_t* block,
                    int64_t max_out) {
  using Coef = typename TP::M::Coef;
  constexpr int kPermHigh = 6;
  const int min_chunk = sizeof(typename TP::Glob) == 16 ? 3 : 4;
  const int max_coefs =
      TP::kStagePlan ? std::min(qs::kTileMaxCoefs, qs::kTileMaxCoefBytes / (int)sizeof(Coef)) : qs::kTileMaxCoefs;
  const qs::fuser::Limits lim{qs::kTileMaxOps - 2, max_coefs, qs::kTileMaxPermBytes};
  if (max_high > qs::kTileMaxHigh) max_high = qs::kTileMaxHigh;
  std::vector<char> taken(gates.size(), 0);
  int64_t w = 0;
  int32_t b = 0;
  size_t next = 0;
  while (next < gates.size()) {
    if (taken[next]) {
      ++next;
      continue;
    }
    qs::fuser::Geom geom;
    std::vector<size_t> members;
    if (gates[next].kind == QS_GATE_PERM && max_high < kPermHigh) {
      members = qs::fuser::choose_block(gates, taken, next, n, TP::kTileLog, kPermHigh, min_chunk, lim, 512, &geom,
                                        true);
      if (members.size() <= 1) members.clear();
    }
    if (members.empty())
      members = qs::fuser::choose_block(gates, taken, next, n, TP::kTileLog, max_high, min_chunk, lim, 512, &geom);
    size_t emitted = 0;
    if (members.size() > 1) {
      qs::fuser::BlockOut<Coef> bo;
      qs::fuser::PlanBuilder<typename TP::M> pb(&bo, geom, lim);
      for (size_t idx : members) {
        if (!pb.add(gates[idx])) break;
        taken[idx] = 1;
        if (w >= max_out) return -1;
        order[w] = (int64_t)idx;
        block[w++] = b;
        ++emitted;
      }
    }
    if (emitted == 0) {
      taken[next] = 1;
      if (w >= max_out) return -1;
      order[w] = (int64_t)next;
      block[w++] = b;
    }
    ++b;
  }
  return w;
}

}  // namespace

// dtype: QS_C128 (the float-float tile) or QS_C64.  Returns the number of
// entries written (the rewritten list's length), or -1 if out is too small.
extern "C" int64_t rw_block_order(const qs_circuit* c, int n, int dtype, int max_high, int64_t* order, int32_t* block,
                                  int64_t max_out) {
  XPusher xp;
  DenseFuser df;
  MatFuser mf;
  const std::vector<FGate> gates = rewritten(c, xp, df, mf);
  return dtype == QS_C128 ? block_order<qs::TileDF>(gates, n, max_high, order, block, max_out)
                          : block_order<qs::TileF32>(gates, n, max_high, order, block, max_out);
}
