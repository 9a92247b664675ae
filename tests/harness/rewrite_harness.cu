// Test harness, not part of the library: runs the host-side rewrites that
// qs_fuse_run applies to a gate list before it forms blocks (X gates pushed
// through diagonals, dense gates on 3..5 targets composed with the gates
// after them, consecutive 1q/2q gates multiplied), and hands the rewritten
// list back so that a CPU test can apply it and the original with the
// oracle and compare the states.  Built by tests/test_host_rewrites.py and
// linked against the in-tree libqs.so.
#include <cstring>
#include <vector>

#include "qs_densefuse.h"
#include "qs_fuser.h"
#include "qs_matfuse.h"

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
