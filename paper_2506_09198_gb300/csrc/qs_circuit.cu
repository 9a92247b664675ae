// Circuit runner: validation of qs_circuit records and gate-by-gate dispatch.
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "qs_internal.h"

namespace qs {

qs_status run_fused(qs_state s, const qs_circuit* c, int max_high);  // qs_tile.cu
void release_batch_cache(qs_state s);           // qs_batch.cu

void release_plan_cache(qs_state s) { release_batch_cache(s); }

// Fusion width chosen by qs_autotune, per (device, dtype, math, qubits).
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int, int>, int> g_tuned;
constexpr int kDefaultMaxFuse = 4;

int fuse_width_for(qs_state s);

static int tuned_max_fuse(qs_state s) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tuned.find(std::make_tuple(s->device, (int)s->dtype, (int)s->math, s->n));
  return it == g_tuned.end() ? kDefaultMaxFuse : it->second;
}

int fuse_width_for(qs_state s) { return tuned_max_fuse(s); }

// Validates one gate record against the state and returns its control mask.
qs_status check_gate(const qs_state s, const qs_circuit* c, int64_t gi) {
  const qs_gate& g = c->gates[gi];
  if (g.k < 1 || g.k > QS_MAX_TARGETS) return fail(QS_ERR_ARG, "gate %lld: k = %d out of range", (long long)gi, g.k);
  uint64_t used = 0;
  for (int j = 0; j < g.k; ++j) {
    const int t = g.targets[j];
    if (t < 0 || t >= s->n || ((used >> t) & 1ull))
      return fail(QS_ERR_ARG, "gate %lld: bad or repeated target %d", (long long)gi, t);
    used |= 1ull << t;
  }
  if (s->n < 64 && (g.ctrl_mask >> s->n) != 0)
    return fail(QS_ERR_ARG, "gate %lld: control outside the register", (long long)gi);
  if (g.ctrl_mask & used) return fail(QS_ERR_ARG, "gate %lld: control also a target", (long long)gi);
  if (g.offset < 0) return fail(QS_ERR_ARG, "gate %lld: negative offset", (long long)gi);
  switch (g.kind) {
    case QS_GATE_U1:
      if (g.k != 1) return fail(QS_ERR_ARG, "gate %lld: U1 needs k = 1", (long long)gi);
      if (!c->data) return fail(QS_ERR_ARG, "circuit has no data pool");
      break;
    case QS_GATE_UK: {
      if (!c->data) return fail(QS_ERR_ARG, "circuit has no data pool");
      if (g.k <= 5) break;
      // Larger matrices are accepted when they are diagonal or permutations.
      const int dim = 1 << g.k;
      const double* M = c->data + g.offset;
      bool diag = true, permlike = true;
      for (int col = 0; col < dim; ++col) {
        int ones = 0;
        for (int r = 0; r < dim; ++r) {
          const double* z = M + 2 * (r * dim + col);
          const bool zero = z[0] == 0.0 && z[1] == 0.0;
          if (r != col && !zero) diag = false;
          if (z[0] == 1.0 && z[1] == 0.0)
            ++ones;
          else if (!zero)
            permlike = false;
        }
        if (ones != 1) permlike = false;
      }
      if (!diag && !permlike)
        return fail(QS_ERR_UNSUPPORTED, "gate %lld: dense matrices on %d targets are not supported (at most 5)",
                    (long long)gi, g.k);
      break;
    }
    case QS_GATE_DIAG:
      if (!c->data) return fail(QS_ERR_ARG, "circuit has no data pool");
      break;
    case QS_GATE_PERM: {
      if (!c->perm) return fail(QS_ERR_ARG, "circuit has no permutation pool");
      const uint32_t* p = c->perm + g.offset;
      std::vector<char> seen((size_t)1 << g.k, 0);
      for (int v = 0; v < (1 << g.k); ++v) {
        if (p[v] >= (1u << g.k) || seen[p[v]]) return fail(QS_ERR_ARG, "gate %lld: not a bijection", (long long)gi);
        seen[p[v]] = 1;
      }
      break;
    }
    default:
      return fail(QS_ERR_ARG, "gate %lld: unknown kind %d", (long long)gi, g.kind);
  }
  return QS_OK;
}

qs_status apply_gate_record(qs_state s, const qs_circuit* c, const qs_gate& g);

qs_status qs_fuse_run_gatewise(qs_state s, const qs_circuit* c) {
  for (int64_t i = 0; i < c->n_gates; ++i) {
    qs_status st = apply_gate_record(s, c, c->gates[i]);
    if (st != QS_OK) return st;
  }
  return QS_OK;
}

qs_status apply_gate_record(qs_state s, const qs_circuit* c, const qs_gate& g) {
  switch (g.kind) {
    case QS_GATE_U1:
      return dispatch_u1(s, g.targets[0], g.ctrl_mask, c->data + g.offset);
    case QS_GATE_UK:
      return dispatch_uk(s, g.targets, g.k, g.ctrl_mask, c->data + g.offset);
    case QS_GATE_DIAG:
      return dispatch_diag(s, g.targets, g.k, g.ctrl_mask, c->data + g.offset);
    case QS_GATE_PERM:
      return dispatch_perm(s, g.targets, g.k, g.ctrl_mask, c->perm + g.offset);
  }
  return fail(QS_ERR_ARG, "unknown gate kind");
}

}  // namespace qs

using namespace qs;

extern "C" {

qs_status qs_fuse_run(qs_state s, const qs_circuit* c, const qs_run_opts* opts) {
  if (!s) return fail(QS_ERR_ARG, "state handle is NULL");
  if (!c || c->n_gates < 0 || (c->n_gates > 0 && !c->gates)) return fail(QS_ERR_ARG, "bad circuit");
  const int max_fuse = opts ? opts->max_fuse : 0;
  if (max_fuse < 0 || max_fuse > 6) return fail(QS_ERR_ARG, "max_fuse = %d outside [0, 6]", max_fuse);
  for (int64_t i = 0; i < c->n_gates; ++i) {
    qs_status st = check_gate(s, c, i);
    if (st != QS_OK) return st;
  }
  s->run_fused_launches = 0;
  s->run_gate_launches = 0;
  s->run_dense_blocks = 0;
  s->run_dense_gates = 0;
  if (c->n_gates == 0) return QS_OK;
  if (s->split) return split_run(s, c, max_fuse);
  if (max_fuse != 1) return run_fused(s, c, max_fuse == 0 ? tuned_max_fuse(s) : max_fuse);
  s->run_gate_launches = c->n_gates;
  return qs_fuse_run_gatewise(s, c);
}

qs_status qs_last_run_stats(qs_state s, qs_run_stats* out) {
  if (!s) return fail(QS_ERR_ARG, "state handle is NULL");
  if (!out) return fail(QS_ERR_ARG, "out is NULL");
  std::memset(out, 0, sizeof(*out));
  out->fused_launches = s->run_fused_launches;
  out->gate_launches = s->run_gate_launches;
  out->dense_blocks = s->run_dense_blocks;
  out->dense_gates = s->run_dense_gates;
  return QS_OK;
}

qs_status qs_autotune(qs_state s, const qs_circuit* c, int* best_max_fuse, double* best_ms) {
  if (!s) return fail(QS_ERR_ARG, "state handle is NULL");
  if (s->split) return fail(QS_ERR_UNSUPPORTED, "autotuning takes a state in one allocation");
  if (!c || c->n_gates < 0 || (c->n_gates > 0 && !c->gates)) return fail(QS_ERR_ARG, "bad circuit");
  for (int64_t i = 0; i < c->n_gates; ++i) {
    qs_status st = check_gate(s, c, i);
    if (st != QS_OK) return st;
  }
  cudaEvent_t a, b;
  QS_CUDA(cudaEventCreate(&a));
  QS_CUDA(cudaEventCreate(&b));
  int best = 1;
  float best_t = 0.f;
  qs_status st = QS_OK;
  constexpr int kTimedReps = 3;
  for (int mf = 1; mf <= 6 && st == QS_OK; ++mf) {
    // one untimed run (kernel loading), then the fastest of kTimedReps
    float ms = 0.f;
    for (int rep = 0; rep <= kTimedReps && st == QS_OK; ++rep) {
      st = launch_init_basis(s, 0);
      if (st != QS_OK) break;
      if (rep > 0 && cudaEventRecord(a, s->stream) != cudaSuccess) st = fail(QS_ERR_CUDA, "event record");
      if (st == QS_OK) st = mf == 1 ? qs_fuse_run_gatewise(s, c) : run_fused(s, c, mf);
      if (st != QS_OK || rep == 0) continue;
      if (cudaEventRecord(b, s->stream) != cudaSuccess) {
        st = fail(QS_ERR_CUDA, "event record");
      } else if (cudaEventSynchronize(b) != cudaSuccess) {
        st = fail(QS_ERR_CUDA, "event synchronize");
      } else {
        float t = 0.f;
        cudaEventElapsedTime(&t, a, b);
        if (rep == 1 || t < ms) ms = t;
      }
    }
    if (st != QS_OK) break;
    if (mf == 1 || ms < best_t) {
      best = mf;
      best_t = ms;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (st != QS_OK) return st;
  if (best == 1) best = 2;  // max_fuse = 0 always fuses; keep the narrowest block if gate-by-gate won
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[std::make_tuple(s->device, (int)s->dtype, (int)s->math, s->n)] = best;
  }
  if (best_max_fuse) *best_max_fuse = best;
  if (best_ms) *best_ms = best_t;
  return device_error_check(s);
}

}  // extern "C"
