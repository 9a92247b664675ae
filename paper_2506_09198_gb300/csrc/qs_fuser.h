// Host-side fuser: turns a gate list into fused blocks of tile ops.
//
// A block is a set of gates applied in one pass over the state: their targets
// must be tile qubits (the low qubits plus at most max_high "high" qubits,
// see qs_tile.cuh); diagonal gates need no tile qubits.  Blocks are grown
// greedily over a window of the remaining gates: a gate that cannot join
// blocks the qubits it touches for every later gate, so later gates only move
// ahead of gates they commute with (disjoint qubits).  Used by the per-circuit
// runner (qs_tile.cu) and by the batched kernel (qs_batch.cu).
#pragma once
#include <algorithm>
#include <cmath>
#include <cstring>
#include <deque>
#include <functional>
#include <vector>

#include "qs_internal.h"
#include "qs_tile.cuh"

namespace qs {
namespace fuser {

inline bool is_c(const double* z, double re, double im) { return z[0] == re && z[1] == im; }

// A coefficient on the 2^-32-turn grid: c = exp(2 pi i m / 2^32) to within
// 1e-15 per component (the rounding of cos and sin).
inline bool dyadic_turn(const double* c, uint32_t* m) {
  const double t = std::atan2(c[1], c[0]) * (4294967296.0 / 6.283185307179586476925286766559);
  const double r = std::nearbyint(t);
  if (!(std::fabs(t - r) <= 1e-3)) return false;
  const uint32_t mm = (uint32_t)(uint64_t)(int64_t)r;
  double cr, ci;
  turn_cos_sin(mm, &cr, &ci);
  if (!(std::fabs(cr - c[0]) <= 1e-15 && std::fabs(ci - c[1]) <= 1e-15)) return false;
  *m = mm;
  return true;
}

// Smallest e with sum_c (|re u_rc| + |im u_rc|) (entries rounded to float)
// < 2^e, stored biased by 128: the anchored float-float accumulation of
// dense rows needs this bound.
inline uint8_t row_exp_biased(const double* U, int row, int dim) {
  double sum = 0.0;
  for (int c = 0; c < dim; ++c) {
    const double* z = U + 2 * (row * dim + c);
    sum += std::fabs((double)(float)z[0]) + std::fabs((double)(float)z[1]);
  }
  int e = -126;
  if (sum > 0.0) std::frexp(sum, &e);
  if (e < -126) e = -126;
  if (e > 127) e = 127;
  return (uint8_t)(e + 128);
}

// Internal gate kind (never in a qs_circuit): multiply the amplitudes whose
// bits under pmask equal ppat by the complex number at data.
constexpr int kGatePattern = 100;

// One gate record in normalised form.
struct FGate {
  int kind;  // QS_GATE_* or kGatePattern
  int k;
  int targets[QS_MAX_TARGETS];
  uint64_t ctrl;
  const double* data;
  const uint32_t* perm;
  bool diagonal;        // needs no tile qubits
  uint64_t qubit_mask;  // targets | controls
  uint64_t tmask;       // targets that must be tile qubits
  uint64_t pmask, ppat;  // kGatePattern
};

inline bool matrix_is_diag(const double* M, int dim) {
  for (int r = 0; r < dim; ++r)
    for (int c = 0; c < dim; ++c)
      if (r != c && !is_c(M + 2 * (r * dim + c), 0, 0)) return false;
  return true;
}

inline FGate normalise(const qs_circuit* c, const qs_gate& g) {
  FGate f;
  std::memset(&f, 0, sizeof(f));
  f.kind = g.kind;
  f.k = g.k;
  for (int j = 0; j < g.k; ++j) f.targets[j] = g.targets[j];
  f.ctrl = g.ctrl_mask;
  if (g.kind == QS_GATE_PERM)
    f.perm = c->perm + g.offset;
  else
    f.data = c->data + g.offset;
  uint64_t tm = 0;
  for (int j = 0; j < g.k; ++j) tm |= 1ull << g.targets[j];
  f.qubit_mask = tm | g.ctrl_mask;
  if (g.kind == QS_GATE_DIAG)
    f.diagonal = true;
  else if (g.kind == QS_GATE_U1 || g.kind == QS_GATE_UK)
    f.diagonal = matrix_is_diag(f.data, 1 << g.k);
  f.tmask = f.diagonal ? 0 : tm;
  return f;
}

// Uncontrolled X given as a 2x2 matrix or a one-qubit permutation.
inline bool is_plain_x(const FGate& g) {
  if (g.ctrl != 0 || g.k != 1) return false;
  if (g.kind == QS_GATE_PERM) return g.perm[0] == 1u && g.perm[1] == 0u;
  if (g.kind == QS_GATE_U1)
    return is_c(g.data, 0, 0) && is_c(g.data + 2, 1, 0) && is_c(g.data + 4, 1, 0) && is_c(g.data + 6, 0, 0);
  return false;
}

// Diagonal entry v of a diagonal gate (DIAG table, or the diagonal of a
// U1 / UK matrix).
inline const double* diag_entry(const FGate& g, int v) {
  if (g.kind == QS_GATE_DIAG) return g.data + 2 * v;
  const int dim = 1 << g.k;
  return g.data + 2 * (v * dim + v);
}

// Moves uncontrolled X gates later in the circuit past diagonal gates, which
// they conjugate (X_q D = D' X_q, D' = D with index bit q flipped), so that
// two X on one qubit cancel.  An X-conjugated multi-controlled phase (a
// Grover oracle or diffusion core) becomes one phase on a bit pattern that
// needs no tile qubits.  A pending X is emitted before the first gate that
// is not diagonal on its qubit (or that this pass cannot conjugate), and at
// the end.  Moves and phases are exact, so the circuit's arithmetic is
// unchanged.  The tables and coefficients it creates live in this object.
class XPusher {
 public:
  std::vector<FGate> run(const std::vector<FGate>& in) {
    std::vector<FGate> out;
    out.reserve(in.size());
    uint64_t pend = 0;
    auto flush = [&](uint64_t qm) {
      const uint64_t f = qm & pend;
      for (int q = 0; q < 64; ++q)
        if ((f >> q) & 1ull) out.push_back(make_x(q));
      pend &= ~qm;
    };
    for (const FGate& g : in) {
      if (is_plain_x(g)) {
        pend ^= 1ull << g.targets[0];
        continue;
      }
      const uint64_t hit = g.qubit_mask & pend;
      if (!hit) {
        out.push_back(g);
        continue;
      }
      if (g.diagonal && g.kind != kGatePattern) {
        const int dim = 1 << g.k;
        int n_other = 0, v_other = 0;
        for (int v = 0; v < dim; ++v)
          if (!is_c(diag_entry(g, v), 1, 0)) {
            ++n_other;
            v_other = v;
          }
        if (n_other == 0) continue;  // identity
        uint64_t tbits = 0, vbits = 0;
        for (int j = 0; j < g.k; ++j) {
          tbits |= 1ull << g.targets[j];
          if ((v_other >> j) & 1) vbits |= 1ull << g.targets[j];
        }
        if (n_other == 1) {
          const uint64_t mask = tbits | g.ctrl;
          out.push_back(make_pattern(mask, (vbits | g.ctrl) ^ hit, diag_entry(g, v_other)));
          continue;
        }
        if ((hit & g.ctrl) == 0) {
          // X on targets: the table's index bits flip
          uint32_t flip = 0;
          for (int j = 0; j < g.k; ++j)
            if ((hit >> g.targets[j]) & 1ull) flip |= 1u << j;
          store_.emplace_back(2 * dim);
          std::vector<double>& t = store_.back();
          for (int v = 0; v < dim; ++v) {
            const double* e = diag_entry(g, v ^ (int)flip);
            t[2 * v] = e[0];
            t[2 * v + 1] = e[1];
          }
          FGate d = g;
          d.kind = QS_GATE_DIAG;
          d.data = t.data();
          out.push_back(d);
          continue;
        }
      }
      if (g.kind == kGatePattern) {
        FGate p = g;
        p.ppat ^= hit;
        out.push_back(p);
        continue;
      }
      flush(g.qubit_mask);
      out.push_back(g);
    }
    flush(~0ull);
    return out;
  }

 private:
  std::deque<std::vector<double>> store_;
  static constexpr uint32_t kXPerm[2] = {1u, 0u};

  static FGate blank() {
    FGate f;
    std::memset(&f, 0, sizeof(f));
    return f;
  }
  FGate make_x(int q) const {
    FGate f = blank();
    f.kind = QS_GATE_PERM;
    f.k = 1;
    f.targets[0] = q;
    f.perm = kXPerm;
    f.qubit_mask = 1ull << q;
    f.tmask = 1ull << q;
    return f;
  }
  FGate make_pattern(uint64_t mask, uint64_t pattern, const double* c) {
    store_.emplace_back(2);
    store_.back()[0] = c[0];
    store_.back()[1] = c[1];
    FGate f = blank();
    f.kind = kGatePattern;
    f.data = store_.back().data();
    f.diagonal = true;
    f.qubit_mask = mask;
    f.pmask = mask;
    f.ppat = pattern;
    return f;
  }
};

// Gates a tile op can express: dense matrices on at most 2 targets,
// diagonals and permutations on at most 8.
inline bool tileable(const FGate& g) {
  if (g.kind == kGatePattern) return true;
  if (g.kind == QS_GATE_DIAG || g.kind == QS_GATE_PERM || g.diagonal) return g.k <= 8;
  return g.k <= 2;
}

struct Geom {
  int L = 0, m = 0;
  int hq[kTileMaxHigh] = {0};
};

// Smallest tile geometry whose tile qubits include `need`: L = tile_log - m
// low qubits and the needed qubits at or above L as high qubits (m of them).
inline bool geometry(uint64_t need, int n, int tile_log, int max_high, int min_chunk_log, Geom* g) {
  if (n <= tile_log) {
    g->L = n;
    g->m = 0;
    return true;
  }
  for (int m = 0; m <= max_high && m <= kTileMaxHigh; ++m) {
    const int L = tile_log - m;
    if (L < min_chunk_log) return false;
    int cnt = 0;
    for (int q = L; q < n; ++q)
      if ((need >> q) & 1ull) {
        if (cnt < kTileMaxHigh) g->hq[cnt] = q;
        ++cnt;
      }
    if (cnt <= m) {  // the smallest feasible m has cnt == m
      g->L = L;
      g->m = cnt;
      return true;
    }
  }
  return false;
}

struct Limits {
  int ops, coefs, perm_bytes;
};

template <class Coef>
struct BlockOut {
  Geom geom;
  std::vector<TileOp> ops;
  std::vector<Coef> coefs;
  std::vector<uint8_t> perm;
};

// Translates gates into tile ops for one block geometry.
template <class P>
struct PlanBuilder {
  using Coef = typename P::Coef;
  BlockOut<Coef>* out;
  Limits lim;
  int local_of[64];

  PlanBuilder(BlockOut<Coef>* o, const Geom& g, Limits l) : out(o), lim(l) {
    out->geom = g;
    out->ops.clear();
    out->coefs.clear();
    out->perm.clear();
    for (int q = 0; q < 64; ++q) local_of[q] = -1;
    for (int q = 0; q < g.L; ++q) local_of[q] = q;
    for (int j = 0; j < g.m; ++j) local_of[g.hq[j]] = g.L + j;
  }

  bool room(int ops, int coefs, int perm_bytes) const {
    return (int)out->ops.size() + ops <= lim.ops && (int)out->coefs.size() + coefs <= lim.coefs &&
           (int)out->perm.size() + perm_bytes <= lim.perm_bytes;
  }

  static TileOp blank() {
    TileOp op;
    std::memset(&op, 0, sizeof(op));
    return op;
  }

  // Local controls form the op's local mask; controls on free qubits
  // become its tile predicate.
  void controls(TileOp& op, uint64_t ctrl) const {
    for (int q = 0; q < 64; ++q) {
      if (!((ctrl >> q) & 1ull)) continue;
      if (local_of[q] >= 0) {
        op.lmask |= 1u << local_of[q];
      } else {
        op.gmask |= 1ull << q;
        op.gpat |= 1ull << q;
      }
    }
  }

  uint32_t add_coefs(const double* z, int count) {
    const uint32_t at = (uint32_t)out->coefs.size();
    for (int j = 0; j < count; ++j) out->coefs.push_back(P::make_coef(z[2 * j], z[2 * j + 1]));
    return at;
  }

  bool phase(uint64_t mask, uint64_t pattern, const double* c) {
    if (!room(1, 1, 0)) return false;
    TileOp op = blank();
    for (int q = 0; q < 64; ++q) {
      if (!((mask >> q) & 1ull)) continue;
      const bool one = (pattern >> q) & 1ull;
      if (local_of[q] >= 0) {
        op.lmask |= 1u << local_of[q];
        if (one) op.lpat |= 1u << local_of[q];
      } else {
        op.gmask |= 1ull << q;
        if (one) op.gpat |= 1ull << q;
      }
    }
    // Phases on the 2^-32-turn grid become terms; group_terms turns runs
    // of them into TOP_POLY runs and the rest back into PHASE / NEG ops.
    uint32_t m = 0;
    if (is_c(c, -1, 0)) {
      op.kind = TOP_TERM;
      op.neg = 1;
      op.ptab = 0x80000000u;
    } else if (dyadic_turn(c, &m)) {
      op.kind = TOP_TERM;
      op.ptab = m;
      op.coef = add_coefs(c, 1);
    } else {
      op.kind = TOP_PHASE;
      op.coef = add_coefs(c, 1);
    }
    out->ops.push_back(op);
    return true;
  }

  bool diag(const int* targets, int k, uint64_t ctrl, const double* d) {
    int n_other = 0, v_other = -1;
    for (int v = 0; v < (1 << k); ++v)
      if (!is_c(d + 2 * v, 1, 0)) {
        ++n_other;
        v_other = v;
      }
    if (n_other == 0) return true;
    if (n_other == 1) {
      uint64_t mask = ctrl, pattern = ctrl;
      for (int j = 0; j < k; ++j) {
        mask |= 1ull << targets[j];
        if ((v_other >> j) & 1) pattern |= 1ull << targets[j];
      }
      return phase(mask, pattern, d + 2 * v_other);
    }
    if (!room(1, 1 << k, 0)) return false;
    TileOp op = blank();
    op.kind = TOP_DIAG;
    op.k = (uint8_t)k;
    controls(op, ctrl);
    int nl = 0;
    for (int j = 0; j < k; ++j) {
      const int lq = local_of[targets[j]];
      if (lq >= 0) {
        op.tpos[nl] = (uint8_t)lq;
        op.tj[nl] = (uint8_t)j;
        ++nl;
        op.gq[j] = 0xFF;
      } else {
        op.gq[j] = (uint8_t)targets[j];
      }
    }
    op.nloc = (uint8_t)nl;
    op.coef = add_coefs(d, 1 << k);
    out->ops.push_back(op);
    return true;
  }

  bool pairs(uint8_t kind, int t, uint64_t ctrl, const double* U) {
    if (!room(1, U ? 4 : 0, 0)) return false;
    TileOp op = blank();
    op.kind = kind;
    op.tpos[0] = (uint8_t)local_of[t];
    controls(op, ctrl);
    if (U) {
      op.coef = add_coefs(U, 4);
      // Real matrices (H, rotations about y) skip the imaginary terms.
      op.nloc = (U[1] == 0.0 && U[3] == 0.0 && U[5] == 0.0 && U[7] == 0.0) ? 1 : 0;
    }
    out->ops.push_back(op);
    return true;
  }

  bool dense2(int t0, int t1, uint64_t ctrl, const double* U) {
    if (!room(1, 16, 0)) return false;
    TileOp op = blank();
    op.kind = TOP_DENSE2;
    op.tpos[0] = (uint8_t)local_of[t0];
    op.tpos[1] = (uint8_t)local_of[t1];
    controls(op, ctrl);
    op.coef = add_coefs(U, 16);
    for (int r = 0; r < 4; ++r) op.tj[r] = row_exp_biased(U, r, 4);
    out->ops.push_back(op);
    return true;
  }

  bool perm(const int* targets, int k, uint64_t ctrl, const uint32_t* p) {
    if (k == 2 && ctrl == 0 && p[0] == 0 && p[1] == 2 && p[2] == 1 && p[3] == 3) {  // SWAP: relabel only
      if (!room(1, 0, 0)) return false;
      TileOp op = blank();
      op.kind = TOP_SWAPBITS;
      op.tpos[0] = (uint8_t)local_of[targets[0]];
      op.tpos[1] = (uint8_t)local_of[targets[1]];
      out->ops.push_back(op);
      return true;
    }
    if (k > 8 || !room(1, 0, 1 << k)) return false;
    TileOp op = blank();
    op.kind = TOP_PERM;
    op.k = (uint8_t)k;
    for (int j = 0; j < k; ++j) op.tpos[j] = (uint8_t)local_of[targets[j]];
    controls(op, ctrl);
    op.ptab = (uint32_t)out->perm.size();
    const size_t at = out->perm.size();
    out->perm.resize(at + (1u << k));
    for (int v = 0; v < (1 << k); ++v) out->perm[at + p[v]] = (uint8_t)v;  // inverse table
    out->ops.push_back(op);
    return true;
  }

  // Translate one gate; false if the block has no room for it.
  bool add(const FGate& g) {
    if (g.kind == kGatePattern) return phase(g.pmask, g.ppat, g.data);
    if (g.kind == QS_GATE_DIAG) return diag(g.targets, g.k, g.ctrl, g.data);
    if (g.kind == QS_GATE_PERM) {
      bool ident = true;
      for (int v = 0; v < (1 << g.k); ++v) ident = ident && g.perm[v] == (uint32_t)v;
      if (ident) return true;
      if (g.k == 1) return pairs(TOP_XSWAP, g.targets[0], g.ctrl, nullptr);
      return perm(g.targets, g.k, g.ctrl, g.perm);
    }
    const int dim = 1 << g.k;
    if (g.diagonal) {
      std::vector<double> d(2 * dim);
      for (int v = 0; v < dim; ++v) {
        d[2 * v] = g.data[2 * (v * dim + v)];
        d[2 * v + 1] = g.data[2 * (v * dim + v) + 1];
      }
      return diag(g.targets, g.k, g.ctrl, d.data());
    }
    if (g.k == 1) {
      const double* U = g.data;
      if (is_c(U, 0, 0) && is_c(U + 6, 0, 0)) {
        if (is_c(U + 2, 1, 0) && is_c(U + 4, 1, 0)) return pairs(TOP_XSWAP, g.targets[0], g.ctrl, nullptr);
        if (is_c(U + 2, 0, -1) && is_c(U + 4, 0, 1)) return pairs(TOP_Y, g.targets[0], g.ctrl, nullptr);
      }
      return pairs(TOP_DENSE1, g.targets[0], g.ctrl, U);
    }
    if (g.k == 2) {
      // Permutation matrices given densely become table permutations.
      bool permlike = true;
      uint32_t p[4] = {0, 0, 0, 0};
      for (int c = 0; c < 4 && permlike; ++c) {
        int ones = 0;
        for (int r = 0; r < 4; ++r) {
          const double* z = g.data + 2 * (r * 4 + c);
          if (is_c(z, 1, 0)) {
            ++ones;
            p[c] = (uint32_t)r;
          } else if (!is_c(z, 0, 0)) {
            permlike = false;
          }
        }
        if (ones != 1) permlike = false;
      }
      if (permlike) return perm(g.targets, 2, g.ctrl, p);
      return dense2(g.targets[0], g.targets[1], g.ctrl, g.data);
    }
    return false;
  }
};

// Local bits that must be register bits for an op (dense gates and moves).
inline uint32_t reg_need(const TileOp& op) {
  if (op.kind == TOP_DENSE1 || op.kind == TOP_XSWAP || op.kind == TOP_Y) return 1u << op.tpos[0];
  if (op.kind == TOP_DENSE2) return (1u << op.tpos[0]) | (1u << op.tpos[1]);
  return 0u;
}

// Insert layout changes so that every dense op finds its targets in
// registers, and rewrite those targets as register bit indices.  A new layout
// takes the targets of the op that needs it plus those of the following ops,
// in order, while they fit in rb register bits; free register slots take the
// highest remaining local bits.
//
// The staged tile sits in shared memory in plain order, so the first read and
// the last write are free of bank conflicts only when the lowest `bank_bits`
// local bits are thread bits (lanes then touch consecutive amplitudes).  If
// the first layout needs one of those bits in registers, the tile is read in
// a bank-friendly layout first and transposed (layout changes go through a
// swizzled arrangement); likewise before the final write.
inline std::vector<TileOp> schedule_layouts(const std::vector<TileOp>& ops, int tile_log, int reg_bits,
                                            int bank_bits) {
  const int rb = tile_log < reg_bits ? tile_log : reg_bits;
  const uint32_t low = tile_log > bank_bits + rb ? ((1u << bank_bits) - 1u) : 0u;
  std::vector<TileOp> out;
  out.reserve(ops.size() + 8);
  uint32_t cur = 0;
  int pos_of[32];
  bool have = false;
  auto emit = [&](uint32_t set) {
    TileOp lay;
    std::memset(&lay, 0, sizeof(lay));
    lay.kind = TOP_LAYOUT;
    lay.k = (uint8_t)rb;
    int j = 0;
    for (int b = 0; b < tile_log; ++b)
      if ((set >> b) & 1u) {
        lay.tpos[j] = (uint8_t)b;
        pos_of[b] = j;
        ++j;
      }
    cur = set;
    have = true;
    out.push_back(lay);
  };
  auto fill_high = [&](uint32_t set) {
    int cnt = __builtin_popcount(set);
    for (int b = tile_log - 1; b >= 0 && cnt < rb; --b)
      if (!((set >> b) & 1u)) {
        set |= 1u << b;
        ++cnt;
      }
    return set;
  };
  auto make_layout = [&](size_t i) {
    uint32_t set = 0;
    for (size_t j = i; j < ops.size(); ++j) {
      if (ops[j].kind == TOP_SWAPBITS) break;  // later needs refer to relabelled bits
      const uint32_t need = reg_need(ops[j]);
      if (!need) continue;
      const uint32_t u = set | need;
      if (__builtin_popcount(u) > rb) break;
      set = u;
    }
    set = fill_high(set);
    if (!have && (set & low)) emit(fill_high(0));  // bank-friendly first read
    emit(set);
  };
  for (size_t i = 0; i < ops.size(); ++i) {
    const uint32_t need = reg_need(ops[i]);
    if (!have || (need & ~cur)) make_layout(i);
    if (ops[i].kind == TOP_SWAPBITS) {
      // The register that held local bit a now holds bit b, and vice versa.
      const int a = ops[i].tpos[0], b = ops[i].tpos[1];
      const bool ra = (cur >> a) & 1u, rb_ = (cur >> b) & 1u;
      if (ra && rb_) {
        std::swap(pos_of[a], pos_of[b]);
      } else if (ra || rb_) {
        const int from = ra ? a : b, to = ra ? b : a;
        cur = (cur & ~(1u << from)) | (1u << to);
        pos_of[to] = pos_of[from];
      }
      out.push_back(ops[i]);
      continue;
    }
    if (ops[i].kind == TOP_POLY) {
      // Split each term's local condition into its thread bits (lmask,
      // lpat) and its register bits (tj[0], tj[1] in register-index space),
      // then order the run's terms by register condition (they commute), so
      // that the kernel sums each group per thread and adds it to the
      // group's registers once.
      const size_t cnt = ops[i].k;
      std::vector<TileOp> run(ops.begin() + i, ops.begin() + i + cnt);
      const uint8_t count = run[0].k, first = run[0].nloc;
      for (TileOp& t : run) {
        uint32_t rm = 0, rp = 0;
        for (int b = 0; b < tile_log; ++b) {
          if (!((cur >> b) & 1u) || !((t.lmask >> b) & 1u)) continue;
          rm |= 1u << pos_of[b];
          if ((t.lpat >> b) & 1u) rp |= 1u << pos_of[b];
        }
        t.tj[0] = (uint8_t)rm;
        t.tj[1] = (uint8_t)rp;
        t.lmask &= ~cur;
        t.lpat &= ~cur;
      }
      std::stable_sort(run.begin(), run.end(), [](const TileOp& x, const TileOp& y) {
        return x.tj[0] != y.tj[0] ? x.tj[0] < y.tj[0] : x.tj[1] < y.tj[1];
      });
      for (size_t t = 0; t < cnt; ++t) run[t].kind = t == 0 ? TOP_POLY : TOP_TERM;
      run[0].k = count;
      run[0].nloc = first;
      // Complex multiplications per thread: accumulate mode, one per
      // register and byte; factored mode, a table product per group plus
      // one per matching register and group.
      if (first < 4) {
        const int R = 1 << rb, bytes = 4 - first;
        int fact = 0;
        for (size_t g0 = 0; g0 < cnt;) {
          size_t g1 = g0 + 1;
          while (g1 < cnt && run[g1].tj[0] == run[g0].tj[0] && run[g1].tj[1] == run[g0].tj[1]) ++g1;
          uint32_t any = 0;
          for (size_t t = g0; t < g1; ++t) any |= run[t].ptab;
          const int gfirst = any == 0 ? 3 : __builtin_ctz(any) / 8;  // the group's lowest nonzero byte
          for (size_t t = g0; t < g1; ++t) run[t].tj[2] = (uint8_t)gfirst;
          fact += (4 - gfirst) + (R >> __builtin_popcount(run[g0].tj[0]));
          g0 = g1;
        }
        run[0].tpos[0] = fact < bytes * R ? 1 : 0;
      }
      for (TileOp& t : run) t.coef = (uint32_t)t.tj[0] | (uint32_t)t.tj[1] << 8 | (uint32_t)t.tj[2] << 16;
      out.insert(out.end(), run.begin(), run.end());
      i += cnt - 1;
      continue;
    }
    TileOp op = ops[i];
    if (need) {
      op.tpos[0] = (uint8_t)pos_of[ops[i].tpos[0]];
      if (op.kind == TOP_DENSE2) op.tpos[1] = (uint8_t)pos_of[ops[i].tpos[1]];
    }
    out.push_back(op);
  }
  if (!have) make_layout(0);
  if (cur & low) emit(fill_high(0));  // bank-friendly last write
  return out;
}

// Runs of at least kPolyMinRun consecutive terms become TOP_POLY runs of at
// most kPolyMaxRun terms; shorter runs go back to single PHASE / NEG ops.
// Runs before schedule_layouts, which then splits each term's condition
// into thread and register bits.
inline void group_terms(std::vector<TileOp>& ops) {
  size_t i = 0;
  while (i < ops.size()) {
    if (ops[i].kind != TOP_TERM) {
      ++i;
      continue;
    }
    size_t j = i;
    while (j < ops.size() && ops[j].kind == TOP_TERM) ++j;
    if (j - i < (size_t)kPolyMinRun) {
      for (size_t t = i; t < j; ++t) ops[t].kind = ops[t].neg ? TOP_NEG : TOP_PHASE;
    } else {
      for (size_t s = i; s < j; s += kPolyMaxRun) {
        const size_t e = std::min(j, s + (size_t)kPolyMaxRun);
        uint32_t any = 0;
        for (size_t t = s; t < e; ++t) any |= ops[t].ptab;
        TileOp& h = ops[s];
        h.kind = TOP_POLY;
        h.k = (uint8_t)(e - s);
        // The sum of the m's has no bits below the lowest bit set in any m.
        h.nloc = any == 0 ? 5 : any == 0x80000000u ? 4 : (uint8_t)(__builtin_ctz(any) / 8);
      }
    }
    i = j;
  }
}

// Ops that only move amplitudes or flip signs: a block of these runs exactly
// in any precision policy.
inline bool moves_only(const std::vector<TileOp>& ops) {
  for (const TileOp& op : ops) {
    switch (op.kind) {
      case TOP_LAYOUT: case TOP_XSWAP: case TOP_Y: case TOP_NEG: case TOP_PERM: case TOP_SWAPBITS: break;
      case TOP_POLY: if (op.nloc < 4) return false; break;
      case TOP_TERM: break;
      default: return false;
    }
  }
  return true;
}

// Scheduled-op cost of one gate: an op, plus a layout change for gates that
// need register bits (diagonal gates never do).
inline int op_weight(const FGate& g) { return g.diagonal ? 1 : 2; }

// Estimated pool use of one gate.
inline void pool_need(const FGate& g, int* coefs, int* perm_bytes) {
  *coefs = 0;
  *perm_bytes = 0;
  if (g.kind == kGatePattern)
    *coefs = 1;
  else if (g.kind == QS_GATE_PERM)
    *perm_bytes = 1 << g.k;
  else if (g.kind == QS_GATE_DIAG || g.diagonal)
    *coefs = 1 << g.k;
  else if (g.k == 2)
    *coefs = 16;  // or a 4-entry permutation table
  else
    *coefs = 4;
  if (g.k == 2 && !g.diagonal && g.kind == QS_GATE_UK) *perm_bytes = 4;
}

// Choose the next block starting at the first untaken gate.  Returns the
// member indices (in application order) and the geometry; an empty result
// means gate `next` cannot be placed in a tile with these limits.  With
// perms_only, only permutation gates join (moves cost no arithmetic, so such
// a block can take more high qubits than the arithmetic blocks).
inline std::vector<size_t> choose_block(const std::vector<FGate>& gates, const std::vector<char>& taken, size_t next,
                                        int n, int tile_log, int max_high, int min_chunk_log, Limits lim,
                                        size_t window, Geom* geom_out, bool perms_only = false) {
  std::vector<size_t> members;
  const FGate& g0 = gates[next];
  Geom geom;
  if (!tileable(g0) || !geometry(g0.tmask, n, tile_log, max_high, min_chunk_log, &geom)) return members;
  uint64_t need = 0, blocked = 0;
  const uint64_t all = n >= 64 ? ~0ull : ((1ull << n) - 1ull);
  int ops = 0, coefs = 0, pbytes = 0;
  for (size_t i = next; i < gates.size() && i < next + window; ++i) {
    if (taken[i]) continue;
    const FGate& g = gates[i];
    bool ok = tileable(g) && !(g.qubit_mask & blocked) && (!perms_only || g.kind == QS_GATE_PERM);
    Geom trial;
    int c_need = 0, p_need = 0;
    pool_need(g, &c_need, &p_need);
    if (ok) ok = geometry(need | g.tmask, n, tile_log, max_high, min_chunk_log, &trial);
    if (ok && (ops + op_weight(g) > lim.ops || coefs + c_need > lim.coefs || pbytes + p_need > lim.perm_bytes))
      ok = false;
    if (ok) {
      members.push_back(i);
      need |= g.tmask;
      geom = trial;
      ops += op_weight(g);
      coefs += c_need;
      pbytes += p_need;
    } else {
      blocked |= g.qubit_mask;
      if (blocked == all) break;
    }
  }
  *geom_out = geom;
  return members;
}

}  // namespace fuser
}  // namespace qs
