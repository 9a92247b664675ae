// Dense-block fusion ahead of block formation (host).
//
// A dense gate on more than two targets has no tile op: it costs one pass of
// its own (the dense-gate kernels).  Starting from such a gate, the gates
// after it that act only on the block's qubits, or that widen the block to at
// most QS_MAX_DENSE qubits while touching it, are multiplied into one
// 2^m x 2^m matrix in FP64 (m <= 5).  A gate that cannot join is stepped over,
// and the qubits it touches are closed to the block from then on, so every
// absorbed gate commutes with every gate stepped over; the product takes the
// place of the first absorbed gate.  One pass then applies what would have
// taken one pass per dense gate (gate fusion, Sec. I).
#pragma once
#include <complex>
#include <deque>
#include <vector>

#include "qs_fuser.h"

namespace qs {
namespace fuser {

// Apply gate g to a vector over the ordered qubits q[0..m-1] (local bit j of
// the index is qubit q[j]); every target, control and pattern bit of g is
// one of them.
inline void apply_local(const FGate& g, const int* q, int m, std::complex<double>* v) {
  using cplx = std::complex<double>;
  const int d = 1 << m;
  auto lbit = [&](int qubit) {
    for (int j = 0; j < m; ++j)
      if (q[j] == qubit) return j;
    return 0;
  };
  if (g.kind == kGatePattern) {
    uint32_t pm = 0, pv = 0;
    for (int j = 0; j < m; ++j)
      if ((g.pmask >> q[j]) & 1ull) {
        pm |= 1u << j;
        if ((g.ppat >> q[j]) & 1ull) pv |= 1u << j;
      }
    const cplx c(g.data[0], g.data[1]);
    for (int i = 0; i < d; ++i)
      if (((uint32_t)i & pm) == pv) v[i] *= c;
    return;
  }
  uint32_t cm = 0;
  for (int j = 0; j < m; ++j)
    if ((g.ctrl >> q[j]) & 1ull) cm |= 1u << j;
  int lt[QS_MAX_TARGETS];
  for (int j = 0; j < g.k; ++j) lt[j] = lbit(g.targets[j]);
  std::vector<cplx> out(v, v + d);
  const int dim = 1 << g.k;
  for (int i = 0; i < d; ++i) {
    if (((uint32_t)i & cm) != cm) continue;
    int sub = 0, rest = i;
    for (int j = 0; j < g.k; ++j) {
      sub |= ((i >> lt[j]) & 1) << j;
      rest &= ~(1 << lt[j]);
    }
    auto index = [&](int s) {
      int x = rest;
      for (int j = 0; j < g.k; ++j) x |= ((s >> j) & 1) << lt[j];
      return x;
    };
    if (g.kind == QS_GATE_DIAG) {
      out[i] = cplx(g.data[2 * sub], g.data[2 * sub + 1]) * v[i];
    } else if (g.kind == QS_GATE_PERM) {
      out[index((int)g.perm[sub])] = v[i];
    } else {
      cplx acc = 0.0;
      for (int c = 0; c < dim; ++c) acc += cplx(g.data[2 * (sub * dim + c)], g.data[2 * (sub * dim + c) + 1]) * v[index(c)];
      out[i] = acc;
    }
  }
  for (int i = 0; i < d; ++i) v[i] = out[i];
}

class DenseFuser {
 public:
  // Returns the gate list with dense blocks composed; matrices it creates
  // live in this object.
  std::vector<FGate> run(const std::vector<FGate>& in) {
    store_.clear();
    blocks_ = absorbed_ = 0;
    std::vector<FGate> out;
    out.reserve(in.size());
    std::vector<char> used(in.size(), 0);
    for (size_t i = 0; i < in.size(); ++i) {
      if (used[i]) continue;
      const FGate& g = in[i];
      if (!seed(g) || __builtin_popcountll(g.qubit_mask) > QS_MAX_DENSE) {
        out.push_back(g);
        continue;
      }
      uint64_t Q = g.qubit_mask, blocked = 0;
      std::vector<size_t> members{i};
      for (size_t j = i + 1; j < in.size() && j < i + kWindow; ++j) {
        if (used[j]) continue;
        const uint64_t hm = in[j].qubit_mask;
        const bool fits = (hm & blocked) == 0 && (hm & Q) != 0 && __builtin_popcountll(Q | hm) <= QS_MAX_DENSE;
        if (fits) {
          Q |= hm;
          members.push_back(j);
        } else {
          blocked |= hm;
          if ((Q & ~blocked) == 0) break;  // nothing can join any more
        }
      }
      if (members.size() < 2) {
        out.push_back(g);
        continue;
      }
      for (size_t j : members) used[j] = 1;
      out.push_back(compose(in, members, Q));
      ++blocks_;
      absorbed_ += (int64_t)members.size();
    }
    return out;
  }

  int64_t blocks() const { return blocks_; }
  int64_t absorbed() const { return absorbed_; }

 private:
  static constexpr size_t kWindow = 256;
  std::deque<std::vector<double>> store_;
  int64_t blocks_ = 0, absorbed_ = 0;

  // A dense gate no tile op expresses.
  static bool seed(const FGate& g) { return g.kind == QS_GATE_UK && !g.diagonal && !tileable(g); }

  FGate compose(const std::vector<FGate>& in, const std::vector<size_t>& members, uint64_t Q) {
    int q[QS_MAX_DENSE];
    int m = 0;
    for (int b = 0; b < 64; ++b)
      if ((Q >> b) & 1ull) q[m++] = b;
    const int d = 1 << m;
    store_.emplace_back((size_t)2 * d * d);
    std::vector<double>& M = store_.back();
    std::vector<std::complex<double>> v(d);
    for (int c = 0; c < d; ++c) {
      for (int r = 0; r < d; ++r) v[r] = r == c ? 1.0 : 0.0;
      for (size_t j : members) apply_local(in[j], q, m, v.data());
      for (int r = 0; r < d; ++r) {
        M[2 * (r * d + c)] = v[r].real();
        M[2 * (r * d + c) + 1] = v[r].imag();
      }
    }
    FGate f;
    std::memset(&f, 0, sizeof(f));
    f.kind = QS_GATE_UK;
    f.k = m;
    for (int j = 0; j < m; ++j) f.targets[j] = q[j];
    f.data = M.data();
    f.diagonal = matrix_is_diag(f.data, d);
    f.qubit_mask = Q;
    f.tmask = f.diagonal ? 0 : Q;
    return f;
  }
};

}  // namespace fuser
}  // namespace qs
