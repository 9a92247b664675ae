// Gate-matrix fusion ahead of block formation (host).
//
// Consecutive gates on the same one or two qubits are multiplied into one
// 2x2 or 4x4 matrix in FP64, so a fused block applies their product once
// (the block product of the fused k-qubit gates, composed in double
// precision).  In a random circuit, the two 1q gates of a pair, the CZ
// between them and the next layer's 1q gates on the pair become one 4x4.
// A fused matrix is kept only when its estimated cost is below that of the
// gates it replaces; permutations always stay as they are (they move
// amplitudes exactly).
#pragma once
#include <complex>
#include <deque>
#include <vector>

#include "qs_fuser.h"

namespace qs {
namespace fuser {

using cplx = std::complex<double>;

// Apply gate g to a state over the ordered qubits (q[0], q[1]) (q[1] < 0
// for one qubit): local bit j of the index is qubit q[j].  Every target and
// control of g is one of them.
inline void apply_small(const FGate& g, const int* q, int nq, cplx* v) {
  const int d = 1 << nq;
  auto bit_of = [&](int qubit) { return qubit == q[0] ? 0 : 1; };
  uint32_t cm = 0;
  for (int j = 0; j < nq; ++j)
    if ((g.ctrl >> q[j]) & 1ull) cm |= 1u << j;
  int lt[2] = {0, 0};
  for (int j = 0; j < g.k; ++j) lt[j] = bit_of(g.targets[j]);
  cplx out[4];
  for (int i = 0; i < d; ++i) out[i] = v[i];
  const int dim = 1 << g.k;
  for (int i = 0; i < d; ++i) {
    if ((i & cm) != cm) continue;
    int sub = 0;
    for (int j = 0; j < g.k; ++j) sub |= ((i >> lt[j]) & 1) << j;
    int rest = i;
    for (int j = 0; j < g.k; ++j) rest &= ~(1 << lt[j]);
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
      for (int c = 0; c < dim; ++c) {
        const double* z = g.data + 2 * (sub * dim + c);
        acc += cplx(z[0], z[1]) * v[index(c)];
      }
      out[i] = acc;
    }
  }
  for (int i = 0; i < d; ++i) v[i] = out[i];
}

// Estimated arithmetic per amplitude of one gate inside a tile (float-float
// instruction units; the complex64 ratios are alike).
inline double tile_cost(const FGate& g) {
  if (g.kind == QS_GATE_PERM) return 2.0;
  if (g.diagonal) return 20.0;
  if (g.k == 2) return 65.0;
  const double* U = g.data;
  if (is_c(U, 0, 0) && is_c(U + 6, 0, 0)) return 2.0;  // X / Y-like moves
  const bool real = U[1] == 0.0 && U[3] == 0.0 && U[5] == 0.0 && U[7] == 0.0;
  return real ? 18.0 : 40.0;
}

class MatFuser {
 public:
  // Returns the fused gate list; matrices it creates live in this object.
  std::vector<FGate> run(const std::vector<FGate>& in) {
    in_ = &in;
    out_.clear();
    blocks_.clear();
    store_.clear();
    for (int q = 0; q < 64; ++q) owner_[q] = -1;
    for (size_t i = 0; i < in.size(); ++i) take(i);
    for (size_t b = 0; b < blocks_.size(); ++b)
      if (blocks_[b].alive) flush((int)b);
    return out_;
  }

 private:
  struct Block {
    bool alive = false;
    int q[2] = {-1, -1};
    int nq = 0;
    cplx M[16];  // row-major, dim 2^nq
    std::vector<size_t> members;
    double cost = 0.0;
  };

  const std::vector<FGate>* in_ = nullptr;
  std::vector<FGate> out_;
  std::vector<Block> blocks_;
  std::deque<std::vector<double>> store_;
  int owner_[64];

  static bool mergeable(const FGate& g) {
    if (g.kind == QS_GATE_PERM || g.kind == kGatePattern) return false;
    if (!tileable(g)) return false;
    return __builtin_popcountll(g.qubit_mask) <= 2;
  }
  // Worth opening a block for: a dense (non-diagonal, non-move) matrix.
  static bool starter(const FGate& g) { return !g.diagonal && tile_cost(g) >= 18.0; }

  void flush(int b) {
    Block& B = blocks_[b];
    const int dim = 1 << B.nq;
    FGate f;
    std::memset(&f, 0, sizeof(f));
    f.kind = B.nq == 1 ? QS_GATE_U1 : QS_GATE_UK;
    f.k = B.nq;
    f.targets[0] = B.q[0];
    if (B.nq == 2) f.targets[1] = B.q[1];
    store_.emplace_back(2 * dim * dim);
    std::vector<double>& m = store_.back();
    for (int i = 0; i < dim * dim; ++i) {
      m[2 * i] = B.M[i].real();
      m[2 * i + 1] = B.M[i].imag();
    }
    f.data = m.data();
    f.diagonal = matrix_is_diag(f.data, dim);
    f.qubit_mask = (1ull << B.q[0]) | (B.nq == 2 ? 1ull << B.q[1] : 0ull);
    f.tmask = f.diagonal ? 0 : f.qubit_mask;
    if (B.members.size() > 1 && tile_cost(f) < B.cost) {
      out_.push_back(f);
    } else {
      for (size_t i : B.members) out_.push_back((*in_)[i]);
    }
    for (int j = 0; j < B.nq; ++j) owner_[B.q[j]] = -1;
    B.alive = false;
  }

  // The matrix of gate g on the block's qubits, multiplied in after B.
  void absorb(Block& B, size_t gi) {
    const FGate& g = (*in_)[gi];
    const int dim = 1 << B.nq;
    cplx G[16];
    for (int c = 0; c < dim; ++c) {
      cplx v[4] = {0.0, 0.0, 0.0, 0.0};
      v[c] = 1.0;
      apply_small(g, B.q, B.nq, v);
      for (int r = 0; r < dim; ++r) G[r * dim + c] = v[r];
    }
    cplx P[16];
    for (int r = 0; r < dim; ++r)
      for (int c = 0; c < dim; ++c) {
        cplx acc = 0.0;
        for (int k = 0; k < dim; ++k) acc += G[r * dim + k] * B.M[k * dim + c];
        P[r * dim + c] = acc;
      }
    for (int i = 0; i < dim * dim; ++i) B.M[i] = P[i];
    B.members.push_back(gi);
    B.cost += tile_cost(g);
  }

  int open(int nq, int q0, int q1) {
    Block B;
    B.alive = true;
    B.nq = nq;
    B.q[0] = q0;
    B.q[1] = q1;
    const int dim = 1 << nq;
    for (int i = 0; i < dim * dim; ++i) B.M[i] = (i % (dim + 1) == 0) ? 1.0 : 0.0;
    blocks_.push_back(B);
    const int b = (int)blocks_.size() - 1;
    for (int j = 0; j < nq; ++j) owner_[blocks_[b].q[j]] = b;
    return b;
  }

  // Embed a pending one-qubit block into the two-qubit block `to`.
  void embed(int from, int to) {
    Block& A = blocks_[from];
    Block& B = blocks_[to];
    const int bit = A.q[0] == B.q[0] ? 0 : 1;
    cplx P[16];
    for (int r = 0; r < 4; ++r)
      for (int c = 0; c < 4; ++c) {
        const int ro = (r >> (1 - bit)) & 1, co = (c >> (1 - bit)) & 1;  // the other qubit's bits
        P[r * 4 + c] = ro == co ? A.M[((r >> bit) & 1) * 2 + ((c >> bit) & 1)] : 0.0;
      }
    cplx Q[16];
    for (int r = 0; r < 4; ++r)
      for (int c = 0; c < 4; ++c) {
        cplx acc = 0.0;
        for (int k = 0; k < 4; ++k) acc += P[r * 4 + k] * B.M[k * 4 + c];
        Q[r * 4 + c] = acc;
      }
    for (int i = 0; i < 16; ++i) B.M[i] = Q[i];
    B.members.insert(B.members.end(), A.members.begin(), A.members.end());
    B.cost += A.cost;
    A.alive = false;
    owner_[A.q[0]] = to;
  }

  void take(size_t i) {
    const FGate& g = (*in_)[i];
    int qs_[2] = {-1, -1}, nq = 0;
    for (int q = 0; q < 64 && nq <= 2; ++q)
      if ((g.qubit_mask >> q) & 1ull) {
        if (nq < 2) qs_[nq] = q;
        ++nq;
      }
    if (!mergeable(g) || nq > 2 || nq == 0) {
      for (int j = 0; j < 64; ++j)
        if (((g.qubit_mask >> j) & 1ull) && owner_[j] >= 0) flush(owner_[j]);
      out_.push_back(g);
      return;
    }
    if (nq == 1) {
      const int b = owner_[qs_[0]];
      if (b >= 0) {
        absorb(blocks_[b], i);
      } else if (starter(g)) {
        absorb(blocks_[open(1, qs_[0], -1)], i);
      } else {
        out_.push_back(g);
      }
      return;
    }
    const int a = qs_[0], c = qs_[1];
    const int ba = owner_[a], bc = owner_[c];
    if (ba >= 0 && ba == bc) {  // the pair's block
      absorb(blocks_[ba], i);
      return;
    }
    // Blocks pairing a or c with another qubit end here.
    if (ba >= 0 && blocks_[ba].nq == 2) flush(ba);
    if (bc >= 0 && blocks_[bc].nq == 2) flush(bc);
    const int pa = owner_[a], pc = owner_[c];
    if (pa < 0 && pc < 0 && !starter(g)) {
      out_.push_back(g);
      return;
    }
    const int b = open(2, a, c);
    if (pa >= 0) embed(pa, b);
    if (pc >= 0) embed(pc, b);
    absorb(blocks_[b], i);
  }
};

}  // namespace fuser
}  // namespace qs
