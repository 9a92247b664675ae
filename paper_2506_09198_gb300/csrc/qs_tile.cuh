// Fused-block ("tile") engine: plan layout shared by the host fuser and the
// kernel.
//
// A tile is 2^(L+m) amplitudes: 2^m chunks of 2^L contiguous amplitudes,
// chunk c at global offset base + sum_j bit_j(c) 2^hq[j].  Local index
// lambda = c 2^L + o maps local bit b < L to global qubit b and local bit
// L + j to global qubit hq[j]; the remaining ("free") qubits select the tile
// (its base).  Every gate of a block whose targets are tile qubits is applied
// in shared memory, so the whole block costs one read and one write of the
// state.  Diagonal gates need no tile qubits at all: their free-qubit bits are
// constant per tile.
#pragma once
#include <cstdint>

#include "qs_math.cuh"

namespace qs {

constexpr int kTileMaxOps = 40;
constexpr int kTileMaxHigh = 8;
constexpr int kTileMaxChunks = 1 << kTileMaxHigh;
constexpr int kTileMaxCoefs = 320;
constexpr int kTileMaxPermBytes = 512;
constexpr int kTileMaxPos = 14;  // inserted local bit positions per op

enum TileOpKind : uint8_t {
  TOP_DENSE1 = 0,  // 2x2 on local bit tpos[0]
  TOP_DENSE2 = 1,  // 4x4 on local bits tpos[0], tpos[1] (index b0 + 2 b1)
  TOP_PHASE = 2,   // multiply the amplitudes that match a bit pattern by one coefficient
  TOP_NEG = 3,     // same with coefficient -1 (sign flip)
  TOP_DIAG = 4,    // d[s], s from local target bits and tile-constant bits
  TOP_XSWAP = 5,   // swap pair partners on local bit tpos[0]
  TOP_Y = 6,       // up' = -i lo, lo' = i up
  TOP_PERM = 7     // index permutation of local target bits (inverse table)
};

struct TileOp {
  uint8_t kind;
  uint8_t k;                  // DIAG / PERM: number of targets
  uint8_t npos;               // positions inserted to enumerate items
  uint8_t nloc;               // DIAG: local targets
  uint32_t himask[kTileMaxPos];  // ~((1 << pos) - 1) for the ascending local positions inserted
                                 // (targets' 0s, controls' 1s)
  uint8_t tpos[8];            // local positions of targets
  uint8_t tj[8];              // DIAG: sub-register bit of each local target
  uint8_t gq[8];              // DIAG: global qubit of target j when it is not local, else 0xFF
  uint32_t ifixed;            // bits set after insertion (local controls / pattern ones)
  uint32_t lmask;             // PERM: local control mask
  uint64_t gmask, gpat;       // the op acts on a tile iff (base & gmask) == gpat
  uint16_t coef;              // first coefficient in the plan's pool
  uint16_t ptab;              // PERM: byte offset of the inverse table
};

template <class Coef>
struct TilePlan {
  int n;
  int L, m;                            // chunk = 2^L amplitudes, 2^m chunks per tile
  int nops;
  uint64_t n_tiles;
  uint64_t base_high[kTileMaxHigh];    // ~((1 << hq[j]) - 1), ascending: tile base expansion
  uint64_t chunk_off[kTileMaxChunks];  // amplitude offset of chunk c from the base
  TileOp ops[kTileMaxOps];
  Coef coefs[kTileMaxCoefs];
  uint8_t perm[kTileMaxPermBytes];
};

}  // namespace qs
