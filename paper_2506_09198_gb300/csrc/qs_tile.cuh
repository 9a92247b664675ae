// Fused-block ("tile") engine: op and plan layout shared by the host fuser
// and the kernels.
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

constexpr int kTileMaxOps = 96;  // scheduled ops (gates plus layout changes) per plan
constexpr int kTileMaxHigh = 8;
constexpr int kTileMaxChunks = 1 << kTileMaxHigh;
constexpr int kTileMaxCoefs = 320;
constexpr int kTileMaxPermBytes = 512;
// A block's ops and coefficients are staged in shared memory next to the
// tile ring; this many bytes of coefficients keep two CTAs per SM.
constexpr int kTileMaxCoefBytes = 10752;

// Inside a tile every consumer thread holds 2^RB amplitudes in registers.
// A layout names the RB local bits that index a thread's registers (in
// order); the remaining local bits, ascending, are the thread index.  Gates
// whose targets are register bits run without communication; a layout change
// moves the tile through shared memory.  The host schedules layout changes
// (TOP_LAYOUT) so that every dense gate finds its targets in registers.
enum TileOpKind : uint8_t {
  TOP_LAYOUT = 0,  // new layout: register bit j = local bit tpos[j]
  TOP_DENSE1 = 1,  // 2x2 on register bit tpos[0]; nloc = 1: real coefficients
  TOP_DENSE2 = 2,  // 4x4 on register bits tpos[0], tpos[1] (index b0 + 2 b1)
  TOP_XSWAP = 3,   // swap pair partners on register bit tpos[0]
  TOP_Y = 4,       // up' = -i lo, lo' = i up on register bit tpos[0]
  TOP_PHASE = 5,   // multiply amplitudes with (lambda & lmask) == lpat by one coefficient
  TOP_NEG = 6,     // same with coefficient -1 (sign flip)
  TOP_DIAG = 7,    // d[s]: s from local targets tpos[0..nloc) (sub-register bits tj) and tile bits gq
  TOP_PERM = 8,    // permutation of local targets tpos[0..k), through shared memory
  // A run of k phase terms (this op and the k - 1 TOP_TERM ops after it).
  // Term t adds m_t = ptab (a phase in units of 2^-32 turn) to the
  // accumulator of the amplitude a thread holds in register r when the
  // thread bits match, (lambda & lmask) == lpat, the register bits match,
  // (r & tj[0]) == tj[1], and the tile matches, (base & gmask) == gpat.
  // Terms come grouped by (tj[0], tj[1]).  The amplitude is then multiplied
  // once by exp(2 pi i acc / 2^32), the product of four table entries (one
  // per byte of acc, from byte nloc up); nloc 4: every m is 2^31, so the
  // product is a sign; nloc 5: nothing to do.  tpos[0] = 1 (factored): each
  // group's sum is turned into its phase once per thread and multiplied into
  // the group's registers instead, starting at the group's lowest nonzero
  // byte tj[2].
  TOP_POLY = 9,
  TOP_TERM = 10,
  // Swap of local bits tpos[0], tpos[1] (an uncontrolled SWAP gate): the
  // amplitude a thread holds for local index lambda now belongs at the
  // swapped index, so only the thread's index bookkeeping changes.
  TOP_SWAPBITS = 11
};

// Before scheduling (host), dense gates carry local bit positions in tpos;
// the scheduler rewrites them to register bit indices.
// 64 bytes, 16-byte aligned: the first 16 bytes hold everything a phase
// term reads besides its tile predicate (the next 16), so a term is two
// vector loads.
struct alignas(16) TileOp {
  uint32_t lmask;   // local control mask (PHASE/NEG: pattern mask; POLY/TERM: thread bits)
  uint32_t lpat;    // PHASE/NEG: local pattern (POLY/TERM: thread bits)
  uint32_t coef;    // first coefficient in the pool; POLY/TERM after scheduling:
                    // register mask | register pattern << 8 | first byte << 16
  uint32_t ptab;    // PERM: byte offset of the inverse table; POLY/TERM: m
  uint64_t gmask, gpat;  // the op acts on a tile iff (base & gmask) == gpat
  uint8_t kind;
  uint8_t k;        // DIAG / PERM: number of targets; LAYOUT: register bits
  uint8_t nloc;     // DIAG: local targets
  uint8_t neg;      // TERM before grouping: the term came from a sign flip
  uint8_t tpos[8];
  uint8_t tj[8];    // DIAG: sub-register bit of each local target
  uint8_t gq[8];    // DIAG: global qubit of target j when not local, else 0xFF
  uint8_t pad[4];
};
static_assert(sizeof(TileOp) == 64, "TileOp is 64 bytes");

template <class Coef>
struct TilePlan {
  int n;
  int L, m;                            // chunk = 2^L amplitudes, 2^m chunks per tile
  int nops;
  int ncoefs;
  int fmt;                             // kTileInFF | kTileOutFF: float-float tiles in HBM
  uint64_t n_tiles;
  uint64_t base_high[kTileMaxHigh];    // ~((1 << hq[j]) - 1), ascending: tile base expansion
  uint64_t chunk_off[kTileMaxChunks];  // amplitude offset of chunk c from the base
  TileOp ops[kTileMaxOps];
  Coef coefs[kTileMaxCoefs];
  uint8_t perm[kTileMaxPermBytes];
  const void* phase_tab;               // exp(2 pi i v 2^(8b) / 2^32) at [256 b + v], the policy's format
  uint64_t wait_ns;                    // limit of each bounded wait
};

// Tile storage in HBM between consecutive float-float blocks: the plan's
// input and/or output tile holds (re head, im head, re tail, im tail)
// floats instead of (re, im) doubles.
constexpr int kTileInFF = 1;
constexpr int kTileOutFF = 2;

// Phase terms: runs shorter than this stay single phase ops; a run holds at
// most 255 terms (its count is a byte).
constexpr int kPolyMinRun = 4;
constexpr int kPolyMaxRun = 255;

}  // namespace qs
