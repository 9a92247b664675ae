// Split states: a state of n qubits whose top g qubits select one of 2^g
// contiguous segments of 2^(n-g) amplitudes, each held either in HBM or in
// host memory that the GPU reads and writes directly (pinned, mapped;
// NVLink-C2C on Grace).  This carries the paper's NUMA placement (Sec. II-B:
// the state spread over two memories, each part processed where it lives)
// over to a GPU whose state outgrows its HBM.
//
// Gates on local qubits (the low n - g) run on every segment with the
// ordinary kernels; a control on a global qubit selects the segments whose
// index bit is 1; a diagonal gate's global targets are fixed per segment, so
// each segment gets the sub-table (or a scalar phase).  A gate that needs a
// global qubit as a target first swaps that qubit with the top local one: a
// SWAP between a global and the top local qubit exchanges the upper half of
// one segment with the lower half of its partner (contiguous halves).  A
// logical -> physical qubit map records these swaps; copies out, gathers and
// marginals first restore the identity map.  Two global qubits swap by
// renaming segments (no data moves).
//
// Host-resident segments use only the per-gate kernels (plain loads and
// stores); HBM segments also run fused blocks.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "qs_internal.h"

namespace qs {

qs_status run_fused(qs_state s, const qs_circuit* c, int max_high);  // qs_tile.cu
int fuse_width_for(qs_state s);                                     // qs_circuit.cu
qs_status qs_fuse_run_gatewise(qs_state s, const qs_circuit* c);     // qs_circuit.cu

struct SplitInfo {
  int g = 0, L = 0;
  std::vector<qs_state> seg;  // sub-states of L qubits over the segments
  std::vector<char> on_host;  // segment placement (index = segment)
  std::vector<int> phys;      // logical qubit -> physical position
  std::vector<int> logi;      // physical position -> logical qubit
};

namespace {

SplitInfo* info(qs_state s) { return static_cast<SplitInfo*>(s->split); }

template <class Amp>
__global__ void k_zero(Amp* __restrict__ p, uint64_t count) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  Amp z = {};
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) p[i] = z;
}

template <class Amp>
__global__ void k_one(Amp* __restrict__ p, uint64_t at) {
  Amp one = {};
  one.x = 1;
  p[at] = one;
}

// Exchange a[0..count) with b[0..count) (two halves of two segments).
template <class Amp>
__global__ void k_swap_halves(Amp* __restrict__ a, Amp* __restrict__ b, uint64_t count) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    const Amp x = a[i], y = b[i];
    a[i] = y;
    b[i] = x;
  }
}

unsigned grid_for_count(qs_state s, uint64_t count) {
  const uint64_t want = (count + 255) / 256;
  const uint64_t cap = (uint64_t)sm_count(s->device) * 8;
  return (unsigned)std::max<uint64_t>(1, std::min(want, cap));
}

qs_status zero_segment(qs_state seg) {
  const uint64_t count = 1ull << seg->n;
  if (seg->dtype == QS_C64)
    k_zero<float2><<<grid_for_count(seg, count), 256, 0, seg->stream>>>((float2*)seg->psi, count);
  else
    k_zero<double2><<<grid_for_count(seg, count), 256, 0, seg->stream>>>((double2*)seg->psi, count);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

qs_status set_one(qs_state seg, uint64_t at) {
  if (seg->dtype == QS_C64)
    k_one<float2><<<1, 1, 0, seg->stream>>>((float2*)seg->psi, at);
  else
    k_one<double2><<<1, 1, 0, seg->stream>>>((double2*)seg->psi, at);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

void reset_map(SplitInfo* si, int n) {
  si->phys.resize(n);
  si->logi.resize(n);
  for (int q = 0; q < n; ++q) si->phys[q] = si->logi[q] = q;
}

void swap_map(SplitInfo* si, int p0, int p1) {
  std::swap(si->logi[p0], si->logi[p1]);
  si->phys[si->logi[p0]] = p0;
  si->phys[si->logi[p1]] = p1;
}

const uint32_t kSwapTable[4] = {0u, 2u, 1u, 3u};

// SWAP of two local physical positions on every segment.
qs_status local_swap(qs_state s, int p0, int p1) {
  SplitInfo* si = info(s);
  const int t[2] = {p0, p1};
  for (qs_state seg : si->seg) {
    qs_status st = dispatch_perm(seg, t, 2, 0, kSwapTable);
    if (st != QS_OK) return st;
  }
  swap_map(si, p0, p1);
  return QS_OK;
}

// SWAP of global position P with the top local position L - 1: the upper
// half of each segment whose bit P - L is 0 trades places with the lower half
// of its partner.
qs_status global_swap_top(qs_state s, int P) {
  SplitInfo* si = info(s);
  const int L = si->L;
  const uint32_t bit = 1u << (P - L);
  const uint64_t half = 1ull << (L - 1);
  for (uint32_t a = 0; a < (uint32_t)si->seg.size(); ++a) {
    if (a & bit) continue;
    qs_state sa = si->seg[a], sb = si->seg[a | bit];
    if (s->dtype == QS_C64)
      k_swap_halves<float2><<<grid_for_count(s, half), 256, 0, s->stream>>>((float2*)sa->psi + half, (float2*)sb->psi,
                                                                            half);
    else
      k_swap_halves<double2><<<grid_for_count(s, half), 256, 0, s->stream>>>((double2*)sa->psi + half,
                                                                              (double2*)sb->psi, half);
    QS_CUDA(cudaGetLastError());
  }
  swap_map(si, P, L - 1);
  return QS_OK;
}

// SWAP of two global positions: rename the segments.
void global_rename(qs_state s, int P0, int P1) {
  SplitInfo* si = info(s);
  const int b0 = P0 - si->L, b1 = P1 - si->L;
  std::vector<qs_state> seg(si->seg.size());
  std::vector<char> host(si->seg.size());
  for (uint32_t a = 0; a < (uint32_t)seg.size(); ++a) {
    const uint32_t x = ((a >> b0) ^ (a >> b1)) & 1u;
    const uint32_t to = a ^ ((x << b0) | (x << b1));
    seg[to] = si->seg[a];
    host[to] = si->on_host[a];
  }
  si->seg.swap(seg);
  si->on_host.swap(host);
  swap_map(si, P0, P1);
}

// Make global position P local: it takes the place of the highest local
// position not in `avoid` (moved to L - 1 first if needed).  Returns the
// local position the qubit now occupies (L - 1).
qs_status bring_local(qs_state s, int P, uint64_t avoid) {
  SplitInfo* si = info(s);
  const int L = si->L;
  int V = -1;
  for (int v = L - 1; v >= 0; --v)
    if (!((avoid >> v) & 1ull)) {
      V = v;
      break;
    }
  if (V < 0) return fail(QS_ERR_UNSUPPORTED, "split state: no free local qubit to swap a global qubit into");
  if (V != L - 1) {
    qs_status st = local_swap(s, V, L - 1);
    if (st != QS_OK) return st;
  }
  return global_swap_top(s, P);
}

// Restore the identity map (physical position q holds logical qubit q).
qs_status canonicalize(qs_state s) {
  SplitInfo* si = info(s);
  const int L = si->L, n = s->n;
  for (int P = L; P < n; ++P) {
    if (si->logi[P] == P) continue;
    const int X = si->phys[P];
    if (X >= L) {
      global_rename(s, P, X);
      continue;
    }
    if (X != L - 1) {
      qs_status st = local_swap(s, X, L - 1);
      if (st != QS_OK) return st;
    }
    qs_status st = global_swap_top(s, P);
    if (st != QS_OK) return st;
  }
  for (int p = 0; p < L; ++p) {
    if (si->logi[p] == p) continue;
    qs_status st = local_swap(s, p, si->phys[p]);
    if (st != QS_OK) return st;
  }
  return QS_OK;
}

// One segment's share of a run of gates: records and pools of a qs_circuit.
struct SegCirc {
  std::vector<qs_gate> gates;
  std::vector<double> data;
  std::vector<uint32_t> perm;
  void clear() {
    gates.clear();
    data.clear();
    perm.clear();
  }
  void add(int kind, int k, const int* targets, uint64_t ctrl, const double* d, size_t nd, const uint32_t* p,
           size_t np) {
    qs_gate g;
    std::memset(&g, 0, sizeof(g));
    g.kind = kind;
    g.k = k;
    for (int j = 0; j < k; ++j) g.targets[j] = targets[j];
    g.ctrl_mask = ctrl;
    if (kind == QS_GATE_PERM) {
      g.offset = (int64_t)perm.size();
      perm.insert(perm.end(), p, p + np);
    } else {
      g.offset = (int64_t)data.size();
      data.insert(data.end(), d, d + nd);
    }
    gates.push_back(g);
  }
  qs_circuit view() const {
    qs_circuit c;
    c.n_gates = (int64_t)gates.size();
    c.gates = gates.data();
    c.data = data.empty() ? nullptr : data.data();
    c.perm = perm.empty() ? nullptr : perm.data();
    return c;
  }
};

bool matrix_diagonal(const double* M, int dim) {
  for (int r = 0; r < dim; ++r)
    for (int c = 0; c < dim; ++c)
      if (r != c && (M[2 * (r * dim + c)] != 0.0 || M[2 * (r * dim + c) + 1] != 0.0)) return false;
  return true;
}

// Run every segment's pending share: fused on HBM segments, gate by gate on
// host-resident ones.
qs_status flush_run(qs_state s, std::vector<SegCirc>& pend, int max_fuse) {
  SplitInfo* si = info(s);
  int64_t fused = 0, single = 0;
  for (size_t a = 0; a < pend.size(); ++a) {
    if (pend[a].gates.empty()) continue;
    qs_state seg = si->seg[a];
    const qs_circuit c = pend[a].view();
    qs_status st;
    if (si->on_host[a] || max_fuse == 1) {
      st = qs_fuse_run_gatewise(seg, &c);
      single += c.n_gates;
    } else {
      seg->run_fused_launches = 0;
      seg->run_gate_launches = 0;
      seg->run_dense_blocks = 0;
      seg->run_dense_gates = 0;
      st = run_fused(seg, &c, max_fuse == 0 ? fuse_width_for(seg) : max_fuse);
      fused += seg->run_fused_launches;
      single += seg->run_gate_launches;
      s->run_dense_blocks += seg->run_dense_blocks;
      s->run_dense_gates += seg->run_dense_gates;
    }
    if (st != QS_OK) return st;
    pend[a].clear();
  }
  s->run_fused_launches += fused;
  s->run_gate_launches += single;
  return QS_OK;
}

}  // namespace


// Apply circuit c (gates validated against s) to a split state.
qs_status split_run(qs_state s, const qs_circuit* c, int max_fuse) {
  SplitInfo* si = info(s);
  const int L = si->L;
  const uint64_t lmask = (1ull << L) - 1ull;
  const uint32_t nseg = (uint32_t)si->seg.size();
  std::vector<SegCirc> pend(nseg);
  s->run_fused_launches = 0;
  s->run_gate_launches = 0;
  s->run_dense_blocks = 0;
  s->run_dense_gates = 0;
  for (int64_t gi = 0; gi < c->n_gates; ++gi) {
    const qs_gate& g = c->gates[gi];
    const int k = g.k;
    const int dim = 1 << k;
    const double* d = g.kind == QS_GATE_PERM ? nullptr : c->data + g.offset;
    const uint32_t* pt = g.kind == QS_GATE_PERM ? c->perm + g.offset : nullptr;
    const bool diagonal = g.kind == QS_GATE_DIAG ||
                          ((g.kind == QS_GATE_U1 || g.kind == QS_GATE_UK) && matrix_diagonal(d, dim));
    auto mapped = [&](int* tp, uint64_t* cp) {
      for (int j = 0; j < k; ++j) tp[j] = si->phys[g.targets[j]];
      uint64_t cm = 0;
      for (int q = 0; q < s->n; ++q)
        if ((g.ctrl_mask >> q) & 1ull) cm |= 1ull << si->phys[q];
      *cp = cm;
    };
    int tp[QS_MAX_TARGETS];
    uint64_t cp = 0;
    mapped(tp, &cp);
    if (!diagonal) {
      for (int j = 0; j < k; ++j) {
        if (tp[j] < L) continue;
        qs_status st = flush_run(s, pend, max_fuse);
        if (st != QS_OK) return st;
        uint64_t avoid = cp & lmask;
        for (int i = 0; i < k; ++i)
          if (tp[i] < L) avoid |= 1ull << tp[i];
        st = bring_local(s, tp[j], avoid);
        if (st != QS_OK) return st;
        mapped(tp, &cp);
      }
    }
    const uint64_t cglob = cp >> L, cloc = cp & lmask;
    for (uint32_t a = 0; a < nseg; ++a) {
      if ((cglob & ~(uint64_t)a) != 0) continue;  // a global control is 0 in this segment
      if (!diagonal) {
        pend[a].add(g.kind, k, tp, cloc, d, d ? (size_t)(g.kind == QS_GATE_U1 ? 8 : 2 * dim * dim) : 0, pt,
                    pt ? (size_t)dim : 0);
        continue;
      }
      // Diagonal: the global targets' bits are fixed by the segment.
      int lt[QS_MAX_TARGETS], lj[QS_MAX_TARGETS], nl = 0;
      uint32_t fixed = 0;
      for (int j = 0; j < k; ++j) {
        if (tp[j] < L) {
          lt[nl] = tp[j];
          lj[nl] = j;
          ++nl;
        } else if ((a >> (tp[j] - L)) & 1u) {
          fixed |= 1u << j;
        }
      }
      auto entry = [&](uint32_t v) -> const double* {
        return g.kind == QS_GATE_DIAG ? d + 2 * v : d + 2 * (v * dim + v);
      };
      std::vector<double> sub(2u << nl);
      bool ident = true;
      for (uint32_t u = 0; u < (1u << nl); ++u) {
        uint32_t v = fixed;
        for (int j = 0; j < nl; ++j)
          if ((u >> j) & 1u) v |= 1u << lj[j];
        sub[2 * u] = entry(v)[0];
        sub[2 * u + 1] = entry(v)[1];
        ident = ident && sub[2 * u] == 1.0 && sub[2 * u + 1] == 0.0;
      }
      if (ident) continue;
      if (nl > 0) {
        pend[a].add(QS_GATE_DIAG, nl, lt, cloc, sub.data(), sub.size(), nullptr, 0);
      } else {
        // A scalar phase on the segment (under its local controls): a 1-qubit
        // diagonal diag(z, z) on a local qubit that is not a control.
        int q = 0;
        while ((cloc >> q) & 1ull) ++q;
        const double zz[4] = {sub[0], sub[1], sub[0], sub[1]};
        pend[a].add(QS_GATE_DIAG, 1, &q, cloc, zz, 4, nullptr, 0);
      }
    }
  }
  return flush_run(s, pend, max_fuse);
}

qs_status split_gate(qs_state s, int kind, const int* targets, int k, uint64_t ctrl_mask, const double* data,
                     size_t ndata, const uint32_t* perm) {
  qs_gate g;
  std::memset(&g, 0, sizeof(g));
  g.kind = kind;
  g.k = k;
  for (int j = 0; j < k; ++j) g.targets[j] = targets[j];
  g.ctrl_mask = ctrl_mask;
  g.offset = 0;
  qs_circuit c;
  c.n_gates = 1;
  c.gates = &g;
  c.data = data;
  c.perm = perm;
  (void)ndata;
  return split_run(s, &c, 1);
}

// ---------------------------------------------------------------------------
// State-level operations on split states (called by the C ABI in qs_api.cu)
// ---------------------------------------------------------------------------
qs_status split_init_basis(qs_state s, uint64_t idx) {
  SplitInfo* si = info(s);
  reset_map(si, s->n);
  for (qs_state seg : si->seg) {
    qs_status st = zero_segment(seg);
    if (st != QS_OK) return st;
  }
  return set_one(si->seg[idx >> si->L], idx & ((1ull << si->L) - 1ull));
}

qs_status split_copy_in(qs_state s, const void* host) {
  SplitInfo* si = info(s);
  reset_map(si, s->n);  // the input is in logical order
  const size_t bytes = amp_bytes(s->dtype) << si->L;
  for (size_t a = 0; a < si->seg.size(); ++a)
    QS_CUDA(cudaMemcpyAsync(si->seg[a]->psi, (const char*)host + a * bytes, bytes, cudaMemcpyDefault, s->stream));
  return QS_OK;
}

qs_status split_copy_out(qs_state s, void* host, bool sync) {
  SplitInfo* si = info(s);
  qs_status st = canonicalize(s);
  if (st != QS_OK) return st;
  const size_t bytes = amp_bytes(s->dtype) << si->L;
  for (size_t a = 0; a < si->seg.size(); ++a)
    QS_CUDA(cudaMemcpyAsync((char*)host + a * bytes, si->seg[a]->psi, bytes, cudaMemcpyDefault, s->stream));
  if (!sync) return QS_OK;
  QS_CUDA(cudaStreamSynchronize(s->stream));
  return split_check(s);
}

qs_status split_gather(qs_state s, const uint64_t* idx, int64_t count, void* host_out) {
  SplitInfo* si = info(s);
  qs_status st = canonicalize(s);
  if (st != QS_OK) return st;
  const size_t ab = amp_bytes(s->dtype);
  const uint64_t lmask = (1ull << si->L) - 1ull;
  for (uint32_t a = 0; a < (uint32_t)si->seg.size(); ++a) {
    std::vector<uint64_t> loc;
    std::vector<int64_t> where;
    for (int64_t j = 0; j < count; ++j)
      if ((idx[j] >> si->L) == a) {
        loc.push_back(idx[j] & lmask);
        where.push_back(j);
      }
    if (loc.empty()) continue;
    std::vector<unsigned char> buf(loc.size() * ab);
    st = run_gather(si->seg[a], loc.data(), (int64_t)loc.size(), buf.data());
    if (st != QS_OK) return st;
    for (size_t j = 0; j < loc.size(); ++j) std::memcpy((char*)host_out + where[j] * ab, buf.data() + j * ab, ab);
  }
  return QS_OK;
}

qs_status split_norm(qs_state s, double* out) {
  SplitInfo* si = info(s);
  double sum = 0.0;
  for (qs_state seg : si->seg) {
    double v = 0.0;
    qs_status st = run_norm(seg, &v);
    if (st != QS_OK) return st;
    sum += v;
  }
  *out = sum;
  return QS_OK;
}

// Marginals: each segment contributes its local marginal to the outcomes
// whose global bits are the segment's.
qs_status split_probs(qs_state s, const int* qubits, int k, double* out) {
  SplitInfo* si = info(s);
  qs_status st = canonicalize(s);
  if (st != QS_OK) return st;
  const int L = si->L;
  int lq[16], lj[16], nl = 0;
  for (int j = 0; j < k; ++j)
    if (qubits[j] < L) {
      lq[nl] = qubits[j];
      lj[nl] = j;
      ++nl;
    }
  std::fill(out, out + ((size_t)1 << k), 0.0);
  std::vector<double> part((size_t)1 << nl);
  for (uint32_t a = 0; a < (uint32_t)si->seg.size(); ++a) {
    st = nl ? run_probs(si->seg[a], lq, nl, part.data()) : run_norm(si->seg[a], part.data());
    if (st != QS_OK) return st;
    uint64_t gbits = 0;
    for (int j = 0; j < k; ++j)
      if (qubits[j] >= L && ((a >> (qubits[j] - L)) & 1u)) gbits |= 1ull << j;
    for (uint64_t u = 0; u < part.size(); ++u) {
      uint64_t v = gbits;
      for (int j = 0; j < nl; ++j)
        if ((u >> j) & 1ull) v |= 1ull << lj[j];
      out[v] += part[u];
    }
  }
  return QS_OK;
}

// Device errors recorded by any segment's kernels.
qs_status split_check(qs_state s) {
  qs_status first = QS_OK;
  for (qs_state seg : info(s)->seg) {
    qs_status st = device_error_check(seg);
    if (st != QS_OK && first == QS_OK) first = st;
  }
  return first;
}

void split_set_stream(qs_state s, cudaStream_t stream) {
  for (qs_state seg : info(s)->seg) seg->stream = stream;
}

void split_set_math(qs_state s, qs_math math) {
  for (qs_state seg : info(s)->seg) seg->math = math;
}

void split_set_tensor_cores(qs_state s, int enable) {
  for (qs_state seg : info(s)->seg) seg->tensor_cores = enable;
}

void split_destroy(qs_state s) {
  SplitInfo* si = info(s);
  cudaStreamSynchronize(s->stream);
  for (size_t a = 0; a < si->seg.size(); ++a) {
    qs_state seg = si->seg[a];
    if (!seg) continue;
    if (seg->psi) {
      if (si->on_host[a])
        cudaFreeHost(seg->psi);
      else
        cudaFree(seg->psi);
    }
    seg->psi = nullptr;
    free_sub_state(seg);
  }
  delete si;
  s->split = nullptr;
}

}  // namespace qs

using namespace qs;

extern "C" qs_status qs_create_split(int n, qs_dtype dtype, int g, int hbm_segments, qs_state* out) {
  if (!out) return fail(QS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (dtype != QS_C64 && dtype != QS_C128) return fail(QS_ERR_ARG, "unknown dtype %d", (int)dtype);
  if (g < 1 || g > 6) return fail(QS_ERR_ARG, "g = %d outside [1, 6]", g);
  if (n - g < 10 || n > QS_MAX_QUBITS)
    return fail(QS_ERR_ARG, "n = %d: a split state needs 10 <= n - g and n <= %d", n, (int)QS_MAX_QUBITS);
  if (hbm_segments < 0 || hbm_segments > (1 << g))
    return fail(QS_ERR_ARG, "hbm_segments = %d outside [0, %d]", hbm_segments, 1 << g);
  qs_state s = new_sub_state(n, dtype, nullptr);
  if (!s) return fail(QS_ERR_OOM, "host allocation failed");
  SplitInfo* si = new (std::nothrow) SplitInfo();
  if (!si) {
    free_sub_state(s);
    return fail(QS_ERR_OOM, "host allocation failed");
  }
  s->split = si;
  si->g = g;
  si->L = n - g;
  const size_t bytes = amp_bytes(dtype) << si->L;
  qs_status st = QS_OK;
  for (int a = 0; a < (1 << g) && st == QS_OK; ++a) {
    const bool host = a >= hbm_segments;
    void* p = nullptr;
    cudaError_t e = host ? cudaHostAlloc(&p, bytes, cudaHostAllocPortable | cudaHostAllocMapped) : cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      st = cuda_fail(e, host ? "cudaHostAlloc(segment)" : "cudaMalloc(segment)");
      break;
    }
    qs_state seg = new_sub_state(si->L, dtype, p);
    if (!seg) {
      host ? cudaFreeHost(p) : cudaFree(p);
      st = fail(QS_ERR_OOM, "host allocation failed");
      break;
    }
    seg->device = s->device;
    si->seg.push_back(seg);
    si->on_host.push_back(host ? 1 : 0);
  }
  if (st == QS_OK) st = ensure_phase_tables(s->device);
  if (st == QS_OK) st = split_init_basis(s, 0);
  if (st == QS_OK) {
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) st = cuda_fail(e, "split state init");
  }
  if (st != QS_OK) {
    split_destroy(s);
    free_sub_state(s);
    return st;
  }
  *out = s;
  return QS_OK;
}
