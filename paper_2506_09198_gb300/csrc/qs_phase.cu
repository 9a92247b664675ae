// Phase tables for runs of dyadic phase gates.
//
// A controlled phase of angle 2 pi m / 2^32 (every QFT rotation on up to 32
// qubits, CZ, S, T, Z) adds m to a 32-bit accumulator, which wraps exactly
// at one full turn.  A run of such gates in a fused block then costs one
// integer add per gate and amplitude, and one multiplication by
// exp(2 pi i acc / 2^32) per amplitude, formed from four 256-entry tables
// (one per byte of acc).  The tables live in static device memory: filling
// them is a copy, not an allocation.
#include <array>
#include <cmath>
#include <map>
#include <mutex>

#include "qs_internal.h"

namespace qs {

namespace {

constexpr int kEntries = 4 * 256;
__device__ __align__(16) float2 g_phase_f32[kEntries];
__device__ __align__(16) double2 g_phase_f64[kEntries];
__device__ __align__(16) float4 g_phase_df[kEntries];

std::mutex g_phase_mu;
std::map<int, std::array<void*, 3>> g_phase_ptr;  // per device: f32, f64, df

}  // namespace

// cos and sin of 2 pi m / 2^32, reduced to the first octant so that
// multiples of a quarter turn come out exact (0, +-1).
void turn_cos_sin(uint32_t m, double* c, double* s) {
  const uint32_t quadrant = m >> 30;
  const uint32_t r = m & 0x3FFFFFFFu;
  const double k = 6.283185307179586476925286766559 / 4294967296.0;  // 2 pi / 2^32 (power-of-two scaling)
  double cr, sr;
  if (r == 0) {
    cr = 1.0;
    sr = 0.0;
  } else if (r <= (1u << 29)) {
    cr = std::cos((double)r * k);
    sr = std::sin((double)r * k);
  } else {
    const double a = (double)((1u << 30) - r) * k;  // quarter turn minus the angle
    cr = std::sin(a);
    sr = std::cos(a);
  }
  switch (quadrant) {
    case 0: *c = cr; *s = sr; break;
    case 1: *c = -sr; *s = cr; break;
    case 2: *c = -cr; *s = -sr; break;
    default: *c = sr; *s = -cr; break;
  }
}

qs_status ensure_phase_tables(int device) {
  std::lock_guard<std::mutex> lock(g_phase_mu);
  if (g_phase_ptr.count(device)) return QS_OK;
  static float2 f32[kEntries];
  static double2 f64[kEntries];
  static float4 df[kEntries];
  for (int b = 0; b < 4; ++b)
    for (int v = 0; v < 256; ++v) {
      double c, s;
      turn_cos_sin((uint32_t)v << (8 * b), &c, &s);
      const int i = 256 * b + v;
      f32[i] = make_float2((float)c, (float)s);
      f64[i] = make_double2(c, s);
      const float ch = (float)c, sh = (float)s;
      df[i] = make_float4(ch, sh, (float)(c - (double)ch), (float)(s - (double)sh));
    }
  int prev = 0;
  QS_CUDA(cudaGetDevice(&prev));
  if (prev != device) QS_CUDA(cudaSetDevice(device));
  std::array<void*, 3> ptr{};
  cudaError_t e = cudaMemcpyToSymbol(g_phase_f32, f32, sizeof(f32));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_phase_f64, f64, sizeof(f64));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_phase_df, df, sizeof(df));
  if (e == cudaSuccess) e = cudaGetSymbolAddress(&ptr[0], g_phase_f32);
  if (e == cudaSuccess) e = cudaGetSymbolAddress(&ptr[1], g_phase_f64);
  if (e == cudaSuccess) e = cudaGetSymbolAddress(&ptr[2], g_phase_df);
  if (prev != device) cudaSetDevice(prev);
  if (e != cudaSuccess) return cuda_fail(e, "phase tables");
  g_phase_ptr[device] = ptr;
  return QS_OK;
}

const void* phase_table(int device, int format) {
  std::lock_guard<std::mutex> lock(g_phase_mu);
  auto it = g_phase_ptr.find(device);
  if (it == g_phase_ptr.end() || format < 0 || format > 2) return nullptr;
  return it->second[format];
}

}  // namespace qs
