// Device arithmetic policies for the gate kernels.
//
// Three ways to compute one gate update  out = sum_k m_k * v_k  (complex):
//   MathF32  complex64 state (float2), FP32 FMA arithmetic.
//   MathF64  complex128 state (double2), plain IEEE double arithmetic.
//   MathDF   complex128 state (double2), float-float arithmetic on the FP32
//            pipes: each double is split into head + tail floats, products are
//            formed exactly (TwoProduct via FMA, Dekker 1971) and summed with
//            TwoSum (Knuth, TAOCP vol. 2) error terms; the result is rounded
//            to double by one FP64 add of two exactly converted floats.
// GB300 runs FP64 at about 1/70 of the FP32 rate, so MathDF is the default
// for complex128: about 48 significant bits per product and sum, rounded to
// IEEE double after every gate.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace qs {

// ---------------------------------------------------------------------------
// Exact float <-> double conversions with integer instructions only (the
// F2F conversions run on the slow FP64 pipe of this GPU).
// ---------------------------------------------------------------------------

// Float to double, exact for normal floats; zero and subnormal floats
// (|f| < 2^-126) become a signed zero.
__device__ __forceinline__ double f2d_exact(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t sign = b & 0x80000000u;
  const uint32_t mag = b & 0x7FFFFFFFu;
  uint32_t hi = sign | ((mag >> 3) + (896u << 20));  // rebias 127 -> 1023
  uint32_t lo = mag << 29;
  if (mag < 0x00800000u) {
    hi = sign;
    lo = 0u;
  }
  return __hiloint2double((int)hi, (int)lo);
}

// Double to head + tail floats: head = the leading 24 significant bits
// (truncated), tail = the remaining 29 bits rounded to 24.  |x - h - l| <=
// 2^-48 |x|.  |x| < 2^-74 gives h = l = 0; |x| must be below 2^127.
__device__ __forceinline__ void d2ff(double x, float& h, float& l) {
  const uint32_t lo32 = (uint32_t)__double2loint(x);
  const uint32_t hi32 = (uint32_t)__double2hiint(x);
  // (hi32 << 3) | (lo32 >> 29): exponent bits 7..0 land at 30..23 and the 23
  // leading mantissa bits at 22..0.  Rebias 1023 -> 127 is a flip of bit 30
  // (896 = 3*256 + 128); bit 31 is replaced by the sign.
  const uint32_t fs = __funnelshift_l(lo32, hi32, 3) ^ 0x40000000u;
  uint32_t hb = (fs & 0x7FFFFFFFu) | (hi32 & 0x80000000u);
  // tail = sign * (lo32 & (2^29-1)) * 2^(E-1075); its scale is 2^-52 of the
  // head's exponent, built by lowering the head's exponent field by 52.
  const uint32_t scale_bits = (hb & 0xFF800000u) - (52u << 23);
  float tl = __uint2float_rn(lo32 & 0x1FFFFFFFu) * __uint_as_float(scale_bits);
  const uint32_t e = (hi32 >> 20) & 0x7FFu;
  if (e < 949u) {  // |x| < 2^-74: flush
    hb = 0u;
    tl = 0.0f;
  }
  h = __uint_as_float(hb);
  l = tl;
}

// ---------------------------------------------------------------------------
// Policies.  Each provides:
//   Amp       storage type of one amplitude
//   Val       working value of one amplitude
//   Coef      one complex matrix entry in working form
//   make_coef(re, im)   host-side conversion of a double matrix entry
//   load(Amp) -> Val
//   mac_round<K>(coefs, vals) -> Amp   sum_k coefs[k] * vals[k], rounded to
//                                      the storage type
// ---------------------------------------------------------------------------
struct MathF64 {
  using Amp = double2;
  struct Val { double re, im; };
  struct Coef { double re, im; };
  static __host__ Coef make_coef(double re, double im) { return Coef{re, im}; }
  static __device__ __forceinline__ Val load(const Amp& a) { return Val{a.x, a.y}; }
  static __device__ __forceinline__ Amp pack(const Val& v) { return make_double2(v.re, v.im); }
  template <int K>
  static __device__ __forceinline__ Val mac(const Coef* m, const Val* v) {
    double re = 0.0, im = 0.0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      re = __fma_rn(m[k].re, v[k].re, re);
      re = __fma_rn(-m[k].im, v[k].im, re);
      im = __fma_rn(m[k].re, v[k].im, im);
      im = __fma_rn(m[k].im, v[k].re, im);
    }
    return Val{re, im};
  }
  template <int K>
  static __device__ __forceinline__ Amp mac_round(const Coef* m, const Val* v) { return pack(mac<K>(m, v)); }
};

// ---------------------------------------------------------------------------
// Packed FP32x2 arithmetic (sm_100+): one instruction computes two lanes, so
// the real and imaginary channels of a complex dot product share each issue.
// ---------------------------------------------------------------------------
// Operands are packed into register pairs with mov.b64 {lo, hi}, which the
// assembler resolves to the pair itself (no data movement).
#define QS_F32X2_BINARY(name, op)                                                             \
  __device__ __forceinline__ float2 name(float2 a, float2 b) {                               \
    float2 d;                                                                                 \
    asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"     \
        " " op " rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"                                     \
        : "=f"(d.x), "=f"(d.y)                                                                \
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));                                            \
    return d;                                                                                 \
  }
QS_F32X2_BINARY(add2, "add.rn.f32x2")
QS_F32X2_BINARY(sub2, "sub.rn.f32x2")
QS_F32X2_BINARY(mul2, "mul.rn.f32x2")
#undef QS_F32X2_BINARY

__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n .reg .b64 ra, rb, rc, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
      " mov.b64 rc, {%6, %7};\n fma.rn.f32x2 rd, ra, rb, rc;\n mov.b64 {%0, %1}, rd;\n}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}

// Float-float complex dot product on (re, im) channel pairs.
//   A term multiplies (vr, vi) by (mr, mr); a B term multiplies the swapped
//   value (vi, vr) by (-mi, mi): re += mr vr - mi vi, im += mr vi + mi vr.
// Each vector term: exact product head (mul) and tail (fma against the
// negated head), TwoSum of the head into S, every lower-order part into C.
// A coefficient is carried as three floats, h + l + ll, which equal the
// double exactly (24 + 24 + 24 significant bits >= 53).  With two floats a
// coefficient keeps only ~48 bits, and that truncation is the same in every
// application of the gate: over thousands of gates (Grover's Hadamards) it
// adds up coherently, to several times 1e-12 against FP64.  The third part
// costs one fma per term (ll xh; ll xl and l xl are below 2^-96 |m x|, the
// dropped l xl below 2^-48 and of either sign).
struct DF2Term {
  float2 h, hn, l, ll;  // coefficient head, negated head, tail, second tail (per channel)
};

struct DF2Acc {
  float2 S, C;
  // LL: include the coefficient's second tail (exact double coefficients).
  template <bool LL = true>
  __device__ __forceinline__ void first(const DF2Term& a, float2 xh, float2 xl) {
    S = mul2(a.h, xh);
    const float2 ne = fma2(a.hn, xh, S);  // S - a.h xh = -(product tail), exact
    C = sub2(fma2(a.l, xh, mul2(a.h, xl)), ne);
    if (LL) C = fma2(a.ll, xh, C);
  }
  template <bool LL = true>
  __device__ __forceinline__ void add(const DF2Term& a, float2 xh, float2 xl) {
    const float2 pn = mul2(a.hn, xh);     // -p
    const float2 e = fma2(a.h, xh, pn);   // a.h xh - p, exact
    const float2 s = sub2(S, pn);         // TwoSum(S, p)
    const float2 bb = sub2(s, S);
    const float2 t2 = sub2(S, sub2(s, bb));
    const float2 err = sub2(t2, add2(pn, bb));  // (S - (s - bb)) + (p - bb)
    C = add2(C, add2(err, e));
    C = fma2(a.h, xl, C);
    C = fma2(a.l, xh, C);
    if (LL) C = fma2(a.ll, xh, C);
    S = s;
  }
};

// complex64 with packed FP32x2 multiply-adds: (re, im) += (mr, mr)(vr, vi)
// + (-mi, mi)(vi, vr), two instructions per complex multiply-add.
struct MathF32 {
  using Amp = float2;
  struct Val {
    float2 v, vs;  // (re, im) and (im, re)
  };
  struct alignas(16) Coef {  // 16-byte aligned: one vector load from a staged pool
    float2 a, b;   // (mr, mr) and (-mi, mi)
  };
  static __host__ Coef make_coef(double re, double im) {
    const float r = (float)re, i = (float)im;
    return Coef{make_float2(r, r), make_float2(-i, i)};
  }
  static __device__ __forceinline__ Val load(const Amp& a) { return Val{a, make_float2(a.y, a.x)}; }
  template <int K>
  static __device__ __forceinline__ Amp mac_round(const Coef* m, const Val* v) {
    float2 acc = mul2(m[0].a, v[0].v);
    acc = fma2(m[0].b, v[0].vs, acc);
#pragma unroll
    for (int k = 1; k < K; ++k) {
      acc = fma2(m[k].a, v[k].v, acc);
      acc = fma2(m[k].b, v[k].vs, acc);
    }
    return acc;
  }
};


// Anchored float-float dot product.  The heads are summed into S starting
// from a power-of-two anchor A >= 2 * (bound on |sum of heads|), so every
// addition S + p has |S| >= |p| and its rounding error is exactly
// p - (S' - S) (Fast2Sum, Dekker 1971: 3 operations instead of TwoSum's 6);
// S - A is exact at the end (Sterbenz: S lies within [A/2, 2A]).  The bound
// is sum_k |a_k| * max_k |x_k|: the row sum comes from the host as a power
// of two exponent, the input maximum from the amplitudes.
// With p = fl(a.h xh), s = fl(S + p) and d = S - s (exact: Fast2Sum), the two
// exact error terms (a.h xh - p) + (p - (s - S)) equal a.h xh + d, so one fma
// yields their sum rounded once: 7 packed operations per term.
struct DF2AnchorAcc {
  float2 S, C;
  template <bool LL = true>
  __device__ __forceinline__ void add(const DF2Term& a, float2 xh, float2 xl) {
    const float2 p = mul2(a.h, xh);
    const float2 s = add2(S, p);
    const float2 t = fma2(a.h, xh, sub2(S, s));  // product tail + addition error
    C = add2(C, t);
    C = fma2(a.h, xl, C);
    C = fma2(a.l, xh, C);
    if (LL) C = fma2(a.ll, xh, C);
    S = s;
  }
};

// 2^(e - 127) as a float for an exponent field e clamped to [1, 254].
__device__ __forceinline__ float pow2_field(int e) {
  e = e < 1 ? 1 : (e > 254 ? 254 : e);
  return __uint_as_float((uint32_t)e << 23);
}

template <bool LL>
struct MathDFT {
  using Amp = double2;
  struct Val {
    float2 h, l;    // (re, im) heads and tails
    float2 hs, ls;  // the same, channels swapped (im, re)
  };
  struct Coef {
    DF2Term a, b;   // A term (mr, mr) and B term (-mi, mi)
  };
  // h = fl(x), l = fl(x - h), ll = fl(x - h - l): each difference is exact
  // in double, and ll holds the last <= 5 bits exactly, so h + l + ll == x.
  static __host__ Coef make_coef(double re, double im) {
    const float rh = (float)re, ih = (float)im;
    const float rl = (float)(re - (double)rh), il = (float)(im - (double)ih);
    const float rll = (float)((re - (double)rh) - (double)rl), ill = (float)((im - (double)ih) - (double)il);
    Coef c;
    c.a.h = make_float2(rh, rh);
    c.a.hn = make_float2(-rh, -rh);
    c.a.l = make_float2(rl, rl);
    c.a.ll = make_float2(rll, rll);
    c.b.h = make_float2(-ih, ih);
    c.b.hn = make_float2(ih, -ih);
    c.b.l = make_float2(-il, il);
    c.b.ll = make_float2(-ill, ill);
    return c;
  }
  static __device__ __forceinline__ Val load(const Amp& a) {
    Val v;
    d2ff(a.x, v.h.x, v.l.x);
    d2ff(a.y, v.h.y, v.l.y);
    v.hs = make_float2(v.h.y, v.h.x);
    v.ls = make_float2(v.l.y, v.l.x);
    return v;
  }
  template <int K>
  static __device__ __forceinline__ DF2Acc mac(const Coef* m, const Val* v) {
    DF2Acc acc;
    acc.template first<LL>(m[0].a, v[0].h, v[0].l);
    acc.template add<LL>(m[0].b, v[0].hs, v[0].ls);
#pragma unroll
    for (int k = 1; k < K; ++k) {
      acc.template add<LL>(m[k].a, v[k].h, v[k].l);
      acc.template add<LL>(m[k].b, v[k].hs, v[k].ls);
    }
    return acc;
  }
  // Exponent field of the largest |head| among K input amplitudes.
  template <int K>
  static __device__ __forceinline__ int max_exp_field(const Val* v) {
    float mx = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) mx = fmaxf(mx, fmaxf(fabsf(v[k].h.x), fabsf(v[k].h.y)));
    return (int)(__float_as_uint(mx) >> 23);
  }
  // sum_k m[k] v[k] with the anchored accumulation; row_exp: the row's
  // sum_k (|re m_k| + |im m_k|) < 2^row_exp; mexp: max_exp_field of v.
  template <int K>
  static __device__ __forceinline__ Amp mac_anchor_round(const Coef* m, const Val* v, int row_exp, int mexp) {
    const DF2Acc r = mac_anchor<K>(m, v, row_exp, mexp);
    return make_double2(f2d_exact(r.S.x) + f2d_exact(r.C.x), f2d_exact(r.S.y) + f2d_exact(r.C.y));
  }
  // Anchored accumulation returning (exact head sum, lower-order sum).
  template <int K>
  static __device__ __forceinline__ DF2Acc mac_anchor(const Coef* m, const Val* v, int row_exp, int mexp) {
    const float A = pow2_field(mexp + row_exp + 2);
    DF2AnchorAcc acc;
    acc.S = make_float2(A, A);
    acc.C = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      acc.template add<LL>(m[k].a, v[k].h, v[k].l);
      acc.template add<LL>(m[k].b, v[k].hs, v[k].ls);
    }
    DF2Acc r;
    r.S = sub2(acc.S, make_float2(A, A));
    r.C = acc.C;
    return r;
  }
  template <int K>
  static __device__ __forceinline__ Amp mac_round(const Coef* m, const Val* v) {
    const DF2Acc acc = mac<K>(m, v);
    return make_double2(f2d_exact(acc.S.x) + f2d_exact(acc.C.x), f2d_exact(acc.S.y) + f2d_exact(acc.C.y));
  }
};

// Fused and batched tiles keep the state in float-float form across many
// gates: exact double coefficients (three floats).
using MathDF = MathDFT<true>;
// Per-gate kernels round every result to IEEE double; they leave out the
// second coefficient tail (at most 2^-49 of a coefficient, below their own
// float-float rounding), which keeps them at the memory bound.
using MathDFGate = MathDFT<false>;

}  // namespace qs
