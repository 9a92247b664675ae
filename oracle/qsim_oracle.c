/*
 * Oracle: a plain, slow, obviously correct CPU state-vector simulator in
 * complex128 (IEEE double real and imaginary parts).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this code.  The GPU library never
 * links, calls or reads it, and it shares no code with the GPU library.
 *
 * Conventions (arXiv 2506.09198):
 *   - An n-qubit state is an array of 2^n complex amplitudes (Sec. I).
 *   - Each amplitude is stored as (re, im) side by side: array-of-structures
 *     (Sec. II-A, Fig. 1).
 *   - Qubit q is bit q of the amplitude index, qubit 0 the least significant
 *     bit.  A gate on target t pairs the amplitudes whose indices differ only
 *     in bit t: index "up" has bit t = 0, "lo" = up + 2^t (Algorithm 1).
 *   - A controlled gate acts only where every control bit is 1 (Fig. 4,
 *     Sec. III-A).
 * Readings of points where the paper is silent are stated at each function.
 *
 * Every loop below visits all 2^n indices and skips the ones a gate does not
 * start from; nothing is blocked, fused or reordered.  Arithmetic is plain
 * double with no FMA contraction (built with -ffp-contract=off).
 *
 * Two builds of this one file: the parity build (single thread, the loops
 * run in increasing index order) and a timing build with -fopenmp, where
 * the gate loops are split over threads.  Each index's update reads and
 * writes only its own pair / group, so both builds compute bit-identical
 * states.  The reductions (norm, marginals) stay sequential in both.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads of the gate loops in the timing build (no effect otherwise);
 * returns the count in use (1 in the parity build). */
int oracle_set_threads(int count) {
#ifdef _OPENMP
  if (count > 0) omp_set_num_threads(count);
  return omp_get_max_threads();
#else
  (void)count;
  return 1;
#endif
}

typedef struct {
  double re, im;
} amp_t;

static amp_t c_make(double re, double im) {
  amp_t r;
  r.re = re;
  r.im = im;
  return r;
}

static amp_t c_add(amp_t a, amp_t b) { return c_make(a.re + b.re, a.im + b.im); }

static amp_t c_mul(amp_t a, amp_t b) {
  return c_make(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}

/* Entry (r, c) of a row-major dim x dim complex matrix stored as (re, im). */
static amp_t mat_at(const double* m, int dim, int r, int c) {
  const double* p = m + 2 * (r * dim + c);
  return c_make(p[0], p[1]);
}

static int bit_of(uint64_t i, int q) { return (int)((i >> q) & 1u); }

/* 1 if every qubit in ctrl_mask is 1 in index i. */
static int controls_on(uint64_t i, uint64_t ctrl_mask) { return (i & ctrl_mask) == ctrl_mask; }

/* Sub-register value s = sum_j bit(i, targets[j]) * 2^j. */
static uint64_t sub_index(uint64_t i, const int* targets, int k) {
  uint64_t s = 0;
  for (int j = 0; j < k; ++j) s |= (uint64_t)bit_of(i, targets[j]) << j;
  return s;
}

/* Index i with its target bits replaced by the bits of s (bit j of s goes to
 * qubit targets[j]). */
static uint64_t with_sub(uint64_t i, const int* targets, int k, uint64_t s) {
  for (int j = 0; j < k; ++j) {
    uint64_t m = 1ull << targets[j];
    i = (i & ~m) | (((s >> j) & 1u) ? m : 0u);
  }
  return i;
}

/*
 * Single-qubit gate U (2x2, row-major, (re,im) interleaved) on target t,
 * acting only where all qubits of ctrl_mask are 1 (ctrl_mask = 0: plain gate).
 * For each pair (up, lo = up + 2^t):
 *   up' = u00 up + u01 lo,   lo' = u10 up + u11 lo.
 * Algorithm 1 gives this pairing and loop for the Hadamard (u = 1/sqrt 2
 * (1 1; 1 -1)); "applying gate matrices" (Sec. I) generalises it to any U.
 */
void oracle_apply_1q(amp_t* psi, int n, uint64_t ctrl_mask, int t, const double* U) {
  const uint64_t dim = 1ull << n;
  const uint64_t half = 1ull << t;
  const amp_t u00 = mat_at(U, 2, 0, 0), u01 = mat_at(U, 2, 0, 1);
  const amp_t u10 = mat_at(U, 2, 1, 0), u11 = mat_at(U, 2, 1, 1);
#pragma omp parallel for schedule(static)
  for (uint64_t up = 0; up < dim; ++up) {
    if (bit_of(up, t)) continue;
    if (!controls_on(up, ctrl_mask)) continue;
    const uint64_t lo = up + half;
    const amp_t a = psi[up], b = psi[lo];
    psi[up] = c_add(c_mul(u00, a), c_mul(u01, b));
    psi[lo] = c_add(c_mul(u10, a), c_mul(u11, b));
  }
}

/*
 * Dense k-qubit gate M (2^k x 2^k, row-major, (re,im) interleaved) on
 * targets[0..k-1], under ctrl_mask.  Reading (the paper names two-qubit gates,
 * Sec. III-A, but fixes no basis order): row and column index of M is
 * s = sum_j bit(targets[j]) 2^j, so targets[0] is the least significant.
 * For every index i whose target bits are all 0, gather v[s] = psi[i with
 * sub-register s], then write psi[i with sub-register r] = sum_s M[r][s] v[s].
 * With k = 2 this is the two-qubit update on the quad
 * (a, a+2^t0, a+2^t1, a+2^t0+2^t1).
 */
void oracle_apply_kq(amp_t* psi, int n, uint64_t ctrl_mask, const int* targets, int k, const double* M) {
  const uint64_t dim = 1ull << n;
  const int sub = 1 << k; /* k <= 8: at most 256 entries */
  uint64_t tmask = 0;
  for (int j = 0; j < k; ++j) tmask |= 1ull << targets[j];
#pragma omp parallel for schedule(static)
  for (uint64_t i = 0; i < dim; ++i) {
    amp_t v[256];
    if (i & tmask) continue;
    if (!controls_on(i, ctrl_mask)) continue;
    for (int s = 0; s < sub; ++s) v[s] = psi[with_sub(i, targets, k, (uint64_t)s)];
    for (int r = 0; r < sub; ++r) {
      amp_t acc = c_make(0.0, 0.0);
      for (int s = 0; s < sub; ++s) acc = c_add(acc, c_mul(mat_at(M, sub, r, s), v[s]));
      psi[with_sub(i, targets, k, (uint64_t)r)] = acc;
    }
  }
}

/*
 * Diagonal gate on targets[0..k-1]: psi[i] <- d[s(i)] psi[i], with
 * s(i) = sum_j bit(i, targets[j]) 2^j, applied only where ctrl_mask is on.
 * (Controlled phase shifts of the QFT, Sec. III-B, and a Grover oracle's
 * phase flip are diagonal gates.)
 */
void oracle_apply_diag(amp_t* psi, int n, uint64_t ctrl_mask, const int* targets, int k, const double* d) {
  const uint64_t dim = 1ull << n;
#pragma omp parallel for schedule(static)
  for (uint64_t i = 0; i < dim; ++i) {
    if (!controls_on(i, ctrl_mask)) continue;
    const uint64_t s = sub_index(i, targets, k);
    psi[i] = c_mul(c_make(d[2 * s], d[2 * s + 1]), psi[i]);
  }
}

/*
 * Permutation gate on targets[0..k-1]: the basis state whose sub-register is
 * s moves to sub-register perm[s] (|s> -> |perm(s)>), where ctrl_mask is on.
 * (Controlled modular multiplication of the Shor-like workload, Sec. III-D.)
 * Computed out of place: out[i with sub perm[s]] = in[i with sub s].
 */
void oracle_apply_perm(amp_t* psi, int n, uint64_t ctrl_mask, const int* targets, int k, const uint32_t* perm) {
  const uint64_t dim = 1ull << n;
  amp_t* src = (amp_t*)malloc(sizeof(amp_t) * (size_t)dim);
  if (!src) return;
  memcpy(src, psi, sizeof(amp_t) * (size_t)dim);
#pragma omp parallel for schedule(static)
  for (uint64_t i = 0; i < dim; ++i) {
    if (!controls_on(i, ctrl_mask)) continue;
    const uint64_t s = sub_index(i, targets, k);
    psi[with_sub(i, targets, k, perm[s])] = src[i];
  }
  free(src);
}

/* Kahan-compensated sum of |psi_i|^2 over all i. */
double oracle_norm2(const amp_t* psi, int n) {
  const uint64_t dim = 1ull << n;
  double sum = 0.0, comp = 0.0;
  for (uint64_t i = 0; i < dim; ++i) {
    const double term = psi[i].re * psi[i].re + psi[i].im * psi[i].im;
    const double y = term - comp;
    const double t = sum + y;
    comp = (t - sum) - y;
    sum = t;
  }
  return sum;
}

/* out[s] = sum over i with sub-register s (on qubits[0..k-1]) of |psi_i|^2,
 * each a Kahan-compensated sum. */
void oracle_probs(const amp_t* psi, int n, const int* qubits, int k, double* out) {
  const uint64_t dim = 1ull << n;
  const int sub = 1 << k;
  double* comp = (double*)calloc((size_t)sub, sizeof(double));
  if (!comp) return;
  for (int s = 0; s < sub; ++s) out[s] = 0.0;
  for (uint64_t i = 0; i < dim; ++i) {
    const uint64_t s = sub_index(i, qubits, k);
    const double term = psi[i].re * psi[i].re + psi[i].im * psi[i].im;
    const double y = term - comp[s];
    const double t = out[s] + y;
    comp[s] = (t - out[s]) - y;
    out[s] = t;
  }
  free(comp);
}
