"""Seeded synthetic inputs: states and circuits shaped like the paper's workloads.

This module is shared by the oracle side (tests, CPU baseline) and the GPU
side (tests, benchmark, serving).  It only *generates inputs* — gate lists
with their matrices, permutation tables and starting states — and holds none
of the simulation arithmetic: nothing here applies a gate to a state.

Random numbers come from ``numpy.random.Generator(PCG64(seed))``.

Gate record (``Gate``):
  kind    "u1"   2x2 matrix on targets[0]
          "uk"   dense 2^k x 2^k matrix on targets (row/col index
                 s = sum_j b_targets[j] 2^j, targets[0] least significant)
          "diag" 2^k diagonal entries indexed the same way
          "perm" uint32 table: sub-register value s -> perm[s]
  ctrls   qubits that must all be 1 for the gate to act (may be empty)
  data    complex128 matrix / diagonal, or uint32 table
  name    label only (the simulators look at ``kind`` and ``data``)
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

SQRT1_2 = 1.0 / math.sqrt(2.0)


@dataclass(frozen=True)
class Gate:
    kind: str
    targets: Tuple[int, ...]
    data: np.ndarray
    ctrls: Tuple[int, ...] = ()
    name: str = ""

    def qubits(self) -> Tuple[int, ...]:
        return tuple(self.targets) + tuple(self.ctrls)


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# --------------------------------------------------------------------------
# Fixed gate matrices (textbook definitions)
# --------------------------------------------------------------------------
def mat_h():
    return np.array([[SQRT1_2, SQRT1_2], [SQRT1_2, -SQRT1_2]], dtype=np.complex128)


def mat_x():
    return np.array([[0, 1], [1, 0]], dtype=np.complex128)


def mat_y():
    return np.array([[0, -1j], [1j, 0]], dtype=np.complex128)


def mat_z():
    return np.array([[1, 0], [0, -1]], dtype=np.complex128)


def mat_phase(phi: float):
    return np.array([[1, 0], [0, complex(math.cos(phi), math.sin(phi))]], dtype=np.complex128)


def mat_sqrt_pauli(P):
    """sqrt(P) = ((1+i)/2) I + ((1-i)/2) P for an involutory P."""
    return 0.5 * (1 + 1j) * np.eye(2, dtype=np.complex128) + 0.5 * (1 - 1j) * np.asarray(P, dtype=np.complex128)


def mat_w():
    return (mat_x() + mat_y()) * SQRT1_2


# --------------------------------------------------------------------------
# Gate constructors
# --------------------------------------------------------------------------
def g1(t, U, name="u1", ctrls=()):
    return Gate("u1", (int(t),), np.asarray(U, dtype=np.complex128).reshape(2, 2), tuple(int(c) for c in ctrls), name)


def gk(targets, M, name="uk", ctrls=()):
    k = len(targets)
    return Gate("uk", tuple(int(t) for t in targets), np.asarray(M, dtype=np.complex128).reshape(1 << k, 1 << k),
                tuple(int(c) for c in ctrls), name)


def gdiag(targets, d, name="diag", ctrls=()):
    return Gate("diag", tuple(int(t) for t in targets), np.asarray(d, dtype=np.complex128).reshape(-1),
                tuple(int(c) for c in ctrls), name)


def gperm(targets, perm, name="perm", ctrls=()):
    return Gate("perm", tuple(int(t) for t in targets), np.asarray(perm, dtype=np.uint32).reshape(-1),
                tuple(int(c) for c in ctrls), name)


def H(t):
    return g1(t, mat_h(), "h")


def X(t):
    return g1(t, mat_x(), "x")


def Y(t):
    return g1(t, mat_y(), "y")


def Z(t):
    return g1(t, mat_z(), "z")


def S(t):
    return g1(t, mat_phase(math.pi / 2), "s")


def T(t):
    return g1(t, mat_phase(math.pi / 4), "t")


def CNOT(c, t):
    return g1(t, mat_x(), "cnot", ctrls=(c,))


def CP(c, t, phi):
    """Controlled phase shift: diag(1, e^{i phi}) on t when c = 1."""
    return g1(t, mat_phase(phi), "cp", ctrls=(c,))


def CZ(a, b):
    return gdiag((a, b), [1, 1, 1, -1], "cz")


def SWAP(a, b):
    return gperm((a, b), [0, 2, 1, 3], "swap")


def MCZ(ctrls, t):
    return g1(t, mat_z(), "mcz", ctrls=tuple(ctrls))


def adjoint(g: Gate) -> Gate:
    """The inverse gate (conjugate transpose / inverse table)."""
    if g.kind in ("u1", "uk"):
        return Gate(g.kind, g.targets, np.conj(g.data.T).copy(), g.ctrls, g.name + "^")
    if g.kind == "diag":
        return Gate("diag", g.targets, np.conj(g.data).copy(), g.ctrls, g.name + "^")
    inv = np.empty_like(g.data)
    inv[g.data] = np.arange(g.data.size, dtype=np.uint32)
    return Gate("perm", g.targets, inv, g.ctrls, g.name + "^")


def inverse_circuit(gates: Sequence[Gate]) -> List[Gate]:
    return [adjoint(g) for g in reversed(gates)]


# --------------------------------------------------------------------------
# Random inputs
# --------------------------------------------------------------------------
def haar_unitary(dim: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-random U(dim): QR of a complex Ginibre matrix with the phases of
    R's diagonal moved into Q (Mezzadri 2007)."""
    z = (rng.standard_normal((dim, dim)) + 1j * rng.standard_normal((dim, dim))) * SQRT1_2
    q, r = np.linalg.qr(z)
    d = np.diagonal(r)
    return q * (d / np.abs(d))[None, :]


def random_state(n: int, rng, chunk: int = 1 << 24) -> np.ndarray:
    """i.i.d. complex Gaussian amplitudes (re, im ~ N(0,1)), normalised in
    double.  ``rng`` is a Generator (values drawn in order) or an int seed:
    then chunk j of ``chunk`` doubles is drawn from PCG64 seeded by
    SeedSequence(seed).spawn(...)[j], filled by parallel threads; the values
    do not depend on the thread count."""
    psi = np.empty(1 << n, dtype=np.complex128)
    f = psi.view(np.float64)
    if isinstance(rng, np.random.Generator):
        for lo in range(0, f.size, chunk):
            hi = min(f.size, lo + chunk)
            f[lo:hi] = rng.standard_normal(hi - lo)
    else:
        n_chunks = (f.size + chunk - 1) // chunk
        kids = np.random.SeedSequence(int(rng)).spawn(n_chunks)

        def fill(j):
            lo = j * chunk
            np.random.Generator(np.random.PCG64(kids[j])).standard_normal(out=f[lo:min(f.size, lo + chunk)])

        _parallel(fill, n_chunks)
    partial = np.zeros((f.size + chunk - 1) // chunk)

    def sq(j):
        seg = f[j * chunk:(j + 1) * chunk]
        partial[j] = float(np.dot(seg, seg))

    _parallel(sq, partial.size)
    scale = 1.0 / math.sqrt(float(np.sum(partial)))

    def norm(j):
        f[j * chunk:(j + 1) * chunk] *= scale

    _parallel(norm, partial.size)
    return psi


def _parallel(fn, count):
    if count <= 1:
        for j in range(count):
            fn(j)
        return
    import os
    from concurrent.futures import ThreadPoolExecutor

    with ThreadPoolExecutor(max_workers=min(count, os.cpu_count() or 1)) as ex:
        list(ex.map(fn, range(count)))


def random_distinct(rng, n, k):
    return [int(x) for x in rng.choice(n, size=k, replace=False)]


# --------------------------------------------------------------------------
# Workload circuits
# --------------------------------------------------------------------------
def random_circuit(n: int, n_gates: int, p_cnot: float, seed: int) -> List[Gate]:
    """Each gate: with probability p_cnot a CNOT on a random distinct
    (control, target), else a Haar-random 2x2 on a uniform target."""
    rng = rng_for(seed)
    gates = []
    for _ in range(n_gates):
        if rng.random() < p_cnot:
            c, t = random_distinct(rng, n, 2)
            gates.append(CNOT(c, t))
        else:
            gates.append(g1(int(rng.integers(n)), haar_unitary(2, rng), "haar1"))
    return gates


def gate_sweep(n: int, n_pairs: int, seed: int):
    """One Haar 2x2 on each target 0..n-1, then Haar 4x4 gates on random
    distinct (t0, t1) pairs.  Returns (one_qubit_gates, two_qubit_gates)."""
    rng = rng_for(seed)
    g1s = [g1(t, haar_unitary(2, rng), "haar1") for t in range(n)]
    g2s = []
    for _ in range(n_pairs):
        t0, t1 = random_distinct(rng, n, 2)
        g2s.append(gk((t0, t1), haar_unitary(4, rng), "haar2"))
    return g1s, g2s


def rqc(n: int, layers: int, seed: int) -> List[Gate]:
    """Random quantum circuit of ``layers`` cycles.  Each cycle: one of
    sqrt-X / sqrt-Y / sqrt-W on every qubit (uniform, never the qubit's
    previous choice), then CZ on a brick pattern: (2j, 2j+1) on even
    cycles, (2j+1, 2j+2) on odd cycles."""
    rng = rng_for(seed)
    mats = [mat_sqrt_pauli(mat_x()), mat_sqrt_pauli(mat_y()), mat_sqrt_pauli(mat_w())]
    names = ["sx", "sy", "sw"]
    prev = [-1] * n
    gates = []
    for layer in range(layers):
        for q in range(n):
            choices = [c for c in range(3) if c != prev[q]]
            c = choices[int(rng.integers(len(choices)))]
            prev[q] = c
            gates.append(g1(q, mats[c], names[c]))
        start = layer % 2
        for a in range(start, n - 1, 2):
            gates.append(CZ(a, a + 1))
    return gates


def rqc_ring(n: int, layers: int, seed: int) -> List[Gate]:
    """Random circuit as the paper describes it (Sec. III-C): per layer a
    random single-qubit gate on every qubit, then CNOT i -> (i+1) mod n for
    i = 0..n-1.  The single-qubit gates are Haar-random."""
    rng = rng_for(seed)
    gates = []
    for _ in range(layers):
        for q in range(n):
            gates.append(g1(q, haar_unitary(2, rng), "haar1"))
        for i in range(n):
            gates.append(CNOT(i, (i + 1) % n))
    return gates


def qft(qubits: Sequence[int]) -> List[Gate]:
    """QFT on the register ``qubits`` (qubits[j] holds bit j of the
    register value): from the most significant qubit down, a Hadamard
    followed by controlled phase shifts pi/2^(j-k) from every less
    significant qubit k, then the ending SWAPs that reverse the register."""
    m = len(qubits)
    gates = []
    for j in range(m - 1, -1, -1):
        gates.append(H(qubits[j]))
        for k in range(j - 1, -1, -1):
            gates.append(CP(qubits[k], qubits[j], math.pi / (1 << (j - k))))
    for q in range(m // 2):
        gates.append(SWAP(qubits[q], qubits[m - 1 - q]))
    return gates


def inverse_qft(qubits: Sequence[int]) -> List[Gate]:
    return inverse_circuit(qft(qubits))


def grover_iterations(n: int) -> int:
    theta = math.asin(2.0 ** (-n / 2.0))
    return int(math.floor(math.pi / (4.0 * theta)))


def grover(n: int, marked: int, iterations: int | None = None) -> List[Gate]:
    """Grover search for one marked index.  Oracle: phase flip of |marked>
    (X on the qubits where marked has a 0, multi-controlled Z, X again).
    Diffusion: H, X on all, multi-controlled Z, X, H on all.  Starts from
    |0...0> with H on every qubit."""
    r = grover_iterations(n) if iterations is None else iterations
    allq = list(range(n))
    zeros = [q for q in allq if not (marked >> q) & 1]
    gates = [H(q) for q in allq]
    for _ in range(r):
        gates += [X(q) for q in zeros]
        gates.append(MCZ(allq[:-1], allq[-1]))
        gates += [X(q) for q in zeros]
        gates += [H(q) for q in allq]
        gates += [X(q) for q in allq]
        gates.append(MCZ(allq[:-1], allq[-1]))
        gates += [X(q) for q in allq]
        gates += [H(q) for q in allq]
    return gates


def _is_composite(N: int) -> bool:
    return any(N % p == 0 for p in range(2, int(math.isqrt(N)) + 1))


def shor_params(n: int, rng: np.random.Generator):
    """Work register m = min(8, floor(n/2)) qubits (m >= 4), counting
    register t = n - m; N an odd composite in [max(9, 2^(m-1)), 2^m), a
    random base in (1, N) coprime with N."""
    m = max(4, min(8, n // 2))
    lo = max(9, 1 << (m - 1))
    cands = [N for N in range(lo, 1 << m) if N % 2 == 1 and _is_composite(N)]
    N = int(cands[int(rng.integers(len(cands)))])
    bases = [a for a in range(2, N) if math.gcd(a, N) == 1]
    a = int(bases[int(rng.integers(len(bases)))])
    return m, n - m, N, a


def mulmod_table(mult: int, N: int, m: int) -> np.ndarray:
    """Permutation of 0..2^m-1: x -> mult*x mod N for x < N, x for x >= N."""
    tab = np.arange(1 << m, dtype=np.uint32)
    tab[:N] = (np.arange(N, dtype=np.int64) * mult % N).astype(np.uint32)
    return tab


def shor_like(n: int, seed: int):
    """Order finding (periodicity estimation): counting register on qubits
    0..t-1 under H, work register on qubits t..n-1 starting at |1>, one
    controlled modular multiplication by a^(2^j) per counting qubit j, then
    the inverse QFT on the counting register.  Returns (gates, params)."""
    rng = rng_for(seed)
    m, t, N, a = shor_params(n, rng)
    work = list(range(t, n))
    gates = [X(work[0])]
    gates += [H(q) for q in range(t)]
    for j in range(t):
        gates.append(gperm(work, mulmod_table(pow(a, 1 << j, N), N, m), "cmulmod", ctrls=(j,)))
    gates += inverse_qft(list(range(t)))
    return gates, {"m": m, "t": t, "N": N, "a": a}


def multiplicative_order(a: int, N: int) -> int:
    r, x = 1, a % N
    while x != 1:
        x = x * a % N
        r += 1
    return r
