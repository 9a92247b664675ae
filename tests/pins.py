"""Pins for the oracle: checks against facts fixed independently of its code.

Each ``pin_*`` function raises AssertionError when the oracle disagrees with
  - brute force: a dense 2^n x 2^n operator assembled from Kronecker products
    of one-qubit pieces (qubit 0 = rightmost factor) and projector sums for
    controls, multiplied into the state with numpy;
  - a tensor-network contraction (numpy.tensordot on a (2,)*n tensor);
  - textbook matrices on one and two qubits;
  - closed forms: H^n|0> = 2^(-n/2) everywhere; the QFT of |x> has
    amplitude 2^(-n/2) exp(2 pi i x y / 2^n); Grover's success probability
    sin^2((2r+1) theta), theta = asin(2^(-n/2)); the Shor-like counting
    distribution from the textbook state sum_x |x>|a^x mod N>;
  - invariants: norm preservation, a circuit followed by its inverse,
    exact index permutation for X, CNOT, SWAP and permutation gates.
The functions take the oracle module as an argument so that the mutation
test can run them against deliberately broken oracle builds.
"""
from __future__ import annotations

import math

import numpy as np

import workloads as W

# ---------------------------------------------------------------------------
# Independent brute force
# ---------------------------------------------------------------------------
_KET = [np.array([1, 0], dtype=np.complex128), np.array([0, 1], dtype=np.complex128)]


def _outer(r, c):
    return np.outer(_KET[r], _KET[c])


def local_operator(n, pieces):
    """Kronecker product over qubits n-1 .. 0 (qubit 0 rightmost) of the
    2x2 pieces given in ``pieces`` (dict qubit -> 2x2), identity elsewhere."""
    op = np.array([[1.0 + 0j]])
    for q in range(n - 1, -1, -1):
        op = np.kron(op, pieces.get(q, np.eye(2, dtype=np.complex128)))
    return op


def gate_matrix_on_targets(g):
    k = len(g.targets)
    if g.kind in ("u1", "uk"):
        return np.asarray(g.data, dtype=np.complex128).reshape(1 << k, 1 << k)
    if g.kind == "diag":
        return np.diag(np.asarray(g.data, dtype=np.complex128))
    if g.kind == "perm":
        M = np.zeros((1 << k, 1 << k), dtype=np.complex128)
        for s, ps in enumerate(g.data):
            M[int(ps), s] = 1.0
        return M
    raise ValueError(g.kind)


def full_operator(g, n):
    """Dense 2^n x 2^n operator of gate g (controls as a projector sum)."""
    M = gate_matrix_on_targets(g)
    k = len(g.targets)
    op_t = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    for r in range(1 << k):
        for c in range(1 << k):
            if M[r, c] == 0:
                continue
            pieces = {g.targets[j]: _outer((r >> j) & 1, (c >> j) & 1) for j in range(k)}
            op_t += M[r, c] * local_operator(n, pieces)
    if not g.ctrls:
        return op_t
    P = local_operator(n, {c: _outer(1, 1) for c in g.ctrls})
    eye = np.eye(1 << n, dtype=np.complex128)
    return eye + P @ (op_t - eye)


def brute_force_run(psi, gates, n):
    out = np.array(psi, dtype=np.complex128)
    for g in gates:
        out = full_operator(g, n) @ out
    return out


def tensordot_apply(psi, g, n):
    """Apply gate g by contracting its (2,)*2k tensor with the state tensor.
    Axis a of the state tensor is qubit n-1-a."""
    k = len(g.targets)
    M = gate_matrix_on_targets(g)
    # gate tensor indices: outputs (b_{k-1} .. b_0), inputs (b_{k-1} .. b_0)
    Mt = M.reshape((2,) * (2 * k))
    st = np.asarray(psi, dtype=np.complex128).reshape((2,) * n)
    axes_in = [n - 1 - g.targets[j] for j in range(k - 1, -1, -1)]
    if g.ctrls:
        # Split on the control axes: act only on the slice where all are 1.
        idx = [slice(None)] * n
        for c in g.ctrls:
            idx[n - 1 - c] = 1
        sub = st[tuple(idx)]
        # remaining axes keep relative order; remap target axes
        kept = [a for a in range(n) if (n - 1 - a) not in g.ctrls]
        sub_axes = [kept.index(a) for a in axes_in]
        moved = np.tensordot(Mt, sub, axes=(list(range(k, 2 * k)), sub_axes))
        moved = np.moveaxis(moved, list(range(k)), sub_axes)
        st = st.copy()
        st[tuple(idx)] = moved
        return st.reshape(-1)
    moved = np.tensordot(Mt, st, axes=(list(range(k, 2 * k)), axes_in))
    moved = np.moveaxis(moved, list(range(k)), axes_in)
    return moved.reshape(-1)


# ---------------------------------------------------------------------------
# Random gate mix covering every kind, with and without controls
# ---------------------------------------------------------------------------
def random_mixed_circuit(n, n_gates, seed, max_k=3):
    rng = W.rng_for(seed)
    gates = []
    for _ in range(n_gates):
        kind = ["u1", "uk", "diag", "perm"][int(rng.integers(4))]
        kmax = min(max_k, n)
        k = 1 if kind == "u1" else int(rng.integers(1, kmax + 1))
        if kind == "uk" and k < 2 and n >= 2:
            k = 2
        nc = int(rng.integers(0, min(2, n - k) + 1))
        qs = W.random_distinct(rng, n, k + nc)
        tg, cs = qs[:k], qs[k:]
        if kind == "u1":
            gates.append(W.g1(tg[0], W.haar_unitary(2, rng), ctrls=cs))
        elif kind == "uk":
            gates.append(W.gk(tg, W.haar_unitary(1 << k, rng), ctrls=cs))
        elif kind == "diag":
            ph = rng.uniform(0, 2 * math.pi, size=1 << k)
            gates.append(W.gdiag(tg, np.exp(1j * ph), ctrls=cs))
        else:
            gates.append(W.gperm(tg, rng.permutation(1 << k).astype(np.uint32), ctrls=cs))
    return gates


def _maxerr(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))))


# ---------------------------------------------------------------------------
# Pins
# ---------------------------------------------------------------------------
def pin_textbook_1q(O):
    """n = 1: psi' = U psi for H, X, Y, Z, S, T and a Haar U."""
    rng = W.rng_for(11)
    psi0 = rng.standard_normal(2) + 1j * rng.standard_normal(2)
    for U in (W.mat_h(), W.mat_x(), W.mat_y(), W.mat_z(), W.mat_phase(math.pi / 2),
              W.mat_phase(math.pi / 4), W.haar_unitary(2, rng)):
        got = O.apply_1q(psi0.copy(), 0, U)
        assert _maxerr(got, U @ psi0) < 1e-15, "1-qubit gate differs from U psi"
    # H|0> = (|0> + |1>)/sqrt2, H|1> = (|0> - |1>)/sqrt2 (Algorithm 1 formula)
    r2 = 1 / math.sqrt(2)
    assert _maxerr(O.apply_1q(O.basis_state(1, 0), 0, W.mat_h()), [r2, r2]) < 1e-16
    assert _maxerr(O.apply_1q(O.basis_state(1, 1), 0, W.mat_h()), [r2, -r2]) < 1e-16


def pin_textbook_2q(O):
    """n = 2, basis index i = b0 + 2 b1: U (x) I, I (x) U, CNOT, CZ, SWAP, 4x4."""
    rng = W.rng_for(12)
    psi0 = rng.standard_normal(4) + 1j * rng.standard_normal(4)
    U = W.haar_unitary(2, rng)
    I2 = np.eye(2)
    # Gate on qubit 0 acts on the rightmost Kronecker factor.
    assert _maxerr(O.apply_1q(psi0.copy(), 0, U), np.kron(I2, U) @ psi0) < 1e-15
    assert _maxerr(O.apply_1q(psi0.copy(), 1, U), np.kron(U, I2) @ psi0) < 1e-15
    # CNOT control 0 -> target 1 swaps |01> (i=1) and |11> (i=3).
    cnot01 = np.array([[1, 0, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0], [0, 1, 0, 0]], dtype=np.complex128)
    assert _maxerr(O.apply_1q(psi0.copy(), 1, W.mat_x(), ctrls=(0,)), cnot01 @ psi0) == 0.0
    # CNOT control 1 -> target 0 swaps i=2 and i=3.
    cnot10 = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=np.complex128)
    assert _maxerr(O.apply_1q(psi0.copy(), 0, W.mat_x(), ctrls=(1,)), cnot10 @ psi0) == 0.0
    swap = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=np.complex128)
    assert _maxerr(O.apply_perm(psi0.copy(), [0, 1], [0, 2, 1, 3]), swap @ psi0) == 0.0
    cz = np.diag([1, 1, 1, -1]).astype(np.complex128)
    assert _maxerr(O.apply_diag(psi0.copy(), [0, 1], [1, 1, 1, -1]), cz @ psi0) == 0.0
    # Dense 4x4 on (t0, t1) = (0, 1): matrix index b_t0 + 2 b_t1 = basis index.
    U4 = W.haar_unitary(4, rng)
    assert _maxerr(O.apply_2q(psi0.copy(), 0, 1, U4), U4 @ psi0) < 1e-15
    # (t0, t1) = (1, 0): matrix index b1 + 2 b0, i.e. the basis with qubits swapped.
    P = swap.real
    assert _maxerr(O.apply_2q(psi0.copy(), 1, 0, U4), P @ U4 @ P @ psi0) < 1e-15


def pin_bruteforce(O, ns=(1, 2, 3, 4, 5, 6, 7, 8), n_gates=24, seed=100):
    """Every gate kind with 0-2 controls against the dense-operator brute force."""
    for n in ns:
        gates = random_mixed_circuit(n, n_gates, seed + n)
        rng = W.rng_for(seed + 1000 + n)
        psi0 = W.random_state(n, rng)
        ref = brute_force_run(psi0, gates, n)
        got = O.run_circuit(psi0.copy(), gates)
        assert _maxerr(got, ref) < 1e-13, f"n={n}: oracle vs dense operators"


def pin_tensordot(O, n=12, n_gates=40, seed=200):
    """Larger n: each gate checked against a tensordot contraction."""
    gates = random_mixed_circuit(n, n_gates, seed, max_k=3)
    psi = W.random_state(n, W.rng_for(seed + 1))
    for g in gates:
        ref = tensordot_apply(psi, g, n)
        got = O.apply_gate(psi.copy(), g)
        assert _maxerr(got, ref) < 1e-14, f"gate {g.kind} t={g.targets} c={g.ctrls}"
        psi = ref


def pin_dense_wide(O, seed=250):
    """Dense gates on 4 and 5 targets (unsorted, 0-2 controls): against the
    tensordot contraction, and a Kronecker product U_{k-1} (x) ... (x) U_0
    (target j is bit j of the matrix index, the rightmost factor for j = 0)
    against the k single-qubit gates applied one by one."""
    rng = W.rng_for(seed)
    for k in (4, 5):
        for n in (k, k + 2, 9):
            for nc in range(0, min(2, n - k) + 1):
                qs = W.random_distinct(rng, n, k + nc)
                tg, cs = qs[:k], qs[k:]
                psi = W.random_state(n, rng)
                g = W.gk(tg, W.haar_unitary(1 << k, rng), ctrls=cs)
                ref = tensordot_apply(psi, g, n)
                got = O.apply_kq(psi.copy(), tg, g.data, ctrls=cs)
                assert _maxerr(got, ref) < 1e-14, f"k={k} n={n} t={tg} c={cs}"
            facs = [W.haar_unitary(2, rng) for _ in range(k)]
            U = facs[k - 1]
            for j in range(k - 2, -1, -1):
                U = np.kron(U, facs[j])
            tg = W.random_distinct(rng, n, k)
            psi = W.random_state(n, rng)
            want = psi.copy()
            for j in range(k):
                O.apply_1q(want, tg[j], facs[j])
            got = O.apply_kq(psi.copy(), tg, U)
            assert _maxerr(got, want) < 1e-14, f"k={k} n={n}: Kronecker product vs one-qubit gates"


def pin_hadamard_uniform(O, ns=range(1, 15)):
    for n in ns:
        psi = O.run_circuit(O.basis_state(n), [W.H(q) for q in range(n)])
        assert _maxerr(psi, np.full(1 << n, 2.0 ** (-n / 2))) < 1e-15 * n


def qft_closed_form(n, x, ys=None):
    """Amplitudes 2^(-n/2) exp(2 pi i x y / 2^n), phase reduced as the
    integer x*y mod 2^n before scaling."""
    ys = np.arange(1 << n, dtype=np.int64) if ys is None else np.asarray(ys, dtype=np.int64)
    ph = ((int(x) * ys) % (1 << n)).astype(np.float64) * (2 * math.pi / (1 << n))
    return np.exp(1j * ph) * 2.0 ** (-n / 2)


def pin_qft_basis(O, ns=range(1, 12), seed=300):
    rng = W.rng_for(seed)
    for n in ns:
        for x in {0, (1 << n) - 1, int(rng.integers(1 << n))}:
            psi = O.run_circuit(O.basis_state(n, x), W.qft(list(range(n))))
            assert _maxerr(psi, qft_closed_form(n, x)) < 1e-13, f"QFT n={n} x={x}"
            back = O.run_circuit(psi, W.inverse_qft(list(range(n))))
            assert _maxerr(back, O.basis_state(n, x)) < 1e-13


def grover_closed_form(n, marked, r):
    """State after r iterations of the Grover circuit from |0...0>.

    With theta = asin(2^(-n/2)), each textbook iteration rotates by 2 theta in
    the plane of |marked> and the uniform superposition of the other indices,
    so G^r H^n |0> = sin((2r+1) theta) |marked> + cos((2r+1) theta) |rest>,
    |rest> the normalised sum of the other 2^n - 1 basis states.  The circuit
    realises the diffusion as H X MCZ X H = I - 2|s><s|, the negative of the
    textbook 2|s><s| - I, so each iteration also contributes a factor -1."""
    theta = math.asin(2.0 ** (-n / 2))
    sign = -1.0 if r % 2 else 1.0
    psi = np.full(1 << n, sign * math.cos((2 * r + 1) * theta) / math.sqrt((1 << n) - 1), dtype=np.complex128)
    psi[marked] = sign * math.sin((2 * r + 1) * theta)
    return psi


def pin_grover(O, ns=range(2, 13), seed=400):
    rng = W.rng_for(seed)
    for n in ns:
        marked = int(rng.integers(1 << n))
        theta = math.asin(2.0 ** (-n / 2))
        for r in sorted({0, 1, 2, 3, W.grover_iterations(n)}):
            psi = O.run_circuit(O.basis_state(n), W.grover(n, marked, r))
            p = np.abs(psi) ** 2
            assert abs(p[marked] - math.sin((2 * r + 1) * theta) ** 2) < 1e-12, f"Grover n={n} r={r}"
            others = np.delete(psi, marked)
            assert _maxerr(others, np.full(others.size, others[0])) < 1e-12
            # every amplitude, signs included
            assert _maxerr(psi, grover_closed_form(n, marked, r)) < 1e-12, f"Grover state n={n} r={r}"


def shor_counting_distribution(t, a, N):
    """P(y) = sum_s |2^(-t) sum_{x = s mod r, x < 2^t} exp(-2 pi i x y / 2^t)|^2."""
    r = W.multiplicative_order(a, N)
    T = 1 << t
    y = np.arange(T, dtype=np.int64)
    P = np.zeros(T)
    for s in range(r):
        xs = np.arange(s, T, r, dtype=np.int64)
        ph = -2 * math.pi * ((np.outer(y, xs) % T).astype(np.float64)) / T
        P += np.abs(np.exp(1j * ph).sum(axis=1) / T) ** 2
    return P


def pin_shor_like(O, ns=(8, 9, 10, 11, 12), seed=500):
    for n in ns:
        gates, prm = W.shor_like(n, seed + n)
        psi = O.run_circuit(O.basis_state(n), gates)
        got = O.probs(psi, list(range(prm["t"])))
        want = shor_counting_distribution(prm["t"], prm["a"], prm["N"])
        assert _maxerr(got, want) < 1e-12, f"Shor-like n={n} N={prm['N']} a={prm['a']}"


def pin_norm_and_inverse(O, seed=600):
    for n in (3, 6, 9, 12):
        gates = random_mixed_circuit(n, 60, seed + n)
        psi0 = W.random_state(n, W.rng_for(seed + 50 + n))
        psi = O.run_circuit(psi0.copy(), gates)
        assert abs(O.norm2(psi) - 1.0) < 1e-13
        back = O.run_circuit(psi, W.inverse_circuit(gates))
        assert _maxerr(back, psi0) < 1e-12


def pin_moves_exact(O, n=9, seed=700):
    """X, Y, CNOT, SWAP, perm: the result is the input with indices moved
    (and, for Y, multiplied by +-i), bit for bit."""
    rng = W.rng_for(seed)
    psi0 = W.random_state(n, rng)
    idx = np.arange(1 << n)
    for t in range(n):
        got = O.apply_1q(psi0.copy(), t, W.mat_x())
        assert np.array_equal(got, psi0[idx ^ (1 << t)])
        got = O.apply_1q(psi0.copy(), t, W.mat_y())
        src = psi0[idx ^ (1 << t)]
        sign = np.where((idx >> t) & 1, 1j, -1j)
        assert np.array_equal(got, src * sign)
    for _ in range(6):
        c, t = W.random_distinct(rng, n, 2)
        got = O.apply_1q(psi0.copy(), t, W.mat_x(), ctrls=(c,))
        src = np.where((idx >> c) & 1, idx ^ (1 << t), idx)
        assert np.array_equal(got, psi0[src])
        a, b = W.random_distinct(rng, n, 2)
        got = O.apply_perm(psi0.copy(), [a, b], [0, 2, 1, 3])
        ba, bb = (idx >> a) & 1, (idx >> b) & 1
        src = idx ^ ((ba ^ bb) << a) ^ ((ba ^ bb) << b)
        assert np.array_equal(got, psi0[src])
    # general permutation with a control, against explicit index arithmetic
    k = 3
    tg = W.random_distinct(rng, n, k + 1)
    targets, ctrl = tg[:k], tg[k]
    perm = rng.permutation(1 << k).astype(np.uint32)
    inv = np.argsort(perm)
    got = O.apply_perm(psi0.copy(), targets, perm, ctrls=(ctrl,))
    s = sum(((idx >> targets[j]) & 1) << j for j in range(k))
    s_src = inv[s]
    src = idx.copy()
    for j in range(k):
        src = (src & ~(1 << targets[j])) | (((s_src >> j) & 1) << targets[j])
    src = np.where((idx >> ctrl) & 1, src, idx)
    assert np.array_equal(got, psi0[src])


def pin_threaded_build_identical(O, n=14, seed=900):
    """The OpenMP timing build computes bit-identical states: every index's
    update touches only its own pair or group."""
    gates = random_mixed_circuit(n, 40, seed) + W.shor_like(n, seed=seed)[0]
    psi0 = W.random_state(n, W.rng_for(seed))
    a = O.run_circuit(psi0.copy(), gates)
    prev = O.threads()
    try:
        O.set_threads(4)
        b = O.run_circuit(psi0.copy(), gates)
    finally:
        O.set_threads(prev)
    assert np.array_equal(a, b)


def pin_probs(O, n=10, seed=800):
    psi = W.random_state(n, W.rng_for(seed))
    p_all = (np.abs(psi) ** 2).reshape((2,) * n)
    rng = W.rng_for(seed + 1)
    for k in (1, 2, 3):
        qs = W.random_distinct(rng, n, k)
        got = O.probs(psi, qs)
        # marginal by summing the tensor over the other axes (axis a = qubit n-1-a)
        keep = [n - 1 - q for q in qs]
        other = tuple(a for a in range(n) if a not in keep)
        marg = p_all.sum(axis=other)  # remaining axes in increasing axis order
        order = sorted(keep)
        want = np.zeros(1 << k)
        for s in range(1 << k):
            index = tuple(((s >> qs.index(n - 1 - a)) & 1) for a in order)
            want[s] = marg[index]
        assert _maxerr(got, want) < 1e-14
    assert abs(O.norm2(psi) - float(np.sum(np.abs(psi) ** 2))) < 1e-14


ALL_PINS = [
    pin_textbook_1q,
    pin_textbook_2q,
    pin_bruteforce,
    pin_tensordot,
    pin_dense_wide,
    pin_hadamard_uniform,
    pin_qft_basis,
    pin_grover,
    pin_shor_like,
    pin_norm_and_inverse,
    pin_moves_exact,
    pin_probs,
    pin_threaded_build_identical,
]
