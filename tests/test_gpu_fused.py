"""Fused-block parity: qs_fuse_run with the tile engine (gates applied in
shared memory, one HBM pass per block) against the oracle, which applies the
same gates one by one."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import MODES, assert_close, assert_state, fidelity, new_state, qs
from pins import grover_closed_form, qft_closed_form, shor_counting_distribution

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_09198_gb300 import build

    build.build()
    O.build()


def mixed_circuit(n, n_gates, seed):
    """Every kind the fuser handles: dense 2x2 (plain, controlled, X, Y, H),
    diagonal 1q/2q/k, dense 4x4 (plain, controlled), permutations, CZ, SWAP."""
    rng = W.rng_for(seed)
    gates = []
    for _ in range(n_gates):
        r = int(rng.integers(10))
        if r <= 2 or n < 2:
            t = int(rng.integers(n))
            U = [W.haar_unitary(2, rng), W.mat_h(), W.mat_x(), W.mat_y()][int(rng.integers(4))]
            nc = int(rng.integers(0, min(2, n - 1) + 1))
            cs = [q for q in W.random_distinct(rng, n, min(n, nc + 1)) if q != t][:nc]
            gates.append(W.g1(t, U, ctrls=cs))
        elif r == 3:
            t = int(rng.integers(n))
            gates.append(W.g1(t, W.mat_phase(rng.uniform(0, 6.3))))
        elif r == 4:
            k = int(rng.integers(1, min(4, n) + 1))
            q = W.random_distinct(rng, n, k)
            gates.append(W.gdiag(q, np.exp(1j * rng.uniform(0, 6.3, 1 << k))))
        elif r in (5, 6):
            q = W.random_distinct(rng, n, min(n, 4))
            cs = q[2:2 + int(rng.integers(0, 2))] if n >= 3 else []
            gates.append(W.gk(q[:2], W.haar_unitary(4, rng), ctrls=cs))
        elif r == 7:
            q = W.random_distinct(rng, n, 2)
            gates.append(W.CZ(*q))
        elif r == 8:
            q = W.random_distinct(rng, n, 2)
            gates.append(W.SWAP(*q))
        else:
            k = int(rng.integers(1, min(3, n) + 1))
            q = W.random_distinct(rng, n, min(n, k + 1))
            gates.append(W.gperm(q[:k], rng.permutation(1 << k).astype(np.uint32), ctrls=q[k:k + int(rng.integers(0, 2))]))
    return gates


def run_gpu(n, mode, gates, psi0, max_fuse):
    st = new_state(n, mode, psi0)
    st.run(gates, max_fuse=max_fuse)
    got = st.read()
    st.close()
    return got


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("max_fuse", [0, 2, 3, 6])
@pytest.mark.parametrize("n", [1, 2, 5, 11, 12, 13, 17])
def test_fused_mixed(mode, max_fuse, n):
    gates = mixed_circuit(n, 60, seed=8000 + n)
    psi0 = W.random_state(n, W.rng_for(8100 + n))
    ref = O.run_circuit(psi0.copy(), gates)
    got = run_gpu(n, mode, gates, psi0, max_fuse)
    assert_close(got, ref, mode, f"fused n={n} max_fuse={max_fuse}")


@pytest.mark.parametrize("mode", MODES)
def test_fused_qft_closed_form(mode):
    n = 15
    x = 12345
    gates = W.qft(list(range(n)))
    got = run_gpu(n, mode, gates, O.basis_state(n, x), 0)
    assert_close(got, qft_closed_form(n, x), mode, "QFT closed form")


@pytest.mark.parametrize("mode", MODES)
def test_fused_rqc(mode):
    n = 16
    gates = W.rqc(n, 20, seed=2508)
    psi0 = O.basis_state(n)
    ref = O.run_circuit(psi0.copy(), gates)
    got = run_gpu(n, mode, gates, psi0, 0)
    assert_close(got, ref, mode, "RQC 20 layers")


@pytest.mark.parametrize("mode", MODES)
def test_fused_rqc_ring(mode):
    n = 14
    gates = W.rqc_ring(n, 5, seed=2509)
    psi0 = O.basis_state(n)
    ref = O.run_circuit(psi0.copy(), gates)
    got = run_gpu(n, mode, gates, psi0, 0)
    assert_close(got, ref, mode, "RQC CNOT ring")


@pytest.mark.parametrize("mode", MODES)
def test_fused_grover_success_probability(mode):
    """Grover on 11 qubits (25 iterations): the whole state against the
    oracle, and against the closed form of every amplitude (the FP64 oracle
    is within 1e-13 of it here)."""
    n = 11
    marked = 1234
    r = W.grover_iterations(n)
    gates = W.grover(n, marked, r)
    st = new_state(n, mode)
    st.run(gates, max_fuse=0)
    got = st.read()
    p = st.probs(list(range(n)))
    st.close()
    assert_state(got, O.run_circuit(O.basis_state(n), gates), mode, "Grover n=11")
    theta = math.asin(2.0 ** (-n / 2))
    if mode.startswith("c128"):
        assert np.max(np.abs(got - grover_closed_form(n, marked, r))) < 1e-12
        assert abs(p[marked] - math.sin((2 * r + 1) * theta) ** 2) < 1e-12
    else:
        assert fidelity(got, grover_closed_form(n, marked, r)) >= 1 - 1e-5


def x_diag_circuit(n, n_gates, seed):
    """X gates around diagonal gates of every form (phase on one pattern,
    general diagonal tables, controls on X'd qubits), with H and CNOT
    between them: the fuser moves X gates past the diagonals it can
    conjugate and cancels pairs."""
    rng = W.rng_for(seed)
    gates = []
    for _ in range(n_gates):
        r = rng.random()
        if r < 0.35:
            gates.append(W.X(int(rng.integers(n))))
        elif r < 0.5:
            q = W.random_distinct(rng, n, 3)
            gates.append(W.MCZ(q[:2], q[2]))
        elif r < 0.6:
            q = W.random_distinct(rng, n, 2)
            gates.append(W.CP(q[0], q[1], float(rng.uniform(0, 6.2))))
        elif r < 0.72:
            k = int(rng.integers(1, 4))
            q = W.random_distinct(rng, n, k + 2)
            nc = int(rng.integers(0, 3))
            d = np.exp(1j * rng.uniform(0, 6.2, size=1 << k))
            gates.append(W.gdiag(q[:k], d, ctrls=q[k:k + nc]))
        elif r < 0.8:
            gates.append(W.T(int(rng.integers(n))))
        elif r < 0.9:
            gates.append(W.H(int(rng.integers(n))))
        else:
            c, t = W.random_distinct(rng, n, 2)
            gates.append(W.CNOT(c, t))
    return gates


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("max_fuse", [0, 2])
def test_x_conjugation_rewrite(mode, max_fuse):
    for n, seed in ((6, 71), (13, 72), (17, 73)):
        gates = x_diag_circuit(n, 160, seed)
        psi0 = W.random_state(n, W.rng_for(seed + 1))
        ref = O.run_circuit(psi0.copy(), gates)
        got = run_gpu(n, mode, gates, psi0, max_fuse)
        assert_close(got, ref, mode, f"X conjugation n={n} max_fuse={max_fuse}")


@pytest.mark.parametrize("mode", ["c128_df", "c64"])
def test_grover_iteration_takes_few_passes(mode):
    """With the oracle's and the diffusion's X gates moved through their
    multi-controlled Z, a Grover iteration on 16 qubits is two phases on a
    bit pattern and two H layers; each H layer spans two tiles (11 qubits
    complex128, 12 complex64, 4 of them strided), so at most 4 fused passes
    per iteration."""
    n, marked, r = 16, 12345, 20
    st = new_state(n, mode)
    st.run(W.grover(n, marked, r), max_fuse=4)
    passes = qs().qs_last_run_stats(st.h)["fused_launches"]
    got = st.read()
    st.close()
    assert passes <= 4 * r + 4, f"{passes} fused passes for {r} Grover iterations"
    assert_state(got, O.run_circuit(O.basis_state(n), W.grover(n, marked, r)), mode, "Grover 16q")


@pytest.mark.parametrize("mode", MODES)
def test_fused_shor_like(mode):
    n = 13
    gates, prm = W.shor_like(n, seed=2510)
    st = new_state(n, mode)
    st.run(gates, max_fuse=0)
    got = st.probs(list(range(prm["t"])))
    st.close()
    want = shor_counting_distribution(prm["t"], prm["a"], prm["N"])
    tol = 1e-11 if mode.startswith("c128") else 1e-5
    assert np.max(np.abs(got - want)) < tol


@pytest.mark.parametrize("mode", MODES)
def test_fused_equals_unfused_many_tiles(mode):
    n = 21
    gates = mixed_circuit(n, 40, seed=8200)
    psi0 = W.random_state(n, W.rng_for(8201))
    a = run_gpu(n, mode, gates, psi0, 1)
    b = run_gpu(n, mode, gates, psi0, 0)
    assert_close(b, a, mode, "fused vs gate-by-gate")


def test_dense_six_qubit_gate_rejected():
    """Dense matrices go up to QS_MAX_DENSE (5) targets; a dense 6-target
    matrix (neither diagonal nor a permutation) is rejected before any work."""
    q = qs()
    st = new_state(8, "c128_df")
    with pytest.raises(q.QSError) as e:
        st.run([W.gk((0, 2, 4, 5, 6, 7), W.haar_unitary(64, W.rng_for(1)))])
    assert e.value.status == q.QS_ERR_UNSUPPORTED
    st.close()


def swap_heavy_circuit(n, n_gates, seed):
    """SWAPs (relabelled inside a block, no data movement) interleaved with
    dense, controlled and phase gates whose qubits the SWAPs exchange."""
    rng = W.rng_for(seed)
    gates = [W.H(q) for q in range(n)]
    for _ in range(n_gates):
        r = int(rng.integers(6))
        if r <= 1:
            gates.append(W.SWAP(*W.random_distinct(rng, n, 2)))
        elif r == 2:
            gates.append(W.g1(int(rng.integers(n)), W.haar_unitary(2, rng)))
        elif r == 3:
            q = W.random_distinct(rng, n, 3)
            gates.append(W.gk(q[:2], W.haar_unitary(4, rng), ctrls=q[2:] if rng.integers(2) else []))
        elif r == 4:
            gates.append(W.CP(*W.random_distinct(rng, n, 2), float(rng.uniform(0, 6.3))))
        else:
            q = W.random_distinct(rng, n, 3)
            gates.append(W.gperm(q[:2], [0, 2, 1, 3], ctrls=q[2:]))  # a controlled SWAP moves data
    return gates


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n,max_fuse", [(7, 3), (12, 3), (15, 2), (15, 5)])
def test_swap_relabel(mode, n, max_fuse):
    gates = swap_heavy_circuit(n, 60, seed=8500 + n + max_fuse)
    psi0 = W.random_state(n, W.rng_for(8501))
    ref = O.run_circuit(psi0.copy(), gates)
    got = run_gpu(n, mode, gates, psi0, max_fuse)
    assert_close(got, ref, mode, f"swap relabel n={n}")


@pytest.mark.parametrize("mode", MODES)
def test_swap_network_moves_exactly(mode):
    """A register reversal by SWAPs alone moves amplitudes bit for bit."""
    n = 17
    gates = [W.SWAP(q, n - 1 - q) for q in range(n // 2)]
    psi0 = W.random_state(n, W.rng_for(8600))
    ref = O.run_circuit(psi0.copy(), gates)
    got = run_gpu(n, mode, gates, psi0, 3)
    assert np.array_equal(got, ref.astype(got.dtype))
