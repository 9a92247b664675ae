"""Runs of phase gates on the 2^-32-turn grid inside fused blocks: each gate
adds its angle to an integer accumulator per amplitude, and the amplitude is
multiplied once by the accumulated phase.  Parity against the oracle, which
multiplies by every gate's own coefficient in turn."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import MODES, assert_close, new_state, qs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_09198_gb300 import build

    build.build()
    O.build()


def turn(m):
    """Phase angle of m / 2^32 turn, m a signed 32-bit integer."""
    return 2.0 * math.pi * (m / 2.0 ** 32)


def phase_run(n, length, rng, special=True):
    """A run of commuting phase gates: controlled phases with random and
    special angles, CZ, multi-controlled Z, S, T, Z and one-entry diagonals,
    on low (tile-local) and high qubits alike."""
    gates = []
    specials = [1, -1, 1 << 30, -(1 << 30), 1 << 29, (1 << 31) - 1, 3, 1 << 24, 1 << 8]
    for i in range(length):
        r = int(rng.integers(8))
        if r <= 2:
            m = specials[i % len(specials)] if special and i < len(specials) else int(rng.integers(-2 ** 31, 2 ** 31))
            c, t = W.random_distinct(rng, n, 2)
            gates.append(W.CP(c, t, turn(m)))
        elif r == 3:
            gates.append(W.CZ(*W.random_distinct(rng, n, 2)))
        elif r == 4:
            q = W.random_distinct(rng, n, 3)
            gates.append(W.MCZ(q[1:], q[0]))
        elif r == 5:
            gates.append([W.S, W.T, W.Z][int(rng.integers(3))](int(rng.integers(n))))
        elif r == 6:
            q = W.random_distinct(rng, n, 2)
            d = np.ones(4, dtype=np.complex128)
            d[int(rng.integers(4))] = np.exp(1j * turn(int(rng.integers(-2 ** 31, 2 ** 31))))
            gates.append(W.gdiag(q, d))
        else:
            t = int(rng.integers(n))
            gates.append(W.g1(t, W.mat_phase(turn(int(rng.integers(-2 ** 20, 2 ** 20)) << 12))))
    return gates


def circuit(n, seed, runs=6, run_len=30, off_grid=True):
    rng = W.rng_for(seed)
    gates = [W.H(q) for q in range(n)]
    for j in range(runs):
        gates += phase_run(n, run_len, rng)
        if off_grid:  # a phase off the grid splits the run
            gates.append(W.CP(*W.random_distinct(rng, n, 2), rng.uniform(0.1, 3.0)))
        gates += phase_run(n, int(rng.integers(1, 6)), rng, special=False)
        t = int(rng.integers(n))
        gates.append(W.g1(t, W.haar_unitary(2, rng)))
        gates.append(W.H(int(rng.integers(n))))
    return gates


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n,max_fuse", [(9, 3), (14, 3), (16, 6)])
def test_phase_runs_fused(mode, n, max_fuse):
    gates = circuit(n, 8100 + n)
    ref = O.run_circuit(O.basis_state(n), gates)
    st = new_state(n, mode)
    st.run(gates, max_fuse=max_fuse)
    got = st.read()
    st.close()
    assert_close(got, ref, mode, f"phase runs n={n}")


@pytest.mark.parametrize("mode", MODES)
def test_sign_only_runs(mode):
    """Runs of CZ / multi-controlled Z only: the accumulated phase is a sign."""
    n = 13
    rng = W.rng_for(8200)
    gates = [W.H(q) for q in range(n)]
    for _ in range(5):
        for _ in range(12):
            if rng.integers(2):
                gates.append(W.CZ(*W.random_distinct(rng, n, 2)))
            else:
                q = W.random_distinct(rng, n, 3)
                gates.append(W.MCZ(q[1:], q[0]))
        gates.append(W.g1(int(rng.integers(n)), W.haar_unitary(2, rng)))
    psi = W.random_state(n, W.rng_for(8201))
    ref = O.run_circuit(psi.copy(), gates)
    st = new_state(n, mode, psi)
    st.run(gates, max_fuse=3)
    got = st.read()
    st.close()
    assert_close(got, ref, mode, "sign-only runs")


@pytest.mark.parametrize("dtype_name", ["c128", "c64"])
def test_long_runs_batched(dtype_name):
    """The batched kernel puts a whole small circuit in few blocks, so runs
    exceed the 255 terms one run op holds and are split."""
    q = qs()
    dt = q.QS_C128 if dtype_name == "c128" else q.QS_C64
    mode = "c128_df" if dtype_name == "c128" else "c64"
    states, refs = [], []
    circuits = []
    for i, n in enumerate((8, 10, 12, 14)):
        gates = circuit(n, 8300 + i, runs=2, run_len=300, off_grid=(i % 2 == 0))
        refs.append(O.run_circuit(O.basis_state(n), gates))
        states.append(q.State(n, dt))
        circuits.append(q.Circuit(gates))
    q.qs_batch_run([s.h for s in states], circuits)
    for st, ref in zip(states, refs):
        assert_close(st.read(), ref, mode, f"batched long runs n={st.n}")
        st.close()


@pytest.mark.parametrize("mode", MODES)
def test_qft_fused_against_closed_form(mode):
    """QFT of a random basis state (runs of controlled rotations between the
    Hadamards) against the closed form, at a size that spans tiles."""
    from pins import qft_closed_form

    n = 18
    x = int(W.rng_for(8400).integers(1 << n))
    st = new_state(n, mode)
    qs().qs_init_basis(st.h, x)
    st.run(W.qft(list(range(n))), max_fuse=3)
    got = st.read()
    st.close()
    want = qft_closed_form(n, x, np.arange(1 << n, dtype=np.int64))
    assert_close(got, want, mode, "QFT closed form")
