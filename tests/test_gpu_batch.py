"""Batched execution: many states of uneven qubit counts in one persistent
launch (qs_batch_run), each result against the oracle or a closed form."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import MODES, assert_close, mode_args, qs
from pins import shor_counting_distribution
from test_gpu_fused import mixed_circuit

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_09198_gb300 import build

    build.build()
    O.build()


def make_states(ns, mode):
    q = qs()
    dt, math_mode = mode_args(mode)
    return [q.State(n, dt, math_mode) for n in ns]


@pytest.mark.parametrize("mode", MODES)
def test_batch_mixed_sizes_against_oracle(mode):
    q = qs()
    rng = W.rng_for(9000)
    ns = [1, 2, 3, 5, 8, 10, 11, 12, 13, 14, 16, 9, 4, 15, 7, 6]
    circuits, psis, states = [], [], make_states(ns, mode)
    for i, (n, st) in enumerate(zip(ns, states)):
        gates = mixed_circuit(n, 30 + 5 * (i % 4), seed=9100 + i)
        psi0 = W.random_state(n, rng)
        st.load(psi0)
        circuits.append((gates, q.Circuit(gates)))
        psis.append(psi0)
    q.qs_batch_run([s.h for s in states], [c for _, c in circuits])
    for n, st, (gates, _), psi0 in zip(ns, states, circuits, psis):
        ref = O.run_circuit(psi0.copy(), gates)
        assert_close(st.read(), ref, mode, f"batch state n={n}")
        st.close()


@pytest.mark.parametrize("mode", MODES)
def test_batch_grover_and_shor_pins(mode):
    """Half Grover (random marked item, optimal iteration count), half
    Shor-like order finding, qubit counts uniform in 10..14."""
    q = qs()
    rng = W.rng_for(9200)
    count = 24
    ns = [int(x) for x in rng.integers(10, 15, size=count)]
    states = make_states(ns, mode)
    circuits, meta = [], []
    for i, n in enumerate(ns):
        if i % 2 == 0:
            marked = int(rng.integers(1 << n))
            gates = W.grover(n, marked)
            meta.append(("grover", n, marked, W.grover_iterations(n)))
        else:
            gates, prm = W.shor_like(n, seed=9300 + i)
            meta.append(("shor", n, prm, None))
        circuits.append(q.Circuit(gates))
    q.qs_batch_run([s.h for s in states], circuits, q.run_opts(use_graph=1))
    tol = 1e-10 if mode.startswith("c128") else 2e-4
    for st, m in zip(states, meta):
        if m[0] == "grover":
            _, n, marked, r = m
            p = st.probs(list(range(n)))
            theta = math.asin(2.0 ** (-n / 2))
            assert abs(p[marked] - math.sin((2 * r + 1) * theta) ** 2) < tol
        else:
            _, n, prm, _ = m
            got = st.probs(list(range(prm["t"])))
            want = shor_counting_distribution(prm["t"], prm["a"], prm["N"])
            assert np.max(np.abs(got - want)) < tol
        st.close()


@pytest.mark.parametrize("mode", ["c128_df", "c64"])
def test_batch_graph_replay(mode):
    """The second call with use_graph replays the captured launch."""
    q = qs()
    ns = [6, 12, 13]
    states = make_states(ns, mode)
    gates = [mixed_circuit(n, 25, seed=9400 + n) for n in ns]
    psis = [W.random_state(n, W.rng_for(9500 + n)) for n in ns]
    for st, p in zip(states, psis):
        st.load(p)
    circuits = [q.Circuit(g) for g in gates]
    opts = q.run_opts(use_graph=1)
    q.qs_batch_run([s.h for s in states], circuits, opts)
    q.qs_batch_run([s.h for s in states], circuits, opts)
    for st, g, p in zip(states, gates, psis):
        ref = O.run_circuit(O.run_circuit(p.copy(), g), g)
        assert_close(st.read(), ref, mode, "graph replay")
        st.close()


def test_batch_argument_errors():
    q = qs()
    a = q.State(5, q.QS_C128)
    b = q.State(5, q.QS_C64)
    c = q.Circuit([W.H(0)])
    with pytest.raises(q.QSError):
        q.qs_batch_run([a.h, b.h], [c, c])
    with pytest.raises(q.QSError):
        q.qs_batch_run([a.h, a.h], [c, c])
    q.qs_batch_run([], [])
    a.close()
    b.close()
