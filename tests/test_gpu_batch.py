"""Batched execution: many states of uneven qubit counts in one persistent
launch (qs_batch_run), each result against the oracle or a closed form."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import MODES, arith_gates, assert_close, assert_state, c128_tol, mode_args, qs
from pins import grover_closed_form, shor_counting_distribution
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
    Shor-like order finding, qubit counts uniform in 10..14: every state
    against the oracle, and against the closed forms (Grover: every amplitude;
    Shor-like: the counting distribution)."""
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
            meta.append(("grover", n, marked, W.grover_iterations(n), gates))
        else:
            gates, prm = W.shor_like(n, seed=9300 + i)
            meta.append(("shor", n, prm, None, gates))
        circuits.append(q.Circuit(gates))
    q.qs_batch_run([s.h for s in states], circuits, q.run_opts(use_graph=1))
    math_mode = "fp64" if mode == "c128_fp64" else "df"
    for st, m in zip(states, meta):
        got = st.read()
        ref = O.run_circuit(O.basis_state(m[1]), m[4])
        if mode.startswith("c128"):
            # Grover runs 25..100 iterations (up to 2.8k Hadamards per
            # amplitude): the depth term of the tolerance applies
            tol = c128_tol(m[4], math_mode)
            err = float(np.max(np.abs(got - ref)))
            assert err <= tol, f"{m[0]} n={m[1]}: max abs error {err:.3e} > {tol:.3e}"
        else:
            assert_state(got, ref, mode, f"{m[0]} n={m[1]}")
        if m[0] == "grover":
            _, n, marked, r, gates = m
            # the FP64 oracle itself drifts from the closed form by up to
            # 2^-52 per Hadamard (its 1/sqrt 2 is a rounded double)
            if mode.startswith("c128"):
                tol = c128_tol(gates, math_mode) + arith_gates(gates) * 2.0 ** -52
                assert np.max(np.abs(got - grover_closed_form(n, marked, r))) < tol
        else:
            _, n, prm, _, _ = m
            p = st.probs(list(range(prm["t"])))
            want = shor_counting_distribution(prm["t"], prm["a"], prm["N"])
            if mode.startswith("c128"):
                assert np.max(np.abs(p - want)) < 1e-12
            else:
                assert np.max(np.abs(p / p.sum() - want)) < 1e-5
        st.close()


@pytest.mark.parametrize("mode", ["c128_df", "c64"])
def test_batch_run_with_graph_twice(mode):
    """qs_batch_run with use_graph captures and launches each call afresh:
    two calls apply the circuits twice."""
    q = qs()
    ns = [6, 12, 13, 17]
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
        assert_close(st.read(), ref, mode, "graph, two calls")
        st.close()


@pytest.mark.parametrize("mode", ["c128_df", "c64"])
def test_graph_after_states_replaced(mode):
    """States closed and made again (the allocator hands out the same
    addresses) and circuits rebuilt: a later graph run must apply the new
    circuits to the new states."""
    q = qs()
    ns = [5, 11, 12, 14]
    for rnd in range(3):
        states = make_states(ns, mode)
        gates = [mixed_circuit(n, 20, seed=9600 + 10 * rnd + n) for n in ns]
        psis = [W.random_state(n, W.rng_for(9700 + 10 * rnd + n)) for n in ns]
        for st, p in zip(states, psis):
            st.load(p)
        q.qs_batch_run([s.h for s in states], [q.Circuit(g) for g in gates], q.run_opts(use_graph=1))
        for st, g, p in zip(states, gates, psis):
            assert_close(st.read(), O.run_circuit(p.copy(), g), mode, f"round {rnd}")
            st.close()


@pytest.mark.parametrize("mode", MODES)
def test_compiled_batch_launch_twice(mode):
    """qs_batch_compile then two qs_batch_launch: the circuits are applied
    twice, and the circuits may be dropped after compiling."""
    q = qs()
    ns = [3, 9, 11, 12, 15, 18, 21]
    states = make_states(ns, mode)
    gates = [mixed_circuit(n, 20, seed=9800 + n) for n in ns]
    psis = [W.random_state(n, W.rng_for(9900 + n)) for n in ns]
    for st, p in zip(states, psis):
        st.load(p)
    circuits = [q.Circuit(g) for g in gates]
    b = q.qs_batch_compile([s.h for s in states], circuits)
    del circuits
    q.qs_batch_launch(b)
    q.qs_batch_launch(b)
    for st, g, p in zip(states, gates, psis):
        ref = O.run_circuit(O.run_circuit(p.copy(), g), g)
        assert_close(st.read(), ref, mode, f"compiled batch n={st.n}")
    # a destroyed member invalidates the handle
    states[2].close()
    with pytest.raises(q.QSError) as e:
        q.qs_batch_launch(b)
    assert e.value.status == q.QS_ERR_ARG
    q.qs_batch_destroy(b)
    for st in states:
        st.close()


def test_compiled_batch_orders_member_streams():
    """Work queued on a member's own stream before the launch is seen by the
    batch, and work queued there after it sees the batch's result."""
    torch = pytest.importorskip("torch")
    q = qs()
    ns = [10, 13]
    states = make_states(ns, "c128_df")
    streams = [torch.cuda.Stream() for _ in ns]
    for st, s in zip(states, streams):
        q.qs_set_stream(st.h, s.cuda_stream)
    gates = [mixed_circuit(n, 30, seed=9950 + n) for n in ns]
    b = q.qs_batch_compile([s.h for s in states], [q.Circuit(g) for g in gates])
    pre = [W.H(q_) for q_ in range(4)]
    for st in states:
        q.qs_init_basis(st.h, 3)
        st.run(pre, max_fuse=1)       # queued on the member's own stream
    q.qs_batch_launch(b)
    for st in states:
        st.run([W.X(0)], max_fuse=1)  # after the batch, on the member's stream
    for st, g, n in zip(states, gates, ns):
        ref = O.run_circuit(O.run_circuit(O.run_circuit(O.basis_state(n, 3), pre), g), [W.X(0)])
        assert_close(st.read(), ref, "c128_df", f"stream order n={n}")
    q.qs_batch_destroy(b)
    for st in states:
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
