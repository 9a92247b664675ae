"""Parity at the full workload sizes, on sampled outputs the oracle computes
one by one, or through properties that hold at any size.

- 30-qubit complex128 gate sweep (16 GiB, the benchmark's launch
  configuration): each checked gate starts from the pristine seeded state
  (a device copy restored before the gate); sampled outputs are compared with
  the oracle applied to the 2- or 4-amplitude sub-state they depend on.
- 32-qubit QFT of a random basis state (complex128 64 GiB, complex64 32 GiB):
  sampled amplitudes against the closed form.
- 32-qubit RQC (20 layers): norm, and complex64 vs complex128 fidelity.
- 24-qubit RQC: full state against the oracle.
- Batched states of 10..20 qubits (Grover and Shor-like): every state
  element by element against the oracle (Grover at n = 17..20 with a few
  iterations, so that the oracle finishes in seconds), and Grover at its
  optimal iteration count, n = 17..20, against its closed-form state.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import C128_TOL, arith_gates, assert_state, c128_tol, fidelity, oracle_threads, qs
from pins import grover_closed_form, qft_closed_form, shor_counting_distribution

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_09198_gb300 import build

    build.build()
    O.build()


def _sample_indices(n, count, seed):
    rng = W.rng_for(seed)
    idx = rng.integers(0, 1 << n, size=count, dtype=np.uint64)
    edges = np.array([0, 1, (1 << n) - 1, (1 << (n - 1)), (1 << (n - 1)) - 1], dtype=np.uint64)
    return np.unique(np.concatenate([idx, edges]))


def test_sweep_30q_c128_sampled():
    torch = pytest.importorskip("torch")
    q = qs()
    n = 30
    psi = W.random_state(n, 2507)  # the benchmark's state
    pristine = torch.from_numpy(psi.view(np.float64)).cuda()
    work = torch.empty_like(pristine)
    stream = torch.cuda.current_stream().cuda_stream
    h = q.qs_wrap(n, q.QS_C128, work.data_ptr(), stream)
    g1s, g2s = W.gate_sweep(n, 64, seed=2507)  # the benchmark's gates
    idx = _sample_indices(n, 4096, seed=11)
    out = np.empty(idx.size, dtype=np.complex128)
    checked = [g1s[t] for t in (0, 1, 2, 4, 5, 9, 17, 28, 29)] + g2s[:6]
    for g in checked:
        work.copy_(pristine)
        q.qs_apply_1q(h, g.targets[0], g.data) if g.kind == "u1" else \
            q.qs_apply_2q(h, g.targets[0], g.targets[1], g.data)
        q.qs_gather(h, idx, out)
        i64 = idx.astype(np.int64)
        if g.kind == "u1":
            t = g.targets[0]
            up = i64 & ~(1 << t)
            sub = np.stack([psi[up], psi[up | (1 << t)]], axis=1)
            want = np.empty(idx.size, dtype=np.complex128)
            for j in range(idx.size):
                res = O.apply_1q(sub[j].copy(), 0, g.data)
                want[j] = res[(i64[j] >> t) & 1]
        else:
            t0, t1 = g.targets
            base = i64 & ~((1 << t0) | (1 << t1))
            quads = np.stack([psi[base], psi[base | (1 << t0)], psi[base | (1 << t1)],
                              psi[base | (1 << t0) | (1 << t1)]], axis=1)
            want = np.empty(idx.size, dtype=np.complex128)
            for j in range(idx.size):
                res = O.apply_kq(quads[j].copy(), [0, 1], g.data)
                want[j] = res[((i64[j] >> t0) & 1) + 2 * ((i64[j] >> t1) & 1)]
        err = float(np.max(np.abs(out - want)))
        assert err <= C128_TOL, f"gate {g.kind} {g.targets}: max error {err:.3e}"
    q.qs_destroy(h)


@pytest.mark.parametrize("dtype_name", ["c128", "c64"])
def test_qft_32q_closed_form_sampled(dtype_name):
    q = qs()
    n = 32
    dt = q.QS_C128 if dtype_name == "c128" else q.QS_C64
    x = int(W.rng_for(2510).integers(1 << n))
    st = q.State(n, dt)
    q.qs_init_basis(st.h, x)
    st.run(W.qft(list(range(n))))
    idx = _sample_indices(n, 1 << 14, seed=12)
    got = st.gather(idx).astype(np.complex128)
    want = qft_closed_form(n, x, idx.astype(np.int64))
    err = float(np.max(np.abs(got - want)))
    # complex128: 1e-12; complex64 amplitudes are 2^-16 in size, FP32 gives ~1e-11
    tol = C128_TOL if dtype_name == "c128" else 1e-9
    assert err <= tol, f"QFT 32q {dtype_name}: max error {err:.3e}"
    assert abs(st.norm() - 1.0) < (1e-12 if dtype_name == "c128" else 1e-4)
    st.close()


def test_rqc_32q_norm_and_c64_fidelity():
    torch = pytest.importorskip("torch")
    q = qs()
    n = 32
    gates = W.rqc(n, 20, seed=2508)
    a = torch.zeros(1 << n, dtype=torch.complex128, device="cuda")
    b = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    ha = q.qs_wrap(n, q.QS_C128, a.data_ptr(), stream)
    hb = q.qs_wrap(n, q.QS_C64, b.data_ptr(), stream)
    q.qs_init_basis(ha, 0)
    q.qs_init_basis(hb, 0)
    c = q.Circuit(gates)
    q.qs_fuse_run(ha, c)
    q.qs_fuse_run(hb, c)
    assert abs(q.qs_norm(ha) - 1.0) < 1e-12
    # fidelity |<b|a>|^2 / (|a|^2 |b|^2), accumulated in FP64 chunk by chunk
    inner = 0j
    na = nb = 0.0
    chunk = 1 << 26
    for lo in range(0, 1 << n, chunk):
        xa = a[lo:lo + chunk]
        xb = b[lo:lo + chunk].to(torch.complex128)
        inner += complex(torch.vdot(xb, xa).item())
        na += float(torch.vdot(xa, xa).real.item())
        nb += float(torch.vdot(xb, xb).real.item())
    fid = abs(inner) ** 2 / (na * nb)
    assert fid >= 1 - 1e-5, f"fidelity {fid}"
    q.qs_destroy(ha)
    q.qs_destroy(hb)


@pytest.mark.parametrize("dtype_name", ["c128_df", "c64"])
def test_rqc_24q_full_state(dtype_name):
    q = qs()
    n = 24
    gates = W.rqc(n, 20, seed=2508)
    ref = O.run_circuit(O.basis_state(n), gates)
    dt = q.QS_C128 if dtype_name == "c128_df" else q.QS_C64
    st = q.State(n, dt)
    st.run(gates)
    got = st.read().astype(np.complex128)
    st.close()
    if dtype_name == "c128_df":
        assert float(np.max(np.abs(got - ref))) <= C128_TOL
    else:
        fid = abs(np.vdot(got, ref)) ** 2 / (np.vdot(got, got).real * np.vdot(ref, ref).real)
        assert fid >= 1 - 1e-5


def _batch_mode(dtype_name):
    q = qs()
    return {"c128": (q.QS_C128, q.QS_MATH_DF, "df"), "c128_fp64": (q.QS_C128, q.QS_MATH_FP64, "fp64"),
            "c64": (q.QS_C64, q.QS_MATH_DF, "c64")}[dtype_name]


@pytest.mark.parametrize("dtype_name", ["c128", "c128_fp64", "c64"])
def test_batched_10_to_20_qubits(dtype_name):
    """Grover (random marked item) and Shor-like states of every size 10..20
    in one batched launch, each compared element by element with the oracle
    (complex128: max amplitude error 1e-12, plus for float-float arithmetic
    2^-49 per arithmetic gate on the deep Grover circuits; FP64 arithmetic:
    1e-12 flat; complex64: fidelity 1 - 1e-5).  Grover runs its optimal
    iteration count up to 16 qubits and 6 iterations above; the Shor-like
    distribution is also checked against its closed form."""
    q = qs()
    dt, mm, math_mode = _batch_mode(dtype_name)
    rng = W.rng_for(2511)
    states, circuits, meta = [], [], []
    for n in range(10, 21):
        marked = int(rng.integers(1 << n))
        r = W.grover_iterations(n) if n <= 16 else 6
        gates = W.grover(n, marked, r)
        states.append(q.State(n, dt, mm))
        circuits.append(q.Circuit(gates))
        meta.append(("grover", n, gates, None))
        gates, prm = W.shor_like(n, seed=2600 + n)
        states.append(q.State(n, dt, mm))
        circuits.append(q.Circuit(gates))
        meta.append(("shor", n, gates, prm))
    q.qs_batch_run([s.h for s in states], circuits)
    with oracle_threads(O):
        for st, (kind, n, gates, prm) in zip(states, meta):
            got = st.read()
            ref = O.run_circuit(O.basis_state(n), gates)
            if dt == q.QS_C128:
                tol = c128_tol(gates, math_mode) if kind == "grover" else C128_TOL
                err = float(np.max(np.abs(got - ref)))
                assert err <= tol, f"batched {kind} n={n}: max abs error {err:.3e} > {tol:.3e}"
            else:
                assert_state(got, ref, "c64", f"batched {kind} n={n}")
            if kind == "shor":
                p = st.probs(list(range(prm["t"])))
                want = shor_counting_distribution(prm["t"], prm["a"], prm["N"])
                tol = 1e-12 if dt == q.QS_C128 else 1e-5
                p = p if dt == q.QS_C128 else p / p.sum()
                assert np.max(np.abs(p - want)) < tol, f"Shor-like n={n}"
            st.close()


@pytest.mark.parametrize("dtype_name", ["c128", "c128_fp64", "c64"])
def test_batched_grover_17_to_20_closed_form(dtype_name):
    """Grover at its optimal iteration count (284..804 iterations, up to 32k
    Hadamards per amplitude) on 17..20 qubits, batched: every amplitude
    against the closed form.  Exact FP64 arithmetic itself drifts from the
    closed form by up to 2^-52 per Hadamard (its 1/sqrt 2 is a rounded double;
    the oracle: 8.6e-13 at 17 qubits, 2.8e-12 at 20), so that term is added to
    the complex128 tolerance, and float-float adds its own 2^-49 per
    arithmetic gate; complex64 keeps the fidelity bar."""
    q = qs()
    dt, mm, math_mode = _batch_mode(dtype_name)
    rng = W.rng_for(2512)
    ns = [17, 18, 19, 20]
    marks = [int(rng.integers(1 << n)) for n in ns]
    circs = [W.grover(n, m) for n, m in zip(ns, marks)]
    states = [q.State(n, dt, mm) for n in ns]
    q.qs_batch_run([s.h for s in states], [q.Circuit(g) for g in circs])
    for st, n, m, gates in zip(states, ns, marks, circs):
        got = st.read().astype(np.complex128)
        want = grover_closed_form(n, m, W.grover_iterations(n))
        if dt == q.QS_C128:
            tol = c128_tol(gates, math_mode) + arith_gates(gates) * 2.0 ** -52
            err = float(np.max(np.abs(got - want)))
            assert err < tol, f"Grover n={n}: max amplitude error {err:.3e} against the closed form (bound {tol:.3e})"
        else:
            f = fidelity(got, want)
            assert f >= 1 - 1e-5, f"Grover n={n}: fidelity {f}"
        st.close()
