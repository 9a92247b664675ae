"""States split over device and host memory (qs_create_split): the top g
qubits select segments, some in HBM and some in pinned host memory; gates
with global targets swap qubits into the local range through a qubit map.
Every result against the oracle: gate by gate, fused, marginals, gathers."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import MODES, assert_close, mode_args, qs
from pins import qft_closed_form
from test_gpu_fused import mixed_circuit

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_09198_gb300 import build

    build.build()
    O.build()


def split_state(n, mode, g, hbm):
    q = qs()
    dt, math = mode_args(mode)
    return q.State.split(n, dt, g, hbm, math)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("g,hbm", [(1, 1), (2, 2), (2, 0), (3, 5), (2, 4)])
def test_split_gate_by_gate_and_fused(mode, g, hbm):
    n = 13
    gates = mixed_circuit(n, 70, seed=9900 + 10 * g + hbm)
    psi0 = W.random_state(n, W.rng_for(9950 + g))
    ref = O.run_circuit(psi0.copy(), gates)
    st = split_state(n, mode, g, hbm)
    st.load(psi0)
    for gt in gates:
        st.apply(gt)
    assert_close(st.read(), ref, mode, f"split g={g} hbm={hbm}, gate by gate")
    st.load(psi0)
    st.run(gates, max_fuse=0)
    assert_close(st.read(), ref, mode, f"split g={g} hbm={hbm}, fused")
    st.close()


@pytest.mark.parametrize("mode", ["c128_df", "c64"])
def test_split_marginals_gather_norm(mode):
    n, g = 14, 2
    gates = mixed_circuit(n, 50, seed=9970)
    psi0 = W.random_state(n, W.rng_for(9971))
    ref = O.run_circuit(psi0.copy(), gates)
    st = split_state(n, mode, g, 1)
    st.load(psi0)
    st.run(gates)  # leaves a non-identity qubit map behind
    tol = 1e-12 if mode.startswith("c128") else 2e-6
    assert abs(st.norm() - O.norm2(ref)) < tol
    for qubits in ([0, 13, 5], [12, 13], [3], list(range(10)), [13, 1, 12, 0]):
        got = st.probs(qubits)
        assert np.max(np.abs(got - O.probs(ref, qubits))) < tol, f"marginals on {qubits}"
    idx = np.array([0, 1, (1 << n) - 1, 4097, 12345, 8191, 8192], dtype=np.uint64)
    got = st.gather(idx).astype(np.complex128)
    assert np.max(np.abs(got - ref[idx.astype(np.int64)])) < tol
    st.close()


@pytest.mark.parametrize("mode", ["c128_df", "c64"])
def test_split_qft_and_grover(mode):
    q = qs()
    n = 14
    x = 11111
    st = split_state(n, mode, 2, 2)
    q.qs_init_basis(st.h, x)
    st.run(W.qft(list(range(n))))
    got = st.read().astype(np.complex128)
    tol = 1e-12 if mode.startswith("c128") else 1e-6
    assert np.max(np.abs(got - qft_closed_form(n, x))) < tol
    gates = W.grover(n, 9876, 6)
    q.qs_init_basis(st.h, 0)
    st.run(gates)
    assert_close(st.read(), O.run_circuit(O.basis_state(n), gates), mode, "Grover on a split state")
    st.close()


def test_split_rejects_what_it_cannot_take():
    q = qs()
    for args in ((12, q.QS_C128, 0, 1), (12, q.QS_C128, 3, 1), (13, q.QS_C128, 2, 5), (12, 9, 1, 1)):
        with pytest.raises(q.QSError) as e:
            q.qs_create_split(*args)
        assert e.value.status == q.QS_ERR_ARG
    st = split_state(12, "c128_df", 1, 1)
    with pytest.raises(q.QSError) as e:
        q.qs_device_ptr(st.h)
    assert e.value.status == q.QS_ERR_UNSUPPORTED
    with pytest.raises(q.QSError):
        q.qs_batch_run([st.h], [q.Circuit([W.H(0)])])
    st.close()
