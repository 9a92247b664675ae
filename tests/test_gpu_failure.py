"""Failure detection without a GPU fault: bounded waits that run out.

- Host side: qs_sync with a deadline shorter than the queued work returns
  QS_ERR_TIMEOUT (the work is not cancelled), and a later qs_sync with a real
  limit returns QS_OK.
- Device side: with the wait limit of the fused and batched kernels set to
  zero, their first wait on a tile copy (or on the warps consuming one) runs
  out; the kernel records QS_ERR_TIMEOUT in the state's own error word, lets
  its own copies land and returns.  The state's next synchronous call reports
  the timeout, other states are unaffected, and the context stays usable:
  with the default limit restored the same circuit gives the oracle's result.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import assert_close, qs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_09198_gb300 import build

    build.build()
    O.build()


@pytest.fixture
def restore_wait_limit():
    yield
    qs().qs_set_wait_limit(2.0)


def test_host_deadline_shorter_than_the_work():
    q = qs()
    st = q.State(28, q.QS_C128)
    st.run(W.rqc(28, 20, seed=2508))  # a few hundred ms of queued device work
    with pytest.raises(q.QSError) as e:
        q.qs_sync(st.h, 0.0)
    assert e.value.status == q.QS_ERR_TIMEOUT
    q.qs_sync(st.h, 120.0)  # the work was not cancelled: it drains
    assert abs(st.norm() - 1.0) < 1e-12
    st.close()


@pytest.mark.parametrize("dtype_name", ["c128", "c64"])
def test_device_wait_runs_out_and_context_survives(dtype_name, restore_wait_limit):
    q = qs()
    dt = q.QS_C128 if dtype_name == "c128" else q.QS_C64
    n = 20
    gates = W.rqc(n, 6, seed=2509)
    bystander = q.State(12, dt)
    bystander.run([W.H(0), W.CNOT(0, 1)])
    st = q.State(n, dt)
    q.qs_set_wait_limit(0.0)
    st.run(gates)  # fused blocks: every launch gives up at its first wait
    q.qs_set_wait_limit(2.0)
    with pytest.raises(q.QSError) as e:
        st.sync()
    assert e.value.status == q.QS_ERR_TIMEOUT
    # the error belonged to st only, and was cleared by reading it
    bystander.sync()
    st.sync()
    # the context still works: the same circuit from |0...0> matches the oracle
    q.qs_init_basis(st.h, 0)
    st.run(gates)
    ref = O.run_circuit(O.basis_state(n), gates)
    assert_close(st.read(), ref, "c128_df" if dtype_name == "c128" else "c64", "after a timeout")
    b = bystander.read()
    assert abs(abs(b[0]) ** 2 - 0.5) < 1e-6 and abs(abs(b[3]) ** 2 - 0.5) < 1e-6
    st.close()
    bystander.close()


def test_batched_wait_runs_out(restore_wait_limit):
    q = qs()
    ns = [8, 11, 13, 15]
    states = [q.State(n, q.QS_C128) for n in ns]
    gates = [W.rqc(n, 8, seed=2600 + n) for n in ns]
    q.qs_set_wait_limit(0.0)
    q.qs_batch_run([s.h for s in states], [q.Circuit(g) for g in gates])
    q.qs_set_wait_limit(2.0)
    with pytest.raises(q.QSError) as e:
        states[0].sync()  # a batch reports through its first state
    assert e.value.status == q.QS_ERR_TIMEOUT
    for st in states:
        q.qs_init_basis(st.h, 0)
    q.qs_batch_run([s.h for s in states], [q.Circuit(g) for g in gates])
    for st, g, n in zip(states, gates, ns):
        assert_close(st.read(), O.run_circuit(O.basis_state(n), g), "c128_df", f"n={n} after a timeout")
        st.close()


def test_wait_limit_argument_errors():
    q = qs()
    for bad in (-1.0, 61.0, float("nan")):
        with pytest.raises(q.QSError) as e:
            q.qs_set_wait_limit(bad)
        assert e.value.status == q.QS_ERR_ARG
