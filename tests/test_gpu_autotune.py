"""The fusion autotuner: times every setting on a scratch state, and
max_fuse = 0 then uses its choice (results unchanged)."""
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


@pytest.mark.parametrize("mode", MODES)
def test_autotune_then_run(mode):
    q = qs()
    n = 17
    gates = W.rqc(n, 6, seed=42)
    c = q.Circuit(gates)
    scratch = new_state(n, mode)
    best, ms = q.qs_autotune(scratch.h, c)
    assert 2 <= best <= 6 and ms > 0
    # the scratch state holds the last trial's result: a full, correct run
    ref = O.run_circuit(O.basis_state(n), gates)
    assert_close(scratch.read(), ref, mode, "autotune trial result")
    scratch.close()
    st = new_state(n, mode)
    st.run(c, max_fuse=0)
    assert_close(st.read(), ref, mode, "tuned run")
    st.close()
