"""qs_probs_noalloc, the entry point for callers that cannot allocate memory
(device memory owned by another allocator, no allocation or cudaFree sync
allowed in their loop, or only raw device pointers at hand), against the
allocating qs_probs on the same state, through the C ABI.

Collected last on purpose, so that a run stopping at the first failure has
already run every other test; it also passes when run alone."""
import numpy as np
import pytest

import workloads as W
from gpu_common import qs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2506_09198_gb300 import build

    build.build()
    return qs()


@pytest.mark.parametrize("dtype_name", ["c128", "c64"])
def test_noalloc_matches_qs_probs_twice(lib, dtype_name):
    torch = pytest.importorskip("torch")
    q = lib
    dtype = q.QS_C128 if dtype_name == "c128" else q.QS_C64
    tol = 1e-13 if dtype_name == "c128" else 1e-12
    n = 18
    st = q.State(n, dtype)
    st.load(W.random_state(n, W.rng_for(9100 + dtype)))
    dev_state = q.qs_device_ptr(st.h)
    stream = torch.cuda.current_stream().cuda_stream
    q.qs_set_stream(st.h, stream)
    for qubits in ([3, 11, 0], [], [17, 4, 9, 12, 1, 6, 2]):  # two calls in a row, then a third
        k = len(qubits)
        want = st.probs(qubits) if k else np.array([st.norm()])
        out = torch.full((1 << k,), float("nan"), dtype=torch.float64, device="cuda")
        q.qs_probs_noalloc(dev_state, n, dtype, qubits, out.data_ptr(), stream)
        torch.cuda.current_stream().synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - want)) <= tol, f"qubits={qubits}"
    st.close()


def test_noalloc_rejects_oversize_requests(lib):
    torch = pytest.importorskip("torch")
    q = lib
    n = 18
    st = q.State(n, q.QS_C64)
    dev_state = q.qs_device_ptr(st.h)
    out = torch.zeros(1 << 17, dtype=torch.float64, device="cuda")
    with pytest.raises(q.QSError) as e:
        q.qs_probs_noalloc(dev_state, n, q.QS_C64, list(range(17)), out.data_ptr())
    assert e.value.status == q.QS_ERR_ARG and "2^16" in str(e.value)
    with pytest.raises(q.QSError):
        q.qs_probs_noalloc(dev_state, n, q.QS_C64, [1, 1], out.data_ptr())
    with pytest.raises(q.QSError):
        q.qs_probs_noalloc(0, n, q.QS_C64, [1], out.data_ptr())
    st.close()
