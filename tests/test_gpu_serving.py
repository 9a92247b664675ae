"""Serving loop: admission by HBM footprint, continuous batching of gate
layers, and the same result for every request alone and in the mix."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import qs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_09198_gb300 import build

    build.build()
    O.build()


def serving():
    from paper_2506_09198_gb300 import serving as S

    return S


def clone(req):
    S = serving()
    return S.Request(rid=req.rid, n=req.n, gates=req.gates, arrival=0.0, kind=req.kind)


@pytest.mark.parametrize("dtype_name", ["c128", "c64"])
def test_alone_equals_in_mix(dtype_name):
    q, S = qs(), serving()
    dtype = q.QS_C128 if dtype_name == "c128" else q.QS_C64
    reqs = S.make_requests(28, seed=7000, n_min=12, n_max=19, rate=400.0)
    srv = S.Server(dtype, hbm_budget_bytes=1 << 27, small_n=15, chunk_gates=64)
    for r in reqs:
        srv.submit(r)
    done = srv.run()
    assert len(done) == len(reqs)
    assert srv.peak_used <= srv.arena.capacity
    assert max(r.admitted - r.arrival for r in done) >= 0.0
    for r in done:
        alone = S.Server(dtype, hbm_budget_bytes=1 << 27, small_n=15, chunk_gates=64)
        a = clone(r)
        alone.submit(a)
        alone.run()
        assert np.array_equal(a.probs, r.probs), f"request {r.rid} ({r.kind}, n={r.n}) differs alone vs mix"
        # complex64 gate matrices carry FP32 rounding (1/sqrt2 is 1.7e-8 low),
        # so the norm drifts by ~3e-8 per H gate over a circuit.
        tol = 1e-12 if dtype_name == "c128" else 1e-4
        assert abs(r.norm - 1.0) < tol


@pytest.mark.parametrize("dtype_name", ["c128", "c64"])
def test_served_results_against_oracle_and_closed_forms(dtype_name):
    q, S = qs(), serving()
    dtype = q.QS_C128 if dtype_name == "c128" else q.QS_C64
    tol = 1e-12 if dtype_name == "c128" else 2e-6
    reqs = S.make_requests(18, seed=7100, n_min=12, n_max=17, rate=0.0)
    srv = S.Server(dtype, hbm_budget_bytes=1 << 26, small_n=14, chunk_gates=100)
    for r in reqs:
        srv.submit(r)
    done = {r.rid: r for r in srv.run()}
    for r in reqs:
        got = done[r.rid].probs
        k = min(8, r.n)
        if r.kind == "qft":
            # QFT of a basis state: every outcome has probability 2^-n.
            assert np.max(np.abs(got - 2.0 ** -k)) < tol
        ref_state = O.run_circuit(O.basis_state(r.n), r.gates)
        want = O.probs(ref_state, list(range(k)))
        assert np.max(np.abs(got - want)) < tol, f"{r.kind} n={r.n}"


def test_admission_respects_footprint():
    q, S = qs(), serving()
    # Budget of 2^22 bytes holds two 17-qubit complex128 states at most.
    srv = S.Server(q.QS_C128, hbm_budget_bytes=1 << 22, small_n=12, chunk_gates=200)
    reqs = [S.Request(rid=i, n=17, gates=W.qft(list(range(17)))) for i in range(5)]
    for r in reqs:
        srv.submit(r)
    done = srv.run()
    assert len(done) == 5
    assert srv.peak_used <= 2 * (16 << 17)
    with pytest.raises(ValueError):
        srv.submit(S.Request(rid=9, n=19, gates=[]))


def test_buddy_arena_merges():
    S = serving()
    a = S.BuddyArena(1 << 20)
    x = a.alloc(1 << 18)
    y = a.alloc(1 << 18)
    z = a.alloc(1 << 19)
    assert None not in (x, y, z) and len({x, y, z}) == 3
    assert a.alloc(1 << 12) is None
    a.release(x, 1 << 18)
    a.release(y, 1 << 18)
    a.release(z, 1 << 19)
    assert a.alloc(1 << 20) == 0
