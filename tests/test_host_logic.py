"""Host-side logic that needs no GPU: the serving loop's buddy arena and
request mix, circuit marshalling into the C ABI's records, and the bench's
aggregation over ranks (world size 2 over gloo on the CPU)."""
import ctypes
import math
import os
import socket
import sys

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def serving():
    pytest.importorskip("torch")
    from paper_2506_09198_gb300 import serving as S

    return S


def test_buddy_allocator_splits_and_merges():
    S = serving()
    a = S.BuddyAllocator(1 << 20)
    blocks = [a.alloc(1 << 16) for _ in range(16)]
    assert None not in blocks and len(set(blocks)) == 16
    assert all(b % (1 << 16) == 0 and 0 <= b < (1 << 20) for b in blocks)
    assert a.alloc(1 << 12) is None  # full
    for b in blocks[::2]:
        a.release(b, 1 << 16)
    assert a.alloc(1 << 17) is None  # free space is fragmented into 64 KiB holes
    for b in blocks[1::2]:
        a.release(b, 1 << 16)
    assert a.alloc(1 << 20) == 0  # everything merged back


def test_buddy_allocator_rounds_up_and_aligns():
    S = serving()
    a = S.BuddyAllocator(1 << 20)
    x = a.alloc(3000)  # rounds up to 4096
    y = a.alloc(4096)
    assert x is not None and y is not None and abs(x - y) >= 4096
    assert x % 4096 == 0 and y % 4096 == 0


def test_request_mix_and_sizes():
    S = serving()
    reqs = S.make_requests(400, seed=11, n_min=12, n_max=24, rate=50.0)
    kinds = [r.kind for r in reqs]
    assert abs(kinds.count("rqc") / 400 - 0.4) < 0.08
    assert abs(kinds.count("qft") / 400 - 0.3) < 0.08
    assert abs(kinds.count("grover") / 400 - 0.3) < 0.08
    ns = np.array([r.n for r in reqs])
    assert ns.min() >= 12 and ns.max() <= 24
    # log-uniform: the median sits near sqrt(12 * 24), below the midpoint 18
    assert 15 <= np.median(ns) <= 18
    arrivals = np.array([r.arrival for r in reqs])
    assert np.all(np.diff(arrivals) >= 0)
    assert abs(arrivals[-1] / 400 - 1 / 50.0) < 0.01  # Poisson rate 50/s
    for r in reqs:
        if r.kind == "grover":
            assert sum(1 for g in r.gates if g.name == "mcz") <= 2 * 16  # iterations capped at 16


def test_circuit_marshalling_records():
    pytest.importorskip("torch")
    try:
        from paper_2506_09198_gb300 import qs
    except ImportError:
        pytest.skip("libqs not built")
    rng = W.rng_for(5)
    gates = [W.H(3), W.CNOT(1, 4), W.gk((0, 2), W.haar_unitary(4, rng), ctrls=(5,)),
             W.gperm((1, 2, 3), rng.permutation(8).astype(np.uint32)), W.gdiag((4,), [1, -1]), W.SWAP(0, 6)]
    c = qs.Circuit(gates)
    assert c.n_gates == len(gates) and c.c.n_gates == len(gates)
    d_off = p_off = 0
    for i, g in enumerate(gates):
        rec = c.gates[i]
        assert rec.kind == qs._KIND[g.kind]
        assert rec.k == len(g.targets) and list(rec.targets)[:rec.k] == list(g.targets)
        assert rec.ctrl_mask == sum(1 << q for q in g.ctrls)
        if g.kind == "perm":
            assert rec.offset == p_off
            assert np.array_equal(c.perm[p_off:p_off + len(g.data)], g.data)
            p_off += len(g.data)
        else:
            flat = np.asarray(g.data, dtype=np.complex128).reshape(-1)
            assert rec.offset == d_off
            assert np.array_equal(c.data[d_off:d_off + 2 * flat.size].view(np.complex128), flat)
            d_off += 2 * flat.size


def test_circuit_slices_share_records_and_pools():
    """A serving chunk is a gate-range view: its records are the parent's,
    its pools the parent's (record offsets index the whole circuit's pools)."""
    pytest.importorskip("torch")
    try:
        from paper_2506_09198_gb300 import qs
    except ImportError:
        pytest.skip("libqs not built")
    gates = W.rqc(6, 4, seed=1) + W.shor_like(10, seed=3)[0][:5]
    c = qs.Circuit(gates)
    addr = lambda p: ctypes.cast(p, ctypes.c_void_p).value  # noqa: E731
    for first, count in ((0, 4), (5, 7), (c.n_gates - 3, 10), (c.n_gates, 5)):
        s = c.slice(first, count)
        want = max(0, min(count, c.n_gates - first))
        assert s.n_gates == want and s.c.n_gates == want
        assert addr(s.c.data) == addr(c.c.data) and addr(s.c.perm) == addr(c.c.perm)
        for j in range(want):
            a, b = c.gates[first + j], s.c.gates[j]
            assert (a.kind, a.k, a.ctrl_mask, a.offset) == (b.kind, b.k, b.ctrl_mask, b.offset)
            assert list(a.targets) == list(b.targets)


def test_repeated_circuit_equals_the_flat_one():
    """Circuit.repeated (each part marshalled once, records tiled, pools
    shared) gives the same gate sequence as marshalling the flat list."""
    pytest.importorskip("torch")
    try:
        from paper_2506_09198_gb300 import qs
    except ImportError:
        pytest.skip("libqs not built")
    n, m = 9, 300
    r = W.grover_iterations(n)
    shor = W.shor_like(10, seed=4)[0]
    cases = [(W.grover(n, m), [(W.grover(n, m, 0), 1), (W.grover(n, m, 1)[n:], r)]),
             (shor[:4] * 3 + shor[4:], [(shor[:4], 3), (shor[4:], 1)])]
    for flat, parts in cases:
        a, b = qs.Circuit(flat), qs.Circuit.repeated(parts)
        assert a.n_gates == b.n_gates == len(flat)
        for i in range(a.n_gates):
            x, y = a.gates[i], b.gates[i]
            assert (x.kind, x.k, list(x.targets), x.ctrl_mask) == (y.kind, y.k, list(y.targets), y.ctrl_mask)
            if x.kind == qs.QS_GATE_PERM:
                k = 1 << x.k
                assert np.array_equal(a.perm[x.offset:x.offset + k], b.perm[y.offset:y.offset + k])
            else:
                size = {qs.QS_GATE_U1: 8, qs.QS_GATE_UK: 2 * (1 << x.k) ** 2, qs.QS_GATE_DIAG: 2 * (1 << x.k)}[x.kind]
                assert np.array_equal(a.data[x.offset:x.offset + size], b.data[y.offset:y.offset + size])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(times[rank], world)
    out[rank] = (ms, bench.job_throughput(1e9, 5, ms, world))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    mgr = mp.Manager()
    out = mgr.dict()
    times = [100.0, 125.0]
    port = _free_port()
    procs = [mp.Process(target=_rank_main, args=(r, 2, port, times, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        ms, value = out[r]
        assert ms == 125.0  # every rank sees the slowest rank's time
        assert math.isclose(value, 2 * 1e9 * 5 / 0.125 / 1e9)


def test_reference_arm_other_ranks_do_nothing(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    bench.run_reference(bench.parse())
    assert capsys.readouterr().out == ""


# -- circuit generators: structure as the workload readings state it --------
def test_rqc_structure():
    n, layers = 9, 6
    gates = W.rqc(n, layers, seed=3)
    per_layer = [n + len(range(layer % 2, n - 1, 2)) for layer in range(layers)]
    assert len(gates) == sum(per_layer)
    pos, prev = 0, [None] * n
    for layer in range(layers):
        ones = gates[pos:pos + n]
        assert [g.targets[0] for g in ones] == list(range(n))
        for q, g in enumerate(ones):
            assert g.name in ("sx", "sy", "sw") and g.name != prev[q]  # never the previous choice
            prev[q] = g.name
            U = np.asarray(g.data)
            assert np.allclose(U @ U.conj().T, np.eye(2), atol=1e-15)
        czs = gates[pos + n:pos + per_layer[layer]]
        assert [g.targets for g in czs] == [(a, a + 1) for a in range(layer % 2, n - 1, 2)]
        pos += per_layer[layer]


def test_qft_structure():
    n = 7
    gates = W.qft(list(range(n)))
    hs = [g for g in gates if g.name == "h"]
    cps = [g for g in gates if g.name == "cp"]
    swaps = [g for g in gates if g.name == "swap"]
    assert len(hs) == n and len(cps) == n * (n - 1) // 2 and len(swaps) == n // 2
    for g in cps:  # CP(pi / 2^(j-k)) controlled by k < j on target j
        k, j = g.ctrls[0], g.targets[0]
        assert k < j
        assert np.isclose(np.angle(np.asarray(g.data)[1, 1]), math.pi / (1 << (j - k)))
    assert [g.targets for g in swaps] == [(q, n - 1 - q) for q in range(n // 2)]


def test_grover_and_shor_parameters():
    for n in range(2, 21):
        theta = math.asin(2.0 ** (-n / 2))
        r = W.grover_iterations(n)
        assert (2 * r + 1) * theta <= math.pi / 2 + theta and r == math.floor(math.pi / (4 * theta))
    rng = W.rng_for(9)
    for n in range(8, 21):
        m, t, N, a = W.shor_params(n, rng)
        assert m == max(4, min(8, n // 2)) and t == n - m
        assert N % 2 == 1 and any(N % p == 0 for p in range(3, N)) and max(9, 1 << (m - 1)) <= N < (1 << m)
        assert 1 < a < N and math.gcd(a, N) == 1
        tab = W.mulmod_table(pow(a, 2, N), N, m)
        assert sorted(tab.tolist()) == list(range(1 << m))  # a permutation
