"""Continuous-batching serving loop over the libqs C ABI.

Requests (a circuit on n qubits) arrive over time.  The server admits a
waiting request when its state fits the HBM budget (2^n amplitudes x 8 or 16
bytes) and a slot is free, keeps admitted states resident on the device, and
every scheduler tick advances every resident circuit by its next chunk of
gates ("layer"):
  - states of at most ``small_n`` qubits: one ``qs_batch_run`` launch carries
    the next chunk of all of them;
  - larger states: ``qs_fuse_run`` of their next chunk on their own stream.
New arrivals join at the next tick, so their work overlaps on the device with
the requests already running.  When a circuit's last chunk is done the server
reads its result (marginal probabilities of the lowest ``result_qubits``
qubits and the norm), frees the state and records the latency (arrival to
result).

Chunk boundaries and fusion depend only on the request's own gates, so a
request's result does not depend on what else is in flight.

All compute runs in libqs kernels; this module only schedules.
"""
from __future__ import annotations

import heapq
import math
import time
from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np

from . import qs


@dataclass
class Request:
    rid: int
    n: int
    gates: list
    arrival: float = 0.0          # seconds on the server clock
    kind: str = ""
    result_qubits: int = 8
    meta: dict = field(default_factory=dict)  # generator parameters (marked item, basis state, ...)
    # filled by the server
    admitted: float = -1.0
    finished: float = -1.0
    probs: Optional[np.ndarray] = None
    norm: float = float("nan")

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


@dataclass
class _Active:
    req: Request
    state: "qs.State"
    offset: int
    n_chunks: int
    pos: int = 0
    stream: object = None
    circuit: object = None  # qs.Circuit of the whole request, marshalled at admission


class BuddyAllocator:
    """Power-of-two sub-allocation bookkeeping (state sizes are powers of
    two, so a freed state's block merges back with its buddy).  Offsets
    only; BuddyArena puts device memory under it."""

    def __init__(self, total_bytes: int, min_bytes: int = 1 << 12):
        self.top = max(int(total_bytes).bit_length() - 1, min_bytes.bit_length() - 1)
        self.min_order = min_bytes.bit_length() - 1
        self.free = {o: set() for o in range(self.min_order, self.top + 1)}
        self.free[self.top].add(0)

    @property
    def capacity(self) -> int:
        return 1 << self.top

    def alloc(self, nbytes: int) -> Optional[int]:
        order = max(self.min_order, (int(nbytes) - 1).bit_length())
        o = order
        while o <= self.top and not self.free[o]:
            o += 1
        if o > self.top:
            return None
        off = min(self.free[o])
        self.free[o].remove(off)
        while o > order:  # split, keeping the lower half
            o -= 1
            self.free[o].add(off + (1 << o))
        return off

    def release(self, off: int, nbytes: int):
        o = max(self.min_order, (int(nbytes) - 1).bit_length())
        while o < self.top:
            buddy = off ^ (1 << o)
            if buddy not in self.free[o]:
                break
            self.free[o].remove(buddy)
            off = min(off, buddy)
            o += 1
        self.free[o].add(off)


class BuddyArena(BuddyAllocator):
    """BuddyAllocator over one device allocation (a torch uint8 tensor)."""

    def __init__(self, total_bytes: int, min_bytes: int = 1 << 12):
        import torch

        super().__init__(total_bytes, min_bytes)
        self.tensor = torch.empty(1 << self.top, dtype=torch.uint8, device="cuda")
        self.base = self.tensor.data_ptr()


class Server:
    def __init__(self, dtype: int = qs.QS_C128, hbm_budget_bytes: int = 64 << 30, max_resident: int = 256,
                 small_n: int = 16, chunk_gates: int = 256, max_fuse: int = 0, result_qubits: int = 8):
        import torch

        self.torch = torch
        self.dtype = dtype
        self.amp_bytes = 8 if dtype == qs.QS_C64 else 16
        self.arena = BuddyArena(hbm_budget_bytes)
        self.max_resident = int(max_resident)
        self.small_n = int(small_n)
        self.chunk_gates = int(chunk_gates)
        self.max_fuse = int(max_fuse)
        self.result_qubits = int(result_qubits)
        self.small_stream = torch.cuda.Stream()
        self.streams = [torch.cuda.Stream() for _ in range(4)]
        self.result_stream = torch.cuda.Stream()
        self.reaper = torch.cuda.Stream()  # never given work: closing a finished state waits on nothing
        # Result slots: reads are issued on the result stream and collected
        # when their event has completed, so the scheduler never waits on them.
        self.n_slots = 64
        width = (1 << self.result_qubits) + 1
        self.result_dev = torch.zeros((self.n_slots, width), dtype=torch.float64, device="cuda")
        self.result_host = torch.zeros((self.n_slots, width), dtype=torch.float64, pin_memory=True)
        self.free_slots = list(range(self.n_slots))
        self.reading: List = []          # (active, slot, event, k)
        self._next_stream = 0
        self.used = 0
        self.active: Dict[int, _Active] = {}
        self.pending: List = []          # heap of (arrival, rid, Request)
        self.done: List[Request] = []
        self.ticks = 0
        self.peak_used = 0

    # -- requests ------------------------------------------------------
    def footprint(self, n: int) -> int:
        return self.amp_bytes << n

    def submit(self, req: Request):
        if self.footprint(req.n) > self.arena.capacity:
            raise ValueError(f"request {req.rid}: {req.n} qubits exceed the HBM budget")
        heapq.heappush(self.pending, (req.arrival, req.rid, req))

    def _n_chunks(self, gates) -> int:
        return max(1, -(-len(gates) // self.chunk_gates))

    def _chunk(self, a: "_Active") -> "qs.CircuitSlice":
        """The request's next chunk: a gate-range view of the circuit that was
        marshalled once at admission (no per-chunk marshalling)."""
        return a.circuit.slice(a.pos * self.chunk_gates, self.chunk_gates)

    def _admit(self, now: float):
        while self.pending and self.pending[0][0] <= now and len(self.active) < self.max_resident:
            req = self.pending[0][2]
            fp = self.footprint(req.n)
            off = self.arena.alloc(fp)
            if off is None:
                break  # admission by footprint: wait for memory to free up
            heapq.heappop(self.pending)
            if req.n <= self.small_n:
                stream = self.small_stream
            else:
                stream = self.streams[self._next_stream % len(self.streams)]
                self._next_stream += 1
            h = qs.qs_wrap(req.n, self.dtype, self.arena.base + off, stream.cuda_stream)
            st = qs.State(req.n, self.dtype, handle=h)
            qs.qs_init_basis(st.h, 0)
            req.admitted = now
            self.active[req.rid] = _Active(req, st, off, self._n_chunks(req.gates), 0, stream,
                                           qs.Circuit(req.gates))
            self.used += fp
            self.peak_used = max(self.peak_used, self.used)

    # -- one scheduler tick ---------------------------------------------
    def _tick(self):
        small = [a for a in self.active.values() if a.req.n <= self.small_n]
        large = [a for a in self.active.values() if a.req.n > self.small_n]
        if small:
            qs.qs_batch_run([a.state.h for a in small], [self._chunk(a) for a in small])
            for a in small:
                a.pos += 1
        for a in large:
            qs.qs_fuse_run(a.state.h, self._chunk(a), qs.run_opts(max_fuse=self.max_fuse))
            a.pos += 1
        self.ticks += 1

    def _start_read(self, a: _Active, slot: int):
        """Marginals of the lowest qubits and the norm, computed without
        allocation on one result stream (so result reads never overlap) and
        copied to pinned host memory asynchronously."""
        torch = self.torch
        k = min(self.result_qubits, a.req.n)
        rs = self.result_stream
        rs.wait_stream(a.stream)
        ptr = self.arena.base + a.offset
        out = self.result_dev[slot].data_ptr()
        qs.qs_probs_noalloc(ptr, a.req.n, self.dtype, list(range(k)), out, rs.cuda_stream)
        qs.qs_probs_noalloc(ptr, a.req.n, self.dtype, [], out + 8 * (1 << k), rs.cuda_stream)
        with torch.cuda.stream(rs):
            self.result_host[slot, : (1 << k) + 1].copy_(self.result_dev[slot, : (1 << k) + 1], non_blocking=True)
        ev = torch.cuda.Event()
        ev.record(rs)
        self.reading.append((a, slot, ev, k))

    def _collect(self, clock, wait: bool = False):
        """Finish the reads whose results have reached the host (with wait,
        at least one)."""
        if wait and self.reading and not any(r[2].query() for r in self.reading):
            self.reading[0][2].synchronize()
        keep = []
        for entry in self.reading:
            a, slot, ev, k = entry
            if not ev.query():
                keep.append(entry)
                continue
            vals = self.result_host[slot, : (1 << k) + 1].numpy()
            a.req.probs = vals[: 1 << k].copy()
            a.req.norm = float(vals[1 << k])
            a.req.finished = clock()
            # the state's memory returns to the arena only after its reads
            qs.qs_set_stream(a.state.h, self.reaper.cuda_stream)
            a.state.close()
            self.arena.release(a.offset, self.footprint(a.req.n))
            self.used -= self.footprint(a.req.n)
            self.free_slots.append(slot)
            self.done.append(a.req)
        self.reading = keep

    def _complete(self, clock):
        for rid in [r for r, a in self.active.items() if a.pos >= a.n_chunks]:
            a = self.active.pop(rid)
            while not self.free_slots:
                self._collect(clock, wait=True)
            self._start_read(a, self.free_slots.pop())
        self._collect(clock)

    def run(self, clock=None, admit_until: Optional[float] = None) -> List[Request]:
        """Serve the submitted requests; arrivals are honoured against
        ``clock`` (seconds, default: wall time since this call).  With
        ``admit_until``, requests not admitted by then are dropped (left in
        ``self.dropped``) and the ones already admitted run to completion."""
        t0 = time.perf_counter()
        clock = clock or (lambda: time.perf_counter() - t0)
        self.dropped: List[Request] = []
        while self.pending or self.active or self.reading:
            now = clock()
            if admit_until is not None and now >= admit_until and self.pending:
                self.dropped.extend(r for _, _, r in self.pending)
                self.pending = []
            self._admit(now)
            if not self.active:
                if self.reading:
                    self._collect(clock, wait=not self.pending)
                if self.pending:
                    wait = self.pending[0][0] - clock()  # idle until the next arrival
                    if wait > 0:
                        time.sleep(min(wait, 0.001 if self.reading else 0.01))
                continue
            self._tick()
            self._complete(clock)
        self.torch.cuda.synchronize()
        return self.done


# ---------------------------------------------------------------------------
# Request streams shaped like the serving workload
# ---------------------------------------------------------------------------
def make_requests(count: int, seed: int, n_min: int = 12, n_max: int = 30, rate: float = 0.0,
                  grover_cap: int = 16, mix=(0.4, 0.3, 0.3)) -> List[Request]:
    """``count`` requests, qubit count log-uniform on [n_min, n_max]
    (n = round(2^U(log2 n_min, log2 n_max))), kinds 40% RQC depth 20 / 30%
    QFT of a random basis state / 30% Grover (iterations capped at
    ``grover_cap``); Poisson arrivals at ``rate`` per second (0: all at t=0)."""
    from workloads import circuits as W

    rng = W.rng_for(seed)
    reqs = []
    t = 0.0
    for i in range(count):
        u = rng.uniform(math.log2(n_min), math.log2(n_max))
        n = int(round(2.0 ** u))
        r = rng.random()
        if r < mix[0]:
            kind, gates = "rqc", W.rqc(n, 20, seed=seed * 100003 + i)
        elif r < mix[0] + mix[1]:
            x = int(rng.integers(1 << n))
            kind, gates = "qft", [W.X(q) for q in range(n) if (x >> q) & 1] + W.qft(list(range(n)))
            meta = {"x": x}
        else:
            marked = int(rng.integers(1 << n))
            iters = min(W.grover_iterations(n), grover_cap)
            kind, gates = "grover", W.grover(n, marked, iters)
            meta = {"marked": marked, "iterations": iters}
        if kind == "rqc":
            meta = {}
        if rate > 0:
            t += rng.exponential(1.0 / rate)
        reqs.append(Request(rid=i, n=n, gates=gates, arrival=t, kind=kind, meta=meta))
    return reqs


def summarize(done: List[Request], wall_s: float) -> dict:
    lat = np.array([r.latency for r in done]) if done else np.zeros(1)
    return {"requests": len(done), "wall_s": wall_s, "circuits_per_s": len(done) / wall_s if wall_s > 0 else 0.0,
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3)}
