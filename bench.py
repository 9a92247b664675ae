"""Benchmark: achieved HBM GB/s per gate on a 30-qubit complex128 state.

Workload (one step): a 30-qubit complex128 state (16 GiB) of normalised
i.i.d. complex Gaussian amplitudes; one Haar-random 2x2 gate on each target
0..29, then Haar-random 4x4 gates on 64 random distinct (t0, t1) pairs.  The
metric is algorithmic bytes (read + write of every amplitude a gate touches,
2 * 16 * 2^30 per gate) over the step's device time.

Prints one JSON line.  --impl reference times the CPU oracle on a bounded
sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "HBM GB/s per gate (30q c128) vs peak; served circuits/s + p99, c64 vs c128"
UNIT = "GB/s"
N_QUBITS = 30
N_PAIRS = 64
SEED_STATE = 2507
SEED_GATES = 2507
WORKLOAD = "gate sweep, 30-qubit complex128 state (16 GiB): Haar 1q on targets 0..29 + Haar 2q on 64 random pairs"
# DRAM bytes (read + write) per launch from one ncu capture at 26 qubits, scaled
# to 30 qubits by the amplitude count (profiles/k_dense_df_26q_c128.md).  Valid
# for the float-float kernels as profiled; other variants report null.
NCU_TRAFFIC_30Q = {("k_dense1", "c128", "df"): (1.073801e9 + 1.012319e9) * 16,
                   ("k_dense2", "c128", "df"): (1.073799e9 + 1.012004e9) * 16}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--dtype", default="c128", choices=["c128", "c64"])
    ap.add_argument("--math", default="df", choices=["df", "fp64"])
    ap.add_argument("--n", type=int, default=N_QUBITS)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the fused-circuit, batched and serving measurements added to the line")
    ap.add_argument("--workload", default="sweep", choices=["sweep", "circuits", "batch", "serve"],
                    help="sweep: the default gate sweep; the others print one line each for the fused "
                         "RQC/QFT circuits, the batched small states and the serving loop")
    ap.add_argument("--count", type=int, default=4096, help="batch: number of states")
    ap.add_argument("--nmin", type=int, default=10)
    ap.add_argument("--nmax", type=int, default=20)
    ap.add_argument("--requests", type=int, default=400, help="serve: number of requests")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# Workload
# ---------------------------------------------------------------------------
def make_gates(n):
    g1s, g2s = W.gate_sweep(n, N_PAIRS, seed=SEED_GATES)
    return g1s + g2s


def gate_bytes(n, amp_bytes):
    return 2 * amp_bytes * (1 << n)


def kernel_kind(g):
    return "k_dense1" if g.kind == "u1" else "k_dense2"


# ---------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
def time_oracle_sample(psi, gates, budget_s):
    """Apply gates one by one with the oracle until budget_s has passed;
    return (GB/s over the gates done, gates done, seconds)."""
    import oracle as O

    O.build()
    n = int(psi.size).bit_length() - 1
    done, t_total, moved = 0, 0.0, 0
    for g in gates:
        t0 = time.perf_counter()
        O.apply_gate(psi, g)
        t_total += time.perf_counter() - t0
        moved += gate_bytes(n, 16)
        done += 1
        if t_total >= budget_s:
            break
    return moved / t_total / 1e9, done, t_total


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n = args.n
    gates = make_gates(n)
    psi = W.random_state(n, SEED_STATE)
    # Each step: the next two gates of the sweep (one 1q, one 2q) on the full
    # state, bounded to about 15 s of single-thread CPU work.
    order = [gates[i % n] if j % 2 == 0 else gates[n + (i % N_PAIRS)] for i in range(64) for j in range(2)]
    cursor = 0

    def step():
        nonlocal cursor
        gbs, done, secs = time_oracle_sample(psi, order[cursor:cursor + 2], budget_s=1e9)
        cursor += done
        return gbs, secs, done

    for _ in range(args.warmup):
        step()
    vals, secs_all, gates_done = [], 0.0, 0
    for _ in range(args.steps):
        gbs, secs, done = step()
        vals.append(gbs)
        secs_all += secs
        gates_done += done
    value = gates_done * gate_bytes(n, 16) / secs_all / 1e9
    sample = f"{gates_done} gates (alternating 1q and 2q from the sweep) on the full {n}-qubit state"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs_all / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_qubits": n, "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Fused circuits, batched states, serving
# ---------------------------------------------------------------------------
def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def measure_circuits(qs, torch, n, fused_only=False):
    """RQC (20 layers of sqrt-X/Y/W + brick CZ) and QFT of a random basis
    state on n qubits, complex128 and complex64, fused (default block size)
    and gate by gate.  Device time per circuit (CUDA events)."""
    stream = torch.cuda.Stream()
    x = int(W.rng_for(2510).integers(1 << n))
    circuits = {"rqc20": W.rqc(n, 20, seed=2508), "qft": [W.X(q) for q in range(n) if (x >> q) & 1] +
                W.qft(list(range(n)))}
    out = {"n_qubits": n}
    for dname, dt, e in (("c128", qs.QS_C128, 16), ("c64", qs.QS_C64, 8)):
        st = qs.State(n, dt)
        qs.qs_set_stream(st.h, stream.cuda_stream)
        for label, gates in circuits.items():
            c = qs.Circuit(gates)
            res = {"gates": len(gates)}
            for mode, mf in (("fused", 0), ("per_gate", 1)):
                if fused_only and mode == "per_gate":
                    continue
                qs.qs_init_basis(st.h, 0)
                st.run(c, max_fuse=mf)  # warm-up (kernel loading, plan caches)
                qs.qs_init_basis(st.h, 0)
                a, b = _events(torch)
                torch.cuda.synchronize()
                a.record(stream)
                st.run(c, max_fuse=mf)
                b.record(stream)
                torch.cuda.synchronize()
                ms = a.elapsed_time(b)
                res[f"{mode}_ms"] = ms
                res[f"{mode}_gate_equiv_gbs"] = len(gates) * 2 * e * (1 << n) / (ms * 1e-3) / 1e9
            res["norm"] = st.norm()
            out[f"{label}_{dname}"] = res
        st.close()
    for label in circuits:
        out[f"{label}_c64_speedup_vs_c128"] = out[f"{label}_c128"]["fused_ms"] / out[f"{label}_c64"]["fused_ms"]
    return out


def measure_batch(qs, torch, count, nmin, nmax, dtype_name="c128", seed=2512):
    """count states, qubit counts uniform in nmin..nmax, half Grover (random
    marked item, optimal iteration count), half Shor-like; one persistent
    graph-captured launch.  Reports circuits/s, gates/s and effective GB/s
    (every gate counted as one read and write of its state)."""
    rng = W.rng_for(seed)
    dt = qs.QS_C128 if dtype_name == "c128" else qs.QS_C64
    e = 16 if dtype_name == "c128" else 8
    ns = [int(v) for v in rng.integers(nmin, nmax + 1, size=count)]
    states, circuits, n_gates, moved = [], [], 0, 0.0
    stream = torch.cuda.Stream()
    for i, n in enumerate(ns):
        gates = W.grover(n, int(rng.integers(1 << n))) if i % 2 == 0 else W.shor_like(n, seed=seed * 7 + i)[0]
        st = qs.State(n, dt)
        qs.qs_set_stream(st.h, stream.cuda_stream)
        states.append(st)
        circuits.append(qs.Circuit(gates))
        n_gates += len(gates)
        moved += len(gates) * 2.0 * e * (1 << n)
    handles = [s.h for s in states]
    opts = qs.run_opts(use_graph=1)
    t0 = time.perf_counter()
    qs.qs_batch_run(handles, circuits, opts)  # compile + capture + first run
    torch.cuda.synchronize()
    compile_and_first_s = time.perf_counter() - t0
    for st in states:
        qs.qs_init_basis(st.h, 0)
    a, b = _events(torch)
    torch.cuda.synchronize()
    a.record(stream)
    qs.qs_batch_run(handles, circuits, opts)  # graph replay
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    for st in states:
        st.close()
    return {"states": count, "dtype": dtype_name, "qubits": [nmin, nmax], "gates": n_gates, "ms": ms,
            "circuits_per_s": count / (ms * 1e-3), "gates_per_s": n_gates / (ms * 1e-3),
            "effective_gbs": moved / (ms * 1e-3) / 1e9, "host_compile_and_first_run_s": compile_and_first_s}


def measure_serving(qs, torch, requests, nmin, nmax, seed=2513):
    """Closed-loop capacity (all requests at t=0), then Poisson arrivals at
    0.7x and 1.0x that capacity; complex64 and complex128."""
    from paper_2506_09198_gb300 import serving as S

    free = torch.cuda.mem_get_info()[0]
    out = {"requests": requests, "qubits": [nmin, nmax], "mix": "40% RQC-20 / 30% QFT / 30% Grover (r <= 16)"}
    for dname, dt in (("c128", qs.QS_C128), ("c64", qs.QS_C64)):
        budget = min(1 << 37, 1 << (int(free * 0.6).bit_length() - 1))
        res = {}
        srv = S.Server(dt, hbm_budget_bytes=budget)
        for r in S.make_requests(requests, seed=seed, n_min=nmin, n_max=nmax, rate=0.0):
            srv.submit(r)
        t0 = time.perf_counter()
        done = srv.run()
        cap = S.summarize(done, time.perf_counter() - t0)
        res["capacity"] = cap
        for frac in (0.7, 1.0):
            rate = frac * cap["circuits_per_s"]
            srv = S.Server(dt, hbm_budget_bytes=budget)
            for r in S.make_requests(requests, seed=seed, n_min=nmin, n_max=nmax, rate=rate):
                srv.submit(r)
            t0 = time.perf_counter()
            done = srv.run()
            summ = S.summarize(done, time.perf_counter() - t0)
            summ["arrival_rate"] = rate
            res[f"poisson_{frac}"] = summ
        res["hbm_budget_bytes"] = budget
        out[dname] = res
        del srv
        torch.cuda.empty_cache()
    out["c64_vs_c128_capacity"] = out["c64"]["capacity"]["circuits_per_s"] / out["c128"]["capacity"]["circuits_per_s"]
    return out


def run_extra_workload(args):
    import torch

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    from paper_2506_09198_gb300 import build

    build.build()
    from paper_2506_09198_gb300 import qs

    if args.workload == "circuits":
        res = measure_circuits(qs, torch, args.n)
        line = {"metric": "fused circuits: RQC-20 and QFT device time, complex128 vs complex64",
                "value": res["rqc20_c64"]["fused_ms"], "unit": "ms", "higher_is_better": False,
                "config": {"workload": f"RQC-20 and QFT on {args.n} qubits"}, "detail": res}
    elif args.workload == "batch":
        res = [measure_batch(qs, torch, args.count, args.nmin, args.nmax, d) for d in ("c128", "c64")]
        line = {"metric": "batched states: circuits/s in one persistent graph-captured launch",
                "value": res[0]["circuits_per_s"], "unit": "circuits/s", "higher_is_better": True,
                "config": {"workload": f"{args.count} states, {args.nmin}..{args.nmax} qubits, half Grover / half "
                                       f"Shor-like"}, "detail": res}
    else:
        res = measure_serving(qs, torch, args.requests, args.nmin, args.nmax)
        line = {"metric": "served circuits/s and p99 latency, complex64 vs complex128",
                "value": res["c128"]["capacity"]["circuits_per_s"], "unit": "circuits/s", "higher_is_better": True,
                "config": {"workload": f"{args.requests} requests, {args.nmin}..{args.nmax} qubits log-uniform"},
                "detail": res}
    line["data"] = "synthetic"
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Multi-rank aggregation (replicas: each rank simulates its own state)
# ---------------------------------------------------------------------------
def max_over_ranks(ms: float, world: int, device=None) -> float:
    """The slowest rank's time: every rank gets the maximum of all ranks'."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(bytes_per_step: float, steps: int, ms: float, world: int) -> float:
    """Whole-job GB/s: the units all ranks processed over the slowest rank's time."""
    return world * bytes_per_step * steps / (ms * 1e-3) / 1e9


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    from paper_2506_09198_gb300 import build

    build.build()
    from paper_2506_09198_gb300 import qs

    n = args.n
    c64 = args.dtype == "c64"
    amp_bytes = 8 if c64 else 16
    dt = qs.QS_C64 if c64 else qs.QS_C128
    math_mode = qs.QS_MATH_FP64 if args.math == "fp64" else qs.QS_MATH_DF
    gates = make_gates(n)
    psi_host = W.random_state(n, SEED_STATE + rank)
    if c64:
        psi_host = psi_host.astype(np.complex64)
    # pinned host copy for the end-to-end measurement
    pinned = torch.empty(psi_host.nbytes, dtype=torch.uint8, pin_memory=True)
    pinned.numpy()[:] = psi_host.view(np.uint8)

    stream = torch.cuda.Stream()
    st = qs.State(n, dt, math_mode)
    qs.qs_set_stream(st.h, stream.cuda_stream)
    host_in = pinned.numpy()
    qs.qs_copy_in(st.h, host_in)
    st.sync()

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    def one_step(events=None):
        for i, g in enumerate(gates):
            if events is not None:
                events[i][0].record(stream)
            st.apply(g)
            if events is not None:
                events[i][1].record(stream)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    barrier()

    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in gates]
          for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    t_start.record(stream)
    for s in range(args.steps):
        one_step(ev[s])
    t_end.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier()
    ms = max_over_ranks(t_start.elapsed_time(t_end), world, device="cuda")
    bytes_step = len(gates) * gate_bytes(n, amp_bytes)
    value = job_throughput(bytes_step, args.steps, ms, world)

    # Per-kernel averages over the timed region.
    per_kind = {}
    for s in range(args.steps):
        for i, g in enumerate(gates):
            d = ev[s][i][0].elapsed_time(ev[s][i][1])
            per_kind.setdefault(kernel_kind(g), []).append(d)
    tot = {k: sum(v) for k, v in per_kind.items()}
    dom = max(tot, key=tot.get)
    dom_ms = statistics.mean(per_kind[dom])
    achieved = gate_bytes(n, amp_bytes) / (dom_ms * 1e-3) / 1e9
    peak, peak_src = peaks()
    per_target = []
    for i, g in enumerate(gates[:n]):
        d = statistics.median(ev[s][i][0].elapsed_time(ev[s][i][1]) for s in range(args.steps))
        per_target.append(round(gate_bytes(n, amp_bytes) / (d * 1e-3) / 1e9, 1))

    # End-to-end through the C ABI with host buffers: every step copies its
    # input state in from pinned host memory, runs the step's gates and copies
    # the resulting state back out, all inside the timed region.  Steps are
    # independent, so two device states on two streams alternate and one
    # step's copies overlap the other's gates (the host link carries about
    # 0.2 TB/s each way on this machine).
    e2e = None
    if not args.no_e2e:
        st2 = qs.State(n, dt, math_mode)
        stream2 = torch.cuda.Stream()
        qs.qs_set_stream(st2.h, stream2.cuda_stream)
        host_out = [torch.empty(psi_host.nbytes, dtype=torch.uint8, pin_memory=True).numpy() for _ in range(2)]
        pairs = [(st, host_out[0]), (st2, host_out[1])]
        # The first copy-in and the last copy-out overlap nothing; 2K steps
        # (at most 10) amortise them the way a longer job would.
        e_steps = max(2, min(2 * args.steps, 10))

        def e2e_step(k):
            s_k, out_k = pairs[k % 2]
            qs.qs_copy_in(s_k.h, host_in)
            for g in gates:
                s_k.apply(g)
            qs.qs_copy_out_async(s_k.h, out_k)

        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for k in range(e_steps):
            e2e_step(k)
        st.sync()
        st2.sync()
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        st2.close()
        e2e = {"value": world * bytes_step * e_steps / el / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": int(psi_host.nbytes), "d2h_bytes_per_step": int(psi_host.nbytes),
               "steps": e_steps, "overlap": "two states on two streams alternate steps"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu and not c64:
        gbs, done, secs = time_oracle_sample(psi_host.copy() if c64 else psi_host, [gates[0], gates[n]], 1e9)
        cpu = {"value": gbs, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{done} gates (first 1q, first 2q of the sweep) on the full {n}-qubit state, "
                         f"{secs:.1f} s single-thread"}

    st.close()
    del pinned
    extras = None
    if rank == 0 and not args.no_extras:
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        extras = {
            "fused_circuits": measure_circuits(qs, torch, 28),
            "batched": measure_batch(qs, torch, 512, 10, 16, "c128"),
            "batched_c64": measure_batch(qs, torch, 512, 10, 16, "c64"),
            "serving": measure_serving(qs, torch, 120, 12, 24),
        }
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": {"c128": {"df": "f64 storage, float-float arithmetic", "fp64": "f64"}[args.math],
                          "c64": "f32"}[args.dtype],
                "data": "synthetic",
                "config": {"workload": WORKLOAD if n == N_QUBITS else WORKLOAD.replace("30-qubit", f"{n}-qubit"),
                           "n_qubits": n, "state": args.dtype, "math": args.math,
                           "gates_per_step": len(gates), "parallelism": f"replicas x{world}",
                           "l2": "inputs larger than L2 (16 GiB state, 129 MB L2)"},
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak,
                             "traffic": NCU_TRAFFIC_30Q.get((dom, args.dtype, args.math)) if n == 30 else None,
                             "kernel": dom, "peak_source": peak_src},
                "per_kernel_ms": {k: statistics.mean(v) for k, v in per_kind.items()},
                "gbs_per_target_1q": per_target,
                "e2e": e2e, "cpu_baseline": cpu, "clocks": clk,
                "gpu_launches": len(gates) * args.steps,
                "extras": extras}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload != "sweep":
        run_extra_workload(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
