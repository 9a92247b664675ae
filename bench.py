"""Benchmark: achieved HBM GB/s per gate on a 30-qubit complex128 state.

Workload (one step): a 30-qubit complex128 state (16 GiB) of normalised
i.i.d. complex Gaussian amplitudes; one Haar-random 2x2 gate on each target
0..29, then Haar-random 4x4 gates on 64 random distinct (t0, t1) pairs.  The
metric is algorithmic bytes (read + write of every amplitude a gate touches,
2 * 16 * 2^30 per gate) over the step's device time.

After the timed region the line gains (bounded in time):
  - the CPU leg: the oracle on a sample of the same gates, timed on every
    host core (OpenMP build) and on one core, and its result against the GPU's
    result of the same gates from the same input (sampled amplitudes);
  - per-kind GB/s of the structured, controlled, diagonal and permutation
    kernels on the same 30-qubit state;
  - the same sweep with FP64 arithmetic and on a complex64 state;
  - fused RQC-20 and QFT circuits on 32 qubits (complex128 and complex64):
    time, HBM passes, GB/s per pass, errors against closed forms and the
    complex64-vs-complex128 fidelity;
  - 4096 batched Grover / Shor-like states of 10..20 qubits (one compiled,
    graph-captured batch), with closed-form checks;
  - the serving loop on a stream of requests of 12..30 qubits (admission
    closed after a stated time), complex64 and complex128;
  - a 32-qubit complex128 state split over HBM and host memory: a gate on a
    local and on the global qubit.
A compact "summary" object closes the line.

Prints one JSON line.  --impl reference times the CPU oracle on a bounded
sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
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
# DRAM bytes (read + write) per launch of the dense kernels: one ncu capture at
# 26 qubits (both kernels as they are now), scaled to 30 qubits by the
# amplitude count (traffic grows in proportion).  Other variants: null.
NCU_TRAFFIC_30Q = {("k_dense1", "c128", "df"): (1.073801e9 + 1.012319e9) * 16,
                   ("k_dense2", "c128", "df"): (1.073799e9 + 1.012004e9) * 16}
NCU_TRAFFIC_NOTE = "ncu dram__bytes at 26 qubits x16 (scaled by amplitude count)"


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
                    help="skip every measurement taken after the timed region")
    ap.add_argument("--extras", default="kinds,variants,dense,circuits,batch,serve,split",
                    help="comma list of the extras to take after the timed region")
    ap.add_argument("--workload", default="sweep", choices=["sweep", "circuits", "batch", "serve", "dense"],
                    help="sweep: the default gate sweep; the others print one line each for the fused "
                         "RQC/QFT circuits, the batched small states, the serving loop and the dense "
                         "3..5-target gates (tensor cores vs CUDA cores, complex64, --n qubits)")
    ap.add_argument("--count", type=int, default=4096, help="batch: number of states")
    ap.add_argument("--nmin", type=int, default=10)
    ap.add_argument("--nmax", type=int, default=20)
    ap.add_argument("--requests", type=int, default=2000, help="serve: number of requests")
    ap.add_argument("--admit-s", type=float, default=0.0,
                    help="serve: close admission after this many seconds (0: serve every request)")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def cpu_count():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


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


class BusySampler:
    """GPU utilisation (nvidia-smi utilization.gpu, 100 ms samples) over a
    region: the fraction of time a kernel was running."""

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.vals = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=utilization.gpu", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            try:
                self.vals.append(float(line.strip()))
            except ValueError:
                pass

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        return {"mean_pct": statistics.mean(self.vals), "samples": len(self.vals)} if self.vals else None


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


def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _sample_indices(n, count, seed):
    rng = W.rng_for(seed)
    idx = rng.integers(0, 1 << n, size=count, dtype=np.uint64)
    edges = np.array([0, 1, (1 << n) - 1, 1 << (n - 1), (1 << (n - 1)) - 1], dtype=np.uint64)
    return np.unique(np.concatenate([idx, edges]))


# ---------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
def time_oracle(psi, gates, threads):
    """Apply gates one by one with the oracle on `threads` threads (the
    OpenMP build of the same source when > 1); returns (GB/s, seconds)."""
    import oracle as O

    O.build()
    used = O.set_threads(threads)
    n = int(psi.size).bit_length() - 1
    t0 = time.perf_counter()
    for g in gates:
        O.apply_gate(psi, g)
    secs = time.perf_counter() - t0
    O.set_threads(1)
    return len(gates) * gate_bytes(n, 16) / secs / 1e9, secs, used


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n = args.n
    gates = make_gates(n)
    psi = W.random_state(n, SEED_STATE)
    cores = cpu_count()
    # Each step: the next two gates of the sweep (one 1q, one 2q) on the full
    # state, on every host core.
    order = [gates[i % n] if j % 2 == 0 else gates[n + (i % N_PAIRS)] for i in range(64) for j in range(2)]
    cursor = 0

    def step():
        nonlocal cursor
        _, secs, used = time_oracle(psi, order[cursor:cursor + 2], cores)
        cursor += 2
        return secs, used

    for _ in range(args.warmup):
        step()
    secs_all, used = 0.0, cores
    for _ in range(args.steps):
        secs, used = step()
        secs_all += secs
    value = 2 * args.steps * gate_bytes(n, 16) / secs_all / 1e9
    sample = (f"{2 * args.steps} gates (alternating 1q and 2q from the sweep) on the full {n}-qubit state, "
              f"oracle gate loops on {used} threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs_all / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_qubits": n, "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_leg(qs, st, psi_host, gates, n):
    """The oracle on a bounded sample of the sweep: timed on every host core
    and on one core, and its result compared with the GPU's result of the
    same gates from the same input state (sampled amplitudes)."""
    import oracle as O

    cores = cpu_count()
    sample = [gates[0], gates[n], gates[n - 1], gates[n + 1]]  # 1q t=0, 2q, 1q t=29, 2q
    psi_cpu = psi_host.copy()
    gbs_all, secs_all, used = time_oracle(psi_cpu, sample, cores)
    psi_one = psi_host.copy()
    gbs_one, secs_one, _ = time_oracle(psi_one, sample[:1], 1)
    # the GPU applies the same four gates to the same input
    qs.qs_copy_in(st.h, psi_host)
    for g in sample:
        st.apply(g)
    idx = _sample_indices(n, 1 << 16, seed=13)
    got = st.gather(idx).astype(np.complex128)
    err = float(np.max(np.abs(got - psi_cpu[idx.astype(np.int64)])))
    del psi_one
    O.set_threads(1)
    return {"value": gbs_all, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"{len(sample)} gates of the sweep (1q t=0, 2q, 1q t={n - 1}, 2q) on the full {n}-qubit state, "
                      f"{secs_all:.1f} s on {used} threads (OpenMP build, bit-identical states)",
            "single_core": {"value": gbs_one, "unit": UNIT, "cores": 1,
                            "sample": f"1 gate (1q t=0) on the full state, {secs_one:.1f} s"},
            "gpu_vs_oracle_max_abs_err": err,
            "gpu_vs_oracle_sample": f"{idx.size} sampled amplitudes after the same 4 gates from the same input"}


# ---------------------------------------------------------------------------
# Extras: per-kind kernels, arithmetic / dtype variants
# ---------------------------------------------------------------------------
def per_kind_gates(n, rng):
    """(label, gate, algorithmic bytes as a multiple of 2 e 2^n) per kind,
    following the per-unit table of algorithmic bytes: a gate moves the
    amplitudes it changes (controls and patterns restrict them)."""
    U = W.haar_unitary(2, rng)
    U4 = W.haar_unitary(4, rng)
    lo, mid, hi = 1, n // 2, n - 1
    ph = np.exp(1j * rng.uniform(0, 2 * math.pi, size=8))
    ph3 = np.exp(1j * rng.uniform(0, 2 * math.pi, size=1 << 3))
    ph8 = np.exp(1j * rng.uniform(0, 2 * math.pi, size=1 << 8))
    p3 = np.roll(np.arange(8, dtype=np.uint32), 3)  # no fixed points
    p8 = np.roll(np.arange(256, dtype=np.uint32), 77)
    kinds = []
    for t in (lo, mid, hi):
        kinds += [(f"dense1_t{t}", W.g1(t, U), 1.0), (f"H_t{t}", W.H(t), 1.0), (f"X_t{t}", W.X(t), 1.0),
                  (f"Y_t{t}", W.Y(t), 1.0), (f"Z_t{t}", W.Z(t), 0.5), (f"T_t{t}", W.T(t), 0.5),
                  (f"phase_t{t}", W.g1(t, np.diag([1, ph[0]])), 0.5)]
    for (c, t) in ((0, hi), (hi, 2), (mid, mid + 1)):
        kinds += [(f"CNOT_c{c}_t{t}", W.CNOT(c, t), 0.5), (f"CZ_{c}_{t}", W.CZ(c, t), 0.25),
                  (f"SWAP_{c}_{t}", W.SWAP(c, t), 0.5), (f"ctrlU_c{c}_t{t}", W.g1(t, U, ctrls=(c,)), 0.5),
                  (f"dense2_{c}_{t}", W.gk((c, t), U4), 1.0)]
    kinds += [("ccU_c0,29_t15", W.g1(15, U, ctrls=(0, hi)), 0.25),
              ("diag1_t5", W.gdiag((5,), ph[:2]), 1.0), ("diag3_t2,17,28", W.gdiag((2, 17, 28), ph3), 1.0),
              ("diag8_low", W.gdiag(tuple(range(8)), ph8), 1.0),
              ("diag8_high", W.gdiag(tuple(range(n - 8, n)), ph8), 1.0),
              ("perm3_t0,9,27", W.gperm((0, 9, 27), p3), 1.0), ("perm8_low", W.gperm(tuple(range(8)), p8), 1.0),
              ("perm8_high", W.gperm(tuple(range(n - 8, n)), p8), 1.0),
              ("cperm8_c29", W.gperm(tuple(range(8, 16)), p8, ctrls=(hi,)), 0.5)]
    return kinds


def measure_per_kind(qs, torch, st, stream, n, amp_bytes, reps=3):
    """Device time of each kind's kernel (CUDA events on the state's stream,
    median of reps) on the resident state; GB/s from its algorithmic bytes."""
    rng = W.rng_for(2520)
    out = {}
    for label, g, frac in per_kind_gates(n, rng):
        st.apply(g)  # warm-up
        ts = []
        for _ in range(reps):
            a, b = _events(torch)
            a.record(stream)
            st.apply(g)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        ms = statistics.median(ts)
        out[label] = {"ms": round(ms, 4), "gbs": round(frac * gate_bytes(n, amp_bytes) / (ms * 1e-3) / 1e9, 1)}
    return out


def measure_sweep_variant(qs, torch, n, dtype_name, math_name, steps):
    """The sweep's gates on a fresh state of another dtype or arithmetic:
    device time per step and GB/s, per-kernel averages."""
    dt = qs.QS_C64 if dtype_name == "c64" else qs.QS_C128
    mm = qs.QS_MATH_FP64 if math_name == "fp64" else qs.QS_MATH_DF
    e = 8 if dtype_name == "c64" else 16
    gates = make_gates(n)
    st = qs.State(n, dt, mm)
    stream = torch.cuda.Stream()
    qs.qs_set_stream(st.h, stream.cuda_stream)
    qs.qs_init_basis(st.h, 0)
    for g in gates[:4]:
        st.apply(g)  # warm-up
    per = {}
    a, b = _events(torch)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(steps):
        for g in gates:
            e0, e1 = _events(torch)
            e0.record(stream)
            st.apply(g)
            e1.record(stream)
            per.setdefault(kernel_kind(g), []).append((e0, e1))
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    st.close()
    per_ms = {k: statistics.mean(x.elapsed_time(y) for x, y in v) for k, v in per.items()}
    return {"dtype": dtype_name, "math": math_name, "steps": steps, "ms_per_step": ms,
            "gbs": len(gates) * gate_bytes(n, e) / (ms * 1e-3) / 1e9,
            "per_kernel_gbs": {k: gate_bytes(n, e) / (v * 1e-3) / 1e9 for k, v in per_ms.items()}}


# ---------------------------------------------------------------------------
# Extras: fused circuits, batched states, serving
# ---------------------------------------------------------------------------
def qft_closed_form(n, x, ys):
    """QFT of basis state |x>: amplitude y is 2^(-n/2) exp(2 pi i x y / 2^n)."""
    ys = np.asarray(ys, dtype=np.int64)
    ph = ((int(x) * ys) % (1 << n)).astype(np.float64) * (2 * math.pi / (1 << n))
    return np.exp(1j * ph) * 2.0 ** (-n / 2)


def grover_closed_form_at(n, marked, r, idx):
    """Grover state after r iterations (circuit diffusion sign (-1)^r) at
    the indices idx: sin((2r+1) theta) on the marked item, cos((2r+1) theta)
    / sqrt(2^n - 1) elsewhere."""
    theta = math.asin(2.0 ** (-n / 2))
    s = -1.0 if r % 2 else 1.0
    idx = np.asarray(idx, dtype=np.int64)
    v = np.full(idx.size, s * math.cos((2 * r + 1) * theta) / math.sqrt((1 << n) - 1), dtype=np.complex128)
    v[idx == marked] = s * math.sin((2 * r + 1) * theta)
    return v


def fidelity_dev(torch, a, b):
    """|<b|a>|^2 / (|a|^2 |b|^2) in FP64 over two device tensors, chunk by chunk."""
    inner, na, nb = 0j, 0.0, 0.0
    chunk = 1 << 26
    for lo in range(0, a.numel(), chunk):
        xa = a[lo:lo + chunk].to(torch.complex128)
        xb = b[lo:lo + chunk].to(torch.complex128)
        inner += complex(torch.vdot(xb, xa).item())
        na += float(torch.vdot(xa, xa).real.item())
        nb += float(torch.vdot(xb, xb).real.item())
    return abs(inner) ** 2 / (na * nb)


def measure_circuits(qs, torch, n, fused_only=False):
    """RQC (20 layers of sqrt-X/Y/W + brick CZ) and QFT of a random basis
    state on n qubits, complex128 and complex64, fused (default block width),
    and gate by gate unless fused_only.  Device time per circuit (CUDA events),
    HBM passes (fused-block launches) and GB/s per pass; QFT against its
    closed form on sampled amplitudes; complex64 vs complex128 fidelity of
    each circuit's final state."""
    peak, _ = peaks()
    stream = torch.cuda.Stream()
    x = int(W.rng_for(2510).integers(1 << n))
    circuits = {"rqc20": W.rqc(n, 20, seed=2508), "qft": W.qft(list(range(n)))}
    start = {"rqc20": 0, "qft": x}
    out = {"n_qubits": n}
    idx = _sample_indices(n, 1 << 15, seed=14)
    for label, gates in circuits.items():
        c = qs.Circuit(gates)
        bufs = {}
        for dname, tdt, e in (("c128", torch.complex128, 16), ("c64", torch.complex64, 8)):
            buf = torch.zeros(1 << n, dtype=tdt, device="cuda")
            h = qs.qs_wrap(n, qs.QS_C128 if dname == "c128" else qs.QS_C64, buf.data_ptr(), stream.cuda_stream)
            res = {"gates": len(gates)}
            for mode, mf in (("per_gate", 1), ("fused", 0)):
                if fused_only and mode == "per_gate":
                    continue
                qs.qs_init_basis(h, start[label])
                qs.qs_fuse_run(h, c, qs.run_opts(mf))  # warm-up (kernel loading)
                qs.qs_init_basis(h, start[label])
                a, b = _events(torch)
                torch.cuda.synchronize()
                a.record(stream)
                qs.qs_fuse_run(h, c, qs.run_opts(mf))
                b.record(stream)
                torch.cuda.synchronize()
                ms = a.elapsed_time(b)
                res[f"{mode}_ms"] = ms
                if mode == "fused":
                    stats = qs.qs_last_run_stats(h)
                    passes = stats["fused_launches"]
                    res["fused_passes"] = passes
                    res["per_gate_launches"] = stats["gate_launches"]
                    if passes:
                        gbs = passes * 2 * e * (1 << n) / (ms * 1e-3) / 1e9
                        res["fused_gbs_per_pass"] = round(gbs, 1)
                        res["fused_frac_of_hbm"] = round(gbs / peak, 3)
            # the buffer now holds the fused run's result
            res["norm_err"] = abs(qs.qs_norm(h) - 1.0)
            if label == "qft":
                got = np.empty(idx.size, dtype=np.complex128 if dname == "c128" else np.complex64)
                qs.qs_gather(h, idx, got)
                res["max_err_vs_closed_form"] = float(np.max(np.abs(got.astype(np.complex128) -
                                                                    qft_closed_form(n, x, idx.astype(np.int64)))))
            qs.qs_destroy(h)
            bufs[dname] = buf
            out[f"{label}_{dname}"] = res
        out[f"{label}_c64_fidelity_vs_c128"] = fidelity_dev(torch, bufs["c64"], bufs["c128"])
        out[f"{label}_c64_speedup_vs_c128"] = out[f"{label}_c128"]["fused_ms"] / out[f"{label}_c64"]["fused_ms"]
        del bufs
        torch.cuda.empty_cache()
    return out


def shor_counting_distribution(t, a, N):
    """Closed form of the counting register's distribution (textbook state
    sum_x |x>|a^x mod N> followed by the inverse QFT)."""
    r = W.multiplicative_order(a, N)
    T = 1 << t
    y = np.arange(T, dtype=np.int64)
    P = np.zeros(T)
    for s in range(r):
        xs = np.arange(s, T, r, dtype=np.int64)
        ph = -2 * math.pi * ((np.outer(y, xs) % T).astype(np.float64)) / T
        P += np.abs(np.exp(1j * ph).sum(axis=1) / T) ** 2
    return P


def measure_batch(qs, torch, count, nmin, nmax, dtype_name="c128", seed=2512, checks=True, launches=2):
    """count states, qubit counts uniform in nmin..nmax, half Grover (random
    marked item, optimal iteration count), half Shor-like; compiled once
    (qs_batch_compile: host compile and graph capture, timed apart) and
    launched (qs_batch_launch, device time by CUDA events).  Reports
    circuits/s, gates/s and effective GB/s (every gate counted as one read
    and write of its state); Grover states against their closed form, a
    sample of Shor-like counting distributions against theirs."""
    rng = W.rng_for(seed)
    dt = qs.QS_C128 if dtype_name == "c128" else qs.QS_C64
    e = 16 if dtype_name == "c128" else 8
    ns = [int(v) for v in rng.integers(nmin, nmax + 1, size=count)]
    states, circuits, meta, n_gates, moved = [], [], [], 0, 0.0
    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    for i, n in enumerate(ns):
        if i % 2 == 0:
            marked = int(rng.integers(1 << n))
            # the H layer, then the iteration repeated (marshalled once)
            c = qs.Circuit.repeated([(W.grover(n, marked, 0), 1), (W.grover(n, marked, 1)[n:],
                                                                   W.grover_iterations(n))])
            meta.append(("grover", n, marked))
        else:
            gates, prm = W.shor_like(n, seed=seed * 7 + i)
            c = qs.Circuit(gates)
            meta.append(("shor", n, prm))
        st = qs.State(n, dt)
        qs.qs_set_stream(st.h, stream.cuda_stream)
        states.append(st)
        circuits.append(c)
        n_gates += c.n_gates
        moved += c.n_gates * 2.0 * e * (1 << n)
    gen_s = time.perf_counter() - t0
    handles = [s.h for s in states]
    t0 = time.perf_counter()
    b = qs.qs_batch_compile(handles, circuits)
    torch.cuda.synchronize()
    compile_s = time.perf_counter() - t0
    del circuits
    ts = []
    for rep in range(launches):
        for st in states:
            qs.qs_init_basis(st.h, 0)
        a, bb = _events(torch)
        torch.cuda.synchronize()
        a.record(stream)
        qs.qs_batch_launch(b)
        bb.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(bb))
    ms = min(ts)
    res = {"states": count, "dtype": dtype_name, "qubits": [nmin, nmax], "gates": n_gates, "ms": ms,
           "launch_ms": ts, "circuits_per_s": count / (ms * 1e-3), "gates_per_s": n_gates / (ms * 1e-3),
           "effective_gbs": moved / (ms * 1e-3) / 1e9, "host_generate_s": gen_s, "host_compile_and_capture_s":
           compile_s}
    if checks:
        g_err, g_fid, s_err, n_shor, n_grover = 0.0, 1.0, 0.0, 0, 0
        for i, (st, m) in enumerate(zip(states, meta)):
            if m[0] == "grover":
                if i % 8:  # every 4th Grover state
                    continue
                n_grover += 1
                _, n, marked = m
                got = st.read().astype(np.complex128)
                want = grover_closed_form_at(n, marked, W.grover_iterations(n), np.arange(1 << n))
                g_err = max(g_err, float(np.max(np.abs(got - want))))
                f = abs(np.vdot(got, want)) ** 2 / (np.vdot(got, got).real * np.vdot(want, want).real)
                g_fid = min(g_fid, f)
            elif n_shor < 32:
                _, n, prm = m
                p = st.probs(list(range(prm["t"])))
                p = p / p.sum()
                s_err = max(s_err, float(np.max(np.abs(p - shor_counting_distribution(prm["t"], prm["a"], prm["N"])))))
                n_shor += 1
        res["grover_max_abs_err_vs_closed_form"] = g_err
        res["grover_min_fidelity_vs_closed_form"] = g_fid
        res["shor_max_err_vs_closed_form"] = s_err
        res["shor_checked"] = n_shor
        res["grover_checked"] = n_grover
    qs.qs_batch_destroy(b)
    for st in states:
        st.close()
    torch.cuda.empty_cache()
    return res


def _served_closed_form_err(reqs):
    """Largest deviation of served marginals (8 lowest qubits) from their
    closed forms: QFT of a basis state is uniform; Grover from its state."""
    err = 0.0
    for r in reqs:
        k = len(r.probs)
        if r.kind == "qft":
            want = np.full(k, 1.0 / k)
        elif r.kind == "grover":
            marked = r.meta["marked"]
            iters = r.meta["iterations"]
            n = r.n
            theta = math.asin(2.0 ** (-n / 2))
            c2 = math.cos((2 * iters + 1) * theta) ** 2 / ((1 << n) - 1)
            want = np.full(k, c2 * (1 << n) / k)
            b = marked % k
            want[b] = math.sin((2 * iters + 1) * theta) ** 2 + c2 * ((1 << n) // k - 1)
        else:
            continue
        err = max(err, float(np.max(np.abs(r.probs - want))))
    return err


def measure_serving(qs, torch, requests, nmin, nmax, admit_s=0.0, seed=2513, fracs=(0.7, 1.0)):
    """Closed-loop capacity (all requests at t=0), then Poisson arrivals at
    fracs x that capacity; complex64 and complex128.  With admit_s > 0,
    admission closes after admit_s seconds of each run (requests not admitted
    by then are counted as dropped, admitted ones run to completion)."""
    from paper_2506_09198_gb300 import serving as S

    free = torch.cuda.mem_get_info()[0]
    out = {"requests": requests, "qubits": [nmin, nmax], "mix": "40% RQC-20 / 30% QFT / 30% Grover (r <= 16)",
           "admission_closes_after_s": admit_s or None}
    results = {}
    for dname, dt in (("c128", qs.QS_C128), ("c64", qs.QS_C64)):
        budget = min(1 << 37, 1 << (int(free * 0.6).bit_length() - 1))
        res = {}
        srv = S.Server(dt, hbm_budget_bytes=budget)
        for r in S.make_requests(requests, seed=seed, n_min=nmin, n_max=nmax, rate=0.0):
            srv.submit(r)
        busy = BusySampler(torch.cuda.current_device())
        busy.start()
        t0 = time.perf_counter()
        done = srv.run(admit_until=admit_s or None)
        cap = S.summarize(done, time.perf_counter() - t0)
        cap["gpu_busy"] = busy.stop()
        cap["dropped"] = len(srv.dropped)
        res["capacity"] = cap
        results[dname] = {r.rid: r for r in done}
        for frac in fracs:
            rate = frac * cap["circuits_per_s"]
            srv = S.Server(dt, hbm_budget_bytes=budget)
            for r in S.make_requests(requests, seed=seed, n_min=nmin, n_max=nmax, rate=rate):
                srv.submit(r)
            t0 = time.perf_counter()
            done = srv.run(admit_until=admit_s or None)
            summ = S.summarize(done, time.perf_counter() - t0)
            summ["arrival_rate"] = rate
            summ["dropped"] = len(srv.dropped)
            res[f"poisson_{frac}"] = summ
        res["max_err_vs_closed_form"] = _served_closed_form_err(results[dname].values())
        res["hbm_budget_bytes"] = budget
        out[dname] = res
        del srv
        torch.cuda.empty_cache()
    # the same requests served in both precisions: marginals side by side
    common = sorted(set(results["c128"]) & set(results["c64"]))
    if common:
        out["c64_vs_c128_max_marginal_diff"] = max(
            float(np.max(np.abs(results["c64"][i].probs / results["c64"][i].norm - results["c128"][i].probs)))
            for i in common)
    out["c64_vs_c128_capacity"] = out["c64"]["capacity"]["circuits_per_s"] / out["c128"]["capacity"]["circuits_per_s"]
    out["c64_vs_c128_state_fidelity"] = served_fidelity_sample(qs, torch, seed, nmin, nmax)
    return out


def served_fidelity_sample(qs, torch, seed, nmin, nmax, count=24, n_cap=24):
    """complex64 vs complex128 state fidelity of served circuits: the first
    `count` requests of the stream with at most n_cap qubits, each run alone
    through qs_fuse_run in both precisions (alone and in the serving mix give
    the same results)."""
    from paper_2506_09198_gb300 import serving as S

    worst = 1.0
    picked = [r for r in S.make_requests(400, seed=seed, n_min=nmin, n_max=nmax, rate=0.0) if r.n <= n_cap][:count]
    for r in picked:
        a = torch.zeros(1 << r.n, dtype=torch.complex128, device="cuda")
        b = torch.zeros(1 << r.n, dtype=torch.complex64, device="cuda")
        ha = qs.qs_wrap(r.n, qs.QS_C128, a.data_ptr(), 0)
        hb = qs.qs_wrap(r.n, qs.QS_C64, b.data_ptr(), 0)
        c = qs.Circuit(r.gates)
        for h in (ha, hb):
            qs.qs_init_basis(h, 0)
            qs.qs_fuse_run(h, c)
        qs.qs_sync(ha, 600)
        qs.qs_sync(hb, 600)
        worst = min(worst, fidelity_dev(torch, b, a))
        qs.qs_destroy(ha)
        qs.qs_destroy(hb)
    return {"min": worst, "requests": len(picked), "qubits_at_most": n_cap}


def measure_split(qs, torch, n=32, seed=2530):
    """A complex128 state of n qubits in two segments, one in HBM and one in
    pinned host memory (NVLink-C2C): device time of a dense gate on a local
    qubit and on the global qubit (which first swaps it in), algorithmic GB/s,
    and the norm after them (FP64 reduction over both segments)."""
    t0 = time.perf_counter()
    st = qs.State.split(n, qs.QS_C128, 1, 1)
    alloc_s = time.perf_counter() - t0
    stream = torch.cuda.Stream()
    qs.qs_set_stream(st.h, stream.cuda_stream)
    U = W.haar_unitary(2, W.rng_for(seed))
    qs.qs_apply_1q(st.h, 0, W.mat_h())  # a state with every amplitude in both segments
    res = {"n_qubits": n, "segments": "2 (1 in HBM, 1 in pinned host memory)", "alloc_s": alloc_s}
    for label, t in (("local_gate_q20", 20), ("global_gate_swap_in", n - 1), ("gate_on_swapped_qubit", n - 1)):
        a, b = _events(torch)
        torch.cuda.synchronize()
        a.record(stream)
        qs.qs_apply_1q(st.h, t, U)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        res[label] = {"ms": ms, "gbs": gate_bytes(n, 16) / (ms * 1e-3) / 1e9}
    res["norm_err"] = abs(st.norm() - 1.0)
    st.close()
    return res


def tf32_peak():
    """TF32 dense tensor peak: the measured bf16 burst figure times the nominal
    TF32 : bf16 ratio (1.1 : 2.25 PFLOP/s)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]) * 1.1 / 2.25, "measured bf16 x 1.1/2.25"
    except Exception:
        return 1900.0 * 1.1 / 2.25, "fallback bf16 x 1.1/2.25"


def measure_dense_k(qs, torch, psi_host, seed=2540):
    """Dense gates on k = 3, 4, 5 targets (low, high and scattered positions)
    of a seeded state (the benchmark's 30-qubit one: 8 GiB) in complex64: device time
    of one launch on the tensor cores (mode 2; k = 3 runs as I (x) U on a
    fourth target) and on the FP32 CUDA cores,
    algorithmic GB/s (one read and one write of the state), useful TFLOP/s
    (8 2^k real flops per amplitude) and, for the tensor cores, the pipe's
    TFLOP/s (three TF32 products: 24 2^k flops per amplitude).  Then sampled
    groups of a k = 5 tensor-core launch against U x in double for each
    32-amplitude group (sub-register order), as the ratio of the error to the
    FP32 bound (4 d + 8) 2^-24 sum_c |U_rc||x_c|."""
    n = int(psi_host.size).bit_length() - 1
    psi64 = psi_host.astype(np.complex64)
    dev = torch.from_numpy(psi64.view(np.float32)).cuda()
    stream = torch.cuda.current_stream()
    h = qs.qs_wrap(n, qs.QS_C64, dev.data_ptr(), stream.cuda_stream)
    rng = W.rng_for(seed)
    peak, peak_src = peaks()
    tpeak, tpeak_src = tf32_peak()
    res = {"n_qubits": n, "state": "c64", "launches": {}}
    best = None
    for k in (3, 4, 5):
        U = W.haar_unitary(1 << k, rng)
        for label, tg in (("low", list(range(k))), ("high", list(range(n - k, n))),
                          ("scattered", [0, 7, 15, 22, n - 1][:k])):
            for eng, flag in (("tc", 2), ("cuda_cores", 0)):
                qs.qs_set_tensor_cores(h, flag)
                qs.qs_apply_dense(h, [], tg, U)
                ts = []
                for _ in range(3):
                    a, b = _events(torch)
                    a.record(stream)
                    qs.qs_apply_dense(h, [], tg, U)
                    b.record(stream)
                    torch.cuda.synchronize()
                    ts.append(a.elapsed_time(b))
                ms = statistics.median(ts)
                gbs = 2 * 8 * 2 ** n / (ms * 1e-3) / 1e9
                v = {"ms": ms, "gbs": gbs, "tflops": 8 * 2 ** k * 2 ** n / (ms * 1e-3) / 1e12}
                if eng == "tc":
                    v["tensor_tflops"] = 24 * 2 ** k * 2 ** n / (ms * 1e-3) / 1e12
                    if k == 5 and (best is None or gbs > best[1]["gbs"]):
                        best = (label, v)
                res["launches"][f"k{k}_{label}_{eng}"] = v
    # Eight dense 3-target gates over one set of 5 qubits through qs_fuse_run:
    # composed into one 5-target matrix (one pass) against one pass per gate.
    qs.qs_set_tensor_cores(h, 2)
    five = [0, 7, 15, 22, n - 1]
    circ = qs.Circuit([W.gk([five[i] for i in rng.choice(5, size=3, replace=False)], W.haar_unitary(8, rng))
                       for _ in range(8)])
    blk = {}
    for label_b, mf in (("composed", 0), ("gate_by_gate", 1)):
        qs.qs_fuse_run(h, circ, qs.run_opts(max_fuse=mf))
        ts = []
        for _ in range(3):
            a, b = _events(torch)
            a.record(stream)
            qs.qs_fuse_run(h, circ, qs.run_opts(max_fuse=mf))
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        blk[label_b] = {"ms": statistics.median(ts), **qs.qs_last_run_stats(h)}
    res["dense_block_8_gates_3q_on_5_qubits"] = blk
    label, v = best
    res["roofline_tc_k5"] = {"bound": "hbm", "targets": label, "achieved": v["gbs"], "peak": peak, "unit": "GB/s",
                             "frac": v["gbs"] / peak, "peak_source": peak_src,
                             "tensor_tflops": v["tensor_tflops"], "tensor_peak_tflops": tpeak,
                             "tensor_frac": v["tensor_tflops"] / tpeak, "tensor_peak_source": tpeak_src}
    # Sampled parity of one k = 5 tensor-core launch from the seeded input.
    dev.copy_(torch.from_numpy(psi64.view(np.float32)))
    tg, cs = [n - 1, 3, 1, 18, 10], [0, n - 5]
    U = W.haar_unitary(32, rng)
    qs.qs_apply_dense(h, cs, tg, U)
    pos = sorted(tg + cs)
    groups = rng.integers(0, 1 << (n - 7), size=256)
    offs = [sum(1 << tg[j] for j in range(5) if (s >> j) & 1) for s in range(32)]
    idx = []
    for g in groups.tolist():
        b = g
        for p_ in pos:
            b = ((b >> p_) << (p_ + 1)) | (b & ((1 << p_) - 1))
        for c in cs:
            b |= 1 << c
        idx += [b | o for o in offs]
    idx = np.array(idx, dtype=np.uint64)
    out = np.empty(idx.size, dtype=np.complex64)
    qs.qs_gather(h, idx, out)
    xin = psi64[idx.astype(np.int64)].astype(np.complex128).reshape(-1, 32)
    got = out.astype(np.complex128).reshape(-1, 32)
    want = xin @ U.T
    bound = np.abs(xin) @ np.abs(U).T
    res["tc_k5_sampled_err_over_fp32_bound"] = float(np.max(np.abs(got - want) / ((4 * 32 + 8) * 2.0 ** -24 * bound)))
    res["tc_k5_sample"] = "256 groups of a 5-target, 2-control gate, each against U x in double on its 32 amplitudes"
    qs.qs_destroy(h)
    del dev
    torch.cuda.empty_cache()
    return res


def run_extra_workload(args):
    import torch

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    from paper_2506_09198_gb300 import build

    build.build()
    from paper_2506_09198_gb300 import qs

    if args.workload == "dense":
        res = measure_dense_k(qs, torch, W.random_state(args.n, SEED_STATE))
        line = {"metric": "dense 5-target gate on the tensor cores: HBM GB/s per launch vs peak",
                "value": res["roofline_tc_k5"]["achieved"], "unit": "GB/s", "higher_is_better": True,
                "config": {"workload": f"dense 3..5-target gates on a {args.n}-qubit complex64 state"},
                "detail": res}
    elif args.workload == "circuits":
        res = measure_circuits(qs, torch, args.n)
        line = {"metric": "fused circuits: RQC-20 and QFT device time, complex128 vs complex64",
                "value": res["rqc20_c64"]["fused_ms"], "unit": "ms", "higher_is_better": False,
                "config": {"workload": f"RQC-20 and QFT on {args.n} qubits"}, "detail": res}
    elif args.workload == "batch":
        res = [measure_batch(qs, torch, args.count, args.nmin, args.nmax, d) for d in ("c128", "c64")]
        line = {"metric": "batched states: circuits/s in one compiled, graph-captured batch",
                "value": res[0]["circuits_per_s"], "unit": "circuits/s", "higher_is_better": True,
                "config": {"workload": f"{args.count} states, {args.nmin}..{args.nmax} qubits, half Grover / half "
                                       f"Shor-like"}, "detail": res}
    else:
        res = measure_serving(qs, torch, args.requests, args.nmin, args.nmax, admit_s=args.admit_s)
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


def summarize_extras(ex, peak):
    """The key figures of the extras in a few hundred characters."""
    s = {}

    def r(x, d=0):
        return None if x is None else round(x, d)

    if "per_kind_30q_c128" in ex:
        pk = ex["per_kind_30q_c128"]
        groups = {}
        for label, v in pk.items():
            kind = label.split("_")[0]
            groups.setdefault(kind, []).append(v["gbs"])
        s["kind_gbs_30q_c128_min"] = {k: r(min(v)) for k, v in groups.items()}
    if "sweep_fp64" in ex:
        s["sweep_fp64_gbs"] = r(ex["sweep_fp64"]["gbs"])
    if "sweep_c64" in ex:
        s["sweep_c64_gbs"] = r(ex["sweep_c64"]["gbs"])
    c = ex.get("circuits_32q")
    if c:
        for lab in ("rqc20", "qft"):
            for d in ("c128", "c64"):
                v = c[f"{lab}_{d}"]
                s[f"{lab}_32q_{d}"] = {"ms": r(v["fused_ms"]), "passes": v.get("fused_passes"),
                                       "frac": v.get("fused_frac_of_hbm")}
            s[f"{lab}_32q_fid_c64"] = c.get(f"{lab}_c64_fidelity_vs_c128")
        s["qft_32q_err_c128"] = c["qft_c128"].get("max_err_vs_closed_form")
    for d in ("c128", "c64"):
        b = ex.get(f"batched_{d}")
        if b:
            s[f"batch4096_{d}"] = {"cps": r(b["circuits_per_s"]), "grover_err": b.get("grover_max_abs_err_vs_closed_form"),
                                   "shor_err": b.get("shor_max_err_vs_closed_form"),
                                   "compile_s": r(b["host_compile_and_capture_s"], 1)}
    sv = ex.get("serving")
    if sv:
        for d in ("c128", "c64"):
            cap = sv[d]["capacity"]
            p7 = sv[d].get("poisson_0.7", {})
            s[f"serve_{d}"] = {"cps": r(cap["circuits_per_s"], 1), "done": cap["requests"],
                               "p50_0.7": r(p7.get("p50_ms"), 1), "p99_0.7": r(p7.get("p99_ms"), 1),
                               "err": sv[d].get("max_err_vs_closed_form")}
        s["serve_fid_c64"] = sv.get("c64_vs_c128_state_fidelity", {}).get("min")
        s["serve_gpu_busy_pct"] = {d: (sv[d]["capacity"].get("gpu_busy") or {}).get("mean_pct") for d in ("c128", "c64")}
    dk = ex.get("dense_k_30q_c64")
    if dk:
        rf = dk["roofline_tc_k5"]
        s["dense_k5_30q_c64"] = {"tc_gbs": r(rf["achieved"]), "tc_frac": r(rf["frac"], 3),
                                 "tc_tensor_frac": r(rf["tensor_frac"], 3),
                                 "cuda_core_gbs": r(max(v["gbs"] for key, v in dk["launches"].items()
                                                        if key.startswith("k5_") and key.endswith("cuda_cores"))),
                                 "err_over_bound": r(dk["tc_k5_sampled_err_over_fp32_bound"], 3),
                                 "block_8x3q_ms": {k: r(v["ms"], 2) for k, v in
                                                   dk.get("dense_block_8_gates_3q_on_5_qubits", {}).items()}}
    sp = ex.get("split_32q_c128")
    if sp:
        s["split_32q_gbs"] = {"local": r(sp["local_gate_q20"]["gbs"]), "global": r(sp["global_gate_swap_in"]["gbs"])}
    return s


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
    # step's copies overlap the other's gates.  A step's gates wait for the
    # previous step's gates (an event), so the GPU computes one step at a time
    # while the copy engines move the other state; without that order the two
    # streams' kernels interleave and the copies overlap them by chance
    # (4.1-5.8 TB/s from run to run on one box).
    e2e = None
    if not args.no_e2e:
        st2 = qs.State(n, dt, math_mode)
        stream2 = torch.cuda.Stream()
        qs.qs_set_stream(st2.h, stream2.cuda_stream)
        host_out = [torch.empty(psi_host.nbytes, dtype=torch.uint8, pin_memory=True).numpy() for _ in range(2)]
        pairs = [(st, host_out[0], stream), (st2, host_out[1], stream2)]
        gates_done = [None]
        # The first copy-in and the last copy-out overlap nothing; 2K steps
        # (at most 10) amortise them the way a longer job would.
        e_steps = max(2, min(2 * args.steps, 10))

        def e2e_step(k):
            s_k, out_k, str_k = pairs[k % 2]
            qs.qs_copy_in(s_k.h, host_in)
            if k > 0:
                str_k.wait_event(gates_done[0])
            for g in gates:
                s_k.apply(g)
            gates_done[0] = torch.cuda.Event()
            gates_done[0].record(str_k)
            qs.qs_copy_out_async(s_k.h, out_k)

        # The run is repeated and the median reported, with every repetition.
        reps = []
        for _ in range(3):
            torch.cuda.synchronize()
            barrier()
            t0 = time.perf_counter()
            for k in range(e_steps):
                e2e_step(k)
            st.sync()
            st2.sync()
            torch.cuda.synchronize()
            el = max_over_ranks(time.perf_counter() - t0, world, device="cuda")
            reps.append(world * bytes_step * e_steps / el / 1e9)
        st2.close()
        del host_out, pairs
        e2e = {"value": statistics.median(reps), "unit": UNIT,
               "h2d_bytes_per_step": int(psi_host.nbytes), "d2h_bytes_per_step": int(psi_host.nbytes),
               "steps": e_steps, "repetitions": reps, "statistic": "median of 3 repetitions",
               "overlap": "two states on two streams alternate steps; a step's gates follow the previous step's"}

    extras = {}
    want = set() if args.no_extras else set(args.extras.split(","))
    if rank == 0 and "kinds" in want:
        extras[f"per_kind_{n}q_{args.dtype}"] = measure_per_kind(qs, torch, st, stream, n, amp_bytes)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu and not c64:
        cpu = cpu_leg(qs, st, psi_host, gates, n)

    st.close()
    del pinned
    if rank == 0:
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        if "variants" in want:
            extras["sweep_fp64"] = measure_sweep_variant(qs, torch, n, "c128", "fp64", 1)
            extras["sweep_c64"] = measure_sweep_variant(qs, torch, n, "c64", "df", 3)
        if "dense" in want and n == 30 and not c64:
            extras["dense_k_30q_c64"] = measure_dense_k(qs, torch, psi_host)
        if "circuits" in want:
            extras["circuits_32q"] = measure_circuits(qs, torch, 32, fused_only=True)
        if "batch" in want:
            extras["batched_c128"] = measure_batch(qs, torch, 4096, 10, 20, "c128", launches=1)
            extras["batched_c64"] = measure_batch(qs, torch, 4096, 10, 20, "c64", launches=1)
        if "serve" in want:
            extras["serving"] = measure_serving(qs, torch, 2000, 12, 30, admit_s=12.0, fracs=(0.7,))
        if "split" in want:
            extras["split_32q_c128"] = measure_split(qs, torch)
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
                             "traffic_source": NCU_TRAFFIC_NOTE,
                             "kernel": dom, "peak_source": peak_src},
                "per_kernel_ms": {k: statistics.mean(v) for k, v in per_kind.items()},
                "gbs_per_target_1q": per_target,
                "e2e": e2e, "cpu_baseline": cpu, "clocks": clk,
                "gpu_launches": len(gates) * args.steps,
                "extras": extras,
                "summary": summarize_extras(extras, peak)}
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
