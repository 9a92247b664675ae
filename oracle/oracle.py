"""Oracle: plain CPU complex128 state-vector simulator (Python wrapper).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this module.  It shares no code with
the GPU library and never imports it.

The arithmetic lives in ``qsim_oracle.c`` (plain loops over all 2^n indices,
double precision, no FMA contraction).  This wrapper only marshals numpy
arrays and walks a circuit gate by gate, never fusing: a fused block on the
GPU side is checked against the sequential application of its gates.

Conventions (arXiv 2506.09198, Sec. II-A and Algorithm 1): amplitude i is
``psi[i]`` (complex128, (re, im) adjacent); qubit q is bit q of i.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qsim_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
# Timing build of the same source with the gate loops split over OpenMP
# threads; every index's update is independent, so its states are bit-identical.
_LIB_OMP_PATH = os.path.join(_BUILD_DIR, "liboracle_omp.so")
_lock = threading.Lock()
_libs = {}
_threads = 1


def _gcc(out, extra):
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", *extra, "-fPIC", "-shared", "-o", tmp, _SRC])
    os.replace(tmp, out)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction): the single-thread
    parity build and the OpenMP timing build.  Returns the parity build's path."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    for path, extra in ((_LIB_PATH, []), (_LIB_OMP_PATH, ["-fopenmp"])):
        stale = (not os.path.exists(path)) or os.path.getmtime(path) < os.path.getmtime(_SRC)
        if force or stale:
            _gcc(path, extra)
    return _LIB_PATH


def set_threads(count: int) -> int:
    """Gate loops on ``count`` threads (the OpenMP build) or, with 1, the
    single-thread parity build (the default).  Returns the threads in use."""
    global _threads
    count = max(1, int(count))
    with _lock:
        _threads = count
    if count == 1:
        return 1
    return int(_load().oracle_set_threads(count))


def threads() -> int:
    return _threads


def _load():
    with _lock:
        omp = _threads > 1
        lib = _libs.get(omp)
        if lib is None:
            build()
            lib = ctypes.CDLL(_LIB_OMP_PATH if omp else _LIB_PATH)
            p_amp = ctypes.c_void_p
            p_i32 = ctypes.POINTER(ctypes.c_int)
            p_f64 = ctypes.POINTER(ctypes.c_double)
            p_u32 = ctypes.POINTER(ctypes.c_uint32)
            u64 = ctypes.c_uint64
            i32 = ctypes.c_int
            lib.oracle_apply_1q.argtypes = [p_amp, i32, u64, i32, p_f64]
            lib.oracle_apply_kq.argtypes = [p_amp, i32, u64, p_i32, i32, p_f64]
            lib.oracle_apply_diag.argtypes = [p_amp, i32, u64, p_i32, i32, p_f64]
            lib.oracle_apply_perm.argtypes = [p_amp, i32, u64, p_i32, i32, p_u32]
            lib.oracle_norm2.argtypes = [p_amp, i32]
            lib.oracle_norm2.restype = ctypes.c_double
            lib.oracle_probs.argtypes = [p_amp, i32, p_i32, i32, p_f64]
            lib.oracle_set_threads.argtypes = [i32]
            lib.oracle_set_threads.restype = i32
            for f in (lib.oracle_apply_1q, lib.oracle_apply_kq, lib.oracle_apply_diag,
                      lib.oracle_apply_perm, lib.oracle_probs):
                f.restype = None
            _libs[omp] = lib
            if omp:
                lib.oracle_set_threads(_threads)
        return lib


def _nqubits(psi: np.ndarray) -> int:
    if psi.dtype != np.complex128 or psi.ndim != 1 or not psi.flags.c_contiguous:
        raise ValueError("oracle states are contiguous 1-D complex128 arrays")
    n = int(psi.size).bit_length() - 1
    if psi.size != (1 << n):
        raise ValueError("state length must be a power of two")
    return n


def _ctrl_mask(ctrls) -> int:
    m = 0
    for c in ctrls:
        m |= 1 << int(c)
    return m


def _i32(xs):
    a = np.ascontiguousarray(np.asarray(xs, dtype=np.int32))
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _f64(m):
    a = np.ascontiguousarray(np.asarray(m, dtype=np.complex128)).view(np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check_qubits(n, targets, ctrls):
    qs = list(targets) + list(ctrls)
    if any(q < 0 or q >= n for q in qs) or len(set(qs)) != len(qs):
        raise ValueError(f"qubits {qs} must be distinct and in [0, {n})")


def apply_1q(psi, t, U, ctrls=()):
    """psi <- (controlled) single-qubit gate U on target t (Algorithm 1 pairing)."""
    n = _nqubits(psi)
    _check_qubits(n, [t], ctrls)
    u, pu = _f64(np.asarray(U).reshape(2, 2))
    _load().oracle_apply_1q(psi.ctypes.data, n, _ctrl_mask(ctrls), int(t), pu)
    return psi


def apply_kq(psi, targets, M, ctrls=()):
    """psi <- (controlled) dense 2^k x 2^k gate M; row/col index = sum_j b_targets[j] 2^j."""
    n = _nqubits(psi)
    _check_qubits(n, targets, ctrls)
    k = len(targets)
    t, pt = _i32(targets)
    m, pm = _f64(np.asarray(M).reshape(1 << k, 1 << k))
    _load().oracle_apply_kq(psi.ctypes.data, n, _ctrl_mask(ctrls), pt, k, pm)
    return psi


def apply_2q(psi, t0, t1, U, ctrls=()):
    """Two-qubit gate: the k = 2 case of ``apply_kq`` (index b_t0 + 2 b_t1)."""
    return apply_kq(psi, [t0, t1], U, ctrls)


def apply_diag(psi, targets, d, ctrls=()):
    """psi_i <- d[s(i)] psi_i, s(i) = sum_j b_targets[j](i) 2^j."""
    n = _nqubits(psi)
    _check_qubits(n, targets, ctrls)
    k = len(targets)
    t, pt = _i32(targets)
    dd, pd = _f64(np.asarray(d).reshape(1 << k))
    _load().oracle_apply_diag(psi.ctypes.data, n, _ctrl_mask(ctrls), pt, k, pd)
    return psi


def apply_perm(psi, targets, perm, ctrls=()):
    """|s> -> |perm[s]> on the target sub-register where all controls are 1."""
    n = _nqubits(psi)
    _check_qubits(n, targets, ctrls)
    k = len(targets)
    p = np.ascontiguousarray(np.asarray(perm, dtype=np.uint32))
    if p.size != (1 << k) or sorted(p.tolist()) != list(range(1 << k)):
        raise ValueError("perm must be a bijection of 0..2^k-1")
    t, pt = _i32(targets)
    _load().oracle_apply_perm(psi.ctypes.data, n, _ctrl_mask(ctrls), pt, k,
                              p.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    return psi


def norm2(psi) -> float:
    """Kahan-summed sum of |psi_i|^2 in double."""
    n = _nqubits(psi)
    return float(_load().oracle_norm2(psi.ctypes.data, n))


def probs(psi, qubits) -> np.ndarray:
    """Marginal probabilities of the sub-register on ``qubits`` (2^k entries)."""
    n = _nqubits(psi)
    _check_qubits(n, qubits, ())
    k = len(qubits)
    out = np.zeros(1 << k, dtype=np.float64)
    q, pq = _i32(qubits)
    _load().oracle_probs(psi.ctypes.data, n, pq, k,
                         out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def apply_gate(psi, g):
    """Apply one gate record (see ``workloads.circuits.Gate``)."""
    if g.kind == "u1":
        return apply_1q(psi, g.targets[0], g.data, g.ctrls)
    if g.kind == "uk":
        return apply_kq(psi, g.targets, g.data, g.ctrls)
    if g.kind == "diag":
        return apply_diag(psi, g.targets, g.data, g.ctrls)
    if g.kind == "perm":
        return apply_perm(psi, g.targets, g.data, g.ctrls)
    raise ValueError(f"unknown gate kind {g.kind!r}")


def run_circuit(psi, gates):
    """Apply ``gates`` one by one, in order, in place."""
    for g in gates:
        apply_gate(psi, g)
    return psi


def basis_state(n: int, x: int = 0) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[x] = 1.0
    return psi
