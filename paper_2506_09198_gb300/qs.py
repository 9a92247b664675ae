"""Python binding of libqs: the C ABI of include/qs.h through ctypes.

Argument marshalling only — every step of a gate application runs in the
library's CUDA kernels.  Functions keep the C names (qs_create, qs_apply_1q,
...) and raise ``QSError`` on a non-zero status.  PyTorch is used by callers
only for device memory and streams (``qs_wrap`` takes a tensor's pointer).

If the shared library has not been built, importing this module raises
ImportError: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libqs.so")

QS_OK, QS_ERR_ARG, QS_ERR_OOM, QS_ERR_CUDA, QS_ERR_TIMEOUT, QS_ERR_UNSUPPORTED, QS_ERR_DEVICE = range(7)
QS_C64, QS_C128 = 0, 1
QS_MATH_DF, QS_MATH_FP64 = 0, 1
QS_MAX_QUBITS, QS_MAX_TARGETS, QS_MAX_DENSE = 40, 8, 5
QS_GATE_U1, QS_GATE_UK, QS_GATE_DIAG, QS_GATE_PERM = 0, 1, 2, 3
STATUS_NAMES = {0: "QS_OK", 1: "QS_ERR_ARG", 2: "QS_ERR_OOM", 3: "QS_ERR_CUDA", 4: "QS_ERR_TIMEOUT",
                5: "QS_ERR_UNSUPPORTED", 6: "QS_ERR_DEVICE"}


class QSError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class qs_gate(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("k", ctypes.c_int32), ("targets", ctypes.c_int32 * QS_MAX_TARGETS),
                ("ctrl_mask", ctypes.c_uint64), ("offset", ctypes.c_int64)]


class qs_circuit(ctypes.Structure):
    _fields_ = [("n_gates", ctypes.c_int64), ("gates", ctypes.POINTER(qs_gate)),
                ("data", ctypes.POINTER(ctypes.c_double)), ("perm", ctypes.POINTER(ctypes.c_uint32))]


class qs_run_stats(ctypes.Structure):
    _fields_ = [("fused_launches", ctypes.c_int64), ("gate_launches", ctypes.c_int64),
                ("dense_blocks", ctypes.c_int64), ("dense_gates", ctypes.c_int64),
                ("reserved", ctypes.c_int64 * 4)]


class qs_run_opts(ctypes.Structure):
    _fields_ = [("max_fuse", ctypes.c_int32), ("use_graph", ctypes.c_int32), ("reserved", ctypes.c_int32 * 6)]


if not os.path.exists(LIB_PATH):
    raise ImportError(f"libqs is not built ({LIB_PATH} missing): run __graft_entry__.build() first")

_lib = ctypes.CDLL(LIB_PATH)
_P = ctypes.c_void_p
_I = ctypes.c_int
_PI = ctypes.POINTER(ctypes.c_int)
_PD = ctypes.POINTER(ctypes.c_double)
_PU32 = ctypes.POINTER(ctypes.c_uint32)
_PU64 = ctypes.POINTER(ctypes.c_uint64)
_SIGS = {
    "qs_create": [_I, _I, ctypes.POINTER(_P)],
    "qs_wrap": [_I, _I, _P, _P, ctypes.POINTER(_P)],
    "qs_destroy": [_P],
    "qs_set_stream": [_P, _P],
    "qs_set_math": [_P, _I],
    "qs_num_qubits": [_P, _PI],
    "qs_device_ptr": [_P, ctypes.POINTER(_P)],
    "qs_init_basis": [_P, ctypes.c_uint64],
    "qs_copy_in": [_P, _P],
    "qs_copy_out": [_P, _P],
    "qs_copy_out_async": [_P, _P],
    "qs_gather": [_P, _PU64, ctypes.c_int64, _P],
    "qs_apply_1q": [_P, _I, _PD],
    "qs_apply_2q": [_P, _I, _I, _PD],
    "qs_apply_ctrl": [_P, _PI, _I, _I, _PD],
    "qs_apply_diag": [_P, _PI, _I, _PD],
    "qs_apply_dense": [_P, _PI, _I, _PI, _I, _PD],
    "qs_set_tensor_cores": [_P, _I],
    "qs_apply_perm": [_P, _PI, _I, _PI, _I, _PU32],
    "qs_fuse_run": [_P, ctypes.POINTER(qs_circuit), ctypes.POINTER(qs_run_opts)],
    "qs_batch_run": [ctypes.POINTER(_P), ctypes.POINTER(ctypes.POINTER(qs_circuit)), _I, ctypes.POINTER(qs_run_opts)],
    "qs_norm": [_P, _PD],
    "qs_probs": [_P, _PI, _I, _PD],
    "qs_sync": [_P, ctypes.c_double],
    "qs_probs_noalloc": [_P, _I, _I, _PI, _I, _P, _P],
    "qs_autotune": [_P, ctypes.POINTER(qs_circuit), _PI, _PD],
    "qs_batch_compile": [ctypes.POINTER(_P), ctypes.POINTER(ctypes.POINTER(qs_circuit)), _I, ctypes.POINTER(_P)],
    "qs_batch_launch": [_P],
    "qs_batch_destroy": [_P],
    "qs_set_wait_limit": [ctypes.c_double],
    "qs_last_run_stats": [_P, ctypes.POINTER(qs_run_stats)],
    "qs_create_split": [_I, _I, _I, _I, ctypes.POINTER(_P)],
}
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = ctypes.c_int
_lib.qs_last_error.restype = ctypes.c_char_p
_lib.qs_version.restype = ctypes.c_char_p

EXPORTED = sorted(list(_SIGS) + ["qs_last_error", "qs_version"])


def lib():
    return _lib


def _check(st: int):
    if st != QS_OK:
        raise QSError(st, _lib.qs_last_error().decode(errors="replace"))


def _i32(xs):
    a = np.ascontiguousarray(np.asarray(list(xs), dtype=np.int32))
    return a, (a.ctypes.data_as(_PI) if a.size else None)


def _c128_flat(m, size):
    a = np.ascontiguousarray(np.asarray(m, dtype=np.complex128).reshape(-1))
    if a.size != size:
        raise ValueError(f"expected {size} complex entries, got {a.size}")
    f = a.view(np.float64)
    return f, f.ctypes.data_as(_PD)


def qs_last_error() -> str:
    return _lib.qs_last_error().decode(errors="replace")


def qs_version() -> str:
    return _lib.qs_version().decode()


def qs_create(n: int, dtype: int):
    h = _P()
    _check(_lib.qs_create(n, dtype, ctypes.byref(h)))
    return h


def qs_create_split(n: int, dtype: int, g: int, hbm_segments: int):
    """A state of n qubits in 2^g segments, the first hbm_segments in device
    memory and the rest in pinned host memory."""
    h = _P()
    _check(_lib.qs_create_split(n, dtype, g, hbm_segments, ctypes.byref(h)))
    return h


def qs_wrap(n: int, dtype: int, device_ptr: int, stream: int = 0):
    h = _P()
    _check(_lib.qs_wrap(n, dtype, _P(device_ptr), _P(stream or None), ctypes.byref(h)))
    return h


def qs_destroy(h):
    _check(_lib.qs_destroy(h))


def qs_set_stream(h, stream: int):
    _check(_lib.qs_set_stream(h, _P(stream or None)))


def qs_set_math(h, math: int):
    _check(_lib.qs_set_math(h, math))


def qs_num_qubits(h) -> int:
    n = ctypes.c_int()
    _check(_lib.qs_num_qubits(h, ctypes.byref(n)))
    return n.value


def qs_device_ptr(h) -> int:
    p = _P()
    _check(_lib.qs_device_ptr(h, ctypes.byref(p)))
    return p.value


def qs_init_basis(h, idx: int):
    _check(_lib.qs_init_basis(h, ctypes.c_uint64(idx)))


def qs_copy_in(h, host: np.ndarray):
    if not host.flags.c_contiguous:
        raise ValueError("host buffer must be contiguous")
    _check(_lib.qs_copy_in(h, _P(host.ctypes.data)))


def qs_copy_out(h, host: np.ndarray):
    if not host.flags.c_contiguous or not host.flags.writeable:
        raise ValueError("host buffer must be contiguous and writeable")
    _check(_lib.qs_copy_out(h, _P(host.ctypes.data)))
    return host


def qs_copy_out_async(h, host: np.ndarray):
    if not host.flags.c_contiguous or not host.flags.writeable:
        raise ValueError("host buffer must be contiguous and writeable")
    _check(_lib.qs_copy_out_async(h, _P(host.ctypes.data)))
    return host


def qs_gather(h, idx, out: np.ndarray):
    i = np.ascontiguousarray(np.asarray(idx, dtype=np.uint64))
    _check(_lib.qs_gather(h, i.ctypes.data_as(_PU64), i.size, _P(out.ctypes.data)))
    return out


def qs_apply_1q(h, target: int, U):
    f, p = _c128_flat(U, 4)
    _check(_lib.qs_apply_1q(h, target, p))


def qs_apply_2q(h, t0: int, t1: int, U):
    f, p = _c128_flat(U, 16)
    _check(_lib.qs_apply_2q(h, t0, t1, p))


def qs_apply_ctrl(h, ctrls, target: int, U):
    c, pc = _i32(ctrls)
    f, p = _c128_flat(U, 4)
    _check(_lib.qs_apply_ctrl(h, pc, c.size, target, p))


def qs_apply_dense(h, ctrls, targets, U):
    c, pc = _i32(ctrls)
    t, pt = _i32(targets)
    f, p = _c128_flat(U, 1 << (2 * t.size))
    _check(_lib.qs_apply_dense(h, pc, c.size, pt, t.size, p))


def qs_set_tensor_cores(h, mode: int):
    _check(_lib.qs_set_tensor_cores(h, int(mode)))


def qs_apply_diag(h, targets, d):
    t, pt = _i32(targets)
    f, p = _c128_flat(d, 1 << t.size)
    _check(_lib.qs_apply_diag(h, pt, t.size, p))


def qs_apply_perm(h, ctrls, targets, perm):
    c, pc = _i32(ctrls)
    t, pt = _i32(targets)
    pm = np.ascontiguousarray(np.asarray(perm, dtype=np.uint32))
    _check(_lib.qs_apply_perm(h, pc, c.size, pt, t.size, pm.ctypes.data_as(_PU32)))


def qs_norm(h) -> float:
    out = ctypes.c_double()
    _check(_lib.qs_norm(h, ctypes.byref(out)))
    return out.value


def qs_probs(h, qubits) -> np.ndarray:
    q, pq = _i32(qubits)
    out = np.zeros(1 << q.size, dtype=np.float64)
    _check(_lib.qs_probs(h, pq, q.size, out.ctypes.data_as(_PD)))
    return out


def qs_probs_noalloc(device_state: int, n: int, dtype: int, qubits, device_out: int, stream: int = 0):
    """No-allocation marginals (k = len(qubits), 0 for the norm) into 2^k
    doubles of device memory at device_out, asynchronous on stream."""
    q, pq = _i32(qubits)
    _check(_lib.qs_probs_noalloc(_P(device_state), n, dtype, pq, q.size, _P(device_out), _P(stream or None)))


def qs_sync(h, timeout_s: float = 60.0):
    _check(_lib.qs_sync(h, float(timeout_s)))


# ---------------------------------------------------------------------------
# Circuit marshalling
# ---------------------------------------------------------------------------
_KIND = {"u1": QS_GATE_U1, "uk": QS_GATE_UK, "diag": QS_GATE_DIAG, "perm": QS_GATE_PERM}


class Circuit:
    """Flat qs_circuit built from gate records (objects with kind, targets,
    ctrls and data attributes).  Keeps its arrays alive."""

    def __init__(self, gates):
        gates = list(gates)
        self.gates = (qs_gate * max(1, len(gates)))()
        data, perm = [], []
        nd = npm = 0
        for i, g in enumerate(gates):
            rec = self.gates[i]
            rec.kind = _KIND[g.kind]
            rec.k = len(g.targets)
            for j, t in enumerate(g.targets):
                rec.targets[j] = int(t)
            mask = 0
            for c in g.ctrls:
                mask |= 1 << int(c)
            rec.ctrl_mask = mask
            if g.kind == "perm":
                arr = np.asarray(g.data, dtype=np.uint32).reshape(-1)
                rec.offset = npm
                perm.append(arr)
                npm += arr.size
            else:
                arr = np.asarray(g.data, dtype=np.complex128).reshape(-1).view(np.float64)
                rec.offset = nd
                data.append(arr)
                nd += arr.size
        self.data = np.ascontiguousarray(np.concatenate(data) if data else np.zeros(2))
        self.perm = np.ascontiguousarray(np.concatenate(perm) if perm else np.zeros(1, dtype=np.uint32))
        self.c = qs_circuit(len(gates), self.gates, self.data.ctypes.data_as(_PD), self.perm.ctypes.data_as(_PU32))
        self.n_gates = len(gates)

    @property
    def ptr(self):
        return ctypes.pointer(self.c)

    @classmethod
    def repeated(cls, parts) -> "Circuit":
        """A circuit made of parts [(gates, count), ...]: each part's gates
        repeated count times, in order (Grover iterations, Trotter steps).
        Each part is marshalled once and its records are tiled; every copy
        refers to the same matrices and tables in the pools."""
        subs = [(cls(list(g)), int(cnt)) for g, cnt in parts if cnt > 0 and len(g) > 0]
        self = cls.__new__(cls)
        rec_size = ctypes.sizeof(qs_gate)
        chunks, data, perm = [], [], []
        nd = npm = 0
        for c, cnt in subs:
            raw = np.frombuffer(ctypes.string_at(ctypes.addressof(c.gates), c.n_gates * rec_size), dtype=np.uint8)
            recs = raw.reshape(c.n_gates, rec_size).copy()
            off = recs[:, 48:56].copy().view(np.int64).reshape(-1)
            kind = recs[:, 0:4].copy().view(np.int32).reshape(-1)
            off = np.where(kind == QS_GATE_PERM, off + npm, off + nd)
            recs[:, 48:56] = off.astype(np.int64).view(np.uint8).reshape(-1, 8)
            chunks.append(np.tile(recs, (cnt, 1)))
            data.append(c.data)
            perm.append(c.perm)
            nd += c.data.size
            npm += c.perm.size
        allrec = np.ascontiguousarray(np.concatenate(chunks) if chunks else np.zeros((1, rec_size), np.uint8))
        n = int(sum(c.n_gates * cnt for c, cnt in subs))
        self._rec_buf = allrec
        self.gates = (qs_gate * max(1, n)).from_buffer(allrec)
        self.data = np.ascontiguousarray(np.concatenate(data) if data else np.zeros(2))
        self.perm = np.ascontiguousarray(np.concatenate(perm) if perm else np.zeros(1, dtype=np.uint32))
        self.c = qs_circuit(n, self.gates, self.data.ctypes.data_as(_PD), self.perm.ctypes.data_as(_PU32))
        self.n_gates = n
        return self

    def slice(self, first: int, count: int) -> "CircuitSlice":
        """Gates first .. first + count - 1 as a circuit of their own: the
        records and pools are shared (record offsets index the same pools),
        so nothing is marshalled again."""
        first = max(0, min(int(first), self.n_gates))
        count = max(0, min(int(count), self.n_gates - first))
        return CircuitSlice(self, first, count)


class CircuitSlice:
    """A gate range of a Circuit (keeps the parent alive)."""

    def __init__(self, parent: Circuit, first: int, count: int):
        self.parent = parent
        rec = ctypes.cast(ctypes.byref(parent.gates, first * ctypes.sizeof(qs_gate)), ctypes.POINTER(qs_gate))
        self.c = qs_circuit(count, rec, parent.c.data, parent.c.perm)
        self.n_gates = count

    @property
    def ptr(self):
        return ctypes.pointer(self.c)


def run_opts(max_fuse: int = 0, use_graph: int = 0):
    return qs_run_opts(max_fuse, use_graph)


def qs_fuse_run(h, circuit: Circuit, opts: qs_run_opts | None = None):
    _check(_lib.qs_fuse_run(h, circuit.ptr, ctypes.byref(opts) if opts is not None else None))


def qs_last_run_stats(h) -> dict:
    """Launch counts of the last qs_fuse_run on h."""
    st = qs_run_stats()
    _check(_lib.qs_last_run_stats(h, ctypes.byref(st)))
    return {"fused_launches": st.fused_launches, "gate_launches": st.gate_launches,
            "dense_blocks": st.dense_blocks, "dense_gates": st.dense_gates}


def qs_autotune(h, circuit: Circuit):
    """Time every fusion setting of circuit on the scratch state h; returns
    (best max_fuse, its device time in ms)."""
    best = ctypes.c_int()
    ms = ctypes.c_double()
    _check(_lib.qs_autotune(h, circuit.ptr, ctypes.byref(best), ctypes.byref(ms)))
    return best.value, ms.value


def _batch_arrays(handles, circuits):
    n = len(handles)
    hs = (_P * n)(*[h.value if isinstance(h, _P) else h for h in handles])
    cs = (ctypes.POINTER(qs_circuit) * n)(*[c.ptr for c in circuits])
    return n, hs, cs


def qs_batch_run(handles, circuits, opts: qs_run_opts | None = None):
    n, hs, cs = _batch_arrays(handles, circuits)
    _check(_lib.qs_batch_run(hs, cs, n, ctypes.byref(opts) if opts is not None else None))


def qs_batch_compile(handles, circuits):
    """Compile and capture a batch once; returns a handle for qs_batch_launch."""
    n, hs, cs = _batch_arrays(handles, circuits)
    b = _P()
    _check(_lib.qs_batch_compile(hs, cs, n, ctypes.byref(b)))
    return b


def qs_batch_launch(b):
    _check(_lib.qs_batch_launch(b))


def qs_batch_destroy(b):
    _check(_lib.qs_batch_destroy(b))


def qs_set_wait_limit(seconds: float):
    _check(_lib.qs_set_wait_limit(float(seconds)))


# ---------------------------------------------------------------------------
# Convenience handle
# ---------------------------------------------------------------------------
class State:
    """Owning wrapper of a qs_state handle."""

    def __init__(self, n: int, dtype: int = QS_C128, math: int = QS_MATH_DF, handle=None):
        self.n = n
        self.dtype = dtype
        self.h = handle if handle is not None else qs_create(n, dtype)
        if dtype == QS_C128:
            qs_set_math(self.h, math)

    @property
    def np_dtype(self):
        return np.complex64 if self.dtype == QS_C64 else np.complex128

    @classmethod
    def split(cls, n: int, dtype: int = QS_C128, g: int = 1, hbm_segments: int = 1, math: int = QS_MATH_DF):
        """A state split over device and host memory (qs_create_split)."""
        return cls(n, dtype, math, handle=qs_create_split(n, dtype, g, hbm_segments))

    def close(self):
        if self.h is not None:
            qs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, psi: np.ndarray):
        a = np.ascontiguousarray(np.asarray(psi, dtype=self.np_dtype))
        qs_copy_in(self.h, a)
        qs_sync(self.h)
        return self

    def read(self) -> np.ndarray:
        out = np.empty(1 << self.n, dtype=self.np_dtype)
        return qs_copy_out(self.h, out)

    def gather(self, idx) -> np.ndarray:
        idx = np.asarray(idx, dtype=np.uint64)
        out = np.empty(idx.size, dtype=self.np_dtype)
        return qs_gather(self.h, idx, out)

    def apply(self, g):
        """Apply one gate record (see workloads.circuits.Gate)."""
        if g.kind == "u1":
            if g.ctrls:
                qs_apply_ctrl(self.h, g.ctrls, g.targets[0], g.data)
            else:
                qs_apply_1q(self.h, g.targets[0], g.data)
        elif g.kind == "uk" and len(g.targets) == 2 and not g.ctrls:
            qs_apply_2q(self.h, g.targets[0], g.targets[1], g.data)
        elif g.kind == "uk" and len(g.targets) <= QS_MAX_DENSE:
            qs_apply_dense(self.h, g.ctrls, g.targets, g.data)
        elif g.kind == "diag" and not g.ctrls:
            qs_apply_diag(self.h, g.targets, g.data)
        elif g.kind == "perm":
            qs_apply_perm(self.h, g.ctrls, g.targets, g.data)
        else:
            qs_fuse_run(self.h, Circuit([g]), run_opts(max_fuse=1))
        return self

    def run(self, gates, max_fuse: int = 0, use_graph: int = 0):
        c = gates if isinstance(gates, Circuit) else Circuit(gates)
        qs_fuse_run(self.h, c, run_opts(max_fuse, use_graph))
        return self

    def norm(self) -> float:
        return qs_norm(self.h)

    def probs(self, qubits) -> np.ndarray:
        return qs_probs(self.h, qubits)

    def sync(self, timeout_s: float = 60.0):
        qs_sync(self.h, timeout_s)
