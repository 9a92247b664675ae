"""The host-side gate-list rewrites of qs_fuse_run against the oracle (CPU).

Before it forms blocks, qs_fuse_run rewrites the gate list exactly: X gates
are moved past the diagonal gates they conjugate (two X on one qubit cancel,
a conjugated multi-controlled Z becomes a phase on a bit pattern), a dense
gate on 3..5 targets absorbs the gates after it that stay within 5 qubits
(their product formed in FP64), and consecutive gates on the same one or two
qubits are multiplied into one 2x2 / 4x4 matrix (gate fusion, Sec. I).  These
tests run the rewrites on the CPU through a small harness
(tests/harness/rewrite_harness.cu, linked against the in-tree libqs.so),
apply both the original and the rewritten list to the same seeded state with
the oracle, and require the two states to agree within 1e-12, the
complex128 bar.  They also check that each rewrite fired.

The blocks that follow move gates ahead of gates they commute with (disjoint
qubits; diagonal gates need no tile qubits).  test_block_order applies the
rewritten gates in the order the fused runner executes them, block by block,
for both tile policies and several fusion widths, and compares with the
circuit's own order.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HARNESS = os.path.join(ROOT, "tests", "harness", "rewrite_harness.cu")
OUT_DIR = os.path.join(ROOT, "tests", "_build")

PATTERN = 100  # kind of a phase on a bit pattern
X_PUSH, DENSE, MATFUSE = 1, 2, 4


class RwGate(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("k", ctypes.c_int32), ("targets", ctypes.c_int32 * 8),
                ("ctrl", ctypes.c_uint64), ("pmask", ctypes.c_uint64), ("ppat", ctypes.c_uint64),
                ("data_off", ctypes.c_int64), ("perm_off", ctypes.c_int64)]


@pytest.fixture(scope="module")
def harness(oracle_mod):
    pytest.importorskip("torch")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    from paper_2506_09198_gb300 import build

    lib = build.build()
    libdir = os.path.dirname(lib)
    os.makedirs(OUT_DIR, exist_ok=True)
    out = os.path.join(OUT_DIR, "librewrite.so")
    tmp = f"{out}.{os.getpid()}.tmp"  # concurrent test processes each build, then rename
    cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O1", "-std=c++17", "-Xcompiler", "-fPIC",
           "--expt-relaxed-constexpr", "-shared", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(ROOT, "paper_2506_09198_gb300", "csrc"), HARNESS, "-o", tmp,
           "-L", libdir, "-lqs", "-Xlinker", "-rpath=" + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    os.replace(tmp, out)
    h = ctypes.CDLL(out)
    h.rw_block_order.restype = ctypes.c_int64
    h.rw_block_order.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32), ctypes.c_int64]
    h.rw_rewrite.restype = ctypes.c_int64
    h.rw_rewrite.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(RwGate), ctypes.c_int64,
                             ctypes.POINTER(ctypes.c_double), ctypes.c_int64, ctypes.POINTER(ctypes.c_uint32),
                             ctypes.c_int64]
    return h


def rewrite(h, gates, stages):
    from paper_2506_09198_gb300 import qs

    c = qs.Circuit(gates)
    cap = 4 * len(gates) + 16
    out = (RwGate * cap)()
    data = np.zeros(1 << 22)
    perm = np.zeros(1 << 16, dtype=np.uint32)
    cnt = h.rw_rewrite(ctypes.cast(c.ptr, ctypes.c_void_p), stages, out, cap,
                       data.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), data.size,
                       perm.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), perm.size)
    assert cnt >= 0
    return [(out[i], data, perm) for i in range(cnt)]


def ctrl_list(mask):
    return [q for q in range(64) if (mask >> q) & 1]


def apply_rewritten(O, psi, rewritten):
    n = int(psi.size).bit_length() - 1
    idx = np.arange(psi.size, dtype=np.uint64)
    for g, data, perm in rewritten:
        t = [int(g.targets[j]) for j in range(g.k)]
        dim = 1 << g.k
        cs = ctrl_list(int(g.ctrl))
        z = data[g.data_off:g.data_off + 2 * dim * dim].view(np.complex128) if g.kind in (0, 1) else None
        if g.kind == PATTERN:
            c = complex(data[g.data_off], data[g.data_off + 1])
            sel = (idx & np.uint64(g.pmask)) == np.uint64(g.ppat)
            psi[sel] *= c
        elif g.kind == 0:
            O.apply_1q(psi, t[0], z.reshape(2, 2), cs)
        elif g.kind == 1:
            O.apply_kq(psi, t, z.reshape(dim, dim), cs)
        elif g.kind == 2:
            O.apply_diag(psi, t, data[g.data_off:g.data_off + 2 * dim].view(np.complex128), cs)
        elif g.kind == 3:
            O.apply_perm(psi, t, perm[g.perm_off:g.perm_off + dim].copy(), cs)
        else:
            raise AssertionError(f"unknown kind {g.kind}")
    assert n >= 1
    return psi


def varied_circuit(n, n_gates, seed):
    """1q/2q dense, X, controlled gates, phases, diagonals, CZ, SWAP,
    permutations, multi-controlled Z, and dense gates on 3..5 targets."""
    rng = W.rng_for(seed)
    gates = []
    for _ in range(n_gates):
        r = int(rng.integers(12))
        if r <= 1:
            t = int(rng.integers(n))
            U = [W.haar_unitary(2, rng), W.mat_h(), W.mat_x()][int(rng.integers(3))]
            nc = int(rng.integers(0, 2))
            cs = [q for q in W.random_distinct(rng, n, nc + 1) if q != t][:nc]
            gates.append(W.g1(t, U, ctrls=cs))
        elif r == 2:
            gates.append(W.X(int(rng.integers(n))))
        elif r == 3:
            gates.append(W.g1(int(rng.integers(n)), W.mat_phase(rng.uniform(0, 6.3))))
        elif r == 4:
            k = int(rng.integers(1, 4))
            gates.append(W.gdiag(W.random_distinct(rng, n, k), np.exp(1j * rng.uniform(0, 6.3, 1 << k))))
        elif r == 5:
            q = W.random_distinct(rng, n, 3)
            gates.append(W.gk(q[:2], W.haar_unitary(4, rng), ctrls=q[2:2 + int(rng.integers(0, 2))]))
        elif r == 6:
            gates.append(W.CZ(*W.random_distinct(rng, n, 2)))
        elif r == 7:
            gates.append(W.SWAP(*W.random_distinct(rng, n, 2)))
        elif r == 8:
            k = int(rng.integers(1, 3))
            q = W.random_distinct(rng, n, k + 1)
            gates.append(W.gperm(q[:k], rng.permutation(1 << k).astype(np.uint32), ctrls=q[k:k + int(rng.integers(0, 2))]))
        elif r == 9:
            q = W.random_distinct(rng, n, int(rng.integers(2, 5)))
            gates.append(W.MCZ(q[1:], q[0]))
        else:
            k = int(rng.integers(3, 6))
            q = W.random_distinct(rng, n, min(n, k + 1))
            gates.append(W.gk(q[:k], W.haar_unitary(1 << k, rng), ctrls=q[k:k + int(rng.integers(0, 2))]))
    return gates


def check(O, h, n, gates, stages, seed):
    psi0 = W.random_state(n, W.rng_for(seed))
    want = O.run_circuit(psi0.copy(), gates)
    rw = rewrite(h, gates, stages)
    got = apply_rewritten(O, psi0.copy(), rw)
    err = float(np.max(np.abs(got - want)))
    assert err <= 1e-12, f"stages {stages}: max |diff| {err:.3e}"
    return rw


@pytest.mark.parametrize("stages", [X_PUSH, DENSE, MATFUSE, X_PUSH | DENSE | MATFUSE])
@pytest.mark.parametrize("seed", [9100, 9101, 9102])
def test_varied_circuits(oracle_mod, harness, stages, seed):
    n = 8
    gates = varied_circuit(n, 160, seed)
    check(oracle_mod, harness, n, gates, stages, seed + 50)


def test_each_rewrite_fires(oracle_mod, harness):
    n = 8
    rng = W.rng_for(9200)
    # X on a control of a multi-controlled Z, on both sides: the X gates meet and
    # cancel, and the Z becomes a phase on the pattern with that control bit 0
    gates = [W.X(1), W.MCZ([0, 1, 2], 5), W.X(1)]
    rw = check(oracle_mod, harness, n, gates, X_PUSH, 9201)
    assert len(rw) == 1 and rw[0][0].kind == PATTERN
    # a dense 3-target gate absorbs the 1q/2q gates on its qubits after it
    gates = [W.gk([1, 4, 6], W.haar_unitary(8, rng)), W.H(4), W.CNOT(1, 6), W.g1(6, W.haar_unitary(2, rng)),
             W.gk([2, 4, 6], W.haar_unitary(8, rng))]
    rw = check(oracle_mod, harness, n, gates, DENSE, 9202)
    assert len(rw) == 1 and rw[0][0].kind == 1 and rw[0][0].k == 4
    # consecutive gates on one pair of qubits become one 4x4
    gates = [W.g1(2, W.haar_unitary(2, rng)), W.g1(5, W.haar_unitary(2, rng)), W.CZ(2, 5),
             W.g1(2, W.haar_unitary(2, rng)), W.g1(5, W.haar_unitary(2, rng))]
    rw = check(oracle_mod, harness, n, gates, MATFUSE, 9203)
    assert len(rw) < len(gates)


@pytest.mark.parametrize("name", ["qft", "grover", "rqc", "shor"])
def test_workload_circuits(oracle_mod, harness, name):
    n = 9
    if name == "qft":
        gates = W.qft(list(range(n)))
    elif name == "grover":
        gates = W.grover(n, 77, 4)
    elif name == "rqc":
        gates = W.rqc(n, 8, seed=9300)
    else:
        gates = W.shor_like(n, seed=9301)[0]
    check(oracle_mod, harness, n, gates, X_PUSH | DENSE | MATFUSE, 9302)


@pytest.mark.parametrize("dtype_name", ["c128", "c64"])
@pytest.mark.parametrize("max_high", [2, 4, 6])
@pytest.mark.parametrize("name", ["varied", "qft", "rqc", "grover", "shor"])
def test_block_order(oracle_mod, harness, dtype_name, max_high, name):
    from paper_2506_09198_gb300 import qs

    O = oracle_mod
    n = 14
    if name == "varied":
        gates = varied_circuit(n, 220, 9400 + max_high)
    elif name == "qft":
        gates = W.qft(list(range(n)))
    elif name == "rqc":
        gates = W.rqc(n, 10, seed=9401)
    elif name == "grover":
        gates = W.grover(n, 4321, 3)
    else:
        gates = W.shor_like(n, seed=9402)[0]
    rw = rewrite(harness, gates, X_PUSH | DENSE | MATFUSE)
    c = qs.Circuit(gates)
    cap = len(rw) + 8
    order = np.zeros(cap, dtype=np.int64)
    block = np.zeros(cap, dtype=np.int32)
    dt = qs.QS_C128 if dtype_name == "c128" else qs.QS_C64
    cnt = harness.rw_block_order(ctypes.cast(c.ptr, ctypes.c_void_p), n, dt, max_high,
                                 order.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                 block.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), cap)
    assert cnt == len(rw)
    order, block = order[:cnt], block[:cnt]
    assert sorted(order.tolist()) == list(range(cnt))  # every gate exactly once
    assert np.all(np.diff(block) >= 0)
    psi0 = W.random_state(n, W.rng_for(9403))
    want = O.run_circuit(psi0.copy(), gates)
    got = apply_rewritten(O, psi0.copy(), [rw[i] for i in order])
    err = float(np.max(np.abs(got - want)))
    assert err <= 1e-12, f"max |diff| {err:.3e}"
    if name in ("varied", "qft", "rqc"):
        assert block[-1] + 1 < cnt  # blocks of several gates formed
