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
