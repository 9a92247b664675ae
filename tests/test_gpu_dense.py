"""Dense gates on 3..5 targets through the C ABI against the oracle.

complex64 states run on the tensor cores (3xTF32 split; mode 2 takes them
wherever they apply: 3 and 4 targets as the 5-target gate I (x) U on free
qubits, 4 targets on the 4-target kernel when no qubit is free), on the
default mix (mode 1) or on the FP32 CUDA cores (mode 0); complex128 states on
FP64 CUDA cores.  Sizes span one group (n = k), a partial tile (fewer than 128
groups), many tiles and more tiles than resident CTAs; targets low, high and
scattered (unsorted); 0-2 controls.

complex64 bar, per amplitude: |got - ref| <= (4d + 8) 2^-24 sum_c |U_rc||x_c|
(d = 2^k), where the sum is the oracle applied to |x| with |U|.  A sum of 2d
FP32 products has error below 2d 2^-24 of that sum; the TF32 head/remainder
split adds about 2^-23 per product.  Dropping one of the three TF32 products
(error about 2^-12) fails it by a factor of 30.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import C128_TOL, oracle_threads, qs

pytestmark = pytest.mark.gpu

MODES = ["c64_tc", "c64_auto", "c64_cc", "c128_df", "c128_fp64"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_09198_gb300 import build

    build.build()
    O.build()


def make_state(n, mode, psi):
    q = qs()
    if mode.startswith("c64"):
        st = q.State(n, q.QS_C64)
        q.qs_set_tensor_cores(st.h, {"c64_tc": 2, "c64_auto": 1, "c64_cc": 0}[mode])
    else:
        st = q.State(n, q.QS_C128, q.QS_MATH_DF if mode == "c128_df" else q.QS_MATH_FP64)
    st.load(psi)
    return st


def stored_input(psi, mode):
    """The amplitudes as the device holds them (complex64 rounding), in double."""
    return psi.astype(np.complex64).astype(np.complex128) if mode.startswith("c64") else psi.copy()


def check(got, x_in, gates, mode, what):
    ref = x_in.copy()
    bound = np.abs(x_in).astype(np.complex128)
    with oracle_threads(O):
        for g in gates:
            O.apply_gate(ref, g)
            O.apply_gate(bound, W.Gate(g.kind, g.targets, np.abs(g.data).astype(np.complex128), g.ctrls))
    err = np.abs(np.asarray(got, dtype=np.complex128) - ref)
    if mode.startswith("c128"):
        assert float(err.max()) <= C128_TOL, f"{what}: max abs error {err.max():.3e}"
        return float(err.max())
    d = max(g.data.shape[0] for g in gates)
    gamma = (4 * d + 8) * 2.0 ** -24 * len(gates)
    ratio = err / np.maximum(gamma * bound.real, 1e-300)
    worst = int(np.argmax(ratio))
    assert ratio[worst] <= 1.0, (f"{what}: amplitude {worst} error {err[worst]:.3e} above "
                                 f"{gamma:.2e} x {bound.real[worst]:.3e}")
    return float(err.max())


def target_sets(n, k, rng):
    sets = {"low": list(range(k)), "high": list(range(n - k, n))}
    sets["scattered"] = W.random_distinct(rng, n, k)
    return sets


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("k", [3, 4, 5])
@pytest.mark.parametrize("n_extra", [0, 3, 9, 15, 17])
def test_dense_k_parity(mode, k, n_extra):
    n = k + n_extra
    q = qs()
    rng = W.rng_for(7000 + 100 * k + n)
    sets = target_sets(n, k, rng)
    if n_extra == 17:  # more tiles than resident CTAs: one scattered case
        sets = {"scattered": sets["scattered"]}
    for name, tg in sets.items():
        for nc in ([1] if n_extra == 17 else range(0, min(2, n - k) + 1)):
            free = [x for x in range(n) if x not in tg]
            cs = [free[int(i)] for i in rng.choice(len(free), size=nc, replace=False)] if nc else []
            U = W.haar_unitary(1 << k, rng)
            psi = W.random_state(n, rng)
            x_in = stored_input(psi, mode)
            st = make_state(n, mode, psi)
            q.qs_apply_dense(st.h, cs, tg, U)
            got = st.read()
            st.close()
            check(got, x_in, [W.gk(tg, U, ctrls=cs)], mode, f"n={n} k={k} {name} t={tg} c={cs}")


@pytest.mark.parametrize("mode", ["c64_tc", "c64_cc", "c128_df"])
def test_dense_k_closed_forms(mode):
    """H on k qubits as one dense matrix maps |0> to the uniform state; the
    QFT matrix on k qubits maps |x> to 2^-k/2 sum_y e^{2 pi i x y / 2^k} |y>."""
    q = qs()
    for k in (3, 4, 5):
        d = 1 << k
        Hk = np.ones((1, 1))
        for _ in range(k):
            Hk = np.kron(Hk, W.mat_h())
        n = k + 4
        tg = [1, 3, 4, 6, 8][:k]
        st = make_state(n, mode, O.basis_state(n, 0))
        q.qs_apply_dense(st.h, [], tg, Hk)
        got = st.read()
        st.close()
        want = np.zeros(1 << n, dtype=np.complex128)
        for s in range(d):
            want[sum(1 << tg[j] for j in range(k) if (s >> j) & 1)] = d ** -0.5
        tol = 1e-15 if mode.startswith("c128") else 4e-7
        assert float(np.max(np.abs(got - want))) <= tol, f"H^{k}"
        F = np.array([[np.exp(2j * math.pi * x * y / d) for x in range(d)] for y in range(d)]) / math.sqrt(d)
        x = 5 % d
        idx = sum(1 << tg[j] for j in range(k) if (x >> j) & 1)
        st = make_state(n, mode, O.basis_state(n, idx))
        q.qs_apply_dense(st.h, [], tg, F)
        got = st.read()
        st.close()
        want = np.zeros(1 << n, dtype=np.complex128)
        for y in range(d):
            want[sum(1 << tg[j] for j in range(k) if (y >> j) & 1)] = np.exp(2j * math.pi * x * y / d) / math.sqrt(d)
        assert float(np.max(np.abs(got - want))) <= tol, f"QFT_{k}"


@pytest.mark.parametrize("mode", MODES)
def test_dense_k_in_fused_runs(mode):
    """Dense 3..5-qubit gates inside a circuit run by qs_fuse_run: the fused
    blocks around them and the per-gate launches for them agree with the
    oracle, and the launches are counted as per-gate launches."""
    q = qs()
    n = 16
    rng = W.rng_for(7500)
    gates = [W.g1(t, W.mat_h()) for t in range(n)]
    gates.append(W.gk([0, 3, 7, 9, 12], W.haar_unitary(32, rng)))
    gates += [W.g1(t, W.haar_unitary(2, rng)) for t in (1, 5, 9, 15)]
    gates.append(W.gk([15, 2, 8], W.haar_unitary(8, rng), ctrls=(5,)))
    gates.append(W.gk([11, 12, 13, 14], W.haar_unitary(16, rng), ctrls=(0, 1)))
    gates += [W.gk([t, t + 1], W.haar_unitary(4, rng)) for t in (0, 4, 10)]
    psi = W.random_state(n, rng)
    x_in = stored_input(psi, mode)
    st = make_state(n, mode, psi)
    st.run(gates)
    stats = q.qs_last_run_stats(st.h)
    got = st.read()
    st.close()
    assert stats["gate_launches"] >= 3
    if mode.startswith("c128"):
        ref = O.run_circuit(x_in.copy(), gates)
        assert float(np.max(np.abs(got - ref))) <= C128_TOL
    else:
        ref = O.run_circuit(x_in.copy(), gates)
        f = abs(np.vdot(got, ref)) ** 2 / (np.vdot(got, got).real * np.vdot(ref, ref).real)
        assert f >= 1 - 1e-6 and float(np.max(np.abs(got - ref))) <= 2e-6


@pytest.mark.parametrize("mode", ["c64_tc", "c128_df"])
def test_dense_k_on_split_states(mode):
    """Split states (top 2 qubits select 4 segments, two in host memory):
    dense gates with targets and controls on global qubits are made local
    first; the result matches the oracle."""
    q = qs()
    n = 14
    rng = W.rng_for(7600)
    dt = q.QS_C64 if mode.startswith("c64") else q.QS_C128
    st = q.State.split(n, dt, g=2, hbm_segments=2)
    if mode == "c64_tc":
        q.qs_set_tensor_cores(st.h, 2)
    psi = W.random_state(n, rng)
    st.load(psi)
    x_in = stored_input(psi, mode)
    gates = [W.gk([13, 12, 3, 0, 7], W.haar_unitary(32, rng)),
             W.gk([1, 12, 5], W.haar_unitary(8, rng), ctrls=(13,)),
             W.gk([2, 6, 9, 13], W.haar_unitary(16, rng), ctrls=(11,))]
    for g in gates:
        st.apply(g)
    got = st.read()
    st.close()
    check(got, x_in, gates, mode, "split")


def test_dense_k_30q_c64_sampled():
    """30-qubit complex64 state (8 GiB, the dense-gate benchmark's size): a
    5-qubit gate on the tensor cores; sampled groups against the oracle
    applied to the 32-amplitude group alone."""
    torch = pytest.importorskip("torch")
    q = qs()
    n, k = 30, 5
    psi = W.random_state(n, 2600).astype(np.complex64)
    dev = torch.from_numpy(psi.view(np.float32)).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    h = q.qs_wrap(n, q.QS_C64, dev.data_ptr(), stream)
    rng = W.rng_for(2601)
    for tg, cs in (([0, 7, 15, 22, 29], []), ([29, 3, 1, 18, 10], [0, 25]), ([2, 3, 4, 5, 6], [])):
        U = W.haar_unitary(1 << k, rng)
        x = psi
        q.qs_apply_dense(h, cs, tg, U)
        groups = rng.integers(0, 1 << (n - k - len(cs)), size=256, dtype=np.uint64)
        pos = sorted(tg + cs)
        bases = []
        for g in groups.tolist():
            b = g
            for p in pos:
                b = ((b >> p) << (p + 1)) | (b & ((1 << p) - 1))
            for c in cs:
                b |= 1 << c
            bases.append(b)
        offs = [sum(1 << tg[j] for j in range(k) if (s >> j) & 1) for s in range(1 << k)]
        idx = np.array([b | o for b in bases for o in offs], dtype=np.uint64)
        out = np.empty(idx.size, dtype=np.complex64)
        q.qs_gather(h, idx, out)
        xin = x[idx.astype(np.int64)].astype(np.complex128).reshape(-1, 1 << k)
        got = out.astype(np.complex128).reshape(-1, 1 << k)
        gamma = (4 * 32 + 8) * 2.0 ** -24
        for j in range(len(bases)):
            want = O.apply_kq(xin[j].copy(), list(range(k)), U)
            bound = O.apply_kq(np.abs(xin[j]).astype(np.complex128), list(range(k)), np.abs(U).astype(np.complex128))
            assert np.all(np.abs(got[j] - want) <= gamma * bound.real), f"t={tg} c={cs} group {j}"
        # Restore the input for the next gate.
        dev.copy_(torch.from_numpy(psi.view(np.float32)))
    q.qs_destroy(h)


def test_tensor_core_switch_arguments():
    q = qs()
    st = q.State(6, q.QS_C64)
    with pytest.raises(q.QSError):
        q.qs_set_tensor_cores(st.h, 3)
    U = W.haar_unitary(64, W.rng_for(1))
    with pytest.raises(q.QSError):
        q.qs_apply_dense(st.h, [], [0, 1, 2, 3, 4, 5], U)  # 6 targets: above QS_MAX_DENSE
    with pytest.raises(q.QSError):
        q.qs_apply_dense(st.h, [0], [0, 1, 2], W.haar_unitary(8, W.rng_for(2)))  # control is a target
    st.close()


@pytest.fixture
def restore_wait_limit():
    yield
    qs().qs_set_wait_limit(2.0)


def test_dense_tc_wait_runs_out_and_context_survives(restore_wait_limit):
    """With a zero wait limit the tensor-core kernel's bounded mbarrier waits
    give up: the state's next sync reports QS_ERR_TIMEOUT, the kernel has
    freed its tensor memory and returned, and the same context then applies
    the gate correctly."""
    q = qs()
    n = 20
    tg = [0, 5, 9, 14, 19]
    U = W.haar_unitary(32, W.rng_for(7700))
    st = q.State(n, q.QS_C64)
    q.qs_set_tensor_cores(st.h, 2)
    q.qs_set_wait_limit(0.0)
    for _ in range(4):
        q.qs_apply_dense(st.h, [], tg, U)
    q.qs_set_wait_limit(2.0)
    with pytest.raises(q.QSError) as e:
        st.sync()
    assert e.value.status == q.QS_ERR_TIMEOUT
    st.sync()  # reading the error cleared it
    psi = W.random_state(n, W.rng_for(7701))
    st.load(psi)
    q.qs_apply_dense(st.h, [], tg, U)
    got = st.read()
    st.close()
    check(got, stored_input(psi, "c64_tc"), [W.gk(tg, U)], "c64_tc", "after a timeout")


@pytest.mark.parametrize("mode", ["c64_tc", "c64_cc", "c128_df"])
def test_dense_blocks_composed_in_fused_runs(mode):
    """qs_fuse_run composes a dense gate on 3..5 targets with the gates after
    it that stay within 5 qubits (one pass instead of one per dense gate):
    gates on other qubits are stepped over and close their qubits to the
    block, so a gate after a stepped-over gate on a shared qubit is not moved
    ahead of it.  The result matches the oracle, and the three dense gates
    form one composed block."""
    q = qs()
    n = 14
    rng = W.rng_for(7800)
    gates = [W.g1(t, W.mat_h()) for t in range(n)]
    gates += [W.gk([2, 5, 9], W.haar_unitary(8, rng)),                  # starts a block on {2, 5, 9}
              W.g1(0, W.haar_unitary(2, rng)),                          # disjoint: stepped over
              W.g1(5, W.haar_unitary(2, rng)),                          # inside: absorbed
              W.CNOT(2, 11),                                            # widens to {2, 5, 9, 11}
              W.gk([9, 11, 5], W.haar_unitary(8, rng), ctrls=(2,)),     # inside
              W.CNOT(0, 1),                                             # disjoint
              W.gk([2, 5, 9, 11, 12], W.haar_unitary(32, rng)),         # widens to 5 qubits
              W.CZ(12, 13),                                             # 13 outside: stepped over, closes 12, 13
              W.g1(12, W.mat_h()),                                      # on a closed qubit: stays after the CZ
              W.g1(9, W.haar_unitary(2, rng)),                          # inside, open: absorbed
              W.g1(13, W.haar_unitary(2, rng))]
    psi = W.random_state(n, rng)
    x_in = stored_input(psi, mode)
    st = make_state(n, mode, psi)
    st.run(gates)
    stats = q.qs_last_run_stats(st.h)
    got = st.read()
    st.close()
    ref = O.run_circuit(x_in.copy(), gates)
    if mode.startswith("c128"):
        assert float(np.max(np.abs(got - ref))) <= C128_TOL
    else:
        f = abs(np.vdot(got, ref)) ** 2 / (np.vdot(got, got).real * np.vdot(ref, ref).real)
        assert f >= 1 - 1e-6 and float(np.max(np.abs(got - ref))) <= 2e-6
    # One block: the three dense gates, g1(5), CNOT(2, 11) and the trailing
    # g1(9).
    assert stats["dense_blocks"] == 1 and stats["dense_gates"] == 6, stats
