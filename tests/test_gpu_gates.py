"""Per-gate parity: every gate kernel, through the C ABI, against the oracle
on the same seeded inputs, for complex128 (float-float and FP64 arithmetic)
and complex64, across target positions below, at and above the warp and
vector spans, with and without controls."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import MODES, assert_close, new_state, qs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_09198_gb300 import build

    build.build()
    O.build()


def _run_both(n, mode, gates, seed, psi0=None):
    psi0 = W.random_state(n, W.rng_for(seed)) if psi0 is None else psi0
    ref = O.run_circuit(psi0.copy(), gates)
    st = new_state(n, mode, psi0)
    for g in gates:
        st.apply(g)
    got = st.read()
    st.close()
    return got, ref


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n", [1, 2, 3, 5, 6, 7, 9, 12])
def test_dense_1q_every_target(mode, n):
    rng = W.rng_for(1000 + n)
    psi = W.random_state(n, rng)
    st = new_state(n, mode, psi)
    ref = psi.copy()
    for t in range(n):
        U = W.haar_unitary(2, rng)
        st.apply(W.g1(t, U))
        O.apply_1q(ref, t, U)
        assert_close(st.read(), ref, mode, f"n={n} t={t}")
    st.close()


@pytest.mark.parametrize("mode", MODES)
def test_structured_1q(mode):
    n = 8
    rng = W.rng_for(2000)
    mats = {"h": W.mat_h(), "x": W.mat_x(), "y": W.mat_y(), "z": W.mat_z(), "s": W.mat_phase(math.pi / 2),
            "t": W.mat_phase(math.pi / 4), "p": W.mat_phase(0.3), "id": np.eye(2),
            "d": np.diag([np.exp(0.2j), np.exp(-1.1j)]), "d0": np.diag([np.exp(0.7j), 1.0]),
            "ad": np.array([[0, np.exp(0.4j)], [np.exp(-0.9j), 0]]), "sx": W.mat_sqrt_pauli(W.mat_x())}
    for name, U in mats.items():
        for t in (0, 1, 4, 5, 7):
            got, ref = _run_both(n, mode, [W.g1(t, U)], 2100 + t)
            assert_close(got, ref, mode, f"{name} t={t}")
            if name in ("x", "y", "z", "id"):
                assert np.array_equal(got, ref.astype(got.dtype)), f"{name} must move amplitudes exactly"


@pytest.mark.parametrize("mode", MODES)
def test_controlled_1q(mode):
    n = 9
    rng = W.rng_for(3000)
    gates = []
    for _ in range(40):
        nc = int(rng.integers(1, 4))
        qs_ = W.random_distinct(rng, n, nc + 1)
        kind = int(rng.integers(4))
        U = [W.haar_unitary(2, rng), W.mat_x(), W.mat_z(), W.mat_phase(rng.uniform(0, 6.28))][kind]
        gates.append(W.g1(qs_[0], U, ctrls=qs_[1:]))
    got, ref = _run_both(n, mode, gates, 3001)
    assert_close(got, ref, mode, "controlled gates")


@pytest.mark.parametrize("mode", MODES)
def test_cnot_exact(mode):
    n = 10
    rng = W.rng_for(3100)
    gates = [W.CNOT(*W.random_distinct(rng, n, 2)) for _ in range(30)]
    got, ref = _run_both(n, mode, gates, 3101)
    assert np.array_equal(got, ref.astype(got.dtype))


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n", [2, 3, 6, 11])
def test_dense_2q_pairs(mode, n):
    rng = W.rng_for(4000 + n)
    pairs = [(a, b) for a in range(n) for b in range(n) if a != b]
    if len(pairs) > 40:
        pairs = [pairs[i] for i in rng.choice(len(pairs), 40, replace=False)]
    psi = W.random_state(n, rng)
    st = new_state(n, mode, psi)
    ref = psi.copy()
    for t0, t1 in pairs:
        U = W.haar_unitary(4, rng)
        st.apply(W.gk((t0, t1), U))
        O.apply_2q(ref, t0, t1, U)
        assert_close(st.read(), ref, mode, f"n={n} t0={t0} t1={t1}")
    st.close()


@pytest.mark.parametrize("mode", MODES)
def test_controlled_2q_and_structured_2q(mode):
    n = 8
    rng = W.rng_for(4100)
    gates = []
    for _ in range(12):
        q = W.random_distinct(rng, n, 4)
        gates.append(W.gk(q[:2], W.haar_unitary(4, rng), ctrls=q[2:2 + int(rng.integers(0, 3))]))
        gates.append(W.CZ(q[0], q[1]))
        gates.append(W.SWAP(q[2], q[3]))
        swapmat = np.eye(4)[[0, 2, 1, 3]]
        gates.append(W.gk((q[0], q[3]), swapmat))  # a permutation matrix given densely
        gates.append(W.gk((q[1], q[2]), np.diag(np.exp(1j * rng.uniform(0, 6, 4)))))  # diagonal given densely
    got, ref = _run_both(n, mode, gates, 4101)
    assert_close(got, ref, mode, "2q mix")


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("k", [1, 2, 3, 5, 8])
def test_diag_k(mode, k):
    n = 10
    rng = W.rng_for(5000 + k)
    gates = []
    for _ in range(4):
        q = W.random_distinct(rng, n, k + 2)
        d = np.exp(1j * rng.uniform(0, 2 * math.pi, 1 << k))
        gates.append(W.gdiag(q[:k], d))
        gates.append(W.gdiag(q[:k], d, ctrls=q[k:k + 1]))
        one_hot = np.ones(1 << k, dtype=np.complex128)
        one_hot[int(rng.integers(1 << k))] = -1
        gates.append(W.gdiag(q[:k], one_hot, ctrls=q[k + 1:]))
    got, ref = _run_both(n, mode, gates, 5100 + k)
    assert_close(got, ref, mode, f"diag k={k}")


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("k", [1, 2, 3, 4, 6, 8])
def test_perm_k_exact(mode, k):
    n = 11
    rng = W.rng_for(6000 + k)
    gates = []
    for nc in (0, 1, 2):
        q = W.random_distinct(rng, n, k + nc)
        gates.append(W.gperm(q[:k], rng.permutation(1 << k).astype(np.uint32), ctrls=q[k:]))
    got, ref = _run_both(n, mode, gates, 6100 + k)
    assert np.array_equal(got, ref.astype(got.dtype)), f"perm k={k} must move amplitudes exactly"


@pytest.mark.parametrize("mode", MODES)
def test_single_transpositions_exact(mode):
    """Permutations that exchange exactly two sub-register values (SWAP is
    01 <-> 10) run on the pair-exchange kernel: bit-exact against the oracle,
    with and without controls, on low, high and mixed qubits."""
    n = 13
    rng = W.rng_for(6400)
    gates = [W.SWAP(0, 1), W.SWAP(0, 12), W.SWAP(7, 3), W.gperm((5, 6), np.array([0, 1, 2, 3][::-1], np.uint32)),
             W.SWAP(2, 9)]
    gates[-1] = W.Gate("perm", (2, 9), np.array([0, 2, 1, 3], np.uint32), ctrls=(4, 11), name="cswap")
    for k in (2, 3, 5):
        for nc in (0, 2):
            q = W.random_distinct(rng, n, k + nc)
            p = np.arange(1 << k, dtype=np.uint32)
            a, b = (int(x) for x in rng.choice(1 << k, size=2, replace=False))
            p[a], p[b] = b, a
            gates.append(W.gperm(q[:k], p, ctrls=q[k:]))
    got, ref = _run_both(n, mode, gates, 6401)
    assert np.array_equal(got, ref.astype(got.dtype)), "transpositions must move amplitudes exactly"


@pytest.mark.parametrize("mode", MODES)
def test_perm_whole_register(mode):
    n = 8
    rng = W.rng_for(6500)
    g = W.gperm(list(range(n)), rng.permutation(1 << n).astype(np.uint32))
    got, ref = _run_both(n, mode, [g], 6501)
    assert np.array_equal(got, ref.astype(got.dtype))


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n", [1, 4, 12, 17])
def test_norm_and_probs(mode, n):
    rng = W.rng_for(7000 + n)
    psi = W.random_state(n, rng) * 0.8
    st = new_state(n, mode, psi)
    stored = psi.astype(st.np_dtype).astype(np.complex128)
    tol = 1e-13 if mode.startswith("c128") else 1e-12
    assert abs(st.norm() - O.norm2(stored)) <= tol
    for k in sorted({1, min(3, n), min(n, 6)}):
        qubits = W.random_distinct(rng, n, k)
        got = st.probs(qubits)
        want = O.probs(stored, qubits)
        assert np.max(np.abs(got - want)) <= tol, f"probs k={k}"
    st.close()


@pytest.mark.parametrize("mode", MODES)
def test_init_copy_gather(mode):
    n = 13
    st = new_state(n, mode)
    out = st.read()
    assert out[0] == 1 and np.count_nonzero(out) == 1
    qs().qs_init_basis(st.h, 4097)
    out = st.read()
    assert out[4097] == 1 and np.count_nonzero(out) == 1
    psi = W.random_state(n, W.rng_for(7100)).astype(st.np_dtype)
    st.load(psi)
    assert np.array_equal(st.read(), psi)
    idx = np.array([0, 1, 4097, (1 << n) - 1, 77], dtype=np.uint64)
    assert np.array_equal(st.gather(idx), psi[idx.astype(np.int64)])
    out = np.zeros_like(psi)
    qs().qs_copy_out_async(st.h, out)
    st.sync()
    assert np.array_equal(out, psi)
    st.close()


@pytest.mark.parametrize("max_fuse", [1, 0, 6])
@pytest.mark.parametrize("mode", MODES)
def test_random_circuit_400_gates_n20(mode, max_fuse):
    """20-qubit state from |0...0>, 400 gates: Haar 2x2 on uniform targets,
    CNOT on random distinct pairs at 30% of gates; full-state check, gate by
    gate (max_fuse 1) and through the fuser (0: the default width; 6: the
    widest blocks)."""
    n = 20
    gates = W.random_circuit(n, 400, 0.3, seed=2506)
    psi0 = O.basis_state(n)
    ref = O.run_circuit(psi0.copy(), gates)
    st = new_state(n, mode)
    st.run(gates, max_fuse=max_fuse)
    got = st.read()
    st.close()
    assert_close(got, ref, mode, f"random circuit n=20, max_fuse={max_fuse}")


def test_errors_on_gpu():
    q = qs()
    st = new_state(5, "c128_df")
    with pytest.raises(q.QSError) as e:
        q.qs_apply_1q(st.h, 5, np.eye(2))
    assert e.value.status == q.QS_ERR_ARG
    with pytest.raises(q.QSError):
        q.qs_apply_ctrl(st.h, [1, 1], 0, np.eye(2))
    with pytest.raises(q.QSError):
        q.qs_apply_perm(st.h, [], [0, 1], [0, 1, 1, 3])
    with pytest.raises(q.QSError):
        q.qs_apply_1q(st.h, 0, np.array([[np.nan, 0], [0, 1]]))
    with pytest.raises(q.QSError):
        q.qs_probs(st.h, [0, 0])
    st.run([])  # empty circuit is a no-op
    st.sync(5.0)
    st.close()


def test_torch_owned_memory():
    """A torch complex128 tensor wrapped as a state on torch's stream."""
    torch = pytest.importorskip("torch")
    q = qs()
    n = 12
    psi = W.random_state(n, W.rng_for(7200))
    t = torch.from_numpy(psi.copy()).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    h = q.qs_wrap(n, q.QS_C128, t.data_ptr(), stream)
    U = W.haar_unitary(2, W.rng_for(7201))
    q.qs_apply_1q(h, 7, U)
    q.qs_sync(h)
    got = t.cpu().numpy()
    q.qs_destroy(h)
    ref = O.apply_1q(psi.copy(), 7, U)
    assert_close(got, ref, "c128_df", "wrapped torch tensor")
