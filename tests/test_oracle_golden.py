"""The oracle's single-qubit access pattern against the paper (CPU only).

tests/golden/access_6q.txt lists, for a 6-qubit state, the amplitude pairs
that a single-qubit gate on each target mixes (the pattern Fig. 3 draws for
targets 0..5) and the pairs that a gate controlled by qubit 2 updates
(Fig. 4: only pairs whose control bit is 1).  The file is written by
tests/golden/make_golden.py from the oracle.  Here it is checked three ways:
the oracle still produces it; its pairs, in order, are those of the paper's
Hadamard kernel (Algorithm 1, Sec. II-B), where task k of target t works on the lower
index made of k's bits above t shifted up by one place and k's bits below t,
and on that index plus 2^t; and the controlled pairs are exactly those whose
lower index has bit 2 set.
"""
import importlib.util
import os

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")
N = 6


def _load_make_golden():
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(GOLDEN, "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _read():
    pairs, ctrl = {}, {}
    with open(os.path.join(GOLDEN, "access_6q.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            head, body = line.split(":", 1)
            kind, t = head.split()
            t = int(t.split("=")[1])
            if kind == "pairs":
                pairs[t] = [tuple(int(x) for x in p.split("-")) for p in body.split()]
            else:
                ctrl[t] = [int(x) for x in body.split()]
    return pairs, ctrl


def test_fixture_is_what_the_oracle_writes(oracle_mod):
    with open(os.path.join(GOLDEN, "access_6q.txt")) as f:
        assert f.read() == _load_make_golden().render()


@pytest.mark.parametrize("t", range(N))
def test_pairs_follow_the_hadamard_kernel_task_order(t):
    pairs, _ = _read()
    half = 1 << t
    want = []
    for k in range(1 << (N - 1)):
        lo = ((k >> t) << (t + 1)) | (k & (half - 1))
        want.append((lo, lo + half))
    assert pairs[t] == want


@pytest.mark.parametrize("t", [0, 1, 3, 4, 5])
def test_controlled_gate_updates_only_control_one_pairs(t):
    pairs, ctrl = _read()
    assert ctrl[t] == [lo for lo, _ in pairs[t] if (lo >> 2) & 1]
    assert len(ctrl[t]) == len(pairs[t]) // 2
