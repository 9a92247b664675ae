"""Writes the fixtures in this folder.  Every stored value comes from the
oracle (``oracle/``); nothing here comes from the CUDA library.

access_6q.txt: which amplitude indices a single-qubit gate mixes on a
6-qubit state, for each target 0..5 (the access pattern of Fig. 3), and
which of those pairs a gate controlled by qubit 2 updates (Fig. 4).  The
pairs are found by applying the oracle's Hadamard to every basis state: a
basis state |i> with bit t clear spreads over exactly {i, partner}.  They are
listed in ascending order of the lower index, which is the task order of the
paper's Hadamard kernel (Algorithm 1, Sec. II-B).

Run from the repository root: python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402

N = 6
CONTROL = 2
H = np.array([[1.0, 1.0], [1.0, -1.0]], dtype=np.complex128) / np.sqrt(2.0)


def _touched(i, t, ctrls=()):
    psi = oracle.basis_state(N, i)
    oracle.apply_1q(psi, t, H, ctrls)
    return [int(j) for j in np.flatnonzero(np.abs(psi) > 0.0)]


def pairs(t):
    """(lower, upper) index pairs that H on target t mixes, lower ascending."""
    out = []
    for i in range(1 << N):
        nz = _touched(i, t)
        if len(nz) == 2 and nz[0] == i:
            out.append((nz[0], nz[1]))
    return out


def controlled_updates(t):
    """Lower indices of the pairs that H on t controlled by CONTROL changes."""
    return [lo for lo, _ in pairs(t) if _touched(lo, t, (CONTROL,)) != [lo]]


def render() -> str:
    lines = [
        "# Amplitude index pairs mixed by a single-qubit gate on a 6-qubit state (Fig. 3),",
        "# lower index ascending = task order of the Hadamard kernel (Algorithm 1), and the pairs",
        f"# a gate controlled by qubit {CONTROL} updates (Fig. 4).  Written by make_golden.py from the oracle.",
    ]
    for t in range(N):
        lines.append(f"pairs t={t}: " + " ".join(f"{a}-{b}" for a, b in pairs(t)))
    for t in range(N):
        if t != CONTROL:
            lines.append(f"ctrl{CONTROL} t={t}: " + " ".join(str(a) for a in controlled_updates(t)))
    return "\n".join(lines) + "\n"


if __name__ == "__main__":
    oracle.build()
    with open(os.path.join(HERE, "access_6q.txt"), "w") as f:
        f.write(render())
