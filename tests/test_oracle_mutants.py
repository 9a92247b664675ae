"""Plant plausible mistakes in copies of the oracle source and check that the
pins catch every one (CPU only).  Each mutant is built into a temporary
directory and exercised in a child process; the committed oracle is untouched."""
import os
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "qsim_oracle.c")

# (name, original text, planted text); each original must occur in the source.
MUTANTS = [
    ("transposed_1q", "psi[up] = c_add(c_mul(u00, a), c_mul(u01, b));",
     "psi[up] = c_add(c_mul(u00, a), c_mul(u10, b));"),
    ("cmul_sign", "a.re * b.im + a.im * b.re", "a.re * b.im - a.im * b.re"),
    ("sub_index_order", "s |= (uint64_t)bit_of(i, targets[j]) << j;",
     "s |= (uint64_t)bit_of(i, targets[j]) << (k - 1 - j);"),
    ("any_control", "return (i & ctrl_mask) == ctrl_mask;", "return ctrl_mask == 0 || (i & ctrl_mask) != 0;"),
    ("perm_inverse", "psi[with_sub(i, targets, k, perm[s])] = src[i];",
     "psi[i] = src[with_sub(i, targets, k, perm[s])];"),
    ("kq_transposed", "mat_at(M, sub, r, s)", "mat_at(M, sub, s, r)"),
    ("diag_conjugate", "c_make(d[2 * s], d[2 * s + 1])", "c_make(d[2 * s], -d[2 * s + 1])"),
    ("lo_row_dropped_term", "psi[lo] = c_add(c_mul(u10, a), c_mul(u11, b));", "psi[lo] = c_mul(u11, b);"),
    ("norm_drops_imag", "const double term = psi[i].re * psi[i].re + psi[i].im * psi[i].im;\n    const double y = term - comp;",
     "const double term = psi[i].re * psi[i].re;\n    const double y = term - comp;"),
    ("probs_wrong_bucket", "const uint64_t s = sub_index(i, qubits, k);",
     "const uint64_t s = sub_index(i, qubits, k) ^ 1u;"),
    ("with_sub_clears_wrong", "i = (i & ~m) | (((s >> j) & 1u) ? m : 0u);", "i = i | (((s >> j) & 1u) ? m : 0u);"),
]

CHILD = textwrap.dedent(
    """
    import sys
    sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
    import oracle.oracle as o
    o._SRC = {src!r}; o._BUILD_DIR = {bdir!r}; o._LIB_PATH = {lib!r}; o._LIB_OMP_PATH = {lib_omp!r}
    o.build(force=True)
    import pins
    failed = []
    for pin in pins.ALL_PINS:
        try:
            pin(o)
        except AssertionError:
            failed.append(pin.__name__)
        except Exception as e:  # a crash also counts as caught
            failed.append(pin.__name__ + ':' + type(e).__name__)
    # the threaded build of the same mutant source computes the same states
    failed = [f for f in failed if f != 'pin_threaded_build_identical']
    print('CAUGHT' if failed else 'MISSED', failed)
    """
)


@pytest.mark.parametrize("name,orig,planted", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(tmp_path, name, orig, planted):
    src = open(SRC).read()
    assert orig in src, f"mutation anchor for {name} not found in the oracle source"
    msrc = tmp_path / "qsim_oracle.c"
    msrc.write_text(src.replace(orig, planted, 1))
    code = CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"), src=str(msrc), bdir=str(tmp_path),
                        lib=str(tmp_path / "liboracle.so"), lib_omp=str(tmp_path / "liboracle_omp.so"))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    out = r.stdout + r.stderr
    assert r.returncode != 0 or "CAUGHT" in r.stdout, f"mutant {name} survived every pin:\n{out}"
