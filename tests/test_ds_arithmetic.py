"""Double-single primitives of the mixed-precision path (Sec. 2.4, Algorithm 1)
on the GPU against exact rational arithmetic: sums and products to the
paper's 44-bit effective precision, normalised results, and exact two-sum /
two-product error terms (which any contraction of the error-free
transformations into fused operations would break)."""
import os
import subprocess
from fractions import Fraction as Fr

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _program(tmp_path):
    import shutil
    if shutil.which("nvcc") is None:
        pytest.skip("nvcc not available")
    exe = tmp_path / "ds_unit"
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "-I", os.path.join(ROOT, "paper_0912_3824_gb300", "csrc"), "-o", str(exe),
                    os.path.join(HERE, "ds_unit.cu")], check=True)
    return exe


def _normalise(hi, lo):
    """(hi, lo) as float32 with hi = fl(hi + lo): a valid double-single value."""
    h = np.float32(np.float64(hi) + np.float64(lo))
    return h, np.float32(np.float64(hi) + np.float64(lo) - np.float64(h))


def _operands(rng, n):
    out = []
    for k in range(n):
        e1, e2 = rng.integers(-20, 20, 2)
        a = _normalise(rng.standard_normal() * 2.0 ** e1, rng.standard_normal() * 2.0 ** (e1 - 26))
        if k % 4 == 1:                  # near cancellation: b close to -a
            b = _normalise(-np.float64(a[0]) * (1 + rng.standard_normal() * 1e-6), rng.standard_normal() * 2.0 ** (e1 - 30))
        elif k % 4 == 2:                # low words zero: the error-free transformations alone
            a = (a[0], np.float32(0.0))
            b = (np.float32(rng.standard_normal() * 2.0 ** e2), np.float32(0.0))
        else:
            b = _normalise(rng.standard_normal() * 2.0 ** e2, rng.standard_normal() * 2.0 ** (e2 - 26))
        out.append((a[0], a[1], b[0], b[1]))
    return np.array(out, dtype=np.float32)


def test_ds_add_mul_against_exact_rationals(tmp_path):
    exe = _program(tmp_path)
    ops = _operands(np.random.default_rng(7), 4000)
    inp, outp = tmp_path / "in.bin", tmp_path / "out.bin"
    with open(inp, "wb") as f:
        f.write(np.int32(len(ops)).tobytes())
        f.write(ops.tobytes())
    subprocess.run([str(exe), str(inp), str(outp)], check=True)
    res = np.fromfile(outp, dtype=np.float32).reshape(-1, 6)
    tol = Fr(1, 2 ** 44)
    for (ah, al, bh, bl), (sh, sl, ph, pl, qh, ql), k in zip(ops, res, range(len(ops))):
        a, b = Fr(float(ah)) + Fr(float(al)), Fr(float(bh)) + Fr(float(bl))
        for hi, lo in ((sh, sl), (ph, pl), (qh, ql)):
            assert np.float32(np.float64(hi) + np.float64(lo)) == hi      # normalised
        s = Fr(float(sh)) + Fr(float(sl))
        assert abs(s - (a + b)) <= tol * (abs(a) + abs(b))
        p = Fr(float(ph)) + Fr(float(pl))
        assert abs(p - a * b) <= tol * abs(a * b)
        q = Fr(float(qh)) + Fr(float(ql))
        assert abs(q - a * Fr(float(bh))) <= tol * abs(a * Fr(float(bh)))
        if al == 0 and bl == 0:         # two-sum and two-product are exact
            assert s == a + b
            assert p == a * b and q == a * b
