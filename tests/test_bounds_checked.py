"""Bounds-checked run of the parity tests.  compute-sanitizer is not available
where these tests run, so the library is rebuilt with MD_CHECK_BOUNDS: every
index the kernels read from device memory (neighbour-list entries, cell keys,
permutation slots, staged candidates) is tested against its array, and a
violation stops the step loop with MD_E_BOUNDS instead of touching memory
outside the array.  A selection of the GPU parity tests then runs against that
library in a child process; they check md_sync() == MD_OK, so any violation
fails them."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

SELECTION = ("forces_energy_virial or ragged or replicas_match or pairs_at_the_cutoff or neighbour_lists "
             "or smoothed_and_wca or lists_cover or fp64_trajectory or overflow_during_run or andersen_collision")


def test_parity_selection_with_bounds_checks():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0912_3824_gb300 import build
    lib = build.build(checked=True)
    env = dict(os.environ, MDGB300_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-m", "gpu",
                        os.path.join(HERE, "test_gpu_parity.py"), "-k", SELECTION],
                       env=env, cwd=ROOT, capture_output=True, text=True)
    tail = "\n".join((r.stdout + r.stderr).splitlines()[-15:])
    assert r.returncode == 0, tail
    assert " passed" in r.stdout, tail
