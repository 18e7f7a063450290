"""Host-side logic of bench.py that needs no GPU: the energy-drift estimate
and the lookup of the committed ncu traffic figure."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_0912_3824_gb300 import md  # noqa: E402


def _obs(steps, e_pot, e_kin):
    o = np.zeros(len(steps), dtype=md.OBS_DTYPE)
    o["step"], o["e_pot"], o["e_kin"] = steps, e_pot, e_kin
    return o


def test_energy_drift_recovers_a_linear_slope():
    """E/N = -5 + 1e-9 t (per step): slope relative to |E/N| = 2e-10; the largest
    deviation from the first sample is the whole rise."""
    n = 1000
    t = np.arange(0, 10001, 100)
    e = (-5.0 + 1e-9 * t) * n
    drift, maxdev = bench.energy_drift(_obs(t, e * 0.7, e * 0.3), n)
    mean = abs(np.mean(e / n))
    assert abs(drift - 1e-9 / mean) < 1e-15
    assert abs(maxdev - 1e-9 * 10000 / mean) < 1e-12


def test_energy_drift_needs_three_samples():
    assert bench.energy_drift(_obs([0, 100], [1.0, 1.0], [0.0, 0.0]), 10) == (None, None)


def test_profiled_traffic_only_for_the_captured_kernel_and_skin():
    """The committed summary covers one kernel at one skin, captured from the
    kernel sources whose hash it records: its figure is returned for exactly
    that kernel, skin and source state, None otherwise."""
    import hashlib
    fields = {}
    for line in open(os.path.join(ROOT, "profiles", "k_step_ka65536_mixed.md")):
        k, sep, v = line.partition(":")
        if sep and k in ("traffic_bytes_per_launch", "kernel", "skin", "source_sha256"):
            fields[k] = v.strip()
    kernel, skin = fields["kernel"], float(fields["skin"])
    now = " ".join(hashlib.sha256(open(os.path.join(ROOT, f), "rb").read()).hexdigest()
                   for f in bench.KERNEL_SOURCES)
    got = bench.profiled_traffic(kernel, skin)
    if now == fields["source_sha256"]:
        assert got == float(fields["traffic_bytes_per_launch"])
        assert 20e6 < got < 40e6                  # one cold launch at KA N=65536: list + state
    else:
        assert got is None                        # sources changed since the capture
    assert bench.profiled_traffic("k_step<0, 4, 0>", skin) is None
    assert bench.profiled_traffic(kernel, skin + 0.1) is None
