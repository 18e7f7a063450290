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
    assert bench.profiled_traffic("k_step<0, 4, 0, 0>", skin) is None
    assert bench.profiled_traffic(kernel, skin + 0.1) is None


def _line(prec, drift, pmax, msd):
    return {"precision": prec, "energy_drift_per_step_rel": drift, "max_abs_momentum_per_particle": pmax,
            "msd_A": {str(k): v for k, v in msd.items()}}


def test_stats_summary_means_errors_and_z_scores():
    """Over independent runs: mean and standard error (sample std / sqrt(k)) per
    precision and quantity; z of a precision against the reference is the
    difference of means over the combined standard error; the MSD verdict
    holds only if every lag is within 3 standard errors."""
    lines = [_line("fp64", d, p, {10: m10, 100: m100}) for d, p, m10, m100 in
             [(1.0, 1e-9, 0.10, 1.00), (3.0, 3e-9, 0.12, 1.10), (2.0, 2e-9, 0.11, 1.05), (2.0, 2e-9, 0.11, 1.05)]]
    lines += [_line("mixed", d, p, {10: m10, 100: m100}) for d, p, m10, m100 in
              [(1.5, 1e-9, 0.10, 1.00), (2.5, 3e-9, 0.12, 1.10), (2.0, 2e-9, 0.11, 1.05), (2.0, 2e-9, 0.11, 1.05)]]
    lines += [_line("fp32", d, p, {10: m10, 100: m100}) for d, p, m10, m100 in
              [(9.0, 1e-7, 0.30, 1.00), (9.5, 3e-7, 0.31, 1.10), (9.2, 2e-7, 0.32, 1.05), (9.3, 2e-7, 0.30, 1.05)]]
    out = bench.stats_summary(lines)
    s64 = out["summary"]["fp64"]
    v = np.array([1.0, 3.0, 2.0, 2.0])
    assert s64["drift_per_step"]["mean"] == 2.0
    assert abs(s64["drift_per_step"]["se"] - v.std(ddof=1) / 2.0) < 1e-15
    assert s64["runs"] == 4 and s64["msd_A"]["10"]["n"] == 4
    mixed = out["comparison"]["mixed"]
    assert mixed["msd_A_within_3se"] and abs(mixed["z_msd_A"]["10"]) < 1e-9
    fp32 = out["comparison"]["fp32"]
    assert not fp32["msd_A_within_3se"] and fp32["z_msd_A"]["10"] > 3
    se32 = np.array([0.30, 0.31, 0.32, 0.30]).std(ddof=1) / 2
    se64 = np.array([0.10, 0.12, 0.11, 0.11]).std(ddof=1) / 2
    want = (0.3075 - 0.11) / np.sqrt(se32 ** 2 + se64 ** 2)
    assert abs(fp32["z_msd_A"]["10"] - want) < 1e-9
    assert abs(fp32["momentum_ratio"] - 100.0) < 1e-9


def test_paper_workload_constants_match_the_generators_and_bench():
    """The workload constants printed in the paper (tests/golden/paper_workloads.txt,
    each with its section) are the ones the input generator and the bench use."""
    from paper_0912_3824_gb300 import synth
    const = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "paper_workloads.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()[:2]
            const[k] = float(v)
    assert synth.lj_params()["rcut"][0][0] == const["lj_rcut_sigma"]
    ka = synth.ka_params()
    assert ka["rcut"][0][0] == const["lj_rcut_sigma"] * ka["sigma"][0][0]      # 2.5 sigma_ab
    s = synth.ka_mixture(n=int(const["ka_n_a"] + const["ka_n_b"]) // 100, temperature=0.5, seed=1)
    assert abs(s.n / s.box ** 3 - const["ka_density"]) < 1e-12
    assert abs((s.species == 1).mean() - const["ka_n_b"] / (const["ka_n_a"] + const["ka_n_b"])) < 1e-3
    # the performance sweep of Sec. 3, the stability protocol of Sec. 4 and the
    # Kob-Andersen time step of Sec. 5 as the bench runs them
    assert bench.E1 == {"temperature": const["lj_perf_temperature"], "dt": const["lj_perf_dt"],
                        "skin": const["lj_perf_skin_gpu"]}
    st = bench.STABILITY
    assert (st["n"], st["density"], st["temperature"]) == (const["stab_n"], const["stab_density"],
                                                           const["stab_temperature"])
    assert bench.KA_DT == const["ka_dt"]


def test_median_of_groups():
    """Five consecutive groups of the timed iterations; the median of their means."""
    it = [1.0, 1.0, 2.0, 2.0, 3.0, 3.0, 4.0, 4.0, 9.0, 9.0]
    assert bench.median_of_groups(it) == 3.0
    assert bench.median_of_groups([1.0, 2.0]) is None
