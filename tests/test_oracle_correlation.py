"""Pins for the blocking correlator of the oracle (Sec. 2.5) and the wavevector
shell of the input generator: closed forms for free flight, and the scheme
against a direct average over the same time origins."""
import math

import numpy as np
import pytest

from oracle.correlation import BlockingCorrelator, pair_sums
from paper_0912_3824_gb300 import synth


def test_shell_wavevectors_lie_on_the_reciprocal_lattice_near_q():
    L = 37.94
    q = synth.shell_wavevectors(L, 7.25, count=24, seed=3)
    n = q * L / (2 * math.pi)
    assert np.abs(n - np.round(n)).max() < 1e-9
    norm = np.linalg.norm(q, axis=1)
    assert np.abs(norm - 7.25).max() <= 0.5 * 2 * math.pi / L + 1e-12
    assert len({tuple(x) for x in np.round(n).astype(int)}) == 24
    assert np.array_equal(q, synth.shell_wavevectors(L, 7.25, count=24, seed=3))


def test_free_flight_msd_is_exact_and_fs_is_gaussian():
    """Ballistic motion r(t) = r(0) + v t: MSD(t) = <|v|^2> t^2 exactly, and for
    Maxwell-Boltzmann velocities F_s(q, t) = exp(-q^2 T t^2 / 2m) up to sampling
    noise (20000 particles x 16 wavevectors)."""
    n, T, dts = 20000, 0.6, 0.05
    st = synth.Stream(17)
    v = st.normal(3 * n).reshape(n, 3) * math.sqrt(T)
    r0 = st.uniform(3 * n).reshape(n, 3) * 30.0
    species = (np.arange(n) % 5 == 0).astype(np.int32)
    qv = synth.shell_wavevectors(30.0, 7.25, count=16, seed=1)
    c = BlockingCorrelator(3, 5, species, qv)
    for m in range(60):
        c.sample(r0 + v * (m * dts))
    lags, msd, fs, org = c.result()
    for a in (0, 1):
        v2 = (v[species == a] ** 2).sum(axis=1).mean()
        ok = org > 0
        assert np.allclose(msd[..., a][ok], v2 * (lags[ok] * dts) ** 2, rtol=1e-11)
        qq = (qv ** 2).sum(axis=1)
        ref = np.array([np.exp(-qq * T * (t * dts) ** 2 / 2).mean() for t in lags[ok]])
        assert np.abs(fs[..., a][ok] - ref).max() < 0.03
    assert (org[2] == 0).all()          # 60 samples cannot fill a block of spacing 25


def test_blocking_equals_direct_average_over_its_origins():
    """Block n correlates the origins m0 = t l^n with m0 + (l-1) l^n < M, each
    with its l-1 successors; the scheme's sums equal that direct double loop."""
    k, l, M, n = 3, 4, 137, 40
    st = synth.Stream(5)
    traj = np.cumsum(st.normal(M * n * 3).reshape(M, n, 3) * 0.1, axis=0)
    species = (np.arange(n) % 3 == 0).astype(np.int32)
    qv = synth.shell_wavevectors(12.0, 7.25, count=5, seed=2)
    c = BlockingCorrelator(k, l, species, qv)
    for m in range(M):
        c.sample(traj[m])
    for b in range(k):
        sp = l ** b
        origins = [m0 for m0 in range(0, M, sp) if m0 + (l - 1) * sp <= M - 1]
        for j in range(1, l):
            ref = sum((pair_sums(traj[m0], traj[m0 + j * sp], species, qv) for m0 in origins),
                      np.zeros((2, 3)))
            assert c.origins[b, j - 1] == len(origins)
            assert np.allclose(c.sums[b, j - 1], ref, rtol=1e-12, atol=1e-12)


def test_random_walk_msd_is_linear_in_time():
    """Gaussian increments of variance s^2 per component and sample: MSD(t) = 3 s^2 t."""
    n, M, s = 4000, 300, 0.05
    st = synth.Stream(8)
    traj = np.cumsum(st.normal(M * n * 3).reshape(M, n, 3) * s, axis=0)
    c = BlockingCorrelator(3, 6, np.zeros(n, np.int32), np.array([[1.0, 0.0, 0.0]]))
    for m in range(M):
        c.sample(traj[m])
    lags, msd, _, org = c.result()
    ok = org > 0
    assert np.allclose(msd[..., 0][ok], 3 * s * s * lags[ok], rtol=0.05)
