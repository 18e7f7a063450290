"""Pins for the FP64 CPU oracle, against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms
of the 12-6 potential (Sec. 3 definition), the parameter table printed in
Sec. 5, finite differences of its own energy, an independent lattice-sum
enumeration, an independent numpy distance matrix, exact symmetries (Newton's
third law, translation invariance, time reversibility of velocity Verlet) and
the harmonic limit of a bound dimer.  A dropped term, a wrong sign or index,
or a transposed parameter in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_0912_3824_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _lj_noshift():
    return synth.lj_params(shift=False)


# --------------------------------------------------------------------------
# pair potential: closed forms
# --------------------------------------------------------------------------

def test_lj_minimum_depth_and_position():
    """V_LJ has its minimum -eps at r = 2^(1/6) sigma, where the force vanishes."""
    rmin = 2.0 ** (1.0 / 6.0)
    v, fr = oracle.pair(_lj_noshift(), 0, 0, rmin * rmin)
    assert v == pytest.approx(-1.0, rel=1e-14)
    assert abs(fr) < 1e-13


def test_lj_zero_at_sigma_and_signs():
    v, fr = oracle.pair(_lj_noshift(), 0, 0, 1.0)
    assert abs(v) < 1e-15
    assert fr > 0                      # repulsive inside the minimum
    v2, fr2 = oracle.pair(_lj_noshift(), 0, 0, 1.5 ** 2)
    assert v2 < 0 and fr2 < 0          # attractive beyond it


def test_shift_constant_at_rc_2p5():
    """(sigma/r_c) = 0.4: V_LJ(r_c) = 4(0.4^12 - 0.4^6) = -0.016316891136 eps
    exactly in decimal, so the shifted potential at r = sigma is +0.016316891136."""
    v_shift, _ = oracle.pair(synth.lj_params(shift=True), 0, 0, 1.0)
    assert v_shift == pytest.approx(0.016316891136, rel=1e-12)
    v_raw, _ = oracle.pair(_lj_noshift(), 0, 0, 2.4999999999 ** 2)
    assert v_raw == pytest.approx(-0.016316891136, rel=1e-9)


def test_shifted_potential_continuous_at_cutoff_and_zero_beyond():
    p = synth.lj_params(shift=True)
    v_in, fr_in = oracle.pair(p, 0, 0, (2.5 * (1 - 1e-13)) ** 2)
    assert abs(v_in) < 1e-12
    assert fr_in < 0                    # the force jumps at r_c; the shift does not remove it
    v_out, fr_out = oracle.pair(p, 0, 0, 2.5 ** 2)   # r == r_c: strictly outside
    assert v_out == 0.0 and fr_out == 0.0


@pytest.mark.parametrize("r", [0.9, 1.0, 1.05, 1.122462, 1.3, 1.7, 2.2, 2.45])
def test_force_is_minus_derivative_of_potential(r):
    """fr = -V'(r)/r, checked by central differences of V."""
    p = _lj_noshift()
    h = 1e-6
    vp, _ = oracle.pair(p, 0, 0, (r + h) ** 2)
    vm, _ = oracle.pair(p, 0, 0, (r - h) ** 2)
    _, fr = oracle.pair(p, 0, 0, r * r)
    dvdr = (vp - vm) / (2 * h)
    assert -fr * r == pytest.approx(dvdr, rel=2e-7, abs=1e-8)


def test_ka_parameters_match_paper_table():
    rows = {}
    with open(os.path.join(GOLDEN, "ka_parameters.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, s, e = line.split()
                rows[k] = (float(s), float(e))
    p = synth.ka_params()
    idx = {"AA": (0, 0), "BB": (1, 1), "AB": (0, 1)}
    for k, (s, e) in rows.items():
        a, b = idx[k]
        assert p["sigma"][a][b] == s and p["sigma"][b][a] == s
        assert p["eps"][a][b] == e and p["eps"][b][a] == e
        assert p["rcut"][a][b] == pytest.approx(2.5 * s)
    assert p["mass"][0] == p["mass"][1]


@pytest.mark.parametrize("a,b", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_ka_pair_scaling(a, b):
    """V_ab(r) = eps_ab V_11(r / sigma_ab): minimum -eps_ab at 2^(1/6) sigma_ab and
    shift -0.016316891136 eps_ab at r_c = 2.5 sigma_ab, for every species pair."""
    p = synth.ka_params(shift=False)
    s, e = p["sigma"][a][b], p["eps"][a][b]
    rmin = 2.0 ** (1.0 / 6.0) * s
    v, fr = oracle.pair(p, a, b, rmin * rmin)
    assert v == pytest.approx(-e, rel=1e-14)
    assert abs(fr) < 1e-12
    ps = synth.ka_params(shift=True)
    v_sig, _ = oracle.pair(ps, a, b, s * s)
    assert v_sig == pytest.approx(0.016316891136 * e, rel=1e-12)
    v_out, _ = oracle.pair(ps, a, b, (2.5 * s * 1.0000001) ** 2)
    assert v_out == 0.0


# --------------------------------------------------------------------------
# N-body sums
# --------------------------------------------------------------------------

def _liquid(n, params, density, seed, amp=0.1, temperature=1.0):
    s = synth.make_system(n, density, temperature, seed, params)
    return synth.perturb(s, amp, seed + 1000)


def _fcc_vectors(a, rc):
    """All fcc lattice vectors 0 < |R| < rc (cubic cell a), by enumeration."""
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    m = int(math.ceil(rc / a)) + 1
    g = np.arange(-m, m + 1)
    cells = np.array(np.meshgrid(g, g, g, indexing="ij")).reshape(3, -1).T
    R = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3) * a
    d = np.linalg.norm(R, axis=1)
    return d[(d > 0) & (d < rc)]


@pytest.mark.parametrize("density,nc", [(0.8442, 4), (1.2, 5)])
def test_fcc_lattice_energy_virial_and_zero_force(density, nc):
    """On a perfect fcc lattice every force vanishes by symmetry, and the energy
    and virial per particle equal half the lattice sums over neighbour shells,
    enumerated here independently of the oracle's minimum-image loop."""
    p = synth.lj_params(shift=True)
    n = 4 * nc ** 3
    s = synth.make_system(n, density, 1.0, 3, p)
    a = s.box / nc
    for fn in (oracle.forces_brute, oracle.forces_cells):
        f, e, w7 = fn(p, s.box, s.species, s.pos)
        assert np.abs(f).max() < 1e-11
        d = _fcc_vectors(a, 2.5)
        vs = np.array([oracle.pair(p, 0, 0, x * x)[0] for x in d])
        frs = np.array([oracle.pair(p, 0, 0, x * x)[1] for x in d])
        assert e.sum() / n == pytest.approx(0.5 * vs.sum(), rel=1e-12)
        assert np.allclose(e, e[0], rtol=1e-12, atol=1e-14)
        assert w7[0] / n == pytest.approx(0.5 * (frs * d * d).sum(), rel=1e-12)
        # cubic symmetry: diagonal tensor entries equal, off-diagonal zero
        assert w7[1] == pytest.approx(w7[0] / 3, rel=1e-12)
        assert abs(w7[4]) < 1e-9 * abs(w7[0])


@pytest.mark.parametrize("n,density,kind", [(216, 0.8442, "lj"), (500, 0.8442, "lj"),
                                            (864, 0.8442, "lj"), (1000, 1.2, "ka"),
                                            (256, 1.2, "ka")])
def test_brute_force_equals_cell_list(n, density, kind):
    """Two independently written summations agree (216 and 256 particles give
    2 cells per edge, 500 gives 3)."""
    p = synth.lj_params() if kind == "lj" else synth.ka_params()
    s = _liquid(n, p, density, seed=11)
    fb, eb, wb = oracle.forces_brute(p, s.box, s.species, s.pos)
    fc, ec, wc = oracle.forces_cells(p, s.box, s.species, s.pos)
    scale = np.sqrt((fb ** 2).sum(axis=1).mean())
    assert np.abs(fb - fc).max() <= 1e-13 * scale * 10
    assert np.abs(eb - ec).max() <= 1e-13 * np.abs(eb).max() * 10
    assert np.allclose(wb, wc, rtol=1e-12, atol=1e-12 * abs(wb[0]))


@pytest.mark.parametrize("kind", ["lj", "ka"])
def test_newton_third_law_and_translation_invariance(kind):
    p = synth.lj_params() if kind == "lj" else synth.ka_params()
    s = _liquid(500 if kind == "lj" else 1000, p, 0.8442 if kind == "lj" else 1.2, seed=21)
    f, e, w = oracle.forces_cells(p, s.box, s.species, s.pos)
    scale = np.sqrt((f ** 2).sum(axis=1).mean())
    assert np.abs(f.sum(axis=0)).max() < 1e-12 * scale * s.n
    shift = np.array([0.3712, -1.234, 2.0])
    pos2 = np.mod(s.pos + shift, s.box)
    f2, e2, w2 = oracle.forces_cells(p, s.box, s.species, pos2)
    assert np.abs(f2 - f).max() < 1e-10 * scale
    assert e2.sum() == pytest.approx(e.sum(), rel=1e-12)


@pytest.mark.parametrize("kind", ["lj", "ka"])
def test_forces_are_minus_gradient_of_total_energy(kind):
    p = synth.lj_params() if kind == "lj" else synth.ka_params()
    s = _liquid(256, p, 0.8442 if kind == "lj" else 1.2, seed=31, amp=0.08)
    f, e, _ = oracle.forces_brute(p, s.box, s.species, s.pos)
    h = 1e-6
    rng = np.random.default_rng(0)
    for i in rng.choice(s.n, 6, replace=False):
        for k in range(3):
            pp = s.pos.copy(); pp[i, k] += h
            pm = s.pos.copy(); pm[i, k] -= h
            ep = oracle.forces_brute(p, s.box, s.species, pp)[1].sum()
            em = oracle.forces_brute(p, s.box, s.species, pm)[1].sum()
            assert -(ep - em) / (2 * h) == pytest.approx(f[i, k], rel=1e-5, abs=1e-5)


@pytest.mark.parametrize("kind", ["lj", "ka"])
def test_virial_is_minus_volume_scaling_derivative(kind):
    """E(lam) = sum V(lam r_ij) for positions and box scaled by lam gives
    dE/dlam at lam = 1 equal to  -W = -sum r_ij . F_ij."""
    p = synth.lj_params() if kind == "lj" else synth.ka_params()
    s = _liquid(500, p, 0.8442 if kind == "lj" else 1.2, seed=41)
    _, _, w7 = oracle.forces_cells(p, s.box, s.species, s.pos)
    h = 1e-6
    ep = oracle.forces_cells(p, s.box * (1 + h), s.species, s.pos * (1 + h))[1].sum()
    em = oracle.forces_cells(p, s.box * (1 - h), s.species, s.pos * (1 - h))[1].sum()
    assert (ep - em) / (2 * h) == pytest.approx(-w7[0], rel=1e-5)
    assert w7[1] + w7[2] + w7[3] == pytest.approx(w7[0], rel=1e-12)


def test_neighbour_pairs_match_numpy_distance_matrix():
    p = synth.ka_params()
    s = _liquid(300, p, 1.2, seed=51)
    skin = 0.3
    counts, lists = oracle.neighbours_brute(p, s.box, s.species, s.pos, skin, kmax=256)
    d = s.pos[:, None, :] - s.pos[None, :, :]
    d -= s.box * np.round(d / s.box)
    r = np.sqrt((d ** 2).sum(-1))
    rc = np.asarray(p["rcut"])[s.species[:, None], s.species[None, :]] + skin
    mask = (r < rc) & ~np.eye(s.n, dtype=bool)
    assert (counts == mask.sum(1)).all()
    for i in range(0, s.n, 17):
        assert set(lists[i, :counts[i]].tolist()) == set(np.nonzero(mask[i])[0].tolist())


# --------------------------------------------------------------------------
# velocity Verlet and reductions
# --------------------------------------------------------------------------

def test_synth_velocities_have_exact_temperature_and_zero_momentum():
    p = synth.ka_params()
    s = synth.ka_mixture(n=4000, temperature=0.7, seed=5)
    ek, mom = oracle.kinetic(p, s.species, s.vel)
    assert 2 * ek / (3 * s.n - 3) == pytest.approx(0.7, rel=1e-13)
    assert np.abs(mom).max() < 1e-11
    nb = int((s.species == 1).sum())
    assert nb == round(0.2 * 4000)


def test_rescale_sets_temperature_exactly():
    p = synth.lj_params()
    s = synth.lj_fluid(n=500, temperature=1.3, seed=2)
    v = oracle.rescale(p, s.species, s.vel * 1.7, 0.5)
    ek, _ = oracle.kinetic(p, s.species, v)
    assert 2 * ek / (3 * s.n - 3) == pytest.approx(0.5, rel=1e-14)


def _dimer(delta):
    p = synth.lj_params()
    L = 10.0
    rmin = 2.0 ** (1.0 / 6.0)
    pos = np.array([[5.0 - 0.5 * (rmin + delta), 5.0, 5.0], [5.0 + 0.5 * (rmin + delta), 5.0, 5.0]])
    return p, L, np.zeros(2, np.int32), pos, np.zeros((2, 3)), np.zeros((2, 3), np.int32)


def test_dimer_small_oscillation_period():
    """Harmonic limit of a bound LJ dimer: V''(r_min) = 72 * 2^(-1/3) eps/sigma^2,
    reduced mass m/2, so the period is 2 pi / sqrt(144 * 2^(-1/3))."""
    p, L, sp, pos, vel, img = _dimer(1e-3)
    dt, nsteps = 2e-4, 8000
    xs = []
    for _ in range(nsteps // 50):
        pos, vel, img, _, _ = oracle.vv_run(p, L, sp, pos, vel, img, dt, 50)
        xs.append(pos[1, 0] - pos[0, 0] - 2.0 ** (1.0 / 6.0))
    xs = np.array(xs)
    t = (np.arange(len(xs)) + 1) * 50 * dt
    zc = [t[k] - xs[k] * (t[k + 1] - t[k]) / (xs[k + 1] - xs[k])
          for k in range(len(xs) - 1) if xs[k] > 0 >= xs[k + 1]]
    period = np.diff(zc).mean()
    assert period == pytest.approx(2 * math.pi / math.sqrt(144 * 2 ** (-1.0 / 3.0)), rel=2e-3)


def test_energy_error_scales_as_dt_squared():
    """Velocity Verlet on a smooth orbit: max |E(t) - E(0)| over a fixed time
    drops by 4 when dt halves (Sec. 4.3)."""
    errs = []
    for dt in (0.004, 0.002):
        p, L, sp, pos, vel, img = _dimer(0.08)
        steps = int(round(2.0 / dt))
        *_, rec = oracle.vv_run(p, L, sp, pos, vel, img, dt, steps, sample=1)
        e = rec["e_pot"] + rec["e_kin"]
        errs.append(np.abs(e - e[0]).max())
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.1)


def test_verlet_time_reversibility_and_momentum():
    p = synth.lj_params()
    s = synth.perturb(synth.lj_fluid(n=256, temperature=0.722, seed=7), 0.05, 8)
    pos, vel, img, _, rec = oracle.vv_run(p, s.box, s.species, s.pos, s.vel, s.image,
                                          0.005, 200, sample=20)
    assert np.abs(rec["p"]).max() < 1e-11
    e = rec["e_pot"] + rec["e_kin"]
    assert np.abs(e - e[0]).max() < 2e-3 * abs(e[0])
    pos2, vel2, img2, _, _ = oracle.vv_run(p, s.box, s.species, pos, -vel, img, 0.005, 200)
    unwrapped0 = s.pos + s.image * s.box
    unwrapped2 = pos2 + img2 * s.box
    assert np.abs(unwrapped2 - unwrapped0).max() < 1e-8
    assert np.abs(-vel2 - s.vel).max() < 1e-8


def test_oracle_regression_fixture():
    """Oracle output for a fixed seeded 108-particle KA configuration, stored by
    tests/golden/make_golden.py (which calls only the oracle)."""
    path = os.path.join(GOLDEN, "oracle_ka108.txt")
    with open(path) as fh:
        lines = fh.readlines()
    w7_ref = np.array([float(x) for x in lines[2].split(":")[1].split()])
    tab = np.loadtxt(path, comments="#")
    p = synth.ka_params()
    s = _liquid(108, p, 1.2, seed=61)
    assert np.array_equal(s.species, tab[:, 0].astype(np.int32))
    assert np.allclose(s.pos, tab[:, 1:4], rtol=0, atol=1e-14)
    f, e, w7 = oracle.forces_brute(p, s.box, s.species, s.pos)
    assert np.allclose(f, tab[:, 4:7], rtol=0, atol=1e-12 * np.abs(tab[:, 4:7]).max())
    assert np.allclose(e, tab[:, 7], rtol=1e-13, atol=1e-14)
    assert np.allclose(w7, w7_ref, rtol=1e-13, atol=1e-12)


def test_dimer_period_scales_with_sqrt_mass():
    """Doubling both masses doubles the reduced mass: the period grows by sqrt(2)."""
    periods = []
    for m in (1.0, 2.0):
        p, L, sp, pos, vel, img = _dimer(1e-3)
        p = dict(p, mass=[m, m])
        dt = 2e-4
        xs = []
        for _ in range(240):
            pos, vel, img, _, _ = oracle.vv_run(p, L, sp, pos, vel, img, dt, 50)
            xs.append(pos[1, 0] - pos[0, 0] - 2.0 ** (1.0 / 6.0))
        xs = np.array(xs)
        t = (np.arange(len(xs)) + 1) * 50 * dt
        zc = [t[k] - xs[k] * (t[k + 1] - t[k]) / (xs[k + 1] - xs[k])
              for k in range(len(xs) - 1) if xs[k] > 0 >= xs[k + 1]]
        periods.append(np.diff(zc).mean())
    assert periods[1] / periods[0] == pytest.approx(math.sqrt(2.0), rel=2e-3)


def test_single_particle_force_matches_full_sum():
    p = synth.ka_params()
    s = _liquid(400, p, 1.2, seed=71)
    f, e, _ = oracle.forces_brute(p, s.box, s.species, s.pos)
    idx = [0, 5, 17, 399]
    f1, e1 = oracle.force_on(p, s.box, s.species, s.pos, idx)
    assert np.allclose(f1, f[idx], rtol=0, atol=1e-12 * np.abs(f).max())
    assert np.allclose(e1, e[idx], rtol=1e-13, atol=1e-14)


# --------------------------------------------------------------------------
# Sec. 4: purely repulsive WCA potential and the smoothing function
# g(x) = x^4 / (1 + x^4), x = (r - r_c) / (h sigma_ab)
# --------------------------------------------------------------------------

def test_wca_closed_forms():
    """WCA = V_LJ + eps cut at the minimum 2^(1/6) sigma: V(sigma) = eps, and
    both V and the force go to zero at r_c (the force is continuous there)."""
    p = synth.wca_params()
    v, fr = oracle.pair(p, 0, 0, 1.0)
    assert v == pytest.approx(1.0, rel=1e-14)
    assert fr == pytest.approx(24.0, rel=1e-14)          # 48 (1 - 1/2)
    rc = synth.WCA_RCUT
    v, fr = oracle.pair(p, 0, 0, (rc * (1 - 1e-9)) ** 2)
    assert 0 <= v < 1e-15 and abs(fr) < 1e-6
    assert oracle.pair(p, 0, 0, rc * rc) == (0.0, 0.0)


@pytest.mark.parametrize("shift", [True, False])
def test_smoothing_at_one_h_inside_cutoff(shift):
    """At x = -1: g = 1/2 and g'(x) = 4x^3/(1+x^4)^2 = -1, so the smoothed pair
    has V/2 and force factor fr/2 + V/(h sigma_ab r).  Checked on the KA A-B
    pair (sigma_AB = 0.8), which also fixes that the length scale of x is the
    pair's own sigma."""
    h = 0.005
    raw = synth.ka_params(shift=shift)
    smo = synth.ka_params(shift=shift, smooth=h)
    hs = h * 0.8
    r = 2.0 - hs                       # r_c,AB = 2.5 * 0.8
    v0, f0 = oracle.pair(raw, 0, 1, r * r)
    v1, f1 = oracle.pair(smo, 0, 1, r * r)
    assert v1 == pytest.approx(0.5 * v0, rel=1e-12)
    assert f1 == pytest.approx(0.5 * f0 + v0 / (hs * r), rel=1e-9)


@pytest.mark.parametrize("shift,pv,pf", [(False, 4, 3), (True, 5, 4)])
def test_smoothed_potential_vanishes_with_its_derivatives_at_cutoff(shift, pv, pf):
    """U = V g behaves as (r_c - r)^4 V(r_c) near the cutoff (as (r_c - r)^5
    when V(r_c) = 0 by the shift), its force one power lower: U, U' and U''
    all vanish at r_c, the C^2 continuity claimed in Sec. 4."""
    p = synth.lj_params(shift=shift, smooth=0.005)
    d = 0.005 * 1e-3
    v1, f1 = oracle.pair(p, 0, 0, (2.5 - d) ** 2)
    v2, f2 = oracle.pair(p, 0, 0, (2.5 - 2 * d) ** 2)
    assert v2 / v1 == pytest.approx(2.0 ** pv, rel=1e-2)
    assert f2 / f1 == pytest.approx(2.0 ** pf, rel=1e-2)
    assert abs(v1) < 1e-13 and abs(f1) < 1e-7


def test_smoothing_far_inside_cutoff_recovers_potential():
    """At x = -50, g = 50^4 / (1 + 50^4)."""
    h = 0.005
    r = 2.5 - 50 * h
    v0, _ = oracle.pair(synth.lj_params(), 0, 0, r * r)
    v1, _ = oracle.pair(synth.lj_params(smooth=h), 0, 0, r * r)
    assert v1 == pytest.approx(v0 * 50.0 ** 4 / (1 + 50.0 ** 4), rel=1e-13)


@pytest.mark.parametrize("params", [synth.lj_params(smooth=0.005), synth.wca_params(smooth=0.005),
                                    synth.ka_params(smooth=0.005)])
@pytest.mark.parametrize("frac", [0.9, 0.97, 0.995, 0.999])
def test_smoothed_force_is_minus_derivative(params, frac):
    """fr = -U'(r)/r by central differences, down to r_c - 0.25 h sigma."""
    for a, b in ((0, 0), (0, 1)) if params["n_species"] == 2 else ((0, 0),):
        rc = params["rcut"][a][b]
        r = rc * frac
        d = 1e-7
        vp, _ = oracle.pair(params, a, b, (r + d) ** 2)
        vm, _ = oracle.pair(params, a, b, (r - d) ** 2)
        _, fr = oracle.pair(params, a, b, r * r)
        assert -fr * r == pytest.approx((vp - vm) / (2 * d), rel=1e-5, abs=1e-8)


def test_wca_liquid_energy_error_scales_as_dt_squared():
    """Velocity Verlet on a smoothed WCA liquid (rho = 0.75, T = 1.12, the
    state point of Sec. 4): the largest energy deviation over a fixed time
    drops by 4 when dt halves."""
    s = synth.make_system(256, 0.75, 1.12, 11, synth.wca_params(smooth=0.005))
    pos, vel, img, _, _ = oracle.vv_run(s.params, s.box, s.species, s.pos, s.vel, s.image, 0.002, 300)
    errs = []
    for dt in (0.002, 0.001):
        *_, rec = oracle.vv_run(s.params, s.box, s.species, pos, vel, img, dt, int(round(0.4 / dt)),
                                sample=1)
        e = rec["e_pot"] + rec["e_kin"]
        errs.append(np.abs(e - e[0]).max())
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.25)


# --------------------------------------------------------------------------
# Sec. 2.3: rand48 with leapfrogging, and the Andersen heat bath
# --------------------------------------------------------------------------

def _libc():
    import ctypes
    import ctypes.util
    libc = ctypes.CDLL(ctypes.util.find_library("c") or None)
    libc.drand48.restype = ctypes.c_double
    libc.srand48.argtypes = [ctypes.c_long]
    return libc


@pytest.mark.parametrize("seed", [0, 1, 12345, 2 ** 31 + 7])
def test_rand48_matches_the_c_library(seed):
    """The oracle's rand48 against the C library's drand48 (an independent
    implementation of the same published recurrence), bit for bit."""
    libc = _libc()
    libc.srand48(seed)
    ref = np.array([libc.drand48() for _ in range(2000)])
    assert np.array_equal(oracle.rand48_uniforms(seed, 0, 2000), ref)
    assert np.array_equal(oracle.rand48_uniforms(seed, 1500, 500), ref[1500:])


@pytest.mark.parametrize("T", [1, 2, 7, 1000, 65536])
def test_rand48_leapfrog_equals_sequential_steps(T):
    """x_{n+T} = A_T x_n + C_T with A_T = a^T, C_T = c sum a^n (mod 2^48)."""
    A, Cc = oracle.rand48_leapfrog(T)
    if T == 1:
        assert (A, Cc) == (0x5DEECE66D, 0xB)
    for x in (0x330E, 0xFFFFFFFFFFFF, 0x123456789ABC, oracle.rand48_seed(99)):
        assert (A * x + Cc) % 2 ** 48 == oracle.rand48_step(x, T)


def test_andersen_draws_from_interleaved_leapfrog_streams():
    """Particle i of N uses the deviates (4e + k) N + i of the C library's
    drand48 sequence for collision e; Box-Muller, mean removal and exact
    rescaling then give the velocities."""
    n, seed, event, T = 50, 777, 2, 1.3
    libc = _libc()
    libc.srand48(seed)
    d = np.array([libc.drand48() for _ in range(4 * n * (event + 1))])
    u = d[4 * n * event:].reshape(4, n)
    r1, r2 = np.sqrt(-2 * np.log1p(-u[0])), np.sqrt(-2 * np.log1p(-u[2]))
    v = np.stack([r1 * np.cos(2 * np.pi * u[1]), r1 * np.sin(2 * np.pi * u[1]),
                  r2 * np.cos(2 * np.pi * u[3])], axis=1) * np.sqrt(T)
    v -= v.mean(axis=0)
    v *= np.sqrt(T * (3 * n - 3) / (v * v).sum())
    got = oracle.andersen(synth.lj_params(), np.zeros(n, np.int32), np.zeros((n, 3)), T, seed, event)
    assert np.abs(got - v).max() < 1e-13


def test_andersen_temperature_momentum_and_distribution():
    p = synth.ka_params()
    s = synth.ka_mixture(6000, temperature=1.0, seed=4)
    v = oracle.andersen(p, s.species, s.vel, 0.8, 4242, 0)
    ek, mom = oracle.kinetic(p, s.species, v)
    assert 2 * ek / (3 * s.n - 3) == pytest.approx(0.8, rel=1e-13)
    assert np.abs(mom).max() < 1e-11
    x = v.ravel() / np.sqrt(0.8)
    assert abs(np.mean(x ** 4) / np.mean(x ** 2) ** 2 - 3.0) < 0.15     # Gaussian kurtosis
    v2 = oracle.andersen(p, s.species, s.vel, 0.8, 4242, 1)
    assert np.abs(v2 - v).min() > 0 and abs(np.corrcoef(v.ravel(), v2.ravel())[0, 1]) < 0.05
    assert np.array_equal(v, oracle.andersen(p, s.species, s.vel, 0.8, 4242, 0))
