"""GPU parity: the CUDA path against the FP64 CPU oracle, through the C ABI.

Tolerances (per call, identical configurations):
  forces       max_i |F_gpu - F_ref| / rms|F_ref|   <= 1e-12 (FP64), 1e-5 (MIXED)
  E_pot        |E_gpu - E_ref| / |E_ref|             <= 1e-13 (FP64), 1e-6 (MIXED)
  e_i          max_i |e_gpu - e_ref| / rms|e_ref|    <= 1e-12 (FP64), 1e-5 (MIXED)
FP32 (positions themselves single precision) is compared with the oracle
evaluated at the single-precision positions it actually holds; its remaining
error is the rounding of a pair separation across the periodic boundary, at
most ulp(L)/2 per component, so it gets 2e-4 on forces and 1e-5 on E_pot.
"""
import numpy as np
import pytest

import oracle
from paper_0912_3824_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_F = {"fp64": 1e-12, "mixed": 1e-5, "fp32": 2e-4}
TOL_E = {"fp64": 1e-13, "mixed": 1e-6, "fp32": 1e-5}


@pytest.fixture(scope="module")
def md():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0912_3824_gb300 import build
    build.build()
    from paper_0912_3824_gb300 import md as m
    return m


def _system(kind, n, seed=3, amp=0.1, temperature=None):
    if kind == "lj":
        s = synth.make_system(n, 0.8442, temperature or 0.722, seed, synth.lj_params())
    else:
        s = synth.make_system(n, 1.2, temperature or 0.7, seed, synth.ka_params())
    return synth.perturb(s, amp, seed + 100) if amp > 0 else s


def _sim(md, s, prec, dt=0.001, **kw):
    return md.System.from_synth(s, dt=dt, precision=md.PRECISIONS[prec], **kw)


def _ref_pos(s, prec):
    if prec == "fp32":
        return s.pos.astype(np.float32).astype(np.float64)
    return s.pos


def _ferr(f, ref):
    return np.abs(f - ref).max() / np.sqrt((ref ** 2).sum(axis=1).mean())


CASES = [("lj", 864), ("ka", 1000), ("ka", 4000), ("ka", 500), ("lj", 2000)]


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
@pytest.mark.parametrize("kind,n", CASES)
def test_forces_energy_virial_match_oracle(md, prec, kind, n):
    s = _system(kind, n)
    sim = _sim(md, s, prec)
    f, e, tot = sim.forces()
    fr, er, w7 = oracle.forces_cells(s.params, s.box, s.species, _ref_pos(s, prec))
    assert _ferr(f, fr) <= TOL_F[prec]
    assert abs(tot["e_pot"][0] - er.sum()) <= TOL_E[prec] * abs(er.sum())
    assert np.abs(e - er).max() <= TOL_F[prec] * np.sqrt((er ** 2).mean())
    assert abs(tot["virial"][0] - w7[0]) <= 10 * TOL_E[prec] * abs(w7[0]) + 1e-9
    assert np.allclose(tot["w"][0], w7[1:], rtol=0, atol=10 * TOL_E[prec] * abs(w7[0]) + 1e-9)
    ek, mom = oracle.kinetic(s.params, s.species, s.vel)
    assert tot["e_kin"][0] == pytest.approx(ek, rel=1e-6 if prec == "fp32" else 1e-13)
    # total momentum (velocities held as double-single in MIXED: exact to ~2^-48)
    assert np.abs(tot["p"][0] - mom).max() <= {"fp64": 1e-12, "mixed": 1e-10, "fp32": 1e-4}[prec]
    assert tot["max_disp"][0] == 0.0                  # lists just rebuilt
    sim.close()


def _melted(pot, n, density, temperature, seed=3, steps=300, dt=0.002):
    """fcc start melted by 300 oracle steps: a liquid configuration."""
    s = synth.make_system(n, density, temperature, seed, pot)
    s.pos, s.vel, s.image, _, _ = oracle.vv_run(s.params, s.box, s.species, s.pos, s.vel, s.image, dt, steps)
    return s


SMOOTH_CASES = [("lj", 0.005), ("ka", 0.005), ("wca", 0.005), ("wca", 0.0)]


def _smooth_system(kind, h):
    if kind == "lj":
        return _melted(synth.lj_params(smooth=h), 864, 0.8442, 1.0)
    if kind == "wca":                     # the state point of Sec. 4
        return _melted(synth.wca_params(smooth=h), 1000, 0.75, 1.12)
    return _melted(synth.ka_params(smooth=h), 1000, 1.2, 1.0)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
@pytest.mark.parametrize("kind,h", SMOOTH_CASES)
def test_smoothed_and_wca_forces_match_oracle(md, prec, kind, h):
    """Sec. 4 potentials: the C^2-smoothed LJ, KA and WCA pair sums and the plain
    WCA potential against the oracle."""
    s = _smooth_system(kind, h)
    sim = _sim(md, s, prec)
    f, e, tot = sim.forces()
    fr, er, w7 = oracle.forces_cells(s.params, s.box, s.species, _ref_pos(s, prec))
    assert _ferr(f, fr) <= TOL_F[prec]
    assert abs(tot["e_pot"][0] - er.sum()) <= TOL_E[prec] * abs(er.sum())
    assert np.abs(e - er).max() <= TOL_F[prec] * np.sqrt((er ** 2).mean())
    assert abs(tot["virial"][0] - w7[0]) <= 10 * TOL_E[prec] * abs(w7[0]) + 1e-9
    sim.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("mixed", 1e-5)])
def test_smoothed_wca_trajectory_matches_oracle(md, prec, tol):
    s = _smooth_system("wca", 0.005)
    pos, vel, img, obs, info = _trajectory(md, s, prec, 0.002, 200, 20)
    rp, rv, ri, _, rec = oracle.vv_run(s.params, s.box, s.species, s.pos, s.vel, s.image, 0.002, 200, sample=20)
    assert info["rebuilds"] >= 2
    assert np.abs((pos + img * s.box) - (rp + ri * s.box)).max() < tol
    assert np.allclose(obs["e_pot"], rec["e_pot"], rtol=1e-11 if prec == "fp64" else 1e-5)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_melted_liquid_forces(md, prec):
    """A configuration taken from an oracle trajectory (fcc melted for 300 steps)."""
    s = _system("ka", 2000, amp=0.0, temperature=1.5)
    pos, vel, img, _, _ = oracle.vv_run(s.params, s.box, s.species, s.pos, s.vel, s.image, 0.002, 300)
    s.pos, s.vel, s.image = pos, vel, img
    sim = _sim(md, s, prec)
    f, e, tot = sim.forces()
    fr, er, _ = oracle.forces_cells(s.params, s.box, s.species, s.pos)
    assert _ferr(f, fr) <= TOL_F[prec]
    assert abs(tot["e_pot"][0] - er.sum()) <= TOL_E[prec] * abs(er.sum())
    sim.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
def test_neighbour_lists_contain_all_pairs_within_list_radius(md, prec):
    s = _system("ka", 3000)
    skin = 0.3
    sim = _sim(md, s, prec)
    counts, lists = sim.neighbours()
    inner, inner_l = oracle.neighbours_brute(s.params, s.box, s.species, s.pos, skin - 1e-4, kmax=256)
    outer, outer_l = oracle.neighbours_brute(s.params, s.box, s.species, s.pos, skin + 1e-3, kmax=256)
    assert (counts >= inner).all() and (counts <= outer).all()
    for i in range(0, s.n, 7):
        got = set(lists[i, :counts[i]].tolist())
        assert set(inner_l[i, :inner[i]].tolist()) <= got <= set(outer_l[i, :outer[i]].tolist())
        assert len(got) == counts[i]       # no duplicates
    sim.close()


def _trajectory(md, s, prec, dt, nsteps, sample, **kw):
    sim = _sim(md, s, prec, dt=dt, sample_interval=sample, **kw)
    sim.step(nsteps)
    assert sim.sync() == md.MD_OK
    pos, vel, img = sim.get_state()
    obs = sim.observables()
    info = sim.info()
    sim.close()
    return pos, vel, img, obs[:, 0], info


@pytest.mark.parametrize("use_graph,check", [(True, 0), (False, 0), (True, 1), (True, 16)])
def test_fp64_trajectory_matches_oracle(md, use_graph, check):
    """200 velocity-Verlet steps of the LJ fluid (several list rebuilds), with
    the rebuild checked every 4 steps (the automatic interval here), every
    step, and every 16 steps."""
    s = _system("lj", 864, amp=0.02)
    pos, vel, img, obs, info = _trajectory(md, s, "fp64", 0.005, 200, 20, use_graph=use_graph,
                                           check_interval=check)
    assert info["check_interval"] == (check or 4)
    rp, rv, ri, _, rec = oracle.vv_run(s.params, s.box, s.species, s.pos, s.vel, s.image, 0.005, 200,
                                       sample=20)
    assert info["rebuilds"] >= 3
    assert np.abs((pos + img * s.box) - (rp + ri * s.box)).max() < 1e-9
    assert np.abs(vel - rv).max() < 1e-8
    assert (obs["step"] == rec["step"]).all()
    assert np.allclose(obs["e_pot"], rec["e_pot"], rtol=1e-11)
    assert np.allclose(obs["e_kin"], rec["e_kin"], rtol=1e-11)
    assert np.abs(obs["p"]).max() < 1e-10


@pytest.mark.parametrize("prec,tpp", [("fp64", 4), ("mixed", 4), ("mixed", 8), ("mixed", 2), ("fp32", 4)])
def test_ragged_particle_count_trajectory(md, prec, tpp):
    """N = 1001: the last warp of the step kernel holds padding lanes."""
    s = _system("ka", 1001, amp=0.03)
    pos, vel, img, obs, info = _trajectory(md, s, prec, 0.002, 40, 10, threads_per_particle=tpp)
    rp, rv, ri, _, rec = oracle.vv_run(s.params, s.box, s.species, s.pos, s.vel, s.image, 0.002, 40, sample=10)
    tol = {"fp64": 1e-9, "mixed": 1e-5, "fp32": 1e-3}[prec]
    assert np.abs((pos + img * s.box) - (rp + ri * s.box)).max() < tol
    assert np.allclose(obs["e_pot"], rec["e_pot"], rtol=1e-11 if prec == "fp64" else 1e-5)


def test_mixed_trajectory_close_to_oracle(md):
    s = _system("ka", 2000, amp=0.02)
    pos, vel, img, obs, info = _trajectory(md, s, "mixed", 0.001, 300, 50)
    rp, rv, ri, _, rec = oracle.vv_run(s.params, s.box, s.species, s.pos, s.vel, s.image, 0.001, 300,
                                       sample=50)
    assert np.abs((pos + img * s.box) - (rp + ri * s.box)).max() < 1e-5
    e_gpu = obs["e_pot"] + obs["e_kin"]
    e_ref = rec["e_pot"] + rec["e_kin"]
    assert np.allclose(e_gpu, e_ref, rtol=1e-6)
    assert np.abs(obs["p"]).max() < 1e-6 * s.n


@pytest.mark.parametrize("prec,steps,tol", [("fp64", 100, 1e-11), ("mixed", 50, 1e-6)])
@pytest.mark.parametrize("use_graph", [True, False])
def test_epot_every_step_matches_oracle(md, prec, steps, tol, use_graph):
    """The potential energy at every MD step (a per-step reduction of Sec. 2.2),
    against the oracle's trajectory sampled at every step; at the sample steps
    it equals the e_pot of the observables record bit for bit; a second call
    returns only the steps recorded since the first."""
    s = _system("lj", 864, amp=0.02)
    sim = _sim(md, s, prec, dt=0.005, sample_interval=10, use_graph=use_graph)
    sim.step(steps)
    assert sim.sync() == md.MD_OK
    st, e = sim.epot_series()
    obs = sim.observables()[:, 0]
    _, _, _, _, rec = oracle.vv_run(s.params, s.box, s.species, s.pos, s.vel, s.image, 0.005, steps, sample=1)
    assert np.array_equal(st, np.arange(steps + 1))
    assert np.abs(e[:, 0] - rec["e_pot"]).max() <= tol * np.abs(rec["e_pot"]).max()
    assert np.array_equal(e[obs["step"], 0], obs["e_pot"])
    sim.step(7)
    st2, e2 = sim.epot_series()
    assert np.array_equal(st2, np.arange(steps + 1, steps + 8))
    assert sim.epot_series()[0].size == 0
    sim.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
def test_max_displacement_matches_host_displacement(md, prec):
    """max_disp of a sample record is the largest displacement of that step's
    positions from those of the last list build.  With a wide skin no rebuild
    happens in 30 steps, so it is max_i |r_i(t) - r_i(0)|, computed here from
    the oracle's trajectory (the device tests it in single precision against
    positions rounded at the build: a few 1e-6 sigma)."""
    s = _system("ka", 1000, amp=0.02)
    sim = _sim(md, s, prec, dt=0.001, sample_interval=10, skin=0.6)
    sim.step(30)
    assert sim.sync() == md.MD_OK
    assert sim.info()["rebuilds"] == 1              # the build of md_create only
    obs = sim.observables()[:, 0]
    sim.close()
    r0 = s.pos + s.image * s.box
    for t, got in zip(obs["step"], obs["max_disp"]):
        rp, _, ri, _, _ = oracle.vv_run(s.params, s.box, s.species, s.pos, s.vel, s.image, 0.001, int(t))
        want = np.sqrt((((rp + ri * s.box) - r0) ** 2).sum(axis=1)).max()
        assert abs(got - want) <= 2e-5, (t, got, want)
    assert obs["max_disp"][0] == 0.0 and obs["max_disp"][-1] > 1e-3


def test_e1_sparse_corner_trajectory(md):
    """The sparse corner of the performance measurement of Sec. 3: LJ at
    density 0.2, T = 1.5, skin 0.5, dt = 0.001, N = 1372 (4 x 7^3).  FP64
    follows the oracle trajectory; MIXED stays within the mixed tolerances."""
    s = synth.perturb(synth.lj_fluid(1372, density=0.2, temperature=1.5, seed=4), 0.05, 41)
    rp, rv, ri, _, rec = oracle.vv_run(s.params, s.box, s.species, s.pos, s.vel, s.image, 0.001, 300,
                                       sample=50)
    pos, vel, img, obs, info = _trajectory(md, s, "fp64", 0.001, 300, 50, skin=0.5)
    assert np.abs((pos + img * s.box) - (rp + ri * s.box)).max() < 1e-9
    assert np.allclose(obs["e_pot"], rec["e_pot"], rtol=1e-11)
    assert np.allclose(obs["p"], rec["p"], rtol=0, atol=1e-11)
    pos, vel, img, obs, info = _trajectory(md, s, "mixed", 0.001, 300, 50, skin=0.5)
    assert np.abs((pos + img * s.box) - (rp + ri * s.box)).max() < 1e-5
    assert np.allclose(obs["e_pot"] + obs["e_kin"], rec["e_pot"] + rec["e_kin"], rtol=1e-6)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
@pytest.mark.parametrize("kind,n,skin", [("ka", 4000, 0.3), ("lj", 2048, 0.3), ("ka", 6000, 0.9)])
def test_build_forms_give_the_same_lists_and_trajectory(md, prec, kind, n, skin):
    """The neighbour build with one warp per cell and with one block per cell
    (the handle picks by the cell count) write the same rows in the same
    order: equal lists at creation and equal positions after 200 steps with
    several rebuilds, bit for bit.  Skin 0.9 makes cells of ~45 particles, so
    the warp form takes each cell's particles in two batches of lanes."""
    s = _system(kind, n, amp=0.02)
    runs = []
    for form in (1, 2):
        sim = _sim(md, s, prec, dt=0.005 if kind == "lj" else 0.002, build_form=form, skin=skin)
        assert sim.info()["build_form"] == form
        counts, lists = sim.neighbours()
        sim.step(200 if skin < 0.5 else 1500)
        assert sim.sync() == md.MD_OK
        info = sim.info()
        pos, vel, img = sim.get_state()
        runs.append((counts, lists, pos, vel, img, info["rebuilds"]))
        sim.close()
    (c1, l1, p1, v1, i1, r1), (c2, l2, p2, v2, i2, r2) = runs
    assert np.array_equal(c1, c2) and np.array_equal(l1, l2)
    assert r1 == r2 and r1 >= (3 if skin < 0.5 else 1)
    assert np.array_equal(p1, p2) and np.array_equal(v1, v2) and np.array_equal(i1, i2)


@pytest.mark.parametrize("prec", ["mixed", "fp32"])
@pytest.mark.parametrize("kind,n,tpp,smooth", [("lj", 262144, 1, 0.0), ("ka", 4000, 2, 0.0), ("ka", 4000, 2, 0.005),
                                               ("lj", 300, 1, 0.0)])
def test_step_forms_give_the_same_trajectory(md, prec, kind, n, tpp, smooth):
    """The step kernel with one block per chunk and with the resident blocks
    sweeping runs of chunks compute every particle and every chunk's partial
    sums the same way: equal positions, velocities, images, samples and
    per-step energies after 150 steps with rebuilds, bit for bit.  LJ at
    N = 262,144 and 1 lane needs more blocks than are resident (the automatic
    choice is the sweep); the small systems force it on fewer chunks than
    resident blocks (N = 300: fewer chunks than SMs)."""
    s = _system(kind, n, amp=0.02)
    if smooth:
        s.params["smooth"] = smooth
    runs = []
    for form in (1, 2):
        sim = _sim(md, s, prec, dt=0.005 if kind == "lj" else 0.002, step_form=form, threads_per_particle=tpp,
                   sample_interval=10)
        assert sim.info()["step_form"] == form
        sim.step(150)
        assert sim.sync() == md.MD_OK
        info = sim.info()
        pos, vel, img = sim.get_state()
        st, e = sim.epot_series()
        runs.append((pos, vel, img, sim.observables(), st, e, info["rebuilds"]))
        sim.close()
    (p1, v1, i1, o1, s1, e1, r1), (p2, v2, i2, o2, s2, e2, r2) = runs
    assert r1 == r2 and r1 >= 2
    assert np.array_equal(p1, p2) and np.array_equal(v1, v2) and np.array_equal(i1, i2)
    assert np.array_equal(o1, o2)
    assert np.array_equal(s1, s2) and np.array_equal(e1, e2) and len(s1) == 151
    if n == 262144:
        auto = _sim(md, s, prec, dt=0.005, threads_per_particle=tpp)
        assert auto.info()["step_form"] == 2
        auto.close()


def test_automatic_build_form_follows_cells_per_sm_and_cell_occupancy(md):
    """The automatic neighbour build takes a warp per cell from 8 cells per SM
    with at most 32 particles per cell on average, a block per cell otherwise."""
    import torch
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    for kind, n in (("lj", 4096), ("lj", 32768), ("ka", 65536)):
        s = _system(kind, n, amp=0.0)
        sim = _sim(md, s, "mixed")
        info = sim.info()
        sim.close()
        ncell = info["cells_per_edge"] ** 3
        want = 1 if (ncell >= 8 * nsm and n <= 32 * ncell) else 2
        assert info["build_form"] == want, (kind, n, ncell)
    if nsm == 152:                      # GB300: the measured crossover
        for kind, n, form in (("lj", 4096, 2), ("ka", 65536, 1)):
            sim = _sim(md, _system(kind, n, amp=0.0), "mixed")
            assert sim.info()["build_form"] == form
            sim.close()


def test_step_form_two_needs_a_single_precision_pair_loop(md):
    s = _system("ka", 1000)
    for prec, tpp in (("fp64", 4), ("mixed", 4)):
        with pytest.raises(md.MDError) as ei:
            _sim(md, s, prec, step_form=2, threads_per_particle=tpp)
        assert ei.value.code == md.MD_E_INVAL
    sim = _sim(md, s, "fp64")
    assert sim.info()["step_form"] == 1
    sim.close()


def test_epot_series_with_many_replicas(md):
    """More than 8 replicas (each replica summed by one thread): every
    replica's per-step potential energy equals that of the same system run
    alone, within the summation-order rounding of FP64."""
    sizes = [500, 777, 1000, 640, 900, 512, 1500, 700, 1200, 850, 600, 1100]
    reps = [synth.perturb(synth.ka_mixture(n=m, temperature=0.7, seed=70 + r), 0.05, 170 + r)
            for r, m in enumerate(sizes)]
    p = md.make_params(reps[0].params, 0.002, precision=md.MD_PREC_FP64, sample_interval=25)
    cat = lambda f: np.concatenate([getattr(r, f) for r in reps])
    one = md.System(p, sizes, [r.box for r in reps], cat("species"), cat("pos"), cat("vel"), cat("image"))
    one.step(60)
    assert one.sync() == md.MD_OK
    st, e = one.epot_series()
    one.close()
    assert np.array_equal(st, np.arange(61)) and e.shape == (61, len(sizes))
    for k in (0, 5, 11):
        r = reps[k]
        alone = md.System(p, [r.n], [r.box], r.species, r.pos, r.vel, r.image)
        alone.step(60)
        st1, e1 = alone.epot_series()
        alone.close()
        assert np.array_equal(st1, st)
        assert np.allclose(e[:, k], e1[:, 0], rtol=1e-12, atol=0)


def test_epot_series_survives_force_evaluations_and_state_changes(md):
    """The energies of a step still awaiting their sum are added up before a
    force evaluation outside the loop reuses the partials: the series stays
    complete, one value per step, across md_compute_forces and md_set_state."""
    s = _system("ka", 1000, amp=0.02)
    sim = _sim(md, s, "mixed", dt=0.002, sample_interval=7)
    sim.step(31)
    f, e, tot = sim.forces()
    sim.step(20)
    pos, vel, img = sim.get_state()
    sim.set_state(pos, vel, img)
    sim.step(9)
    assert sim.sync() == md.MD_OK
    st, ep = sim.epot_series()
    obs = sim.observables()[:, 0]
    sim.close()
    assert np.array_equal(st, np.arange(61))
    assert np.array_equal(ep[obs["step"], 0], obs["e_pot"])
    assert abs(ep[31, 0] - tot["e_pot"][0]) <= 1e-6 * abs(tot["e_pot"][0])


def test_graph_and_stream_launches_agree_bitwise(md):
    s = _system("ka", 3000, amp=0.05)
    a = _trajectory(md, s, "mixed", 0.002, 150, 10, use_graph=True)
    b = _trajectory(md, s, "mixed", 0.002, 150, 10, use_graph=False)
    assert a[4]["rebuilds"] == b[4]["rebuilds"] >= 2
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    assert np.array_equal(a[3]["e_pot"], b[3]["e_pot"])


def test_repeated_runs_are_deterministic(md):
    s = _system("lj", 2000, amp=0.05)
    a = _trajectory(md, s, "fp64", 0.005, 100, 10)
    b = _trajectory(md, s, "fp64", 0.005, 100, 10)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_reorder_does_not_change_forces(md, prec):
    """Cells in x-fastest, Morton and Hilbert order: the same forces, and a short
    trajectory that stays together."""
    s = _system("ka", 4000)
    f0, _, t0 = _sim(md, s, prec, reorder=0).forces()
    for r in (1, 2):
        f1, _, t1 = _sim(md, s, prec, reorder=r).forces()
        assert _ferr(f1, f0) <= TOL_F[prec]
        assert t1["e_pot"][0] == pytest.approx(t0["e_pot"][0], rel=TOL_E[prec])
    a = _trajectory(md, s, prec, 0.002, 60, 20, reorder=2)
    b = _trajectory(md, s, prec, 0.002, 60, 20, reorder=0)
    assert np.abs((a[0] + a[2] * s.box) - (b[0] + b[2] * s.box)).max() < (1e-9 if prec == "fp64" else 1e-5)


@pytest.mark.parametrize("tpp", [1, 2, 4, 16, 32])
def test_threads_per_particle_variants(md, tpp):
    s = _system("ka", 1500)
    f, _, tot = _sim(md, s, "mixed", threads_per_particle=tpp).forces()
    fr, er, _ = oracle.forces_cells(s.params, s.box, s.species, s.pos)
    assert _ferr(f, fr) <= TOL_F["mixed"]
    assert abs(tot["e_pot"][0] - er.sum()) <= TOL_E["mixed"] * abs(er.sum())


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
def test_state_roundtrip(md, prec):
    s = _system("ka", 1000)
    sim = _sim(md, s, prec)
    pos, vel, img = sim.get_state()
    unwrapped = pos + img * s.box
    tol = {"fp64": 0.0, "mixed": 1e-12, "fp32": 4e-6}[prec]
    assert np.abs(unwrapped - (s.pos + s.image * s.box)).max() <= tol
    assert np.abs(vel - s.vel).max() <= {"fp64": 0.0, "mixed": 1e-12, "fp32": 1e-6}[prec]
    assert (pos >= 0).all() and (pos < s.box).all()
    # set_state with shifted positions, then read back
    sim.set_state(s.pos + 0.5, -s.vel)
    p2, v2, i2 = sim.get_state()
    assert np.abs((p2 + i2 * s.box) - (s.pos + 0.5)).max() <= max(tol, 1e-12) * 10
    assert np.abs(v2 + s.vel).max() <= {"fp64": 0.0, "mixed": 1e-12, "fp32": 1e-6}[prec]
    sim.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
def test_wrap_just_below_zero_keeps_unwrapped_position(md, prec):
    """A coordinate that leaves the box by less than half an ulp of L wraps to
    a value that rounds to L; the stored position and its image counter must
    still describe the same unwrapped point (perfect fcc lattice at rest, so
    the moving particle feels almost no force)."""
    s = synth.make_system(864, 0.8442, 0.0, 1, synth.lj_params())
    k = 0
    p0 = np.mod(s.pos - s.pos[k], s.box)      # translate the lattice: particle k at the origin
    assert (p0[k] == 0.0).all()
    vel = np.zeros_like(p0)
    vel[k, 0] = -1e-4                           # leaves the box by 1e-7 < ulp(L)/2 in FP32
    tol = 1e-5 if prec == "fp32" else 1e-9
    sim = md.System(md.make_params(s.params, 0.001, precision=md.PRECISIONS[prec]), [s.n], [s.box],
                    s.species, p0, vel, s.image)
    sim.step(1)
    pos, _, img = sim.get_state()
    assert (pos[:, 0] >= 0).all() and (pos[:, 0] <= s.box).all()
    assert pos[k, 0] + img[k, 0] * s.box == pytest.approx(-1e-7, abs=tol)
    # the same through set_state: a coordinate 1e-9 below zero
    p2 = p0.copy()
    p2[k, 0] = -1e-9
    sim.set_state(p2, np.zeros_like(p2))
    pos, _, img = sim.get_state()
    assert pos[k, 0] + img[k, 0] * s.box == pytest.approx(-1e-9, abs=tol)
    sim.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-12), ("fp32", 2e-6)])
def test_andersen_collision_matches_oracle(md, prec, tol):
    """Sec. 2.3 heat bath: the velocities drawn on the device (rand48 jump-ahead
    per particle) equal the oracle's sequential stream, whatever the particles'
    order in memory (10 steps re-sort them first)."""
    s = _system("ka", 3000)
    sim = _sim(md, s, prec)
    sim.step(10)
    sim.andersen(0.8, 4242, 3)
    _, vel, _ = sim.get_state()
    ref = oracle.andersen(s.params, s.species, s.vel, 0.8, 4242, 3)
    assert np.abs(vel - ref).max() <= tol * np.sqrt((ref ** 2).mean())
    ek, mom = oracle.kinetic(s.params, s.species, vel)
    assert 2 * ek / (3 * s.n - 3) == pytest.approx(0.8, rel=1e-12 if prec != "fp32" else 1e-6)
    assert np.abs(mom).max() < (1e-10 if prec != "fp32" else 1e-3)
    sim.close()


def test_andersen_replicas_share_one_leapfrog(md):
    """Two replicas in one handle: replica r's particles are the threads
    start_r + i of one leapfrog over all particles; each gets its own target."""
    p = synth.ka_params()
    a = synth.ka_mixture(500, temperature=0.7, seed=21)
    b = synth.ka_mixture(800, temperature=0.7, seed=22)
    cat = lambda f: np.concatenate([getattr(a, f), getattr(b, f)])
    sim = md.System(md.make_params(p, 0.001, precision=md.MD_PREC_FP64), [a.n, b.n], [a.box, b.box],
                    cat("species"), cat("pos"), cat("vel"), cat("image"))
    sim.andersen([0.5, 1.0], 99, 1)
    _, vel, _ = sim.get_state()
    ra = oracle.andersen(p, a.species, a.vel, 0.5, 99, 1, nthreads=1300, first_index=0)
    rb = oracle.andersen(p, b.species, b.vel, 1.0, 99, 1, nthreads=1300, first_index=500)
    assert np.abs(vel[:500] - ra).max() < 1e-12 and np.abs(vel[500:] - rb).max() < 1e-12
    sim.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_rescale_sets_temperature(md, prec):
    s = _system("ka", 2000)
    sim = _sim(md, s, prec)
    sim.step(10)
    sim.rescale(0.5)
    _, vel, _ = sim.get_state()
    ek, _ = oracle.kinetic(s.params, s.species, vel)
    assert 2 * ek / (3 * s.n - 3) == pytest.approx(0.5, rel=1e-12 if prec == "fp64" else 1e-7)
    sim.close()


def test_replicas_match_independent_systems(md):
    """Three replicas of different size and box in one handle: each one's forces
    and trajectory equal those of the oracle run on it alone."""
    systems = [_system("ka", n, seed=10 + k) for k, n in enumerate([700, 1500, 2222])]
    sizes = [x.n for x in systems]
    p = md.make_params(systems[0].params, 0.002, precision=md.MD_PREC_FP64, sample_interval=25)
    sim = md.System(p, sizes, [x.box for x in systems],
                    np.concatenate([x.species for x in systems]),
                    np.concatenate([x.pos for x in systems]), np.concatenate([x.vel for x in systems]))
    f, _, tot = sim.forces()
    off = np.cumsum([0] + sizes)
    for k, x in enumerate(systems):
        fr, er, _ = oracle.forces_cells(x.params, x.box, x.species, x.pos)
        assert _ferr(f[off[k]:off[k + 1]], fr) <= 1e-12
        assert tot["e_pot"][k] == pytest.approx(er.sum(), rel=1e-13)
    sim.step(100)
    assert sim.sync() == md.MD_OK
    pos, vel, img = sim.get_state()
    obs = sim.observables()
    for k, x in enumerate(systems):
        rp, rv, ri, _, rec = oracle.vv_run(x.params, x.box, x.species, x.pos, x.vel, x.image, 0.002, 100,
                                           sample=25)
        sl = slice(off[k], off[k + 1])
        assert np.abs((pos[sl] + img[sl] * x.box) - (rp + ri * x.box)).max() < 1e-9
        assert np.allclose(obs[:, k]["e_pot"], rec["e_pot"], rtol=1e-11)
    sim.close()


def test_momentum_conserved_over_long_mixed_run(md):
    s = _system("ka", 4000, amp=0.0, temperature=1.0)
    sim = _sim(md, s, "mixed", dt=0.002, sample_interval=500)
    sim.step(5000)
    assert sim.sync() == md.MD_OK
    obs = sim.observables()[:, 0]
    assert np.abs(obs["p"]).max() < 1e-7 * s.n
    e = obs["e_pot"] + obs["e_kin"]
    assert np.abs(e[2:] - e[2]).max() < 2e-4 * abs(e[2])
    sim.close()


def test_capacity_past_the_cap_is_reported(md):
    """A list longer than the cap neigh_capacity_max is the one capacity
    error (MD_E_CAPACITY), here at the first build of md_create."""
    s = _system("ka", 1000)
    with pytest.raises(md.MDError) as ei:
        _sim(md, s, "mixed", neigh_capacity=16, neigh_capacity_max=16)
    assert ei.value.code == md.MD_E_CAPACITY
    with pytest.raises(md.MDError) as ei:       # default cap: twice the start, still too small
        _sim(md, s, "mixed", neigh_capacity=16)
    assert ei.value.code == md.MD_E_CAPACITY


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
def test_capacity_grows_at_create_within_the_cap(md, prec):
    """A starting capacity far below the lists (fixed-size list of Sec. 2.2):
    the first build grows it on the device and is redone; the forces equal
    those of a handle created with room to spare, bit for bit."""
    s = _system("ka", 1000)
    sim = _sim(md, s, prec, neigh_capacity=16, neigh_capacity_max=256)
    info = sim.info()
    mx = info["max_neighbours"]
    assert info["regrows"] == 1
    assert info["neigh_capacity"] == min(256, -(-(mx + (mx + 3) // 4) // 8) * 8)
    assert info["neigh_capacity"] >= mx and info["neigh_capacity_max"] == 256
    f, e, tot = sim.forces()
    sim.close()
    ref = _sim(md, s, prec, neigh_capacity=256)
    fr, er, totr = ref.forces()
    assert ref.info()["regrows"] == 0
    ref.close()
    assert np.array_equal(f, fr) and np.array_equal(e, er)
    assert tot["e_pot"][0] == totr["e_pot"][0] and tot["virial"][0] == totr["virial"][0]


def _heated_run(md, s, nsteps, use_graph, **kw):
    sim = _sim(md, s, "mixed", dt=0.002, use_graph=use_graph, **kw)
    sim.rescale(2.0)
    sim.step(nsteps)
    return sim


@pytest.mark.parametrize("use_graph", [True, False])
def test_capacity_grows_during_a_run(md, use_graph):
    """A capacity that fits the start but not the heated liquid, with a cap to
    grow into: the run finishes with MD_OK, the capacity has grown in place
    (a redone build inside the CUDA graph's rebuild branch, or in the stream
    launches), and the trajectory equals that of a run with room to spare from
    the start, bit for bit (the list contents and their order do not depend on
    the capacity)."""
    s = _melted(synth.ka_params(), 2000, 1.2, 1.0)     # longest list 112 at the start, on a
    probe = _sim(md, s, "mixed")                        # multiple of 8: no slack in the capacity
    cap = (probe.info()["max_neighbours"] + 7) // 8 * 8
    probe.close()
    sim = _heated_run(md, s, 3000, use_graph, neigh_capacity=cap, neigh_capacity_max=2 * cap)
    assert sim.sync() == md.MD_OK
    info = sim.info()
    assert info["step"] == 3000
    assert info["regrows"] >= 1 and info["neigh_capacity"] > cap
    assert info["neigh_capacity"] >= info["max_neighbours"]
    pos, vel, img = sim.get_state()
    obs = sim.observables()
    sim.close()
    ref = _heated_run(md, s, 3000, use_graph, neigh_capacity=2 * cap)
    assert ref.sync() == md.MD_OK
    assert ref.info()["regrows"] == 0
    rp, rv, ri = ref.get_state()
    robs = ref.observables()
    ref.close()
    assert np.array_equal(pos, rp) and np.array_equal(img, ri) and np.array_equal(vel, rv)
    assert np.array_equal(obs["e_pot"], robs["e_pot"])


@pytest.mark.parametrize("use_graph", [True, False])
def test_overflow_past_the_cap_keeps_the_last_consistent_state(md, use_graph):
    """The same heated run with the capacity fixed (cap = start): the step loop
    stops at the rebuild whose list exceeds the cap, MD_E_CAPACITY is reported,
    and the buffers stay those of the last completed step (the build's last
    block does not make the half-written permutation current), so the
    positions equal those of an unconstrained run after the same number of
    steps."""
    s = _melted(synth.ka_params(), 2000, 1.2, 1.0)
    probe = _sim(md, s, "mixed")
    cap = (probe.info()["max_neighbours"] + 7) // 8 * 8
    probe.close()
    sim = _heated_run(md, s, 3000, use_graph, neigh_capacity=cap, neigh_capacity_max=cap)
    assert sim.sync() == md.MD_E_CAPACITY
    k = sim.info()["step"]
    assert 0 < k < 3000
    pos, _, img = sim.get_state()
    sim.close()
    ref = _heated_run(md, s, k, use_graph)
    assert ref.sync() == md.MD_OK
    rp, _, ri = ref.get_state()
    ref.close()
    assert np.isfinite(pos).all()
    assert np.array_equal(pos + img * s.box, rp + ri * s.box)


def test_instability_is_reported_and_state_kept(md):
    s = _system("lj", 864)
    sim = _sim(md, s, "fp64", dt=50.0)
    sim.step(5)
    assert sim.sync() == md.MD_E_UNSTABLE
    assert sim.sync() == md.MD_OK          # reported once
    info = sim.info()
    assert info["step"] <= 1
    sim.close()


@pytest.mark.parametrize("use_graph", [True, False])
def test_exhausted_step_budget_is_reported_and_state_kept(md, use_graph):
    """md_step's device loop is bounded.  With the bound lowered to 40 step-
    kernel executions (step_budget), md_step(100) stops inside the loop with
    MD_E_TIMEOUT, reported once, and the positions are those of an
    unconstrained run of the same number of steps."""
    s = _system("ka", 1000)
    sim = _sim(md, s, "mixed", step_budget=40, use_graph=use_graph)
    sim.step(100)
    assert sim.sync() == md.MD_E_TIMEOUT
    assert sim.sync() == md.MD_OK               # reported once
    k = sim.info()["step"]
    assert 30 <= k <= 42
    pos, _, img = sim.get_state()
    sim.close()
    ref = _sim(md, s, "mixed", use_graph=use_graph)
    ref.step(k)
    assert ref.sync() == md.MD_OK
    rp, _, ri = ref.get_state()
    ref.close()
    assert np.array_equal(pos + img * s.box, rp + ri * s.box)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
def test_nonfinite_state_is_reported(md, prec):
    """A NaN velocity planted on the host through md_set_state: the first drift
    makes that position non-finite, md_step stops with MD_E_NONFINITE (reported
    once), and the current positions stay those before the step."""
    s = _system("ka", 1000)
    sim = _sim(md, s, prec)
    pos, vel, img = sim.get_state()
    vel[17, 1] = np.nan
    sim.set_state(pos, vel, img)
    sim.step(50)
    assert sim.sync() == md.MD_E_NONFINITE
    assert sim.sync() == md.MD_OK
    assert sim.info()["step"] == 0
    p2, _, i2 = sim.get_state()
    sim.close()
    assert np.array_equal(p2 + i2 * s.box, pos + img * s.box)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
def test_overlapping_particles_are_reported(md, prec):
    """Two particles 1e-3 sigma apart (repulsion ~ 48 / r^13): the first step
    either overflows single precision (MD_E_NONFINITE) or throws a particle
    more than a quarter box (MD_E_UNSTABLE); the run stops at step 0 with
    finite positions."""
    s = _system("lj", 864)
    s.pos[5] = s.pos[4] + np.array([1e-3, 0.0, 0.0])
    sim = _sim(md, s, prec, dt=0.005)
    sim.step(10)
    assert sim.sync() in (md.MD_E_NONFINITE, md.MD_E_UNSTABLE)
    assert sim.info()["step"] == 0
    pos, _, _ = sim.get_state()
    sim.close()
    assert np.isfinite(pos).all()


def test_full_size_sampled_parity_ka65536(md):
    """The benchmark's system (KA, N = 65536, mixed, default launch shape):
    after 200 graph-driven steps, forces on 256 sampled particles equal the
    oracle's one-by-one brute-force sums; Newton's third law holds for the
    total; E_pot equals the oracle cell-list sum."""
    s = synth.ka_mixture(n=65536, temperature=0.7, seed=5)
    sim = _sim(md, s, "mixed", dt=0.001, sample_interval=100)
    sim.step(200)
    assert sim.sync() == md.MD_OK
    pos, vel, img = sim.get_state()
    f, e, tot = sim.forces()
    idx = np.random.default_rng(0).choice(s.n, 256, replace=False)
    fr, er = oracle.force_on(s.params, s.box, s.species, pos, idx)
    rms = np.sqrt((f ** 2).sum(axis=1).mean())
    assert np.abs(f[idx] - fr).max() <= TOL_F["mixed"] * rms
    assert np.abs(e[idx] - er).max() <= TOL_F["mixed"] * np.sqrt((e ** 2).mean())
    assert np.abs(f.sum(axis=0)).max() < 1e-3 * rms
    _, ec, _ = oracle.forces_cells(s.params, s.box, s.species, pos)
    assert abs(tot["e_pot"][0] - ec.sum()) <= TOL_E["mixed"] * abs(ec.sum())
    sim.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_correlator_matches_blocking_oracle(md, prec):
    """Sec. 2.5 blocking scheme on the device (snapshots, block bookkeeping,
    MSD and F_s sums) against the oracle fed with the same unwrapped states."""
    from oracle.correlation import BlockingCorrelator
    s = _system("ka", 2000, amp=0.05, temperature=1.0)
    sim = _sim(md, s, prec)
    q = synth.shell_wavevectors(s.box, 7.25, count=12, seed=3)
    corr = md.Correlator(sim, 3, 4, q)
    ref = BlockingCorrelator(3, 4, s.species, q)
    for _ in range(70):
        corr.sample()
        pos, _, img = sim.get_state()
        ref.sample(pos + img * s.box)
        sim.step(5)
    lags, msd, fs, org = corr.result()
    rl, rmsd, rfs, rorg = ref.result()
    assert np.array_equal(lags, rl) and np.array_equal(org, rorg)
    ok = org > 0
    assert ok.sum() >= 6
    assert np.allclose(msd[ok], rmsd[ok], rtol=1e-12, atol=0)
    assert np.abs(fs[ok] - rfs[ok]).max() < 1e-5
    assert np.isnan(msd[~ok]).all()
    corr.close()
    sim.close()


@pytest.mark.parametrize("use_graph", [True, False])
def test_step_kernel_device_timer(md, use_graph):
    """Every step-kernel launch adds its device duration (first block start to
    last block end) to md_info: one launch per MD step, graph or not."""
    s = _system("ka", 4000, amp=0.05)
    sim = _sim(md, s, "mixed", use_graph=use_graph)
    sim.step(10)
    a = sim.info()
    sim.step(200)
    b = sim.info()
    n = b["step_device_launches"] - a["step_device_launches"]
    assert n == 200
    per = (b["step_device_ms"] - a["step_device_ms"]) / n
    assert 1e-4 < per < 5.0
    sim.close()


def test_autotuner_picks_a_timed_candidate(md):
    """The autotuner times each candidate (lanes per particle x skin) on the
    caller's state and returns the fastest, with the list capacity set from the
    longest list seen; the tuned system runs and matches the oracle forces."""
    from paper_0912_3824_gb300 import tune
    s = _system("ka", 4000, amp=0.05)
    base = md.make_params(s.params, 0.001, precision=md.MD_PREC_MIXED)
    p, trials = tune.autotune(base, [s.n], [s.box], s.species, s.pos, s.vel, s.image,
                              lanes=(1, 2), skins=(0.25, 0.3), steps=100, repeats=2)
    assert len(trials) == 4 and all(t["status"] == "MD_OK" for t in trials)
    fastest = min(trials, key=lambda t: t["ms_per_step"])
    assert (p.threads_per_particle, p.skin) == (fastest["threads_per_particle"], fastest["skin"])
    assert p.neigh_capacity % 32 == 0 and p.neigh_capacity >= 1.25 * fastest["max_neighbours"]
    sim = md.System(p, [s.n], [s.box], s.species, s.pos, s.vel, s.image)
    f, _, _ = sim.forces()
    fr, _, _ = oracle.forces_cells(s.params, s.box, s.species, s.pos)
    assert _ferr(f, fr) <= TOL_F["mixed"]
    sim.step(200)
    assert sim.sync() == md.MD_OK
    sim.close()


@pytest.fixture(scope="module")
def ka65536_reference():
    """KA N=65536 start and the oracle's 24 velocity-Verlet steps from it (dt 0.002)."""
    s = synth.perturb(synth.ka_mixture(n=65536, temperature=0.7, seed=5), 0.05, 9)
    return s, oracle.vv_run(s.params, s.box, s.species, s.pos, s.vel, s.image, 0.002, 24, sample=8)


@pytest.mark.parametrize("prec,tpp,skin,tol", [("mixed", 2, 0.2, 2e-6), ("mixed", 0, 0.3, 2e-6),
                                               ("fp64", 4, 0.3, 1e-10)])
def test_full_size_step_kernel_trajectory_ka65536(md, ka65536_reference, prec, tpp, skin, tol):
    """The bench's system and launch shape (KA N=65536; the autotuner's usual
    pick of 2 lanes and skin 0.2, and the defaults): 24 steps of the step
    kernel in the CUDA graph, with list rebuilds, against the oracle's
    velocity Verlet from the same start; every particle's position and the
    sampled E_pot and E_kin."""
    s, (rp, rv, ri, _, rec) = ka65536_reference
    pos, vel, img, obs, info = _trajectory(md, s, prec, 0.002, 24, 8, threads_per_particle=tpp, skin=skin)
    assert info["rebuilds"] >= 2
    assert np.abs((pos + img * s.box) - (rp + ri * s.box)).max() < tol
    assert (obs["step"] == rec["step"]).all()
    assert np.allclose(obs["e_pot"], rec["e_pot"], rtol=1e-6 if prec == "mixed" else 1e-12)
    assert np.allclose(obs["e_kin"], rec["e_kin"], rtol=1e-6 if prec == "mixed" else 1e-12)


def _near_cutoff(params, box, species, pos, rel=1e-6):
    """Particles with a partner at |r^2 / r_c,ab^2 - 1| < rel: whether such a pair
    is inside the cutoff depends on the last rounding of r^2, so single and
    double precision may both be right and still disagree (the force jumps by
    F(r_c) there); the comparison leaves these particles out.  rel = 1e-6 is
    several times the single-precision rounding of r^2 (about 3e-7)."""
    from scipy.spatial import cKDTree
    rc = np.asarray(params["rcut"], dtype=np.float64)
    x = np.mod(pos, box)
    pr = cKDTree(x, boxsize=box).query_pairs(rc.max() * (1 + 1e-3), output_type="ndarray")
    d = x[pr[:, 0]] - x[pr[:, 1]]
    d -= box * np.rint(d / box)
    near = np.abs((d * d).sum(1) / rc[species[pr[:, 0]], species[pr[:, 1]]] ** 2 - 1.0) < rel
    return set(pr[near].ravel().tolist())


def test_full_size_replica_ensemble_sampled(md):
    """The 256-replica ensemble (N_r uniform in 500..8000, seed 4) in one handle:
    after 20 steps, six replicas (first, last and four drawn at random) equal
    their own oracle runs particle by particle (particles that met a pair at
    the cutoff within rounding are left out, see _near_cutoff)."""
    pytest.importorskip("scipy")
    sizes = synth.ensemble_sizes(256, 500, 8000, seed=4)
    reps = [synth.ka_mixture(n=m, temperature=0.8, seed=4000 + r) for r, m in enumerate(sizes)]
    cat = lambda f: np.concatenate([getattr(r, f) for r in reps])
    p = md.make_params(reps[0].params, 0.001, precision=md.MD_PREC_MIXED, sample_interval=10)
    sim = md.System(p, sizes, [r.box for r in reps], cat("species"), cat("pos"), cat("vel"), cat("image"))
    sim.step(20)
    assert sim.sync() == md.MD_OK
    pos, vel, img = sim.get_state()
    start = np.concatenate([[0], np.cumsum(sizes)])
    pick = [0, 255] + list(np.random.default_rng(1).choice(np.arange(1, 255), 4, replace=False))
    for r in pick:
        q = reps[r]
        rp, rv, ri = q.pos, q.vel, q.image
        skip = _near_cutoff(q.params, q.box, q.species, rp)
        for _ in range(20):
            rp, rv, ri, _, _ = oracle.vv_run(q.params, q.box, q.species, rp, rv, ri, 0.001, 1)
            skip |= _near_cutoff(q.params, q.box, q.species, rp)
        keep = np.setdiff1d(np.arange(q.n), np.fromiter(skip, dtype=np.int64, count=len(skip)))
        assert len(keep) >= q.n - 40
        sl = slice(start[r], start[r + 1])
        assert np.abs((pos[sl] + img[sl] * q.box) - (rp + ri * q.box))[keep].max() < 1e-6
        assert np.abs(vel[sl] - rv)[keep].max() < 1e-5
    sim.close()


def test_full_size_lj_1m_two_steps(md):
    """The largest size of the LJ sweep (N = 1,048,576, rho 0.8442, dt 0.005,
    mixed, default launch shape): two steps against the oracle, every
    particle."""
    s = synth.perturb(synth.lj_fluid(n=1048576, density=0.8442, temperature=1.0, seed=3), 0.03, 4)
    pos, vel, img, obs, info = _trajectory(md, s, "mixed", 0.005, 2, 1)
    assert info["check_interval"] == 1          # automatic from 262,144 particles on
    rp, rv, ri, _, rec = oracle.vv_run(s.params, s.box, s.species, s.pos, s.vel, s.image, 0.005, 2, sample=1)
    assert np.abs((pos + img * s.box) - (rp + ri * s.box)).max() < 1e-6
    assert np.allclose(obs["e_pot"], rec["e_pot"], rtol=1e-6)


# ---------------------------------------------------------------------------
# edge placements: pairs at the cutoff and at the list radius, and pairs that
# straddle a face, an edge or a corner of the periodic box
# ---------------------------------------------------------------------------
def _placed_pairs():
    """LJ (r_c = 2.5, list radius 2.8 at skin 0.3) in a box of 24: isolated
    pairs centred on a 4^3 grid of spacing 6 (centres at 0 lie on the faces,
    edges and corner of the box, so those pairs straddle the boundary); any two
    particles of different pairs are more than 3.2 apart."""
    rc, rl = 2.5, 2.8
    seps = [rc * (1 - 1e-5), rc * (1 + 1e-5), rl * (1 - 1e-5), rl * (1 + 1e-3), 1.12, 1.0, 0.95, 2.0]
    dirs = [np.array(d, dtype=np.float64) / np.linalg.norm(d) for d in
            ([1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 0], [1, 0, 1], [0, 1, 1], [1, 1, 1], [1, -1, 1])]
    L = 24.0
    pos, tags = [], []
    k = 0
    for i in range(4):
        for j in range(4):
            for m in range(4):
                c = np.array([6.0 * i, 6.0 * j, 6.0 * m])
                d = seps[k % len(seps)]
                u = dirs[(k // len(seps)) % len(dirs)]
                pos += [c - 0.5 * d * u, c + 0.5 * d * u]
                tags.append(d)
                k += 1
    pos = np.mod(np.array(pos), L)
    n = len(pos)
    s = synth.System(n=n, box=L, species=np.zeros(n, dtype=np.int32), pos=pos,
                     vel=np.zeros((n, 3)), image=np.zeros((n, 3), dtype=np.int32),
                     params=synth.lj_params(), seed=0)
    return s, np.repeat(np.array(tags), 2), rc, rl


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
def test_pairs_at_the_cutoff_and_across_the_box_faces(md, prec):
    """Forces of pairs 1e-5 inside and outside r_c, and of pairs across faces,
    edges and the corner of the box, against the oracle; a particle whose
    partner is just beyond r_c feels exactly zero force; the lists hold the
    partner just inside the list radius and not the one 1e-3 beyond it."""
    s, sep, rc, rl = _placed_pairs()
    sim = _sim(md, s, prec, skin=0.3)
    f, e, tot = sim.forces()
    counts, lists = sim.neighbours()
    sim.close()
    fr, er, _ = oracle.forces_brute(s.params, s.box, s.species, _ref_pos(s, prec))
    assert _ferr(f, fr) <= TOL_F[prec]
    outside = sep > rc
    assert (f[outside] == 0.0).all() and (np.abs(fr[outside]).max() == 0.0)
    assert (np.abs(f[sep == rc * (1 - 1e-5)]) > 0.0).any(axis=1).all()
    partner = np.arange(s.n) ^ 1
    listed = np.array([partner[i] in lists[i, :counts[i]] for i in range(s.n)])
    assert listed[sep < rl].all()
    assert not listed[sep > rl * 1.0005].any()
    assert (counts <= 1).all()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_lists_cover_the_cutoff_between_rebuilds(md, prec):
    """At arbitrary steps between rebuilds every pair inside r_c,ab is still in
    the list built earlier (the displacement criterion of Sec. 2.2)."""
    s = _system("ka", 3000, amp=0.05, temperature=1.5)
    sim = _sim(md, s, prec, dt=0.002, skin=0.3)
    seen = 0
    for n in (13, 29, 41):
        sim.step(n)
        assert sim.sync() == md.MD_OK
        pos, _, _ = sim.get_state()
        counts, lists = sim.neighbours()
        inner, inner_l = oracle.neighbours_brute(s.params, s.box, s.species, pos, -1e-6, kmax=256)
        for i in range(s.n):
            assert set(inner_l[i, :inner[i]].tolist()) <= set(lists[i, :counts[i]].tolist())
        seen += int(inner.sum())
    assert seen > 0
    sim.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-6)])
def test_checkpoint_and_resume(md, prec, tol):
    """A run stopped after 100 steps, its state read back (md_get_state, original
    order) and a new handle created from it continues like the uninterrupted
    run: positions and velocities after 200 steps agree to the rounding of a
    different list order (the resumed handle bins and builds afresh)."""
    s = _system("lj", 2000, amp=0.02)
    whole = _sim(md, s, prec, dt=0.004)
    whole.step(200)
    assert whole.sync() == md.MD_OK
    pa, va, ia = whole.get_state()
    whole.close()
    first = _sim(md, s, prec, dt=0.004)
    first.step(100)
    assert first.sync() == md.MD_OK
    pos, vel, img = first.get_state()
    first.close()
    ck = synth.System(n=s.n, box=s.box, species=s.species, pos=pos, vel=vel, image=img, params=s.params,
                      seed=s.seed)
    second = _sim(md, ck, prec, dt=0.004)
    second.step(100)
    assert second.sync() == md.MD_OK
    pb, vb, ib = second.get_state()
    second.close()
    assert np.abs((pa + ia * s.box) - (pb + ib * s.box)).max() < tol
    assert np.abs(va - vb).max() < 10 * tol
