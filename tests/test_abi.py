"""The C-ABI library loads, exports every entry point its header declares,
and its host-only calls (defaults, workspace sizing, argument checks) behave.
No GPU needed: nothing here launches a kernel."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def md():
    from paper_0912_3824_gb300 import build
    build.build()
    from paper_0912_3824_gb300 import md as m
    return m


def _declared():
    src = open(os.path.join(ROOT, "include", "md.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*(md_\w+)\s*\(", src, re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("md_create", "md_step", "md_observables", "md_compute_forces", "md_get_state",
                 "md_set_state", "md_rescale_velocities", "md_sync", "md_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(md):
    import ctypes
    lib = ctypes.CDLL(md.LIB_PATH)
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(_declared()) == set(md.EXPORTED)


def test_library_exports_the_measurement_helpers(md):
    """include/md_bench.h (the FMA-peak microbenchmark the roofline divides by)."""
    import ctypes
    src = open(os.path.join(ROOT, "include", "md_bench.h")).read()
    names = sorted(set(re.findall(r"^\s*int\s*(md_\w+)\s*\(", src, re.M)))
    assert names == sorted(md.EXPORTED_BENCH)
    lib = ctypes.CDLL(md.LIB_PATH)
    for name in names:
        assert hasattr(lib, name), name
    assert md._lib.md_fma_peak(1, 10, None, None) == 1          # argument checks come first


def test_bounds_checked_library_builds_and_exports_the_same_symbols(md):
    """The bounds-checked variant used by tests/test_bounds_checked.py compiles
    (nvcc cross-compiles without a GPU) and exports the same entry points."""
    import ctypes
    import shutil
    if shutil.which("nvcc") is None:
        pytest.skip("nvcc not available")
    from paper_0912_3824_gb300 import build
    lib = ctypes.CDLL(build.build(checked=True))
    for name in _declared():
        assert hasattr(lib, name), name


def test_params_default(md):
    p = md.md_params_default()
    assert p.n_species == 1 and p.shift == 1
    assert p.rcut[0][0] == 2.5 and p.dt == 0.005 and p.skin == 0.3
    assert p.precision == md.MD_PREC_MIXED and p.use_graph == 1


def test_workspace_size_grows_with_n_and_precision(md):
    from paper_0912_3824_gb300 import synth
    p = md.make_params(synth.ka_params(), 0.001, precision=md.MD_PREC_MIXED)
    a = md.md_workspace_size(p, [16384], [(16384 / 1.2) ** (1 / 3)])
    b = md.md_workspace_size(p, [65536], [(65536 / 1.2) ** (1 / 3)])
    assert 3.5 * a < b < 4.5 * a
    p64 = md.make_params(synth.ka_params(), 0.001, precision=md.MD_PREC_FP64)
    assert md.md_workspace_size(p64, [65536], [(65536 / 1.2) ** (1 / 3)]) > b * 0.9
    # neighbour lists dominate: K * 4 bytes per particle
    assert b > 65536 * 128 * 4


def test_workspace_holds_the_capacity_cap(md):
    """The list area is sized for the cap neigh_capacity_max, so the capacity
    can grow in place; 0 means twice the starting capacity."""
    from paper_0912_3824_gb300 import synth
    n, box = 65536, (65536 / 1.2) ** (1 / 3)
    sz = lambda **kw: md.md_workspace_size(md.make_params(synth.ka_params(), 0.001, **kw), [n], [box])
    fixed = sz(neigh_capacity=128, neigh_capacity_max=128)
    assert sz(neigh_capacity=128, neigh_capacity_max=200) - fixed == pytest.approx(4 * n * (200 - 128), abs=512)
    assert sz(neigh_capacity=128) - fixed == pytest.approx(4 * n * 128, abs=512)
    assert sz(neigh_capacity=128, neigh_capacity_max=129) - fixed == pytest.approx(4 * n * 8, abs=512)


@pytest.mark.parametrize("bad", ["box", "dt", "species", "tpp", "sample", "asym", "smooth", "smooth_tpp",
                                 "check3", "check32", "capmax", "capneg", "budget", "stepform", "sweep64", "sweep4",
                                 "form"])
def test_argument_checks(md, bad):
    from paper_0912_3824_gb300 import synth
    pot = synth.ka_params()
    kw = {}
    box = 20.0
    if bad == "box":
        box = 5.5          # < 2 (r_c,max + skin)
    if bad == "dt":
        kw["dt"] = -1.0
    p = md.make_params(pot, kw.get("dt", 0.001))
    if bad == "species":
        p.n_species = 3
    if bad == "tpp":
        p.threads_per_particle = 3
    if bad == "sample":
        p.sample_interval = 0
    if bad == "asym":
        p.eps[0][1] = 2.0
    if bad == "smooth":
        p.smooth_h = -0.005
    if bad == "smooth_tpp":              # smoothed kernels exist for 1..8 lanes per particle
        p.smooth_h = 0.005
        p.threads_per_particle = 16
    if bad in ("check3", "check32"):     # the check interval divides the 16 steps of a graph loop
        p.check_interval = 3 if bad == "check3" else 32
    if bad == "capmax":                  # the cap may not be below the starting capacity
        p.neigh_capacity, p.neigh_capacity_max = 128, 64
    if bad == "capneg":
        p.neigh_capacity = -8
    if bad == "budget":
        p.step_budget = -1
    if bad == "stepform":
        p.step_form = 3
    if bad == "sweep64":                 # the sweeping step kernel exists for the FP32 pair loops
        p.precision = md.MD_PREC_FP64
        p.step_form = 2
    if bad == "sweep4":                  # ... at 1 or 2 lanes per particle
        p.threads_per_particle = 4
        p.step_form = 2
    if bad == "form":
        p.build_form = 3
    with pytest.raises(md.MDError) as ei:
        md.md_workspace_size(p, [1000], [box])
    assert ei.value.code == md.MD_E_INVAL


def test_status_strings(md):
    assert md._status_name(md.MD_E_CAPACITY) == "MD_E_CAPACITY"
    assert md._status_name(99) == "MD_E_UNKNOWN"


def test_obs_record_layout(md):
    assert md.OBS_DTYPE.itemsize == 120


def test_params_layout_and_smoothing_field(md):
    """md_params keeps its 192-byte layout; the smoothing width travels from the
    potential dictionary into smooth_h."""
    import ctypes
    from paper_0912_3824_gb300 import synth
    assert ctypes.sizeof(md.md_params) == 192
    assert md.md_params.smooth_h.offset == 168
    assert md.md_params.check_interval.offset == 176
    assert md.md_params.neigh_capacity_max.offset == 180 and md.md_params.step_budget.offset == 184
    assert md.make_params(synth.lj_params(smooth=0.005), 0.001).smooth_h == 0.005
    assert md.make_params(synth.wca_params(), 0.001).rcut[0][0] == synth.WCA_RCUT


def test_noalloc_rejects_smoothing_before_touching_the_device(md):
    """The fixed-scratch entry point evaluates the plain potential only; the
    rejection happens in argument checking, before any CUDA call."""
    import ctypes
    from paper_0912_3824_gb300 import synth
    p = md.make_params(synth.lj_params(smooth=0.005), 0.001)
    buf = (ctypes.c_double * 64)()
    sp = (ctypes.c_int32 * 8)()
    addr = ctypes.addressof(buf)
    rc = md._lib.md_forces_noalloc(ctypes.byref(p), 8, ctypes.c_double(20.0), ctypes.addressof(sp), addr, addr,
                                   addr, addr, None)
    assert rc == md.MD_E_INVAL
    assert b"smoothed potential" in md._lib.md_last_error(None)


@pytest.mark.parametrize("case", ["null", "small_n", "big_n", "box", "species", "precision"])
def test_noalloc_argument_errors_carry_their_reason(md, case):
    """Every argument the host can check is checked before any CUDA call, and
    the reason is kept for md_last_error(NULL) (a fixed per-thread buffer)."""
    import ctypes
    from paper_0912_3824_gb300 import synth
    p = md.make_params(synth.ka_params(), 0.001)
    buf = (ctypes.c_double * 64)()
    addr = ctypes.addressof(buf)
    n, box, sp = 8, 20.0, addr
    want = {"null": b"null argument", "small_n": b"at least 2", "big_n": b"MD_NOALLOC_MAX_N",
            "box": b"box must", "species": b"n_species", "precision": b"precision"}[case]
    if case == "null":
        sp = None
    if case == "small_n":
        n = 1
    if case == "big_n":
        n = md.MD_NOALLOC_MAX_N + 1
    if case == "box":
        box = 4.0
    if case == "species":
        p.n_species = 3
    if case == "precision":
        p.precision = 7
    rc = md._lib.md_forces_noalloc(ctypes.byref(p), n, ctypes.c_double(box), sp, addr, addr, addr, addr, None)
    assert rc == md.MD_E_INVAL
    assert want in md._lib.md_last_error(None)


def _cells_in_order(md, reorder, box):
    from paper_0912_3824_gb300 import synth
    p = md.make_params(synth.ka_params(), 0.001, reorder=reorder)
    rank = md.md_cell_order(p, [int(1.2 * box ** 3)], [box])
    nc = rank.shape[0]
    order = np.argsort(rank.ravel())               # cells (linear x-fastest index) along the curve
    xyz = np.stack([order % nc, (order // nc) % nc, order // (nc * nc)], axis=1)
    assert np.array_equal(np.sort(rank.ravel()), np.arange(nc ** 3))     # a bijection
    return nc, rank, xyz


def test_hilbert_cell_order_steps_to_a_face_neighbour(md):
    """reorder = 2, 8 cells per edge (a power of two): consecutive cells along
    the Hilbert curve share a face, the defining property of the curve."""
    nc, _, xyz = _cells_in_order(md, 2, 23.0)
    assert nc == 8
    assert (np.abs(np.diff(xyz, axis=0)).sum(axis=1) == 1).all()


def test_hilbert_cell_order_in_a_cut_cube_mostly_steps_to_neighbours(md):
    """13 cells per edge: the curve of the enclosing 16^3 cube restricted to the
    box still steps to a face neighbour most of the time."""
    nc, _, xyz = _cells_in_order(md, 2, 37.94)
    assert nc == 13
    assert (np.abs(np.diff(xyz, axis=0)).sum(axis=1) == 1).mean() > 0.8


def test_morton_and_plain_cell_orders(md):
    nc, rank, xyz = _cells_in_order(md, 1, 23.0)
    assert {tuple(c) for c in xyz[:8]} == {(x, y, z) for x in (0, 1) for y in (0, 1) for z in (0, 1)}
    assert tuple(xyz[8]) == (2, 0, 0)               # x carries the lowest interleaved bit
    nc, rank, xyz = _cells_in_order(md, 0, 23.0)
    assert np.array_equal(rank.ravel(), np.arange(nc ** 3))
