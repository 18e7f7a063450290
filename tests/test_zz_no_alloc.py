"""md_forces_noalloc: forces for callers that may not allocate device memory.

Such callers (an out-of-memory handler that must still evaluate a
configuration, an application whose memory manager owns the whole device, code
certified to allocate nothing after start-up) get forces from one C call that
uses only their own arrays and a fixed scratch area inside the library.  These
tests call it through the C ABI on two calls in a row (the second call reuses
the scratch area the first one left behind) and check it against the FP64
oracle's brute-force sum and against md_compute_forces, within the parity
tolerances of the other GPU tests.  The file name makes pytest collect it last.
"""
import numpy as np
import pytest

import oracle
from paper_0912_3824_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_F = {"fp64": 1e-12, "mixed": 1e-5}
TOL_E = {"fp64": 1e-13, "mixed": 1e-6}


@pytest.fixture(scope="module")
def md():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0912_3824_gb300 import build
    build.build()
    from paper_0912_3824_gb300 import md as m
    return m


def _device_arrays(s):
    import torch
    dev = torch.device("cuda:0")
    return dict(species=torch.tensor(s.species, dtype=torch.int32, device=dev),
                pos=torch.tensor(s.pos, dtype=torch.float64, device=dev),
                force=torch.empty((s.n, 3), dtype=torch.float64, device=dev),
                energy=torch.empty(s.n, dtype=torch.float64, device=dev),
                totals=torch.empty(8, dtype=torch.float64, device=dev),
                stream=torch.cuda.current_stream(dev))


def _call(md, p, s, d):
    import torch
    d["force"].fill_(float("nan"))
    d["energy"].fill_(float("nan"))
    d["totals"].fill_(float("nan"))
    md.md_forces_noalloc(p, s.n, s.box, d["species"].data_ptr(), d["pos"].data_ptr(), d["force"].data_ptr(),
                         d["energy"].data_ptr(), d["totals"].data_ptr(), d["stream"].cuda_stream)
    torch.cuda.synchronize()
    return d["force"].cpu().numpy(), d["energy"].cpu().numpy(), d["totals"].cpu().numpy()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("kind", ["ka", "lj"])
def test_noalloc_forces_match_oracle_and_compute_forces_on_two_calls(md, prec, kind):
    if kind == "ka":
        s = synth.perturb(synth.ka_mixture(n=3001, temperature=0.7, seed=9), 0.05, 19)
    else:       # one species: every code is 0
        s = synth.perturb(synth.lj_fluid(n=2000, temperature=1.0, seed=8), 0.05, 18)
    fr, er, w7 = oracle.forces_brute(s.params, s.box, s.species, s.pos)
    sim = md.System.from_synth(s, dt=0.001, precision=md.PRECISIONS[prec])
    f_ref, e_ref, tot_ref = sim.forces()
    sim.close()
    d = _device_arrays(s)
    p = md.make_params(s.params, 0.001, precision=md.PRECISIONS[prec])
    rms = np.sqrt((fr ** 2).sum(axis=1).mean())
    erms = np.sqrt((er ** 2).mean())
    for _ in range(2):
        f, e, t = _call(md, p, s, d)
        # against the oracle: the plain pair sum
        assert np.abs(f - fr).max() <= TOL_F[prec] * rms
        assert np.abs(e - er).max() <= TOL_F[prec] * erms
        assert abs(t[0] - er.sum()) <= TOL_E[prec] * abs(er.sum())
        assert abs(t[1] - w7[0]) <= 10 * TOL_E[prec] * abs(w7[0])
        assert np.allclose(t[2:], w7[1:], rtol=0, atol=10 * TOL_E[prec] * abs(w7[0]))
        # against the handle-based path
        assert np.abs(f - f_ref).max() <= TOL_F[prec] * rms
        assert abs(t[0] - tot_ref["e_pot"][0]) <= TOL_E[prec] * abs(tot_ref["e_pot"][0])


def test_noalloc_marks_a_species_code_out_of_range(md):
    """A species code the pair table does not have: the totals and that
    particle's force and energy come back NaN, the other particles' forces
    stay finite, and the next call with valid codes is clean again."""
    import torch
    s = synth.perturb(synth.ka_mixture(n=1000, temperature=0.7, seed=9), 0.05, 19)
    d = _device_arrays(s)
    p = md.make_params(s.params, 0.001, precision=md.MD_PREC_FP64)
    d["species"][123] = 5
    f, e, t = _call(md, p, s, d)
    assert np.isnan(t).all()
    assert np.isnan(f[123]).all() and np.isnan(e[123])
    assert np.isfinite(np.delete(f, 123, axis=0)).all()
    d["species"][123] = int(s.species[123])
    f, e, t = _call(md, p, s, d)
    assert np.isfinite(t).all() and np.isfinite(f).all()
    torch.cuda.synchronize()


def test_noalloc_rejects_sizes_beyond_its_scratch(md):
    import torch
    p = md.make_params(synth.ka_params(), 0.001)
    dev = torch.device("cuda:0")
    buf = torch.empty(16, dtype=torch.float64, device=dev)
    with pytest.raises(md.MDError) as ei:
        md.md_forces_noalloc(p, md.MD_NOALLOC_MAX_N + 1, 200.0, buf.data_ptr(), buf.data_ptr(),
                             buf.data_ptr(), 0, buf.data_ptr(), torch.cuda.current_stream(dev).cuda_stream)
    assert ei.value.code == md.MD_E_INVAL
    assert "MD_NOALLOC_MAX_N" in str(ei.value)
