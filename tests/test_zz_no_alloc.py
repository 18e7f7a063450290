"""md_forces_noalloc: forces for callers that may not allocate device memory.

Such callers (an out-of-memory handler that must still evaluate a
configuration, an application whose memory manager owns the whole device, code
certified to allocate nothing after start-up) get forces from one C call that
uses only their own arrays and a fixed scratch area inside the library.  This
test checks, through the C ABI, that the call returns the same forces, energies
and totals as md_compute_forces within the parity tolerances of the other GPU
tests, on two calls in a row (the second call reuses the scratch area the
first one left behind).  The file name makes pytest collect it last.
"""
import numpy as np
import pytest

from paper_0912_3824_gb300 import synth

TOL_F = {"fp64": 1e-12, "mixed": 1e-5}
TOL_E = {"fp64": 1e-13, "mixed": 1e-6}


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_noalloc_forces_match_compute_forces_on_two_calls(prec):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0912_3824_gb300 import build
    build.build()
    from paper_0912_3824_gb300 import md

    s = synth.perturb(synth.ka_mixture(n=3001, temperature=0.7, seed=9), 0.05, 19)
    sim = md.System.from_synth(s, dt=0.001, precision=md.PRECISIONS[prec])
    f_ref, e_ref, tot_ref = sim.forces()
    sim.close()

    dev = torch.device("cuda:0")
    species = torch.tensor(s.species, dtype=torch.int32, device=dev)
    pos = torch.tensor(s.pos, dtype=torch.float64, device=dev)
    force = torch.empty((s.n, 3), dtype=torch.float64, device=dev)
    energy = torch.empty(s.n, dtype=torch.float64, device=dev)
    totals = torch.empty(8, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    p = md.make_params(s.params, 0.001, precision=md.PRECISIONS[prec])
    rms = np.sqrt((f_ref ** 2).sum(axis=1).mean())
    for _ in range(2):
        force.fill_(float("nan"))
        totals.fill_(float("nan"))
        md.md_forces_noalloc(p, s.n, s.box, species.data_ptr(), pos.data_ptr(), force.data_ptr(),
                             energy.data_ptr(), totals.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        f = force.cpu().numpy()
        e = energy.cpu().numpy()
        t = totals.cpu().numpy()
        assert np.abs(f - f_ref).max() <= TOL_F[prec] * rms
        assert np.abs(e - e_ref).max() <= TOL_F[prec] * np.sqrt((e_ref ** 2).mean())
        assert abs(t[0] - tot_ref["e_pot"][0]) <= TOL_E[prec] * abs(tot_ref["e_pot"][0])
        assert abs(t[1] - tot_ref["virial"][0]) <= 10 * TOL_E[prec] * abs(tot_ref["virial"][0])
        assert np.allclose(t[2:], tot_ref["w"][0], rtol=0, atol=10 * TOL_E[prec] * abs(tot_ref["virial"][0]))


@pytest.mark.gpu
def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0912_3824_gb300 import md
    p = md.make_params(synth.ka_params(), 0.001)
    dev = torch.device("cuda:0")
    buf = torch.empty(16, dtype=torch.float64, device=dev)
    with pytest.raises(md.MDError) as ei:
        md.md_forces_noalloc(p, md.MD_NOALLOC_MAX_N + 1, 200.0, buf.data_ptr(), buf.data_ptr(),
                             buf.data_ptr(), 0, buf.data_ptr(), torch.cuda.current_stream(dev).cuda_stream)
    assert ei.value.code == md.MD_E_INVAL
