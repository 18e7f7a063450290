"""Python binding of the C ABI in include/md.h (argument marshalling only).

Every function below has the name of the C entry point it wraps and does no
computation of its own: all simulation work runs in the CUDA library
libmdgb300.so.  Importing this module raises if that library is missing -- there
is no CPU fallback.  PyTorch supplies the device workspace and the CUDA stream.

    from paper_0912_3824_gb300 import md, synth
    s = synth.ka_mixture(n=65536)
    sim = md.System.from_synth(s, dt=0.001, precision=md.MD_PREC_MIXED)
    sim.step(1000)
    obs = sim.observables()
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("MDGB300_LIB", os.path.join(_HERE, "libmdgb300.so"))

(MD_OK, MD_E_INVAL, MD_E_NOMEM, MD_E_CUDA, MD_E_NONFINITE, MD_E_UNSTABLE, MD_E_TIMEOUT, MD_E_CAPACITY,
 MD_E_BOUNDS) = range(9)
MD_PREC_FP64, MD_PREC_MIXED, MD_PREC_FP32 = 0, 1, 2
PRECISIONS = {"fp64": MD_PREC_FP64, "mixed": MD_PREC_MIXED, "fp32": MD_PREC_FP32}


class md_params(C.Structure):
    _fields_ = [("n_species", C.c_int32), ("shift", C.c_int32),
                ("eps", (C.c_double * 2) * 2), ("sigma", (C.c_double * 2) * 2),
                ("rcut", (C.c_double * 2) * 2), ("mass", C.c_double * 2),
                ("dt", C.c_double), ("skin", C.c_double),
                ("precision", C.c_int32), ("neigh_capacity", C.c_int32),
                ("sample_interval", C.c_int32), ("obs_capacity", C.c_int32),
                ("threads_per_particle", C.c_int32), ("use_graph", C.c_int32),
                ("reorder", C.c_int32), ("step_form", C.c_int32), ("smooth_h", C.c_double),
                ("check_interval", C.c_int32), ("neigh_capacity_max", C.c_int32),
                ("step_budget", C.c_int32), ("build_form", C.c_int32)]


class md_obs(C.Structure):
    _fields_ = [("step", C.c_int64), ("e_pot", C.c_double), ("e_kin", C.c_double),
                ("virial", C.c_double), ("w", C.c_double * 6), ("p", C.c_double * 3),
                ("max_disp", C.c_double), ("rebuilds", C.c_int64)]


class md_info_t(C.Structure):
    _fields_ = [("n_total", C.c_int64), ("n_replicas", C.c_int32),
                ("neigh_capacity", C.c_int32), ("threads_per_particle", C.c_int32),
                ("cells_per_edge", C.c_int32), ("step", C.c_int64), ("rebuilds", C.c_int64),
                ("kernel_launches", C.c_int64), ("max_neighbours", C.c_int32),
                ("status", C.c_int32), ("step_ms", C.c_double), ("step_launches", C.c_int64),
                ("rebuild_ms", C.c_double), ("rebuild_checks", C.c_int64),
                ("step_device_ms", C.c_double), ("step_device_launches", C.c_int64),
                ("check_interval", C.c_int32), ("neigh_capacity_max", C.c_int32),
                ("regrows", C.c_int64), ("build_form", C.c_int32), ("step_form", C.c_int32)]


OBS_DTYPE = np.dtype([("step", np.int64), ("e_pot", np.float64), ("e_kin", np.float64),
                      ("virial", np.float64), ("w", np.float64, (6,)), ("p", np.float64, (3,)),
                      ("max_disp", np.float64), ("rebuilds", np.int64)])
assert OBS_DTYPE.itemsize == C.sizeof(md_obs)


class MDError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"{_status_name(code)}: {message}")
        self.code = code


def _load() -> C.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library not built: {LIB_PATH} (run paper_0912_3824_gb300.build)")
    lib = C.CDLL(LIB_PATH)
    H = C.c_void_p
    P = C.POINTER(md_params)
    d = C.POINTER(C.c_double)
    i32 = C.POINTER(C.c_int32)
    i64 = C.POINTER(C.c_int64)
    sig = {
        "md_params_default": ([P], C.c_int),
        "md_workspace_size": ([P, C.c_int32, i64, d, C.POINTER(C.c_size_t)], C.c_int),
        "md_cell_order": ([P, C.c_int32, i64, d, i32, i32], C.c_int),
        "md_create": ([C.POINTER(H), P, C.c_int32, i64, d, i32, d, d, i32, C.c_void_p, C.c_size_t,
                       C.c_void_p], C.c_int),
        "md_step": ([H, C.c_int64], C.c_int),
        "md_rescale_velocities": ([H, d], C.c_int),
        "md_andersen": ([H, d, C.c_uint64, C.c_int64], C.c_int),
        "md_corr_workspace_size": ([H, C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_size_t)], C.c_int),
        "md_corr_create": ([C.POINTER(C.c_void_p), H, C.c_int32, C.c_int32, C.c_int32, d, C.c_void_p,
                            C.c_size_t], C.c_int),
        "md_corr_sample": ([C.c_void_p], C.c_int),
        "md_corr_result": ([C.c_void_p, i64, d, d, i64], C.c_int),
        "md_corr_destroy": ([C.c_void_p], C.c_int),
        "md_compute_forces": ([H, d, d, C.POINTER(md_obs)], C.c_int),
        "md_observables": ([H, C.POINTER(md_obs), C.c_int32, i32], C.c_int),
        "md_epot_series": ([H, i64, d, C.c_int32, i32], C.c_int),
        "md_get_state": ([H, d, d, i32], C.c_int),
        "md_set_state": ([H, d, d, i32], C.c_int),
        "md_get_neighbours": ([H, i32, i32, C.c_int32], C.c_int),
        "md_info": ([H, C.POINTER(md_info_t)], C.c_int),
        "md_sync": ([H], C.c_int),
        "md_destroy": ([H], C.c_int),
        "md_last_error": ([H], C.c_char_p),
        "md_status_string": ([C.c_int], C.c_char_p),
        "md_forces_noalloc": ([P, C.c_int64, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                               C.c_void_p, C.c_void_p], C.c_int),
        # measurement helper (include/md_bench.h)
        "md_fma_peak": ([C.c_int32, C.c_int64, d, d], C.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


_lib = _load()
EXPORTED = ("md_params_default", "md_workspace_size", "md_create", "md_step",
            "md_rescale_velocities", "md_compute_forces", "md_observables", "md_get_state",
            "md_set_state", "md_get_neighbours", "md_info", "md_sync", "md_destroy",
            "md_last_error", "md_status_string", "md_forces_noalloc", "md_andersen",
            "md_corr_workspace_size", "md_corr_create", "md_corr_sample", "md_corr_result",
            "md_corr_destroy", "md_cell_order", "md_epot_series")
MD_NOALLOC_MAX_N = 1048576
EXPORTED_BENCH = ("md_fma_peak",)


def _status_name(code: int) -> str:
    return _lib.md_status_string(code).decode()


def _check(rc: int, h=None):
    if rc != MD_OK:
        msg = _lib.md_last_error(h).decode() if h else ""
        raise MDError(rc, msg)


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def _iptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32)) if a is not None else None


def _f64(a, shape):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(shape))


def _i32(a, shape):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32).reshape(shape))


# ---------------------------------------------------------------------------
# one Python function per C entry point
# ---------------------------------------------------------------------------
def md_params_default() -> md_params:
    p = md_params()
    _check(_lib.md_params_default(C.byref(p)))
    return p


def md_workspace_size(p: md_params, n_per_replica, box) -> int:
    n = np.ascontiguousarray(n_per_replica, dtype=np.int64)
    b = np.ascontiguousarray(box, dtype=np.float64)
    out = C.c_size_t()
    _check(_lib.md_workspace_size(C.byref(p), len(n), n.ctypes.data_as(C.POINTER(C.c_int64)),
                                  _dptr(b), C.byref(out)))
    return out.value


def md_cell_order(p: md_params, n_per_replica, box):
    """Position along the cell curve of every cell (x, y, z) of replica 0, as an
    array [nc, nc, nc] indexed [z, y, x]."""
    nr = np.ascontiguousarray(n_per_replica, dtype=np.int64)
    bx = np.ascontiguousarray(box, dtype=np.float64)
    nc = C.c_int32()
    _check(_lib.md_cell_order(C.byref(p), len(nr), nr.ctypes.data_as(C.POINTER(C.c_int64)), _dptr(bx), None,
                              C.byref(nc)))
    rank = np.empty(nc.value ** 3, dtype=np.int32)
    _check(_lib.md_cell_order(C.byref(p), len(nr), nr.ctypes.data_as(C.POINTER(C.c_int64)), _dptr(bx),
                              _iptr(rank), C.byref(nc)))
    return rank.reshape(nc.value, nc.value, nc.value)


def md_create(p: md_params, n_per_replica, box, species, pos, vel, image, workspace_ptr: int,
              workspace_bytes: int, stream_ptr: int):
    n = np.ascontiguousarray(n_per_replica, dtype=np.int64)
    b = np.ascontiguousarray(box, dtype=np.float64)
    ntot = int(n.sum())
    sp = _i32(species, (ntot,))
    ps = _f64(pos, (ntot, 3))
    vs = _f64(vel, (ntot, 3))
    im = _i32(image, (ntot, 3)) if image is not None else None
    h = C.c_void_p()
    rc = _lib.md_create(C.byref(h), C.byref(p), len(n), n.ctypes.data_as(C.POINTER(C.c_int64)),
                        _dptr(b), _iptr(sp), _dptr(ps), _dptr(vs), _iptr(im),
                        C.c_void_p(workspace_ptr), workspace_bytes, C.c_void_p(stream_ptr))
    _check(rc)
    return h


def md_step(h, nsteps: int):
    _check(_lib.md_step(h, int(nsteps)), h)


def md_rescale_velocities(h, T_target):
    t = np.ascontiguousarray(T_target, dtype=np.float64)
    _check(_lib.md_rescale_velocities(h, _dptr(t)), h)


def md_andersen(h, T_target, seed: int, event: int):
    t = np.ascontiguousarray(T_target, dtype=np.float64)
    _check(_lib.md_andersen(h, _dptr(t), int(seed), int(event)), h)


def md_compute_forces(h, n_total: int, n_replicas: int):
    f = np.empty((n_total, 3))
    e = np.empty(n_total)
    tot = (md_obs * n_replicas)()
    _check(_lib.md_compute_forces(h, _dptr(f), _dptr(e), tot), h)
    return f, e, np.frombuffer(tot, dtype=OBS_DTYPE).copy()


def md_observables(h, n_replicas: int, max_samples: int = 1 << 16):
    buf = (md_obs * (max_samples * n_replicas))()
    n = C.c_int32()
    _check(_lib.md_observables(h, buf, max_samples, C.byref(n)), h)
    arr = np.frombuffer(buf, dtype=OBS_DTYPE)[: n.value * n_replicas].copy()
    return arr.reshape(n.value, n_replicas)


def md_epot_series(h, n_replicas: int, max_steps: int = 1 << 16):
    """(steps [n], e_pot [n, n_replicas]): the per-step potential energies
    recorded since the previous call, oldest first."""
    steps = np.empty(max_steps, dtype=np.int64)
    e = np.empty((max_steps, n_replicas))
    n = C.c_int32()
    _check(_lib.md_epot_series(h, steps.ctypes.data_as(C.POINTER(C.c_int64)), _dptr(e), max_steps, C.byref(n)), h)
    return steps[: n.value].copy(), e[: n.value].copy()


def md_get_state(h, n_total: int):
    pos = np.empty((n_total, 3))
    vel = np.empty((n_total, 3))
    img = np.empty((n_total, 3), dtype=np.int32)
    _check(_lib.md_get_state(h, _dptr(pos), _dptr(vel), _iptr(img)), h)
    return pos, vel, img


def md_set_state(h, pos, vel, image=None):
    n = np.asarray(pos).size // 3
    ps = _f64(pos, (n, 3))
    vs = _f64(vel, (n, 3))
    im = _i32(image, (n, 3)) if image is not None else None
    _check(_lib.md_set_state(h, _dptr(ps), _dptr(vs), _iptr(im)), h)


def md_get_neighbours(h, n_total: int, kmax: int):
    counts = np.empty(n_total, dtype=np.int32)
    lists = np.empty((n_total, kmax), dtype=np.int32)
    _check(_lib.md_get_neighbours(h, _iptr(counts), _iptr(lists), kmax), h)
    return counts, lists


def md_info(h) -> dict:
    out = md_info_t()
    _check(_lib.md_info(h, C.byref(out)), h)
    return {k: getattr(out, k) for k, _ in md_info_t._fields_}


def md_sync(h) -> int:
    """Returns the pending device status code (does not raise)."""
    return _lib.md_sync(h)


def md_destroy(h):
    _check(_lib.md_destroy(h))


def md_last_error(h) -> str:
    return _lib.md_last_error(h).decode()


def md_fma_peak(precision: int, iters: int = 2000) -> tuple[float, float]:
    """Measured CUDA-core FMA peak of the current GPU (md_bench.h): (TFLOP/s,
    ms of the fastest timed launch) for precision MD_PREC_FP64 or MD_PREC_FP32."""
    t = C.c_double()
    ms = C.c_double()
    rc = _lib.md_fma_peak(int(precision), int(iters), C.byref(t), C.byref(ms))
    if rc != 0:
        raise MDError(rc, "md_fma_peak failed")
    return t.value, ms.value


def md_forces_noalloc(p: md_params, n: int, box: float, species_ptr: int, pos_ptr: int, force_ptr: int,
                      energy_ptr: int, totals_ptr: int, stream_ptr: int):
    """Direct-sum forces without any device allocation; every pointer is a
    caller-owned device address (see md.h for the layouts)."""
    rc = _lib.md_forces_noalloc(C.byref(p), int(n), float(box), C.c_void_p(species_ptr),
                                C.c_void_p(pos_ptr), C.c_void_p(force_ptr),
                                C.c_void_p(energy_ptr) if energy_ptr else None,
                                C.c_void_p(totals_ptr), C.c_void_p(stream_ptr))
    if rc != MD_OK:          # the handle-free call keeps its message per thread
        raise MDError(rc, _lib.md_last_error(None).decode())


# ---------------------------------------------------------------------------
# convenience: parameters from the input generator's dictionaries, and a
# handle that owns its torch workspace
# ---------------------------------------------------------------------------
def make_params(pot: dict, dt: float, skin: float = 0.3, precision: int = MD_PREC_MIXED,
                sample_interval: int = 100, neigh_capacity: int = 0, threads_per_particle: int = 0,
                use_graph: bool = True, reorder: int = 1, obs_capacity: int = 0,
                check_interval: int = 0, neigh_capacity_max: int = 0, step_budget: int = 0,
                build_form: int = 0, step_form: int = 0) -> md_params:
    p = md_params_default()
    p.n_species = int(pot["n_species"])
    p.shift = 1 if pot.get("shift", True) else 0
    for a in range(2):
        for b in range(2):
            p.eps[a][b] = float(pot["eps"][a][b])
            p.sigma[a][b] = float(pot["sigma"][a][b])
            p.rcut[a][b] = float(pot["rcut"][a][b])
        p.mass[a] = float(pot["mass"][a])
    p.smooth_h = float(pot.get("smooth", 0.0))
    p.dt = float(dt)
    p.skin = float(skin)
    p.precision = int(precision)
    p.sample_interval = int(sample_interval)
    p.neigh_capacity = int(neigh_capacity)
    p.threads_per_particle = int(threads_per_particle)
    p.use_graph = 1 if use_graph else 0
    p.reorder = int(reorder)          # 0 x-fastest, 1 Morton, 2 Hilbert (True / False: 1 / 0)
    p.obs_capacity = int(obs_capacity)
    p.check_interval = int(check_interval)   # 0 automatic, else 1, 2, 4, 8, 16
    p.neigh_capacity_max = int(neigh_capacity_max)   # 0: twice the starting capacity
    p.step_budget = int(step_budget)         # 0: automatic bound of md_step's device loop
    p.build_form = int(build_form)           # 0 automatic, 1 warp per cell, 2 block per cell
    p.step_form = int(step_form)             # 0 automatic, 1 block per chunk, 2 resident blocks sweep
    return p


class System:
    """A handle plus the torch-owned device workspace it lives in."""

    def __init__(self, params: md_params, n_per_replica, box, species, pos, vel, image=None,
                 device: str = "cuda", stream=None):
        import torch
        self.params = params
        self.n_per_replica = np.ascontiguousarray(n_per_replica, dtype=np.int64)
        self.box = np.ascontiguousarray(box, dtype=np.float64)
        self.n = int(self.n_per_replica.sum())
        self.species = np.ascontiguousarray(species, dtype=np.int32)
        self.nrep = len(self.n_per_replica)
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        nbytes = md_workspace_size(params, self.n_per_replica, self.box)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        self.workspace_bytes = nbytes
        self.h = md_create(params, self.n_per_replica, self.box, species, pos, vel, image,
                           self._ws_ptr, nbytes, self.stream.cuda_stream)

    @classmethod
    def from_synth(cls, sysm, dt: float, **kw):
        device = kw.pop("device", "cuda")
        stream = kw.pop("stream", None)
        p = make_params(sysm.params, dt, **kw)
        return cls(p, [sysm.n], [sysm.box], sysm.species, sysm.pos, sysm.vel, sysm.image,
                   device=device, stream=stream)

    def step(self, n: int):
        md_step(self.h, n)

    def rescale(self, temperature):
        t = np.broadcast_to(np.asarray(temperature, dtype=np.float64), (self.nrep,))
        md_rescale_velocities(self.h, t)

    def andersen(self, temperature, seed: int, event: int):
        """One Andersen heat-bath collision of every particle (Sec. 2.3)."""
        t = np.broadcast_to(np.asarray(temperature, dtype=np.float64), (self.nrep,))
        md_andersen(self.h, t, seed, event)

    def forces(self):
        return md_compute_forces(self.h, self.n, self.nrep)

    def observables(self, max_samples: int = 1 << 16):
        return md_observables(self.h, self.nrep, max_samples)

    def epot_series(self, max_steps: int = 1 << 16):
        return md_epot_series(self.h, self.nrep, max_steps)

    def get_state(self):
        return md_get_state(self.h, self.n)

    def set_state(self, pos, vel, image=None):
        md_set_state(self.h, pos, vel, image)

    def neighbours(self, kmax: int | None = None):
        k = kmax if kmax is not None else self.info()["neigh_capacity"]
        return md_get_neighbours(self.h, self.n, k)

    def info(self) -> dict:
        return md_info(self.h)

    def sync(self) -> int:
        return md_sync(self.h)

    def close(self):
        if getattr(self, "h", None):
            md_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Correlator:
    """Blocking-scheme time-correlation functions (Sec. 2.5) of one System:
    k blocks of l entries, tagged-particle MSD and F_s over the wavevectors q
    ([n_q, 3]); the workspace is a torch tensor on the system's device."""

    def __init__(self, system: "System", k: int, l: int, q):
        import torch
        self.system = system
        self.k, self.l = int(k), int(l)
        self.q = np.ascontiguousarray(q, dtype=np.float64).reshape(-1, 3)
        nb = C.c_size_t()
        _check(_lib.md_corr_workspace_size(system.h, self.k, self.l, self.q.shape[0], C.byref(nb)), system.h)
        self.workspace = torch.empty(nb.value + 256, dtype=torch.uint8, device=system.workspace.device)
        ptr = (self.workspace.data_ptr() + 255) // 256 * 256
        c = C.c_void_p()
        _check(_lib.md_corr_create(C.byref(c), system.h, self.k, self.l, self.q.shape[0], _dptr(self.q),
                                   ptr, nb.value), system.h)
        self.c = c

    def sample(self):
        _check(_lib.md_corr_sample(self.c), self.system.h)

    def result(self):
        """lags [k, l-1] (samples), msd and fs [k, l-1, 2], origins [k, l-1]."""
        m = self.k * (self.l - 1)
        lags = np.empty(m, dtype=np.int64)
        org = np.empty(m, dtype=np.int64)
        msd = np.empty(2 * m)
        fs = np.empty(2 * m)
        _check(_lib.md_corr_result(self.c, lags.ctypes.data_as(C.POINTER(C.c_int64)), _dptr(msd), _dptr(fs),
                                   org.ctypes.data_as(C.POINTER(C.c_int64))), self.system.h)
        sh = (self.k, self.l - 1)
        return lags.reshape(sh), msd.reshape(sh + (2,)), fs.reshape(sh + (2,)), org.reshape(sh)

    def close(self):
        if getattr(self, "c", None):
            _lib.md_corr_destroy(self.c)
            self.c = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
