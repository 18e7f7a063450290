"""FP64 CPU oracle for the molecular-dynamics step (test infrastructure).

TEST INFRASTRUCTURE ONLY: the reference that the CUDA library is checked
against.  Only the test-suite, the smoke check and the benchmark's CPU
baseline leg may import this package.  It never imports the CUDA library or
its Python binding, and the CUDA library never imports it.

The arithmetic lives in ``md_oracle.c`` (plain C, IEEE double, no fused
multiply-add); this module compiles it with gcc on first use and wraps it with
ctypes.  Potential parameters arrive as the plain dictionaries produced by the
seeded input generator.

Functions (all arrays float64 / int32, original particle order):
  pair(params, a, b, r2)                 -> (V, F/r) for one pair   (Sec. 3, 4, 5)
  forces_brute(params, L, species, pos)  -> (f[n,3], e[n], w7[7])   O(N^2)
  forces_cells(params, L, species, pos)  -> same, linked cells
  kinetic(params, species, vel)          -> (E_kin, P[3])
  vv_run(params, L, species, pos, vel, image, dt, nsteps, sample)
                                         -> (pos, vel, image, f, obs)  (Sec. 2.2)
  rescale(params, species, vel, T)       -> vel scaled to T         (Sec. 2.3)
  neighbours_brute(params, L, species, pos, skin, kmax)
                                         -> (counts[n], lists[n,kmax])
  rand48_seed / rand48_step / rand48_leapfrog / rand48_uniforms
                                         the rand48 generator and its leapfrog (Sec. 2.3)
  andersen(params, species, vel, T, seed, event)
                                         one Andersen heat-bath collision      (Sec. 2.3)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "md_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile md_oracle.c into oracle/liboracle.so (gcc, -ffp-contract=off)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Pot(C.Structure):
    _fields_ = [("n_species", C.c_int), ("shift", C.c_int),
                ("eps", C.c_double * 4), ("sigma", C.c_double * 4),
                ("rcut", C.c_double * 4), ("mass", C.c_double * 2), ("smooth_h", C.c_double)]


class _Obs(C.Structure):
    _fields_ = [("step", C.c_longlong), ("e_pot", C.c_double), ("e_kin", C.c_double),
                ("virial", C.c_double), ("w", C.c_double * 6), ("p", C.c_double * 3)]


OBS_FIELDS = ["step", "e_pot", "e_kin", "virial", "w", "p"]

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.POINTER(_Pot)
            lib.orc_pair.argtypes = [P, C.c_int, C.c_int, C.c_double,
                                     C.POINTER(C.c_double), C.POINTER(C.c_double)]
            lib.orc_pair.restype = C.c_int
            for fn in (lib.orc_forces_brute, lib.orc_forces_cells):
                fn.argtypes = [P, C.c_long, C.c_double, _ip, _dp, _dp, _dp, _dp]
                fn.restype = None
            lib.orc_kinetic.argtypes = [P, C.c_long, _ip, _dp, C.POINTER(C.c_double), _dp]
            lib.orc_kinetic.restype = None
            lib.orc_vv_run.argtypes = [P, C.c_long, C.c_double, _ip, _dp, _dp, _ip, _dp,
                                       C.c_double, C.c_longlong, C.c_longlong,
                                       C.POINTER(_Obs), C.c_long]
            lib.orc_vv_run.restype = C.c_long
            lib.orc_rescale.argtypes = [P, C.c_long, _ip, _dp, C.c_double]
            u64 = C.c_ulonglong
            lib.orc_rand48_seed.argtypes = [u64]
            lib.orc_rand48_seed.restype = u64
            lib.orc_rand48_step.argtypes = [u64, C.c_longlong]
            lib.orc_rand48_step.restype = u64
            lib.orc_rand48_leapfrog.argtypes = [C.c_longlong, C.POINTER(u64), C.POINTER(u64)]
            lib.orc_rand48_uniforms.argtypes = [u64, C.c_longlong, C.c_longlong, _dp]
            lib.orc_andersen.argtypes = [P, C.c_long, _ip, _dp, C.c_double, u64, C.c_longlong,
                                         C.c_longlong, C.c_longlong]
            lib.orc_rescale.restype = None
            lib.orc_neighbours_brute.argtypes = [P, C.c_long, C.c_double, _ip, _dp, C.c_double,
                                                 _ip, C.c_void_p, C.c_long]
            lib.orc_neighbours_brute.restype = C.c_long
            lib.orc_force_one.argtypes = [P, C.c_long, C.c_double, _ip, _dp, C.c_long, _dp,
                                          C.POINTER(C.c_double)]
            lib.orc_force_one.restype = None
            _lib = lib
    return _lib


def _pot(params: dict) -> _Pot:
    p = _Pot()
    p.n_species = int(params["n_species"])
    p.shift = 1 if params.get("shift", True) else 0
    for a in range(2):
        for b in range(2):
            p.eps[2 * a + b] = float(params["eps"][a][b])
            p.sigma[2 * a + b] = float(params["sigma"][a][b])
            p.rcut[2 * a + b] = float(params["rcut"][a][b])
    for a in range(2):
        p.mass[a] = float(params["mass"][a])
    p.smooth_h = float(params.get("smooth", 0.0))
    return p


def _f64(x, shape=None):
    a = np.ascontiguousarray(x, dtype=np.float64)
    return a if shape is None else a.reshape(shape)


def _i32(x, shape=None):
    a = np.ascontiguousarray(x, dtype=np.int32)
    return a if shape is None else a.reshape(shape)


def pair(params: dict, a: int, b: int, r2: float) -> tuple[float, float]:
    lib = _load()
    v, fr = C.c_double(), C.c_double()
    lib.orc_pair(C.byref(_pot(params)), a, b, float(r2), C.byref(v), C.byref(fr))
    return v.value, fr.value


def _forces(fn, params, box, species, pos):
    n = len(species)
    pos = _f64(pos, (n, 3)).copy()
    f = np.zeros((n, 3))
    e = np.zeros(n)
    w7 = np.zeros(7)
    fn(C.byref(_pot(params)), n, float(box), _i32(species), pos, f, e, w7)
    return f, e, w7


def forces_brute(params, box, species, pos):
    return _forces(_load().orc_forces_brute, params, box, species, pos)


def forces_cells(params, box, species, pos):
    return _forces(_load().orc_forces_cells, params, box, species, pos)


def force_on(params, box, species, pos, idx):
    """Brute-force force and energy share on each particle in idx: (f[k,3], e[k])."""
    n = len(species)
    pos = _f64(pos, (n, 3))
    sp = _i32(species)
    lib = _load()
    p = _pot(params)
    f = np.zeros((len(idx), 3))
    e = np.zeros(len(idx))
    f3 = np.zeros(3)
    ei = C.c_double()
    for k, i in enumerate(idx):
        lib.orc_force_one(C.byref(p), n, float(box), sp, pos, int(i), f3, C.byref(ei))
        f[k] = f3
        e[k] = ei.value
    return f, e


def kinetic(params, species, vel):
    n = len(species)
    ek = C.c_double()
    mom = np.zeros(3)
    _load().orc_kinetic(C.byref(_pot(params)), n, _i32(species), _f64(vel, (n, 3)),
                        C.byref(ek), mom)
    return ek.value, mom


def vv_run(params, box, species, pos, vel, image, dt, nsteps, sample=0):
    """Velocity-Verlet from (pos, vel, image); returns the final state, the
    final forces and a structured array of observables at steps 0, sample, ..."""
    n = len(species)
    pos = _f64(pos, (n, 3)).copy()
    vel = _f64(vel, (n, 3)).copy()
    image = _i32(image, (n, 3)).copy()
    f = np.zeros((n, 3))
    nobs = (nsteps // sample + 1) if sample > 0 else 0
    obs = (_Obs * max(nobs, 1))()
    nrec = _load().orc_vv_run(C.byref(_pot(params)), n, float(box), _i32(species), pos, vel,
                              image, f, float(dt), int(nsteps), int(sample), obs, nobs)
    rec = {
        "step": np.array([obs[k].step for k in range(nrec)], dtype=np.int64),
        "e_pot": np.array([obs[k].e_pot for k in range(nrec)]),
        "e_kin": np.array([obs[k].e_kin for k in range(nrec)]),
        "virial": np.array([obs[k].virial for k in range(nrec)]),
        "w": np.array([list(obs[k].w) for k in range(nrec)]).reshape(nrec, 6),
        "p": np.array([list(obs[k].p) for k in range(nrec)]).reshape(nrec, 3),
    }
    return pos, vel, image, f, rec


def rescale(params, species, vel, temperature):
    n = len(species)
    v = _f64(vel, (n, 3)).copy()
    _load().orc_rescale(C.byref(_pot(params)), n, _i32(species), v, float(temperature))
    return v


def rand48_seed(seed: int) -> int:
    return int(_load().orc_rand48_seed(seed))


def rand48_step(x: int, n: int) -> int:
    """n steps of the rand48 recurrence from state x, one at a time."""
    return int(_load().orc_rand48_step(x, n))


def rand48_leapfrog(T: int) -> tuple[int, int]:
    """(A_T, C_T) of the leapfrog over T threads, from their definitions."""
    A, Cc = C.c_ulonglong(), C.c_ulonglong()
    _load().orc_rand48_leapfrog(T, C.byref(A), C.byref(Cc))
    return int(A.value), int(Cc.value)


def rand48_uniforms(seed: int, first: int, count: int) -> np.ndarray:
    u = np.empty(count)
    _load().orc_rand48_uniforms(seed, first, count, _f64(u))
    return u


def andersen(params, species, vel, temperature, seed, event, nthreads=None, first_index=0):
    """One Andersen collision of every particle (Sec. 2.3): returns new
    velocities (original order); particle i is thread first_index + i of a
    leapfrog over nthreads (default: the particle count) threads."""
    sp = _i32(species)
    n = sp.shape[0]
    v = _f64(np.array(vel, dtype=np.float64, copy=True), (n, 3))
    _load().orc_andersen(C.byref(_pot(params)), n, sp, v, float(temperature), int(seed), int(event),
                         int(nthreads if nthreads is not None else n), int(first_index))
    return v


def neighbours_brute(params, box, species, pos, skin, kmax=0):
    n = len(species)
    counts = np.zeros(n, dtype=np.int32)
    lists = np.full((n, max(kmax, 1)), -1, dtype=np.int32) if kmax > 0 else None
    _load().orc_neighbours_brute(C.byref(_pot(params)), n, float(box), _i32(species),
                                 _f64(pos, (n, 3)), float(skin), counts,
                                 lists.ctypes.data if lists is not None else None, int(kmax))
    return counts, lists
