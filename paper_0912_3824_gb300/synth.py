"""Seeded synthetic inputs for the molecular-dynamics workloads.

This module only draws random numbers and lays out particles; it contains none
of the simulation arithmetic (no forces, no integration, no reductions beyond
the initial temperature scaling of the drawn velocities).  It is the single
input source shared by the CUDA path, its tests, the benchmark and the CPU
oracle, which receive its arrays as plain data.

Workloads follow the paper's systems: fcc start lattices (Sec. 3, Sec. 4), the
Lennard-Jones 12-6 potential cut at r_c = 2.5 sigma (Sec. 3) and the
Kob-Andersen binary mixture with 80% A / 20% B particles of equal mass
(Sec. 5).  Reduced units: sigma_AA, epsilon_AA, m.

Random stream: SplitMix64 (Steele, Lea, Flood 2014) on a 64-bit counter,
53-bit uniform doubles, Box-Muller normals.  One stream per system, drawn in
the fixed order: lattice-site choice, species choice, velocities.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


class Stream:
    """Counter-based SplitMix64 stream: output k is mix(seed + (k+1)*gamma)."""

    def __init__(self, seed: int):
        self.seed = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        self.counter = 0

    def u64(self, n: int) -> np.ndarray:
        k = np.arange(self.counter + 1, self.counter + 1 + n, dtype=np.uint64)
        self.counter += n
        with np.errstate(over="ignore"):
            z = self.seed + k * _GAMMA
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, n: int) -> np.ndarray:
        """Doubles in [0, 1) with 53 random bits."""
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def normal(self, n: int) -> np.ndarray:
        """Standard normals by Box-Muller, two per pair of uniforms."""
        m = (n + 1) // 2
        u1 = 1.0 - self.uniform(m)          # (0, 1]
        u2 = self.uniform(m)
        r = np.sqrt(-2.0 * np.log(u1))
        z = np.concatenate([r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)])
        return z[:n]

    def permutation(self, n: int) -> np.ndarray:
        """Uniform random permutation: order of n independent 64-bit keys."""
        return np.argsort(self.u64(n), kind="stable")


def lj_params(rcut: float = 2.5, shift: bool = True, smooth: float = 0.0) -> dict:
    """Monatomic 12-6 Lennard-Jones, eps = sigma = m = 1, cut at rcut (Sec. 3);
    smooth = h > 0 multiplies it by g((r - r_c) / (h sigma)) (Sec. 4)."""
    one = [[1.0, 1.0], [1.0, 1.0]]
    return {
        "n_species": 1,
        "eps": one,
        "sigma": one,
        "rcut": [[rcut, rcut], [rcut, rcut]],
        "shift": bool(shift),
        "mass": [1.0, 1.0],
        "smooth": float(smooth),
    }


WCA_RCUT = 2.0 ** (1.0 / 6.0)


def wca_params(smooth: float = 0.0) -> dict:
    """Purely repulsive Weeks-Chandler-Andersen potential (Sec. 4): the 12-6
    potential shifted up by eps and cut at its minimum, r_c = 2^(1/6) sigma."""
    return lj_params(rcut=WCA_RCUT, shift=True, smooth=smooth)


def ka_params(rcut_factor: float = 2.5, shift: bool = True, smooth: float = 0.0) -> dict:
    """Kob-Andersen A/B mixture (Sec. 5): sigma_AA=1, sigma_BB=0.88,
    sigma_AB=0.8, eps_AA=1, eps_BB=0.5, eps_AB=1.5, equal masses.
    Each pair is cut at rcut_factor * sigma_ab."""
    eps = [[1.0, 1.5], [1.5, 0.5]]
    sig = [[1.0, 0.8], [0.8, 0.88]]
    rc = [[rcut_factor * s for s in row] for row in sig]
    return {"n_species": 2, "eps": eps, "sigma": sig, "rcut": rc,
            "shift": bool(shift), "mass": [1.0, 1.0], "smooth": float(smooth)}


def max_rcut(params: dict) -> float:
    ns = params["n_species"]
    return max(params["rcut"][a][b] for a in range(ns) for b in range(ns))


@dataclass
class System:
    """One periodic cubic system: arrays in the original particle order."""
    n: int
    box: float
    species: np.ndarray      # int32 [n]
    pos: np.ndarray          # float64 [n, 3], wrapped into [0, box)
    vel: np.ndarray          # float64 [n, 3]
    image: np.ndarray        # int32 [n, 3]
    params: dict
    seed: int


def fcc_sites(nc: int, a: float) -> np.ndarray:
    """All 4*nc^3 sites of an fcc lattice of nc^3 cubic cells of edge a,
    offset by a/4 so that no site lies on a cell face of the box."""
    basis = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
    g = np.arange(nc, dtype=np.float64)
    cz, cy, cx = np.meshgrid(g, g, g, indexing="ij")
    cells = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], axis=1)
    sites = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3)
    return (sites + 0.25) * a


def make_system(n: int, density: float, temperature: float, seed: int,
                params: dict | None = None, frac_b: float = 0.2) -> System:
    """fcc start lattice at the given number density with Maxwell-Boltzmann
    velocities.

    n_c = ceil((n/4)^(1/3)) fcc cells per edge; when 4 n_c^3 > n the occupied
    sites are a seeded uniform choice (vacancies spread at random).  For a
    two-species mixture, round(frac_b * n) particles (half to even) chosen
    from a seeded permutation are B (species 1).  Velocity components are
    N(0, T/m); the mass-weighted mean is removed and the set is scaled so that
    2 E_kin / (3n - 3) equals the temperature exactly.
    """
    params = params if params is not None else lj_params()
    st = Stream(seed)
    box = (n / density) ** (1.0 / 3.0)
    nc = int(math.ceil((n / 4.0) ** (1.0 / 3.0) - 1e-9))
    while 4 * nc ** 3 < n:
        nc += 1
    sites = fcc_sites(nc, box / nc)
    if sites.shape[0] > n:
        chosen = np.sort(st.permutation(sites.shape[0])[:n])
        sites = sites[chosen]
    pos = np.mod(sites, box)
    species = np.zeros(n, dtype=np.int32)
    if params["n_species"] == 2:
        nb = int(round(frac_b * n))
        species[st.permutation(n)[:nb]] = 1
    mass = np.asarray(params["mass"], dtype=np.float64)[species]
    vel = st.normal(3 * n).reshape(n, 3) * np.sqrt(temperature / mass)[:, None]
    vel -= (mass[:, None] * vel).sum(axis=0) / mass.sum()
    if n > 1 and temperature > 0:
        ekin = 0.5 * float((mass[:, None] * vel * vel).sum())
        vel *= math.sqrt(temperature * (3 * n - 3) / (2.0 * ekin))
    return System(n=n, box=box, species=species, pos=pos, vel=vel,
                  image=np.zeros((n, 3), dtype=np.int32), params=params, seed=seed)


def perturb(sysm: System, amplitude: float, seed: int) -> System:
    """Copy of the system with every coordinate displaced uniformly in
    [-amplitude, amplitude) and wrapped back into the box (image counters
    updated), giving liquid-like, force-carrying configurations."""
    st = Stream(seed)
    d = (st.uniform(3 * sysm.n).reshape(sysm.n, 3) * 2.0 - 1.0) * amplitude
    raw = sysm.pos + d
    shift = np.floor(raw / sysm.box)
    pos = raw - shift * sysm.box
    pos = np.where(pos >= sysm.box, pos - sysm.box, pos)
    return System(n=sysm.n, box=sysm.box, species=sysm.species.copy(), pos=pos,
                  vel=sysm.vel.copy(), image=sysm.image + shift.astype(np.int32),
                  params=sysm.params, seed=sysm.seed)


# Workloads with the shapes of the paper's systems.
def lj_fluid(n: int = 864, density: float = 0.8442, temperature: float = 0.722,
             seed: int = 1) -> System:
    """Monatomic LJ fluid, r_c = 2.5 sigma, truncated and shifted."""
    return make_system(n, density, temperature, seed, lj_params())


def ka_mixture(n: int = 65536, density: float = 1.2, temperature: float = 0.7,
               seed: int = 5) -> System:
    """Kob-Andersen 80:20 mixture at density 1.2 (Sec. 5)."""
    return make_system(n, density, temperature, seed, ka_params())


def ensemble_sizes(n_replicas: int = 256, lo: int = 500, hi: int = 8000,
                   seed: int = 4) -> list[int]:
    """Replica sizes drawn uniformly from {lo, ..., hi}."""
    st = Stream(seed)
    u = st.uniform(n_replicas)
    return [int(lo + math.floor(x * (hi - lo + 1))) for x in u]


def shell_wavevectors(box: float, q: float, count: int = 16, seed: int = 9) -> np.ndarray:
    """`count` wavevectors of the box's reciprocal lattice (2 pi / L) Z^3 whose
    length is within half a lattice spacing of q, chosen by a seeded uniform
    permutation of the whole shell (so that orientations are sampled evenly).
    Returns float64 [count, 3]."""
    dq = 2.0 * math.pi / box
    nmax = int(math.ceil(q / dq + 1))
    r = np.arange(-nmax, nmax + 1)
    n = np.stack(np.meshgrid(r, r, r, indexing="ij"), axis=-1).reshape(-1, 3)
    norm = np.sqrt((n * n).sum(axis=1)) * dq
    shell = n[np.abs(norm - q) <= 0.5 * dq]
    if shell.shape[0] == 0:
        raise ValueError("no wavevector of the box near q")
    pick = Stream(seed).permutation(shell.shape[0])[:count]
    return shell[np.sort(pick)].astype(np.float64) * dq
