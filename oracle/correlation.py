"""Blocking scheme for time-correlation functions (Sec. 2.5) -- TEST
INFRASTRUCTURE ONLY (the reference the CUDA correlator is checked against;
only the tests, the smoke check and the benchmark's CPU leg may use it).

The trajectory is sampled at times m * dt_s, m = 0, 1, 2, ...  Block n
(n = 0 .. k-1) holds at most l samples spaced l^n dt_s apart: it receives the
samples whose index m is a multiple of l^n.  When a block becomes full, its
first (oldest) entry is correlated with each of the other l - 1 entries --
time lags j l^n dt_s, j = 1 .. l-1 -- and is then discarded.  Memory: k l
snapshots for a trajectory of length l^k dt_s.

Observables of a pair of snapshots (unwrapped positions r(0), r(t)), per
species a, summed over the particles of that species:
  - mean-square displacement      |r_i(t) - r_i(0)|^2                 (Sec. 5)
  - self intermediate scattering  (1/n_q) sum_q cos(q . (r_i(t) - r_i(0)))
    over a given set of wavevectors q, the orientational average of
    F_s(q, t) = < rho_q(t) rho_-q(0) > for one particle (Sec. 5).
Averages are these sums divided by (number of correlated origins) x (number
of particles of the species).
"""
from __future__ import annotations

import numpy as np


def pair_sums(r0, rt, species, qvecs):
    """Per species: (sum |d|^2, sum of the q-averaged cos(q . d), particle count)
    for d = rt - r0.  Returns float64 [2, 3]."""
    d = np.asarray(rt, dtype=np.float64) - np.asarray(r0, dtype=np.float64)
    d2 = (d * d).sum(axis=1)
    cs = np.cos(d @ np.asarray(qvecs, dtype=np.float64).T).mean(axis=1)
    out = np.zeros((2, 3))
    for a in range(2):
        sel = species == a
        out[a] = (d2[sel].sum(), cs[sel].sum(), sel.sum())
    return out


class BlockingCorrelator:
    """k blocks of l entries, filled sample by sample (Sec. 2.5)."""

    def __init__(self, k: int, l: int, species, qvecs):
        if k < 1 or l < 2:
            raise ValueError("need k >= 1 blocks of l >= 2 entries")
        self.k, self.l = k, l
        self.species = np.asarray(species, dtype=np.int32)
        self.qvecs = np.asarray(qvecs, dtype=np.float64)
        self.blocks = [[] for _ in range(k)]          # entries (m, snapshot)
        self.sums = np.zeros((k, l - 1, 2, 3))
        self.origins = np.zeros((k, l - 1), dtype=np.int64)
        self.m = 0

    def sample(self, r):
        """Insert the unwrapped positions of sample index self.m."""
        m = self.m
        for n in range(self.k):
            if m % self.l ** n:
                break
            blk = self.blocks[n]
            blk.append((m, np.array(r, dtype=np.float64, copy=True)))
            if len(blk) == self.l:
                m0, r0 = blk[0]
                for j in range(1, self.l):
                    mj, rj = blk[j]
                    assert mj - m0 == j * self.l ** n
                    self.sums[n, j - 1] += pair_sums(r0, rj, self.species, self.qvecs)
                    self.origins[n, j - 1] += 1
                blk.pop(0)
        self.m += 1

    def result(self):
        """lags [k, l-1] in sample intervals, msd and fs [k, l-1, 2] (NaN where no
        origin or no particle of the species), origins [k, l-1]."""
        lags = np.array([[j * self.l ** n for j in range(1, self.l)] for n in range(self.k)])
        cnt = self.sums[..., 2]
        with np.errstate(invalid="ignore", divide="ignore"):
            msd = np.where(cnt > 0, self.sums[..., 0] / cnt, np.nan)
            fs = np.where(cnt > 0, self.sums[..., 1] / cnt, np.nan)
        return lags, msd, fs, self.origins.copy()
