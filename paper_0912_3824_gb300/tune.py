"""Autotuner for the step kernel's launch shape and the neighbour-list
parameters.

The throughput of the step depends on how many lanes share a particle (the
shape of the step kernel's blocks: 1, 2, 4 or 8 lanes, 128 threads per
block), on the skin (a longer list against rarer rebuilds; the result of the
method does not depend on it, Sec. 2.2) and, through memory, on the list
capacity.  `autotune` times short runs of the caller's own configuration for
every candidate and returns the fastest parameters, with the list capacity
set from the longest list seen (25 % headroom, a multiple of 32).

Host logic only: every candidate runs the library's own kernels through the
C ABI; nothing here computes a step.
"""
from __future__ import annotations

import copy
import math

import numpy as np

from . import md


def _clone(p: md.md_params) -> md.md_params:
    q = md.md_params()
    for name, _ in md.md_params._fields_:
        setattr(q, name, copy.deepcopy(getattr(p, name)))
    return q


def _time(torch, sim, steps, repeats):
    ms = []
    for _ in range(repeats):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(sim.stream)
        sim.step(steps)
        e1.record(sim.stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return float(np.median(ms)) / steps


def autotune(base: md.md_params, n_per_replica, box, species, pos, vel, image=None, device: str = "cuda",
             lanes=None, skins=(0.15, 0.2, 0.25, 0.3), steps: int = 400, repeats: int = 3):
    """Returns (best md_params, table of trials).  The state (pos, vel, image,
    original order) is the starting point of every trial; each trial warms up
    for `steps` MD steps (several list rebuilds) and is then timed `repeats`
    times over `steps` steps with CUDA events (median)."""
    import torch
    if lanes is None:
        lanes = (2, 4, 8) if base.precision == md.MD_PREC_FP64 else (1, 2, 4)
    if base.smooth_h > 0:
        lanes = tuple(t for t in lanes if t <= 8)
    trials = []
    best = None
    for skin in skins:
        for tpp in lanes:
            p = _clone(base)
            p.skin = float(skin)
            p.threads_per_particle = int(tpp)
            p.neigh_capacity = 0
            sim = md.System(p, n_per_replica, box, species, pos, vel, image, device=device)
            sim.step(steps)
            status = sim.sync()
            ms = _time(torch, sim, steps, repeats) if status == md.MD_OK else math.inf
            info = sim.info()
            sim.close()
            trials.append({"skin": float(skin), "threads_per_particle": int(tpp), "ms_per_step": ms,
                           "max_neighbours": int(info["max_neighbours"]),
                           "neigh_capacity": int(info["neigh_capacity"]), "status": md._status_name(status)})
            if best is None or ms < best[0]:
                best = (ms, p, info)
    ms, p, info = best
    # capacity: the longest list seen with 25 % headroom, never below the automatic choice's need
    p.neigh_capacity = int(math.ceil(1.25 * info["max_neighbours"] / 32.0) * 32)
    return p, trials
