"""Seeded synthetic initial conditions for the force solve.

This module only draws inputs: positions, velocities and masses of star
clusters. It holds none of the FMM arithmetic, and both the GPU path and the
CPU oracle consume what it returns.

Models (Section 3 of the paper: Plummer spheres in Henon units, G = M = 1,
E0 = -1/4; the paper generated them with MCLUSTER, which is not available, so
these generators stand in for it):

* ``plummer``   -- Plummer sphere with scale a = 3*pi/16 (virial radius 1),
                   radius by inverse CDF truncated at r = 20, isotropic
                   directions, speeds by rejection from q^2 (1-q^2)^(7/2).
* ``kroupa_masses`` -- broken power-law IMF, dN/dm ~ m^-1.3 on [0.08, 0.5]
                   and m^-2.3 on [0.5, 150] solar masses, renormalised so that
                   the total mass is 1.
* ``ensemble``  -- many Plummer clusters of log-uniform N and uniform virial
                   radius, for the batched solve.
* ``nucleus``   -- a Plummer sphere of mass 0.99 plus a point mass of 0.01 at
                   rest at the origin.

The random stream is numpy's PCG64 seeded with the given integer, so a seed
gives the same doubles on every platform.
"""
from __future__ import annotations

import math

import numpy as np

PLUMMER_A = 3.0 * math.pi / 16.0  # Plummer scale radius for virial radius 1
TRUNCATION_RADIUS = 20.0


def _plummer_mass_fraction(r: float, a: float) -> float:
    return r ** 3 / (r * r + a * a) ** 1.5


def plummer(n: int, seed: int, *, a: float = PLUMMER_A, rmax: float = TRUNCATION_RADIUS,
            total_mass: float = 1.0, virial_radius: float = 1.0, center: bool = True):
    """Return (pos[n,3], vel[n,3], mass[n]) of a seeded Plummer sphere.

    Lengths scale with ``virial_radius`` (positions x R_v, velocities x R_v^-1/2),
    so the default is the Henon-unit model. Masses are equal, total_mass / n.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    if n <= 0:
        return (np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0))
    xmax = _plummer_mass_fraction(rmax, a)
    u = rng.random(n)
    x = xmax * (1.0 - u)  # in (0, xmax]
    r = a / np.sqrt(x ** (-2.0 / 3.0) - 1.0)
    cth = 2.0 * rng.random(n) - 1.0
    phi = 2.0 * math.pi * rng.random(n)
    sth = np.sqrt(np.maximum(0.0, 1.0 - cth * cth))
    pos = np.stack([r * sth * np.cos(phi), r * sth * np.sin(phi), r * cth], axis=1)

    # speed fraction q of the local escape speed, by rejection from g(q)
    q = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        qq = rng.random(todo.size)
        yy = 0.1 * rng.random(todo.size)
        ok = yy < qq * qq * (1.0 - qq * qq) ** 3.5
        q[todo[ok]] = qq[ok]
        todo = todo[~ok]
    vesc = np.sqrt(2.0 * total_mass) * (r * r + a * a) ** (-0.25)
    v = q * vesc
    cth = 2.0 * rng.random(n) - 1.0
    phi = 2.0 * math.pi * rng.random(n)
    sth = np.sqrt(np.maximum(0.0, 1.0 - cth * cth))
    vel = np.stack([v * sth * np.cos(phi), v * sth * np.sin(phi), v * cth], axis=1)

    mass = np.full(n, total_mass / n)
    if center:
        pos -= (mass[:, None] * pos).sum(0) / mass.sum()
        vel -= (mass[:, None] * vel).sum(0) / mass.sum()
    pos *= virial_radius
    vel /= math.sqrt(virial_radius)
    return pos, vel, mass


def kroupa_masses(n: int, seed: int, *, mlo: float = 0.08, mbreak: float = 0.5,
                  mhi: float = 150.0, total_mass: float = 1.0) -> np.ndarray:
    """Kroupa (2001) broken power-law masses by piecewise inverse CDF."""
    rng = np.random.Generator(np.random.PCG64(seed))
    a1, a2 = 1.3, 2.3
    # dN/dm = k1 m^-a1 below the break, k2 m^-a2 above, continuous at the break
    k1 = 1.0
    k2 = k1 * mbreak ** (a2 - a1)
    w1 = k1 * (mbreak ** (1 - a1) - mlo ** (1 - a1)) / (1 - a1)
    w2 = k2 * (mhi ** (1 - a2) - mbreak ** (1 - a2)) / (1 - a2)
    u = rng.random(n) * (w1 + w2)
    m = np.empty(n)
    lo = u < w1
    m[lo] = (mlo ** (1 - a1) + u[lo] * (1 - a1) / k1) ** (1.0 / (1 - a1))
    uu = u[~lo] - w1
    m[~lo] = (mbreak ** (1 - a2) + uu * (1 - a2) / k2) ** (1.0 / (1 - a2))
    m = np.clip(m, mlo, mhi)
    return m * (total_mass / m.sum())


def ensemble(nclusters: int, seed: int, *, log2n_lo: float = 10.0, log2n_hi: float = 17.0,
             rv_lo: float = 0.5, rv_hi: float = 2.0, cluster_seed0: int = 1000):
    """Return (offsets[nclusters+1], pos[N,3], mass[N], sizes, virial radii).

    Cluster c has N_c = floor(2^U[lo,hi]) equal-mass stars of total mass 1,
    virial radius U[rv_lo, rv_hi], drawn with seed cluster_seed0 + c.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = np.floor(2.0 ** rng.uniform(log2n_lo, log2n_hi, nclusters)).astype(np.int64)
    rvs = rng.uniform(rv_lo, rv_hi, nclusters)
    pos, mass = [], []
    for c in range(nclusters):
        p, _, m = plummer(int(sizes[c]), cluster_seed0 + c, virial_radius=float(rvs[c]))
        pos.append(p)
        mass.append(m)
    offsets = np.zeros(nclusters + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    return offsets, np.concatenate(pos), np.concatenate(mass), sizes, rvs


def nucleus(n: int, seed: int, *, bh_mass: float = 0.01):
    """Plummer sphere of n stars (total 1 - bh_mass) plus a point mass at the origin."""
    pos, vel, mass = plummer(n, seed, total_mass=1.0 - bh_mass)
    pos = np.concatenate([pos, np.zeros((1, 3))])
    vel = np.concatenate([vel, np.zeros((1, 3))])
    mass = np.concatenate([mass, [bh_mass]])
    return pos, vel, mass


def config_inputs(name: str):
    """Named workloads (positions, masses) used by tests and the benchmark.

    'plummer4k'   : N = 4096, equal masses, seed 1.
    'plummer1m'   : N = 1,048,576, equal masses, seed 2.
    'kroupa1m'    : the same positions, Kroupa masses drawn with seed 3.
    """
    if name == "plummer4k":
        p, _, m = plummer(4096, 1)
        return p, m
    if name == "plummer1m":
        p, _, m = plummer(1 << 20, 2)
        return p, m
    if name == "kroupa1m":
        p, _, _ = plummer(1 << 20, 2)
        return p, kroupa_masses(1 << 20, 3)
    raise KeyError(name)
