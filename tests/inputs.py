"""Seeded synthetic inputs shared by the oracle tests and the GPU parity tests.

This module holds no arithmetic of the method: it only draws positions,
species and velocities with numpy's seeded generator, with the shapes and
value distributions of the paper's workloads (uniform random nucleons in a
periodic cube, Sec. III.B; compact drops standing in for nuclei; Maxwell
velocities at the paper's temperatures).
"""
from __future__ import annotations

import numpy as np

M_NUCLEON = 939.0


def box_side(N: int, rho: float) -> float:
    return (N / rho) ** (1.0 / 3.0)


def species(N: int, Yp: float) -> np.ndarray:
    """Protons first: type 1 for the first floor(Yp*N + 0.5) particles."""
    Np = int(np.floor(Yp * N + 0.5))
    t = np.zeros(N, dtype=np.int8)
    t[:Np] = 1
    return t


def uniform(N: int, Yp: float, L: float, seed: int, min_sep: float = 0.0):
    """Uniform random positions in [0, L)^3; optional minimum separation by
    rejection (nearest image), for small N only."""
    rng = np.random.default_rng(seed)
    if min_sep <= 0.0:
        x = rng.random((N, 3)) * L
    else:
        pts = []
        while len(pts) < N:
            p = rng.random(3) * L
            ok = True
            for q in pts:
                d = p - q
                d -= L * np.round(d / L)
                if d @ d < min_sep * min_sep:
                    ok = False
                    break
            if ok:
                pts.append(p)
        x = np.array(pts)
    return x, species(N, Yp)


def lattice_liquid(N: int, Yp: float, L: float, seed: int, jitter: float = 0.35):
    """Jittered simple-cubic lattice filling the box (a dense, overlap-free
    stand-in for relaxed nuclear matter); species shuffled over sites."""
    rng = np.random.default_rng(seed)
    n = int(np.ceil(N ** (1.0 / 3.0)))
    a = L / n
    g = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1).reshape(-1, 3)
    sites = g[rng.permutation(len(g))[:N]].astype(np.float64)
    x = (sites + 0.5 + jitter * (rng.random((N, 3)) - 0.5)) * a
    x = np.mod(x, L)
    return x, species(N, Yp)


def drop(n_p: int, n_n: int, L: float, center, seed: int, spacing: float = 1.9):
    """A compact nucleus-like drop: jittered cubic lattice points nearest the
    centre; protons and neutrons interleaved.  Positions wrapped into [0, L)."""
    rng = np.random.default_rng(seed)
    N = n_p + n_n
    k = int(np.ceil(N ** (1.0 / 3.0))) + 2
    g = np.stack(np.meshgrid(*(np.arange(-k, k + 1),) * 3, indexing="ij"), -1).reshape(-1, 3).astype(np.float64)
    order = np.argsort((g * g).sum(1), kind="stable")
    pts = g[order[:N]] * spacing + 0.15 * spacing * (rng.random((N, 3)) - 0.5)
    x = np.mod(pts + np.asarray(center, dtype=np.float64), L)
    t = np.zeros(N, dtype=np.int8)
    t[rng.permutation(N)[:n_p]] = 1
    perm = np.argsort(-t, kind="stable")       # protons first
    return x[perm], t[perm]


def maxwell(N: int, T: float, seed: int) -> np.ndarray:
    """Maxwell-Boltzmann velocities (c = 1) at temperature T (MeV)."""
    rng = np.random.default_rng(seed)
    v = rng.normal(0.0, np.sqrt(T / M_NUCLEON), (N, 3))
    return v - v.mean(0)
