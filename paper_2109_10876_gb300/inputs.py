"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no force, integrator or neighbour-list arithmetic: it only
places particles and draws velocities, so that the CUDA library and the CPU
oracle can be fed identical inputs.  Every generator is deterministic in its
seed (numpy PCG64).  Arrays are (N, 3) float64, coordinates in [0, L).

Workloads (reduced LJ units, Sec. 4 of arXiv:2109.10876: m = eps = sigma = 1):
  lj_fluid      fcc lattice at density rho, Gaussian velocities at T with zero
                net momentum (the paper starts its LJ fluid from a lattice at
                rho = 0.8442; its lattice is cubic, the workloads here use fcc)
  perturbed     the same lattice with seeded uniform displacements, so forces
                are non-zero from the first step
  slab          liquid/vapour slab: liquid at rho_l in the central quarter of
                z, vapour at rho_v elsewhere, random sequential placement with
                a minimum separation (an inhomogeneous load, Sec. 5)
  melt          linear bead-spring chains grown as random walks (Sec. 4 polymer
                melt; chain growth rejects near overlaps where it can)
  ensemble      per-replica sizes, log-uniform, and LJ parameters
"""
import math

import numpy as np

FCC_BASIS = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])


def fcc_lattice(ncell, rho):
    """fcc lattice of ncell^3 unit cells (4 sites each) at number density rho.

    Returns (x (N,3), box (3,)).  Lattice constant a = (4/rho)^(1/3)."""
    a = (4.0 / rho) ** (1.0 / 3.0)
    g = np.arange(ncell, dtype=np.float64)
    cz, cy, cx = np.meshgrid(g, g, g, indexing="ij")
    cells = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], axis=1)
    x = (cells[:, None, :] + FCC_BASIS[None, :, :]).reshape(-1, 3) * a
    L = ncell * a
    return x, np.array([L, L, L])


def maxwell_velocities(n, T, seed, mass=1.0):
    """Gaussian velocities, net momentum removed, rescaled so that the
    instantaneous temperature with 3N - 3 degrees of freedom equals T."""
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.standard_normal((n, 3))
    if n > 1:
        v -= v.mean(axis=0, keepdims=True)
        ekin2 = mass * float(np.sum(v * v))  # = 2 K
        dof = 3 * n - 3
        v *= math.sqrt(T * dof / ekin2)
    else:
        v[:] = 0.0
    return v


def wrap(x, box):
    x = np.mod(x, box)
    x[x >= box] = 0.0
    return x


def lj_fluid(ncell, rho=0.8442, T=0.72, seed=1):
    """fcc LJ fluid start: positions, velocities, box."""
    x, box = fcc_lattice(ncell, rho)
    v = maxwell_velocities(len(x), T, seed)
    return x, v, box


def perturbed_lattice(ncell, rho=0.8442, T=0.72, seed=1, amp=0.1):
    """fcc lattice with seeded uniform displacements in [-amp, amp]^3."""
    x, box = fcc_lattice(ncell, rho)
    rng = np.random.Generator(np.random.PCG64(seed + 1000003))
    x = wrap(x + rng.uniform(-amp, amp, size=x.shape), box)
    v = maxwell_velocities(len(x), T, seed)
    return x, v, box


def random_gas(n, box, seed, rmin=0.0):
    """n uniform random points in the box; if rmin > 0, sequential placement
    rejecting any candidate closer than rmin (minimum image) to earlier points."""
    box = np.broadcast_to(np.asarray(box, dtype=np.float64), (3,)).copy()
    rng = np.random.Generator(np.random.PCG64(seed))
    if rmin <= 0.0:
        return rng.uniform(0.0, 1.0, size=(n, 3)) * box
    return _rsa(n, box, rng, rmin, lo=np.zeros(3), hi=box.copy())


def _rsa(n, box, rng, rmin, lo, hi, existing=None):
    """Random sequential placement of n points uniformly in [lo, hi) inside a
    periodic box, each at least rmin (minimum image) from all earlier points
    and from `existing`.  Uses a bucket grid of edge >= rmin."""
    nb = np.maximum((box // rmin).astype(int), 1)
    edge = box / nb
    buckets = {}
    pts = []

    def key(p):
        return tuple((np.floor(p / edge).astype(int)) % nb)

    def ok(p):
        k = key(p)
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    kk = ((k[0] + dx) % nb[0], (k[1] + dy) % nb[1], (k[2] + dz) % nb[2])
                    for q in buckets.get(kk, ()):
                        d = p - q
                        d -= box * np.round(d / box)
                        if d @ d < rmin * rmin:
                            return False
        return True

    if existing is not None:
        for q in existing:
            buckets.setdefault(key(q), []).append(q)
    span = hi - lo
    tries = 0
    while len(pts) < n:
        batch = lo + rng.uniform(0.0, 1.0, size=(4096, 3)) * span
        for p in batch:
            tries += 1
            if ok(p):
                pts.append(p)
                buckets.setdefault(key(p), []).append(p)
                if len(pts) == n:
                    break
        if tries > 200 * n + 100000:
            raise RuntimeError("random sequential placement did not converge")
    return np.array(pts).reshape(-1, 3)
