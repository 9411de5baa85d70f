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


def rsa_fast(n, box, lo, hi, rmin, rng, existing=None, batch=20000):
    """Random sequential placement, vectorised: uniform candidates in [lo, hi),
    each kept if at least rmin (minimum image) from every point kept before it
    (and from `existing`).  A grid of cell edge rmin / sqrt(3) holds at most one
    point per cell, so a candidate is checked against the 5 x 5 x 5 cells
    around it; conflicts inside a batch are resolved in candidate order."""
    from scipy.spatial import cKDTree
    box = np.asarray(box, dtype=np.float64)
    lo, hi = np.asarray(lo, dtype=np.float64), np.asarray(hi, dtype=np.float64)
    # edge <= rmin / sqrt(3): two kept points never share a cell; edge >= rmin / 2:
    # everything within rmin lies in the 5 x 5 x 5 cells around a point
    ng = np.maximum(np.ceil(box / (rmin / math.sqrt(3.0))).astype(np.int64), 1)
    edge = box / ng
    if np.any(edge < 0.5 * rmin) and np.any(ng > 4):
        raise ValueError("box too small for the placement grid")
    grid = np.full(int(ng[0] * ng[1] * ng[2]), -1, dtype=np.int64)
    pts = np.zeros((n + (0 if existing is None else len(existing)), 3))
    m = 0

    def cell_of(p):
        c = np.floor(p / edge).astype(np.int64) % ng
        return (c[:, 2] * ng[1] + c[:, 1]) * ng[0] + c[:, 0], c

    if existing is not None and len(existing):
        k, _ = cell_of(existing)
        pts[:len(existing)] = existing
        grid[k] = np.arange(len(existing))
        m = len(existing)
    start = m
    o5 = np.arange(-2, 3)
    tries = 0
    while m - start < n:
        cand = lo + rng.uniform(0.0, 1.0, size=(batch, 3)) * (hi - lo)
        cand = np.mod(cand, box)
        _, cc = cell_of(cand)
        # the 5 x 5 x 5 cells around each candidate, wrapped per axis
        ax = [(cc[:, k, None] + o5[None, :]) % ng[k] for k in range(3)]
        nbk = ((ax[2][:, None, None, :] * ng[1] + ax[1][:, None, :, None]) * ng[0] +
               ax[0][:, :, None, None]).reshape(len(cand), 125)
        idx = grid[nbk]                                   # (batch, 125)
        # distances to the occupied cells only (most of the 125 are empty)
        row, col = np.nonzero(idx >= 0)
        d = cand[row] - pts[idx[row, col]]
        d -= box * np.round(d / box)
        close = np.zeros(len(cand), dtype=bool)
        close[row[np.sum(d * d, axis=1) < rmin * rmin]] = True
        ok = ~close
        good = np.nonzero(ok)[0]
        # conflicts among this batch's survivors: keep the earlier candidate
        if len(good) > 1:
            tree = cKDTree(cand[good], boxsize=box)
            drop = np.zeros(len(good), dtype=bool)
            for a, b in sorted(tree.query_pairs(rmin)):
                if not drop[a]:
                    drop[b] = True
            good = good[~drop]
        good = good[:n - (m - start)]
        k, _ = cell_of(cand[good])
        pts[m:m + len(good)] = cand[good]
        grid[k] = np.arange(m, m + len(good))
        m += len(good)
        tries += batch
        if tries > 400 * n + 10 * batch:
            raise RuntimeError("random sequential placement did not converge")
    return pts[start:m]


def slab(n, rho_l=0.80, rho_v=0.02, T=0.8, seed=3, rmin=0.8):
    """Liquid/vapour slab: a periodic box with Lz = 4 Lx = 4 Ly; liquid at rho_l
    in the central quarter of z (z in [3 Lz / 8, 5 Lz / 8)), vapour at rho_v
    elsewhere; positions by random sequential placement with minimum separation
    rmin (liquid first, then vapour), Gaussian velocities at T.  The particle
    numbers split as n_liq = round(n rho_l / 4 / (rho_l / 4 + 3 rho_v / 4))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    frac = 0.25 * rho_l / (0.25 * rho_l + 0.75 * rho_v)
    lx = (n / (4.0 * (0.25 * rho_l + 0.75 * rho_v))) ** (1.0 / 3.0)
    box = np.array([lx, lx, 4.0 * lx])
    n_liq = int(round(n * frac))
    liq = rsa_fast(n_liq, box, [0.0, 0.0, 1.5 * lx], [lx, lx, 2.5 * lx], rmin, rng)
    # vapour: uniform in the two outer regions (total length 3 lx), placed against the liquid
    vap = rsa_fast(n - n_liq, box, [0.0, 0.0, 2.5 * lx], [lx, lx, 5.5 * lx], rmin, rng, existing=liq)
    x = wrap(np.concatenate([liq, vap]), box)
    v = maxwell_velocities(n, T, seed + 17)
    return x, v, box


def chains(nchain, nbead, box, seed, bond=0.97, rmin=0.75):
    """Linear chains grown as self-avoiding random walks: bond length `bond`,
    no two beads closer than rmin (minimum image).  For the small, dilute test
    systems; returns positions and the bond list (pairs of particle indices)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    box = np.asarray(box, dtype=np.float64)
    pts, bonds = [], []
    for c in range(nchain):
        for k in range(nbead):
            for _ in range(10000):
                if k == 0:
                    p = rng.uniform(0, 1, 3) * box
                else:
                    u = rng.normal(size=3)
                    p = pts[-1] + bond * u / np.linalg.norm(u)
                if not pts:
                    break
                d = np.array(pts) - p
                d -= box * np.round(d / box)
                if np.min(np.sum(d * d, axis=1)) >= rmin * rmin:
                    break
            else:
                raise RuntimeError("chain growth failed")
            if k > 0:
                bonds.append((len(pts) - 1, len(pts)))
            pts.append(p)
    return wrap(np.array(pts), box), np.array(bonds, dtype=np.int32)


def lattice_fluid(n, rho=0.8442, T=0.72, seed=1, sigma=1.0, amp=0.05):
    """n particles at number density rho (in units of sigma^-3) in a cubic box
    of edge L = sigma (n / rho)^(1/3): the sites of the smallest fcc lattice
    with at least n sites, scaled to the box, with 4 k^3 - n of them chosen at
    random and left empty, then uniform displacements in [-amp, amp] sigma;
    Gaussian velocities at T.  Returns (x, v, box)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    L = sigma * (n / rho) ** (1.0 / 3.0)
    k = 1
    while 4 * k ** 3 < n:
        k += 1
    a = L / k
    g = np.arange(k, dtype=np.float64)
    cz, cy, cx = np.meshgrid(g, g, g, indexing="ij")
    cells = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], axis=1)
    sites = (cells[:, None, :] + FCC_BASIS[None, :, :]).reshape(-1, 3) * a
    keep = np.sort(rng.permutation(len(sites))[:n])
    box = np.array([L, L, L])
    x = wrap(sites[keep] + rng.uniform(-amp * sigma, amp * sigma, size=(n, 3)), box)
    v = maxwell_velocities(n, T, seed + 7919)
    return x, v, box


def ensemble(nrep=64, nmin=500, nmax=32000, rho=0.8442, T=0.72, seed=11,
             eps_range=(0.9, 1.1), sigma_range=(0.95, 1.05)):
    """Batched ensemble of LJ-fluid replicas: sizes log-uniform in [nmin, nmax],
    per-replica eps and sigma uniform in the given ranges, each replica a
    lattice_fluid at density rho in units of its own sigma.  Returns
    (sizes (R,), boxes (R, 3), eps (R,), sigma (R,), x (N, 3), v (N, 3)) with
    the replicas concatenated in order."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = np.rint(np.exp(rng.uniform(math.log(nmin), math.log(nmax), size=nrep))).astype(np.int64)
    eps = rng.uniform(eps_range[0], eps_range[1], size=nrep)
    sig = rng.uniform(sigma_range[0], sigma_range[1], size=nrep)
    xs, vs, boxes = [], [], []
    for r in range(nrep):
        x, v, box = lattice_fluid(int(sizes[r]), rho, T, seed + 101 * (r + 1), sigma=float(sig[r]))
        xs.append(x)
        vs.append(v)
        boxes.append(box)
    return sizes, np.array(boxes), eps, sig, np.concatenate(xs), np.concatenate(vs)


def melt(nchain=2000, nbead=200, rho=0.85, T=1.0, seed=4, bond=0.97):
    """Linear bead-spring chains for the polymer melt (Sec. 4): nchain chains
    of nbead beads at bead density rho in a cubic box, each a free random
    walk of fixed bond length `bond` from a uniform random start (overlaps are
    left for the soft push-off to remove); Gaussian velocities at T.
    Returns (x (N, 3), v (N, 3), box (3,), bonds (nchain (nbead - 1), 2))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = nchain * nbead
    L = (n / rho) ** (1.0 / 3.0)
    box = np.array([L, L, L])
    start = rng.uniform(0.0, L, size=(nchain, 1, 3))
    u = rng.standard_normal((nchain, nbead - 1, 3))
    u *= bond / np.linalg.norm(u, axis=2, keepdims=True)
    walk = np.concatenate([np.zeros((nchain, 1, 3)), np.cumsum(u, axis=1)], axis=1)
    x = wrap((start + walk).reshape(-1, 3), box)
    first = (np.arange(nchain)[:, None] * nbead + np.arange(nbead - 1)[None, :]).ravel()
    bonds = np.stack([first, first + 1], axis=1).astype(np.int32)
    v = maxwell_velocities(n, T, seed + 31)
    return x, v, box, bonds


def sphere(n=2_580_000, L=271.0, rho=0.8442, T=0.1, seed=6):
    """Spherical inhomogeneous LJ system (Sec. 4.2): a cubic box of edge L
    with n particles at density rho in a central sphere and vacuum around it.
    The particles are the n fcc sites (lattice constant (4/rho)^(1/3), one
    site at the box centre) closest to the centre, so the sphere radius is
    about (3 n / (4 pi rho))^(1/3); Gaussian velocities at T."""
    a = (4.0 / rho) ** (1.0 / 3.0)
    R = (3.0 * n / (4.0 * math.pi * rho)) ** (1.0 / 3.0)
    k = int(math.ceil((R + 2 * a) / a))
    g = np.arange(-k, k, dtype=np.float64)
    cz, cy, cx = np.meshgrid(g, g, g, indexing="ij")
    cells = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], axis=1)
    sites = (cells[:, None, :] + FCC_BASIS[None, :, :]).reshape(-1, 3) * a
    r2 = np.einsum("ij,ij->i", sites, sites)
    order = np.argsort(r2, kind="stable")[:n]
    box = np.array([L, L, L])
    x = wrap(sites[np.sort(order)] + 0.5 * L, box)
    v = maxwell_velocities(n, T, seed)
    return x, v, box


def rings(nring=1600, length=200, rho=0.85, T=1.0, seed=7, bond=0.97):
    """Ring polymers (Sec. 4: rings of 200 beads at density 0.85): each ring a
    closed random walk (bond steps of length `bond` in random directions, their
    mean subtracted so that the walk closes), from a uniform random start;
    overlaps are left for the soft push-off.  Returns (x, v, box, bonds
    (nring length, 2), angles (nring length, 3): the triples (k-1, k, k+1) of
    every ring, middle bead second)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = nring * length
    L = (n / rho) ** (1.0 / 3.0)
    box = np.array([L, L, L])
    u = rng.standard_normal((nring, length, 3))
    u *= bond / np.linalg.norm(u, axis=2, keepdims=True)
    u -= u.mean(axis=1, keepdims=True)
    walk = np.concatenate([np.zeros((nring, 1, 3)), np.cumsum(u[:, :-1], axis=1)], axis=1)
    start = rng.uniform(0.0, L, size=(nring, 1, 3))
    x = wrap((start + walk).reshape(-1, 3), box)
    base = (np.arange(nring) * length)[:, None]
    k = np.arange(length)[None, :]
    bonds = np.stack([(base + k).ravel(), (base + (k + 1) % length).ravel()], axis=1).astype(np.int32)
    angles = np.stack([(base + (k - 1) % length).ravel(), (base + k).ravel(),
                       (base + (k + 1) % length).ravel()], axis=1).astype(np.int32)
    v = maxwell_velocities(n, T, seed + 43)
    return x, v, box, bonds, angles
