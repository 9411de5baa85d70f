"""Parity at the full size of the LJ-fluid bench: N = 2,048,000 (fcc 80^3 x 4),
reduced density 0.8442, T* = 0.72, r_cut = 2.5 sigma (shifted), r_skin = 0.3,
dt = 0.005, FP32 pair arithmetic with 64-bit fixed-point sums (and the plain
FP64 path where stated), in the launch configuration the bench times: the
tile size picked by md_autotune and md_step as one graph launch.

The O(N^2) oracle cannot evaluate the whole system, so it is compared on
outputs it computes one particle at a time (forces and neighbour rows of
sampled particles, each summed over all N), and the rest through properties
that hold at any size: the fcc neighbour count and lattice energy, exact
zero total force in fixed point, momentum and energy conservation, and the
time reversibility of velocity Verlet (Fig. 1).  Tolerances as in the small
parity tests: neighbour rows bit-exact (pairs within 1e-9 sigma of
r_cut + r_skin excepted), forces 1e-5 (FP32) and 1e-12 (FP64) relative.
"""
import numpy as np
import pytest

import oracle
from paper_2109_10876_gb300 import inputs
from tests.helpers import force_rel_err, min_image_diff

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NC, N = 80, 2_048_000
RHO, T0, RC, SKIN, DT = 0.8442, 0.72, 2.5, 0.3, 0.005
RL = RC + SKIN


@pytest.fixture(scope="module")
def md():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_10876_gb300 import md as m
    return m


@pytest.fixture(scope="module")
def lattice():
    """The bench's own input: the fcc lattice with Gaussian velocities, seed 2."""
    return inputs.lj_fluid(NC, rho=RHO, T=T0, seed=2)


@pytest.fixture(scope="module")
def perturbed():
    """The bench's force-error input: the lattice displaced by up to 0.1 sigma."""
    return inputs.perturbed_lattice(NC, rho=RHO, T=T0, seed=5, amp=0.1)


def dev(a):
    return torch.tensor(np.ascontiguousarray(np.asarray(a).T), dtype=torch.float64, device="cuda")


def bench_handle(md, x, v, box, precision):
    h = md.md_create(N, box, rc_over_sigma=RC, skin=SKIN, dt=DT, precision=precision)
    md.md_set_state(h, dev(x), dev(v))
    md.md_build_neighbors(h)
    if precision == md.MD_FP32_FIXED:
        md.md_autotune(h, 10)       # as the bench does; the state is restored
    return h


def gpu_forces(md, h):
    f = torch.zeros(3, N, dtype=torch.float64, device="cuda")
    euw = torch.zeros(1, 3, dtype=torch.float64, device="cuda")
    md.md_compute_forces(h, f, euw)
    md.md_sync(h)
    return f.cpu().numpy().T.copy(), euw.cpu().numpy()[0]


def gpu_state(md, h):
    xo = torch.zeros(3, N, dtype=torch.float64, device="cuda")
    vo = torch.zeros_like(xo)
    md.md_get_state(h, xo, vo)
    return xo.cpu().numpy().T.copy(), vo.cpu().numpy().T.copy()


def gpu_rows(md, h, idx, n_particles=N):
    """Neighbour rows of the particles idx from the exported Verlet list."""
    n = md.md_export_pairs(h, None, 0)
    out = np.zeros((n, 2), dtype=np.int32)
    assert md.md_export_pairs(h, out, n) == n
    sel = np.zeros(n_particles, dtype=bool)
    sel[idx] = True
    a, b = out[:, 0], out[:, 1]
    ma, mb = sel[a], sel[b]
    owner = np.concatenate([a[ma], b[mb]])
    other = np.concatenate([b[ma], a[mb]])
    order = np.lexsort((other, owner))
    owner, other = owner[order], other[order]
    rows = {}
    for i in idx:
        lo, hi = np.searchsorted(owner, i), np.searchsorted(owner, i, side="right")
        rows[int(i)] = other[lo:hi]
    return n, rows


def first_step_bound(F, tol):
    """Largest admissible |x_1 - (x_0 + dt v_0 + dt^2/2m F)| per particle when
    the force carries the relative error tol of the force tests (normalised by
    max(|F_i|, F_rms)), plus FP64 rounding of the position."""
    mag = np.linalg.norm(F, axis=1)
    rms = np.sqrt(np.mean(mag ** 2))
    return 0.5 * DT * DT * tol * np.maximum(mag, rms) + 1e-11


def check_rows(md, h, x, box, idx):
    """GPU rows equal the oracle's brute-force rows, except pairs within 1e-9
    sigma of the list radius (which either side may round across)."""
    s = oracle.System(N, box, rc=RC)
    want = oracle.neighbours_sample(s, x, idx, RL)
    n, got = gpu_rows(md, h, idx)
    for i, (j, r2) in zip(idx, want):
        band = np.abs(np.sqrt(r2) - RL) < 1e-9
        g = got[int(i)]
        g = g[~np.isin(g, j[band])]
        np.testing.assert_array_equal(g, j[~band])
    return n


def test_full_size_lattice(md, lattice):
    """The bench input at step 0: every fcc site has exactly 78 neighbours
    within r_cut + r_skin (79,872,000 pairs), the net force on every site
    vanishes, U/N = -6.3328120 with the shifted potential, K = 1/2 sum v^2,
    and the sampled neighbour rows are those of brute force."""
    x, v, box = lattice
    h = bench_handle(md, x, v, box, md.MD_FP32_FIXED)
    st = md.md_get_stats(h)
    assert st["list_entries"] == 78 * N and st["max_list_len"] == 78
    F, euw = gpu_forces(md, h)
    assert np.max(np.abs(F)) < 1e-5
    assert np.all(F.sum(axis=0) == 0.0)
    assert euw[0] / N == pytest.approx(-6.3328120, rel=1e-5)
    assert euw[1] == pytest.approx(0.5 * np.sum(v * v), rel=1e-9)
    # virial per site from the four fcc shells inside r_cut (12, 6, 24, 12
    # sites at a sqrt(m/2)): 1/2 sum count * 24 (2 r^-12 - r^-6)
    a = (4 / RHO) ** (1 / 3)
    w = 0.5 * sum(c * 24 * (2 * r ** -12 - r ** -6)
                  for c, r in zip([12, 6, 24, 12], a * np.sqrt(np.arange(1, 5) / 2)))
    assert euw[2] / N == pytest.approx(w, rel=1e-5)
    idx = np.random.default_rng(21).choice(N, 1024, replace=False)
    assert check_rows(md, h, x, box, idx) == 39 * N
    h.destroy()


@pytest.mark.parametrize("precision,tol", [(1, 1e-5), (0, 1e-12)])
def test_full_size_perturbed_forces_and_rows(md, perturbed, precision, tol):
    """The displaced lattice (non-zero forces everywhere): forces on 4096
    sampled particles follow the oracle's exact O(N) sums for them, the
    sampled neighbour rows are brute force's, and in fixed point the forces
    of the whole system sum to exactly zero."""
    x, v, box = perturbed
    h = bench_handle(md, x, v, box, precision)
    F, euw = gpu_forces(md, h)
    idx = np.random.default_rng(22).choice(N, 4096, replace=False)
    Fo, _, _ = oracle.forces_sample(oracle.System(N, box, rc=RC), x, idx)
    assert force_rel_err(F[idx], Fo) <= tol
    if precision == 1:
        assert np.all(F.sum(axis=0) == 0.0)
    check_rows(md, h, x, box, idx[:1024])
    h.destroy()


def test_full_size_first_step(md, perturbed):
    """One graph-launched md_step from the displaced lattice: for sampled
    particles x_1 = x_0 + dt v_0 + dt^2/(2m) F(x_0) (Fig. 1), with F from the
    oracle's exact sums, within what the FP32 force tolerance allows."""
    x, v, box = perturbed
    h = bench_handle(md, x, v, box, md.MD_FP32_FIXED)
    md.md_step(h, 1)
    x1, _ = gpu_state(md, h)
    idx = np.random.default_rng(23).choice(N, 4096, replace=False)
    Fo, _, _ = oracle.forces_sample(oracle.System(N, box, rc=RC), x, idx)
    want = x[idx] + DT * v[idx] + 0.5 * DT * DT * Fo
    err = np.linalg.norm(min_image_diff(x1[idx], want, box), axis=1)
    assert np.all(err <= first_step_bound(Fo, 1e-5))
    h.destroy()


def test_full_size_reversibility_momentum_energy(md, perturbed):
    """20 graph-launched steps forward with (U, K, W) every step, velocities
    negated, 20 steps back: the positions return to the start (velocity Verlet
    is time-reversible; a force that depended on anything but the positions,
    or a list missing a pair, would break it), total momentum stays at its
    start value, and the energy stays within 5e-4 of its start."""
    x, v, box = perturbed
    h = bench_handle(md, x, v, box, md.MD_FP32_FIXED)
    th = np.zeros((20, 3))
    md.md_step(h, 20, 1, th)
    x20, v20 = gpu_state(md, h)
    st = md.md_get_stats(h)
    assert st["rebuilds"] >= 2
    p0 = v.sum(axis=0)
    assert np.max(np.abs(v20.sum(axis=0) - p0)) < 1e-9
    E = th[:, 0] + th[:, 1]
    assert np.max(np.abs(E - E[0])) / abs(E[0]) < 5e-4
    md.md_set_state(h, dev(x20), dev(-v20))
    md.md_step(h, 20)
    xb, vb = gpu_state(md, h)
    assert np.max(np.abs(min_image_diff(xb, x, box))) < 1e-8
    assert np.max(np.abs(vb + v)) < 1e-6
    h.destroy()


# ------------------------------------------------------------------ the other workloads at full size
def sampled_check(md, h, n, sysm, x, idx, tol, bonded=False):
    """Forces of md_compute_forces on particles idx against the oracle's
    exact sums for them (non-bonded over all j, plus the bonded terms)."""
    f = torch.zeros(3, n, dtype=torch.float64, device="cuda")
    md.md_compute_forces(h, f, None)
    md.md_sync(h)
    F = f.cpu().numpy().T
    Fo, _, _ = oracle.forces_sample(sysm, x, idx)
    if bonded:
        Fo = Fo + oracle.bonded_sample(sysm, x, idx)
    assert force_rel_err(F[idx], Fo) <= tol
    return F


def test_full_size_slab(md, report):
    """The liquid/vapour slab of the bench (N = 1,000,000, Lz = 4 Lx, liquid
    0.80 in the central quarter of z, vapour 0.02): forces of 2048 sampled
    particles, half of them from the vapour, and the neighbour rows of 512;
    the first graph-launched step for the same particles; then the invariants
    of a 300-step FP32 run (momentum, energy, reversibility)."""
    x, v, box = inputs.slab(1_000_000, rho_l=0.80, rho_v=0.02, T=0.8, seed=3, rmin=0.8)
    n = len(x)
    h = md.md_create(n, box, rc_over_sigma=RC, skin=SKIN, dt=DT, precision=md.MD_FP32_FIXED)
    md.md_set_state(h, dev(x), dev(v))
    md.md_build_neighbors(h)
    md.md_autotune(h, 10)
    z = x[:, 2] / box[2]
    liquid = (z >= 0.375) & (z < 0.625)
    rng = np.random.default_rng(31)
    idx = np.concatenate([rng.choice(np.nonzero(liquid)[0], 1024, replace=False),
                          rng.choice(np.nonzero(~liquid)[0], 1024, replace=False)])
    s = oracle.System(n, box, rc=RC)
    F = sampled_check(md, h, n, s, x, idx, 1e-5)
    assert np.all(F.sum(axis=0) == 0.0)
    want = oracle.neighbours_sample(s, x, idx[::4], RL)
    _, got = gpu_rows(md, h, idx[::4], n)
    for i, (j, r2) in zip(idx[::4], want):
        band = np.abs(np.sqrt(r2) - RL) < 1e-9
        g = got[int(i)]
        np.testing.assert_array_equal(g[~np.isin(g, j[band])], j[~band])
    md.md_step(h, 1)
    xo = torch.zeros(3, n, dtype=torch.float64, device="cuda")
    md.md_get_state(h, xo, None)
    x1 = xo.cpu().numpy().T
    Fo, _, _ = oracle.forces_sample(s, x, idx)
    err = np.linalg.norm(min_image_diff(x1[idx], x[idx] + DT * v[idx] + 0.5 * DT * DT * Fo, box), axis=1)
    assert np.all(err <= first_step_bound(Fo, 1e-5))
    # the timed run itself: 300 graph-launched FP32 steps with (U, K, W) every
    # step.  The fixed-point forces sum to exactly zero, so the total momentum
    # moves only by the FP64 rounding of the kicks; 20 steps back with negated
    # velocities return to the start.  The random placement (pairs down to
    # 0.8 sigma) starts violent collisions, so the energy error is the time
    # step's: the same time at dt / 2 cuts it about fourfold (second order).
    def state(hh):
        xo = torch.zeros(3, n, dtype=torch.float64, device="cuda")
        vo = torch.zeros_like(xo)
        md.md_get_state(hh, xo, vo)
        return xo.cpu().numpy().T.copy(), vo.cpu().numpy().T.copy()

    th = np.zeros((300, 3))
    md.md_step(h, 300, 1, th)
    x300, v300 = state(h)
    p1 = v300.sum(axis=0)
    E = th[:, 0] + th[:, 1]
    dE = float(np.max(np.abs(E - E[0])) / abs(E[0]))
    st = md.md_get_stats(h)
    h2 = md.md_create(n, box, rc_over_sigma=RC, skin=SKIN, dt=DT / 2, precision=md.MD_FP32_FIXED)
    md.md_set_state(h2, dev(x), dev(v))
    md.md_step(h2, 2)
    th2 = np.zeros((602, 3))
    md.md_step(h2, 602, 1, th2)
    E2 = th2[:, 0] + th2[:, 1]
    dE2 = float(np.max(np.abs(E2 - E2[0])) / abs(E2[0]))
    h2.destroy()
    report(f"slab N={n}, 300 FP32 steps: rebuilds {st['rebuilds']}, |sum p| {np.max(np.abs(p1)):.2e}, "
           f"max |E - E0| / |E0| {dE:.2e} at dt {DT}, {dE2:.2e} at dt {DT / 2}")
    assert np.max(np.abs(p1 - v.sum(axis=0))) < 1e-8
    assert dE2 < dE / 2.5
    md.md_step(h, 20)
    x20, v20 = state(h)
    md.md_set_state(h, dev(x20), dev(-v20))
    md.md_step(h, 20)
    xb, vb = state(h)
    rev = float(np.max(np.abs(min_image_diff(xb, x300, box))))
    report(f"slab N={n}: 20 steps forward and back, max |x - x0| {rev:.2e}")
    assert rev < 1e-7
    h.destroy()


def test_full_size_sphere_langevin(md):
    """The paper's spherical system (2,580,000 particles in a sphere of radius
    90 in a box of edge 271, Langevin at T = 0.1, gamma = 0.5): conservative
    forces of 2048 sampled particles, half of them within 3 sigma of the
    surface (where the forces do not cancel); after one graph-launched step,
    x_1 = x_0 + dt v_0 + dt^2/2m (F + F_L) with the oracle's Langevin force
    (Philox noise of step 0) for the same particles."""
    x, v, box = inputs.sphere()
    n = len(x)
    h = md.md_create(n, box, rc_over_sigma=RC, skin=SKIN, dt=DT, precision=md.MD_FP32_FIXED,
                     langevin_gamma=0.5, kT=0.1, seed=6)
    md.md_set_state(h, dev(x), dev(v))
    md.md_build_neighbors(h)
    md.md_autotune(h, 10)
    r = np.linalg.norm(x - 0.5 * box, axis=1)
    rng = np.random.default_rng(32)
    idx = np.concatenate([rng.choice(np.nonzero(r > r.max() - 3.0)[0], 1024, replace=False),
                          rng.choice(np.nonzero(r <= r.max() - 3.0)[0], 1024, replace=False)])
    s = oracle.System(n, box, rc=RC, dt=DT, gamma=0.5, kT=0.1, seed=6)
    sampled_check(md, h, n, s, x, idx, 1e-5)
    md.md_step(h, 1)
    xo = torch.zeros(3, n, dtype=torch.float64, device="cuda")
    md.md_get_state(h, xo, None)
    x1 = xo.cpu().numpy().T
    Fo, _, _ = oracle.forces_sample(s, x, idx)
    FL = oracle.langevin_sample(s, idx, v[idx], 0)
    want = x[idx] + DT * v[idx] + 0.5 * DT * DT * (Fo + FL)
    err = np.linalg.norm(min_image_diff(x1[idx], want, box), axis=1)
    assert np.all(err <= first_step_bound(Fo, 1e-5))
    h.destroy()


@pytest.mark.parametrize("system", ["melt", "rings"])
def test_full_size_polymer_preparation(md, system):
    """The polymer melts of the bench at full size (2000 x 200 linear chains,
    1600 x 200 rings with the angle term), as generated (free random walks,
    overlaps left in), in the first stage of the bench's preparation: the
    cosine push-off (A = 1) with FENE bonds in FP64.  Forces of 2048 sampled
    particles (non-bonded plus bonded) against the oracle, and their
    neighbour rows.  In FP32 + fixed point the same overlapping chains under
    WCA exceed the fixed-point range, and the library reports it."""
    rc = 2 ** (1 / 6)
    if system == "melt":
        x, v, box, bonds = inputs.melt(2000, 200, rho=0.85, T=1.0, seed=4)
        angles, aK = None, 0.0
    else:
        x, v, box, bonds, angles = inputs.rings(1600, 200, rho=0.85, T=1.0, seed=7)
        aK = 1.5
    n = len(x)
    common = dict(skin=0.4, bonds=bonds, fene_K=30.0, fene_R0=1.5, langevin_gamma=0.5, kT=1.0,
                  angles=angles, angle_K=aK)
    h = md.md_create(n, box, potential=md.MD_SOFT, rc_over_sigma=rc, eps=1.0, dt=0.005,
                     precision=md.MD_FP64, seed=100, **common)
    md.md_set_state(h, dev(x), dev(v))
    md.md_build_neighbors(h)
    idx = np.random.default_rng(33).choice(n, 2048, replace=False)
    s = oracle.System(n, box, eps=1.0, rc=rc, soft=True, bonds=bonds, fene_K=30.0, fene_R0=1.5,
                      angles=angles, angle_K=aK)
    sampled_check(md, h, n, s, x, idx, 1e-12, bonded=True)
    rl = rc + 0.4
    want = oracle.neighbours_sample(s, x, idx[:512], rl)
    _, got = gpu_rows(md, h, idx[:512], n)
    for i, (j, r2) in zip(idx[:512], want):
        band = np.abs(np.sqrt(r2) - rl) < 1e-9
        g = got[int(i)]
        np.testing.assert_array_equal(g[~np.isin(g, j[band])], j[~band])
    h.destroy()
    hw = md.md_create(n, box, potential=md.MD_WCA, dt=0.005, precision=md.MD_FP32_FIXED, seed=200, **common)
    md.md_set_state(hw, dev(x), dev(v))
    md.md_build_neighbors(hw)
    f = torch.zeros(3, n, dtype=torch.float64, device="cuda")
    md.md_compute_forces(hw, f, None)
    with pytest.raises(md.MDError) as e:
        md.md_sync(hw)
    assert e.value.status == md.MD_ERR_FIXED_OVERFLOW
    hw.destroy()


def test_full_size_ensemble_forces_and_adjoint(md):
    """The batched ensemble of the bench (64 replicas, N log-uniform in
    [500, 32000], 412,837 particles, per-replica eps and sigma, r_cut = 2.5
    sigma): forces of 16 sampled particles per replica against the oracle run
    on each replica alone.  Then the adjoint of every replica's loss
    U/N + (2K + W)/(3V) after an FP64 forward of 5 steps against central
    differences of that forward (all replicas displaced at once: they are
    independent), to 1e-4 relative: d/d(eps) with the LJ potential
    (h = 1e-8 eps), d/d(sigma) with WCA (h = 1e-6 sigma).  With LJ, r_cut =
    2.5 sigma moves with sigma and the force and virial jump there, so among
    400,000 particles some pair would cross r_cut inside any difference wide
    enough to resolve; WCA's force and virial vanish at r_cut, so crossings
    leave the derivative intact."""
    sizes, boxes, eps, sig, x, v = inputs.ensemble()
    n = int(sizes.sum())
    R = len(sizes)
    off = np.concatenate([[0], np.cumsum(sizes)])
    h = md.md_create(sizes, boxes, eps=eps, sigma=sig, rc_over_sigma=RC, skin=SKIN, dt=DT,
                     precision=md.MD_FP32_FIXED)
    md.md_set_state(h, dev(x), dev(v))
    md.md_build_neighbors(h)
    f = torch.zeros(3, n, dtype=torch.float64, device="cuda")
    md.md_compute_forces(h, f, None)
    md.md_sync(h)
    F = f.cpu().numpy().T
    rng = np.random.default_rng(34)
    for r in range(R):
        xr = x[off[r]:off[r + 1]]
        s = oracle.System(int(sizes[r]), boxes[r], eps=float(eps[r]), sigma=float(sig[r]), rc=RC * float(sig[r]))
        idx = rng.choice(int(sizes[r]), 16, replace=False)
        Fo, _, _ = oracle.forces_sample(s, xr, idx)
        assert force_rel_err(F[off[r] + idx], Fo) <= 1e-5
    h.destroy()

    vol = np.prod(boxes, axis=1)
    coef = np.stack([1.0 / sizes, 2.0 / (3.0 * vol), 1.0 / (3.0 * vol)], axis=1)

    def forward(e, sg, pot, keep=False):
        hh = md.md_create(sizes, boxes, eps=e, sigma=sg, rc_over_sigma=RC, skin=SKIN, dt=DT,
                          potential=pot, precision=md.MD_FP64)
        md.md_set_state(hh, dev(x), dev(v))
        md.md_build_neighbors(hh)
        euw = np.zeros((R, 3))
        md.md_forward(hh, 5, 5, euw)
        loss = np.sum(coef * euw, axis=1)
        if keep:
            return hh, loss
        hh.destroy()
        return loss

    for pot, which, hrel in ((md.MD_LJ, 0, 1e-8), (md.MD_WCA, 1, 1e-6)):
        h0, _ = forward(eps, sig, pot, keep=True)
        ge, gs = np.zeros(R), np.zeros(R)
        md.md_backward(h0, None, None, coef, ge, gs)
        h0.destroy()
        if which == 0:
            fd = (forward(eps * (1 + hrel), sig, pot) - forward(eps * (1 - hrel), sig, pot)) / (2 * hrel * eps)
            np.testing.assert_allclose(ge, fd, rtol=1e-4)
        else:
            fd = (forward(eps, sig * (1 + hrel), pot) - forward(eps, sig * (1 - hrel), pot)) / (2 * hrel * sig)
            np.testing.assert_allclose(gs, fd, rtol=1e-4)
