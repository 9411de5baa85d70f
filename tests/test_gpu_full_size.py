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


def gpu_rows(md, h, idx):
    """Neighbour rows of the particles idx from the exported Verlet list."""
    n = md.md_export_pairs(h, None, 0)
    out = np.zeros((n, 2), dtype=np.int32)
    assert md.md_export_pairs(h, out, n) == n
    sel = np.zeros(N, dtype=bool)
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
    oracle's exact sums."""
    x, v, box = perturbed
    h = bench_handle(md, x, v, box, md.MD_FP32_FIXED)
    md.md_step(h, 1)
    x1, _ = gpu_state(md, h)
    idx = np.random.default_rng(23).choice(N, 4096, replace=False)
    Fo, _, _ = oracle.forces_sample(oracle.System(N, box, rc=RC), x, idx)
    want = x[idx] + DT * v[idx] + 0.5 * DT * DT * Fo
    assert np.max(np.abs(min_image_diff(x1[idx], want, box))) < 1e-8
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
