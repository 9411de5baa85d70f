"""Parity of the CUDA path with the FP64 oracle on the other workload shapes:
several independent replicas in one handle, FENE-bonded chains with WCA, the
Langevin thermostat, and an inhomogeneous liquid/vapour slab."""
import numpy as np
import pytest

import oracle
from paper_2109_10876_gb300 import inputs
from tests.helpers import force_rel_err, min_image_diff

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


@pytest.fixture(scope="module")
def md():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_10876_gb300 import md as m
    return m


def dev(a):
    return torch.tensor(np.ascontiguousarray(np.asarray(a).T), dtype=torch.float64, device="cuda")


def host(t):
    return t.cpu().numpy().T.copy()


@pytest.mark.parametrize("precision", [0, 1])
def test_replicas_forces_energies_pairs(md, precision):
    """Replicas of uneven size with their own box, eps and sigma (rc = 2.5 sigma
    each): forces, (U, K, W) per replica and the pair set match the oracle run
    on each replica alone."""
    sizes, boxes, eps, sig = [], [], [], []
    xs, vs = [], []
    rng = np.random.default_rng(31)
    for r, nc in enumerate([5, 6, 7, 5]):
        s = rng.uniform(0.95, 1.05)
        x, v, box = inputs.perturbed_lattice(nc, rho=0.8442, T=0.72, seed=40 + r, amp=0.12)
        x, box = x * s, box * s                       # density 0.8442 in units of sigma
        cut = [500, 864, 1372 - 7, 500][r]            # ragged replica sizes
        xs.append(x[:cut]); vs.append(v[:cut])
        sizes.append(cut); boxes.append(box); eps.append(rng.uniform(0.9, 1.1)); sig.append(s)
    X, V = np.concatenate(xs), np.concatenate(vs)
    N = len(X)
    h = md.md_create(sizes, np.array(boxes), eps=np.array(eps), sigma=np.array(sig), precision=precision)
    md.md_set_state(h, dev(X), dev(V))
    md.md_build_neighbors(h)
    f = torch.zeros(3, N, dtype=torch.float64, device="cuda")
    euw = torch.zeros(len(sizes), 3, dtype=torch.float64, device="cuda")
    md.md_compute_forces(h, f, euw)
    md.md_sync(h)
    F, E = host(f), euw.cpu().numpy()
    pairs = md.export_pairs_sorted(h)
    off = np.concatenate([[0], np.cumsum(sizes)])
    for r in range(len(sizes)):
        s = oracle.System(sizes[r], boxes[r], eps=eps[r], sigma=sig[r], rc=2.5 * sig[r])
        Fr, er = oracle.forces(s, xs[r], vs[r])
        assert force_rel_err(F[off[r]:off[r + 1]], Fr) <= TOL[precision]
        np.testing.assert_allclose(E[r], er, rtol=TOL[precision], atol=TOL[precision] * sizes[r])
        want, _ = oracle.pairs(s, xs[r], 2.5 * sig[r] + 0.3)
        got = pairs[(pairs[:, 0] >= off[r]) & (pairs[:, 0] < off[r + 1])] - off[r]
        np.testing.assert_array_equal(got, want)
    assert np.all(pairs[:, 1] < np.repeat(off[1:], np.diff(off))[pairs[:, 0]])   # no pair across replicas


def test_many_replicas_energy_sums(md):
    """160 replicas of 500 particles (about 1,400 tiles, more than the
    persistent blocks, so most blocks take tiles of several replicas in turn
    and add their energy sums per replica as the replica changes): forces and
    (U, K, W) of every replica match the oracle run on it alone, in FP32 with
    fixed-point sums; 10 steps with (U, K, W) recorded every step keep every
    record finite and the last one equal to a force evaluation of the final
    state in U and W."""
    R = 160
    rng = np.random.default_rng(77)
    sizes, boxes, eps, sig, xs, vs = [], [], [], [], [], []
    for r in range(R):
        s = rng.uniform(0.95, 1.05)
        x, v, box = inputs.perturbed_lattice(5, seed=300 + r, amp=0.1)
        xs.append(x * s); vs.append(v)
        sizes.append(len(x)); boxes.append(box * s); eps.append(rng.uniform(0.9, 1.1)); sig.append(s)
    X, V = np.concatenate(xs), np.concatenate(vs)
    N = len(X)
    h = md.md_create(sizes, np.array(boxes), eps=np.array(eps), sigma=np.array(sig), precision=md.MD_FP32_FIXED)
    md.md_set_state(h, dev(X), dev(V))
    md.md_build_neighbors(h)
    f = torch.zeros(3, N, dtype=torch.float64, device="cuda")
    euw = torch.zeros(R, 3, dtype=torch.float64, device="cuda")
    md.md_compute_forces(h, f, euw)
    md.md_sync(h)
    F, E = host(f), euw.cpu().numpy()
    off = np.concatenate([[0], np.cumsum(sizes)])
    for r in range(R):
        s = oracle.System(sizes[r], boxes[r], eps=eps[r], sigma=sig[r], rc=2.5 * sig[r])
        Fr, er = oracle.forces(s, xs[r], vs[r])
        assert force_rel_err(F[off[r]:off[r + 1]], Fr) <= TOL[1]
        np.testing.assert_allclose(E[r], er, rtol=TOL[1], atol=TOL[1] * sizes[r])
    # a second evaluation gives the same sums (the accumulators were cleared)
    euw2 = torch.zeros(R, 3, dtype=torch.float64, device="cuda")
    md.md_compute_forces(h, f, euw2)
    md.md_sync(h)
    np.testing.assert_array_equal(euw2.cpu().numpy(), E)
    th = np.zeros((10, R, 3))
    md.md_step(h, 10, 1, th)
    assert np.all(np.isfinite(th))
    euw3 = torch.zeros(R, 3, dtype=torch.float64, device="cuda")
    md.md_compute_forces(h, f, euw3)
    md.md_sync(h)
    e3 = euw3.cpu().numpy()
    np.testing.assert_array_equal(th[-1][:, 0], e3[:, 0])
    np.testing.assert_array_equal(th[-1][:, 2], e3[:, 2])


def test_replicas_trajectory_fp64(md):
    """Two replicas stepped together follow the oracle run on each alone."""
    a = inputs.lj_fluid(5, T=0.72, seed=51)
    b = inputs.perturbed_lattice(6, T=1.0, seed=52, amp=0.1)
    X, V = np.concatenate([a[0], b[0]]), np.concatenate([a[1], b[1]])
    h = md.md_create([len(a[0]), len(b[0])], np.array([a[2], b[2]]), precision=0)
    md.md_set_state(h, dev(X), dev(V))
    md.md_build_neighbors(h)
    md.md_step(h, 50)
    xo = torch.zeros(3, len(X), dtype=torch.float64, device="cuda")
    vo = torch.zeros_like(xo)
    md.md_get_state(h, xo, vo)
    xg = host(xo)
    for (x, v, box), sl in ((a, slice(0, len(a[0]))), (b, slice(len(a[0]), len(X)))):
        x1, v1, _ = oracle.vv_run(oracle.System(len(x), box, rc=2.5), x, v, 50)
        assert np.max(np.abs(min_image_diff(xg[sl], x1, box))) < 1e-10


@pytest.mark.parametrize("precision", [0, 1])
def test_fene_wca_forces(md, precision):
    box = np.array([9.0, 9.0, 9.0])
    x, bonds = inputs.chains(12, 25, box, seed=61)
    n = len(x)
    v = inputs.maxwell_velocities(n, 1.0, 62)
    h = md.md_create(n, box, potential=md.MD_WCA, skin=0.4, bonds=bonds, fene_K=30.0, fene_R0=1.5,
                     precision=precision)
    md.md_set_state(h, dev(x), dev(v))
    md.md_build_neighbors(h)
    f = torch.zeros(3, n, dtype=torch.float64, device="cuda")
    euw = torch.zeros(3, dtype=torch.float64, device="cuda")
    md.md_compute_forces(h, f, euw)
    md.md_sync(h)
    s = oracle.System(n, box, rc=2 ** (1 / 6), bonds=bonds, fene_K=30.0, fene_R0=1.5)
    Fr, er = oracle.forces(s, x, v)
    assert force_rel_err(host(f), Fr) <= TOL[precision]
    np.testing.assert_allclose(euw.cpu().numpy(), er, rtol=TOL[precision], atol=TOL[precision] * n)
    if precision == 1:
        assert np.all(host(f).sum(axis=0) == 0.0)


def test_langevin_melt_steps_fp64(md):
    """Kremer-Grest style chains, WCA + FENE + Langevin (gamma 0.5, T 1,
    dt 0.01): 20 steps follow the oracle, whose Philox noise is implemented
    independently from the same published definition."""
    box = np.array([9.0, 9.0, 9.0])
    x, bonds = inputs.chains(12, 25, box, seed=63)
    n = len(x)
    v = inputs.maxwell_velocities(n, 1.0, 64)
    kw = dict(potential=md.MD_WCA, skin=0.4, bonds=bonds, fene_K=30.0, fene_R0=1.5, dt=0.01,
              langevin_gamma=0.5, kT=1.0, seed=12345)
    h = md.md_create(n, box, precision=0, **kw)
    md.md_set_state(h, dev(x), dev(v))
    md.md_build_neighbors(h)
    md.md_step(h, 20)
    xo = torch.zeros(3, n, dtype=torch.float64, device="cuda")
    vo = torch.zeros_like(xo)
    md.md_get_state(h, xo, vo)
    s = oracle.System(n, box, rc=2 ** (1 / 6), bonds=bonds, fene_K=30.0, fene_R0=1.5, dt=0.01,
                      gamma=0.5, kT=1.0, seed=12345)
    x1, v1, _ = oracle.vv_run(s, x, v, 20)
    assert np.max(np.abs(min_image_diff(host(xo), x1, box))) < 1e-10
    assert np.max(np.abs(host(vo) - v1)) < 1e-9


def test_bond_broken_is_reported(md):
    box = np.array([9.0, 9.0, 9.0])
    x = np.array([[1.0, 1.0, 1.0], [2.6, 1.0, 1.0], [5.0, 5.0, 5.0]])
    h = md.md_create(3, box, potential=md.MD_WCA, skin=0.4, bonds=[[0, 1]], fene_R0=1.5)
    md.md_set_state(h, dev(x), dev(np.zeros_like(x)))
    md.md_build_neighbors(h)
    md.md_compute_forces(h, None, None)
    with pytest.raises(md.MDError) as e:
        md.md_sync(h)
    assert e.value.status == md.MD_ERR_BOND_BROKEN


@pytest.mark.parametrize("precision", [0, 1])
def test_slab_forces_and_pairs(md, precision):
    """Liquid/vapour slab (Lz = 4 Lx, liquid at 0.8 in the central quarter of z,
    vapour 0.02 elsewhere): very uneven cell occupancy and a non-cubic box."""
    x, v, box = inputs.slab(3000, rho_l=0.8, rho_v=0.02, T=0.8, seed=71)
    n = len(x)
    h = md.md_create(n, box, precision=precision)
    md.md_set_state(h, dev(x), dev(v))
    md.md_build_neighbors(h)
    f = torch.zeros(3, n, dtype=torch.float64, device="cuda")
    euw = torch.zeros(3, dtype=torch.float64, device="cuda")
    md.md_compute_forces(h, f, euw)
    md.md_sync(h)
    s = oracle.System(n, box, rc=2.5)
    Fr, er = oracle.forces(s, x, v)
    assert force_rel_err(host(f), Fr) <= TOL[precision]
    np.testing.assert_allclose(euw.cpu().numpy(), er, rtol=TOL[precision], atol=TOL[precision] * n)
    want, _ = oracle.pairs(s, x, 2.8)
    np.testing.assert_array_equal(md.export_pairs_sorted(h), want)


def test_soft_pushoff_fene_langevin_fp64(md):
    """Melt preparation: free random-walk chains (overlapping beads, some
    coincident) under the cosine push-off with FENE bonds and the Langevin
    thermostat.  Forces and energies match the oracle at the start, and 20
    steps follow the oracle's trajectory."""
    x, v, box, bonds = inputs.melt(nchain=10, nbead=20, rho=0.85, seed=41)
    n = len(x)
    rc = 2 ** (1 / 6)
    kw = dict(potential=md.MD_SOFT, rc_over_sigma=rc, eps=5.0, skin=0.4, bonds=bonds, fene_K=30.0,
              fene_R0=1.5, dt=0.005, langevin_gamma=0.5, kT=1.0, seed=77)
    h = md.md_create(n, box, precision=0, **kw)
    md.md_set_state(h, dev(x), dev(v))
    md.md_build_neighbors(h)
    f = torch.zeros(3, n, dtype=torch.float64, device="cuda")
    euw = torch.zeros(1, 3, dtype=torch.float64, device="cuda")
    md.md_compute_forces(h, f, euw)
    md.md_sync(h)
    s = oracle.System(n, box, eps=5.0, rc=rc, soft=True, bonds=bonds, fene_K=30.0, fene_R0=1.5, dt=0.005,
                      gamma=0.5, kT=1.0, seed=77)
    Fo, eo = oracle.forces(s, x, v)
    assert force_rel_err(host(f), Fo) <= 1e-12
    np.testing.assert_allclose(euw.cpu().numpy()[0], eo, rtol=1e-12, atol=1e-12 * n)
    md.md_step(h, 20)
    xo = torch.zeros(3, n, dtype=torch.float64, device="cuda")
    vo = torch.zeros_like(xo)
    md.md_get_state(h, xo, vo)
    x1, v1, _ = oracle.vv_run(s, x, v, 20)
    assert np.max(np.abs(min_image_diff(host(xo), x1, box))) < 1e-10
    assert np.max(np.abs(host(vo) - v1)) < 1e-9


def test_soft_pushoff_needs_fp64(md):
    x, v, box, bonds = inputs.melt(nchain=4, nbead=10, rho=0.85, seed=42)
    with pytest.raises(md.MDError):
        md.md_create(len(x), box, potential=md.MD_SOFT, rc_over_sigma=2 ** (1 / 6), precision=1)


def test_rings_with_angles_fp64(md):
    """Ring polymers (Sec. 4) under the push-off with FENE bonds, the cosine
    angle term and the Langevin thermostat: forces and energies match the
    oracle, and 20 steps follow its trajectory."""
    x, v, box, bonds, angles = inputs.rings(8, 30, rho=0.6, seed=51)
    n = len(x)
    rc = 2 ** (1 / 6)
    kw = dict(potential=md.MD_SOFT, rc_over_sigma=rc, eps=5.0, skin=0.4, bonds=bonds, angles=angles,
              angle_K=1.5, dt=0.005, langevin_gamma=0.5, kT=1.0, seed=5)
    h = md.md_create(n, box, precision=0, **kw)
    md.md_set_state(h, dev(x), dev(v))
    md.md_build_neighbors(h)
    f = torch.zeros(3, n, dtype=torch.float64, device="cuda")
    euw = torch.zeros(1, 3, dtype=torch.float64, device="cuda")
    md.md_compute_forces(h, f, euw)
    md.md_sync(h)
    s = oracle.System(n, box, eps=5.0, rc=rc, soft=True, bonds=bonds, angles=angles, angle_K=1.5, dt=0.005,
                      gamma=0.5, kT=1.0, seed=5)
    Fo, eo = oracle.forces(s, x, v)
    assert force_rel_err(host(f), Fo) <= 1e-12
    np.testing.assert_allclose(euw.cpu().numpy()[0], eo, rtol=1e-12, atol=1e-12 * n)
    md.md_step(h, 20)
    xo = torch.zeros(3, n, dtype=torch.float64, device="cuda")
    vo = torch.zeros_like(xo)
    md.md_get_state(h, xo, vo)
    x1, v1, _ = oracle.vv_run(s, x, v, 20)
    assert np.max(np.abs(min_image_diff(host(xo), x1, box))) < 1e-10
    assert np.max(np.abs(host(vo) - v1)) < 1e-9


def test_chains_wca_fene_angles_fp32(md):
    """Self-avoiding linear chains with WCA, FENE and the angle term on every
    interior triple, FP32 pairs and fixed-point sums: forces and energies
    within 1e-5 of the oracle, and the total force is exactly zero."""
    box = np.array([9.0, 9.0, 9.0])
    x, bonds = inputs.chains(12, 25, box, seed=52)
    n = len(x)
    v = inputs.maxwell_velocities(n, 1.0, 53)
    angles = np.array([(c * 25 + k - 1, c * 25 + k, c * 25 + k + 1) for c in range(12) for k in range(1, 24)],
                      dtype=np.int32)
    kw = dict(potential=md.MD_WCA, skin=0.4, bonds=bonds, fene_K=30.0, fene_R0=1.5, angles=angles, angle_K=1.5)
    h = md.md_create(n, box, precision=1, **kw)
    md.md_set_state(h, dev(x), dev(v))
    md.md_build_neighbors(h)
    f = torch.zeros(3, n, dtype=torch.float64, device="cuda")
    euw = torch.zeros(1, 3, dtype=torch.float64, device="cuda")
    md.md_compute_forces(h, f, euw)
    md.md_sync(h)
    s = oracle.System(n, box, rc=2 ** (1 / 6), bonds=bonds, fene_K=30.0, fene_R0=1.5, angles=angles, angle_K=1.5)
    Fo, eo = oracle.forces(s, x, v)
    F = host(f)
    assert force_rel_err(F, Fo) <= 1e-5
    np.testing.assert_allclose(euw.cpu().numpy()[0], eo, rtol=1e-5, atol=1e-5 * n)
    assert np.all(F.sum(axis=0) == 0.0)


def test_angles_rejected_by_the_adjoint(md):
    x, v, box, bonds, angles = inputs.rings(2, 10, rho=0.2, seed=54)
    h = md.md_create(len(x), box, precision=0, potential=md.MD_WCA, bonds=bonds, angles=angles, angle_K=1.0)
    md.md_set_state(h, dev(x), dev(v))
    with pytest.raises(md.MDError) as e:
        md.md_forward(h, 2, 1, np.zeros(3))
    assert e.value.status == md.MD_ERR_ARG
