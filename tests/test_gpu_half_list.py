"""The half Verlet list of Newton's third law (Sec. 2.1.2) against the oracle
and against the full list, through the C ABI.

Each pair is stored once and its force goes to both particles, the partner's
share by 64-bit fixed-point atomic adds.  Because every pair force is rounded
to the fixed point identically from either end (the rounding is an odd
function and the separations are exact integers), the half-list forces must
equal the full-list forces bit for bit, and so must whole trajectories.
Pair sets: bit-exact against brute force, each pair once.  Forces: 1e-5
relative against the FP64 oracle (the FP32 bound); energies to the same
relative bound.
"""
import numpy as np
import pytest

import oracle
from paper_2109_10876_gb300 import inputs
from tests.helpers import force_rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RC, SKIN = 2.5, 0.3
TOL = 1e-5


@pytest.fixture(scope="module")
def md():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_10876_gb300 import md as m
    return m


def dev(a):
    return torch.tensor(np.ascontiguousarray(np.asarray(a).T), dtype=torch.float64, device="cuda")


def make(md, x, v, box, half, **kw):
    h = md.md_create(len(x), box, precision=md.MD_FP32_FIXED, skin=kw.pop("skin", SKIN), **kw)
    if half:
        md.md_set_half_list(h, True)
    md.md_set_state(h, dev(x), dev(v))
    md.md_build_neighbors(h)
    return h


def forces(md, h, n, nrep=1):
    f = torch.zeros(3, n, dtype=torch.float64, device="cuda")
    euw = torch.zeros(nrep, 3, dtype=torch.float64, device="cuda")
    md.md_compute_forces(h, f, euw)
    md.md_sync(h)
    return f.cpu().numpy().T.copy(), euw.cpu().numpy().copy()


def state(md, h, n):
    xo = torch.zeros(3, n, dtype=torch.float64, device="cuda")
    vo = torch.zeros_like(xo)
    md.md_get_state(h, xo, vo)
    return xo.cpu().numpy().T.copy(), vo.cpu().numpy().T.copy()


def test_half_pair_set_fcc_4000(md):
    """fcc N = 4000: 78 neighbours within r_cut + r_skin, so the half list
    holds 156000 entries, one per pair, equal to the brute-force pair set."""
    x, v, box = inputs.lj_fluid(10, seed=1)
    h = make(md, x, v, box, True)
    got = md.export_pairs_sorted(h)
    want, _ = oracle.pairs(oracle.System(len(x), box, rc=RC), x, RC + SKIN)
    assert len(got) == 156000
    np.testing.assert_array_equal(got, want)
    st = md.md_get_stats(h)
    assert st["list_entries"] == 156000


@pytest.mark.parametrize("n,boxl,seed", [(4000, 16.796, 2), (777, 9.1, 3), (60, 5.7, 4), (1, 6.0, 5)])
def test_half_pair_set_random(md, n, boxl, seed):
    """Random points (ragged N, boxes of 1 to 3 cells per axis, pairs across
    the periodic boundary, a lone particle): each pair exactly once, equal to
    brute force."""
    box = np.array([boxl, boxl * 1.03, boxl * 0.98]) if boxl > 5.7 else np.array([boxl] * 3)
    x = inputs.random_gas(n, box, seed=seed)
    h = make(md, x, np.zeros_like(x), box, True)
    got = md.export_pairs_sorted(h)
    want, _ = oracle.pairs(oracle.System(n, box, rc=RC), x, RC + SKIN)
    np.testing.assert_array_equal(got.reshape(-1, 2), want.reshape(-1, 2))
    assert md.md_get_stats(h)["list_entries"] == len(want.reshape(-1, 2))


def test_half_empty_and_single_particle_replicas(md):
    """Replicas of 0, 1 and 500 particles in one handle: forces and energies
    with the half list equal the full list's; 20 steps stay identical."""
    x3, v3, b3 = inputs.perturbed_lattice(5, seed=61, amp=0.1)
    x = np.concatenate([[[1.0, 2.0, 3.0]], x3])
    v = np.concatenate([[[0.1, -0.2, 0.3]], v3])
    sizes = [0, 1, len(x3)]
    boxes = np.array([[9.0, 9.0, 9.0], [7.0, 8.0, 9.0], b3])
    res = []
    for half in (False, True):
        h = md.md_create(sizes, boxes)
        if half:
            md.md_set_half_list(h, True)
        md.md_set_state(h, dev(x), dev(v))
        md.md_build_neighbors(h)
        F, euw = forces(md, h, len(x), 3)
        md.md_step(h, 20)
        res.append((F, euw, state(md, h, len(x))))
    np.testing.assert_array_equal(res[1][0], res[0][0])
    assert np.all(res[1][1][0] == 0.0) and res[1][1][1][0] == 0.0
    np.testing.assert_allclose(res[1][1], res[0][1], rtol=1e-6, atol=1e-6 * len(x))
    np.testing.assert_array_equal(res[1][2][0], res[0][2][0])
    np.testing.assert_array_equal(res[1][2][1], res[0][2][1])


@pytest.mark.parametrize("case", ["liquid", "gas_small_box", "wca"])
def test_half_forces_equal_full_list_bit_for_bit(md, case):
    """Forces from the half list are the full list's bit for bit, sum to
    exactly zero, and follow the FP64 oracle to 1e-5; energies and virial
    agree with the oracle to 1e-5 relative."""
    kw = {}
    rc = RC
    if case == "liquid":
        x, v, box = inputs.perturbed_lattice(10, seed=7, amp=0.2)
        x, v = x[:3999], v[:3999]
    elif case == "gas_small_box":
        box = np.array([6.1, 6.1, 6.1])
        x = inputs.random_gas(90, box, seed=9, rmin=0.85)
        v = inputs.maxwell_velocities(90, 1.0, 10)
    else:
        box = np.array([9.0, 9.0, 9.0])
        x = inputs.random_gas(600, box, seed=12, rmin=0.8)
        v = np.zeros_like(x)
        kw = dict(potential=md.MD_WCA, skin=0.4)
        rc = 2 ** (1 / 6)
    n = len(x)
    Ff, Ef = forces(md, make(md, x, v, box, False, **dict(kw)), n)
    Fh, Eh = forces(md, make(md, x, v, box, True, **dict(kw)), n)
    np.testing.assert_array_equal(Fh, Ff)
    assert np.all(Fh.sum(axis=0) == 0.0)
    F_ref, e_ref = oracle.forces(oracle.System(n, box, rc=rc), x, v)
    assert force_rel_err(Fh, F_ref) <= TOL
    for k in range(3):
        assert Eh[0, k] == pytest.approx(e_ref[k], rel=TOL, abs=TOL * n)
    np.testing.assert_allclose(Eh, Ef, rtol=1e-6, atol=1e-6 * n)


@pytest.mark.parametrize("mode", ["graph", "graph_energies", "stream"])
def test_half_trajectory_equals_full_list(md, mode):
    """100 steps of the N = 4000 LJ fluid (dt = 0.005, rebuilds on the way):
    positions and velocities with the half list equal the full list's bit for
    bit, through the graph-launched step loop (with and without energies every
    step) and through stream launches (section timers on)."""
    x, v, box = inputs.lj_fluid(10, T=0.72, seed=1)
    n = len(x)
    out = []
    for half in (False, True):
        h = make(md, x, v, box, half)
        if mode == "stream":
            md.md_set_timing(h, True)
        if mode == "graph_energies":
            th = np.zeros((100, 3))
            md.md_step(h, 100, 1, th)
        else:
            th = None
            md.md_step(h, 100)
        out.append((state(md, h, n), th, md.md_get_stats(h)))
    (xf, vf), thf, sf = out[0]
    (xh, vh), thh, sh = out[1]
    np.testing.assert_array_equal(xh, xf)
    np.testing.assert_array_equal(vh, vf)
    assert sh["rebuilds"] == sf["rebuilds"] >= 2
    assert 2 * sh["list_entries"] == sf["list_entries"]
    if thf is not None:
        np.testing.assert_allclose(thh, thf, rtol=1e-6, atol=1e-6 * n)


def test_half_langevin_and_replicas(md):
    """Three replicas of uneven size with their own eps, sigma and box, under
    the Langevin thermostat: 40 steps with the half list equal the full list's
    bit for bit."""
    sizes, boxes, eps, sig, xs, vs = [], [], [], [], [], []
    rng = np.random.default_rng(5)
    for r, nc in enumerate([5, 6, 5]):
        s = rng.uniform(0.95, 1.05)
        x, v, box = inputs.perturbed_lattice(nc, seed=60 + r, amp=0.1)
        cut = [500, 851, 433][r]
        xs.append(x[:cut] * s); vs.append(v[:cut])
        sizes.append(cut); boxes.append(box * s); eps.append(rng.uniform(0.9, 1.1)); sig.append(s)
    X, V = np.concatenate(xs), np.concatenate(vs)
    N = len(X)
    res = []
    for half in (False, True):
        h = md.md_create(sizes, np.array(boxes), eps=np.array(eps), sigma=np.array(sig),
                         langevin_gamma=0.5, kT=1.0, seed=99)
        if half:
            md.md_set_half_list(h, True)
        md.md_set_state(h, dev(X), dev(V))
        md.md_step(h, 40)
        res.append(state(md, h, N))
    np.testing.assert_array_equal(res[1][0], res[0][0])
    np.testing.assert_array_equal(res[1][1], res[0][1])


def test_half_switching_and_arguments(md):
    """Switching the list form between md_step calls keeps the trajectory of
    a full-list run bit for bit; the half list is refused for FP64, for
    bonded systems and by the adjoint."""
    x, v, box = inputs.perturbed_lattice(6, seed=13, amp=0.1)
    n = len(x)
    h1 = make(md, x, v, box, False)
    md.md_step(h1, 30)
    a = state(md, h1, n)
    h2 = make(md, x, v, box, False)
    md.md_step(h2, 10)
    md.md_set_half_list(h2, True)
    md.md_step(h2, 10)
    md.md_set_half_list(h2, False)
    md.md_step(h2, 10)
    b = state(md, h2, n)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])

    h64 = md.md_create(n, box, precision=md.MD_FP64)
    with pytest.raises(md.MDError) as e:
        md.md_set_half_list(h64, True)
    assert e.value.status == md.MD_ERR_ARG
    hb = md.md_create(4, np.array([8.0, 8.0, 8.0]), bonds=np.array([[0, 1], [2, 3]], dtype=np.int32))
    with pytest.raises(md.MDError) as e:
        md.md_set_half_list(hb, True)
    assert e.value.status == md.MD_ERR_ARG
    md.md_set_half_list(h2, True)
    with pytest.raises(md.MDError) as e:
        md.md_forward(h2, 5, 5)
    assert e.value.status == md.MD_ERR_ARG
