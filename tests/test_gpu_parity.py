"""CUDA path vs the FP64 CPU oracle, through the C ABI, on seeded inputs.

Tolerances: pair sets bit-exact; forces max relative error (per particle,
normalised by max(|F_i|, F_rms)) <= 1e-12 in FP64 and <= 1e-5 in FP32 with
fixed-point accumulation; energies and virial to the same relative bounds.
"""
import numpy as np
import pytest

import oracle
from paper_2109_10876_gb300 import inputs
from tests.helpers import force_rel_err, min_image_diff

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RC, SKIN = 2.5, 0.3
TOL = {0: 1e-12, 1: 1e-5}     # MD_FP64, MD_FP32_FIXED


@pytest.fixture(scope="module")
def md():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_10876_gb300 import md as m
    return m


def dev(a):
    return torch.tensor(np.ascontiguousarray(np.asarray(a).T), dtype=torch.float64, device="cuda")


def make(md, x, v, box, precision, **kw):
    n = len(x)
    h = md.md_create(n, box, precision=precision, skin=kw.pop("skin", SKIN), **kw)
    md.md_set_state(h, dev(x), dev(v))
    md.md_build_neighbors(h)
    return h


def gpu_forces(md, h, n, nrep=1):
    f = torch.zeros(3, n, dtype=torch.float64, device="cuda")
    euw = torch.zeros(nrep, 3, dtype=torch.float64, device="cuda")
    md.md_compute_forces(h, f, euw)
    md.md_sync(h)
    return f.cpu().numpy().T.copy(), euw.cpu().numpy().copy()


# ----------------------------------------------------------------- pair sets
@pytest.mark.parametrize("precision", [0, 1])
def test_pair_set_fcc_4000(md, precision):
    """N = 4000 fcc (the N = 4000 LJ-fluid start): every particle has 78
    neighbours within r_cut + r_skin; 156000 pairs, equal to brute force."""
    x, v, box = inputs.lj_fluid(10, seed=1)
    h = make(md, x, v, box, precision)
    got = md.export_pairs_sorted(h)
    want, _ = oracle.pairs(oracle.System(len(x), box, rc=RC), x, RC + SKIN)
    assert len(got) == 156000
    np.testing.assert_array_equal(got, want)
    st = md.md_get_stats(h)
    assert st["list_entries"] == 312000 and st["max_list_len"] == 78
    assert st["ncell"] == [5, 5, 5]


@pytest.mark.parametrize("n,boxl,seed", [(4000, 16.796, 2), (777, 9.1, 3), (60, 5.7, 4), (1, 6.0, 5)])
def test_pair_set_random(md, n, boxl, seed):
    """Uniform random points (ragged N, boxes with 1-3 cells per axis, pairs
    across the periodic boundary): the list equals the brute-force pair set."""
    box = np.array([boxl, boxl * 1.03, boxl * 0.98]) if boxl > 5.7 else np.array([boxl] * 3)
    x = inputs.random_gas(n, box, seed=seed)
    v = np.zeros_like(x)
    h = make(md, x, v, box, 1)
    got = md.export_pairs_sorted(h)
    want, _ = oracle.pairs(oracle.System(n, box, rc=RC), x, RC + SKIN)
    np.testing.assert_array_equal(got.reshape(-1, 2), want.reshape(-1, 2))


@pytest.mark.parametrize("half", [False, True])
def test_pair_set_short_lists(md, half):
    """A melt of free random-walk chains (2000 beads at density 0.85, overlaps
    left in) with the WCA list radius 2^(1/6) + 0.4: short lists (about 12
    entries) from cells of three particles; the list (full or half) equals the
    brute-force pair set."""
    x, v, box, bonds = inputs.melt(40, 50, rho=0.85, T=1.0, seed=19)
    n = len(x)
    rl = 2 ** (1 / 6) + 0.4
    h = md.md_create(n, box, potential=md.MD_WCA, skin=0.4, precision=md.MD_FP32_FIXED)
    if half:
        md.md_set_half_list(h, True)
    md.md_set_state(h, dev(x), dev(v))
    md.md_build_neighbors(h)
    got = md.export_pairs_sorted(h)
    want, _ = oracle.pairs(oracle.System(n, box, rc=2 ** (1 / 6)), x, rl)
    np.testing.assert_array_equal(got, want)


# ----------------------------------------------------------------- forces
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("case", ["liquid", "fcc", "gas_small_box"])
def test_forces_and_energies(md, precision, case):
    if case == "liquid":
        x, v, box = inputs.perturbed_lattice(10, seed=7, amp=0.2)      # N = 4000
        x, v = x[:3999], v[:3999]                                    # ragged tail
    elif case == "fcc":
        x, v, box = inputs.lj_fluid(10, seed=8)
    else:
        box = np.array([6.1, 6.1, 6.1])
        x = inputs.random_gas(90, box, seed=9, rmin=0.85)
        v = inputs.maxwell_velocities(90, 1.0, 10)
    n = len(x)
    h = make(md, x, v, box, precision)
    F, euw = gpu_forces(md, h, n)
    F_ref, e_ref = oracle.forces(oracle.System(n, box, rc=RC), x, v)
    tol = TOL[precision]
    if case == "fcc":
        assert np.max(np.abs(F)) < (1e-11 if precision == 0 else 1e-5)
    else:
        assert force_rel_err(F, F_ref) <= tol
    for k in range(3):
        assert euw[0, k] == pytest.approx(e_ref[k], rel=tol, abs=tol * n)
    if precision == 1:
        # fixed-point accumulation: f_ij = -f_ji bit for bit, so the total is exactly zero
        assert np.all(F.sum(axis=0) == 0.0)


@pytest.mark.parametrize("precision", [0, 1])
def test_wca_forces(md, precision):
    box = np.array([9.0, 9.0, 9.0])
    x = inputs.random_gas(600, box, seed=12, rmin=0.8)
    v = np.zeros_like(x)
    h = make(md, x, v, box, precision, potential=md.MD_WCA, skin=0.4)
    F, euw = gpu_forces(md, h, len(x))
    F_ref, e_ref = oracle.forces(oracle.System(len(x), box, rc=2 ** (1 / 6)), x, v)
    assert force_rel_err(F, F_ref) <= TOL[precision]
    assert euw[0, 0] == pytest.approx(e_ref[0], rel=TOL[precision])


# ----------------------------------------------------------------- trajectories
def run_gpu(md, h, n, nsteps, thermo_every=0):
    th = None
    if thermo_every:
        th = torch.zeros(nsteps // thermo_every, 1, 3, dtype=torch.float64, device="cuda")
    md.md_step(h, nsteps, thermo_every, th)
    xo = torch.zeros(3, n, dtype=torch.float64, device="cuda")
    vo = torch.zeros(3, n, dtype=torch.float64, device="cuda")
    md.md_get_state(h, xo, vo)
    out = (xo.cpu().numpy().T.copy(), vo.cpu().numpy().T.copy())
    if thermo_every:
        out += (th.cpu().numpy()[:, 0, :],)
    return out


def test_trajectory_fp64_100_steps(md):
    """N = 4000 LJ fluid from fcc at T = 0.72, 100 steps of dt = 0.005: FP64
    path follows the oracle to 1e-10 in positions; thermo (U, K, W) agrees."""
    x, v, box = inputs.lj_fluid(10, T=0.72, seed=1)
    n = len(x)
    h = make(md, x, v, box, 0, dt=0.005)
    xg, vg, th = run_gpu(md, h, n, 100, thermo_every=10)
    xo, vo, Fo, tho = oracle.vv_run(oracle.System(n, box, rc=RC, dt=0.005), x, v, 100, thermo=True)
    assert np.max(np.abs(min_image_diff(xg, xo, box))) < 1e-10
    assert np.max(np.abs(vg - vo)) < 1e-9
    np.testing.assert_allclose(th, tho[9::10], rtol=1e-10, atol=1e-9)
    st = md.md_get_stats(h)
    assert st["steps"] == 100 and st["rebuilds"] >= 1


def test_trajectory_fp32_fixed(md):
    """Same run in FP32 / fixed point.  Per-step force errors of ~1e-6
    relative grow along the chaotic trajectory: after 10 steps the positions
    agree to 1e-6, after 100 steps (t = 0.5) to 1e-4; total momentum stays
    zero and the energy agrees to 1e-5."""
    x, v, box = inputs.lj_fluid(10, T=0.72, seed=1)
    n = len(x)
    h = make(md, x, v, box, 1, dt=0.005)
    x10, _ = run_gpu(md, h, n, 10)
    xo10, _, _ = oracle.vv_run(oracle.System(n, box, rc=RC, dt=0.005), x, v, 10)
    assert np.max(np.abs(min_image_diff(x10, xo10, box))) < 1e-6
    h = make(md, x, v, box, 1, dt=0.005)
    xg, vg, th = run_gpu(md, h, n, 100, thermo_every=100)
    xo, vo, Fo, tho = oracle.vv_run(oracle.System(n, box, rc=RC, dt=0.005), x, v, 100, thermo=True)
    assert np.max(np.abs(min_image_diff(xg, xo, box))) < 1e-4
    assert np.max(np.abs(vg.sum(axis=0))) < 1e-9
    assert th[-1, 0] == pytest.approx(tho[-1, 0], rel=1e-5)


def test_step_splitting_is_seamless(md):
    """md_step(h, 30) equals md_step(h, 10) three times (FP64)."""
    x, v, box = inputs.perturbed_lattice(6, seed=13, amp=0.1)
    n = len(x)
    h1 = make(md, x, v, box, 0)
    a = run_gpu(md, h1, n, 30)
    h2 = make(md, x, v, box, 0)
    md.md_step(h2, 10)
    md.md_step(h2, 10)
    b = run_gpu(md, h2, n, 10)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


# ----------------------------------------------------------------- errors
def test_list_overflow_is_reported(md):
    x, v, box = inputs.lj_fluid(6, seed=14)
    h = md.md_create(len(x), box, list_capacity=32)
    md.md_set_state(h, dev(x), dev(v))
    md.md_build_neighbors(h)
    with pytest.raises(md.MDError) as e:
        md.md_sync(h)
    assert e.value.status == md.MD_ERR_LIST_OVERFLOW


def test_given_capacity_is_rounded_up(md):
    """A list capacity that is not a multiple of 32 (here 90) is rounded up
    to one (96), so every tile's list block stays aligned for the 16-byte
    copies; the pair set is exact."""
    x, v, box = inputs.lj_fluid(10, seed=1)
    h = md.md_create(len(x), box, list_capacity=90)
    md.md_set_state(h, dev(x), dev(v))
    md.md_build_neighbors(h)
    assert md.md_get_stats(h)["list_capacity"] == 96
    want, _ = oracle.pairs(oracle.System(len(x), box, rc=RC), x, RC + SKIN)
    np.testing.assert_array_equal(md.export_pairs_sorted(h), want)
    f = torch.zeros(3, len(x), dtype=torch.float64, device="cuda")
    md.md_compute_forces(h, f, None)
    md.md_step(h, 20)
    md.md_sync(h)


def test_automatic_capacity_grows(md):
    """A dense clump in a dilute box overflows the density-based capacity
    estimate; md_build_neighbors grows the list and the pair set is exact."""
    box = np.array([30.0, 30.0, 30.0])
    x = np.concatenate([inputs.random_gas(400, box, seed=15),
                        5.0 + inputs.random_gas(700, np.array([9.5, 9.5, 9.5]), seed=16, rmin=0.8)])
    v = np.zeros_like(x)
    h = make(md, x, v, box, 1)
    got = md.export_pairs_sorted(h)
    want, _ = oracle.pairs(oracle.System(len(x), box, rc=RC), x, RC + SKIN)
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("precision", [0, 1])
def test_lists_longer_than_the_shared_stage(md, precision):
    """A compressed fcc crystal (rho = 1.2, N = 4000) with a skin of 0.8: about
    180 neighbours within r_cut + r_skin, more rows than the list build stages
    in shared memory for a tile of about 125 particles (12288 entries), so the
    rows beyond the stage are written straight to global memory, and the force
    kernel reads those tiles' lists from global memory instead of staging
    them.  The pair set equals brute force, forces and energies follow the
    oracle, and 10 steps split 4 + 6 equal 10 in one call bit for bit."""
    skin = 0.8
    x, v, box = inputs.perturbed_lattice(10, rho=1.2, seed=21, amp=0.05)
    n = len(x)
    h = make(md, x, v, box, precision, skin=skin)
    assert md.md_get_stats(h)["max_list_len"] > 128
    got = md.export_pairs_sorted(h)
    want, _ = oracle.pairs(oracle.System(n, box, rc=RC), x, RC + skin)
    np.testing.assert_array_equal(got, want)
    F, euw = gpu_forces(md, h, n)
    F_ref, e_ref = oracle.forces(oracle.System(n, box, rc=RC), x, v)
    tol = TOL[precision]
    assert force_rel_err(F, F_ref) <= tol
    for k in range(3):
        assert euw[0, k] == pytest.approx(e_ref[k], rel=tol, abs=tol * n)
    states = []
    for parts in ((10,), (4, 6)):
        hs = make(md, x, v, box, precision, skin=skin)
        for k in parts:
            md.md_step(hs, k)
        xo = torch.zeros(3, n, dtype=torch.float64, device="cuda")
        vo = torch.zeros_like(xo)
        md.md_get_state(hs, xo, vo)
        states.append((xo.cpu().numpy(), vo.cpu().numpy()))
    np.testing.assert_array_equal(states[0][0], states[1][0])
    np.testing.assert_array_equal(states[0][1], states[1][1])


def test_thermo_every_step_graph_equals_stream_launches(md):
    """md_step with (U, K, W) every step runs as one graph launch; with the
    section timers on the same kernels are launched one by one.  Both give
    the same records and the same state, bit for bit, and the records follow
    the oracle's energies."""
    x, v, box = inputs.perturbed_lattice(6, seed=17, amp=0.1)
    n = len(x)
    out = []
    for timing in (False, True):
        h = make(md, x, v, box, 1)
        md.md_set_timing(h, timing)
        th = np.zeros((30, 3))
        md.md_step(h, 30, 1, th)
        xo = torch.zeros(3, n, dtype=torch.float64, device="cuda")
        vo = torch.zeros_like(xo)
        md.md_get_state(h, xo, vo)
        out.append((th.copy(), xo.cpu().numpy(), vo.cpu().numpy()))
    for a, b in zip(out[0], out[1]):
        np.testing.assert_array_equal(a, b)
    xo, vo, Fo, tho = oracle.vv_run(oracle.System(n, box, rc=RC, dt=0.005), x, v, 30, thermo=True)
    np.testing.assert_allclose(out[0][0], tho, rtol=1e-5, atol=1e-5 * n)
