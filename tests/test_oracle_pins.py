"""Pins for the FP64 CPU oracle, against facts that do not come from the oracle.

Each test checks the oracle against a closed form, a symbolic derivative, a
lattice sum by integer enumeration, a conservation law, an ODE solution from
an independent integrator, or a published known-answer vector, chosen so that
a dropped term, a wrong sign or factor, or a swapped operand fails one of them.
"""
import itertools
import math
import os

import numpy as np
import pytest
import sympy as sp

import oracle
from paper_2109_10876_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RC = 2.5
SKIN = 0.3


# ---------------------------------------------------------------- Eq. 2 pins
def test_lj_closed_forms():
    """V(sigma)=0, F(sigma)=24 eps/sigma, minimum V=-eps with F=0 at 2^(1/6) sigma."""
    for eps, sig in [(1.0, 1.0), (0.9, 1.05), (1.1, 0.95)]:
        assert abs(oracle.lj_energy(sig, eps, sig)) < 1e-14
        assert oracle.lj_force(sig, eps, sig) == pytest.approx(24.0 * eps / sig, rel=1e-14)
        rm = 2 ** (1 / 6) * sig
        assert oracle.lj_energy(rm, eps, sig) == pytest.approx(-eps, rel=1e-14)
        assert abs(oracle.lj_force(rm, eps, sig)) < 1e-12


def test_lj_force_is_symbolic_derivative():
    """Force magnitude equals -dV/dr of Eq. 2 from sympy at many r, eps, sigma."""
    r, e, s = sp.symbols("r e s", positive=True)
    V = 4 * e * ((s / r) ** 12 - (s / r) ** 6)
    dV = sp.lambdify((r, e, s), -sp.diff(V, r), "mpmath")
    Vl = sp.lambdify((r, e, s), V, "mpmath")
    rng = np.random.default_rng(0)
    for _ in range(200):
        rr, ee, ss = rng.uniform(0.8, 3.0), rng.uniform(0.5, 2.0), rng.uniform(0.8, 1.2)
        assert oracle.lj_force(rr, ee, ss) == pytest.approx(float(dV(rr, ee, ss)), rel=1e-12, abs=1e-14)
        assert oracle.lj_energy(rr, ee, ss) == pytest.approx(float(Vl(rr, ee, ss)), rel=1e-12, abs=1e-14)
    # value at the LJ-fluid cutoff used by every LJ workload
    assert oracle.lj_force(2.5) == pytest.approx(-0.0389995, abs=5e-8)
    assert oracle.lj_energy(2.5) == pytest.approx(-0.0163169, abs=5e-8)


def test_min_image_matches_image_enumeration():
    """Minimum-image r^2 equals the smallest r^2 over the 27 periodic images."""
    rng = np.random.default_rng(1)
    for _ in range(500):
        box = rng.uniform(5.0, 12.0, size=3)
        xi, xj = rng.uniform(0, 1, 3) * box, rng.uniform(0, 1, 3) * box
        best = min(float(np.sum((xi - xj - np.array(s) * box) ** 2))
                   for s in itertools.product((-1, 0, 1), repeat=3))
        assert oracle.min_image_r2(xi, xj, box) == pytest.approx(best, rel=1e-13)


# ------------------------------------------------- tiny boxes by brute force
def test_two_particles_across_boundary():
    """Two particles separated across the periodic boundary: force along d,
    magnitude -dV/dr, equal and opposite; energy shifted to 0 at the cutoff."""
    box = np.array([10.0, 9.0, 8.0])
    x = np.array([[0.2, 4.0, 7.9], [9.4, 4.3, 0.1]])
    s = oracle.System(2, box, rc=RC)
    F, euw = oracle.forces(s, x)
    d = np.array([0.2 - 9.4 + 10.0, 4.0 - 4.3, 7.9 - 0.1 - 8.0])
    r = np.linalg.norm(d)
    fm = 24 * (2 * r ** -13 - r ** -7)
    np.testing.assert_allclose(F[0], fm * d / r, rtol=1e-13)
    np.testing.assert_allclose(F[1], -F[0], rtol=0, atol=0)
    V = 4 * (r ** -12 - r ** -6) - 4 * (RC ** -12 - RC ** -6)
    assert euw[0] == pytest.approx(V, rel=1e-13)
    assert euw[2] == pytest.approx(fm * r, rel=1e-13)   # virial d . f = r * f(r)


def test_cutoff_is_strict_and_particle_at_box_edge():
    box = np.array([8.0, 8.0, 8.0])
    L = 8.0
    # at exactly r = rc: no interaction (strict r < r_cut); just inside: interaction
    x = np.array([[1.0, 1.0, 1.0], [1.0 + RC, 1.0, 1.0]])
    F, _ = oracle.forces(oracle.System(2, box, rc=RC), x)
    assert np.all(F == 0.0)
    x[1, 0] = 1.0 + RC - 1e-9
    F, _ = oracle.forces(oracle.System(2, box, rc=RC), x)
    # attractive at r ~ 2.5: particle 0 is pulled towards particle 1 (+x)
    assert F[0, 0] == pytest.approx(-oracle.lj_force(RC - 1e-9), rel=1e-9) and F[1, 0] == -F[0, 0]
    # a particle at the largest double below L interacts with one at 0.5
    x = np.array([[np.nextafter(L, 0), 2.0, 2.0], [0.5, 2.0, 2.0]])
    F, _ = oracle.forces(oracle.System(2, box, rc=RC), x)
    r = 0.5 + (L - np.nextafter(L, 0))
    assert F[1, 0] == pytest.approx(24 * (2 * r ** -13 - r ** -7), rel=1e-12)


def test_pair_set_matches_image_enumeration():
    """Pair set within r_cut + r_skin equals an enumeration over images."""
    rng = np.random.default_rng(2)
    for n in (3, 8, 40):
        box = np.array([6.0, 6.5, 7.0])
        x = rng.uniform(0, 1, (n, 3)) * box
        s = oracle.System(n, box, rc=RC)
        got, counts = oracle.pairs(s, x, RC + SKIN)
        want = []
        for i in range(n):
            for j in range(i + 1, n):
                m = min(float(np.sum((x[i] - x[j] - np.array(t) * box) ** 2))
                        for t in itertools.product((-1, 0, 1), repeat=3))
                if m < (RC + SKIN) ** 2:
                    want.append((i, j))
        assert [tuple(p) for p in got] == want
        assert counts.sum() == 2 * len(want)


# ------------------------------------------------------------- fcc lattice pins
def _fcc_golden():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "fcc_shells.txt")) if l[0] != "#"]
    return [(int(m), float(d), int(c)) for m, d, c in rows]


def test_fcc_shells_golden_is_lattice_fact():
    a = (4 / 0.8442) ** (1 / 3)
    for m, d, c in _fcc_golden():
        assert a * math.sqrt(m / 2) == pytest.approx(d, abs=5e-7)
    B = inputs.FCC_BASIS
    dist = {}
    for n in itertools.product(range(-2, 3), repeat=3):
        for b in B:
            v = (np.array(n) + b)
            m = int(round(2 * v @ v))
            if m:
                dist[m] = dist.get(m, 0) + 1
    assert [dist[m] for m in range(1, 7)] == [c for _, _, c in _fcc_golden()]


def test_fcc_4000_pins():
    """N = 4000 fcc at rho = 0.8442: 54 / 78 neighbours, 108000 / 156000 pairs,
    zero net force per site, U/N = -6.3328120 with the shifted potential."""
    x, box = inputs.fcc_lattice(10, 0.8442)
    assert len(x) == 4000
    s = oracle.System(4000, box, rc=RC)
    pr, counts = oracle.pairs(s, x, RC)
    assert len(pr) == 108000 and np.all(counts == 54)
    pl, countsl = oracle.pairs(s, x, RC + SKIN)
    assert len(pl) == 156000 and np.all(countsl == 78)
    F, euw = oracle.forces(s, x)
    assert np.max(np.abs(F)) < 1e-11
    assert euw[0] / 4000 == pytest.approx(-6.3328120, abs=5e-8)
    # the same number from the shell table: 1/2 sum_shells count (V(r) - V(rc))
    Vs = lambda r: 4 * (r ** -12 - r ** -6) - 4 * (RC ** -12 - RC ** -6)
    shell = 0.5 * sum(c * Vs((4 / 0.8442) ** (1 / 3) * math.sqrt(m / 2))
                      for m, _, c in _fcc_golden() if m <= 4)
    assert euw[0] / 4000 == pytest.approx(shell, rel=1e-12)


def test_neighbours_sample_pins():
    """Sampled neighbour rows: on the fcc lattice every site has the 78
    neighbours of the first five shells, at the shell distances a sqrt(m/2);
    on a random gas in a small box (pairs across the boundary) the rows are
    exactly those of the brute-force pair set."""
    x, box = inputs.fcc_lattice(10, 0.8442)
    s = oracle.System(len(x), box, rc=RC)
    a = (4 / 0.8442) ** (1 / 3)
    for j, r2 in oracle.neighbours_sample(s, x, [0, 1, 1234, 3999], RC + SKIN):
        assert len(j) == 78 and np.all(np.diff(j) > 0)
        m = np.round(2 * r2 / a ** 2).astype(int)
        np.testing.assert_allclose(r2, a ** 2 * m / 2, rtol=1e-12)
        assert [int(np.sum(m == k)) for k in range(1, 6)] == [c for k, _, c in _fcc_golden() if k <= 5]
    box = np.array([6.3, 6.6, 6.1])
    x = inputs.random_gas(300, box, seed=77)
    s = oracle.System(300, box, rc=RC)
    pr, _ = oracle.pairs(s, x, RC + SKIN)
    rows = oracle.neighbours_sample(s, x, np.arange(300), RC + SKIN)
    for i in range(300):
        want = np.sort(np.concatenate([pr[pr[:, 0] == i, 1], pr[pr[:, 1] == i, 0]]))
        np.testing.assert_array_equal(rows[i][0], want)
        for j, r2 in zip(*rows[i]):
            assert r2 == oracle.min_image_r2(x[i], x[j], box)


def test_bonded_sample_pins():
    """Bonded forces of chosen particles: one FENE bond along x gives
    F = -K r / (1 - r^2/R0^2) on its first particle and the opposite on the
    second; on chains with angle triples, the sampled non-bonded plus bonded
    forces equal the whole-system oracle forces."""
    box = np.array([8.0, 8.0, 8.0])
    r = 1.1
    x = np.array([[1.0, 2.0, 3.0], [1.0 + r, 2.0, 3.0]])
    s = oracle.System(2, box, rc=2 ** (1 / 6), bonds=np.array([[0, 1]]), fene_K=30.0, fene_R0=1.5)
    Fb = oracle.bonded_sample(s, x, [0, 1])
    f = 30.0 * r / (1 - r * r / 2.25)
    np.testing.assert_allclose(Fb, [[f, 0, 0], [-f, 0, 0]], rtol=1e-14)
    box = np.array([9.0, 9.0, 9.0])
    x, bonds = inputs.chains(6, 20, box, seed=5)
    ang = np.array([[c * 20 + k - 1, c * 20 + k, c * 20 + k + 1] for c in range(6) for k in range(1, 19)])
    s = oracle.System(len(x), box, rc=2 ** (1 / 6), bonds=bonds, angles=ang, angle_K=1.5)
    F, _ = oracle.forces(s, x)
    idx = np.arange(len(x))
    Fn, _, _ = oracle.forces_sample(s, x, idx)
    np.testing.assert_allclose(Fn + oracle.bonded_sample(s, x, idx), F, rtol=0, atol=1e-12 * np.max(np.abs(F)))


def test_langevin_sample_fluctuation_dissipation():
    """The sampled Langevin force has mean -gamma m v (the friction) and
    variance 2 gamma kT m / dt per component (the fluctuation-dissipation
    relation of the force-form thermostat), over 200000 particle draws."""
    n = 200_000
    s = oracle.System(n, [50.0, 50.0, 50.0], gamma=0.5, kT=1.3, mass=1.0, dt=0.01, seed=11)
    v = np.random.default_rng(3).normal(size=(n, 3))
    F = oracle.langevin_sample(s, np.arange(n), v, 17)
    noise = F + 0.5 * 1.0 * v
    assert abs(noise.mean()) < 5 * math.sqrt(2 * 0.5 * 1.3 / 0.01 / (3 * n))
    assert noise.var() == pytest.approx(2 * 0.5 * 1.3 / 0.01, rel=0.01)


def test_cell_rule_from_paper():
    """N = 262144 at rho = 0.8442 gives a 24^3 cell grid with cell edge >= r_cut + r_skin
    (Sec. 5 quotes the (24, 24, 24) grid)."""
    L = (262144 / 0.8442) ** (1 / 3)
    assert math.floor(L / (RC + SKIN)) == 24


# ------------------------------------------------------------------ invariants
def _liquid(ncell=5, seed=3, amp=0.15):
    x, v, box = inputs.perturbed_lattice(ncell, seed=seed, amp=amp)
    return x, v, box


def test_newton_third_law_and_force_is_minus_grad_U():
    x, v, box = _liquid()
    n = len(x)
    s = oracle.System(n, box, rc=RC)
    F, euw = oracle.forces(s, x)
    assert np.max(np.abs(F.sum(axis=0))) < 1e-12 * np.max(np.abs(F)) * n
    # F = -grad U (Eq. 1) by central differences of the shifted energy
    rng = np.random.default_rng(4)
    h = 1e-6
    for i in rng.choice(n, 6, replace=False):
        for k in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, k] += h
            xm[i, k] -= h
            up = oracle.forces(s, xp)[1][0]
            um = oracle.forces(s, xm)[1][0]
            assert F[i, k] == pytest.approx(-(up - um) / (2 * h), abs=2e-5 * max(1, abs(F[i, k])))


def test_virial_scaling_identity():
    """With r_cut = 2.5 sigma scaling with sigma and V shifted to zero at r_cut,
    U depends on sigma only through r / sigma, so sigma dU/dsigma = W (the
    virial sum of d . f), and eps dU/deps = U."""
    x, v, box = _liquid(seed=5)
    n = len(x)
    sig, h = 1.0, 1e-6
    U0, W0 = oracle.forces(oracle.System(n, box, sigma=sig, rc=RC * sig), x)[1][[0, 2]]
    Up = oracle.forces(oracle.System(n, box, sigma=sig + h, rc=RC * (sig + h)), x)[1][0]
    Um = oracle.forces(oracle.System(n, box, sigma=sig - h, rc=RC * (sig - h)), x)[1][0]
    assert sig * (Up - Um) / (2 * h) == pytest.approx(W0, rel=1e-6)
    Ue = oracle.forces(oracle.System(n, box, eps=1.3, rc=RC), x)[1][0]
    assert Ue == pytest.approx(1.3 * U0, rel=1e-13)


def test_nve_conservation_and_reversibility():
    """Velocity Verlet (Fig. 1): momentum conserved, the energy error is
    second order in dt (ratio ~4 when dt halves) and small, and the map is
    time-reversible."""
    x, v, box = inputs.lj_fluid(5, T=0.72, seed=6)
    n = len(x)
    dE = []
    for dt in (0.005, 0.0025):
        s = oracle.System(n, box, rc=RC, dt=dt)
        F0, e0 = oracle.forces(s, x, v)
        E0 = e0[0] + e0[1]
        x1, v1, F1, th = oracle.vv_run(s, x, v, int(round(0.5 / dt)), thermo=True)
        E = th[:, 0] + th[:, 1]
        dE.append(np.max(np.abs(E - E0)) / n)
        assert np.max(np.abs(v1.sum(axis=0))) < 1e-10
    assert dE[0] < 1e-3
    assert 3.0 < dE[0] / dE[1] < 5.0
    # reverse: negate v, run the same steps back, negate again -> initial state
    s = oracle.System(n, box, rc=RC, dt=0.005)
    x1, v1, _ = oracle.vv_run(s, x, v, 100)
    x2, v2, _ = oracle.vv_run(s, x1, -v1, 100)
    d = x2 - x
    d -= box * np.round(d / box)
    assert np.max(np.abs(d)) < 1e-9
    assert np.max(np.abs(-v2 - v)) < 1e-9


def test_velocity_verlet_is_second_order_against_ode_solver():
    """Two LJ particles: the oracle's trajectory converges to scipy's DOP853
    solution of m x'' = F with error ratio ~4 when dt halves."""
    from scipy.integrate import solve_ivp
    box = np.array([20.0, 20.0, 20.0])
    x0 = np.array([[5.0, 5.0, 5.0], [6.15, 5.3, 5.1]])
    v0 = np.array([[0.3, -0.2, 0.1], [-0.3, 0.2, -0.1]])
    T = 0.64

    def rhs(t, y):
        p = y[:6].reshape(2, 3)
        d = p[0] - p[1]
        r = np.linalg.norm(d)
        f = 24 * (2 * r ** -13 - r ** -7) * d / r if r < RC else 0 * d
        return np.concatenate([y[6:], f, -f])

    sol = solve_ivp(rhs, (0, T), np.concatenate([x0.ravel(), v0.ravel()]), method="DOP853",
                    rtol=1e-12, atol=1e-12)
    xe = sol.y[:6, -1].reshape(2, 3)
    errs = []
    for dt in (0.004, 0.002, 0.001):
        s = oracle.System(2, box, rc=RC, dt=dt)
        x1, v1, _ = oracle.vv_run(s, x0, v0, int(round(T / dt)))
        errs.append(np.max(np.abs(x1 - xe)))
    assert errs[2] < 1e-4
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


# ------------------------------------------------------------------ FENE, Langevin
def test_fene_matches_symbolic_derivative_and_breaks():
    r, K, R0 = sp.symbols("r K R0", positive=True)
    U = -sp.Rational(1, 2) * K * R0 ** 2 * sp.log(1 - r ** 2 / R0 ** 2)
    f = sp.lambdify((r, K, R0), -sp.diff(U, r), "mpmath")
    Ul = sp.lambdify((r, K, R0), U, "mpmath")
    box = np.array([10.0, 10.0, 10.0])
    for rr in (0.5, 0.97, 1.2, 1.45):
        x = np.array([[1.0, 2.0, 3.0], [1.0 + rr * 0.6, 2.0 + rr * 0.8, 3.0]])
        s = oracle.System(2, box, rc=1e-3, shift=False, bonds=[[0, 1]], fene_K=30, fene_R0=1.5)
        F, euw = oracle.forces(s, x)
        d = x[0] - x[1]
        np.testing.assert_allclose(F[0], float(f(rr, 30, 1.5)) * d / rr, rtol=1e-12)
        np.testing.assert_allclose(F[1], -F[0], rtol=1e-15)
        assert euw[0] == pytest.approx(float(Ul(rr, 30, 1.5)), rel=1e-12)
    x = np.array([[1.0, 2.0, 3.0], [2.6, 2.0, 3.0]])
    with pytest.raises(RuntimeError):
        oracle.forces(oracle.System(2, box, rc=1e-3, bonds=[[0, 1]], fene_R0=1.5), x)


def test_philox_known_answers():
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(t, 16) for t in line.split()]
        assert oracle.philox4x32_10(w[0:4], w[4:6]) == w[6:10]


def test_langevin_uniforms_moments_and_thermostat_temperature():
    u = np.array([oracle.langevin_uniforms(7, i, s) for i in range(200) for s in range(50)])
    assert np.all(np.abs(u) < 0.5)
    assert abs(u.mean()) < 0.01 and u.var() == pytest.approx(1 / 12, rel=0.03)
    # ideal gas (no pair forces within a tiny cutoff) under the thermostat: <T> -> kT
    n = 64
    box = np.array([20.0, 20.0, 20.0])
    x = inputs.random_gas(n, box, seed=8)
    v = np.zeros((n, 3))
    s = oracle.System(n, box, rc=1e-3, dt=0.01, gamma=1.0, kT=1.3, seed=9)
    x, v, F, th = oracle.vv_run(s, x, v, 4000, thermo=True)
    T = 2 * th[1000:, 1] / (3 * n)
    assert T.mean() == pytest.approx(1.3, rel=0.06)


# ------------------------------------------------------------------ adjoint pins
def _loss(x, v, box, eps, sig, T, rc, cU, cK, cW):
    n = len(x)
    s = oracle.System(n, box, eps=eps, sigma=sig, rc=rc, dt=0.005)
    x1, v1, _ = oracle.vv_run(s, x, v, T)
    _, euw = oracle.forces(s, x1, v1)
    return cU * euw[0] + cK * euw[1] + cW * euw[2]


def test_hvp_is_derivative_of_forces():
    """(J w) from the oracle equals the directional derivative of the forces,
    F(x + h w) - F(x - h w) over 2h, and the parameter projections equal the
    derivatives of w . F in eps and sigma (r_cut held fixed)."""
    x, v, box = _liquid(ncell=3, seed=9, amp=0.1)
    n = len(x)
    rng = np.random.default_rng(10)
    w = rng.normal(size=(n, 3))
    s = oracle.System(n, box, rc=2.5)
    hv, pe, ps = oracle.hvp(s, x, w)
    h = 1e-6
    Fp, _ = oracle.forces(s, x + h * w)
    Fm, _ = oracle.forces(s, x - h * w)
    np.testing.assert_allclose(hv, (Fp - Fm) / (2 * h), rtol=1e-6, atol=1e-5)
    F0, _ = oracle.forces(s, x)
    Fe, _ = oracle.forces(oracle.System(n, box, eps=1 + h, rc=2.5), x)
    assert pe == pytest.approx(np.sum(w * (Fe - F0)) / h, rel=1e-6)
    Fsp, _ = oracle.forces(oracle.System(n, box, sigma=1 + h, rc=2.5), x)
    Fsm, _ = oracle.forces(oracle.System(n, box, sigma=1 - h, rc=2.5), x)
    assert ps == pytest.approx(np.sum(w * (Fsp - Fsm)) / (2 * h), rel=1e-6)


@pytest.mark.parametrize("T", [0, 1, 5])
def test_adjoint_matches_central_differences(T):
    """d L / d(eps, sigma) by the reverse pass equals central differences of
    the forward (h = 1e-4) for L = U/N + (2K + W)/(3V) after T steps.  For
    sigma the cutoff is held fixed: a cutoff that moves with sigma sweeps pairs
    across r_cut, where the virial jumps, which no pointwise derivative sees."""
    x, v, box = _liquid(ncell=3, seed=5, amp=0.1)
    n = len(x)
    V = float(np.prod(box))
    c = (1.0 / n, 2.0 / (3 * V), 1.0 / (3 * V))
    s = oracle.System(n, box, rc=2.5, dt=0.005)
    h = 1e-4
    _, ge, _, _, _ = oracle.vv_adjoint(s, x, v, T, *c)
    fe = (_loss(x, v, box, 1 + h, 1, T, 2.5 * (1 + 0), *c) - _loss(x, v, box, 1 - h, 1, T, 2.5, *c)) / (2 * h)
    assert ge == pytest.approx(fe, rel=1e-6)
    _, _, gs, _, _ = oracle.vv_adjoint(s, x, v, T, *c, rc_fixed=True)
    fs = (_loss(x, v, box, 1, 1 + h, T, 2.5, *c) - _loss(x, v, box, 1, 1 - h, T, 2.5, *c)) / (2 * h)
    assert gs == pytest.approx(fs, rel=1e-5)


def test_adjoint_initial_state_gradient():
    """The adjoint of the initial positions and velocities is the gradient of
    the loss after T steps (central differences along random directions)."""
    x, v, box = _liquid(ncell=3, seed=6, amp=0.1)
    n = len(x)
    V = float(np.prod(box))
    c = (1.0 / n, 2.0 / (3 * V), 1.0 / (3 * V))
    s = oracle.System(n, box, rc=2.5, dt=0.005)
    _, _, _, lx, lv = oracle.vv_adjoint(s, x, v, 4, *c)
    rng = np.random.default_rng(11)
    h = 1e-6
    for _ in range(2):
        dx, dv = rng.normal(size=(n, 3)), rng.normal(size=(n, 3))
        fx = (_loss(x + h * dx, v, box, 1, 1, 4, 2.5, *c) - _loss(x - h * dx, v, box, 1, 1, 4, 2.5, *c)) / (2 * h)
        fv = (_loss(x, v + h * dv, box, 1, 1, 4, 2.5, *c) - _loss(x, v - h * dv, box, 1, 1, 4, 2.5, *c)) / (2 * h)
        assert np.sum(lx * dx) == pytest.approx(fx, rel=1e-5)
        assert np.sum(lv * dv) == pytest.approx(fv, rel=1e-5)


def test_adjoint_of_a_loss_on_the_final_state():
    """A loss on the end point itself, L = gx . x_T + gv . v_T: with gx and gv
    as the terminal adjoints the reverse pass gives dL/deps, dL/dsigma and
    dL/d(x0, v0) equal to central differences of the forward (r_cut held
    fixed for sigma; x_T compared by minimum image, as positions wrap)."""
    x, v, box = _liquid(ncell=3, seed=7, amp=0.1)
    n = len(x)
    T = 4
    rng = np.random.default_rng(12)
    gx, gv = rng.normal(size=(n, 3)), rng.normal(size=(n, 3))

    def end(eps=1.0, sig=1.0, xx=x, vv=v):
        s = oracle.System(n, box, eps=eps, sigma=sig, rc=2.5, dt=0.005)
        x1, v1, _ = oracle.vv_run(s, xx, vv, T)
        return x1, v1

    def dL(a, b):
        d = a[0] - b[0]
        d -= box * np.round(d / box)
        return float(np.sum(gx * d) + np.sum(gv * (a[1] - b[1])))

    s = oracle.System(n, box, rc=2.5, dt=0.005)
    euw, ge, gs, lx, lv = oracle.vv_adjoint(s, x, v, T, 0.0, 0.0, 0.0, rc_fixed=True, gx=gx, gv=gv)
    h = 1e-6
    assert ge == pytest.approx(dL(end(eps=1 + h), end(eps=1 - h)) / (2 * h), rel=1e-6)
    assert gs == pytest.approx(dL(end(sig=1 + h), end(sig=1 - h)) / (2 * h), rel=1e-6)
    dx, dv = rng.normal(size=(n, 3)), rng.normal(size=(n, 3))
    assert np.sum(lx * dx) == pytest.approx(dL(end(xx=x + h * dx), end(xx=x - h * dx)) / (2 * h), rel=1e-6)
    assert np.sum(lv * dv) == pytest.approx(dL(end(vv=v + h * dv), end(vv=v - h * dv)) / (2 * h), rel=1e-6)
    # the terms add: the energy loss and the end-point loss together give the sum
    c = (1.0 / n, 0.3, 0.2)
    _, ge_c, gs_c, _, _ = oracle.vv_adjoint(s, x, v, T, *c, rc_fixed=True)
    _, ge_b, gs_b, _, _ = oracle.vv_adjoint(s, x, v, T, *c, rc_fixed=True, gx=gx, gv=gv)
    assert ge_b == pytest.approx(ge_c + ge, rel=1e-12)
    assert gs_b == pytest.approx(gs_c + gs, rel=1e-12)


# ---------------------------------------------------------------- soft push-off
def test_soft_pushoff_closed_forms_and_derivative():
    """Cosine push-off A (1 + cos(pi r / rc)): V(0) = 2A, V(rc/2) = A, V(rc) = 0;
    the force is the sympy derivative -dV/dr, pi A / rc at rc / 2 and zero at
    0 and rc (continuous at the cutoff); coincident beads feel no force."""
    rc = 2 ** (1 / 6)
    for A in (1.0, 7.5, 100.0):
        assert oracle.soft_energy(0.0, A, rc) == pytest.approx(2 * A, rel=1e-15)
        assert oracle.soft_energy(0.5 * rc, A, rc) == pytest.approx(A, rel=1e-14)
        assert abs(oracle.soft_energy(rc, A, rc)) < 1e-14 * A
        assert oracle.soft_force(0.5 * rc, A, rc) == pytest.approx(math.pi * A / rc, rel=1e-14)
        assert abs(oracle.soft_force(rc, A, rc)) < 1e-13 * A
        assert oracle.soft_force(0.0, A, rc) == 0.0
    r, a, c = sp.symbols("r a c", positive=True)
    V = a * (1 + sp.cos(sp.pi * r / c))
    dV = sp.lambdify((r, a, c), -sp.diff(V, r), "mpmath")
    for rr in np.linspace(0.05, 1.1, 23):
        assert oracle.soft_force(rr, 3.0, rc) == pytest.approx(float(dV(rr, 3.0, rc)), rel=1e-12, abs=1e-13)
    box = np.array([4.0, 4.0, 4.0])
    x = np.array([[1.0, 1.0, 1.0], [1.0, 1.0, 1.0], [1.3, 1.0, 1.0]])
    s = oracle.System(3, box, eps=2.0, rc=rc, soft=True)
    F, euw = oracle.forces(s, x)
    f01 = oracle.soft_force(0.3, 2.0, rc)          # j = 2 pushes 0 and 1 towards -x
    np.testing.assert_allclose(F[0], [-f01, 0, 0], rtol=1e-14)
    np.testing.assert_allclose(F[1], [-f01, 0, 0], rtol=1e-14)
    np.testing.assert_allclose(F[2], [2 * f01, 0, 0], rtol=1e-14)
    assert euw[0] == pytest.approx(2 * 2.0 + 2 * oracle.soft_energy(0.3, 2.0, rc), rel=1e-14)


def test_soft_pushoff_force_is_minus_grad_U_and_nve_second_order():
    """On a random gas: forces are -grad U by central differences, Newton's
    third law holds, and velocity Verlet conserves energy to second order."""
    box = np.array([6.0, 6.0, 6.0])
    x = inputs.random_gas(300, box, seed=21)
    n = len(x)
    s = oracle.System(n, box, eps=5.0, rc=2 ** (1 / 6), soft=True)
    F, euw = oracle.forces(s, x)
    assert np.max(np.abs(F.sum(axis=0))) < 1e-12 * np.max(np.abs(F)) * n
    h = 1e-6
    for i in np.random.default_rng(3).choice(n, 5, replace=False):
        for k in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, k] += h
            xm[i, k] -= h
            d = -(oracle.forces(s, xp)[1][0] - oracle.forces(s, xm)[1][0]) / (2 * h)
            assert F[i, k] == pytest.approx(d, abs=1e-6 * max(1.0, abs(F[i, k])))
    v = inputs.maxwell_velocities(n, 1.0, 22)
    dE = []
    for dt in (0.004, 0.002):
        s = oracle.System(n, box, eps=5.0, rc=2 ** (1 / 6), soft=True, dt=dt)
        e0 = oracle.forces(s, x, v)[1]
        th = oracle.vv_run(s, x, v, int(round(0.4 / dt)), thermo=True)[3]
        dE.append(np.max(np.abs(th[:, 0] + th[:, 1] - e0[0] - e0[1])))
    assert 3.0 < dE[0] / dE[1] < 5.0


# ---------------------------------------------------------------- angle term
def test_angle_term_closed_forms_and_sympy_gradient():
    """Cosine angle term K (1 - cos theta) between consecutive bond vectors:
    zero force on a straight triple; the right angle gives U = K and forces
    along the other bond; at random triples the forces are sympy's
    -grad U, sum to zero, exert no torque and have zero virial."""
    box = np.array([20.0, 20.0, 20.0])
    K = 1.5
    fa, fb, fc, u = oracle.angle_triple([1, 1, 1], [2, 1, 1], [3, 1, 1], box, K)
    assert u == 0.0 and np.all(np.abs(np.concatenate([fa, fb, fc])) < 1e-15)
    fa, fb, fc, u = oracle.angle_triple([1, 1, 1], [2, 1, 1], [2, 3, 1], box, K)
    assert u == pytest.approx(K, rel=1e-15)
    np.testing.assert_allclose(fa, [0, -K, 0], atol=1e-15)     # |b2| = 2 scales out of fa's direction only
    np.testing.assert_allclose(fc, [K / 2, 0, 0], atol=1e-15)
    for theta in (0.3, 1.0, 2.0, 3.0):
        xc = [2 + np.cos(theta), 1 + np.sin(theta), 1]
        assert oracle.angle_triple([1, 1, 1], [2, 1, 1], xc, box, K)[3] == pytest.approx(K * (1 - np.cos(theta)), rel=1e-13)
    X = sp.symbols("ax ay az bx by bz cx cy cz")
    a, b, c = sp.Matrix(X[0:3]), sp.Matrix(X[3:6]), sp.Matrix(X[6:9])
    b1, b2 = b - a, c - b
    U = K * (1 - b1.dot(b2) / (sp.sqrt(b1.dot(b1)) * sp.sqrt(b2.dot(b2))))
    grad = sp.lambdify(X, [-sp.diff(U, q) for q in X], "mpmath")
    rng = np.random.default_rng(8)
    for _ in range(10):
        pts = 5 + rng.uniform(-1, 1, (3, 3))
        fa, fb, fc, u = oracle.angle_triple(pts[0], pts[1], pts[2], box, K)
        want = np.array([float(g) for g in grad(*pts.ravel())])
        np.testing.assert_allclose(np.concatenate([fa, fb, fc]), want, rtol=1e-11, atol=1e-12)
        F = np.stack([fa, fb, fc])
        assert np.max(np.abs(F.sum(axis=0))) < 1e-12
        assert np.max(np.abs(np.cross(pts - pts[1], F).sum(axis=0))) < 1e-12
        assert abs(np.sum((pts - pts[1]) * F)) < 1e-12


def test_angle_term_in_forces_and_nve():
    """Rings with FENE, the soft push-off and the angle term: forces are -grad U by
    central differences across the periodic boundary, and velocity Verlet
    conserves energy to second order."""
    x, v, box, bonds, angles = inputs.rings(3, 12, rho=0.3, seed=9)
    n = len(x)
    s = oracle.System(n, box, eps=5.0, rc=2 ** (1 / 6), soft=True, bonds=bonds, angles=angles, angle_K=1.5, dt=0.002)
    F, euw = oracle.forces(s, x)
    assert np.max(np.abs(F.sum(axis=0))) < 1e-10 * max(1.0, np.max(np.abs(F)))
    h = 1e-6
    for i in (0, 5, 17, 30):
        for k in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, k] += h
            xm[i, k] -= h
            d = -(oracle.forces(s, xp)[1][0] - oracle.forces(s, xm)[1][0]) / (2 * h)
            assert F[i, k] == pytest.approx(d, abs=1e-5 * max(1.0, abs(F[i, k])))
    dE = []
    for dt in (0.002, 0.001):
        s = oracle.System(n, box, eps=5.0, rc=2 ** (1 / 6), soft=True, bonds=bonds, angles=angles, angle_K=1.5, dt=dt)
        e0 = oracle.forces(s, x, v)[1]
        th = oracle.vv_run(s, x, v, int(round(0.2 / dt)), thermo=True)[3]
        dE.append(np.max(np.abs(th[:, 0] + th[:, 1] - e0[0] - e0[1])))
    assert 3.0 < dE[0] / dE[1] < 5.0
