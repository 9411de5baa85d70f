"""Cases run under the checked build (libmd_gb300_checked.so, device-side
bounds checks).  Not collected by the default pytest run: test_gpu_checked.py
runs this file in a child process with MD_GB300_CHECKED=1, so that the
binding loads the checked library.

- Every path of the library -- binning, re-sort, tiling, the list build, the
  FP32 and FP64 force kernels, the half list, bonded terms, uneven replicas
  with two to four cells per axis, the reverse pass -- runs with every check
  armed and agrees with the oracle: no check fails on valid inputs.
- Each check site, made to fail on purpose (md_check_bounds_selftest, with an
  index that is in range), is reported as MD_ERR_BOUNDS with that site, and
  md_set_state clears it: the handle then computes the oracle's forces again.
"""
import numpy as np
import pytest

import oracle
from paper_2109_10876_gb300 import inputs
from tests.helpers import force_rel_err, min_image_diff

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def forces(md, h, n, nrep=1):
    f = torch.zeros(3, n, dtype=torch.float64, device="cuda")
    euw = torch.zeros(nrep, 3, dtype=torch.float64, device="cuda")
    md.md_compute_forces(h, f, euw)
    md.md_sync(h)
    return host(f), euw.cpu().numpy()


def test_the_checked_library_is_loaded(md):
    assert md.CHECKED and md.LIB_PATH.endswith("libmd_gb300_checked.so")
    assert md.md_build_flags() & md.MD_BUILD_CHECKED


@pytest.mark.parametrize("precision", [1, 0])
def test_fluid_forces_and_trajectory(md, precision):
    """LJ fluid, 4000 particles: forces at the start and 100 steps with
    rebuilds, every check armed; parity as in the default build."""
    x, v, box = inputs.perturbed_lattice(10, seed=91, amp=0.1)
    n = len(x)
    h = md.md_create(n, box, precision=precision)
    md.md_set_state(h, dev(x), dev(v))
    md.md_build_neighbors(h)
    F, _ = forces(md, h, n)
    s = oracle.System(n, box, rc=2.5, dt=0.005)
    Fo, _ = oracle.forces(s, x, v)
    assert force_rel_err(F, Fo) <= (1e-5 if precision == 1 else 1e-12)
    md.md_step(h, 100)
    xg = torch.zeros(3, n, dtype=torch.float64, device="cuda")
    vg = torch.zeros_like(xg)
    md.md_get_state(h, xg, vg)
    st = md.md_get_stats(h)
    assert st["rebuilds"] >= 2 and st["bad_site"] == 0 and st["error_word"] == 0
    if precision == 0:
        x1, _, _ = oracle.vv_run(s, x, v, 100)
        assert np.max(np.abs(min_image_diff(host(xg), x1, box))) < 1e-10


def test_uneven_replicas_of_small_boxes(md):
    """Random gases in boxes of two to four cells per axis (halo rows that
    wrap onto themselves, whole-row halos) as replicas of one handle."""
    boxes = np.array([[6.0, 6.0, 6.0], [9.0, 6.5, 12.0], [12.0, 12.0, 12.0]])
    sizes = [120, 400, 1000]
    xs = [inputs.random_gas(nr, b, seed=92 + r, rmin=0.9) for r, (nr, b) in enumerate(zip(sizes, boxes))]
    vs = [inputs.maxwell_velocities(nr, 1.0, 95 + r) for r, nr in enumerate(sizes)]
    for precision in (1, 0):
        h = md.md_create(sizes, boxes, precision=precision)
        md.md_set_state(h, dev(np.concatenate(xs)), dev(np.concatenate(vs)))
        md.md_build_neighbors(h)
        F, _ = forces(md, h, sum(sizes), nrep=3)
        a = 0
        for r, nr in enumerate(sizes):
            Fo, _ = oracle.forces(oracle.System(nr, boxes[r], rc=2.5), xs[r], vs[r])
            assert force_rel_err(F[a:a + nr], Fo) <= (1e-5 if precision == 1 else 1e-12)
            a += nr
        md.md_step(h, 30)
        assert md.md_get_stats(h)["bad_site"] == 0


def chains_system(md, precision=1):
    box = np.array([9.0, 9.0, 9.0])
    x, bonds = inputs.chains(12, 25, box, seed=52)
    n = len(x)
    v = inputs.maxwell_velocities(n, 1.0, 53)
    angles = np.array([(c * 25 + k - 1, c * 25 + k, c * 25 + k + 1) for c in range(12) for k in range(1, 24)],
                      dtype=np.int32)
    h = md.md_create(n, box, precision=precision, potential=md.MD_WCA, skin=0.4, bonds=bonds, fene_K=30.0,
                     fene_R0=1.5, angles=angles, angle_K=1.5)
    s = oracle.System(n, box, rc=2 ** (1 / 6), bonds=bonds, fene_K=30.0, fene_R0=1.5, angles=angles, angle_K=1.5)
    return h, s, x, v


@pytest.mark.parametrize("precision", [1, 0])
def test_bonded_chains(md, precision):
    h, s, x, v = chains_system(md, precision)
    md.md_set_state(h, dev(x), dev(v))
    md.md_build_neighbors(h)
    F, _ = forces(md, h, len(x))
    Fo, _ = oracle.forces(s, x, v)
    assert force_rel_err(F, Fo) <= (1e-5 if precision == 1 else 1e-12)
    md.md_step(h, 20)
    assert md.md_get_stats(h)["bad_site"] == 0


def test_half_list(md):
    x, v, box = inputs.perturbed_lattice(8, seed=97, amp=0.1)
    n = len(x)
    h = md.md_create(n, box, precision=1)
    md.md_set_half_list(h, True)
    md.md_set_state(h, dev(x), dev(v))
    md.md_build_neighbors(h)
    F, _ = forces(md, h, n)
    Fo, _ = oracle.forces(oracle.System(n, box, rc=2.5), x, v)
    assert force_rel_err(F, Fo) <= 1e-5
    md.md_step(h, 20)
    assert md.md_get_stats(h)["bad_site"] == 0


@pytest.mark.parametrize("precision,tol", [(0, 1e-8), (1, 2e-4)])
def test_reverse_pass(md, precision, tol):
    x, v, box = inputs.perturbed_lattice(5, T=0.9, seed=82, amp=0.08)
    n = len(x)
    h = md.md_create(n, box, precision=precision)
    md.md_set_state(h, dev(x), dev(v))
    md.md_build_neighbors(h)
    md.md_forward(h, 7, 3, None)
    V = float(np.prod(box))
    c = np.array([[1.0 / n, 2.0 / (3 * V), 1.0 / (3 * V)]])
    ge, gs = np.zeros(1), np.zeros(1)
    md.md_backward(h, None, None, c, ge, gs)
    _, ge_ref, gs_ref, _, _ = oracle.vv_adjoint(oracle.System(n, box, rc=2.5, dt=0.005), x, v, 7, *c[0])
    assert ge[0] == pytest.approx(ge_ref, rel=tol)
    assert gs[0] == pytest.approx(gs_ref, rel=tol)


# Each site with the system and the call that evaluates it: "build" (the
# re-sort, tiling and list build), "force" (md_compute_forces after a clean
# build) or "backward" (md_backward after a clean md_forward).
SITES = [
    (1, "fluid", "build"), (2, "fluid", "build"), (3, "fluid", "build"), (4, "chains", "build"),
    (5, "fluid", "build"), (6, "fluid", "build"), (7, "fluid", "build"), (8, "fluid", "build"),
    (9, "fluid", "force"), (10, "fluid", "force"), (11, "half", "force"), (12, "chains", "force"),
    (13, "fluid", "backward"),
]


@pytest.mark.parametrize("site,system,call", SITES)
def test_each_site_reports_its_failure_and_recovers(md, site, system, call):
    if system == "chains":
        h, s, x, v = chains_system(md)
    else:
        x, v, box = inputs.perturbed_lattice(6, seed=98, amp=0.1)
        h = md.md_create(len(x), box, precision=1)
        if system == "half":
            md.md_set_half_list(h, True)
        s = oracle.System(len(x), box, rc=2.5, dt=0.005)
    n = len(x)
    md.md_set_state(h, dev(x), dev(v))
    if call != "build":
        md.md_build_neighbors(h)
    if call == "backward":
        md.md_forward(h, 3, 3, None)
    md.md_check_bounds_selftest(h, site)
    with pytest.raises(md.MDError) as e:
        if call == "build":
            md.md_build_neighbors(h)
        elif call == "force":
            forces(md, h, n)
        else:
            md.md_backward(h, None, None, np.array([[1.0, 0.0, 0.0]]), np.zeros(1), np.zeros(1))
            md.md_sync(h)
    assert e.value.status == md.MD_ERR_BOUNDS
    assert f"site {site} " in str(e.value)
    st = md.md_get_stats(h, check=False)
    assert st["bad_site"] == site and st["error_word"] & 32
    # md_set_state disarms the site and clears the error: the oracle's forces again
    md.md_set_state(h, dev(x), dev(v))
    md.md_build_neighbors(h)
    F, _ = forces(md, h, n)
    Fo, _ = oracle.forces(s, x, v)
    assert force_rel_err(F, Fo) <= 1e-5
    assert md.md_get_stats(h)["bad_site"] == 0
