"""Degenerate inputs through the C ABI: an empty replica and a one-particle
replica beside ordinary ones, a lone pair across the periodic boundary, and
a particle exactly on the box edge; each against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2109_10876_gb300 import inputs
from tests.helpers import force_rel_err

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


def forces(md, h, n, nrep):
    f = torch.zeros(3, max(n, 1), dtype=torch.float64, device="cuda")
    euw = torch.zeros(nrep, 3, dtype=torch.float64, device="cuda")
    md.md_compute_forces(h, f, euw)
    md.md_sync(h)
    return f.cpu().numpy().T[:n], euw.cpu().numpy()


@pytest.mark.parametrize("precision", [0, 1])
def test_empty_and_single_particle_replicas(md, precision):
    """Replicas of 0, 1 and 500 particles in one handle: the empty one has no
    energy, the lone particle feels no force, the full one matches the oracle;
    20 steps run without error."""
    x3, v3, b3 = inputs.perturbed_lattice(5, seed=61, amp=0.1)
    x1 = np.array([[1.0, 2.0, 3.0]])
    v1 = np.array([[0.1, -0.2, 0.3]])
    sizes = [0, 1, len(x3)]
    boxes = np.array([[9.0, 9.0, 9.0], [7.0, 8.0, 9.0], b3])
    x = np.concatenate([x1, x3])
    v = np.concatenate([v1, v3])
    h = md.md_create(sizes, boxes, precision=precision)
    md.md_set_state(h, dev(x), dev(v))
    md.md_build_neighbors(h)
    F, euw = forces(md, h, len(x), 3)
    assert np.all(euw[0] == 0.0)
    assert np.all(F[0] == 0.0) and euw[1][0] == 0.0 and euw[1][2] == 0.0
    assert euw[1][1] == pytest.approx(0.5 * np.sum(v1 ** 2), rel=1e-6)
    Fo, eo = oracle.forces(oracle.System(len(x3), b3, rc=2.5), x3, v3)
    tol = 1e-12 if precision == 0 else 1e-5
    assert force_rel_err(F[1:], Fo) <= tol
    np.testing.assert_allclose(euw[2], eo, rtol=tol, atol=tol * len(x3))
    md.md_step(h, 20)
    md.md_sync(h)


@pytest.mark.parametrize("precision", [0, 1])
def test_lone_pair_across_the_boundary_and_on_the_edge(md, precision):
    """Two particles 1.1 apart through the periodic boundary (one at x = 0,
    the other just below L): the force is the LJ force of r = 1.1 along x,
    equal and opposite; a third particle placed exactly at x = L is wrapped
    to 0 and interacts as such."""
    L = 12.0
    box = np.array([L, L, L])
    x = np.array([[0.0, 5.0, 5.0], [L - 1.1, 5.0, 5.0], [L, 9.0, 9.0], [0.9, 9.0, 9.0]])
    v = np.zeros_like(x)
    h = md.md_create(4, box, precision=precision)
    md.md_set_state(h, dev(x), dev(v))
    md.md_build_neighbors(h)
    F, euw = forces(md, h, 4, 1)
    f11 = oracle.lj_force(1.1)
    f09 = oracle.lj_force(0.9)
    tol = 1e-12 if precision == 0 else 1e-6
    np.testing.assert_allclose(F[0], [f11, 0, 0], rtol=tol, atol=tol)
    np.testing.assert_allclose(F[1], [-f11, 0, 0], rtol=tol, atol=tol)
    np.testing.assert_allclose(F[2], [-f09, 0, 0], rtol=tol, atol=tol)
    np.testing.assert_allclose(F[3], [f09, 0, 0], rtol=tol, atol=tol)
    Fo, eo = oracle.forces(oracle.System(4, box, rc=2.5), x, v)
    np.testing.assert_allclose(euw[0], eo, rtol=tol, atol=tol)
