"""Tile size: parity at every size the tuner can pick, and md_autotune.

A tile is the GPU's unit of work, the counterpart of the paper's HPX subnode
(Sec. 3.3); its size is tuned the way the paper tunes the subnode count
(Sec. 4.2).  The pair set, the FP32 fixed-point forces and the trajectory
must not depend on it: the pair set and the fixed-point sums are exact.
"""
import numpy as np
import pytest

import oracle
from paper_2109_10876_gb300 import inputs
from tests.helpers import force_rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RC, SKIN = 2.5, 0.3


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


def state(md, h, n):
    xo = torch.zeros(3, n, dtype=torch.float64, device="cuda")
    vo = torch.zeros_like(xo)
    md.md_get_state(h, xo, vo)
    return host(xo), host(vo)


@pytest.fixture(scope="module")
def fluid():
    """N = 16384 perturbed fcc at rho = 0.8442: a 9^3 cell grid, about 22
    particles per cell, so tiles of 128 span several cells and tiles of 8
    are single cells."""
    x, v, box = inputs.perturbed_lattice(16, seed=71, amp=0.1)
    return x, v, box


def test_pairs_and_forces_every_tile_size(md, fluid):
    x, v, box = fluid
    n = len(x)
    sysm = oracle.System(n, box, rc=RC)
    want_pairs, _ = oracle.pairs(sysm, x, RC + SKIN)
    Fo, euwo = oracle.forces(sysm, x, v)
    h = md.md_create(n, box, precision=1, skin=SKIN)
    md.md_set_state(h, dev(x), dev(v))
    ref = None
    tiles = []
    for size in (128, 112, 96, 80, 64, 32, 16, 8, 1):
        md.md_set_tile_size(h, size)
        md.md_build_neighbors(h)
        np.testing.assert_array_equal(md.export_pairs_sorted(h), want_pairs)
        f = torch.zeros(3, n, dtype=torch.float64, device="cuda")
        euw = torch.zeros(1, 3, dtype=torch.float64, device="cuda")
        md.md_compute_forces(h, f, euw)
        md.md_sync(h)
        F = host(f)
        assert force_rel_err(F, Fo) <= 1e-5
        np.testing.assert_allclose(euw.cpu().numpy()[0], euwo, rtol=1e-5, atol=1e-5 * n)
        if ref is None:
            ref = F
        else:
            np.testing.assert_array_equal(F, ref)   # fixed-point sums: order-free
        st = md.md_get_stats(h)
        assert st["tile_size"] == size
        tiles.append(st["n_tiles"])
    assert all(a <= b for a, b in zip(tiles, tiles[1:]))
    assert tiles[-1] == 9 ** 3          # one cell per tile
    assert tiles[0] < tiles[-1]


def test_set_tile_size_rejects_out_of_range(md, fluid):
    x, v, box = fluid
    h = md.md_create(len(x), box)
    for bad in (0, -1, 129):
        with pytest.raises(md.MDError) as e:
            md.md_set_tile_size(h, bad)
        assert e.value.status == md.MD_ERR_ARG


def test_autotune_keeps_the_trajectory(md, fluid):
    """Langevin (so the step counter feeds the noise): 10 steps, md_autotune,
    10 steps equals 20 steps straight, bit for bit, in FP32 fixed point."""
    x, v, box = fluid
    n = len(x)
    kw = dict(precision=1, skin=SKIN, langevin_gamma=0.5, kT=0.72, seed=99)
    h1 = md.md_create(n, box, **kw)
    md.md_set_state(h1, dev(x), dev(v))
    md.md_build_neighbors(h1)
    md.md_step(h1, 20)
    a = state(md, h1, n)
    h2 = md.md_create(n, box, **kw)
    md.md_set_state(h2, dev(x), dev(v))
    md.md_build_neighbors(h2)
    md.md_step(h2, 10)
    chosen = md.md_autotune(h2, 5)
    assert chosen in (128, 112, 96, 80, 64, 32, 16, 8)
    st = md.md_get_stats(h2)
    assert st["tile_size"] == chosen and st["steps"] == 10
    md.md_step(h2, 10)
    b = state(md, h2, n)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
