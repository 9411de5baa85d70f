"""The allocation-free force entry point (md_compute_forces_noalloc) agrees with
md_compute_forces on the same positions, on two calls in a row.

It serves callers that cannot allocate device memory (for instance code that
runs while a stream is captured into a CUDA graph).  This file is collected
last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

from paper_2109_10876_gb300 import inputs
from tests.helpers import force_rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


@pytest.fixture(scope="module")
def md():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_10876_gb300 import md as m
    return m


@pytest.mark.parametrize("precision", [1, 0])
def test_noalloc_matches_compute_forces_twice(md, precision):
    for call, seed in enumerate((21, 22)):          # two calls in a row, new positions each time
        x, v, box = inputs.perturbed_lattice(8, seed=seed, amp=0.15)   # N = 2048
        x, v = x[:2001], v[:2001]                                       # ragged tail
        n = len(x)
        xt = torch.tensor(x.T.copy(), device="cuda")
        vt = torch.tensor(v.T.copy(), device="cuda")
        h = md.md_create(n, box, precision=precision)
        md.md_set_state(h, xt, vt)
        md.md_build_neighbors(h)
        f_ref = torch.zeros(3, n, dtype=torch.float64, device="cuda")
        e_ref = torch.zeros(3, dtype=torch.float64, device="cuda")
        md.md_compute_forces(h, f_ref, e_ref)
        md.md_sync(h)
        h.destroy()
        f = torch.full((3, n), float("nan"), dtype=torch.float64, device="cuda")
        e = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
        md.md_compute_forces_noalloc(xt, vt, n, box, f, e, precision=precision)
        torch.cuda.synchronize()
        F, Fr = f.cpu().numpy().T, f_ref.cpu().numpy().T
        assert force_rel_err(F, Fr) <= TOL[precision], f"call {call}"
        er, eg = e_ref.cpu().numpy(), e.cpu().numpy()
        np.testing.assert_allclose(eg, er, rtol=TOL[precision], atol=TOL[precision] * n)


def test_noalloc_rejects_oversize(md):
    x = torch.zeros(3, 8, dtype=torch.float64, device="cuda")
    f = torch.zeros(3, 8, dtype=torch.float64, device="cuda")
    with pytest.raises(md.MDError) as e:
        md.md_compute_forces_noalloc(x, None, 600000, [100.0, 100.0, 100.0], f)
    assert e.value.status == md.MD_ERR_ARG and "524288" in str(e.value)
