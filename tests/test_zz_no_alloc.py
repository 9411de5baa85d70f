"""The allocation-free force entry point, md_compute_forces_noalloc.

It is for callers that cannot call cudaMalloc: a host framework that owns all
device memory through its own pool, or a process held to a fixed memory
budget.  Its only scratch is a fixed array inside the library.  Checked here,
through the C ABI, on two calls in a row (the shared scratch keeps the last
call's contents):
  - against md_compute_forces on the same positions, at the tolerances of the
    other force tests (1e-5 in FP32 + fixed point, 1e-12 in FP64);
  - element by element against the FP64 oracle's direct pair sum, with the
    device's free memory unchanged by the call;
  - a pair closer than the fixed-point range (r = 0.3 sigma) poisons the two
    particles' force rows and U, W with NaN in FP32 + fixed point;
  - sizes beyond the fixed scratch are rejected with a message.
This file is collected last so that a run stopping at the first failure has
run every other test.
"""
import numpy as np
import pytest

import oracle
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


def system(seed):
    x, v, box = inputs.perturbed_lattice(8, seed=seed, amp=0.15)   # N = 2048
    return x[:2001], v[:2001], box                                  # ragged tail


@pytest.mark.parametrize("precision", [1, 0])
def test_noalloc_matches_compute_forces_twice(md, precision):
    for call, seed in enumerate((21, 22)):          # two calls in a row, new positions each time
        x, v, box = system(seed)
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


@pytest.mark.parametrize("precision", [1, 0])
def test_noalloc_matches_oracle_twice(md, precision):
    # one untimed call first: with lazy module loading the library's kernels
    # and its fixed scratch array are loaded onto the device at their first use
    x, v, box = system(23)
    xt = torch.tensor(x.T.copy(), device="cuda")
    md.md_compute_forces_noalloc(xt, None, len(x), box, torch.empty(3, len(x), dtype=torch.float64, device="cuda"),
                                 precision=precision)
    torch.cuda.synchronize()
    for call, seed in enumerate((23, 24)):
        x, v, box = system(seed)
        n = len(x)
        s = oracle.System(n, box, rc=2.5)
        F_ref, euw_ref = oracle.forces(s, x, v)
        xt = torch.tensor(x.T.copy(), device="cuda")
        vt = torch.tensor(v.T.copy(), device="cuda")
        f = torch.full((3, n), float("nan"), dtype=torch.float64, device="cuda")
        e = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        alloc0 = torch.cuda.memory_allocated()
        md.md_compute_forces_noalloc(xt, vt, n, box, f, e, precision=precision)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        # nothing allocated: the device's free memory and torch's pool are unchanged
        assert free1 == free0 and torch.cuda.memory_allocated() == alloc0, f"call {call}"
        F = f.cpu().numpy().T
        assert force_rel_err(F, F_ref) <= TOL[precision], f"call {call}"
        np.testing.assert_allclose(e.cpu().numpy(), euw_ref, rtol=TOL[precision], atol=TOL[precision] * n)


def test_noalloc_reports_too_close_pair(md):
    """Two particles 0.3 sigma apart: the LJ force there (about 2.7e7) is
    outside the 64-bit fixed-point range of the FP32 path, so both particles'
    force rows and U, W come back NaN; the other rows are the
    oracle's.  The next call with clean positions is clean again."""
    x, v, box = system(25)
    n = len(x)
    x = x.copy()
    x[5] = x[4] + np.array([0.3, 0.0, 0.0])
    xt = torch.tensor(x.T.copy(), device="cuda")
    f = torch.zeros(3, n, dtype=torch.float64, device="cuda")
    e = torch.zeros(3, dtype=torch.float64, device="cuda")
    md.md_compute_forces_noalloc(xt, None, n, box, f, e, precision=md.MD_FP32_FIXED)
    torch.cuda.synchronize()
    F = f.cpu().numpy().T
    eu = e.cpu().numpy()
    assert np.all(np.isnan(F[[4, 5]])) and np.isnan(eu[0]) and np.isnan(eu[2]) and eu[1] == 0.0   # no v: K = 0
    ok = np.ones(n, dtype=bool)
    ok[[4, 5]] = False
    assert np.all(np.isfinite(F[ok]))
    F_ref, _ = oracle.forces(oracle.System(n, box, rc=2.5), x)
    far = ok & (np.linalg.norm(F_ref, axis=1) < 1e4)    # rows not touched by the huge pair
    assert force_rel_err(F[far], F_ref[far]) <= TOL[1]
    x2, v2, _ = system(26)
    md.md_compute_forces_noalloc(torch.tensor(x2.T.copy(), device="cuda"), None, n, box, f, e)
    torch.cuda.synchronize()
    assert np.all(np.isfinite(f.cpu().numpy())) and np.all(np.isfinite(e.cpu().numpy()))


def test_noalloc_rejects_oversize(md):
    x = torch.zeros(3, 8, dtype=torch.float64, device="cuda")
    f = torch.zeros(3, 8, dtype=torch.float64, device="cuda")
    with pytest.raises(md.MDError) as e:
        md.md_compute_forces_noalloc(x, None, 600000, [100.0, 100.0, 100.0], f)
    assert e.value.status == md.MD_ERR_ARG and "524288" in str(e.value)
