"""Failure detection and recovery, exercised without faulting the GPU.

- A non-finite input is reported as MD_ERR_NONFINITE, and md_set_state clears it.
- A pair closer than the FP32 path's fixed-point sums allow is reported as
  MD_ERR_FIXED_OVERFLOW, with the full list and with the half list.
- A bounded device wait that runs out is reported as MD_ERR_TIMEOUT, and the
  handle keeps working (the library's self-test waits on a barrier that
  nothing completes, with the same bounded wait as the tile kernels).
- An error latched inside a graph-launched md_step ends the step loop: the
  call returns and the next synchronising call reports the error.
- md_set_recovery: a neighbour-list overflow inside md_step (a collapsing gas
  outgrows the automatic capacity) is recovered by growing the list and
  finishing the call, with the same result as a run that never overflowed.
- md_get_checkpoint / md_set_checkpoint: a Langevin run saved and resumed in a
  new handle continues bit for bit (the step counter keys the noise).
"""
import numpy as np
import pytest

from paper_2109_10876_gb300 import inputs

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


def state(md, h, n):
    x = torch.zeros(3, n, dtype=torch.float64, device="cuda")
    v = torch.zeros(3, n, dtype=torch.float64, device="cuda")
    md.md_get_state(h, x, v)
    return host(x), host(v)


# ----------------------------------------------------------------- non-finite input
@pytest.mark.parametrize("precision,which", [(1, "x"), (0, "v")])
def test_nonfinite_state_is_reported_and_cleared(md, precision, which):
    x, v, box = inputs.perturbed_lattice(5, seed=31, amp=0.1)
    n = len(x)
    bad_x, bad_v = x.copy(), v.copy()
    (bad_x if which == "x" else bad_v)[17, 1] = np.nan
    h = md.md_create(n, box, precision=precision)
    md.md_set_state(h, dev(bad_x), dev(bad_v))
    with pytest.raises(md.MDError) as e:
        md.md_sync(h)
    assert e.value.status == md.MD_ERR_NONFINITE
    # a new state clears the error word; the handle then steps normally and
    # agrees with a fresh handle bit for bit
    md.md_set_state(h, dev(x), dev(v))
    md.md_step(h, 10)
    a = state(md, h, n)
    h2 = md.md_create(n, box, precision=precision)
    md.md_set_state(h2, dev(x), dev(v))
    md.md_step(h2, 10)
    b = state(md, h2, n)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


# ----------------------------------------------------------------- fixed-point range
@pytest.mark.parametrize("half", [False, True])
def test_too_close_pair_is_reported(md, half):
    """FP32 + fixed point: one pair at r = 0.3 sigma, whose LJ force is beyond
    the range of the fixed-point sums.  The pair loop flags the rare case and
    the settling pass names it; a clean state afterwards gives the oracle's
    forces."""
    import oracle
    from tests.helpers import force_rel_err
    x, v, box = inputs.perturbed_lattice(5, seed=41, amp=0.05)
    n = len(x)
    bad = x.copy()
    bad[1] = (bad[0] + np.array([0.3, 0.0, 0.0])) % box
    h = md.md_create(n, box, precision=1)
    md.md_set_half_list(h, half)
    md.md_set_state(h, dev(bad), dev(v))
    md.md_build_neighbors(h)
    f = torch.zeros(3, n, dtype=torch.float64, device="cuda")
    md.md_compute_forces(h, f, None)
    with pytest.raises(md.MDError) as e:
        md.md_sync(h)
    assert e.value.status == md.MD_ERR_FIXED_OVERFLOW
    md.md_set_state(h, dev(x), dev(v))
    md.md_build_neighbors(h)
    md.md_compute_forces(h, f, None)
    md.md_sync(h)
    Fo, _ = oracle.forces(oracle.System(n, box, rc=2.5), x, v)
    assert force_rel_err(host(f), Fo) <= 1e-5


# ----------------------------------------------------------------- bounded waits
def test_wait_timeout_is_reported_and_handle_recovers(md):
    x, v, box = inputs.perturbed_lattice(5, seed=32, amp=0.1)
    n = len(x)
    h = md.md_create(n, box)
    md.md_set_state(h, dev(x), dev(v))
    md.md_step(h, 3)
    md.md_sync(h)
    md.md_check_wait_timeout(h, 1000)
    with pytest.raises(md.MDError) as e:
        md.md_sync(h)
    assert e.value.status == md.MD_ERR_TIMEOUT
    # kernels launched while the error is latched return at once (md_step is
    # graph-launched here and must end), and the error stays reported
    md.md_step(h, 5)
    with pytest.raises(md.MDError) as e:
        md.md_sync(h)
    assert e.value.status == md.MD_ERR_TIMEOUT
    md.md_set_state(h, dev(x), dev(v))
    md.md_step(h, 8)
    a = state(md, h, n)
    h2 = md.md_create(n, box)
    md.md_set_state(h2, dev(x), dev(v))
    md.md_step(h2, 8)
    b = state(md, h2, n)
    np.testing.assert_array_equal(a[0], b[0])


def test_wait_timeout_rejects_bad_poll_count(md):
    x, v, box = inputs.perturbed_lattice(4, seed=33, amp=0.1)
    h = md.md_create(len(x), box)
    for polls in (0, 70000):
        with pytest.raises(md.MDError) as e:
            md.md_check_wait_timeout(h, polls)
        assert e.value.status == md.MD_ERR_ARG


# ----------------------------------------------------------------- errors inside the step graph
def collapsing_gas(n=2000, rho=0.15, alpha=0.5, seed=5):
    """A dilute gas (rho = 0.15) whose particles all move towards the box
    centre (v = -alpha (x - c) plus thermal noise): the density in the middle
    rises to liquid values within about 200 steps, so the neighbour lists
    outgrow a capacity sized for the initial gas."""
    L = (n / rho) ** (1.0 / 3.0)
    box = np.array([L, L, L])
    x = inputs.random_gas(n, box, seed=seed, rmin=0.9)
    rng = np.random.default_rng(seed + 7)
    v = -alpha * (x - box / 2) + rng.normal(scale=0.5, size=(n, 3))
    v -= v.mean(axis=0)
    return x, v, box


def test_overflow_inside_step_graph_ends_the_call(md):
    """Without recovery the overflow is latched, the graph-launched step loop
    ends, and the next synchronising call reports it."""
    x, v, box = collapsing_gas()
    h = md.md_create(len(x), box)
    md.md_set_state(h, dev(x), dev(v))
    md.md_build_neighbors(h)
    md.md_step(h, 300)
    with pytest.raises(md.MDError) as e:
        md.md_sync(h)
    assert e.value.status == md.MD_ERR_LIST_OVERFLOW
    # the handle is usable again after a new state
    md.md_set_state(h, dev(x), dev(v))
    md.md_step(h, 20)
    md.md_sync(h)


@pytest.mark.parametrize("thermo_every", [0, 1, 7])
def test_overflow_recovery_matches_uninterrupted_run(md, thermo_every):
    """FP32 + fixed point: forces do not depend on the list capacity or on when
    the list was built, so the recovered run equals a run with room to spare
    bit for bit, energy records included (graph launch without and with
    per-step records, and stream launches for records every 7 steps)."""
    x, v, box = collapsing_gas()
    n = len(x)
    nsteps = 300
    outs = []
    for cap, recover in ((0, True), (256, False)):
        h = md.md_create(n, box, list_capacity=cap)
        md.md_set_recovery(h, recover)
        md.md_set_state(h, dev(x), dev(v))
        md.md_build_neighbors(h)
        K0 = md.md_get_stats(h)["list_capacity"]
        nrec = nsteps // thermo_every if thermo_every else 0
        th = torch.zeros(max(nrec, 1), 3, dtype=torch.float64, device="cuda")
        md.md_step(h, nsteps, thermo_every, th if nrec else None)
        st = md.md_get_stats(h)
        outs.append((state(md, h, n), th.cpu().numpy()[:nrec], st, K0))
    (xa, va), tha, sa, K0a = outs[0]
    (xb, vb), thb, sb, _ = outs[1]
    assert K0a == 64 and sa["recoveries"] >= 1 and sa["list_capacity"] > 64
    assert sb["recoveries"] == 0 and sa["steps"] == sb["steps"] == nsteps
    np.testing.assert_array_equal(xa, xb)
    np.testing.assert_array_equal(va, vb)
    np.testing.assert_array_equal(tha, thb)   # exact 64-bit sums


# ----------------------------------------------------------------- checkpoint and resume
@pytest.mark.parametrize("precision", [1, 0])
def test_checkpoint_resume_continues_langevin_run(md, precision):
    """Langevin LJ liquid: 25 steps, checkpoint, resume in a new handle, 25
    more steps; equal to 50 steps in one handle (two calls), bit for bit in
    FP32 + fixed point and to rounding in FP64.  md_set_state alone restarts
    the noise from step 0, which the same test shows differs."""
    x, v, box = inputs.perturbed_lattice(8, seed=34, amp=0.1)
    n = len(x)
    kw = dict(precision=precision, langevin_gamma=0.5, kT=1.0, seed=77)
    ha = md.md_create(n, box, **kw)
    md.md_set_state(ha, dev(x), dev(v))
    md.md_step(ha, 25)
    md.md_step(ha, 25)
    xa, va = state(md, ha, n)

    hb = md.md_create(n, box, **kw)
    md.md_set_state(hb, dev(x), dev(v))
    md.md_step(hb, 25)
    cx = torch.zeros(3, n, dtype=torch.float64, device="cuda")
    cv, cf = torch.zeros_like(cx), torch.zeros_like(cx)
    step = md.md_get_checkpoint(hb, cx, cv, cf)
    assert step == 25
    hb.destroy()
    hc = md.md_create(n, box, **kw)
    md.md_set_checkpoint(hc, cx.cpu(), cv.cpu(), cf.cpu(), step)   # host copies: any memory works
    md.md_step(hc, 25)
    xc, vc = state(md, hc, n)
    assert md.md_get_stats(hc)["steps"] == 50
    if precision == 1:
        np.testing.assert_array_equal(xc, xa)
        np.testing.assert_array_equal(vc, va)
    else:
        np.testing.assert_allclose(xc, xa, rtol=0, atol=1e-10)
        np.testing.assert_allclose(vc, va, rtol=0, atol=1e-9)
    # restarting from the same (x, v) without the step counter replays the
    # noise of steps 0..24: a different trajectory
    hd = md.md_create(n, box, **kw)
    md.md_set_state(hd, cx, cv)
    md.md_step(hd, 25)
    xd, _ = state(md, hd, n)
    assert np.max(np.abs(xd - xa)) > 1e-6


def test_checkpoint_arguments(md):
    x, v, box = inputs.perturbed_lattice(4, seed=35, amp=0.1)
    n = len(x)
    h = md.md_create(n, box)
    t = torch.zeros(3, n, dtype=torch.float64, device="cuda")
    with pytest.raises(md.MDError) as e:
        md.md_get_checkpoint(h, t, t, t)                 # before md_set_state
    assert e.value.status == md.MD_ERR_ARG
    with pytest.raises(md.MDError) as e:
        md.md_set_checkpoint(h, dev(x), dev(v), t, -1)
    assert e.value.status == md.MD_ERR_ARG
    # a checkpoint taken right after md_set_state evaluates the stored force
    md.md_set_state(h, dev(x), dev(v))
    f = torch.zeros(3, n, dtype=torch.float64, device="cuda")
    assert md.md_get_checkpoint(h, t.clone(), t.clone(), f) == 0
    f_ref = torch.zeros(3, n, dtype=torch.float64, device="cuda")
    md.md_compute_forces(h, f_ref, None)
    md.md_sync(h)
    np.testing.assert_array_equal(f.cpu().numpy(), f_ref.cpu().numpy())
