"""Python face of the FP64 CPU oracle (oracle.c), via ctypes and numpy.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py, never by the product package.  Positions,
velocities and forces are (N, 3) float64 arrays here.

What each function follows in arXiv:2109.10876:
  lj_energy / lj_force      Eq. 2 (LJ pair potential), F = -dV/dr (Eq. 1)
  soft_energy / soft_force  cosine push-off for overlapping chains (the melt of
                            Sec. 4 needs a preparation the paper leaves open)
  angle_triple              cosine angle term on chain triples (Sec. 4)
  forces                    direct O(N^2) minimum-image pair sum under r < r_cut
  forces_sample             the same sum for chosen particles only
  bonded_sample             FENE and angle forces (Sec. 4) on chosen particles
  pairs                     the Verlet pair set within r_cut + r_skin (Sec. 2.1.2)
  neighbours_sample         the same set's rows for chosen particles only
  vv_run                    velocity Verlet in two half steps (Fig. 1)
  philox4x32_10             counter-based generator (Salmon et al., SC'11) for the
                            Langevin noise (Sec. 4 names the thermostat only)
"""
import ctypes as C
import os

import numpy as np

from . import build_oracle

_lib = None


class OrcSystem(C.Structure):
    _fields_ = [
        ("n", C.c_int64),
        ("box", C.c_double * 3),
        ("eps", C.c_double),
        ("sigma", C.c_double),
        ("rc", C.c_double),
        ("shift", C.c_int32),
        ("mass", C.c_double),
        ("dt", C.c_double),
        ("gamma", C.c_double),
        ("kT", C.c_double),
        ("seed", C.c_uint64),
        ("n_bonds", C.c_int64),
        ("bonds", C.POINTER(C.c_int32)),
        ("fene_K", C.c_double),
        ("fene_R0", C.c_double),
        ("pot", C.c_int32),
        ("angle_K", C.c_double),
        ("n_angles", C.c_int64),
        ("angles", C.POINTER(C.c_int32)),
    ]


def lib():
    global _lib
    if _lib is None:
        path = build_oracle.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        sp = C.POINTER(OrcSystem)
        L.orc_lj_energy.restype = C.c_double
        L.orc_lj_energy.argtypes = [C.c_double, C.c_double, C.c_double]
        L.orc_lj_force.restype = C.c_double
        L.orc_lj_force.argtypes = [C.c_double, C.c_double, C.c_double]
        L.orc_soft_energy.restype = C.c_double
        L.orc_soft_energy.argtypes = [C.c_double, C.c_double, C.c_double]
        L.orc_soft_force.restype = C.c_double
        L.orc_soft_force.argtypes = [C.c_double, C.c_double, C.c_double]
        L.orc_angle_triple.restype = None
        L.orc_angle_triple.argtypes = [dp, dp, dp, dp, C.c_double, dp, dp, dp, dp]
        L.orc_min_image_r2.restype = C.c_double
        L.orc_min_image_r2.argtypes = [dp, dp, dp]
        L.orc_forces.restype = C.c_int
        L.orc_forces.argtypes = [sp, dp, dp, dp, dp]
        L.orc_forces_sample.restype = C.c_int
        L.orc_forces_sample.argtypes = [sp, dp, C.c_int64, C.POINTER(C.c_int64), dp, dp, dp]
        L.orc_bonded_sample.restype = C.c_int
        L.orc_bonded_sample.argtypes = [sp, dp, C.c_int64, C.POINTER(C.c_int64), dp]
        L.orc_langevin_sample.restype = None
        L.orc_langevin_sample.argtypes = [sp, C.c_int64, C.POINTER(C.c_int64), dp, C.c_int64, dp]
        L.orc_vv_run.restype = C.c_int
        L.orc_vv_run.argtypes = [sp, dp, dp, dp, C.c_int64, C.c_int64, dp]
        L.orc_pairs.restype = C.c_int64
        L.orc_pairs.argtypes = [sp, dp, C.c_double, C.c_int64,
                                C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
        L.orc_neighbours_sample.restype = C.c_int64
        L.orc_neighbours_sample.argtypes = [sp, dp, C.c_double, C.c_int64, C.POINTER(C.c_int64), C.c_int64,
                                            C.POINTER(C.c_int32), dp, C.POINTER(C.c_int32)]
        L.orc_philox4x32_10.restype = None
        L.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                                        C.POINTER(C.c_uint32)]
        L.orc_langevin_uniforms.restype = None
        L.orc_langevin_uniforms.argtypes = [C.c_uint64, C.c_int64, C.c_int64, dp]
        L.orc_hvp.restype = None
        L.orc_hvp.argtypes = [sp, dp, dp, dp, dp, dp]
        L.orc_loss_grad.restype = None
        L.orc_loss_grad.argtypes = [sp, dp, dp, C.c_double, C.c_double, C.c_double, dp, dp, dp, dp]
        L.orc_vv_adjoint.restype = C.c_int
        L.orc_vv_adjoint.argtypes = [sp, dp, dp, C.c_int64, C.c_double, C.c_double, C.c_double, dp, dp, dp, dp, dp,
                                     dp, dp]
        L.orc_set_rc_fixed.restype = None
        L.orc_set_rc_fixed.argtypes = [C.c_int]
        L.orc_num_threads.restype = C.c_int
        L.orc_set_num_threads.restype = None
        L.orc_set_num_threads.argtypes = [C.c_int]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


class System:
    """Parameters of one periodic system (reduced units, Sec. 4: m = eps = sigma = 1).

    rc is absolute (for the LJ fluid 2.5 sigma; for WCA 2**(1/6) sigma).
    shift=True subtracts V(rc) so the pair energy is continuous at the cutoff.
    soft=True replaces the LJ pair by the cosine push-off A (1 + cos(pi r / rc))
    with A = eps (sigma and shift unused).
    """

    def __init__(self, n, box, eps=1.0, sigma=1.0, rc=2.5, shift=True, mass=1.0,
                 dt=0.005, gamma=0.0, kT=1.0, seed=0, bonds=None, fene_K=30.0,
                 fene_R0=1.5, soft=False, angles=None, angle_K=0.0):
        self.n = int(n)
        box = np.broadcast_to(np.asarray(box, dtype=np.float64), (3,)).copy()
        self.box = box
        self.eps, self.sigma, self.rc, self.shift = float(eps), float(sigma), float(rc), bool(shift)
        self.mass, self.dt, self.gamma, self.kT, self.seed = float(mass), float(dt), float(gamma), float(kT), int(seed)
        self.bonds = None if bonds is None else np.ascontiguousarray(bonds, dtype=np.int32).reshape(-1, 2)
        self.fene_K, self.fene_R0 = float(fene_K), float(fene_R0)
        self.soft = bool(soft)
        self.angles = None if angles is None else np.ascontiguousarray(angles, dtype=np.int32).reshape(-1, 3)
        self.angle_K = float(angle_K)

    def c(self):
        s = OrcSystem()
        s.n = self.n
        for k in range(3):
            s.box[k] = self.box[k]
        s.eps, s.sigma, s.rc, s.shift = self.eps, self.sigma, self.rc, int(self.shift)
        s.mass, s.dt, s.gamma, s.kT, s.seed = self.mass, self.dt, self.gamma, self.kT, self.seed
        if self.bonds is not None and len(self.bonds):
            s.n_bonds = len(self.bonds)
            s.bonds = self.bonds.ctypes.data_as(C.POINTER(C.c_int32))
        else:
            s.n_bonds = 0
            s.bonds = C.POINTER(C.c_int32)()
        s.fene_K, s.fene_R0 = self.fene_K, self.fene_R0
        s.pot = 1 if self.soft else 0
        s.angle_K = self.angle_K
        if self.angles is not None and len(self.angles):
            s.n_angles = len(self.angles)
            s.angles = self.angles.ctypes.data_as(C.POINTER(C.c_int32))
        else:
            s.n_angles = 0
            s.angles = C.POINTER(C.c_int32)()
        return s


def lj_energy(r, eps=1.0, sigma=1.0):
    return lib().orc_lj_energy(float(r), float(eps), float(sigma))


def lj_force(r, eps=1.0, sigma=1.0):
    return lib().orc_lj_force(float(r), float(eps), float(sigma))


def soft_energy(r, A=1.0, rc=2 ** (1 / 6)):
    return lib().orc_soft_energy(float(r), float(A), float(rc))


def soft_force(r, A=1.0, rc=2 ** (1 / 6)):
    return lib().orc_soft_force(float(r), float(A), float(rc))


def angle_triple(xa, xb, xc, box, K):
    """Forces (fa, fb, fc) and energy of one cosine angle triple."""
    xa, xb, xc, box = _f64(xa, 3), _f64(xb, 3), _f64(xc, 3), _f64(box, 3)
    fa, fb, fc, u = np.zeros(3), np.zeros(3), np.zeros(3), np.zeros(1)
    lib().orc_angle_triple(_dp(xa), _dp(xb), _dp(xc), _dp(box), float(K), _dp(fa), _dp(fb), _dp(fc), _dp(u))
    return fa, fb, fc, float(u[0])


def min_image_r2(xi, xj, box):
    xi, xj, box = _f64(xi, 3), _f64(xj, 3), _f64(box, 3)
    return lib().orc_min_image_r2(_dp(xi), _dp(xj), _dp(box))


def forces(sysm, x, v=None):
    """Forces (N,3), and (U, K, W) for positions x (N,3). Raises on a broken bond."""
    x = _f64(x, (sysm.n, 3))
    F = np.zeros((sysm.n, 3))
    euw = np.zeros(3)
    vv = None if v is None else _f64(v, (sysm.n, 3))
    s = sysm.c()
    rc = lib().orc_forces(C.byref(s), _dp(x), None if vv is None else _dp(vv), _dp(F), _dp(euw))
    if rc != 0:
        raise RuntimeError(f"oracle forces failed: {rc}")
    return F, euw


def forces_sample(sysm, x, idx):
    """Exact non-bonded forces on particles idx (each summed over all j).

    Returns (F (n,3), U_i halves (n,), W_i halves (n,))."""
    x = _f64(x, (sysm.n, 3))
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    F = np.zeros((len(idx), 3))
    ui = np.zeros(len(idx))
    wi = np.zeros(len(idx))
    s = sysm.c()
    rc = lib().orc_forces_sample(C.byref(s), _dp(x), len(idx),
                                 idx.ctypes.data_as(C.POINTER(C.c_int64)), _dp(F), _dp(ui), _dp(wi))
    if rc != 0:
        raise RuntimeError(f"oracle forces_sample failed: {rc}")
    return F, ui, wi


def bonded_sample(sysm, x, idx):
    """FENE and angle-term forces (Sec. 4) on particles idx only, (n, 3).
    Raises on a broken bond."""
    x = _f64(x, (sysm.n, 3))
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    F = np.zeros((len(idx), 3))
    s = sysm.c()
    rc = lib().orc_bonded_sample(C.byref(s), _dp(x), len(idx), idx.ctypes.data_as(C.POINTER(C.c_int64)), _dp(F))
    if rc != 0:
        raise RuntimeError(f"oracle bonded_sample failed: {rc}")
    return F


def vv_run(sysm, x, v, nsteps, step0=0, thermo=False):
    """Velocity Verlet from (x, v); returns (x, v, F[, thermo (nsteps,3)])."""
    x = _f64(x, (sysm.n, 3)).copy()
    v = _f64(v, (sysm.n, 3)).copy()
    F = np.zeros((sysm.n, 3))
    th = np.zeros((max(int(nsteps), 1), 3)) if thermo else None
    s = sysm.c()
    rc = lib().orc_vv_run(C.byref(s), _dp(x), _dp(v), _dp(F), int(step0), int(nsteps),
                          None if th is None else _dp(th))
    if rc != 0:
        raise RuntimeError(f"oracle vv_run failed: {rc}")
    if thermo:
        return x, v, F, th[:nsteps]
    return x, v, F


def pairs(sysm, x, r):
    """Brute-force pair set {(i, j): i < j, |d_ij| < r}, lexicographic, and per-particle counts."""
    x = _f64(x, (sysm.n, 3))
    s = sysm.c()
    counts = np.zeros(sysm.n, dtype=np.int32)
    m = lib().orc_pairs(C.byref(s), _dp(x), float(r), 0, None,
                        counts.ctypes.data_as(C.POINTER(C.c_int32)))
    out = np.zeros((max(m, 1), 2), dtype=np.int32)
    m2 = lib().orc_pairs(C.byref(s), _dp(x), float(r), m,
                         out.ctypes.data_as(C.POINTER(C.c_int32)), None)
    assert m2 == m
    return out[:m], counts


def neighbours_sample(sysm, x, idx, r):
    """Neighbours within r of the particles idx, by brute force over all j
    (the rows of the pair set of Sec. 2.1.2 for those particles).

    Returns a list with, per sampled particle, (j (ascending int array),
    r^2 of each pair (FP64, the formula of `pairs`))."""
    x = _f64(x, (sysm.n, 3))
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    counts = np.zeros(len(idx), dtype=np.int32)
    s = sysm.c()
    ip = idx.ctypes.data_as(C.POINTER(C.c_int64))
    mx = lib().orc_neighbours_sample(C.byref(s), _dp(x), float(r), len(idx), ip, 0, None, None,
                                     counts.ctypes.data_as(C.POINTER(C.c_int32)))
    if mx < 0:
        raise ValueError("neighbours_sample: index out of range")
    cap = max(int(mx), 1)
    nbr = np.zeros((len(idx), cap), dtype=np.int32)
    r2 = np.zeros((len(idx), cap))
    lib().orc_neighbours_sample(C.byref(s), _dp(x), float(r), len(idx), ip, cap,
                                nbr.ctypes.data_as(C.POINTER(C.c_int32)), _dp(r2),
                                counts.ctypes.data_as(C.POINTER(C.c_int32)))
    return [(nbr[q, :counts[q]].copy(), r2[q, :counts[q]].copy()) for q in range(len(idx))]


def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*[int(t) & 0xFFFFFFFF for t in ctr])
    k = (C.c_uint32 * 2)(*[int(t) & 0xFFFFFFFF for t in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(o[i]) for i in range(4)]


def langevin_uniforms(seed, pid, step):
    u = np.zeros(3)
    lib().orc_langevin_uniforms(int(seed), int(pid), int(step), _dp(u))
    return u


def langevin_sample(sysm, idx, v_idx, step):
    """The Langevin force -gamma m v + sqrt(24 gamma kT m / dt) u (u from
    Philox, keyed by the seed, the particle and the step) on particles idx
    with velocities v_idx (n, 3)."""
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    vv = _f64(v_idx, (len(idx), 3))
    F = np.zeros((len(idx), 3))
    s = sysm.c()
    lib().orc_langevin_sample(C.byref(s), len(idx), idx.ctypes.data_as(C.POINTER(C.c_int64)), _dp(vv),
                              int(step), _dp(F))
    return F


def hvp(sysm, x, w):
    """(J w) of the pair forces at x, and (sum_i w_i . dF_i/deps, sum_i w_i . dF_i/dsigma)."""
    x = _f64(x, (sysm.n, 3))
    w = _f64(w, (sysm.n, 3))
    hv = np.zeros((sysm.n, 3))
    pe, ps = C.c_double(), C.c_double()
    s = sysm.c()
    lib().orc_hvp(C.byref(s), _dp(x), _dp(w), _dp(hv), C.byref(pe), C.byref(ps))
    return hv, pe.value, ps.value


def vv_adjoint(sysm, x, v, nsteps, cU, cK, cW, rc_fixed=False, gx=None, gv=None):
    """Adjoint of nsteps NVE velocity-Verlet steps for L = cU U + cK K + cW W +
    gx . x_T + gv . v_T at the end (gx, gv: (N, 3) gradients of the loss in
    the final positions and velocities, or None).  Returns (euw_T, dL/deps,
    dL/dsigma, lx0, lv0).  By default r_cut moves with sigma (sysm.rc is
    rc_over_sigma * sigma); rc_fixed=True holds it."""
    lib().orc_set_rc_fixed(1 if rc_fixed else 0)
    x = _f64(x, (sysm.n, 3))
    v = _f64(v, (sysm.n, 3))
    gxa = None if gx is None else _f64(gx, (sysm.n, 3))
    gva = None if gv is None else _f64(gv, (sysm.n, 3))
    euw = np.zeros(3)
    ge, gs = C.c_double(), C.c_double()
    lx = np.zeros((sysm.n, 3))
    lv = np.zeros((sysm.n, 3))
    s = sysm.c()
    rc = lib().orc_vv_adjoint(C.byref(s), _dp(x), _dp(v), int(nsteps), float(cU), float(cK), float(cW),
                              None if gxa is None else _dp(gxa), None if gva is None else _dp(gva),
                              _dp(euw), C.byref(ge), C.byref(gs), _dp(lx), _dp(lv))
    if rc != 0:
        raise RuntimeError(f"oracle vv_adjoint failed: {rc}")
    return euw, ge.value, gs.value, lx, lv


def num_threads():
    return lib().orc_num_threads()


def set_num_threads(n):
    """Threads of the oracle's OpenMP loops from now on."""
    lib().orc_set_num_threads(int(n))
