"""Thin ctypes binding of the C ABI in include/md.h (same function names).

Argument marshalling only: every step of the computation runs in the CUDA
library lib/libmd_gb300.so.  Arrays may be torch tensors (CUDA or CPU) or
numpy arrays; their data pointers are passed straight through, so they must
be contiguous float64 (positions, velocities, forces) in the (3, N)
component-major layout.  Streams are torch.cuda.Stream objects, raw
cudaStream_t integers, or None for the current torch stream.

Importing this module loads the library and raises if it is missing: there
is no fallback implementation.  With MD_GB300_CHECKED=1 in the environment it
loads the checked build lib/libmd_gb300_checked.so instead (device-side
bounds checks, md_build_flags() & MD_BUILD_CHECKED).
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
CHECKED = os.environ.get("MD_GB300_CHECKED", "0") not in ("", "0")
LIB_PATH = os.path.join(_HERE, "lib", "libmd_gb300_checked.so" if CHECKED else "libmd_gb300.so")

MD_OK = 0
MD_ERR_ARG = -1
MD_ERR_CUDA = -2
MD_ERR_LIST_OVERFLOW = -3
MD_ERR_NONFINITE = -4
MD_ERR_BOND_BROKEN = -5
MD_ERR_FIXED_OVERFLOW = -6
MD_ERR_TIMEOUT = -7
MD_ERR_BOX_TOO_SMALL = -8
MD_ERR_BOUNDS = -9
STATUS_NAMES = {0: "MD_OK", -1: "MD_ERR_ARG", -2: "MD_ERR_CUDA", -3: "MD_ERR_LIST_OVERFLOW",
                -4: "MD_ERR_NONFINITE", -5: "MD_ERR_BOND_BROKEN", -6: "MD_ERR_FIXED_OVERFLOW",
                -7: "MD_ERR_TIMEOUT", -8: "MD_ERR_BOX_TOO_SMALL", -9: "MD_ERR_BOUNDS"}
MD_BUILD_CHECKED = 1
# md_check_site
MD_SITES = {1: "MD_SITE_BIN_CELL", 2: "MD_SITE_SCATTER", 3: "MD_SITE_REORDER", 4: "MD_SITE_TOPOLOGY",
            5: "MD_SITE_TILE_WRITE", 6: "MD_SITE_PIECES", 7: "MD_SITE_LIST_RANGE", 8: "MD_SITE_LIST_SELF",
            9: "MD_SITE_FORCE_HALO", 10: "MD_SITE_FORCE_OWN", 11: "MD_SITE_FORCE_SLOT", 12: "MD_SITE_BOND_SLOT",
            13: "MD_SITE_ADJ"}
globals().update({v: k for k, v in MD_SITES.items()})
MD_LJ, MD_WCA, MD_SOFT = 0, 1, 2
MD_SECT_NEIGH, MD_SECT_FORCE, MD_SECT_OTHER, MD_NSECT = 0, 1, 2, 3
MD_FP64, MD_FP32_FIXED = 0, 1


class md_params(C.Structure):
    _fields_ = [
        ("n_replicas", C.c_int32),
        ("replica_offsets", C.POINTER(C.c_int64)),
        ("box", C.POINTER(C.c_double)),
        ("eps", C.POINTER(C.c_double)),
        ("sigma", C.POINTER(C.c_double)),
        ("rc_over_sigma", C.c_double),
        ("skin", C.c_double),
        ("dt", C.c_double),
        ("mass", C.c_double),
        ("potential", C.c_int32),
        ("precision", C.c_int32),
        ("langevin_gamma", C.c_double),
        ("kT", C.c_double),
        ("seed", C.c_uint64),
        ("fene_K", C.c_double),
        ("fene_R0", C.c_double),
        ("n_bonds", C.c_int64),
        ("bonds", C.POINTER(C.c_int32)),
        ("list_capacity", C.c_int32),
        ("reserved0", C.c_int32),
        ("angle_K", C.c_double),
        ("n_angles", C.c_int64),
        ("angles", C.POINTER(C.c_int32)),
    ]


class md_stats(C.Structure):
    _fields_ = [
        ("steps", C.c_int64),
        ("rebuilds", C.c_int64),
        ("list_entries", C.c_int64),
        ("max_list_len", C.c_int32),
        ("list_capacity", C.c_int32),
        ("max_cell_occupancy", C.c_int32),
        ("error_word", C.c_int32),
        ("ncell", C.c_int32 * 3),
        ("n_replicas", C.c_int32),
        ("n_particles", C.c_int64),
        ("n_tiles", C.c_int32),
        ("max_halo", C.c_int32),
        ("halo_capacity", C.c_int32),
        ("tile_size", C.c_int32),
        ("recoveries", C.c_int64),
        ("bad_index", C.c_int64),
        ("bad_site", C.c_int32),
    ]


if not os.path.exists(LIB_PATH):
    raise ImportError(f"CUDA library not built: {LIB_PATH} is missing "
                      "(run paper_2109_10876_gb300/build.py or __graft_entry__.build())")
_lib = C.CDLL(LIB_PATH)
_vp = C.c_void_p
_H = C.c_void_p
_lib.md_create.restype = C.c_int
_lib.md_create.argtypes = [C.POINTER(md_params), C.POINTER(_H)]
_lib.md_destroy.restype = None
_lib.md_destroy.argtypes = [_H]
_lib.md_set_state.restype = C.c_int
_lib.md_set_state.argtypes = [_H, _vp, _vp, _vp]
_lib.md_get_state.restype = C.c_int
_lib.md_get_state.argtypes = [_H, _vp, _vp, _vp]
_lib.md_build_neighbors.restype = C.c_int
_lib.md_build_neighbors.argtypes = [_H, _vp]
_lib.md_compute_forces.restype = C.c_int
_lib.md_compute_forces.argtypes = [_H, _vp, _vp, _vp]
_lib.md_step.restype = C.c_int
_lib.md_step.argtypes = [_H, C.c_int32, C.c_int32, _vp, _vp]
_lib.md_export_pairs.restype = C.c_int
_lib.md_export_pairs.argtypes = [_H, _vp, C.c_int64, C.POINTER(C.c_int64), _vp]
_lib.md_sync.restype = C.c_int
_lib.md_sync.argtypes = [_H, _vp]
_lib.md_get_stats.restype = C.c_int
_lib.md_get_stats.argtypes = [_H, C.POINTER(md_stats)]
_lib.md_forward.restype = C.c_int
_lib.md_forward.argtypes = [_H, C.c_int32, C.c_int32, _vp, _vp]
_lib.md_backward.restype = C.c_int
_lib.md_backward.argtypes = [_H, _vp, _vp, _vp, _vp, _vp, _vp]
_lib.md_get_checkpoint.restype = C.c_int
_lib.md_get_checkpoint.argtypes = [_H, _vp, _vp, _vp, C.POINTER(C.c_int64), _vp]
_lib.md_set_checkpoint.restype = C.c_int
_lib.md_set_checkpoint.argtypes = [_H, _vp, _vp, _vp, C.c_int64, _vp]
_lib.md_set_recovery.restype = C.c_int
_lib.md_set_recovery.argtypes = [_H, C.c_int32]
_lib.md_check_wait_timeout.restype = C.c_int
_lib.md_check_wait_timeout.argtypes = [_H, C.c_int32, _vp]
_lib.md_build_flags.restype = C.c_int
_lib.md_build_flags.argtypes = []
_lib.md_check_bounds_selftest.restype = C.c_int
_lib.md_check_bounds_selftest.argtypes = [_H, C.c_int32, _vp]
_lib.md_autotune.restype = C.c_int
_lib.md_autotune.argtypes = [_H, C.c_int32, C.POINTER(C.c_int32), _vp]
_lib.md_set_tile_size.restype = C.c_int
_lib.md_set_tile_size.argtypes = [_H, C.c_int32, _vp]
_lib.md_set_half_list.restype = C.c_int
_lib.md_set_half_list.argtypes = [_H, C.c_int32, _vp]
_lib.md_set_timing.restype = C.c_int
_lib.md_set_timing.argtypes = [_H, C.c_int32]
_lib.md_get_timing.restype = C.c_int
_lib.md_get_timing.argtypes = [_H, C.POINTER(C.c_double), C.POINTER(C.c_int64)]
_lib.md_compute_forces_noalloc.restype = C.c_int
_lib.md_compute_forces_noalloc.argtypes = [_vp, _vp, C.c_int64, C.POINTER(C.c_double), C.c_double, C.c_double,
                                           C.c_double, C.c_int32, C.c_int32, C.c_double, _vp, _vp,
                                           C.c_char_p, C.c_int32, _vp]
_lib.md_probe_fp64_fma.restype = C.c_int
_lib.md_probe_fp64_fma.argtypes = [C.c_int64, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double), _vp]
_lib.md_last_error.restype = C.c_char_p
_lib.md_last_error.argtypes = [_H]


class MDError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def lib():
    return _lib


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return int(a)


def _stream(s):
    if s is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream
    return int(s)


def _check(h, status):
    if status != MD_OK:
        msg = _lib.md_last_error(h)
        raise MDError(status, msg.decode() if msg else "")
    return status


class Handle:
    """Owns an md_handle*; keeps the host arrays passed to md_create alive."""

    def __init__(self, ptr, keep):
        self.ptr = ptr
        self._keep = keep

    def __del__(self):
        self.destroy()

    def destroy(self):
        if getattr(self, "ptr", None):
            _lib.md_destroy(self.ptr)
            self.ptr = None


def md_create(n_per_replica, box, eps=1.0, sigma=1.0, rc_over_sigma=2.5, skin=0.3, dt=0.005, mass=1.0,
              potential=MD_LJ, precision=MD_FP32_FIXED, langevin_gamma=0.0, kT=1.0, seed=0,
              fene_K=30.0, fene_R0=1.5, bonds=None, list_capacity=0, angles=None, angle_K=0.0):
    """md_create: n_per_replica is an int or a list of per-replica counts;
    box is (3,) or (R, 3); eps, sigma scalars or per replica."""
    sizes = np.atleast_1d(np.asarray(n_per_replica, dtype=np.int64))
    R = len(sizes)
    off = np.zeros(R + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    boxa = np.ascontiguousarray(np.broadcast_to(np.asarray(box, dtype=np.float64), (R, 3)))
    epsa = np.ascontiguousarray(np.broadcast_to(np.asarray(eps, dtype=np.float64), (R,)))
    siga = np.ascontiguousarray(np.broadcast_to(np.asarray(sigma, dtype=np.float64), (R,)))
    p = md_params()
    p.n_replicas = R
    p.replica_offsets = off.ctypes.data_as(C.POINTER(C.c_int64))
    p.box = boxa.ctypes.data_as(C.POINTER(C.c_double))
    p.eps = epsa.ctypes.data_as(C.POINTER(C.c_double))
    p.sigma = siga.ctypes.data_as(C.POINTER(C.c_double))
    p.rc_over_sigma = rc_over_sigma
    p.skin = skin
    p.dt = dt
    p.mass = mass
    p.potential = potential
    p.precision = precision
    p.langevin_gamma = langevin_gamma
    p.kT = kT
    p.seed = seed
    p.fene_K = fene_K
    p.fene_R0 = fene_R0
    bonda = None
    if bonds is not None and len(bonds):
        bonda = np.ascontiguousarray(bonds, dtype=np.int32).reshape(-1, 2)
        p.n_bonds = len(bonda)
        p.bonds = bonda.ctypes.data_as(C.POINTER(C.c_int32))
    p.list_capacity = list_capacity
    anga = None
    if angles is not None and len(angles):
        anga = np.ascontiguousarray(angles, dtype=np.int32).reshape(-1, 3)
        p.n_angles = len(anga)
        p.angles = anga.ctypes.data_as(C.POINTER(C.c_int32))
        p.angle_K = angle_K
    h = _H()
    st = _lib.md_create(C.byref(p), C.byref(h))
    if st != MD_OK:
        raise MDError(st, "md_create failed")
    return Handle(h, (off, boxa, epsa, siga, bonda, anga))


def md_destroy(h):
    h.destroy()


def md_set_state(h, x, v, stream=None):
    return _check(h.ptr, _lib.md_set_state(h.ptr, _ptr(x), _ptr(v), _stream(stream)))


def md_get_state(h, x, v, stream=None):
    return _check(h.ptr, _lib.md_get_state(h.ptr, _ptr(x), _ptr(v), _stream(stream)))


def md_build_neighbors(h, stream=None):
    return _check(h.ptr, _lib.md_build_neighbors(h.ptr, _stream(stream)))


def md_compute_forces(h, f_out=None, euw_out=None, stream=None):
    return _check(h.ptr, _lib.md_compute_forces(h.ptr, _ptr(f_out), _ptr(euw_out), _stream(stream)))


def md_step(h, nsteps, thermo_every=0, thermo_out=None, stream=None):
    return _check(h.ptr, _lib.md_step(h.ptr, int(nsteps), int(thermo_every), _ptr(thermo_out), _stream(stream)))


def md_forward(h, nsteps, ckpt_every, euw_out=None, stream=None):
    return _check(h.ptr, _lib.md_forward(h.ptr, int(nsteps), int(ckpt_every), _ptr(euw_out), _stream(stream)))


def md_backward(h, dL_dx, dL_dv, dL_deuw, dL_deps, dL_dsigma, stream=None):
    """md_backward: dL_dx, dL_dv ((3, N) or None) and dL_deuw ((R, 3) or None)
    in; dL_deps, dL_dsigma (R each) out."""
    return _check(h.ptr, _lib.md_backward(h.ptr, _ptr(dL_dx), _ptr(dL_dv), _ptr(dL_deuw), _ptr(dL_deps),
                                          _ptr(dL_dsigma), _stream(stream)))


def md_get_checkpoint(h, x, v, f, stream=None):
    """md_get_checkpoint: fills x, v, f ((3, N) each); returns the step counter."""
    step = C.c_int64(0)
    _check(h.ptr, _lib.md_get_checkpoint(h.ptr, _ptr(x), _ptr(v), _ptr(f), C.byref(step), _stream(stream)))
    return step.value


def md_set_checkpoint(h, x, v, f, step, stream=None):
    return _check(h.ptr, _lib.md_set_checkpoint(h.ptr, _ptr(x), _ptr(v), _ptr(f), int(step), _stream(stream)))


def md_set_recovery(h, enable=True):
    return _check(h.ptr, _lib.md_set_recovery(h.ptr, 1 if enable else 0))


def md_check_wait_timeout(h, polls=1000, stream=None):
    return _check(h.ptr, _lib.md_check_wait_timeout(h.ptr, int(polls), _stream(stream)))


def md_build_flags():
    return int(_lib.md_build_flags())


def md_check_bounds_selftest(h, site, stream=None):
    return _check(h.ptr, _lib.md_check_bounds_selftest(h.ptr, int(site), _stream(stream)))


def md_export_pairs(h, pairs_out, capacity, stream=None):
    n = C.c_int64(0)
    _check(h.ptr, _lib.md_export_pairs(h.ptr, _ptr(pairs_out), int(capacity), C.byref(n), _stream(stream)))
    return n.value


def md_autotune(h, trial_steps=20, stream=None):
    """md_autotune: returns the chosen tile size (particles per tile)."""
    out = C.c_int32(0)
    _check(h.ptr, _lib.md_autotune(h.ptr, int(trial_steps), C.byref(out), _stream(stream)))
    return out.value


def md_set_tile_size(h, tile_size, stream=None):
    return _check(h.ptr, _lib.md_set_tile_size(h.ptr, int(tile_size), _stream(stream)))


def md_set_half_list(h, enable=True, stream=None):
    """md_set_half_list: 1 = half list (Newton's third law), 0 = full list."""
    return _check(h.ptr, _lib.md_set_half_list(h.ptr, 1 if enable else 0, _stream(stream)))


def md_sync(h, stream=None):
    return _check(h.ptr, _lib.md_sync(h.ptr, _stream(stream)))


def md_get_stats(h, check=True):
    """md_get_stats as a dict; check=False returns the figures even when the
    call reports a latched device error (error_word, bad_site, bad_index)."""
    s = md_stats()
    st = _lib.md_get_stats(h.ptr, C.byref(s))
    if check:
        _check(h.ptr, st)
    return {f: (list(getattr(s, f)) if f == "ncell" else getattr(s, f)) for f, _ in md_stats._fields_}


def md_set_timing(h, enable=True):
    return _check(h.ptr, _lib.md_set_timing(h.ptr, 1 if enable else 0))


def md_get_timing(h):
    """(ms[MD_NSECT], counts[MD_NSECT]) accumulated since md_set_timing(h, True)."""
    ms = (C.c_double * MD_NSECT)()
    n = (C.c_int64 * MD_NSECT)()
    _check(h.ptr, _lib.md_get_timing(h.ptr, ms, n))
    return list(ms), list(n)


def md_compute_forces_noalloc(x, v, n, box, f_out, euw_out=None, eps=1.0, sigma=1.0, rc=2.5, shift=True,
                              precision=MD_FP32_FIXED, mass=1.0, stream=None):
    """md_compute_forces_noalloc: direct all-pairs forces for one system, no
    allocation (x, v, f_out, euw_out are device arrays; box is 3 host values)."""
    boxa = (C.c_double * 3)(*[float(t) for t in np.broadcast_to(np.asarray(box, dtype=np.float64), (3,))])
    buf = C.create_string_buffer(256)
    st = _lib.md_compute_forces_noalloc(_ptr(x), _ptr(v), int(n), boxa, float(eps), float(sigma), float(rc),
                                        1 if shift else 0, int(precision), float(mass), _ptr(f_out),
                                        _ptr(euw_out), buf, 256, _stream(stream))
    if st != MD_OK:
        raise MDError(st, buf.value.decode())
    return st


def md_probe_fp64_fma(iters=100000, blocks_per_sm=4, stream=None):
    """md_probe_fp64_fma (include/md_probe.h): measured FP64 FMA rate, returns (TFLOP/s, ms)."""
    tf, ms = C.c_double(0.0), C.c_double(0.0)
    st = _lib.md_probe_fp64_fma(int(iters), int(blocks_per_sm), C.byref(tf), C.byref(ms), _stream(stream))
    if st != 0:
        raise MDError(MD_ERR_CUDA if st == -2 else MD_ERR_ARG, "md_probe_fp64_fma failed")
    return tf.value, ms.value


def md_last_error(h):
    m = _lib.md_last_error(h.ptr)
    return m.decode() if m else ""


def export_pairs_sorted(h, stream=None):
    """All Verlet pairs (i < j) as an (M, 2) int32 array in lexicographic order."""
    n = md_export_pairs(h, None, 0, stream)
    out = np.zeros((max(n, 1), 2), dtype=np.int32)
    m = md_export_pairs(h, out, n, stream)
    assert m == n
    out = out[:n]
    order = np.lexsort((out[:, 1], out[:, 0]))
    return out[order]
