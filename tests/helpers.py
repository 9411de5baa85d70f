"""Shared test helpers: error metrics and small input builders (no method arithmetic)."""
import numpy as np


def force_rel_err(F, F_ref):
    """max_i |F_i - F_ref_i| / max(|F_ref_i|, F_rms): a per-particle relative
    error that stays defined where a force is near zero (F_rms is the RMS
    force magnitude of the reference)."""
    F = np.asarray(F).reshape(-1, 3)
    F_ref = np.asarray(F_ref).reshape(-1, 3)
    mag = np.linalg.norm(F_ref, axis=1)
    rms = max(float(np.sqrt(np.mean(mag ** 2))), 1e-300)
    return float(np.max(np.linalg.norm(F - F_ref, axis=1) / np.maximum(mag, rms)))


def min_image_diff(a, b, box):
    d = np.asarray(a) - np.asarray(b)
    return d - box * np.round(d / box)
