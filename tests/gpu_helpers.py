"""Helpers for the GPU parity tests."""
import numpy as np


def field_scale(ref):
    """Per-zone, per-field scale of the parity measure: |P_v| + max_grid |P_v| +
    floor_v.  The residual is normalised by the rest-mass scale (|U_0|), so the
    solver resolves velocities relative to c (floor 1) and the field-like
    primitives B^i, q~, dP~ (which enter T^{mu nu} through squares and
    products with rho-scaled terms) relative to sqrt(max rho); rho and u are
    relative to themselves."""
    ref = np.asarray(ref).reshape(10, -1)
    sr = np.sqrt(np.abs(ref[0]).max())
    floor = np.array([0, 0, 1, 1, 1, sr, sr, sr, sr, sr], dtype=float)[:, None]
    return np.abs(ref) + np.abs(ref).max(axis=1, keepdims=True) + floor + 1e-300


def rel_field_err(a, b):
    """max over zones of |a - b| / field_scale(b), per field."""
    a = np.asarray(a).reshape(10, -1)
    b = np.asarray(b).reshape(10, -1)
    return (np.abs(a - b) / field_scale(b)).max(axis=1)
