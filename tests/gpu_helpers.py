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


def learned_units(Pn):
    """Per field and zone, the unit of the learned start's targets: P_n for
    rho and u (relative change), |X_n| + rho_n for q~ and dP~, 1 for the
    velocities (Pn: [10, zones])."""
    Pn = np.asarray(Pn).reshape(10, -1)
    unit = np.ones_like(Pn)
    unit[0], unit[1] = Pn[0], Pn[1]
    unit[8] = np.abs(Pn[8]) + Pn[0]
    unit[9] = np.abs(Pn[9]) + Pn[0]
    return unit


def learned_pn_features(Pn):
    """The ten P_n features of the learned start, [zones, 10]."""
    Pn = np.asarray(Pn).reshape(10, -1)
    f = Pn.copy()
    f[0], f[1] = np.log(Pn[0]), np.log(Pn[1])
    f[8] = Pn[8] / (np.abs(Pn[8]) + Pn[0])
    f[9] = Pn[9] / (np.abs(Pn[9]) + Pn[0])
    return f.T
