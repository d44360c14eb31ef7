"""Shared tolerance checks of the GPU parity tests."""
import numpy as np


def prim_check(gp, op, gst, ost, cons):
    """Primitives (field-major [10][n]) of the GPU against the oracle at the
    stated bounds: statuses bit-exact; on points both solved cleanly rho and Ye
    to 1e-10 relative, W v^i to 1e-10 absolute, eps and p to 1e-10 relative
    scaled by max(1, (1 + |q|) / |eps|) with q = tau / D."""
    ok = (gst == 0) & (ost == 0)
    assert np.array_equal(gst, ost)
    rho_g, rho_o = gp[0][ok], op[0][ok]
    assert np.all(np.abs(rho_g - rho_o) <= 1e-10 * rho_o)
    assert np.all(np.abs(gp[7][ok] - op[7][ok]) <= 1e-10 * np.abs(op[7][ok]))
    wv_g = gp[3:6][:, ok] * gp[6][ok]
    wv_o = op[3:6][:, ok] * op[6][ok]
    assert np.all(np.abs(wv_g - wv_o) <= 1e-10)
    q = cons[2][ok] / cons[0][ok]
    kap = np.maximum(1.0, (1.0 + np.abs(q)) / np.maximum(np.abs(op[1][ok]), 1e-300))
    assert np.all(np.abs(gp[1][ok] - op[1][ok]) <= 1e-10 * kap * np.abs(op[1][ok]) + 1e-300)
    assert np.all(np.abs(gp[2][ok] - op[2][ok]) <= 1e-10 * kap * np.abs(op[2][ok]) + 1e-300)


NF = 32


def interior(a, n):
    return a[:, 3:3 + n[2], 3:3 + n[1], 3:3 + n[0]]


def field_err(got, want):
    gg = got.reshape(got.shape[0], -1)
    ww = want.reshape(want.shape[0], -1)
    scale = np.maximum(np.abs(ww).max(axis=1), 1e-30)
    return np.abs(gg - ww).max(axis=1) / scale


def init_ok(Ug, U, dx=None):
    """Initial-data conversion: 1e-13 per field.  Gammahat (fields 15-17) is a
    centred derivative of gt_ij = O(1): its rounding is absolute, ~eps / dx
    (times the extrapolation factor in the ghosts), so it is held to 1e-13 / dx
    absolute (or 1e-10 relative when dx is not given)."""
    e = field_err(Ug, U)
    tol = np.full(NF, 1e-13)
    tol[15:18] = 1e-10
    d = np.abs(Ug - U).reshape(NF, -1).max(axis=1)
    small = np.abs(U).reshape(NF, -1).max(axis=1) < 1e-12
    ok = (e < tol) | (small & (d < 1e-13))
    if dx is not None:
        ok[15:18] |= d[15:18] < 1e-13 / dx
    return bool(np.all(ok)), {f: e[f] for f in range(NF) if not ok[f]}
