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
