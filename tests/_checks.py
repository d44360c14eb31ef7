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


# Right-hand-side parity against the oracle's own rounding floor.
#
# The floor of a state is what the oracle itself changes when every input
# value is moved by one rounding step: the largest per-field difference
# between its right-hand side of U and of U (1 + 1e-16 xi), xi ~ U(-1, 1)
# independently per value, con2prim redone on the moved state (largest over
# two draws).  The GPU evaluates the same formulas with another operation
# order, so its difference from the oracle is of that size: over every field
# of the Fourier, TOV, hybrid-EOS and magnetised-star parity cases it measured
# 0.01-2.9 floors and at most 1.0e-12 of the field's largest right-hand side.
FLOOR_FACTOR = 10.0
RHS_TOL = 1e-11


def _perturbed(U, seed):
    rng = np.random.default_rng(1000 + seed)
    return U * (1.0 + 1e-16 * rng.uniform(-1.0, 1.0, U.shape))


def rhs_floor(O, U, n, dx, want=None, draws=2):
    """Per-field rounding floor of the oracle's interior right-hand side at
    state U (ghosts filled); want: the oracle's right-hand side of U if known."""
    if want is None:
        Uo = U.copy()
        prim, _, _, _ = O.con2prim_patch(Uo, n)
        want = interior(O.rhs_patch(Uo, prim, n, dx), n)
    fl = np.zeros(NF)
    for s in range(draws):
        Up = _perturbed(U, s)
        prim, _, _, _ = O.con2prim_patch(Up, n)
        r = interior(O.rhs_patch(Up, prim, n, dx), n)
        fl = np.maximum(fl, np.abs(r - want).reshape(NF, -1).max(axis=1))
    return fl


def rhs_floor_points(O, U, n, dx, ijk, want, draws=2):
    """The same floor for the right-hand side at sampled points ijk ([m][3])."""
    fl = np.zeros(NF)
    for s in range(draws):
        Up = _perturbed(U, s)
        prim, _, _, _ = O.con2prim_patch(Up, n)
        r = O.rhs_points(Up, prim, n, dx, ijk).T
        fl = np.maximum(fl, np.abs(r - want).reshape(NF, -1).max(axis=1))
    return fl


def rhs_check(got, want, floor, tol=RHS_TOL, factor=FLOOR_FACTOR):
    """Right-hand side parity per field (arrays [32][...]):
    max |gpu - oracle| <= max(tol max |oracle|, factor floor).
    Returns (ok, report); report gives, for every field that fails, the error
    relative to the field's largest right-hand side and in units of the floor."""
    want_n = np.abs(want).reshape(NF, -1).max(axis=1)
    d = np.abs(got - want).reshape(NF, -1).max(axis=1)
    ok = d <= np.maximum(tol * want_n, factor * floor)
    rel = d / np.maximum(want_n, 1e-300)
    flr = d / np.maximum(floor, 1e-300)
    return bool(np.all(ok)), {f: dict(err_rel=rel[f], err_over_floor=flr[f], rhs=want_n[f])
                              for f in range(NF) if not ok[f]}


def rhs_report(got, want, floor):
    """Largest error relative to max |RHS| and in floors, over all fields."""
    want_n = np.abs(want).reshape(NF, -1).max(axis=1)
    d = np.abs(got - want).reshape(NF, -1).max(axis=1)
    return float((d / np.maximum(want_n, 1e-300)).max()), float((d / np.maximum(floor, 1e-300)).max())
