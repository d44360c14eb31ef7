"""Pins of the oracle's fast-magnetosonic speed bound with a magnetic field
(appendix on the characteristic structure, eq. fast_waves, with
a^2 = c_s^2 + c_a^2 - c_s^2 c_a^2) and of the Lax-Friedrichs speed window of
Sec. III C (reading A10: lambda at interface i+1/2 is the largest
max(|lambda^+|, |lambda^-|) over points i-2 .. i+3).

Nothing here re-types the oracle's speed formula.  The speeds are checked
against

* the eigenvalues of the flux Jacobian dF^d/dUbar, differentiated numerically
  through the oracle's own flux vectors (pinned against the covariant
  stress-energy tensor elsewhere) and its con2prim: the characteristic speeds
  of the system by definition.  For propagation perpendicular to the field,
  with the velocity along the propagation axis, the paper's bound is exact, so
  the largest |eigenvalue| must equal the oracle's lambda; for any other state
  it must not exceed it;
* a closed form derived independently: for perpendicular compression the
  field acts as an extra pressure b^2/2 with energy b^2/2 and b proportional
  to the rest-mass density, so v_f^2 = (c_s^2 h + b^2) / (h + b^2) in the fluid
  frame (h the enthalpy density), composed with the velocity by relativistic
  addition in the local Eulerian orthonormal frame, then mapped to
  coordinate speed with the lapse, the shift and sqrt(gamma^xx).
"""
import numpy as np
import pytest

import oracle
import synth

NF, NP = oracle.NF, oracle.NP
GAMMA = 2.0


def _sym(m):
    return np.array([m[0, 0], m[0, 1], m[0, 2], m[1, 1], m[1, 2], m[2, 2]])


def _state(O, g, alpha, beta, rho, eps, v, B):
    """Densitized conserved state (10) and the 32-field point for metric g (3x3),
    lapse alpha, shift beta, primitives (rho, eps, v^i) and field B^i."""
    det = np.linalg.det(g)
    chi = det ** (-1.0 / 3.0)
    gt = chi * g
    p = (GAMMA - 1.0) * rho * eps
    W = 1.0 / np.sqrt(1.0 - v @ g @ v)
    pr = np.zeros(NP)
    pr[0], pr[1], pr[2] = rho, eps, p
    pr[3:6] = v
    pr[6] = W
    pr[7] = 0.1
    cons = oracle.prim2con_point(pr, B, _sym(g))
    sg = np.sqrt(det)
    Ubar = np.zeros(10)
    Ubar[:9] = cons * sg
    U32 = np.zeros(NF)
    U32[0:6] = _sym(gt)
    U32[12] = chi
    U32[18] = alpha
    U32[19:22] = beta
    return Ubar, U32, _sym(gt), chi


def _flux(O, Ubar, U32, gt6, chi, alpha, d):
    st, prim, _, _ = O.c2p_point(Ubar, gt6, chi, alpha)
    assert st == 0, st
    U = U32.copy()
    U[22:32] = Ubar
    return O.flux_point(U, prim, d)


def _jacobian_speeds(O, Ubar, U32, gt6, chi, alpha, d):
    """Eigenvalues of dF^d/dUbar over the fluid and transverse-field variables
    (the divergence-cleaning pair B^d, phi is a separate subsystem with speeds
    +-c_b and is held fixed)."""
    idx = [0, 1, 2, 3, 4, 5] + [6 + a for a in range(3) if a != d]
    J = np.zeros((len(idx), len(idx)))
    for c, j in enumerate(idx):
        h = 1e-6 * max(abs(Ubar[j]), 1e-2 * Ubar[0])
        up, um = Ubar.copy(), Ubar.copy()
        up[j] += h
        um[j] -= h
        Fp, _ = _flux(O, up, U32, gt6, chi, alpha, d)
        Fm, _ = _flux(O, um, U32, gt6, chi, alpha, d)
        J[:, c] = (Fp[idx] - Fm[idx]) / (2 * h)
    return np.linalg.eigvals(J)


def _closed_form(g, alpha, beta, rho, eps, vx, By):
    """Coordinate fast speeds along x for v = (vx, 0, 0), B = (0, By, 0) and a
    diagonal metric: perpendicular fast speed in the fluid frame from the total
    pressure and energy, relativistic velocity addition in the Eulerian frame."""
    p = (GAMMA - 1.0) * rho * eps
    h = rho * (1.0 + eps) + p
    cs2 = GAMMA * p / h
    vhat = np.sqrt(g[0, 0]) * vx             # orthonormal Eulerian velocity
    W = 1.0 / np.sqrt(1.0 - vhat * vhat)
    Bhat = np.array([0.0, np.sqrt(g[1, 1]) * By, 0.0])
    u = W * np.array([1.0, vhat, 0.0, 0.0])
    b0 = W * Bhat[0] * vhat
    bsp = Bhat / W + b0 * u[1:] / W
    b2 = -b0 * b0 + bsp @ bsp
    vf = np.sqrt((cs2 * h + b2) / (h + b2))
    sp = [(vhat + vf) / (1 + vhat * vf), (vhat - vf) / (1 - vhat * vf)]
    return [alpha * s / np.sqrt(g[0, 0]) - beta[0] for s in sp]


CASES = [
    # (label, metric diag, alpha, beta, rho, eps, vx, By)
    ("rest_flat", (1.0, 1.0, 1.0), 1.0, (0.0, 0.0, 0.0), 1e-3, 0.2, 0.0, 0.03),
    ("boost_flat", (1.0, 1.0, 1.0), 1.0, (0.0, 0.0, 0.0), 1e-3, 0.2, 0.45, 0.03),
    ("boost_curved", (1.7, 0.8, 1.3), 0.7, (0.15, 0.0, 0.0), 2e-3, 0.1, -0.35, 0.05),
    ("strong_field", (1.2, 1.1, 0.9), 0.9, (-0.05, 0.0, 0.0), 1e-3, 0.05, 0.2, 0.2),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_perpendicular_fast_speed_equals_jacobian_and_closed_form(case):
    _, gd, alpha, beta, rho, eps, vx, By = case
    O = oracle.Oracle(synth.ideal_params())
    g = np.diag(gd)
    beta = np.array(beta)
    v = np.array([vx, 0.0, 0.0])
    B = np.array([0.0, By, 0.0])
    Ubar, U32, gt6, chi = _state(O, g, alpha, beta, rho, eps, v, B)
    F, lam = _flux(O, Ubar, U32, gt6, chi, alpha, 0)
    lp, lm = _closed_form(g, alpha, beta, rho, eps, vx, By)
    # The field matters: without it the speed is the plain sound speed.
    _, lam0 = _flux(O, *_state(O, g, alpha, beta, rho, eps, v, 0 * B)[:4], alpha, 0)
    assert lam > lam0 * 1.05
    assert abs(lam - max(abs(lp), abs(lm))) < 1e-12 * lam
    ev = _jacobian_speeds(O, Ubar, U32, gt6, chi, alpha, 0)
    assert np.max(np.abs(ev.imag)) < 1e-6 * lam
    assert abs(np.max(np.abs(ev.real)) - lam) < 1e-6 * lam
    # Both fast speeds are characteristic speeds of the system.
    for s in (lp, lm):
        assert np.min(np.abs(ev.real - s)) < 1e-6 * lam


def test_fast_speed_bounds_every_characteristic_speed():
    """Oblique fields, velocities off the axis and a full metric: the paper's
    degenerate-case bound must not be exceeded by any characteristic speed."""
    rng = np.random.default_rng(11)
    O = oracle.Oracle(synth.ideal_params())
    tight = 0
    for _ in range(12):
        Aq = rng.normal(size=(3, 3)) * 0.15
        g = np.eye(3) + 0.5 * (Aq + Aq.T)
        alpha = rng.uniform(0.6, 1.2)
        beta = rng.uniform(-0.2, 0.2, 3)
        rho, eps = 10 ** rng.uniform(-4, -2), rng.uniform(0.05, 0.5)
        v = rng.uniform(-0.3, 0.3, 3)
        B = rng.uniform(-1, 1, 3) * np.sqrt(rho) * rng.uniform(0.1, 1.5)
        Ubar, U32, gt6, chi = _state(O, g, alpha, beta, rho, eps, v, B)
        for d in range(3):
            _, lam = _flux(O, Ubar, U32, gt6, chi, alpha, d)
            ev = _jacobian_speeds(O, Ubar, U32, gt6, chi, alpha, d)
            top = np.max(np.abs(ev.real))
            assert top <= lam * (1 + 1e-6)
            tight += top > 0.9 * lam
    assert tight > 0  # the bound is not vacuous


def _window_patch(O, spike_at, factor, n0=16):
    """Periodic 16x4x4 patch of a fluid at rest (B = 0) whose density varies
    along x; at x index spike_at (on the line j = k = 0) the metric is
    diag(f, 1/f, 1), which leaves sqrt(gamma), the conserved variables and
    every x-flux unchanged but multiplies lambda^x there by 1/sqrt(f)."""
    n = (n0, 4, 4)
    shp = synth.patch_shape(n)
    rng = np.random.default_rng(3)
    rho_x = 1e-3 * (1 + 0.3 * rng.uniform(-1, 1, n0))
    U = np.zeros((NF,) + shp)
    U[0] = U[3] = U[5] = 1.0
    U[12] = 1.0
    U[18] = 1.0
    eps = 0.1
    for i in range(n0):
        pr = np.zeros(NP)
        rho = rho_x[i]
        pr[0], pr[1], pr[2] = rho, eps, (GAMMA - 1) * rho * eps
        pr[6] = 1.0
        pr[7] = 0.1
        cons = oracle.prim2con_point(pr, np.zeros(3), [1.0, 0, 0, 1.0, 0, 1.0])
        U[22:31, :, :, 3 + i] = cons[:, None, None]
    if spike_at is not None:
        U[0, 3, 3, 3 + spike_at] = factor
        U[3, 3, 3, 3 + spike_at] = 1.0 / factor
    O.ghost_fill(U, n)
    prim, status, _, _ = O.con2prim_patch(U, n)
    assert np.all(status == 0)
    return U, prim, n


def _rhs_d(O, U, prim, n, pts, driver):
    """D-bar right-hand side at interior points pts, through the sampled-point
    path or the patch driver (which precomputes the interface fluxes)."""
    if driver == "points":
        return O.rhs_points(U, prim, n, 0.1, pts)[:, 22]
    r = O.rhs_patch(U, prim, n, 0.1)
    return np.array([r[22, 3 + k, 3 + j, 3 + i] for i, j, k in pts])


@pytest.mark.parametrize("driver", ["points", "patch"])
def test_lf_speed_window_is_points_i_minus_2_to_i_plus_3(driver):
    """The D-bar right-hand side at point i (no source; flux difference only)
    changes when one point's lambda^x rises exactly when that point lies in
    i-3 .. i+3, the union of the windows of interfaces i-1/2 (i-3 .. i+2) and
    i+1/2 (i-2 .. i+3); a window shifted or narrowed by one point fails at
    one end."""
    O = oracle.Oracle(synth.ideal_params(bc=0))
    i = 8
    U, prim, n = _window_patch(O, None, 1.0)
    base = _rhs_d(O, U, prim, n, [[i, 0, 0]], driver)[0]
    for off in range(-5, 6):
        U, prim, n = _window_patch(O, i + off, 0.01)  # lambda^x 10x at one point
        # the spike leaves the point's x-flux and conserved state unchanged
        sp = i + off
        Us = U[:, 3, 3, 3 + sp].copy()
        pr = prim[:, 3, 3, 3 + sp].copy()
        Uf = Us.copy()
        Uf[0] = Uf[3] = 1.0  # the same point with the flat metric
        F1, lam1 = O.flux_point(Us, pr, 0)
        F0, lam0 = O.flux_point(Uf, pr, 0)
        assert np.allclose(F1, F0, rtol=1e-14, atol=1e-14 * np.abs(F0).max())
        assert abs(lam1 - 10 * lam0) < 1e-12 * lam1
        got = _rhs_d(O, U, prim, n, [[i, 0, 0]], driver)[0]
        if abs(off) <= 3:
            assert abs(got - base) > 1e-3 * abs(base), off
        else:
            assert got == base, off


@pytest.mark.parametrize("driver", ["points", "patch"])
def test_lf_speed_is_the_window_maximum_not_an_average(driver):
    """Lowering lambda at one point of a uniform-lambda background leaves every
    right-hand side unchanged: only the window's maximum enters."""
    O = oracle.Oracle(synth.ideal_params(bc=0))
    i = 8
    U, prim, n = _window_patch(O, None, 1.0)
    pts = [[m, 0, 0] for m in range(16)]
    base = _rhs_d(O, U, prim, n, pts, driver)
    for off in (-3, 0, 2):
        U, prim, n = _window_patch(O, i + off, 100.0)  # lambda^x / 10 at one point
        got = _rhs_d(O, U, prim, n, pts, driver)
        # rounding of p gamma^xx gamma_xx at the lowered point only
        assert np.abs(got - base).max() <= 1e-12 * np.abs(base).max(), off
