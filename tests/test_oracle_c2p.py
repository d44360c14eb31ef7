"""Pins of the oracle's prim2con, con2prim (Kastaun/Brent) and error policy.

Definitions: Sec. II B, eq. def_con2prim.  Recovery: the appendix
"Conversion from conserved to primitive fields" (steps 1-4 and the error
policy).  Pins: closed forms of the conserved variables in special cases, an
independent textbook recovery for B = 0 (1-D root find on the pressure), the
prim -> cons -> prim round trip, the uniqueness of the master function's root
by brute-force scans, and one crafted state per policy branch.
"""
import numpy as np
import pytest
from scipy.optimize import brentq

import oracle
import synth

NP = oracle.NP
GT_FLAT = np.array([1.0, 0, 0, 1.0, 0, 1.0])


def _prim(rho, eps, p, v, ye=0.1, T=0.0):
    pr = np.zeros(NP)
    pr[0], pr[1], pr[2] = rho, eps, p
    pr[3:6] = v
    pr[7] = ye
    pr[8] = T
    return pr


def _metric(rng, amp=0.1):
    """A random positive-definite gamma_ij and its conformal split (gt, chi)."""
    M = np.eye(3) + amp * rng.normal(size=(3, 3))
    g = M @ M.T
    det = np.linalg.det(g)
    chi = det ** (-1.0 / 3.0)
    gt = chi * g
    s = lambda A: np.array([A[0, 0], A[0, 1], A[0, 2], A[1, 1], A[1, 2], A[2, 2]])
    return s(g), s(gt), chi, np.sqrt(det), g


def test_prim2con_closed_forms():
    g = GT_FLAT
    # At rest, no field: D = rho, tau = rho eps, S = 0.
    c = oracle.prim2con_point(_prim(2e-3, 0.3, 6e-4, [0, 0, 0]), [0, 0, 0], g)
    assert c[0] == 2e-3 and abs(c[2] - 2e-3 * 0.3) < 1e-18 and np.all(c[3:6] == 0)
    # At rest with a field: tau = rho eps + B^2 / 2.
    c = oracle.prim2con_point(_prim(2e-3, 0.3, 6e-4, [0, 0, 0]), [0.01, 0.02, 0], g)
    assert abs(c[2] - (2e-3 * 0.3 + 0.5 * 5e-4)) < 1e-17
    # Moving along x, no field: S_x = rho h W^2 v with h the specific enthalpy.
    rho, eps, p, v = 1e-3, 0.2, 2e-4, 0.6
    W2 = 1.0 / (1 - v * v)
    hs = 1 + eps + p / rho
    c = oracle.prim2con_point(_prim(rho, eps, p, [v, 0, 0]), [0, 0, 0], g)
    assert abs(c[3] - rho * hs * W2 * v) < 1e-15 * c[3]
    assert abs(c[0] - rho * np.sqrt(W2)) < 1e-18
    assert abs(c[2] - (rho * hs * W2 - p - rho * np.sqrt(W2))) < 1e-15


def test_prim2con_matches_covariant_stress_energy():
    """tau + D = T^{00} (alpha = 1) and S_i = T^0_i with the MHD T^{ab} built from b^mu (flat space)."""
    rng = np.random.default_rng(1)
    for _ in range(20):
        rho, eps = 10 ** rng.uniform(-4, -2), rng.uniform(0.05, 1.0)
        p = (2 - 1) * rho * eps
        v = rng.uniform(-0.4, 0.4, 3)
        B = rng.uniform(-0.05, 0.05, 3)
        W = 1 / np.sqrt(1 - v @ v)
        u = np.concatenate([[W], W * v])
        b0 = W * (B @ v)
        b = np.concatenate([[b0], (B + b0 * u[1:]) / W])
        eta = np.diag([-1.0, 1, 1, 1])
        b2 = b @ eta @ b
        hh = rho * (1 + eps) + p
        Tuu = (hh + b2) * np.outer(u, u) + (p + b2 / 2) * np.linalg.inv(eta) - np.outer(b, b)
        c = oracle.prim2con_point(_prim(rho, eps, p, v), B, GT_FLAT)
        assert abs((c[2] + c[0]) - Tuu[0, 0]) < 1e-13 * Tuu[0, 0]
        assert np.allclose(c[3:6], Tuu[0, 1:], rtol=1e-12, atol=1e-16)
        assert abs(c[0] - rho * W) < 1e-16


def _cons_bar(pr, B, gdd, sg):
    c = oracle.prim2con_point(pr, B, gdd)
    cb = np.zeros(10)
    cb[:9] = c * sg
    return cb


def test_round_trip_ideal_gas_to_1e12():
    P = synth.ideal_params()
    O = oracle.Oracle(P)
    rng = np.random.default_rng(2)
    for _ in range(300):
        gdd, gt, chi, sg, _g = _metric(rng)
        rho = 10 ** rng.uniform(-5, -2)
        eps = 10 ** rng.uniform(-2, 0)
        p = rho * eps
        v = rng.uniform(-0.3, 0.3, 3)
        gm = _g
        while v @ gm @ v > 0.6:
            v *= 0.5
        B = rng.uniform(-1, 1, 3) * np.sqrt(rho) * rng.uniform(0, 1)
        pr = _prim(rho, eps, p, v)
        st, out, co, it = O.c2p_point(_cons_bar(pr, B, gdd, sg), gt, chi, 1.0)
        assert st == 0, st
        assert abs(out[0] - rho) < 1e-12 * rho
        assert abs(out[1] - eps) < 1e-12 * max(1.0, 1.0 / eps)
        assert np.all(np.abs(out[3:6] - v) < 1e-12)
        assert abs(out[6] - 1 / np.sqrt(1 - v @ gm @ v)) < 1e-12
        assert it < 60


def test_b_zero_at_rest_mu_closed_form():
    # B = 0, v = 0: q = eps and the recovered state is exact: rho = D, eps = tau / D.
    O = oracle.Oracle(synth.ideal_params())
    rho, eps = 1.7e-3, 0.37
    cb = np.zeros(10)
    cb[0], cb[1], cb[2] = rho, 0.1 * rho, rho * eps
    st, out, co, it = O.c2p_point(cb, GT_FLAT, 1.0, 1.0)
    assert st == 0 and out[0] == rho and abs(out[1] - eps) < 4e-16 and np.all(out[3:6] == 0)


def test_b_zero_against_pressure_rootfind():
    """Independent textbook recovery (B = 0, ideal gas): solve for p in one dimension."""
    O = oracle.Oracle(synth.ideal_params())
    G = 2.0
    rng = np.random.default_rng(3)
    for _ in range(100):
        D = 10 ** rng.uniform(-5, -2)
        S = rng.uniform(0, 1) * D * np.array([0.6, -0.3, 0.2])
        tau = D * rng.uniform(0.05, 1.0) + 0.5 * (S @ S) / D
        E = tau + D

        def resid(p):
            v = np.sqrt(S @ S) / (E + p)
            W = 1 / np.sqrt(1 - v * v)
            rho = D / W
            eps = (E + p) / (D * W) - 1 - p / rho
            return p - (G - 1) * rho * eps

        p = brentq(resid, 1e-30, 10 * E, xtol=1e-300, rtol=1e-15)
        v = S / (E + p)
        W = 1 / np.sqrt(1 - v @ v)
        cb = np.zeros(10)
        cb[0], cb[1], cb[2], cb[3:6] = D, 0.1 * D, tau, S
        st, out, co, it = O.c2p_point(cb, GT_FLAT, 1.0, 1.0)
        assert st == 0
        assert abs(out[2] - p) < 1e-11 * p
        assert np.allclose(out[3:6], v, rtol=1e-11, atol=1e-14)
        assert abs(out[0] - D / W) < 1e-12 * D


@pytest.fixture(scope="module")
def table():
    return synth.make_table(nr=64, nt=48, ny=16)


def test_table_nodes_reproduce_model(table):
    from synth.eos_table import model
    O = oracle.Oracle(synth.table_params(table), table)
    for (ir, it, iy) in [(0, 0, 0), (10, 20, 5), (63, 47, 15), (31, 7, 3)]:
        rho = 10 ** (table["lr0"] + ir * table["dlr"])
        T = 10 ** (table["lt0"] + it * table["dlt"])
        ye = table["ye0"] + iy * table["dye"]
        p, eps, cs2 = model(rho, T, ye)
        out = O.eos_from_T(rho, T, ye)
        assert abs(out[0] - p) < 1e-12 * p and abs(out[1] - eps) < 1e-12 * eps and abs(out[3] - cs2) < 1e-12
        # T inversion then forward evaluation reproduces eps (and T at a node).
        inv = O.eos_from_eps(rho, eps, ye)
        assert abs(inv[1] - eps) <= 4e-16 * eps and abs(inv[2] - T) < 1e-9 * T


def test_table_round_trip_kappa_scaled(table):
    P = synth.table_params(table)
    O = oracle.Oracle(P, table)
    st = synth.c2p_states(2000, seed=7)
    bad = 0
    for q in range(2000):
        rho, T, ye = st["rho"][q], st["T"][q], st["ye"][q]
        pe = O.eos_from_T(rho, T, ye)
        pr = _prim(rho, pe[1], pe[0], st["v"][q], ye=ye)
        cb = _cons_bar(pr, st["B"][q], GT_FLAT, 1.0)
        s, out, co, it = O.c2p_point(cb, GT_FLAT, 1.0, 1.0)
        assert s >= 0
        if s != 0:
            continue
        W = 1 / np.sqrt(1 - st["v"][q] @ st["v"][q])
        q_ = cb[2] / cb[0]
        kap = max(1.0, (1 + q_) / abs(pe[1]))
        ok = (abs(out[0] - rho) <= 1e-10 * rho and abs(out[7] - ye) <= 1e-12
              and np.all(np.abs(out[3:6] * out[6] - st["v"][q] * W) <= 1e-10 * W)
              and abs(out[1] - pe[1]) <= 1e-10 * kap * abs(pe[1]))
        bad += not ok
    assert bad == 0


@pytest.mark.parametrize("kind", ["ideal", "table"])
@pytest.mark.parametrize("tau_scale", [False, True])
def test_master_function_root_is_unique(kind, tau_scale, table):
    """Kastaun et al. prove that the master function changes sign exactly once
    on (0, mu_+].  Brute force: 1000 states x 1000 values of mu.  Physical
    states from prim2con, and the same states with tau scaled by U(0, 2)
    (eps clamps and the velocity bound active).  Where tau is below the
    kinetic energy the velocity bound v_0 makes f(mu_+) = 0 analytically and
    rounding may leave it a few ulps negative: no sign change then, and the
    root is mu_+ itself.  The solver's root lies in the sign-change cell."""
    n_mu = 1000
    if kind == "ideal":
        P = synth.ideal_params()
        O = oracle.Oracle(P)
        rng = np.random.default_rng(11)
        states = []
        for _ in range(1000):
            rho, eps = 10 ** rng.uniform(-8, -2), 10 ** rng.uniform(-3, 1)
            v = rng.normal(size=3)
            v *= rng.uniform(0, 0.995) / np.linalg.norm(v)
            B = rng.normal(size=3) * np.sqrt(rho) * 10 ** rng.uniform(-2, 1)
            states.append(_cons_bar(_prim(rho, eps, rho * eps, v), B, GT_FLAT, 1.0))
    else:
        P = synth.table_params(table)
        O = oracle.Oracle(P, table)
        st = synth.c2p_states(1000, seed=17)
        states = []
        for q in range(1000):
            pe = O.eos_from_T(st["rho"][q], st["T"][q], st["ye"][q])
            pr = _prim(st["rho"][q], pe[1], pe[0], st["v"][q], ye=st["ye"][q])
            states.append(_cons_bar(pr, st["B"][q], GT_FLAT, 1.0))
    cons = np.array(states)
    if tau_scale:
        cons[:, 2] *= np.random.default_rng(5).uniform(0.0, 2.0, len(cons))
    _, status, _, roots, _ = O.c2p_flat_ext(cons)
    endpoint = 0
    for q in range(len(cons)):
        mu_plus, f = O.c2p_master_scan(cons[q], n_mu)
        assert mu_plus > 0 and mu_plus == roots[q, 0]
        assert f[0] < 0
        up = np.nonzero((f[:-1] < 0) & (f[1:] >= 0))[0]
        down = np.nonzero((f[:-1] >= 0) & (f[1:] < 0))[0]
        assert len(down) == 0
        mu = roots[q, 1]
        if f[-1] < 0:
            assert len(up) == 0 and -f[-1] <= 1e-15 * mu_plus and mu == mu_plus
            endpoint += 1
            continue
        assert len(up) <= 1
        k = up[0] + 1 if len(up) else 0  # first grid index with f >= 0
        lo, hi = mu_plus * k / n_mu, mu_plus * (k + 1) / n_mu
        assert lo * (1 - 1e-12) <= mu <= hi * (1 + 1e-12)
    if not tau_scale:
        assert endpoint == 0 and np.all(status == 0)


# ---- error policy -----------------------------------------------------------

def _state(O, rho, eps, v, B=(0, 0, 0), ye=0.1, alpha=1.0):
    pr = _prim(rho, eps, rho * eps, np.array(v, float), ye=ye)
    cb = _cons_bar(pr, np.array(B, float), GT_FLAT, 1.0)
    return O.c2p_point(cb, GT_FLAT, 1.0, alpha)


def test_policy_atmosphere():
    P = synth.ideal_params()
    O = oracle.Oracle(P)
    st, out, co, it = _state(O, 1e-12, 0.1, [0.3, 0, 0])
    assert st == 1 and out[0] == P["rho_atmo"] and np.all(out[3:6] == 0) and out[6] == 1.0
    assert abs(out[2] - P["K_atmo"] * P["rho_atmo"] ** 2) < 1e-30
    # Conserved variables rewritten from the atmosphere state.
    assert co[0] == P["rho_atmo"] and np.all(co[3:6] == 0)


def test_policy_rho_max_fatal():
    O = oracle.Oracle(synth.ideal_params(rho_max=1e-3))
    assert _state(O, 2e-3, 0.1, [0, 0, 0])[0] == -1


def test_policy_eps_max():
    # Dense: fatal.  Low density (rho < rho_low) or inside a BH (alpha < alpha_bh): clamp.
    O = oracle.Oracle(synth.ideal_params(eps_max=0.05))
    assert _state(O, 1e-3, 0.1, [0, 0, 0])[0] == -2
    st, out, _, _ = _state(O, 1e-3, 0.1, [0, 0, 0], alpha=0.1)
    assert st == 2 and out[1] == 0.05
    st, out, _, _ = _state(O, 1e-9, 0.1, [0, 0, 0])
    assert st == 2 and out[1] == 0.05


def test_policy_eps_min_clamp():
    O = oracle.Oracle(synth.ideal_params())
    cb = np.zeros(10)
    cb[0], cb[1], cb[2] = 1e-3, 1e-4, -1e-6  # tau < 0 at rest: eps < 0 = eps_min
    st, out, co, it = O.c2p_point(cb, GT_FLAT, 1.0, 1.0)
    assert st == 2 and out[1] == 0.0 and co[2] == 0.0


def test_policy_velocity_limit():
    P = synth.ideal_params(W_max=5.0)
    O = oracle.Oracle(P)
    v = [np.sqrt(1 - 1 / 8.0 ** 2), 0, 0]  # W = 8 > W_max
    assert _state(O, 1e-3, 0.1, v)[0] == -3
    st, out, co, it = _state(O, 1e-9, 0.1, v)
    assert st == 4 and abs(out[6] - 5.0) < 1e-15
    assert abs(np.sqrt(out[3] ** 2) - np.sqrt(1 - 1 / 25.0)) < 1e-13
    D = co[0]
    assert abs(out[0] - D / 5.0) < 1e-24  # D kept fixed, rho = D / W_max


def test_policy_ye():
    O = oracle.Oracle(synth.ideal_params())
    assert _state(O, 1e-3, 0.1, [0, 0, 0], ye=0.9)[0] == -4
    st, out, _, _ = _state(O, 1e-9, 0.1, [0, 0, 0], ye=0.9)
    assert st == 8 and out[7] == synth.ideal_params()["ye_atmo"]


def test_policy_nonfinite():
    O = oracle.Oracle(synth.ideal_params())
    cb = np.zeros(10)
    cb[0], cb[1], cb[2] = np.nan, 1e-5, 1e-4
    assert O.c2p_point(cb, GT_FLAT, 1.0, 1.0)[0] == -5
