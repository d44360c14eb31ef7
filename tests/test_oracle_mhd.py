"""Pins of the oracle's ideal-MHD right-hand side (Sec. II B eq. mhd_system,
Sec. III C flux splitting / MP5 / LLF2, fast-speed bound eq. fast_waves) and of
the matter coupling to CCZ4 (static TOV star)."""
import numpy as np
import pytest

import oracle
import synth

NF, NP = oracle.NF, oracle.NP


def test_fast_speed_reduces_to_sr_sound_speed():
    for v in (-0.7, -0.2, 0.0, 0.3, 0.9):
        for cs2 in (0.05, 0.2, 1 / 3.0):
            cs = np.sqrt(cs2)
            lp, lm = oracle.fast_speeds(1.0, 0.0, 1.0, v, v * v, cs2)
            assert abs(lp - (v + cs) / (1 + v * cs)) < 1e-15
            assert abs(lm - (v - cs) / (1 - v * cs)) < 1e-15


def test_fast_speed_at_rest_with_lapse_and_shift():
    a2, al, be, gxx = 0.3, 0.8, 0.1, 1.7
    lp, lm = oracle.fast_speeds(al, be, gxx, 0.0, 0.0, a2)
    assert abs(lp - (-be + al * np.sqrt(a2 * gxx))) < 1e-15
    assert abs(lm - (-be - al * np.sqrt(a2 * gxx))) < 1e-15


def _point(rho, eps, v, B, gamma=2.0):
    """32-field state and primitives at one flat-space point (alpha = 1, beta = 0)."""
    U = np.zeros(NF)
    U[0] = U[3] = U[5] = 1.0
    U[12] = 1.0
    U[18] = 1.0
    p = (gamma - 1) * rho * eps
    pr = np.zeros(NP)
    pr[0], pr[1], pr[2] = rho, eps, p
    pr[3:6] = v
    W = 1 / np.sqrt(1 - np.dot(v, v))
    pr[6] = W
    pr[7] = 0.1
    h = rho * (1 + eps) + p
    pr[9] = gamma * p / h
    cons = oracle.prim2con_point(pr, B, [1.0, 0, 0, 1.0, 0, 1.0])
    U[22:31] = cons
    return U, pr


def test_stress_at_rest_is_maxwell_stress():
    B = np.array([0.01, -0.02, 0.015])
    U, pr = _point(1e-3, 0.1, np.zeros(3), B)
    E, S, Sij = oracle.matter_point(U, pr)
    p = pr[2]
    B2 = B @ B
    full = p * np.eye(3) - np.outer(B, B) + 0.5 * np.eye(3) * B2
    want = np.array([full[0, 0], full[0, 1], full[0, 2], full[1, 1], full[1, 2], full[2, 2]])
    assert np.allclose(Sij, want, rtol=1e-14, atol=1e-20)
    assert abs(E - (1e-3 * 1.1 + 0.5 * B2)) < 1e-17


def test_flux_matches_covariant_stress_energy_flat_space():
    rng = np.random.default_rng(4)
    P = synth.ideal_params()
    O = oracle.Oracle(P)
    for _ in range(20):
        rho, eps = 10 ** rng.uniform(-4, -2), rng.uniform(0.05, 1.0)
        v = rng.uniform(-0.4, 0.4, 3)
        B = rng.uniform(-0.05, 0.05, 3)
        U, pr = _point(rho, eps, v, B)
        W = pr[6]
        p = pr[2]
        u = np.concatenate([[W], W * v])
        b0 = W * (B @ v)
        b = np.concatenate([[b0], (B + b0 * u[1:]) / W])
        eta = np.diag([-1.0, 1, 1, 1])
        b2 = b @ eta @ b
        hh = rho * (1 + eps) + p
        Tuu = (hh + b2) * np.outer(u, u) + (p + b2 / 2) * np.linalg.inv(eta) - np.outer(b, b)
        for d in range(3):
            F, lam = O.flux_point(U, pr, d)
            D = rho * W
            assert abs(F[0] - D * v[d]) < 1e-15 * D
            assert abs(F[2] - (Tuu[0, d + 1] - D * v[d])) < 1e-13 * Tuu[0, 0]
            assert np.allclose(F[3:6], Tuu[d + 1, 1:], rtol=1e-12, atol=1e-15 * Tuu[0, 0])
            induction = B * v[d] - B[d] * v
            assert np.allclose(F[6:9], induction, rtol=1e-12, atol=1e-18)
            assert abs(F[9] - P["c_b"] ** 2 * B[d]) < 1e-18


def test_flux_matches_covariant_stress_energy_curved():
    # Lapse, shift and a non-diagonal 3-metric: the conservative fluxes along
    # d are sqrt(-g) times the d-components of the four-dimensional currents,
    # with sqrt(-g) = alpha sqrt(gamma): rho u^d for D, T^d_i for S_i,
    # alpha T^{0 d} - rho u^d for tau, and -*F^{d i} = b^i u^d - b^d u^i
    # (the dual Faraday tensor) for B^i, all built here from u^mu and b^mu.
    rng = np.random.default_rng(7)
    P = synth.ideal_params()
    O = oracle.Oracle(P)
    six = lambda M: np.array([M[0, 0], M[0, 1], M[0, 2], M[1, 1], M[1, 2], M[2, 2]])
    for _ in range(20):
        A = rng.uniform(-0.15, 0.15, (3, 3))
        g = np.eye(3) + 0.5 * (A + A.T)
        al = rng.uniform(0.6, 1.2)
        be = rng.uniform(-0.2, 0.2, 3)
        rho, eps, ye = 10 ** rng.uniform(-4, -2), rng.uniform(0.05, 1.0), 0.1
        v = rng.uniform(-0.3, 0.3, 3)
        B = rng.uniform(-0.05, 0.05, 3)
        sg = np.sqrt(np.linalg.det(g))
        chi = np.linalg.det(g) ** (-1.0 / 3.0)
        p = (P["gamma_th"] - 1.0) * rho * eps
        W = 1.0 / np.sqrt(1.0 - v @ g @ v)
        pr = np.zeros(NP)
        pr[0], pr[1], pr[2], pr[3:6], pr[6], pr[7] = rho, eps, p, v, W, ye
        pr[9] = P["gamma_th"] * p / (rho * (1 + eps) + p)
        U = np.zeros(NF)
        U[0:6] = six(chi * g)
        U[12] = chi
        U[18] = al
        U[19:22] = be
        U[22:31] = np.asarray(oracle.prim2con_point(pr, B, six(g))) * sg
        # Four-dimensional quantities.
        g4 = np.zeros((4, 4))
        bl = g @ be
        g4[0, 0] = -al * al + be @ bl
        g4[0, 1:] = g4[1:, 0] = bl
        g4[1:, 1:] = g
        u = np.concatenate([[W / al], W * (v - be / al)])
        b0 = W * (B @ g @ v) / al
        b = np.concatenate([[b0], (B + al * b0 * u[1:]) / W])
        b2 = b @ g4 @ b
        T = (rho * (1 + eps) + p + b2) * np.outer(u, u) + (p + 0.5 * b2) * np.linalg.inv(g4) - np.outer(b, b)
        Tmix = T @ g4  # T^mu_nu
        sqg = al * sg
        for d in range(3):
            F, lam = O.flux_point(U, pr, d)
            k = d + 1
            scale = sqg * abs(T[0, 0])
            assert abs(F[0] - sqg * rho * u[k]) < 1e-13 * sqg * rho * W
            assert abs(F[1] - sqg * rho * ye * u[k]) < 1e-13 * sqg * rho * W
            assert abs(F[2] - sqg * (al * T[0, k] - rho * u[k])) < 1e-12 * scale
            assert np.allclose(F[3:6], sqg * Tmix[k, 1:], rtol=1e-11, atol=1e-13 * scale)
            induction = sqg * (b[1:] * u[k] - b[k] * u[1:])
            assert np.allclose(F[6:9], induction, rtol=1e-11, atol=1e-14 * np.abs(B).max())


def _uniform_patch(O, n, v, B, rho=1e-3, eps=0.1, dx=0.1):
    shp = synth.patch_shape(n)
    ID = np.zeros((26,) + shp)
    ID[0] = ID[3] = ID[5] = 1.0
    ID[12] = 1.0
    ID[16], ID[17] = rho, eps
    ID[18:21] = np.array(v)[:, None, None, None]
    ID[21:24] = np.array(B)[:, None, None, None]
    ID[24] = 0.1
    U = O.init_state(ID, n, dx)
    return U


def test_uniform_state_flat_space_gives_exact_zero():
    O = oracle.Oracle(synth.ideal_params(bc=0))
    n = (6, 6, 6)
    U = _uniform_patch(O, n, [0.2, -0.1, 0.05], [0.01, 0.02, -0.01])
    prim, st, worst, its = O.con2prim_patch(U, n)
    rhs = O.rhs_patch(U, prim, n, 0.1)
    assert np.all(rhs[22:, 3:-3, 3:-3, 3:-3] == 0.0)


def test_periodic_telescoping_of_dbar():
    n = (12, 12, 12)
    O = oracle.Oracle(synth.ideal_params(bc=0))
    ID = synth.config0_id(n=n, seed=11)
    U = O.init_state(ID, n, 1.0 / 12)
    prim, st, worst, its = O.con2prim_patch(U, n)
    rhs = O.rhs_patch(U, prim, n, 1.0 / 12)
    for f in (22, 23):
        r = rhs[f, 3:-3, 3:-3, 3:-3]
        assert abs(r.sum()) < 1e-13 * np.abs(r).sum()


def test_smooth_advection_converges():
    errs = []
    for N in (16, 32, 64):
        n = (N, 4, 4)
        dx = 1.0 / N
        O = oracle.Oracle(synth.ideal_params(bc=0))
        shp = synth.patch_shape(n)
        zz, yy, xx = synth.grid_coords(n, (0, 0, 0), dx)
        xx = np.broadcast_to(xx, shp)
        ID = np.zeros((26,) + shp)
        ID[0] = ID[3] = ID[5] = 1.0
        ID[12] = 1.0
        rho = 1e-3 * (1 + 0.1 * np.sin(2 * np.pi * xx))
        p0 = 1e-4
        ID[16] = rho
        ID[17] = p0 / rho  # uniform pressure (Gamma = 2): a pure contact wave
        ID[18] = 0.3
        ID[24] = 0.1
        U = O.init_state(ID, n, dx)
        prim, st, worst, its = O.con2prim_patch(U, n)
        rhs = O.rhs_patch(U, prim, n, dx)
        W = 1 / np.sqrt(1 - 0.09)
        exact = -0.3 * W * 1e-3 * 0.1 * 2 * np.pi * np.cos(2 * np.pi * xx)
        e = rhs[22, 3:-3, 3:-3, 3:-3] - exact[3:-3, 3:-3, 3:-3]
        errs.append(np.abs(e).mean())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > 3.5, (errs, rates)


# ---- static TOV star --------------------------------------------------------

@pytest.fixture(scope="module")
def tov():
    return synth.tov_profile()


def _tov_rhs(prof, center, dx, n=8):
    P = synth.ideal_params(bc=1)
    O = oracle.Oracle(P)
    nn = (n, n, n)
    x0 = [c - (n // 2) * dx for c in center]
    ID = synth.tov_id(n=nn, x0=x0, dx=dx, perturb=False, bfield=False, profile=prof)
    U = O.init_state(ID, nn, dx)
    prim, st, worst, its = O.con2prim_patch(U, nn)
    assert worst == 0
    rhs = O.rhs_patch(U, prim, nn, dx)
    c = n // 2 + 3
    return rhs[:, c, c, c], U[:, c, c, c]


def test_static_tov_interior_rhs_converges_to_zero(tov):
    center = (2.0, 2.5, 3.0)
    r1, U1 = _tov_rhs(tov, center, 0.2)
    r2, U2 = _tov_rhs(tov, center, 0.1)
    # Exact zeros: no velocity and no field -> Dbar, DYebar, taubar, Bbar, phibar fluxes vanish
    # up to the Lax-Friedrichs dissipation of MP5 (5th order); S_i balances gravity.
    # Fields whose coarse value is at the rounding floor (gt_ij through ln det gt,
    # Gammahat and beta through Gt ~ 0 of a conformally flat metric) are excluded.
    scale = np.abs(r1).max()
    fields = [f for f in range(NF) if abs(r1[f]) > 1e-5 * scale]
    assert len(fields) >= 16
    rate = np.log2(np.abs(r1[fields]) / np.maximum(np.abs(r2[fields]), 1e-300))
    assert np.all(rate > 3.3), dict(zip(fields, rate))
    # Hydrostatic balance: the momentum RHS at dx = 0.1 is tiny against the gravity source.
    grav = (U1[24] + U1[22]) * 0.05  # (taubar + Dbar) |d alpha|, alpha' ~ 0.05 at r ~ 4.4
    assert np.abs(r2[25:28]).max() < 1e-3 * grav


def test_divergence_cleaning_terms_closed_form():
    """Divergence cleaning of the MHD system (Sec. II B, eq. mhd_system, the
    phibar and Bbar^i equations) on a fluid at rest with uniform B and phibar,
    flat conformal metric (chi = 1, gt = delta, Gammahat = 0), zero shift,
    constant Khat and Theta, and a lapse linear in x, alpha = 1 + a x.  The
    fluxes are then linear in x, which the Lax-Friedrichs split and MP5
    differentiate exactly, and the equations reduce to
      d_t phibar = -alpha (c_b^2 phibar (Khat + 2 Theta) + kappa_b phibar)
        (the flux term -c_b^2 B^x a cancels the source c_b^2 B^k d_k alpha),
      d_t Bbar^x = -a phibar + phibar a / c_b^2,   d_t Bbar^y = d_t Bbar^z = 0.
    c_b^2 = 2 and kappa_b = 0.7 keep every term visible."""
    P = synth.ideal_params(bc=2, c_b=np.sqrt(2.0), kappa_b=0.7)
    O = oracle.Oracle(P)
    n, dx, a = (8, 8, 8), 0.05, 0.3
    shp = synth.patch_shape(n)
    z, y, x = synth.grid_coords(n, (0.0, 0.0, 0.0), dx)
    ID = np.zeros((26,) + shp)
    ID[0] = ID[3] = ID[5] = 1.0
    Kh = 0.02
    ID[6] = ID[9] = ID[11] = Kh / 3.0
    ID[12] = 1.0 + a * x
    ID[16], ID[17] = 1e-3, 0.1
    B = np.array([0.011, -0.007, 0.004])
    ID[21:24] = B[:, None, None, None]
    ID[24] = 0.1
    U = O.init_state(ID, n, dx)
    phi, Th = 3e-3, 0.015
    U[31] = phi      # phibar (sqrt(gamma) = 1)
    U[14] = Th       # Theta
    prim, st, worst, its = O.con2prim_patch(U, n)
    assert worst >= 0
    rhs = O.rhs_patch(U, prim, n, dx)
    inner = (slice(3, -3), slice(3, -3), slice(3, -3))
    al = (1.0 + a * np.broadcast_to(x, shp))[inner]
    Khat = U[13][inner]
    cb2, kb = 2.0, 0.7
    want_phi = -al * (cb2 * phi * (Khat + 2.0 * Th) + kb * phi)
    assert np.allclose(rhs[31][inner], want_phi, rtol=1e-12, atol=1e-18)
    assert np.allclose(rhs[28][inner], -a * phi + phi * a / cb2, rtol=1e-11, atol=1e-17)
    assert np.all(np.abs(rhs[29][inner]) < 1e-17) and np.all(np.abs(rhs[30][inner]) < 1e-17)


def test_energy_and_momentum_sources_closed_form():
    """Geometric sources of the taubar and Sbar_i equations (Sec. II B, eq.
    mhd_system) on a magnetised fluid at rest: flat conformal metric, zero
    shift, constant extrinsic curvature K_ij (so Atilde_ij = K_ij - delta_ij K/3
    and Khat = K), Theta = 0, lapse alpha = 1 + a x.  With
    S_ij = delta_ij (p + B^2/2) - B_i B_j (def_cont at v = 0), tr S = 3p + B^2/2
    and tau + D = rho (1 + eps) + B^2/2:
      d_t taubar = alpha (S^ij Atilde_ij + tr S Khat / 3),
      d_t Sbar_i = -a S^x_i - delta_ix (tau + D) a,
    the flux of Sbar_i being alpha S^x_i, linear in x."""
    P = synth.ideal_params(bc=2)
    O = oracle.Oracle(P)
    n, dx, a = (8, 8, 8), 0.05, 0.3
    shp = synth.patch_shape(n)
    z, y, x = synth.grid_coords(n, (0.0, 0.0, 0.0), dx)
    K = np.array([[0.02, 0.005, -0.003], [0.005, -0.01, 0.004], [-0.003, 0.004, 0.015]])
    ID = np.zeros((26,) + shp)
    ID[0] = ID[3] = ID[5] = 1.0
    for m, (i, j) in enumerate([(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]):
        ID[6 + m] = K[i, j]
    ID[12] = 1.0 + a * x
    rho, eps = 1e-3, 0.1
    ID[16], ID[17] = rho, eps
    B = np.array([0.011, -0.007, 0.004])
    ID[21:24] = B[:, None, None, None]
    ID[24] = 0.1
    U = O.init_state(ID, n, dx)
    prim, st, worst, its = O.con2prim_patch(U, n)
    assert worst >= 0
    rhs = O.rhs_patch(U, prim, n, dx)
    inner = (slice(3, -3), slice(3, -3), slice(3, -3))
    al = (1.0 + a * np.broadcast_to(x, shp))[inner]
    p = (P["gamma_th"] - 1.0) * rho * eps
    B2 = B @ B
    S = np.eye(3) * (p + 0.5 * B2) - np.outer(B, B)
    Kh = np.trace(K)
    At = K - np.eye(3) * Kh / 3.0
    want_tau = al * (np.sum(S * At) + (3 * p + 0.5 * B2) * Kh / 3.0)
    assert np.allclose(rhs[24][inner], want_tau, rtol=1e-11, atol=1e-20)
    tpd = rho * (1 + eps) + 0.5 * B2
    for i in range(3):
        want = -a * S[0, i] - (tpd * a if i == 0 else 0.0)
        assert np.allclose(rhs[25 + i][inner], want, rtol=1e-11, atol=1e-18), i
    assert np.all(np.abs(rhs[22][inner]) < 1e-18)


def test_shift_advection_terms_closed_form():
    """Shift terms of the fluxes of eq. mhd_system on a magnetised fluid at
    rest in flat space with alpha = 1 and a shift linear in x,
    beta = (b x, c x, 0): every flux -beta^k U and the induction terms
    Bbar^i (-beta^k) - Bbar^k (-beta^i) are linear in x, so
      d_t (Dbar, DYebar, taubar) = b (Dbar, DYebar, taubar),  d_t Sbar_i = 0,
      d_t Bbar = (0, b B^y - c B^x, b B^z),  d_t phibar = 0."""
    P = synth.ideal_params(bc=2)
    O = oracle.Oracle(P)
    n, dx, b, c = (8, 8, 8), 0.05, 0.2, -0.15
    shp = synth.patch_shape(n)
    z, y, x = synth.grid_coords(n, (0.0, 0.0, 0.0), dx)
    ID = np.zeros((26,) + shp)
    ID[0] = ID[3] = ID[5] = 1.0
    ID[12] = 1.0
    ID[13] = b * x
    ID[14] = c * x
    ID[16], ID[17] = 1e-3, 0.1
    B = np.array([0.011, -0.007, 0.004])
    ID[21:24] = B[:, None, None, None]
    ID[24] = 0.1
    U = O.init_state(ID, n, dx)
    prim, st, worst, its = O.con2prim_patch(U, n)
    assert worst >= 0
    rhs = O.rhs_patch(U, prim, n, dx)
    inner = (slice(3, -3), slice(3, -3), slice(3, -3))
    for f in (22, 23, 24):
        assert np.allclose(rhs[f][inner], b * U[f][inner], rtol=1e-11, atol=1e-20), f
    for f in (25, 26, 27, 28, 31):
        assert np.all(np.abs(rhs[f][inner]) < 1e-17), f
    assert np.allclose(rhs[29][inner], b * B[1] - c * B[0], rtol=1e-11, atol=1e-18)
    assert np.allclose(rhs[30][inner], b * B[2], rtol=1e-11, atol=1e-18)
