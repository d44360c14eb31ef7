"""Pins of the oracle's LES gradient sub-grid-scale model (Sec. II B;
Appendix "Large Eddy Simulation techniques").

The paper's closed forms H_N, H_NY, H_T, H_M (with Psi_v, Psi_M, Psi_Theta,
H_p, H_Theta, H_v) are checked against the definition they come from: for a
flux F(C) the gradient model's SGS residual is -xi H with
H = grad(dF/dC) . grad C, i.e. H = L(F o C) - (dF/dC) L(C) with the filter's
second-moment operator L = gamma^{ab} d_a d_b.  The brute-force side builds
C(x) from analytic primitives with prim2con, F(x) from the textbook MHD fluxes,
dF/dC from finite differences through prim2con, and L by finite differences,
at one point; the oracle's side is its discrete SGS flux divided by
alpha C xi sqrt(gamma).  Checked on a flat and a constant non-diagonal metric,
for the ideal gas and the hybrid EOS.  This pins the symbol readings
(h the enthalpy density, cE = h W^2, Theta = cE + B^2, E = v x B) and the sign
of every added flux.

- The LES terms change only the D, DYe, S_i and B^i right-hand sides.
- The tabulated EOS has no pressure derivatives here: the oracle refuses it.
"""
import numpy as np
import pytest

import oracle
import synth

NP = oracle.NP
GDD_CURVED = np.array([1.1, 0.05, -0.03, 0.95, 0.02, 1.05])
SYM = [[0, 1, 2], [1, 3, 4], [2, 4, 5]]


def _mat(g6):
    return np.array([[g6[SYM[i][j]] for j in range(3)] for i in range(3)])


def _fields(x, rho0, eps_of):
    X, Y, Z = x
    rho = rho0 * (1 + 0.1 * np.sin(2.1 * X + 0.3) * np.cos(1.3 * Y) + 0.05 * Z)
    eps = eps_of(rho) * (1.4 + 0.2 * np.cos(1.7 * X - 0.8 * Z) + 0.1 * Y)
    v = np.array([0.3 * np.sin(1.1 * Y + 0.5 * Z), 0.2 * np.cos(0.9 * X) + 0.1 * Z, -0.25 * np.sin(1.4 * X + Y)])
    B = np.array([0.02 * np.cos(1.2 * Z + X), 0.015 * np.sin(0.8 * X - Y) + 0.01, 0.03 * np.cos(Y)])
    ye = 0.1 + 0.02 * np.sin(X + 0.7 * Y)
    return rho, eps, v, B, ye


def _case(kind):
    if kind == "ideal":
        P = synth.ideal_params(bc=1)
        return P, 1e-3, (lambda rho: 0.2 + 0.0 * rho)
    P = synth.hybrid_params(bc=1)
    O = oracle.Oracle(P)
    return P, 7e-4, (lambda rho: O.eos_from_T(float(rho), 0.0, 0.1)[1])


def _brute(O, g6, x, fields):
    g = _mat(g6)
    gu = np.linalg.inv(g)

    def prim_vec(xx):
        rho, eps, v, B, ye = fields(xx)
        return np.concatenate([[rho, eps], v, B, [ye]])

    def cons(q):
        rho, eps, v, B, ye = q[0], q[1], q[2:5], q[5:8], q[8]
        pr = np.zeros(NP)
        pr[0], pr[1], pr[2], pr[3:6], pr[7] = rho, eps, O.eos_from_eps(rho, eps, ye)[0], v, ye
        return np.asarray(oracle.prim2con_point(pr, B, g6))  # D, DYe, tau, S_i, B^i

    def flux(q):
        rho, eps, v, B, ye = q[0], q[1], q[2:5], q[5:8], q[8]
        p = O.eos_from_eps(rho, eps, ye)[0]
        c = cons(q)
        D, DY, S = c[0], c[1], c[3:6]
        vd, Bd = g @ v, g @ B
        Bv, B2 = Bd @ v, Bd @ B
        W2 = 1.0 / (1.0 - vd @ v)
        Sij = 0.5 * (np.outer(vd, S) + np.outer(S, vd)) + g * p - (2 * np.outer(Bd, Bd) - g * B2) / (2 * W2) \
            - 0.5 * Bv * (np.outer(Bd, vd) + np.outer(vd, Bd) - g * Bv)
        out = []
        for k in range(3):
            FS = gu[k] @ Sij
            FB = B * v[k] - B[k] * v
            out.append(np.concatenate([[D * v[k], DY * v[k]], FS, FB]))
        return np.array(out)  # (3, 8): D, DYe, S_i, B^i

    def L(f, h=2e-3):
        tot = 0.0
        for a in range(3):
            for b in range(3):
                ea, eb = np.eye(3)[a] * h, np.eye(3)[b] * h
                if a == b:
                    d2 = (-f(x + 2 * ea) + 16 * f(x + ea) - 30 * f(x) + 16 * f(x - ea) - f(x - 2 * ea)) / (12 * h * h)
                else:
                    d2 = (f(x + ea + eb) - f(x + ea - eb) - f(x - ea + eb) + f(x - ea - eb)) / (4 * h * h)
                tot = tot + gu[a, b] * d2
        return tot

    q0 = prim_vec(x)

    def jac(f, q):
        cols = []
        for a in range(q.size):
            dq = np.zeros_like(q)
            dq[a] = 1e-6 * max(abs(q[a]), 1e-3)
            cols.append(((f(q + dq) - f(q - dq)) / (2 * dq[a])).ravel())
        return np.array(cols).T

    dCdP = jac(cons, q0)
    keep = [0, 1, 3, 4, 5, 6, 7, 8]  # conserved D, DYe, S_i, B^i (tau's flux has no SGS term)
    dFdC = jac(flux, q0) @ np.linalg.inv(dCdP)
    LC = L(lambda xx: cons(prim_vec(xx)))
    LF = L(lambda xx: flux(prim_vec(xx)).ravel())
    H = (LF - dFdC @ LC).reshape(3, 8)
    del keep
    return H


@pytest.mark.parametrize("kind", ["ideal", "hybrid"])
@pytest.mark.parametrize("metric", ["flat", "curved"])
def test_closed_forms_match_the_gradient_model(kind, metric):
    P, rho0, eps_of = _case(kind)
    P["les_c"] = (1.0, 1.0, 1.0, 1.0)
    O = oracle.Oracle(P)
    g6 = np.array([1.0, 0, 0, 1.0, 0, 1.0]) if metric == "flat" else GDD_CURVED
    n, dx, x0 = (8, 8, 8), 0.01, np.array([0.09, -0.25, 0.33])
    shp = (n[2] + 6, n[1] + 6, n[0] + 6)
    ID = np.zeros((synth.NID,) + shp)
    ax = [x0[a] + dx * np.arange(-3, n[a] + 3) for a in range(3)]
    Zg, Yg, Xg = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    rho, eps, v, B, ye = _fields((Xg, Yg, Zg), rho0, np.vectorize(eps_of))
    for c in range(6):
        ID[c] = g6[c]
    ID[12] = 1.0
    ID[16], ID[17], ID[24] = rho, eps, ye
    ID[18:21] = v
    ID[21:24] = B
    U = O.init_state(ID, n, dx)
    prim, st, _, _ = O.con2prim_patch(U, n)
    assert np.all(st == 0)
    c = (4, 4, 4)
    xc = x0 + dx * np.array(c)
    Hb = _brute(O, g6, xc, lambda xx: _fields(xx, rho0, eps_of))
    sg = np.sqrt(np.linalg.det(_mat(g6)))
    xi = np.linalg.det(_mat(g6)) ** (1 / 3) * dx * dx / 24
    for d in range(3):
        F = O.les_flux_points(U, prim, n, dx, [c], d)[0]
        Ho = np.concatenate([F[0:2], F[3:9]]) / (xi * sg)
        for sl in (slice(0, 1), slice(1, 2), slice(2, 5), slice(5, 8)):
            scale = np.abs(Hb[:, sl]).max()
            assert np.abs(Ho[sl] - Hb[d, sl]).max() <= 1e-5 * scale, (d, sl, Ho[sl], Hb[d, sl])
        assert F[2] == 0.0 and F[9] == 0.0


def test_les_terms_touch_only_the_fluxed_conserved_fields():
    P = synth.ideal_params(bc=1)
    ID = synth.config0_id(n=(12, 12, 12), seed=3)
    base = oracle.Oracle(P)
    U = base.init_state(ID, (12, 12, 12), 1.0 / 12)
    prim, st, _, _ = base.con2prim_patch(U, (12, 12, 12))
    r0 = base.rhs_patch(U, prim, (12, 12, 12), 1.0 / 12)
    P["les_c"] = (1.0, 1.0, 1.0, 8.0)
    r1 = oracle.Oracle(P).rhs_patch(U, prim, (12, 12, 12), 1.0 / 12)
    same = [f for f in range(32) if f not in (22, 23, 25, 26, 27, 28, 29, 30)]
    assert np.array_equal(r0[same], r1[same])
    for f in (22, 23, 25, 26, 27, 28, 29, 30):
        assert not np.array_equal(r0[f], r1[f]), f


def _table_case():
    table = synth.make_table(nr=64, nt=48, ny=16)
    P = synth.table_params(table, bc=1)
    # A point in the middle of one table cell of (log10 rho, log10 T, Ye), where
    # radiation and gas pressure are comparable (rho ~ 1e-7, T ~ 10 MeV): there
    # dp/dYe at fixed eps is not small (for the gas alone p = 2/3 rho eps).
    lr = table["lr0"] + table["dlr"] * 36.5
    lt = table["lt0"] + table["dlt"] * 31.5
    ye0 = table["ye0"] + table["dye"] * 4.5
    return table, P, lr, lt, ye0


def test_table_pressure_derivatives_are_the_interpolants():
    table, P, _, _, _ = _table_case()
    O = oracle.Oracle(P, table)
    rng = np.random.default_rng(8)
    for _ in range(40):
        # a state well inside one cell of (log10 rho, log10 T, Ye)
        ir, it, iy = rng.integers(2, 60), rng.integers(2, 44), rng.integers(1, 14)
        lr = table["lr0"] + table["dlr"] * (ir + rng.uniform(0.2, 0.8))
        lt = table["lt0"] + table["dlt"] * (it + rng.uniform(0.2, 0.8))
        ye = table["ye0"] + table["dye"] * (iy + rng.uniform(0.2, 0.8))
        rho = 10.0 ** lr
        eps = O.eos_from_T(rho, 10.0 ** lt, ye)[1]
        d = O.eos_derivs(rho, eps, ye)
        h = 1e-6

        def p(r, e, y):
            return O.eos_from_eps(r, e, y)[0]

        fd = [(p(rho * (1 + h), eps, ye) - p(rho * (1 - h), eps, ye)) / (2 * h * rho),
              (p(rho, eps * (1 + h), ye) - p(rho, eps * (1 - h), ye)) / (2 * h * eps),
              (p(rho, eps, ye + h) - p(rho, eps, ye - h)) / (2 * h)]
        pscale = p(rho, eps, ye)
        for a, b, sc in zip(d, fd, (pscale / rho, pscale / eps, pscale)):
            assert abs(a - b) <= 1e-6 * max(abs(b), 1e-3 * sc), (d, fd)


def test_table_pressure_derivatives_against_the_model():
    table, P, lr, lt, ye0 = _table_case()
    O = oracle.Oracle(P, table)
    rho, T, ye = 10.0 ** lr, 10.0 ** lt, ye0
    eps = O.eos_from_T(rho, T, ye)[1]
    d = O.eos_derivs(rho, eps, ye)

    def p_model(r, e, y):
        # invert the analytic model for T at (r, y) so that its eps is e
        lo, hi = -3.0, 3.0
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if synth.eos_table.model(r, 10.0 ** mid, y)[1] < e:
                lo = mid
            else:
                hi = mid
        return synth.eos_table.model(r, 10.0 ** lo, y)[0]

    h = 1e-4
    want = [(p_model(rho * (1 + h), eps, ye) - p_model(rho * (1 - h), eps, ye)) / (2 * h * rho),
            (p_model(rho, eps * (1 + h), ye) - p_model(rho, eps * (1 - h), ye)) / (2 * h * eps),
            (p_model(rho, eps, ye + h) - p_model(rho, eps, ye - h)) / (2 * h)]
    for a, b in zip(d, want):
        assert a == pytest.approx(b, rel=0.05), (d, want)


def test_closed_forms_match_the_gradient_model_table():
    table, P, lr, lt, ye0 = _table_case()
    P["les_c"] = (1.0, 1.0, 1.0, 1.0)
    O = oracle.Oracle(P, table)
    g6 = GDD_CURVED

    def fields(x):
        X, Y, Z = x
        rho = 10.0 ** lr * (1 + 0.02 * np.sin(2.1 * X + 0.3) * np.cos(1.3 * Y) + 0.01 * Z)
        T = 10.0 ** lt * (1 + 0.02 * np.cos(1.7 * X - 0.8 * Z) + 0.01 * Y)
        ye = ye0 + 0.4 * table["dye"] * np.sin(3.0 * X + 2.1 * Y + 1.4 * Z)
        eps = np.vectorize(lambda r, t, y: O.eos_from_T(r, t, y)[1])(rho, T, ye)
        v = np.array([0.3 * np.sin(1.1 * Y + 0.5 * Z), 0.2 * np.cos(0.9 * X) + 0.1 * Z, -0.25 * np.sin(1.4 * X + Y)])
        B = np.array([0.02 * np.cos(1.2 * Z + X), 0.015 * np.sin(0.8 * X - Y) + 0.01, 0.03 * np.cos(Y)]) * 1e-3
        return rho, eps, v, B, ye, T

    n, dx, x0 = (8, 8, 8), 0.01, np.array([0.09, -0.25, 0.33])
    shp = (n[2] + 6, n[1] + 6, n[0] + 6)
    ID = np.zeros((synth.NID,) + shp)
    ax = [x0[a] + dx * np.arange(-3, n[a] + 3) for a in range(3)]
    Zg, Yg, Xg = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    rho, eps, v, B, ye, T = fields((Xg, Yg, Zg))
    for c in range(6):
        ID[c] = g6[c]
    ID[12] = 1.0
    ID[16], ID[17], ID[24], ID[25] = rho, eps, ye, T
    ID[18:21] = v
    ID[21:24] = B
    U = O.init_state(ID, n, dx)
    prim, st, _, _ = O.con2prim_patch(U, n)
    assert np.all(st == 0)
    c = (4, 4, 4)
    xc = x0 + dx * np.array(c)
    Hb = _brute(O, g6, xc, lambda xx: fields(xx)[:5])
    sg = np.sqrt(np.linalg.det(_mat(g6)))
    xi = np.linalg.det(_mat(g6)) ** (1 / 3) * dx * dx / 24
    for d in range(3):
        F = O.les_flux_points(U, prim, n, dx, [c], d)[0]
        Ho = np.concatenate([F[0:2], F[3:9]]) / (xi * sg)
        for sl in (slice(0, 1), slice(1, 2), slice(2, 5), slice(5, 8)):
            scale = np.abs(Hb[:, sl]).max()
            assert np.abs(Ho[sl] - Hb[d, sl]).max() <= 1e-4 * scale, (d, sl, Ho[sl], Hb[d, sl])


def test_density_switch():
    """Flux points below les_rho_min get no SGS flux; the others are unchanged."""
    P, rho0, eps_of = _case("ideal")
    P["les_c"] = (1.0, 1.0, 1.0, 8.0)
    ID = synth.config0_id(n=(10, 10, 10), seed=3)
    base = oracle.Oracle(P)
    U = base.init_state(ID, (10, 10, 10), 0.1)
    prim, _, _, _ = base.con2prim_patch(U, (10, 10, 10))
    pts = [[i, 4, 5] for i in range(10)]
    F0 = base.les_flux_points(U, prim, (10, 10, 10), 0.1, pts, 0)
    rho = np.array([prim[0][5 + 3, 4 + 3, i + 3] for i in range(10)])
    thr = np.median(rho)
    F1 = oracle.Oracle(dict(P, les_rho_min=thr)).les_flux_points(U, prim, (10, 10, 10), 0.1, pts, 0)
    assert np.all(F1[rho < thr] == 0.0)
    assert np.array_equal(F1[rho >= thr], F0[rho >= thr])
    assert np.any(F0[rho < thr] != 0.0)
