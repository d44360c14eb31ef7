"""Pins of the oracle's hybrid EOS (Sec. II B: piecewise-polytropic cold part
plus an ideal-gas thermal part; eq. piecewise_p_eps_cold).

- p_cold and eps_cold are continuous at the dividing densities (the constants
  K_i, a_i are fixed by continuity) while the exponent changes.
- With one piece and Gamma_0 = Gamma_th the hybrid EOS is the ideal gas.
- c_s^2 h equals dp/drho|_eps + p / rho^2 dp/deps|_rho by finite differences.
- con2prim round trips on hybrid-EOS states.
"""
import numpy as np
import pytest

import oracle
import synth

NP = oracle.NP


def _cold(O, rho):
    e_min = O.eos_from_T(rho, 0.0, 0.1)  # cold state: p_cold, eps_cold
    return e_min[0], e_min[1]


def test_cold_part_continuous_at_dividing_densities():
    P = synth.hybrid_params()
    O = oracle.Oracle(P)
    for rb in P["rho_poly"][:2]:
        lo, hi = _cold(O, rb * (1 - 1e-12)), _cold(O, rb * (1 + 1e-12))
        assert abs(lo[0] - hi[0]) <= 1e-9 * lo[0]
        assert abs(lo[1] - hi[1]) <= 1e-9 * lo[1]
        # ... while the exponent d ln p / d ln rho jumps.
        h = 1e-6
        g_lo = np.log(_cold(O, rb * (1 - h))[0] / _cold(O, rb * (1 - 2 * h))[0]) / np.log((1 - h) / (1 - 2 * h))
        g_hi = np.log(_cold(O, rb * (1 + 2 * h))[0] / _cold(O, rb * (1 + h))[0]) / np.log((1 + 2 * h) / (1 + h))
        assert g_hi - g_lo > 0.25


def test_single_piece_with_gamma_th_is_the_ideal_gas():
    Ph = synth.hybrid_params(npoly=1, gamma_th=2.0, gamma_poly=(2.0, 0, 0, 0))
    Pi = synth.ideal_params()
    Oh, Oi = oracle.Oracle(Ph), oracle.Oracle(Pi)
    rng = np.random.default_rng(0)
    for _ in range(50):
        rho = 10 ** rng.uniform(-8, -2)
        # Inside the EOS's domain (eps >= eps_cold); the hybrid form adds the
        # cold and thermal parts, so rounding grows with eps_cold / eps_th.
        eps_c = _cold(Oh, rho)[1]
        eps = eps_c * (1 + 10 ** rng.uniform(-1, 1))
        tol = 1e-15 * (4 + 4 * eps_c / (eps - eps_c))
        a, b = Oh.eos_from_eps(rho, eps, 0.1), Oi.eos_from_eps(rho, eps, 0.1)
        assert abs(a[0] - b[0]) <= tol * b[0]
        assert abs(a[3] - b[3]) <= 2 * tol * b[3]


def test_sound_speed_matches_finite_differences():
    P = synth.hybrid_params()
    O = oracle.Oracle(P)
    for rho in (1e-4, 6e-4, 1.2e-3):
        eps = _cold(O, rho)[1] + 0.05
        p, _, _, cs2 = O.eos_from_eps(rho, eps, 0.1)
        hr, he = 1e-6 * rho, 1e-6 * eps
        dpdr = (O.eos_from_eps(rho + hr, eps, 0.1)[0] - O.eos_from_eps(rho - hr, eps, 0.1)[0]) / (2 * hr)
        dpde = (O.eos_from_eps(rho, eps + he, 0.1)[0] - O.eos_from_eps(rho, eps - he, 0.1)[0]) / (2 * he)
        h = 1 + eps + p / rho
        assert cs2 == pytest.approx((dpdr + p / rho ** 2 * dpde) / h, rel=1e-7)


def test_con2prim_round_trip_hybrid():
    P = synth.hybrid_params()
    O = oracle.Oracle(P)
    rng = np.random.default_rng(1)
    for _ in range(40):
        rho = 10 ** rng.uniform(-6, -2.8)
        eps = _cold(O, rho)[1] + 10 ** rng.uniform(-3, -0.5)
        pr = np.zeros(NP)
        pr[0], pr[1], pr[7] = rho, eps, 0.1
        pr[2] = O.eos_from_eps(rho, eps, 0.1)[0]
        pr[3:6] = rng.uniform(-0.3, 0.3, 3)
        B = rng.normal(size=3) * 1e-3
        cb = np.zeros(10)
        cb[:9] = oracle.prim2con_point(pr, B, [1.0, 0, 0, 1.0, 0, 1.0])
        st, out, _, _ = O.c2p_point(cb, [1.0, 0, 0, 1.0, 0, 1.0], 1.0, 1.0)
        assert st == 0
        assert abs(out[0] - rho) <= 1e-12 * rho
        assert abs(out[1] - eps) <= 1e-11 * eps
        assert np.all(np.abs(out[3:6] - pr[3:6]) <= 1e-12)
