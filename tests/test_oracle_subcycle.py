"""Pins of the oracle's sub-cycling in time (Sec. IV C, BOR) and of the dense
output it rests on (Sec. III A, dense output interpolator).

- The dense output at theta = 1 is the RK step itself (b_j(1) are the
  tableau's weights), for RK4 and SSP-RK3.
- On u' = u^2 (closed-form derivatives u'' = 2 u^3, u''' = 6 u^4,
  f_U u'' = 4 u^4) the dense-output derivatives D_m and J = 4 (k3 - k2)
  approach dt^m u^(m) and dt^3 f_U u'' at fourth order.
- The BOR stage values of a fine step (ratio 2, both halves of the coarse
  step) approach the fine RK stages started from the exact solution at
  fourth order (RK4) and third order (SSP-RK3); without the f_U u'' term RK4
  only reaches third.
- A hierarchy of one level: the sub-cycled step is the plain step.
- Three properly nested levels: the sub-cycled evolution converges to the
  synchronous one (every level at the finest step, restricted at the same
  times) at fourth order (RK4) and third order (SSP-RK3), away from the
  level-0 outer boundary, whose stage-wise extrapolation is the same in both.
- A fine patch whose prolongation stencil leaves the coarser level's
  interiors is an error.
"""
import numpy as np
import pytest

import oracle
import synth

W_RK4 = np.array([1.0, 2.0, 2.0, 1.0]) / 6.0
W_RK3 = np.array([1.0, 1.0, 4.0]) / 6.0


def _rk4_ks(f, u0, dt):
    k1 = dt * f(u0)
    k2 = dt * f(u0 + k1 / 2)
    k3 = dt * f(u0 + k2 / 2)
    k4 = dt * f(u0 + k3)
    return np.array([k1, k2, k3, k4])


def _rk3_ks(f, u0, dt):
    k1 = dt * f(u0)
    k2 = dt * f(u0 + k1)
    k3 = dt * f(u0 + k1 / 4 + k2 / 4)
    return np.array([k1, k2, k3])


def _fine_stages(f, u0, h, rk):
    if rk == 0:
        y2 = u0 + h / 2 * f(u0)
        y3 = u0 + h / 2 * f(y2)
        return [u0, y2, y3, u0 + h * f(y3)]
    y2 = u0 + h * f(u0)
    return [u0, y2, u0 + h / 4 * f(u0) + h / 4 * f(y2)]


def _sq(u):
    return u * u


def _exact(u0, t):
    return u0 / (1.0 - u0 * t)


@pytest.mark.parametrize("rk", [0, 1])
def test_dense_output_at_theta_one_is_the_step(rk):
    rng = np.random.default_rng(0)
    w = W_RK4 if rk == 0 else W_RK3
    for _ in range(20):
        k = rng.normal(size=len(w))
        D = oracle.dense_derivs(rk, k)
        assert D[0] + D[1] / 2 + D[2] / 6 == pytest.approx(float(w @ k), rel=1e-14, abs=1e-15)


def test_dense_output_derivatives_fourth_order():
    u0 = 0.7
    errs = []
    for dt in (0.02, 0.01, 0.005):
        D = oracle.dense_derivs(0, _rk4_ks(_sq, u0, dt))
        assert D[0] == pytest.approx(dt * u0 ** 2, rel=1e-15)
        errs.append([abs(D[1] - dt ** 2 * 2 * u0 ** 3), abs(D[2] - dt ** 3 * 6 * u0 ** 4),
                     abs(D[3] - dt ** 3 * 4 * u0 ** 4)])
    e = np.array(errs)
    assert np.all(e[:-1] / e[1:] > 12.0), e


@pytest.mark.parametrize("rk", [0, 1])
def test_bor_stage_values_order(rk):
    u0 = 0.7
    ns = 4 if rk == 0 else 3
    ks = _rk4_ks if rk == 0 else _rk3_ks
    full, noj = [], []
    for dt in (0.04, 0.02, 0.01):
        D = oracle.dense_derivs(rk, ks(_sq, u0, dt))
        data = np.array([u0, D[0], D[1], D[2], D[3]])
        ef, en = [], []
        for m in range(2):
            t0 = m * dt / 2
            true = _fine_stages(_sq, _exact(u0, t0), dt / 2, rk)
            for s in range(ns):
                c = oracle.bor_coeffs(rk, m, 2, s)
                ef.append(abs(c @ data - true[s]))
                en.append(abs(c[:4] @ data[:4] - true[s]))
        full.append(ef)
        noj.append(en)
    full, noj = np.array(full), np.array(noj)
    floor = 1e-15
    ratio = (full[:-1] + floor) / (full[1:] + floor)
    if rk == 0:
        assert np.all(ratio[:, full[0] > 1e-13] > 12.0), ratio
        # Without f_U u'' the third and fourth stages are only third order.
        rn = noj[:-1, [2, 3, 6, 7]] / noj[1:, [2, 3, 6, 7]]
        assert np.all(rn < 10.0) and np.all(rn > 6.0), rn
    else:
        assert np.all(ratio[:, full[0] > 1e-13] > 6.0), ratio


def _fourier_hierarchy(specs, rk):
    P = synth.ideal_params(bc=3)
    P["rk"] = rk
    _, norm = synth.config0_id(n=(32, 32, 32), seed=0, return_norm=True)
    norm = dict(norm, b_scale=0.1 * norm["b_scale"])
    H = oracle.Hierarchy(oracle.Oracle(P), specs)
    for q, s in enumerate(specs):
        H.init_state(q, synth.config0_id(n=s["n"], seed=0, dx=s["dx"], x0=s["x0"], norm=norm))
    return H


def test_single_level_subcycle_is_the_plain_step():
    specs = [synth.hierarchy.spec((16, 12, 14), 0, (0, 0, 0), 1.0 / 16, (0.0, 0.0, 0.0))]
    A, B = _fourier_hierarchy(specs, 0), _fourier_hierarchy(specs, 0)
    assert A.subcycle_step(0.02) >= 0
    assert B.rk4_step(0.02) >= 0
    assert np.array_equal(A.U[0][0], B.U[0][0])


@pytest.mark.parametrize("rk,halvings,order_ratio", [(0, 2, 10.0), (1, 1, 5.0)])
def test_subcycled_evolution_converges_to_the_synchronous_one(rk, halvings, order_ratio):
    specs = synth.subcycle_hierarchy()
    dx0 = specs[0]["dx"]
    errs = []
    for N in [2 ** i for i in range(halvings + 1)]:
        dt0 = 0.4 * dx0 / N
        S, F = _fourier_hierarchy(specs, rk), _fourier_hierarchy(specs, rk)
        for _ in range(N):
            assert S.subcycle_step(dt0) >= 0
        for c in range(4 * N):
            # Restrict at the sub-cycled run's times: level 2 after every
            # level-1 step (two fine steps), level 1 after every level-0 step.
            m = (1 << 2 if c % 2 == 1 else 0) | (1 << 1 if c % 4 == 3 else 0)
            assert F.rk4_step(dt0 / 4, rmask=m) >= 0
        e = [max(np.abs(S.U[0][q][:, 3:-3, 3:-3, 3:-3] - F.U[0][q][:, 3:-3, 3:-3, 3:-3]).max()
                 for q, s in enumerate(specs) if s["level"] == lev) for lev in (1, 2)]
        e.append(np.abs(S.U[0][0][:, 9:-9, 9:-9, 9:-9] - F.U[0][0][:, 9:-9, 9:-9, 9:-9]).max())
        errs.append(e)
    e = np.array(errs)
    assert np.all(e[:-1] / e[1:] > order_ratio), e


def test_unnested_hierarchy_is_rejected():
    # small_hierarchy's level-2 patches sit within two level-1 points of the
    # level-1 boundary: their stencils reach undefined dense-output ghosts.
    H = _fourier_hierarchy(synth.small_hierarchy(dx0=1.0 / 24, X0=(0.0, 0.0, 0.0)), 0)
    assert H.subcycle_step(0.01) == -4
