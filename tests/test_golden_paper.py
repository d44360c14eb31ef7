"""The oracle's discrete operators reproduce the coefficients the paper prints
(tests/golden/paper_operators.json, each entry citing its passage): the
operators are applied to unit impulses, and each recovered weight must equal
the printed one.  The Runge-Kutta tableaux are checked against the order
conditions of their stated orders (the oracle's RK4 step is pinned to the
exact Taylor polynomial in test_oracle_ccz4.py)."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

G = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_operators.json")))


def _impulse(n, pos):
    u = np.zeros(n)
    u[pos] = 1.0
    return u


def _weights(kind, offsets, *args, scale=1.0, n=9):
    c = n // 2
    return [oracle.fd(kind, _impulse(n, c + o), *args) * scale for o in offsets]


def test_centred_first_derivative():
    e = G["D1_centred"]
    assert _weights("d1", e["offsets"], 1.0 / 12.0) == pytest.approx(e["coefficients"], abs=1e-13)


def test_compact_second_derivative():
    e = G["D2_compact"]
    assert _weights("d2", e["offsets"], 1.0, scale=12.0) == pytest.approx(e["coefficients"], abs=1e-13)


@pytest.mark.parametrize("name,beta", [("D1_advection_beta_negative", -1.0), ("D1_advection_beta_positive", 1.0)])
def test_one_sided_advection(name, beta):
    e = G[name]
    assert _weights("up", e["offsets"], beta, 1.0 / 12.0) == pytest.approx(e["coefficients"], abs=1e-13)


def test_kreiss_oliger():
    e = G["Kreiss_Oliger"]
    # sigma = 64, dx = 1: the operator returns the bracket itself.
    assert _weights("ko", e["offsets"], 64.0, 1.0) == pytest.approx(e["coefficients"], abs=1e-13)


def test_mp5_unlimited_interpolant():
    e = G["MP5_interpolant"]
    # On a steep monotone ramp the limiter leaves the fifth-order value, which is
    # linear in the data: a small impulse on top reveals each weight.
    ramp = np.arange(-2, 3, dtype=float) * 10.0
    base = oracle.mp5(ramp)
    eps = 1e-3
    got = [(oracle.mp5(ramp + eps * _impulse(5, o + 2)) - base) / eps * 60.0 for o in e["offsets"]]
    assert got == pytest.approx(e["coefficients"], abs=1e-7)
    assert base == pytest.approx(sum(c * x for c, x in zip(e["coefficients"], ramp)) / 60.0, abs=1e-12)


def test_prolongation_midpoint_weights():
    e = G["prolongation_midpoint"]
    specs = synth.small_hierarchy()
    H = oracle.Hierarchy(oracle.Oracle(synth.ideal_params(bc=3)), specs)
    # Level 1 patch 1 (o = 12): its ghost i = -3 is the midpoint of coarse x-points 4 and 5.
    # Coarse data = impulse at one x index (constant in y and z: the y and z midpoint
    # formulas then return the value unchanged, their weights summing to 256 / 256).
    got = []
    for o in e["offsets"]:
        for q in range(len(specs)):
            H.U[0][q][...] = 0.0
        H.U[0][0][:, :, :, 3 + 4 + o] = 1.0
        assert H.ghost_fill(0) == 0
        got.append(H.U[0][1][0, 3 + 5, 3 + 5, 0] * 256.0)
    assert got == e["coefficients"]
    assert sum(e["coefficients"]) == 256


def _order_conditions(a, b, c, order):
    A = [[Fraction(x) for x in row] for row in a]
    B = [Fraction(x) for x in b]
    C = [Fraction(x) for x in c]
    s = len(B)
    assert all(sum(A[i]) == C[i] for i in range(s))      # row sums = nodes
    conds = [sum(B) == 1]
    if order >= 2:
        conds.append(sum(B[i] * C[i] for i in range(s)) == Fraction(1, 2))
    if order >= 3:
        conds.append(sum(B[i] * C[i] ** 2 for i in range(s)) == Fraction(1, 3))
        conds.append(sum(B[i] * A[i][j] * C[j] for i in range(s) for j in range(s)) == Fraction(1, 6))
    if order >= 4:
        conds.append(sum(B[i] * C[i] ** 3 for i in range(s)) == Fraction(1, 4))
        conds.append(sum(B[i] * C[i] * A[i][j] * C[j] for i in range(s) for j in range(s)) == Fraction(1, 8))
        conds.append(sum(B[i] * A[i][j] * C[j] ** 2 for i in range(s) for j in range(s)) == Fraction(1, 12))
        conds.append(sum(B[i] * A[i][j] * A[j][k] * C[k] for i in range(s) for j in range(s) for k in range(s))
                     == Fraction(1, 24))
    return all(conds)


def _stability_coefficient(a, b, k):
    """Coefficient of z^k in R(z) = 1 + z b^T (I - z A)^-1 1, i.e. b^T A^(k-1) 1."""
    A = [[Fraction(x) for x in row] for row in a]
    v = [Fraction(1)] * len(A)
    for _ in range(k - 1):
        v = [sum(A[i][j] * v[j] for j in range(len(A))) for i in range(len(A))]
    return sum(Fraction(bi) * vi for bi, vi in zip(b, v))


@pytest.mark.parametrize("name,order", [("RK4_explicit", 4), ("SSP_RK3_explicit", 3)])
def test_runge_kutta_tableaux_have_their_order(name, order):
    e = G[name]
    assert _order_conditions(e["a"], e["b"], e["c"], order)
    fact = 1
    for k in range(1, order + 2):
        fact *= k
        coef = _stability_coefficient(e["a"], e["b"], k)
        if k <= order:
            assert coef == Fraction(1, fact), (k, coef)
        else:
            assert coef != Fraction(1, fact), (k, coef)  # not of order + 1
