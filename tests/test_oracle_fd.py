"""Pins of the oracle's finite-difference operators and MP5 reconstruction.

Sec. III B (D_x, D_xx, mixed D_xy, one-sided advection derivatives, KO
dissipation) and Sec. III C (MP5).  Each operator is checked against exact
polynomial derivatives (the orders the stencils are built for), against a
convergence rate on smooth data, and against exact zero on constants.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.filterwarnings("ignore")


def _poly(coeffs, x):
    return sum(c * x ** k for k, c in enumerate(coeffs))


def _dpoly(coeffs, x, m=1):
    c = np.array(coeffs, dtype=float)
    for _ in range(m):
        c = np.array([k * c[k] for k in range(1, len(c))]) if len(c) > 1 else np.zeros(1)
    return _poly(c, x)


@pytest.mark.parametrize("deg", [0, 1, 2, 3, 4])
def test_d1_exact_to_degree4(deg):
    rng = np.random.default_rng(deg)
    c = rng.normal(size=deg + 1)
    dx = 0.37
    x = 0.3 + dx * np.arange(-2, 3)
    got = oracle.fd("d1", _poly(c, x), dx)
    assert abs(got - _dpoly(c, 0.3)) < 1e-11 * (1 + abs(_dpoly(c, 0.3)))


def test_d1_not_exact_degree5():
    dx = 0.37
    x = dx * np.arange(-2, 3)
    got = oracle.fd("d1", x ** 5, dx)
    # D_x x^5 at 0 = -4 dx^4 (the leading error term of the 4th-order stencil, dx^4 f^(5)/30 * -1)
    assert abs(got - (-4.0 * dx ** 4)) < 1e-12


@pytest.mark.parametrize("deg", [0, 1, 2, 3, 4, 5])
def test_d2_exact_to_degree5(deg):
    rng = np.random.default_rng(10 + deg)
    c = rng.normal(size=deg + 1)
    dx = 0.21
    x = -0.4 + dx * np.arange(-2, 3)
    got = oracle.fd("d2", _poly(c, x), dx)
    want = _dpoly(c, -0.4, 2)
    assert abs(got - want) < 1e-10 * (1 + abs(want))


@pytest.mark.parametrize("beta", [0.7, -0.7])
@pytest.mark.parametrize("deg", [0, 1, 2, 3, 4])
def test_upwind_exact_to_degree4(deg, beta):
    rng = np.random.default_rng(20 + deg)
    c = rng.normal(size=deg + 1)
    dx = 0.19
    x = 0.1 + dx * np.arange(-3, 4)
    got = oracle.fd("up", _poly(c, x), beta, dx)
    want = _dpoly(c, 0.1)
    assert abs(got - want) < 1e-10 * (1 + abs(want))


@pytest.mark.parametrize("beta", [1.0, -1.0])
def test_upwind_uses_upwind_side(beta):
    # A spike outside the one-sided stencil must not change the result.
    dx = 1.0
    u = np.zeros(7)
    if beta > 0:
        u[0] = 1e3   # x_{i-3} is not in the beta > 0 stencil (i-1 .. i+3)
    else:
        u[6] = 1e3   # x_{i+3} is not in the beta < 0 stencil (i-3 .. i+1)
    assert oracle.fd("up", u, beta, dx) == 0.0


@pytest.mark.parametrize("deg", [0, 1, 2, 3, 4, 5])
def test_ko_annihilates_degree5(deg):
    rng = np.random.default_rng(30 + deg)
    c = rng.normal(size=deg + 1)
    dx = 0.23
    x = 0.5 + dx * np.arange(-3, 4)
    got = oracle.fd("ko", _poly(c, x), 0.1, dx)
    assert abs(got) < 1e-11 * np.abs(_poly(c, x)).max()


def test_ko_value_on_degree6_and_sign():
    # sum of the 7-point stencil times x^6 = 6! dx^6, times sigma / (64 dx).
    dx, sigma = 0.5, 0.1
    x = dx * np.arange(-3, 4)
    got = oracle.fd("ko", x ** 6, sigma, dx)
    assert abs(got - sigma / (64 * dx) * 720 * dx ** 6) < 1e-12
    # Dissipative: the Nyquist mode (-1)^i is damped (negative at a +1 point).
    u = np.array([(-1.0) ** i for i in range(-3, 4)])
    assert oracle.fd("ko", u, sigma, dx) == pytest.approx(-64 * sigma / (64 * dx))


@pytest.mark.parametrize("kind,args", [("d1", ()), ("d2", ()), ("up", (0.3,)), ("up", (-0.3,)), ("ko", (0.1,))])
def test_constants_give_exact_zero(kind, args):
    for val in (0.7, 1.0 / 3.0, -123.456, 1e-300):
        n = 7 if kind in ("up", "ko") else 5
        assert oracle.fd(kind, np.full(n, val), *(args + (0.1,))) == 0.0


def test_mixed_derivative_exact_on_products():
    dx = 0.3
    rng = np.random.default_rng(5)
    cx = rng.normal(size=5)  # degree 4 in x
    cy = rng.normal(size=5)  # degree 4 in y
    x = 0.2 + dx * np.arange(-2, 3)
    y = -0.1 + dx * np.arange(-2, 3)
    u = np.outer(_poly(cy, y), _poly(cx, x))
    got = oracle.fd_d11(u, dx)
    want = _dpoly(cy, -0.1) * _dpoly(cx, 0.2)
    assert abs(got - want) < 1e-10 * (1 + abs(want))
    assert oracle.fd_d11(np.full((5, 5), 0.77), dx) == 0.0


@pytest.mark.parametrize("kind", ["d1", "d2", "up"])
def test_convergence_rate_4_on_sine(kind):
    errs = []
    for dx in (0.04, 0.02, 0.01):
        m = 7 if kind == "up" else 5
        x = 0.3 + dx * (np.arange(m) - m // 2)
        u = np.sin(3.0 * x)
        if kind == "d1":
            got, want = oracle.fd("d1", u, dx), 3.0 * np.cos(0.9)
        elif kind == "d2":
            got, want = oracle.fd("d2", u, dx), -9.0 * np.sin(0.9)
        else:
            got, want = oracle.fd("up", u, 1.0, dx), 3.0 * np.cos(0.9)
        errs.append(abs(got - want))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 3.8), rates


def test_ko_scales_as_dx5():
    vals = []
    for dx in (0.1, 0.05):
        x = 0.3 + dx * np.arange(-3, 4)
        vals.append(abs(oracle.fd("ko", np.sin(3.0 * x), 0.1, dx)))
    assert 4.8 < np.log2(vals[0] / vals[1]) < 5.2


# ---- MP5 --------------------------------------------------------------------

def _mp5_flux_derivative(f, x0, dx):
    """(Fhat_{i+1/2} - Fhat_{i-1/2}) / dx from point values of f at x0 + dx*(-3..3)."""
    F = f(x0 + dx * np.arange(-3, 4))
    hp = oracle.mp5(F[1:6])
    hm = oracle.mp5(F[0:5])
    return (hp - hm) / dx


@pytest.mark.parametrize("deg", [1, 2, 3, 4])
def test_mp5_flux_difference_exact_on_monotone_polynomials(deg):
    # Monotone, convex-free data so the limiter keeps the 5th-order value;
    # the conservative difference then reproduces f'(x) exactly up to degree 4.
    f = lambda x: x ** deg + 10.0 * x
    x0, dx = 0.35, 0.01
    got = _mp5_flux_derivative(f, x0, dx)
    want = deg * x0 ** (deg - 1) + 10.0
    assert abs(got - want) < 1e-9 * abs(want)


def test_mp5_unlimited_on_smooth_data_converges_5th_order():
    errs = []
    for dx in (0.02, 0.01):
        errs.append(abs(_mp5_flux_derivative(lambda x: np.exp(x) + 5 * x, 0.1, dx) - (np.exp(0.1) + 5)))
    assert np.log2(errs[0] / errs[1]) > 4.5


def test_mp5_hand_values():
    # Step (0,0,0,1,1): upwind interface value stays at the upwind state 0.
    assert oracle.mp5([0, 0, 0, 1, 1]) == 0.0
    # Linear data: f = i (values -2..2): interface value 0.5, unlimited formula
    # (2*-2 - 13*-1 + 47*0 + 27*1 - 3*2)/60 = (−4 + 13 + 27 − 6)/60 = 0.5, accepted.
    assert oracle.mp5([-2, -1, 0, 1, 2]) == pytest.approx(0.5, abs=1e-15)
    # Constant data: exactly the constant.
    assert oracle.mp5([3.25] * 5) == 3.25
    # Local maximum at c, (0,1,2,1,0).  By hand: f_ip = (0-13+94+27-0)/60 = 1.8,
    # f_MP = 2 + minmod(-1, 4) = 2, (1.8-2)(1.8-2) > 0 -> limiter.  d_{i-1} = 0,
    # d_i = -2, d_{i+1} = 0 -> both d^M4 = 0; f_UL = 6, f_MD = 1.5, f_LC = 2.5;
    # f_min = max(min(2,1,1.5), min(2,6,2.5)) = 2, f_max = min(2, 6) = 2 -> 2.
    assert oracle.mp5([0, 1, 2, 1, 0]) == 2.0


def test_mp5_no_new_extrema_on_steps():
    rng = np.random.default_rng(0)
    for _ in range(500):
        lo, hi = sorted(rng.normal(size=2))
        k = rng.integers(1, 5)
        f = np.array([lo] * k + [hi] * (5 - k))
        v = oracle.mp5(f)
        assert min(f[2], f[3]) - 1e-14 <= v <= max(f[2], f[3]) + 1e-14


def test_minmod4_definition():
    assert oracle.minmod4(1.0, 2.0, 3.0, 0.5) == 0.5
    assert oracle.minmod4(-1.0, -2.0, -3.0, -0.5) == -0.5
    assert oracle.minmod4(1.0, -2.0, 3.0, 0.5) == 0.0
    assert oracle.minmod4(0.0, 2.0, 3.0, 0.5) == 0.0


def test_mp5_accepts_the_unlimited_value_when_the_test_passes():
    """Suresh & Huynh's acceptance test, the paper's strict form: when
    (f_ip - f_i)(f_ip - f_MP) < 0 the interface value is the unlimited
    fifth-order one, f_ip = (2 f_{i-2} - 13 f_{i-1} + 47 f_i + 27 f_{i+1}
    - 3 f_{i+2}) / 60, with f_MP = f_i + minmod(f_{i+1} - f_i, 4 (f_i - f_{i-1}))."""
    rng = np.random.default_rng(21)
    accepted = 0
    for _ in range(4000):
        f = np.cumsum(rng.normal(size=5)) if rng.random() < 0.5 else rng.normal(size=5)
        fip = (2 * f[0] - 13 * f[1] + 47 * f[2] + 27 * f[3] - 3 * f[4]) / 60
        a, b = f[3] - f[2], 4 * (f[2] - f[1])
        mm = np.sign(a) * min(abs(a), abs(b)) if np.sign(a) == np.sign(b) else 0.0
        fmp = f[2] + mm
        if (fip - f[2]) * (fip - fmp) < -1e-12 * np.max(np.abs(f)) ** 2:
            accepted += 1
            assert abs(oracle.mp5(f) - fip) <= 1e-14 * np.max(np.abs(f))
    assert accepted > 500
