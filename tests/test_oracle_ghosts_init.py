"""Pins of the oracle's single-patch ghost fill (three ghost layers per side)

bc 0: periodic, vertex-centred with period n points (point -m is point n-m);
bc 1: the outer-boundary extrapolation read as linear, (1 + m) U_0 - m U_1 at
distance m, exact on data linear in the indices, edges and corners included;
bc 2: the ghost values are left as they are (frozen).  Also the initial-data
conversion to the CCZ4 and conserved variables on constant data."""
import numpy as np
import pytest

import oracle
import synth

NG = 3


def _interior(U, n):
    return U[:, NG:NG + n[2], NG:NG + n[1], NG:NG + n[0]]


@pytest.mark.parametrize("n", [(6, 7, 5), (8, 8, 8)])
def test_periodic_ghosts_wrap(n):
    O = oracle.Oracle(synth.ideal_params(bc=0))
    rng = np.random.default_rng(1)
    U = np.zeros((oracle.NF,) + synth.patch_shape(n))
    _interior(U, n)[...] = rng.normal(size=(oracle.NF, n[2], n[1], n[0]))
    O.ghost_fill(U, n)
    idx = [(np.arange(-NG, m + NG) % m) + NG for m in (n[2], n[1], n[0])]
    want = U[:, idx[0]][:, :, idx[1]][:, :, :, idx[2]]
    assert np.array_equal(U, want)


def test_extrapolated_ghosts_exact_on_linear_data():
    n = (6, 7, 5)
    O = oracle.Oracle(synth.ideal_params(bc=1))
    rng = np.random.default_rng(2)
    shp = synth.patch_shape(n)
    k, j, i = np.meshgrid(*(np.arange(m) - NG for m in shp), indexing="ij")
    c = rng.normal(size=(oracle.NF, 4))
    lin = c[:, 0, None, None, None] + c[:, 1, None, None, None] * i + c[:, 2, None, None, None] * j \
        + c[:, 3, None, None, None] * k
    U = np.zeros((oracle.NF,) + shp)
    _interior(U, n)[...] = _interior(lin, n)
    O.ghost_fill(U, n)
    assert np.allclose(U, lin, rtol=0, atol=1e-12 * np.abs(lin).max())
    # not exact on a quadratic: the extrapolation is first order
    U2 = np.zeros((oracle.NF,) + shp)
    _interior(U2, n)[...] = _interior(lin + i * i, n)
    O.ghost_fill(U2, n)
    assert np.abs(U2[:, NG, NG, 0] - (lin + i * i)[:, NG, NG, 0]).max() > 0.5


def test_frozen_ghosts_untouched():
    n = (5, 5, 5)
    O = oracle.Oracle(synth.ideal_params(bc=2))
    U = np.random.default_rng(3).normal(size=(oracle.NF,) + synth.patch_shape(n))
    before = U.copy()
    O.ghost_fill(U, n)
    assert np.array_equal(U, before)


def test_init_state_conformal_split_of_constant_data():
    """Initial-data conversion to the CCZ4 variables (Sec. II A definitions):
    chi = det(gamma)^(-1/3), gt_ij = chi gamma_ij (so det gt = 1),
    Khat = gamma^ij K_ij, At_ij = chi (K_ij - gamma_ij K / 3) (trace-free with
    respect to gt), Theta = 0, Gammahat = 0 for a constant metric, and the
    densitized rest mass Dbar = sqrt(gamma) rho W."""
    n = (5, 5, 5)
    O = oracle.Oracle(synth.ideal_params(bc=2))
    rng = np.random.default_rng(4)
    M = np.eye(3) + 0.1 * rng.normal(size=(3, 3))
    g = M @ M.T
    K = 0.01 * rng.normal(size=(3, 3))
    K = K + K.T
    sym = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    ID = np.zeros((26,) + synth.patch_shape(n))
    for m, (a, b) in enumerate(sym):
        ID[m] = g[a, b]
        ID[6 + m] = K[a, b]
    ID[12] = 1.0
    rho, eps = 2e-3, 0.2
    v = np.array([0.1, -0.05, 0.02])
    ID[16], ID[17] = rho, eps
    ID[18:21] = v[:, None, None, None]
    ID[24] = 0.1
    U = O.init_state(ID, n, 0.1)
    pt = (slice(None), 4, 4, 4)
    u = U[pt]
    chi = np.linalg.det(g) ** (-1.0 / 3.0)
    gt = np.array([[u[0], u[1], u[2]], [u[1], u[3], u[4]], [u[2], u[4], u[5]]])
    At = np.array([[u[6], u[7], u[8]], [u[7], u[9], u[10]], [u[8], u[10], u[11]]])
    assert abs(u[12] - chi) < 1e-15
    assert np.allclose(gt, chi * g, rtol=1e-14, atol=0)
    assert abs(np.linalg.det(gt) - 1.0) < 1e-14
    Kt = np.trace(np.linalg.solve(g, K))
    assert abs(u[13] - Kt) < 1e-15
    assert np.allclose(At, chi * (K - g * Kt / 3.0), rtol=1e-13, atol=1e-17)
    assert abs(np.trace(np.linalg.solve(gt, At))) < 1e-16
    assert u[14] == 0.0 and np.all(np.abs(u[15:18]) < 1e-15) and u[31] == 0.0
    W = 1.0 / np.sqrt(1.0 - v @ g @ v)
    assert abs(u[22] - np.sqrt(np.linalg.det(g)) * rho * W) < 1e-15 * rho
