"""Pins of the oracle's single-patch ghost fill (three ghost layers per side).

bc 0: periodic, vertex-centred with period n points (point -m is point n-m);
bc 1: the outer-boundary extrapolation read as linear, (1 + m) U_0 - m U_1 at
distance m, exact on data linear in the indices, edges and corners included;
bc 2: the ghost values are left as they are (frozen)."""
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
