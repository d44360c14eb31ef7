"""Pins of the oracle's mesh-refinement ghost fill and restriction (Sec. IV B).

- The six-point Lagrange prolongation reproduces polynomials of degree <= 5 in
  each coordinate exactly, on every ghost point that comes from the coarser
  level (one or three midpoint axes, through two levels).
- A hand-computed value of the paper's midpoint formula on 2^x data.
- Sixth-order convergence of the prolongation on smooth data.
- Same-level ghosts and the restriction are exact copies.
- A ghost point that neither its level nor the coarser one covers is an error.
"""
import numpy as np

import oracle
import synth

NF = oracle.NF


def _coords(s):
    n = s["n"]
    ax = [s["x0"][a] + s["dx"] * np.arange(-3, n[a] + 3) for a in range(3)]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return X, Y, Z


def _interior_mask(s):
    n = s["n"]
    m = np.zeros((n[2] + 6, n[1] + 6, n[0] + 6), dtype=bool)
    m[3:-3, 3:-3, 3:-3] = True
    return m


def _fill(H, fn):
    for q, s in enumerate(H.specs):
        X, Y, Z = _coords(s)
        for f in range(NF):
            H.U[0][q][f] = fn(X, Y, Z, f)


def _hier(specs):
    O = oracle.Oracle(synth.ideal_params(bc=3))
    return oracle.Hierarchy(O, specs)


def _poly(X, Y, Z, f):
    return (1.0 + 0.1 * f + 0.3 * X - 0.02 * X ** 2 * Y + 1e-3 * X ** 5 - 2e-4 * Y ** 5 * Z
            + 5e-4 * Z ** 4 * X + 1e-5 * X ** 3 * Y ** 2 * Z ** 5)


def test_prolongation_exact_on_degree_five_polynomials():
    H = _hier(synth.small_hierarchy())
    _fill(H, _poly)
    # Scramble the ghosts of the fine patches: the fill must rebuild them.
    for q, s in enumerate(H.specs):
        if s["level"] > 0:
            H.U[0][q][:, ~_interior_mask(s)] = 1e30
    assert H.ghost_fill(0) == 0
    for q, s in enumerate(H.specs):
        if s["level"] == 0:
            continue
        X, Y, Z = _coords(s)
        g = ~_interior_mask(s)
        for f in (0, 7, 31):
            want = _poly(X, Y, Z, f)[g]
            got = H.U[0][q][f][g]
            assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want)), (q, f)


def test_midpoint_formula_hand_value():
    # Coarse data 2^(x/dx0) along x only: a level-1 ghost point at a midpoint
    # gets 2^(c-2) (150 (4 + 8) - 25 (2 + 16) + 3 (1 + 32)) / 256 = 2^(c-2) 1449 / 256.
    specs = synth.small_hierarchy()
    H = _hier(specs)
    _fill(H, lambda X, Y, Z, f: 2.0 ** ((X + 12.0) / 1.0))
    assert H.ghost_fill(0) == 0
    s = specs[1]  # level 1, o = (12, 12, 12): ghost i = -3 is level-1 point g = 9 (odd), c = 4
    got = H.U[0][1][0][3 + 5, 3 + 5, 0]
    assert got == 2.0 ** (4 - 2) * 1449.0 / 256.0
    # The coincident ghost i = -2 (g = 10) copies the coarse value 2^5.
    assert H.U[0][1][0][3 + 5, 3 + 5, 1] == 2.0 ** 5
    assert s["level"] == 1


def test_prolongation_sixth_order():
    errs = []
    for dx0 in (0.4, 0.2):
        X0 = (-12.0 * dx0,) * 3
        H = _hier(synth.small_hierarchy(dx0=dx0, X0=X0))
        fn = lambda X, Y, Z, f: np.sin(1.3 * X + 0.4) * np.cos(0.9 * Y - 0.2) * np.sin(0.7 * Z + 1.1)  # noqa: E731
        _fill(H, fn)
        assert H.ghost_fill(0) == 0
        s = H.specs[1]
        X, Y, Z = _coords(s)
        g = ~_interior_mask(s)
        errs.append(np.max(np.abs(H.U[0][1][0][g] - fn(X, Y, Z, 0)[g])))
    rate = np.log2(errs[0] / errs[1])
    assert rate > 5.5, (errs, rate)


def test_same_level_copy_and_restriction_are_copies():
    specs = synth.small_hierarchy()
    H = _hier(specs)
    rng = np.random.default_rng(3)
    for q in range(len(specs)):
        H.U[0][q][...] = rng.normal(size=H.U[0][q].shape)
    assert H.ghost_fill(0) == 0
    # Patch 1 (o = 12, n = 12 in x) has x-ghosts i = 12..14 inside patch 2's interior (o = 24).
    a, b = H.U[0][1], H.U[0][2]
    assert np.array_equal(a[:, 3:-3, 3:-3, 15:18], b[:, 3:-3, 3:-3, 3:6])
    before = [u.copy() for u in H.U[0]]
    assert H.restrict(0) == 0
    # Level-2 patch 3 (o = (30, 28, 28)) overwrites level-1 points g/2 of its even points.
    s3, s1 = specs[3], specs[1]
    fine = before[3][:, 3:-3:2, 3:-3:2, 3:-3:2]  # o even on every axis: i = 0, 2, ...
    lo = [s3["o"][a] // 2 - s1["o"][a] for a in range(3)]
    cnt = [(s3["n"][a] + 1) // 2 for a in range(3)]
    got = H.U[0][1][:, 3 + lo[2]:3 + lo[2] + cnt[2], 3 + lo[1]:3 + lo[1] + cnt[1], 3 + lo[0]:3 + lo[0] + cnt[0]]
    nx = min(cnt[0], s1["n"][0] - lo[0])  # part inside patch 1 (the rest lies in patch 2)
    assert np.array_equal(got[..., :nx], fine[..., :nx])
    # Level-0 points outside every level-1 patch are untouched.
    assert np.array_equal(H.U[0][0][:, :6, :6, :6], before[0][:, :6, :6, :6])


def test_uncovered_ghost_point_is_an_error():
    specs = synth.small_hierarchy()
    specs[1] = synth.hierarchy.spec((12, 12, 12), 1, (1, 12, 12), 1.0, (-12.0,) * 3)  # ghosts below level 0
    H = _hier(specs)
    assert H.ghost_fill(0) == -2
