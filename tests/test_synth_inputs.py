"""Sanity checks of the seeded input generators (no method arithmetic here).

The static star is the standard polytrope K = 100, Gamma = 2,
rho_c = 1.28e-3 in G = c = M_sun = 1, whose gravitational mass 1.400 and
areal radius 9.586 are quoted throughout the numerical-relativity literature;
its isotropic surface radius follows from r = rb (1 + M / (2 rb))^2 outside
the star.  The con2prim state recipe must honour its ranges.
"""
import numpy as np

import synth


def test_tov_star_matches_literature_values():
    p = synth.tov_profile()
    assert abs(p["M"] - 1.400) < 1e-3
    assert abs(p["R"] - 9.586) < 1e-3
    # Exterior Schwarzschild in isotropic coordinates at the surface.
    assert abs(p["Rb"] * (1 + p["M"] / (2 * p["Rb"])) ** 2 - p["R"]) < 1e-9 * p["R"]
    assert abs(p["p_c"] - 100.0 * 1.28e-3 ** 2) < 1e-18


def test_c2p_state_ranges():
    s = synth.c2p_states(1 << 14, seed=3)
    W = 1.0 / np.sqrt(1.0 - np.sum(s["v"] ** 2, axis=1))
    b2 = np.sum(s["B"] ** 2, axis=1) / W ** 2 + np.sum(s["B"] * s["v"], axis=1) ** 2
    assert s["rho"].min() >= 1e-10 and s["rho"].max() <= 1e-2
    assert W.min() >= 1.0 - 1e-12 and W.max() <= 10.0 + 1e-9
    assert s["T"].min() >= 1e-2 and s["T"].max() <= 1e2
    assert s["ye"].min() >= 0.05 and s["ye"].max() <= 0.5
    r = b2 / s["rho"]
    assert r.min() >= 1e-4 * (1 - 1e-9) and r.max() <= 10.0 * (1 + 1e-9)
    # log-uniform density: about a tenth of the states per decade
    dec = np.histogram(np.log10(s["rho"]), bins=8, range=(-10, -2))[0] / len(s["rho"])
    assert np.all(np.abs(dec - 0.125) < 0.02)


def test_batched_layout_recipe():
    specs = synth.batched_specs(npatch=256, seed=2)
    assert len(specs) == 256
    for s in specs:
        assert all(e in synth.EDGES for e in s["n"])
        assert s["dx"] == (1.0 / 32) / 2 ** s["level"] and 0 <= s["level"] < 5
