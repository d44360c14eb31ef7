"""Mesh-refinement hierarchy (bc 3) on the GPU, through the C ABI, against the oracle.

- Ghost fill of every fine patch (same-level copies and six-point Lagrange
  prolongation, through two levels): bit-exact, since both sides round the
  paper's midpoint formula operation by operation in the same order; the
  level-0 outer extrapolation within rounding.
- Restriction: bit-exact copies.
- One RK4 step of the TOV star on the five-patch hierarchy from the identical
  state: interiors within 1e-11 per field (the right-hand side tolerance).
- CUDA-graph replay of hierarchy steps equals eager steps bit for bit.
- A layout whose fine ghosts leave the coarser level is rejected.
"""
import numpy as np
import pytest

import oracle
import synth
from tests._checks import field_err, init_ok, interior

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2510_13965_gb300 as g  # noqa: E402

NF = 32


def _pair(specs, P=None):
    P = P if P is not None else synth.ideal_params(bc=3)
    pt = g.Patches(P, specs)
    H = oracle.Hierarchy(oracle.Oracle(P), specs)
    return pt, H


def _upload_all(pt, H, reg=0):
    for q in range(len(H.specs)):
        pt.U[q][reg].copy_(torch.as_tensor(H.U[reg][q], device="cuda"))
    torch.cuda.synchronize()


def _ghost_mask(s):
    n = s["n"]
    m = np.ones((n[2] + 6, n[1] + 6, n[0] + 6), dtype=bool)
    m[3:-3, 3:-3, 3:-3] = False
    return m


def test_hierarchy_ghost_fill_matches_oracle():
    specs = synth.small_hierarchy()
    pt, H = _pair(specs)
    rng = np.random.default_rng(21)
    for q in range(len(specs)):
        H.U[1][q][...] = rng.normal(size=H.U[1][q].shape)
    _upload_all(pt, H, reg=1)
    assert H.ghost_fill(1) == 0
    pt.ghost_fill(1)
    pt.synchronize()
    for q, s in enumerate(specs):
        got = pt.U[q][1].cpu().numpy()
        if s["level"] == 0:
            assert np.max(np.abs(got - H.U[1][q])) <= 1e-14 * np.max(np.abs(H.U[1][q]))
        else:
            assert np.array_equal(got, H.U[1][q]), q


def test_hierarchy_restriction_matches_oracle():
    specs = synth.small_hierarchy()
    pt, H = _pair(specs)
    rng = np.random.default_rng(22)
    for q in range(len(specs)):
        H.U[0][q][...] = rng.normal(size=H.U[0][q].shape)
    _upload_all(pt, H, reg=0)
    assert H.restrict(0) == 0
    pt.restrict(0)
    pt.synchronize()
    for q in range(len(specs)):
        assert np.array_equal(pt.U[q][0].cpu().numpy(), H.U[0][q]), q


def _tov_hierarchy():
    specs = synth.small_hierarchy()
    ids = [synth.tov_id(n=s["n"], x0=s["x0"], dx=s["dx"], seed=1 + q, perturb=True, bfield=True)
           for q, s in enumerate(specs)]
    return specs, ids


def test_hierarchy_rk4_step_matches_oracle():
    specs, ids = _tov_hierarchy()
    pt, H = _pair(specs)
    for q, ID in enumerate(ids):
        pt.init_state(q, torch.as_tensor(ID, device="cuda"))
        H.init_state(q, ID)
    pt.synchronize()
    for q, s in enumerate(specs):
        ok, e = init_ok(interior(pt.U[q][0].cpu().numpy(), s["n"]), interior(H.U[0][q], s["n"]), dx=s["dx"])
        assert ok, (q, e)
    _upload_all(pt, H, reg=0)
    dt = 0.25 * specs[-1]["dx"]
    pt.step(dt)
    pt.synchronize()
    assert pt.sync_status() == 0
    assert H.rk4_step(dt) >= 0
    for q, s in enumerate(specs):
        got = interior(pt.U[q][0].cpu().numpy(), s["n"])
        want = interior(H.U[0][q], s["n"])
        err = field_err(got, want)
        small = np.abs(want).reshape(NF, -1).max(axis=1) < 1e-12
        d = np.abs(got - want).reshape(NF, -1).max(axis=1)
        ok = (err < 1e-11) | (small & (d < 1e-14))
        assert np.all(ok), (q, {f: err[f] for f in range(NF) if not ok[f]})


def test_hierarchy_graph_replay_equals_eager():
    specs, ids = _tov_hierarchy()
    P = synth.ideal_params(bc=3)
    a = g.Patches(P, specs)
    b = g.Patches(P, specs)
    for pt in (a, b):
        for q, ID in enumerate(ids):
            pt.init_state(q, torch.as_tensor(ID, device="cuda"))
    dt = 0.25 * specs[-1]["dx"]
    b.capture_graph(2, dt)
    a.step(dt)
    a.step(dt)
    b.graph_launch()
    a.synchronize()
    b.synchronize()
    for q in range(len(specs)):
        assert torch.equal(a.U[q][0], b.U[q][0]), q


def test_uncovered_fine_ghosts_are_rejected():
    specs = synth.small_hierarchy()
    specs[1] = synth.hierarchy.spec((12, 12, 12), 1, (1, 12, 12), 1.0, (-12.0,) * 3)
    with pytest.raises(g.GrmhdError):
        g.Patches(synth.ideal_params(bc=3), specs)
