"""Sub-cycling in time (Sec. IV C, BOR) on the GPU, through the C ABI, against the oracle.

- From the identical state, one and three sub-cycled level-0 steps of the
  three-level nested hierarchy (seven level steps, 28 substeps each for RK4)
  agree with the oracle's within 1e-9 per field on every patch (the
  multi-step bound); RK4 (dense registers U^n, D_1..D_3, J) and SSP-RK3
  (U^n, D_1, D_2).  Measured: 3.4e-10 after one step (A~_ij, K^), where the
  oracle against itself from a 1e-14-perturbed start already differs by
  5.5e-9, sub-cycled or not: the data's own rounding sensitivity.  A field
  also passes within 1e-14 absolute: for the static star the components that
  vanish analytically (off-diagonal gt_ij ~ 2e-8, A~_ij ~ 3e-7) hold only
  truncation error, left where O(1e-2) terms cancel, and differ by ~1e-15.
- A one-level hierarchy: the sub-cycled step is the synchronous step, bit for bit.
- CUDA-graph replay of sub-cycled steps equals eager steps bit for bit.
- grmhd_set_subcycling rejects a layout whose prolongation stencils leave
  the coarser level's interiors, and a context without a hierarchy.
- Combinations: sub-cycling with the LES SGS fluxes (C_M = 8), with the
  hybrid EOS (a heated star on the nested layout), and with seeded con2prim
  (an untrained network: poor seeds fall back to the plain bracket, so the
  step equals the plain one to the Brent stop rule).
"""
import numpy as np
import pytest

import oracle
import synth
from tests._checks import field_err, interior

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2510_13965_gb300 as g  # noqa: E402

NF = 32


def _ids(specs):
    _, norm = synth.config0_id(n=(32, 32, 32), seed=0, return_norm=True)
    norm = dict(norm, b_scale=0.1 * norm["b_scale"])
    return [synth.config0_id(n=s["n"], seed=0, dx=s["dx"], x0=s["x0"], norm=norm) for s in specs]


def _pair(specs, rk, P=None, ids=None):
    P = synth.ideal_params(bc=3) if P is None else P
    P["rk"] = rk
    pt = g.Patches(P, specs)
    H = oracle.Hierarchy(oracle.Oracle(P), specs)
    for q, ID in enumerate(_ids(specs) if ids is None else ids):
        H.init_state(q, ID)
        pt.U[q][0].copy_(torch.as_tensor(H.U[0][q], device="cuda"))
    torch.cuda.synchronize()
    return pt, H


def _close(pt, H, specs, tol):
    for q, s in enumerate(specs):
        got = interior(pt.U[q][0].cpu().numpy(), s["n"])
        want = interior(H.U[0][q], s["n"])
        err = field_err(got, want)
        d = np.abs(got - want).reshape(NF, -1).max(axis=1)
        ok = (err < tol) | (d < 1e-14)
        assert np.all(ok), (q, s["level"], {f: err[f] for f in range(NF) if not ok[f]})


@pytest.mark.parametrize("rk", [0, 1])
def test_subcycled_steps_match_oracle(rk):
    specs = synth.subcycle_hierarchy()
    pt, H = _pair(specs, rk)
    pt.set_subcycling(True)
    dt0 = 0.4 * specs[0]["dx"]
    pt.step(dt0)
    pt.synchronize()
    assert pt.sync_status() == 0
    assert H.subcycle_step(dt0) >= 0
    _close(pt, H, specs, 1e-9)
    for _ in range(2):
        pt.step(dt0)
        assert H.subcycle_step(dt0) >= 0
    pt.synchronize()
    assert pt.sync_status() == 0
    _close(pt, H, specs, 1e-9)


def test_single_level_subcycled_step_is_the_synchronous_step():
    specs = [synth.hierarchy.spec((20, 16, 18), 0, (0, 0, 0), 1.0 / 20, (0.0, 0.0, 0.0))]
    a, _ = _pair(specs, 0)
    b, _ = _pair(specs, 0)
    b.set_subcycling(True)
    for pt in (a, b):
        pt.step(0.02)
        pt.step(0.02)
    a.synchronize()
    b.synchronize()
    assert torch.equal(a.U[0][0], b.U[0][0])


def test_subcycled_graph_replay_equals_eager():
    specs = synth.subcycle_hierarchy()
    a, _ = _pair(specs, 0)
    b, _ = _pair(specs, 0)
    for pt in (a, b):
        pt.set_subcycling(True)
    dt0 = 0.4 * specs[0]["dx"]
    b.capture_graph(2, dt0)
    a.step(dt0)
    a.step(dt0)
    b.graph_launch()
    a.synchronize()
    b.synchronize()
    for q in range(len(specs)):
        assert torch.equal(a.U[q][0], b.U[q][0]), q


def test_set_subcycling_rejects_unnested_layouts_and_plain_contexts():
    pt = g.Patches(synth.ideal_params(bc=3), synth.small_hierarchy())
    with pytest.raises(g.GrmhdError):
        pt.set_subcycling(True)
    plain = g.Patches(synth.ideal_params(bc=1), [dict(n=(16, 16, 16), dx=1.0 / 16)])
    with pytest.raises(g.GrmhdError):
        plain.set_subcycling(True)


@pytest.mark.parametrize("combo", ["les", "hybrid"])
def test_subcycling_combined_with_les_and_hybrid_eos(combo):
    specs = synth.subcycle_hierarchy()
    if combo == "les":
        P = synth.ideal_params(bc=3)
        P["les_c"] = (0.0, 0.0, 0.0, 8.0)
        ids = None
    else:
        # A smooth heated star (hybrid EOS, no noise, no field) on the nested
        # layout scaled to [-5, 5)^3; the noisy magnetised star amplifies
        # rounding far beyond the parity bound (the surface layer).
        P = synth.hybrid_params(bc=3)
        ids = [synth.tov_id(n=s["n"], x0=tuple(10.0 * (x - 0.5) for x in s["x0"]), dx=10.0 * s["dx"], seed=7 + q,
                            heat=1.5, perturb=False, bfield=False) for q, s in enumerate(specs)]
        specs = [dict(s, dx=10.0 * s["dx"], x0=tuple(10.0 * (x - 0.5) for x in s["x0"])) for s in specs]
    pt, H = _pair(specs, 0, P=P, ids=ids)
    pt.set_subcycling(True)
    dt0 = 0.4 * specs[0]["dx"]
    pt.step(dt0)
    pt.synchronize()
    assert pt.sync_status() == 0
    assert H.subcycle_step(dt0) >= 0
    _close(pt, H, specs, 1e-9)


def test_subcycling_with_seeded_con2prim_equals_plain():
    specs = synth.subcycle_hierarchy()
    a, _ = _pair(specs, 0)
    b, _ = _pair(specs, 0)
    S = g.Seeder(seed=3)  # untrained: the seeds are poor and fall back to the plain bracket
    b.set_seeder(S, 0.03)
    for pt in (a, b):
        pt.set_subcycling(True)
        pt.step(0.4 * specs[0]["dx"])
    a.synchronize()
    b.synchronize()
    assert a.sync_status() == 0 and b.sync_status() == 0
    for q, s in enumerate(specs):
        e = field_err(interior(b.U[q][0].cpu().numpy(), s["n"]), interior(a.U[q][0].cpu().numpy(), s["n"]))
        assert e.max() < 1e-9, (q, e.max())
