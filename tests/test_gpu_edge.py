"""Edge cases of the CUDA path (through the C ABI) against the oracle.

- Empty inputs: con2prim, prim2con, seeded con2prim and seeder inference of
  zero states return empty outputs and no error.
- The smallest patches the boundary accepts (4 interior points per axis, so
  that three ghost layers can be filled from the interior), mixed with ragged
  ones in one batched context: 4 x 4 x 4, 4 x 9 x 5 and 5 x 4 x 11 (every
  point within two of the ghosts on some axis): initial data, con2prim
  (statuses bit-exact, primitives to 1e-10) and the right-hand side (1e-11
  per field) against the oracle, and a CUDA-graph step equal to the eager one
  bit for bit.
- Smaller patches are refused with GRMHD_ERR_ARG.
"""
import numpy as np
import pytest

import oracle
import synth
from tests._checks import interior, prim_check

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2510_13965_gb300 as g  # noqa: E402
from tests.test_gpu_parity import _rhs_ok  # noqa: E402

SHAPES = [(4, 4, 4), (4, 9, 5), (5, 4, 11)]
DX = 1.0 / 16


def test_empty_inputs():
    P = synth.ideal_params()
    cons = torch.zeros((0, 10), dtype=torch.float64, device="cuda")
    prim, st = g.c2p_flat(P, cons)
    assert prim.shape == (0, g.NP) and st.shape == (0,)
    out = g.prim2con_flat(P, torch.zeros((0, 10), dtype=torch.float64, device="cuda"),
                          torch.zeros((0, 3), dtype=torch.float64, device="cuda"))
    assert out.shape[0] == 0
    res = g.c2p_flat_seeded(P, cons, None)
    assert all(r.shape[0] == 0 for r in res)
    S = g.Seeder(seed=2)
    assert S.infer(cons).shape[0] == 0
    torch.cuda.synchronize()


def _ids():
    _, norm = synth.config0_id(n=(32, 32, 32), seed=4, return_norm=True)
    return [synth.config0_id(n=n, seed=4, dx=DX, x0=(0.1 * q, 0.2, 0.3), norm=norm) for q, n in enumerate(SHAPES)]


def test_degenerate_patch_shapes_match_oracle():
    P = synth.ideal_params(bc=1)
    specs = [dict(n=n, dx=DX, x0=(0.1 * q, 0.2, 0.3)) for q, n in enumerate(SHAPES)]
    pt = g.Patches(P, specs)
    O = oracle.Oracle(P)
    ids = _ids()
    for q, ID in enumerate(ids):
        pt.init_state(q, torch.as_tensor(ID, device="cuda"))
    pt.synchronize()
    Us = []
    for q, (n, ID) in enumerate(zip(SHAPES, ids)):
        U = O.init_state(ID, n, DX)
        pt.U[q][0].copy_(torch.as_tensor(U, device="cuda"))
        Us.append(U)
    torch.cuda.synchronize()
    pt.con2prim(0)
    rhs = pt.rhs_eval(0)
    pt.synchronize()
    assert pt.sync_status() == 0
    for q, (n, U) in enumerate(zip(SHAPES, Us)):
        Uo = U.copy()
        prim_o, st_o, _, _ = O.con2prim_patch(Uo, n)
        assert np.array_equal(pt.status[q].cpu().numpy(), st_o), n
        prim_check(pt.prim[q].cpu().numpy(), prim_o, pt.status[q].cpu().numpy(), st_o, Uo[22:25])
        rhs_o = O.rhs_patch(Uo, prim_o, n, DX)
        ok, bad = _rhs_ok(interior(rhs[q].cpu().numpy(), n), interior(rhs_o, n), O, U, n, DX)
        assert ok, (n, bad)


def test_degenerate_patch_shapes_graph_equals_eager():
    P = synth.ideal_params(bc=1)
    specs = [dict(n=n, dx=DX, x0=(0.1 * q, 0.2, 0.3)) for q, n in enumerate(SHAPES)]
    a, b = g.Patches(P, specs), g.Patches(P, specs)
    for pt in (a, b):
        for q, ID in enumerate(_ids()):
            pt.init_state(q, torch.as_tensor(ID, device="cuda"))
    b.capture_graph(2, 0.25 * DX)
    a.step(0.25 * DX)
    a.step(0.25 * DX)
    b.graph_launch()
    a.synchronize()
    b.synchronize()
    assert a.sync_status() == 0
    for q in range(len(SHAPES)):
        assert torch.equal(a.U[q][0], b.U[q][0]), SHAPES[q]


@pytest.mark.parametrize("n", [(3, 4, 4), (4, 1, 4), (4, 4, 2)])
def test_patches_below_four_points_are_refused(n):
    with pytest.raises(g.GrmhdError):
        g.Patches(synth.ideal_params(bc=1), [dict(n=n, dx=DX)])
