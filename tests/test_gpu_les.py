"""LES gradient sub-grid-scale model on the GPU (through the C ABI) against the oracle.

- Right-hand side with the SGS fluxes on (the paper's default C_M = 8, and
  all four coefficients nonzero) from the identical state: 1e-11 per field,
  as the RHS without LES; on the periodic Fourier data (ideal gas) and on the
  heated, magnetised star with the three-piece hybrid EOS and a smooth flow
  (extrapolated ghosts, so the outermost ghost layer takes the one-sided
  gradients).
- Five RK4 steps with C_M = 8 through a CUDA graph: 1e-9 per field.
- The LES terms off leave the fused step bit for bit as before.
- The tabulated EOS (numerical pressure derivatives): the right-hand side of
  a flowing, magnetised star with the synthetic table, C_M = 8 and all
  coefficients, at 1e-11.
"""
import numpy as np
import pytest

import oracle
import synth
from tests._checks import interior, field_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2510_13965_gb300 as g  # noqa: E402
from tests.test_gpu_parity import _rhs_ok, _setup, _upload  # noqa: E402

NF = 32


def _fourier(les):
    _, norm = synth.config0_id(n=(24, 24, 24), seed=2, return_norm=True)
    norm = dict(norm, b_scale=0.3 * norm["b_scale"])
    P = synth.ideal_params(bc=0)
    P["les_c"] = les
    return P, (24, 24, 24), 1.0 / 24, synth.config0_id(n=(24, 24, 24), seed=2, norm=norm)


def _hybrid_star(les):
    P = synth.hybrid_params(bc=1)
    P["les_c"] = les
    P["les_rho_min"] = 1e-6  # the switch is exercised: the atmosphere gets no SGS flux
    n, x0, dx = (28, 28, 28), (-9.45, -9.45, -9.45), 0.7
    ID = synth.tov_id(n=n, x0=x0, dx=dx, seed=1, heat=1.5)
    # A smooth flow through the magnetised star: the induction SGS term needs
    # velocity gradients (it vanishes for the static star).
    z, y, x = synth.grid_coords(n, x0, dx, 1)
    ID[18] = 0.02 * np.sin(y / 3.0) + 0.0 * x
    ID[19] = 0.02 * np.sin(z / 3.0) + 0.0 * y
    ID[20] = 0.02 * np.sin(x / 3.0) + 0.0 * z
    return P, n, dx, np.ascontiguousarray(ID)


CASES = {"fourier": _fourier, "hybrid_star": _hybrid_star}


@pytest.mark.parametrize("les", [(0.0, 0.0, 0.0, 8.0), (1.0, 1.0, 1.0, 8.0)])
@pytest.mark.parametrize("case", sorted(CASES))
def test_rhs_with_les_matches_oracle(case, les):
    P, n, dx, ID = CASES[case](les)
    pt, O, U = _setup(P, n, dx, ID)
    _upload(pt, U)
    pt.con2prim(0)
    rhs_g = pt.rhs_eval(0)[0]
    pt.synchronize()
    assert pt.sync_status() == 0
    Uo = U.copy()
    prim_o, st_o, _, _ = O.con2prim_patch(Uo, n)
    rhs_o = O.rhs_patch(Uo, prim_o, n, dx)
    # The SGS terms are a visible part of the right-hand side.
    P0 = dict(P, les_c=(0.0, 0.0, 0.0, 0.0))
    rhs_0 = oracle.Oracle(P0).rhs_patch(Uo, prim_o, n, dx)
    assert np.abs(interior(rhs_o - rhs_0, n)[28:31]).max() > 1e-6 * np.abs(interior(rhs_o, n)[28:31]).max()
    ok, bad = _rhs_ok(interior(rhs_g.cpu().numpy(), n), interior(rhs_o, n), O, U, n, dx)
    assert ok, bad


def test_les_steps_match_oracle():
    P, n, dx, ID = _fourier((0.0, 0.0, 0.0, 8.0))
    pt, O, U = _setup(P, n, dx, ID)
    _upload(pt, U)
    regs = [U.copy(), np.zeros_like(U), np.zeros_like(U), np.zeros_like(U)]
    prim = np.zeros((oracle.NP,) + U.shape[1:])
    st = np.zeros(U.shape[1:], dtype=np.int8)
    dt = 0.25 * dx
    pt.capture_graph(5, dt)
    pt.graph_launch()
    for _ in range(5):
        O.rk4_step(regs, prim, st, n, dx, dt)
    pt.synchronize()
    assert pt.sync_status() == 0
    e = field_err(interior(pt.U[0][0].cpu().numpy(), n), interior(regs[0], n))
    assert e.max() < 1e-9, e


def test_les_off_is_the_plain_step():
    P, n, dx, ID = _fourier((0.0, 0.0, 0.0, 0.0))
    a = g.Patches(P, [dict(n=n, dx=dx)])
    b = g.Patches(dict(P, les_c=(0.0, 0.0, 0.0, 0.0)), [dict(n=n, dx=dx)])
    for pt in (a, b):
        pt.init_state(0, torch.as_tensor(ID, device="cuda"))
        pt.step(0.25 * dx)
    a.synchronize()
    b.synchronize()
    assert torch.equal(a.U[0][0], b.U[0][0])


@pytest.mark.parametrize("les", [(0.0, 0.0, 0.0, 8.0), (1.0, 1.0, 1.0, 8.0)])
def test_rhs_with_les_table_eos_matches_oracle(les):
    table = synth.make_table(nr=64, nt=48, ny=16)
    P = synth.table_params(table, bc=1)
    P["les_c"] = les
    P["les_rho_min"] = 1e-6
    n, x0, dx = (28, 28, 28), (-9.45, -9.45, -9.45), 0.7
    ID = synth.tov_id(n=n, x0=x0, dx=dx, seed=1, table=table, rho_atmo=P["rho_atmo"])
    z, y, x = synth.grid_coords(n, x0, dx, 1)
    ID[18] = 0.02 * np.sin(y / 3.0) + 0.0 * x
    ID[19] = 0.02 * np.sin(z / 3.0) + 0.0 * y
    ID[20] = 0.02 * np.sin(x / 3.0) + 0.0 * z
    ID[24] = 0.1 + 0.05 * np.sin((x + y + z) / 4.0)
    ID = np.ascontiguousarray(ID)
    pt, O, U = _setup(P, n, dx, ID, table=table)
    _upload(pt, U)
    pt.con2prim(0)
    rhs_g = pt.rhs_eval(0)[0]
    pt.synchronize()
    assert pt.sync_status() == 0
    Uo = U.copy()
    prim_o, st_o, _, _ = O.con2prim_patch(Uo, n)
    rhs_o = O.rhs_patch(Uo, prim_o, n, dx)
    ok, bad = _rhs_ok(interior(rhs_g.cpu().numpy(), n), interior(rhs_o, n), O, U, n, dx)
    assert ok, bad
