"""Global convergence order of the evolution on the GPU (config-0 data: Fourier
modes on the metric and the magnetised fluid, periodic 1^3 box).

Self-convergence at N = 16, 32, 64 with dt = 0.4 dx to t = 0.05 (before the
strongly magnetised fluid drains its internal energy to the clamp):
rate = log2(|U_16 - U_32| / |U_32 - U_64|) over the points the three grids
share, max norm per field.  Spacetime fields >= 3.5 (fourth-order differences
and RK4), the coupled fluid >= 2 (the MP5 limiter acts at the steep parts).
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2510_13965_gb300 as g  # noqa: E402


def _evolve(n, norm, t_end=0.05):
    dx = 1.0 / n
    P = synth.ideal_params(bc=0)
    ID = synth.config0_id(n=(n, n, n), seed=0, norm=norm)
    pt = g.Patches(P, [dict(n=(n, n, n), dx=dx)])
    pt.init_state(0, torch.as_tensor(ID, device="cuda"))
    dt = 0.4 * dx
    steps = int(round(t_end / dt))
    for _ in range(steps):
        pt.step(dt)
    pt.synchronize()
    assert pt.sync_status() == 0
    return pt.U[0][0][:, 3:-3, 3:-3, 3:-3].cpu().numpy()


def test_global_convergence_order_config0():
    _, norm = synth.config0_id(n=(64, 64, 64), seed=0, return_norm=True)
    u16, u32, u64 = (_evolve(n, norm) for n in (16, 32, 64))
    # Common points: index i on N = 16 is 2i on N = 32 and 4i on N = 64.
    c16 = u16
    c32 = u32[:, ::2, ::2, ::2]
    c64 = u64[:, ::4, ::4, ::4]
    e1 = np.abs(c16 - c32).reshape(32, -1).max(axis=1)
    e2 = np.abs(c32 - c64).reshape(32, -1).max(axis=1)
    ok = e2 > 0
    rate = np.full(32, np.inf)
    rate[ok] = np.log2(e1[ok] / e2[ok])
    # Fields that change (the others stay at their exact constant values).
    moving = e1 > 1e-13
    st = [f for f in range(22) if moving[f]]
    mhd = [f for f in range(22, 31) if moving[f]]
    assert st and mhd
    assert np.all(rate[st] >= 3.5), {f: rate[f] for f in st}
    assert np.all(rate[mhd] >= 2.0), {f: rate[f] for f in mhd}
