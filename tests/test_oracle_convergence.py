"""Global convergence order of the oracle's evolution (Fourier-mode data on
the metric and the magnetised fluid, periodic unit box): self-convergence at
N = 16, 32, 64 with dt = 0.4 dx to t = 0.05, before the strongly magnetised
fluid drains its internal energy to the clamp.  rate = log2(|U_16 - U_32| /
|U_32 - U_64|) over the points the three grids share, max norm per field.
The spacetime fields must converge at >= 3.5 (fourth-order differences and
RK4), the coupled fluid at >= 2 (MP5's limiter acts at the steep parts; the
paper reports orders between 2 and 3 for its MHD tests)."""
import numpy as np

import oracle
import synth


def _evolve(n, norm, t_end=0.05):
    dx = 1.0 / n
    P = synth.ideal_params(bc=0)
    O = oracle.Oracle(P)
    ID = synth.config0_id(n=(n, n, n), seed=0, norm=norm)
    U = O.init_state(ID, (n, n, n), dx)
    regs = [U, np.zeros_like(U), np.zeros_like(U), np.zeros_like(U)]
    prim = np.zeros((oracle.NP,) + U.shape[1:])
    status = np.zeros(U.shape[1:], dtype=np.int8)
    dt = 0.4 * dx
    for _ in range(int(round(t_end / dt))):
        assert O.rk4_step(regs, prim, status, (n, n, n), dx, dt) >= 0
    return regs[0][:, 3:3 + n, 3:3 + n, 3:3 + n]


def test_oracle_global_convergence_order():
    _, norm = synth.config0_id(n=(64, 64, 64), seed=0, return_norm=True)
    u16, u32, u64 = (_evolve(n, norm) for n in (16, 32, 64))
    e1 = np.abs(u16 - u32[:, ::2, ::2, ::2]).reshape(32, -1).max(axis=1)
    e2 = np.abs(u32[:, ::2, ::2, ::2] - u64[:, ::4, ::4, ::4]).reshape(32, -1).max(axis=1)
    ok = e2 > 0
    rate = np.full(32, np.inf)
    rate[ok] = np.log2(e1[ok] / e2[ok])
    moving = e1 > 1e-13
    st = [f for f in range(22) if moving[f]]
    mhd = [f for f in range(22, 31) if moving[f]]
    assert st and mhd
    assert np.all(rate[st] >= 3.5), {f: rate[f] for f in st}
    assert np.all(rate[mhd] >= 2.0), {f: rate[f] for f in mhd}
