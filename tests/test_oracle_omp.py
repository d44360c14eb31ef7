"""The OpenMP build of the oracle (same sources, independent point loops on
several host threads) gives bitwise the serial build's results: initial data,
con2prim (primitives, statuses, corrected conserved variables), right-hand
side and whole RK4 steps, on the magnetised TOV star and on the periodic
Fourier data."""
import numpy as np

import oracle
import synth

NF, NP = oracle.NF, oracle.NP


def _run(O, P, n, dx, ID, steps):
    U = O.init_state(ID, n, dx)
    regs = [U, np.zeros_like(U), np.zeros_like(U), np.zeros_like(U)]
    prim = np.zeros((NP,) + U.shape[1:])
    st = np.zeros(U.shape[1:], dtype=np.int8)
    U0 = U.copy()
    p0, s0, w0, it0 = O.con2prim_patch(U0, n)
    r0 = O.rhs_patch(U0, p0, n, dx)
    for _ in range(steps):
        O.rk4_step(regs, prim, st, n, dx, 0.25 * dx)
    return [U0, p0, s0, np.array([w0, it0]), r0] + regs + [prim, st]


def test_openmp_oracle_is_bitwise_the_serial_oracle():
    cases = [
        (synth.ideal_params(bc=1), (20, 18, 16), 0.5,
         synth.tov_id(n=(20, 18, 16), x0=(-5.0, -4.5, -4.0), dx=0.5, seed=1), 2),
        (synth.ideal_params(bc=0), (12, 12, 12), 1 / 12, synth.config0_id(n=(12, 12, 12), seed=1), 2),
    ]
    for P, n, dx, ID, steps in cases:
        serial = _run(oracle.Oracle(P), P, n, dx, ID, steps)
        Opar = oracle.Oracle(P, threads=4)
        assert Opar.threads == 4
        par = _run(Opar, P, n, dx, ID, steps)
        for a, b in zip(serial, par):
            assert np.array_equal(a, b)
