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


def test_openmp_oracle_flat_con2prim_is_bitwise_the_serial_oracle():
    """The flat-metric con2prim over independent states (the isolated
    con2prim workload's 256 x 128 x 64 table, plain and with seeds)."""
    table = synth.make_table()
    P = synth.table_params(table)
    s = synth.c2p_states(3000, seed=7)
    rho, ye, v, B = s["rho"], s["ye"], s["v"], s["B"]
    p, eps, _ = synth.eos_table.model(rho, s["T"], ye)
    v2 = np.einsum("ij,ij->i", v, v)
    W2 = 1.0 / (1.0 - v2)
    h = rho * (1.0 + eps) + p
    B2 = np.einsum("ij,ij->i", B, B)
    vB = np.einsum("ij,ij->i", v, B)
    cons = np.zeros((3000, 10))
    cons[:, 0] = rho * np.sqrt(W2)
    cons[:, 1] = cons[:, 0] * ye
    cons[:, 2] = h * W2 - p + B2 - 0.5 * (B2 / W2 + vB * vB) - cons[:, 0]
    cons[:, 3:6] = (h * W2 + B2)[:, None] * v - vB[:, None] * B
    cons[:, 6:9] = B
    Os, Op = oracle.Oracle(P, table), oracle.Oracle(P, table, threads=4)
    for a, b in zip(Os.c2p_flat(cons), Op.c2p_flat(cons)):
        assert np.array_equal(a, b)
    _, _, _, roots, _ = Os.c2p_flat_ext(cons)
    seeds = roots * (1.0 + 0.01 * np.random.default_rng(2).uniform(-1.0, 1.0, roots.shape))
    for a, b in zip(Os.c2p_flat_ext(cons, seeds, 0.03), Op.c2p_flat_ext(cons, seeds, 0.03)):
        assert np.array_equal(a, b)
