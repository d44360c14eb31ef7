"""Algorithmic FP64 flops per unit of each substep kernel, counted by the oracle.

Runs the counting build of the oracle (every +, -, *, /, sqrt and
transcendental call counted once; min, max, abs, negation and comparisons
free) on one RK4 substep of a sub-box of the 128^3 TOV workload (same grid
spacing, magnetised and perturbed star) and prints flops per unit:
  con2prim          per ghosted point
  pointwise fluxes  per point-direction where computed
  interface fluxes  per interface
  local RHS         per interior point (CCZ4 + gauge + KO + MHD sources + flux difference)
  RK combination    per interior point (stage 0)
Usage: python -m oracle.count_flops [n]
"""
import json
import sys

import numpy as np

import oracle
import synth


def count(n=24, dx=0.3125, center=(0.0, 0.0, 2.5)):
    P = synth.ideal_params(bc=1)
    nn = (n, n, n)
    x0 = [c - (n // 2) * dx for c in center]
    ID = synth.tov_id(n=nn, x0=x0, dx=dx, seed=1)
    O = oracle.Oracle(P, flops=True)
    U = O.init_state(ID, nn, dx)
    regs = [U, np.zeros_like(U), np.zeros_like(U), np.zeros_like(U)]
    prim = np.zeros((oracle.NP,) + U.shape[1:])
    st = np.zeros(U.shape[1:], dtype=np.int8)
    O.flops(reset=True)
    c = O.substep_counted(regs, prim, st, nn, dx, 0, 0.4 * dx)
    g3 = (n + 6) ** 3
    pt_dirs = 3 * (n + 6) * n * n
    ifaces = 3 * (n + 1) * n * n
    n3 = n ** 3
    return {
        "c2p_per_ghosted_point": c[0] / g3,
        "flux_per_point_direction": c[1] / pt_dirs,
        "iflux_per_interface": c[2] / ifaces,
        "rhs_local_per_interior_point": c[3] / n3,
        "rk_stage0_per_interior_point": c[4] / n3,
        "n": n,
        "dx": dx,
    }


if __name__ == "__main__":
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 24
    print(json.dumps(count(n), indent=1))
