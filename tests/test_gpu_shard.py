"""Sharded hierarchy on the GPU: two shard contexts of one hierarchy, each
evolving its own patches (grmhd_init_shard), driven in lockstep in one
process with the exchange done through device buffers (the packed send list
of one shard is the other's receive buffer), against one context holding
every patch.  Two RK4 steps of the magnetised TOV star on the nested
three-level layout: every patch's interior bit for bit, on its own rank.
The kernels of the two shards never wait on each other."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2510_13965_gb300 as g  # noqa: E402


def _specs():
    return synth.subcycle_hierarchy(dx0=1.0, X0=(-12.0, -12.0, -12.0))


def test_two_shards_equal_one_context_bitwise():
    specs = _specs()
    P = synth.ideal_params(bc=3)
    ids = [synth.tov_id(n=s["n"], x0=s["x0"], dx=s["dx"], seed=1 + q, perturb=True, bfield=True)
           for q, s in enumerate(specs)]
    full = g.Patches(P, specs)
    R = 2
    shards = [g.ShardedHierarchy(P, specs, r, R) for r in range(R)]
    for q, ID in enumerate(ids):
        t = torch.as_tensor(ID, device="cuda")
        full.init_state(q, t)
        shards[shards[0].owner[q]].init_state(q, t)
    for sh in shards:
        assert sum(sh.points_exchanged.values()) > 0
    dt = 0.25 * min(s["dx"] for s in specs)
    for _ in range(2):
        full.step(dt)
        for s, reg in enumerate(shards[0].stage_registers()):
            for sh in shards:
                sh.ghost0(reg)
            sends = [sh.pack(reg, "g") for sh in shards]
            for r, sh in enumerate(shards):
                sh.unpack(reg, "g", {q: sends[q][r] for q in range(R)})
            for sh in shards:
                sh.substep(s, dt)
        sends = [sh.pack(0, "r") for sh in shards]
        for r, sh in enumerate(shards):
            sh.unpack(0, "r", {q: sends[q][r] for q in range(R)})
            sh.restrict()
    full.synchronize()
    for sh in shards:
        sh.synchronize()
        assert sh.sync_status() == 0
    assert full.sync_status() == 0
    for q, s in enumerate(specs):
        n = s["n"]
        sl = (slice(None), slice(3, 3 + n[2]), slice(3, 3 + n[1]), slice(3, 3 + n[0]))
        mine = shards[shards[0].owner[q]]
        assert torch.equal(mine.U[q][0][sl], full.U[q][0][sl]), q
