"""Sharding a mesh-refinement hierarchy across ranks, on the CPU.

The partition and the exchange plan are the library's host code
(grmhd_shard_partition, grmhd_shard_plan); the arithmetic on each emulated
rank is the oracle's.  Each rank holds full arrays for every patch, NaN
except its own patches and the points it receives, so a missing or misplaced
source shows up as a NaN or a mismatch.

- The partition covers every patch, is deterministic and balances interior
  points to within the largest patch.
- Every send list of rank q to rank r matches rank r's receive list from q in
  length, for both phases.
- Emulated exchange (2 and 3 ranks, one process): after the level-0 owner's
  extrapolation, one exchange and a ghost fill of levels 1.., every rank's own
  patches equal the single-domain ghost fill bit for bit; after the
  restriction exchange and restriction, every rank's own patches equal the
  single-domain restriction bit for bit.
- Two gloo ranks (spawned processes) exchanging through the package's
  exchange_buffers: two RK4 steps of the magnetised TOV star, every rank
  advancing only its own patches with the oracle, equal the single-domain
  oracle's steps bit for bit.
"""
import os
import socket
import tempfile

import numpy as np
import pytest

import oracle
import synth

g = pytest.importorskip("paper_2510_13965_gb300")
torch = pytest.importorskip("torch")

NF = oracle.NF


def _lib_available():
    try:
        g.load()
        return True
    except Exception:
        return False


pytestmark = pytest.mark.skipif(not _lib_available(), reason="libgrmhd.so not built")

SPECS = synth.subcycle_hierarchy()


def _gather(H, reg, pts):
    out = np.empty((NF, pts.shape[0]))
    for i, (p, o) in enumerate(pts):
        out[:, i] = H.U[reg][p].reshape(NF, -1)[:, o]
    return out


def _scatter(H, reg, pts, buf):
    for i, (p, o) in enumerate(pts):
        H.U[reg][p].reshape(NF, -1)[:, o] = buf[:, i]


def _level0(specs):
    return [q for q, s in enumerate(specs) if s["level"] == 0][0]


def _rank_copy(O, specs, src, role, regs=(0,)):
    """A rank's arrays: its own patches copied from src, every other value NaN."""
    H = oracle.Hierarchy(O, specs)
    for r in range(4):
        for q in range(len(specs)):
            H.U[r][q][...] = np.nan
    for r in regs:
        for q in range(len(specs)):
            if role[q] == 1:
                H.U[r][q][...] = src.U[r][q]
    return H


def _extrapolate_level0(P, H, specs, reg):
    O1 = oracle.Oracle(dict(P, bc=1))
    p0 = _level0(specs)
    O1.ghost_fill(H.U[reg][p0], specs[p0]["n"])


def test_partition_balanced_and_deterministic():
    specs = synth.amr_tov_layout(scale=0.5)
    pts = np.array([np.prod(s["n"]) for s in specs])
    for R in (2, 3, 4, 8):
        own = g.shard_partition(specs, R)
        assert own == g.shard_partition(specs, R)
        assert sorted(set(own)) == list(range(R))
        load = np.bincount(own, weights=pts, minlength=R)
        assert np.all(np.abs(load - pts.sum() / R) <= pts.max()), load


def test_send_and_receive_lists_match_between_ranks():
    for R in (2, 3, 4):
        own = g.shard_partition(SPECS, R)
        plans = [g.shard_plan(SPECS, own, R, r) for r in range(R)]
        for q in range(R):
            for r in range(R):
                for ph in ("g", "r"):
                    assert plans[q][1][r][ph + "send"].shape == plans[r][1][q][ph + "recv"].shape
                    # a sender sends only points of its own patches
                    for p, _ in plans[q][1][r][ph + "send"]:
                        assert own[p] == q


@pytest.mark.parametrize("R", [2, 3])
def test_exchange_gives_single_domain_ghost_fill_and_restriction(R):
    P = synth.ideal_params(bc=3)
    O = oracle.Oracle(P)
    rng = np.random.default_rng(R)
    src = oracle.Hierarchy(O, SPECS)
    for q in range(len(SPECS)):
        src.U[0][q][...] = rng.normal(size=src.U[0][q].shape)
    truth = oracle.Hierarchy(O, SPECS)
    for q in range(len(SPECS)):
        truth.U[0][q][...] = src.U[0][q]
    assert truth.ghost_fill(0) == 0
    own = g.shard_partition(SPECS, R)
    plans = [g.shard_plan(SPECS, own, R, r) for r in range(R)]
    H = [_rank_copy(O, SPECS, src, plans[r][0]) for r in range(R)]
    p0 = _level0(SPECS)
    _extrapolate_level0(P, H[own[p0]], SPECS, 0)
    for r in range(R):
        for q in range(R):
            _scatter(H[r], 0, plans[r][1][q]["grecv"], _gather(H[q], 0, plans[q][1][r]["gsend"]))
    for r in range(R):
        assert H[r].ghost_fill(0, lmin=1) == 0
        for q in range(len(SPECS)):
            if plans[r][0][q] == 1:
                assert np.array_equal(H[r].U[0][q], truth.U[0][q]), (r, q)
    # Restriction.
    truth2 = oracle.Hierarchy(O, SPECS)
    for q in range(len(SPECS)):
        truth2.U[0][q][...] = src.U[0][q]
    assert truth2.restrict(0) == 0
    H = [_rank_copy(O, SPECS, src, plans[r][0]) for r in range(R)]
    for r in range(R):
        for q in range(R):
            _scatter(H[r], 0, plans[r][1][q]["rrecv"], _gather(H[q], 0, plans[q][1][r]["rsend"]))
    for r in range(R):
        assert H[r].restrict(0) == 0
        for q in range(len(SPECS)):
            if plans[r][0][q] == 1:
                assert np.array_equal(H[r].U[0][q], truth2.U[0][q]), (r, q)


def _tov_ids(specs):
    return [synth.tov_id(n=s["n"], x0=s["x0"], dx=s["dx"], seed=1 + q, perturb=True, bfield=True)
            for q, s in enumerate(specs)]


def _specs_tov():
    # The nested sub-cycling layout scaled onto the star (level 0 on [-12, 12)^3).
    return synth.subcycle_hierarchy(dx0=1.0, X0=(-12.0, -12.0, -12.0))


def _rank_main(rank, world, port, outdir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        specs = _specs_tov()
        P = synth.ideal_params(bc=3)
        O = oracle.Oracle(P)
        ids = _tov_ids(specs)
        src = oracle.Hierarchy(O, specs)
        for q, ID in enumerate(ids):
            src.init_state(q, ID)
        own = g.shard_partition(specs, world)
        role, lists = g.shard_plan(specs, own, world, rank)
        H = _rank_copy(O, specs, src, role, regs=(0,))
        for r in (1, 2, 3):
            for q in range(len(specs)):
                if role[q] == 1:
                    H.U[r][q][...] = 0.0
        prim = [np.zeros((oracle.NP,) + H.U[0][q].shape[1:]) for q in range(len(specs))]
        st = [np.zeros(H.U[0][q].shape[1:], dtype=np.int8) for q in range(len(specs))]
        dt = 0.25 * min(s["dx"] for s in specs)
        p0 = _level0(specs)
        for _ in range(2):
            for stage, reg in enumerate((0, 1, 2, 1)):
                if role[p0] == 1:
                    _extrapolate_level0(P, H, specs, reg)
                send = {q: torch.from_numpy(_gather(H, reg, lists[q]["gsend"])) for q in range(world)}
                recv = {q: torch.empty((NF, lists[q]["grecv"].shape[0]), dtype=torch.float64) for q in range(world)}
                g.exchange_buffers(send, recv, rank, tag=1)
                for q in range(world):
                    _scatter(H, reg, lists[q]["grecv"], recv[q].numpy())
                H.ghost_fill(reg, lmin=1)
                for q in range(len(specs)):
                    if role[q] == 1:
                        regs = [H.U[r][q] for r in range(4)]
                        O.substep(regs, prim[q], st[q], specs[q]["n"], specs[q]["dx"], stage, dt)
            send = {q: torch.from_numpy(_gather(H, 0, lists[q]["rsend"])) for q in range(world)}
            recv = {q: torch.empty((NF, lists[q]["rrecv"].shape[0]), dtype=torch.float64) for q in range(world)}
            g.exchange_buffers(send, recv, rank, tag=2)
            for q in range(world):
                _scatter(H, 0, lists[q]["rrecv"], recv[q].numpy())
            H.restrict(0)
        mine = {q: H.U[0][q] for q in range(len(specs)) if role[q] == 1}
        np.savez(os.path.join(outdir, "rank%d.npz" % rank), **{str(q): v for q, v in mine.items()})
    finally:
        dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_two_gloo_ranks_match_single_domain_oracle_steps():
    import torch.multiprocessing as mp
    specs = _specs_tov()
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_rank_main, args=(2, _free_port(), d), nprocs=2, join=True)
        got = {}
        for r in range(2):
            z = np.load(os.path.join(d, "rank%d.npz" % r))
            for k in z.files:
                got[int(k)] = z[k]
    assert sorted(got) == list(range(len(specs)))
    P = synth.ideal_params(bc=3)
    truth = oracle.Hierarchy(oracle.Oracle(P), specs)
    for q, ID in enumerate(_tov_ids(specs)):
        truth.init_state(q, ID)
    dt = 0.25 * min(s["dx"] for s in specs)
    for _ in range(2):
        assert truth.rk4_step(dt) >= 0
    for q, s in enumerate(specs):
        n = s["n"]
        sl = (slice(None), slice(3, 3 + n[2]), slice(3, 3 + n[1]), slice(3, 3 + n[0]))
        assert np.array_equal(got[q][sl], truth.U[0][q][sl]), q
