"""Mesh-refinement hierarchy (bc 3) on the GPU, through the C ABI, against the oracle.

- Ghost fill of every fine patch (same-level copies and six-point Lagrange
  prolongation, through two levels): bit-exact, since both sides round the
  paper's midpoint formula operation by operation in the same order; the
  level-0 outer extrapolation within rounding.
- Restriction: bit-exact copies.
- One RK4 step of the TOV star on the five-patch hierarchy from the identical
  state: interiors within 1e-11 per field (the right-hand side tolerance).
- CUDA-graph replay of hierarchy steps equals eager steps bit for bit.
- A layout whose fine ghosts leave the coarser level is rejected.
- Full size (the 366-patch star hierarchy, synthetic table): 12 sampled
  patches of the GPU's ghost fill + con2prim + RHS against the oracle.
"""
import numpy as np
import pytest

import oracle
import synth
from tests._checks import field_err, init_ok, interior, rhs_check, rhs_floor, rhs_report

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2510_13965_gb300 as g  # noqa: E402

NF = 32


def _pair(specs, P=None):
    P = P if P is not None else synth.ideal_params(bc=3)
    pt = g.Patches(P, specs)
    H = oracle.Hierarchy(oracle.Oracle(P), specs)
    return pt, H


def _upload_all(pt, H, reg=0):
    for q in range(len(H.specs)):
        pt.U[q][reg].copy_(torch.as_tensor(H.U[reg][q], device="cuda"))
    torch.cuda.synchronize()


def _ghost_mask(s):
    n = s["n"]
    m = np.ones((n[2] + 6, n[1] + 6, n[0] + 6), dtype=bool)
    m[3:-3, 3:-3, 3:-3] = False
    return m


def test_hierarchy_ghost_fill_matches_oracle():
    specs = synth.small_hierarchy()
    pt, H = _pair(specs)
    rng = np.random.default_rng(21)
    for q in range(len(specs)):
        H.U[1][q][...] = rng.normal(size=H.U[1][q].shape)
    _upload_all(pt, H, reg=1)
    assert H.ghost_fill(1) == 0
    pt.ghost_fill(1)
    pt.synchronize()
    for q, s in enumerate(specs):
        got = pt.U[q][1].cpu().numpy()
        if s["level"] == 0:
            assert np.max(np.abs(got - H.U[1][q])) <= 1e-14 * np.max(np.abs(H.U[1][q]))
        else:
            assert np.array_equal(got, H.U[1][q]), q


def test_hierarchy_restriction_matches_oracle():
    specs = synth.small_hierarchy()
    pt, H = _pair(specs)
    rng = np.random.default_rng(22)
    for q in range(len(specs)):
        H.U[0][q][...] = rng.normal(size=H.U[0][q].shape)
    _upload_all(pt, H, reg=0)
    assert H.restrict(0) == 0
    pt.restrict(0)
    pt.synchronize()
    for q in range(len(specs)):
        assert np.array_equal(pt.U[q][0].cpu().numpy(), H.U[0][q]), q


def _tov_hierarchy():
    specs = synth.small_hierarchy()
    ids = [synth.tov_id(n=s["n"], x0=s["x0"], dx=s["dx"], seed=1 + q, perturb=True, bfield=True)
           for q, s in enumerate(specs)]
    return specs, ids


def test_hierarchy_rk4_step_matches_oracle():
    specs, ids = _tov_hierarchy()
    pt, H = _pair(specs)
    for q, ID in enumerate(ids):
        pt.init_state(q, torch.as_tensor(ID, device="cuda"))
        H.init_state(q, ID)
    pt.synchronize()
    for q, s in enumerate(specs):
        ok, e = init_ok(interior(pt.U[q][0].cpu().numpy(), s["n"]), interior(H.U[0][q], s["n"]), dx=s["dx"])
        assert ok, (q, e)
    _upload_all(pt, H, reg=0)
    dt = 0.25 * specs[-1]["dx"]
    pt.step(dt)
    pt.synchronize()
    assert pt.sync_status() == 0
    assert H.rk4_step(dt) >= 0
    for q, s in enumerate(specs):
        got = interior(pt.U[q][0].cpu().numpy(), s["n"])
        want = interior(H.U[0][q], s["n"])
        err = field_err(got, want)
        small = np.abs(want).reshape(NF, -1).max(axis=1) < 1e-12
        d = np.abs(got - want).reshape(NF, -1).max(axis=1)
        ok = (err < 1e-11) | (small & (d < 1e-14))
        assert np.all(ok), (q, {f: err[f] for f in range(NF) if not ok[f]})


def test_hierarchy_graph_replay_equals_eager():
    specs, ids = _tov_hierarchy()
    P = synth.ideal_params(bc=3)
    a = g.Patches(P, specs)
    b = g.Patches(P, specs)
    for pt in (a, b):
        for q, ID in enumerate(ids):
            pt.init_state(q, torch.as_tensor(ID, device="cuda"))
    dt = 0.25 * specs[-1]["dx"]
    b.capture_graph(2, dt)
    a.step(dt)
    a.step(dt)
    b.graph_launch()
    a.synchronize()
    b.synchronize()
    for q in range(len(specs)):
        assert torch.equal(a.U[q][0], b.U[q][0]), q


def test_per_patch_launches_equal_batched_launches_bitwise():
    """The plain per-patch form (one launch per patch and kernel kind) and the
    batched form (one launch per kernel kind over all patches) compute every
    point identically: two RK4 steps of the hierarchy, eager and graph-replayed,
    plain and NN-seeded, agree bit for bit."""
    specs, ids = _tov_hierarchy()
    P = synth.ideal_params(bc=3)
    S = g.Seeder(seed=3)
    for seeded in (False, True):
        a = g.Patches(P, specs)
        b = g.Patches(P, specs)
        for pt in (a, b):
            for q, ID in enumerate(ids):
                pt.init_state(q, torch.as_tensor(ID, device="cuda"))
            if seeded:
                pt.set_seeder(S, 0.05)
        b.set_per_patch(True)
        dt = 0.25 * specs[-1]["dx"]
        a.step(dt)
        b.step(dt)
        b.capture_graph(1, dt)
        a.step(dt)
        b.graph_launch()
        a.synchronize()
        b.synchronize()
        assert a.sync_status() == 0 and b.sync_status() == 0
        assert b.launch_count() > a.launch_count()
        for q in range(len(specs)):
            assert torch.equal(a.U[q][0], b.U[q][0]), (seeded, q)
            assert torch.equal(a.prim[q], b.prim[q]), (seeded, q)


@pytest.mark.parametrize("layout", ["hierarchy", "uneven"])
def test_every_schedule_gives_the_same_result_bitwise(layout):
    """Tile shapes per patch and kernel kind, persistent pools of blocks, and
    the autotuner's own choice compute every point with the same arithmetic:
    two RK4 steps agree bit for bit with the default schedule (linear chunks,
    one block per work item).  Layouts: the five-patch hierarchy (ragged
    tiles at every patch edge) and 12 uneven frozen-ghost patches of the
    batched configuration's edge set."""
    if layout == "hierarchy":
        specs, ids = _tov_hierarchy()
        P = synth.ideal_params(bc=3)
    else:
        specs = synth.batched_specs(npatch=12, seed=5)
        _, norm = synth.config0_id(n=(32, 32, 32), seed=0, return_norm=True)
        ids = [synth.batched_id(s_, seed=0, norm=norm) for s_ in specs]
        P = synth.ideal_params(bc=2)
    rng = np.random.default_rng(9)
    dt = 0.25 * min(s_["dx"] for s_ in specs)
    runs = []
    for variant in ("default", "random", "tuned"):
        pt = g.Patches(P, specs)
        for q, ID in enumerate(ids):
            pt.init_state(q, torch.as_tensor(ID, device="cuda"))
        pt.synchronize()
        if variant == "random":
            shapes = [tuple(int(v) for v in rng.integers(0, 5, 3)) for _ in specs]
            pt.set_schedule(shapes, (1, 1, 0))
            assert pt.get_schedule() == (shapes, (1, 1, 0))
        elif variant == "tuned":
            U0 = [u[0].clone() for u in pt.U]
            pt.autotune(dt, reps=1)
            for u, u0 in zip(pt.U, U0):
                u[0].copy_(u0)
        pt.step(dt)
        pt.capture_graph(1, dt)
        pt.graph_launch()
        pt.synchronize()
        assert pt.sync_status() == 0
        runs.append(pt)
    for pt in runs[1:]:
        for q in range(len(specs)):
            assert torch.equal(runs[0].U[q][0], pt.U[q][0]), q
            assert torch.equal(runs[0].prim[q], pt.prim[q]), q


@pytest.mark.parametrize("seeded", [False, True], ids=["plain", "nn_seeded"])
def test_scaled_star_hierarchy_steps_match_oracle(seeded):
    """Config 4 at scale 0.25 (the magnetised star with the synthetic table on
    5 levels, 13 patches, 0.49 M interior points): 20 synchronous RK4 steps on
    the GPU through a CUDA graph against the oracle's OpenMP build (bitwise the
    serial oracle) from the identical state, and the oracle's twin from a
    1e-14-perturbed start, the problem's rounding sensitivity (reading A26).
    Per field over all patches (a field spans the hierarchy, reading A44):
    max |gpu - oracle| / max |oracle| within max(1e-9, 10 x the twin's drift).
    The NN-seeded variant runs the patch seeding (atmosphere scan, network on
    the listed points) and the seeded con2prim in every substep of the graph
    against the oracle's plain con2prim."""
    table = synth.make_table()
    P = synth.table_params(table, bc=3)
    specs = synth.amr_tov_layout(scale=0.25)
    prof = synth.tov_profile()
    O = oracle.Oracle(P, table, threads=0)
    H, Ht = oracle.Hierarchy(O, specs), oracle.Hierarchy(O, specs)
    for q, s in enumerate(specs):
        H.init_state(q, synth.tov_id(n=s["n"], x0=s["x0"], dx=s["dx"], seed=4000 + q, table=table,
                                     rho_atmo=P["rho_atmo"], profile=prof))
    assert H.restrict(0) == 0
    rng = np.random.default_rng(7)
    for q in range(len(specs)):
        Ht.U[0][q][...] = H.U[0][q] * (1.0 + 1e-14 * rng.uniform(-1.0, 1.0, H.U[0][q].shape))
    T = g.Table(table)
    pt = g.Patches(P, specs, table=T)
    _upload_all(pt, H, reg=0)
    if seeded:
        st_ = synth.c2p_states(1 << 16, seed=13)
        prim = np.zeros((1 << 16, 10))
        prim[:, 0], prim[:, 7], prim[:, 8] = st_["rho"], st_["ye"], st_["T"]
        prim[:, 3:6] = st_["v"]
        cons = g.prim2con_flat(P, torch.as_tensor(prim, device="cuda"), torch.as_tensor(st_["B"], device="cuda"),
                               table=T)
        _, s0, _, roots, _ = g.c2p_flat_seeded(P, cons, None, table=T)
        keep = s0 >= 0
        S = g.Seeder(seed=2)
        S.train(g.seeder_features(cons)[keep].contiguous(), g.seeder_targets(cons, roots)[keep].contiguous(),
                batch=1024, epochs=8, lr=3e-3, lr_final=3e-5)
        pt.set_seeder(S, 3e-2)
    dt = 0.25 * min(s["dx"] for s in specs)
    pt.capture_graph(1, dt)
    for _ in range(20):
        pt.graph_launch()
        assert H.rk4_step(dt) >= 0
        assert Ht.rk4_step(dt) >= 0
    pt.synchronize()
    assert pt.sync_status() == 0
    d_gpu, d_twin, scale = np.zeros(NF), np.zeros(NF), np.zeros(NF)
    for q, s in enumerate(specs):
        want = interior(H.U[0][q], s["n"]).reshape(NF, -1)
        got = interior(pt.U[q][0].cpu().numpy(), s["n"]).reshape(NF, -1)
        twin = interior(Ht.U[0][q], s["n"]).reshape(NF, -1)
        scale = np.maximum(scale, np.abs(want).max(axis=1))
        d_gpu = np.maximum(d_gpu, np.abs(got - want).max(axis=1))
        d_twin = np.maximum(d_twin, np.abs(twin - want).max(axis=1))
    e_gpu, e_twin = d_gpu / np.maximum(scale, 1e-300), d_twin / np.maximum(scale, 1e-300)
    print("scaled star hierarchy (%s), 20 steps: max over fields GPU %.3g, twin %.3g"
          % ("seeded" if seeded else "plain", e_gpu.max(), e_twin.max()))
    bad = {f: (e_gpu[f], e_twin[f]) for f in range(NF) if not e_gpu[f] <= max(1e-9, 10.0 * e_twin[f])}
    assert not bad, bad


def test_uncovered_fine_ghosts_are_rejected():
    specs = synth.small_hierarchy()
    specs[1] = synth.hierarchy.spec((12, 12, 12), 1, (1, 12, 12), 1.0, (-12.0,) * 3)
    with pytest.raises(g.GrmhdError):
        g.Patches(synth.ideal_params(bc=3), specs)


def test_full_size_hierarchy_sampled_patches():
    """The star hierarchy at full size (366 patches, 31.2 M interior points,
    synthetic table): after the GPU's hierarchy ghost fill, con2prim and
    right-hand side of the whole layout in the batched launches the bench
    times, 12 seeded-random patches are redone by the oracle from the GPU's
    own ghost-filled state: statuses bit-exact, primitives to 1e-10, the
    right-hand side to 1e-11 per field."""
    from tests._checks import prim_check
    table = synth.make_table()
    P = synth.table_params(table, bc=3)
    T = g.Table(table)
    specs = synth.amr_tov_layout(scale=1.0)
    prof = synth.tov_profile()
    pt = g.Patches(P, specs, table=T)
    for q, s in enumerate(specs):
        ID = synth.tov_id(n=s["n"], x0=s["x0"], dx=s["dx"], seed=4000 + q, table=table, rho_atmo=P["rho_atmo"],
                          profile=prof)
        pt.init_state(q, torch.as_tensor(ID, device="cuda"))
        pt.synchronize()
    pt.restrict(0)
    pt.ghost_fill(0)
    pt.synchronize()
    rng = np.random.default_rng(11)
    sample = sorted(int(x) for x in rng.choice(len(specs), 12, replace=False))
    U0 = {q: pt.U[q][0].cpu().numpy().copy() for q in sample}
    pt.con2prim(0)
    rhs = pt.rhs_eval(0)
    pt.synchronize()
    assert pt.sync_status() == 0
    O = oracle.Oracle(P, table, threads=0)  # OpenMP build: bitwise the serial oracle, all host cores
    # Each sampled patch's right-hand side against the oracle's from the same
    # ghost-filled state: every field within max(1e-11 of the patch's largest
    # value, 10 floors), the floor being the oracle's own change under a
    # one-rounding-step move of every input value (tests/_checks.py).  Far
    # from the star the spacetime right-hand sides are cancellations of the
    # tidal terms (A~_ij: ~1e-12 out of ~1e-5); the floor measures that.
    worst = (0.0, 0.0)
    for q in sample:
        s = specs[q]
        Uo = U0[q].copy()
        prim_o, st_o, _, _ = O.con2prim_patch(Uo, s["n"])
        assert np.array_equal(pt.status[q].cpu().numpy(), st_o), q
        prim_check(pt.prim[q].cpu().numpy(), prim_o, pt.status[q].cpu().numpy(), st_o, Uo[22:25])
        want = interior(O.rhs_patch(Uo, prim_o, s["n"], s["dx"]), s["n"])
        got = interior(rhs[q].cpu().numpy(), s["n"])
        floor = rhs_floor(O, U0[q], s["n"], s["dx"], want=want)
        ok, bad = rhs_check(got, want, floor)
        assert ok, (q, bad)
        r = rhs_report(got, want, floor)
        worst = (max(worst[0], r[0]), max(worst[1], r[1]))
    print("hierarchy sampled patches: max error / max|RHS| %.3g, max error / floor %.3g" % worst)
