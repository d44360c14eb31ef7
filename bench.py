"""Benchmark: GRMHD zone-updates/s on the magnetised TOV star, 128^3 patch.

One step = one full RK4 step (4 fused substeps: ghost fill, con2prim with the
point-wise fluxes, interface fluxes, CCZ4 + MHD right-hand side with the RK
epilogue) of the static TOV star (K = 100, Gamma = 2, rho_c = 1.28e-3) on a
single 128^3 vertex-centred patch covering [-20, 20]^3, with a 1 % seeded
pressure perturbation, a poloidal field and a 1e-10 atmosphere.  A zone-update
is one interior point advanced by one RK4 step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl grmhd|reference]

--impl reference times the CPU oracle (the plain FP64 restatement of the
method used by the tests) on a bounded sub-box of the same workload.  Under
torchrun every rank advances its own star (replicas; no data-path collective).
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GRMHD zone-updates/s (FP64, 1 GB300); con2prim solves/s plain vs NN-seeded"
UNIT = "zone-updates/s"
N_EDGE = 128
DX = 0.3125
X0 = -20.0
WORKLOAD = "tov_magnetised_128^3_rk4_step"

# Algorithmic FP64 flops per unit, counted by the oracle's flop-counting build
# (python -m oracle.count_flops; one substep of a 24^3 sub-box of this workload
# at the same grid spacing; checked by tests/test_flops_figures.py):
#   right-hand side kernel: CCZ4 + gauge + KO + MHD sources + flux difference
#   (6724 per interior point) plus the RK4 combination (128 for stages 0-2,
#   64 for stage 3).
RHS_FLOPS_PER_POINT = 6724.0
RK_FLOPS_PER_POINT = (128.0 * 3 + 64.0) / 4.0
# DRAM bytes (read + write) per interior point of one k_rhs launch, from the
# ncu capture in profiles/launch_list_tov128.md (64^3 case, k_rhs<1, 128, 0>,
# 192.53 + 208.27 MB over 262,144 points), scaled to a launch by its points;
# set to None whenever k_rhs changes until it is captured again.
RHS_TRAFFIC_BYTES_PER_POINT = (192.530176e6 + 208.266752e6) / 64 ** 3
# FP64 peak derived from the unit counts and clocks: 152 SMs x 4 FP64 flops per
# clock per SM x 2070 MHz (nominal GB300 FP64 1.25 TFLOP/s = 152 x 2.07 GHz x 3.97).
# The line's peak is the measured one (the library's FMA throughput probe,
# timed before the timed region); this derived figure is reported beside it.
FP64_PEAK_TFLOPS = 152 * 4 * 2070e6 / 1e12
# FP64 work k_rhs executes per interior point (ncu, thread-level, on the 64^3
# case; profiles/fp64_instruction_mix_substep_kernels_tov64.md): 5264 flops
# (DADD + DMUL + 2 DFMA), fewer than the algorithmic count since the kernel
# shares differences, reciprocals and the Christoffel contraction, issued as
# 3538 FP64 instructions (all of them adds, multiplies or FMAs).
RHS_EXECUTED_FLOPS_PER_POINT = 5264.0
RHS_FP64_INST_PER_POINT = 3538.0
# The other substep kernels' FP64 instructions from the same capture: k_iflux
# 386 per interior point = 380 per interface (65 x 64^2 interfaces per
# launch), k_c2p 529 per interior point = 404 per ghosted point (70^3 points
# per launch), scaled to other sizes by interfaces and ghosted points (the
# same star on the same domain).
IFLUX_FP64_INST_PER_IFACE = 386.0 * 64 ** 3 / (65 * 64 ** 2)
C2P_FP64_INST_PER_POINT = 529.0 * 64 ** 3 / 70 ** 3


def _args():
    a = argparse.ArgumentParser()
    a.add_argument("--gpus", type=int, default=1)
    a.add_argument("--steps", type=int, default=10)
    a.add_argument("--warmup", type=int, default=3)
    a.add_argument("--impl", default="grmhd", choices=["grmhd", "reference"])
    a.add_argument("--no-cpu-baseline", action="store_true")
    a.add_argument("--no-c2p", action="store_true",
                   help="skip the con2prim plain-vs-NN-seeded section of the default line")
    a.add_argument("--e2e-steps", type=int, default=3)
    a.add_argument("--workload", default="tov", choices=["tov", "batched", "c2p", "amr"],
                   help="tov: the 128^3 TOV star (default); batched: 256 uneven patches over 5 levels; "
                        "c2p: con2prim of 2^24 tabulated-EOS states, plain vs NN-seeded; "
                        "amr: tabulated-EOS magnetised star on a 5-level, 366-patch hierarchy")
    a.add_argument("--c2p-states", type=int, default=1 << 24)
    a.add_argument("--train-pairs", type=int, default=1 << 20)
    a.add_argument("--train-epochs", type=int, default=40)
    a.add_argument("--amr-scale", type=float, default=1.0,
                   help="point counts of the hierarchy workload relative to the 366-patch layout")
    a.add_argument("--amr-seeded", action="store_true",
                   help="also time the hierarchy with NN-seeded con2prim")
    a.add_argument("--amr-per-patch", action="store_true",
                   help="also time the hierarchy with one launch per patch and kernel kind")
    a.add_argument("--no-configs", action="store_true",
                   help="default line: skip the batched (256 patches) and hierarchy (366 patches) sections")
    a.add_argument("--amr-delta", type=float, default=3e-2,
                   help="seed bracket half-width of the NN-seeded hierarchy and batched timings")
    a.add_argument("--no-autotune", action="store_true",
                   help="tov workload: keep 128-thread blocks instead of the library's timed choice")
    a.add_argument("--les-cm", type=float, default=0.0,
                   help="tov and amr workloads: LES gradient SGS model with C_M (the paper's default is 8)")
    a.add_argument("--amr-run", type=int, default=0,
                   help="amr workload: then advance this many finest-level steps (the configuration's run is 200; "
                        "with --amr-subcycle as level-0 steps of 2^L of them) and report the central density")
    a.add_argument("--amr-subcycle", action="store_true",
                   help="amr workload: also time sub-cycled steps (BOR) over the same physical time")
    a.add_argument("--edge", type=int, default=N_EDGE,
                   help="interior points per axis (the same [-20,20]^3 star; 128 is the benchmark workload)")
    return a.parse_args()


def _workload_id(seed, edge=N_EDGE):
    import synth
    return synth.tov_id(n=(edge,) * 3, x0=(X0,) * 3, dx=40.0 / edge, seed=seed)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.strip().split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].strip() == "Active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def _schedule_summary(pt):
    """The launch schedule the autotuner kept: per kernel kind, how many
    patches use each tile shape (0 linear chunks, 1 row segments, 2 32x2xb,
    3 16x4xb, 4 8x8xb boxes), and the persistent-pool flags."""
    shapes, pers = pt.get_schedule()
    out = {}
    for k, name in enumerate(("c2p", "iflux", "rhs")):
        hist = {}
        for t in shapes:
            hist[str(t[k])] = hist.get(str(t[k]), 0) + 1
        out[name] = {"tile_shape_patches": hist, "persistent": bool(pers[k])}
    return out


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(ws, x):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _whole_job_rate(ws, steps, units_per_rank_step, ms_max):
    """Units all ranks processed per second, timed by the slowest rank."""
    return ws * steps * units_per_rank_step / (ms_max / 1e3)


def cpu_baseline(n=48, budget_s=8.0):
    """The oracle as it stands on a sub-box of the workload (same dx, star
    centre): its OpenMP build on all host cores (the line's value), and the
    serial build on one core beside it."""
    import oracle
    import synth
    P = synth.ideal_params(bc=1)
    nn = (n, n, n)
    ID = synth.tov_id(n=nn, x0=(-(n // 2) * DX,) * 3, dx=DX, seed=1)
    res = {}
    for threads in (0, None):
        O = oracle.Oracle(P, threads=threads)
        U = O.init_state(ID, nn, DX)
        regs = [U, np.zeros_like(U), np.zeros_like(U), np.zeros_like(U)]
        prim = np.zeros((oracle.NP,) + U.shape[1:])
        st = np.zeros(U.shape[1:], dtype=np.int8)
        steps, t0 = 0, time.perf_counter()
        while True:
            O.rk4_step(regs, prim, st, nn, DX, 0.4 * DX)
            steps += 1
            el = time.perf_counter() - t0
            if el > budget_s or steps >= 50:
                break
        res[threads] = (steps * n ** 3 / el, steps, el, getattr(O, "threads", 1))
    v, steps, el, cores = res[0]
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d RK4 steps of a %d^3 sub-box of the TOV workload (same dx, star centre), the C++ "
                      "oracle's OpenMP build on %d host threads, %.1f s" % (steps, n, cores, el),
            "serial_1_core": {"value": res[None][0], "steps": res[None][1], "seconds": res[None][2]}}


def cpu_baseline_c2p(n=1 << 19):
    """The oracle's flat-metric con2prim (plain brackets) on n states of the
    isolated-con2prim workload made by the oracle's own prim2con: its OpenMP
    build on all host cores (the value), the serial build on one core beside it."""
    import oracle
    import synth
    table = synth.make_table()
    O = oracle.Oracle(synth.table_params(table), table)
    st = synth.c2p_states(n, seed=3)
    cons = np.zeros((n, 10))
    for q in range(n):
        pr = np.zeros(oracle.NP)
        pr[0], pr[7] = st["rho"][q], st["ye"][q]
        e = O.eos_from_T(st["rho"][q], st["T"][q], st["ye"][q])
        pr[1], pr[2] = e[1], e[0]
        pr[3:6] = st["v"][q]
        cons[q, :9] = oracle.prim2con_point(pr, st["B"][q], [1.0, 0, 0, 1.0, 0, 1.0])
    t0 = time.perf_counter()
    O.c2p_flat_ext(cons)
    el = time.perf_counter() - t0
    Op = oracle.Oracle(synth.table_params(table), table, threads=0)
    t0 = time.perf_counter()
    Op.c2p_flat_ext(cons)
    elp = time.perf_counter() - t0
    cores = getattr(Op, "threads", 1)
    return {"value": n / elp, "unit": "con2prim solves/s", "cores": cores, "kind": "oracle",
            "sample": "%d states (seed 3) of the workload, plain brackets, the C++ oracle's OpenMP build on %d "
                      "host threads, %.2f s" % (n, cores, elp),
            "serial_1_core": {"value": n / el, "seconds": el}}


def cpu_baseline_amr(scale=0.25):
    """One RK4 step of the hierarchy workload at a reduced scale on the oracle
    (every level at the finest time step, restriction at the end): its OpenMP
    build on all host cores (the value), the serial build on one core beside it."""
    import oracle
    import synth
    table = synth.make_table()
    P = synth.table_params(table, bc=3)
    specs = synth.amr_tov_layout(scale=scale)
    prof = synth.tov_profile()
    ids = [synth.tov_id(n=s_["n"], x0=s_["x0"], dx=s_["dx"], seed=4000 + q, table=table,
                        rho_atmo=P["rho_atmo"], profile=prof) for q, s_ in enumerate(specs)]
    zones = int(sum(np.prod(s_["n"]) for s_ in specs))
    res = {}
    for threads in (0, None):
        O = oracle.Oracle(P, table, threads=threads)
        H = oracle.Hierarchy(O, specs)
        for q, ID in enumerate(ids):
            H.init_state(q, ID)
        H.restrict(0)
        t0 = time.perf_counter()
        H.rk4_step(0.25 * min(s_["dx"] for s_ in specs))
        el = time.perf_counter() - t0
        res[threads] = (zones / el, el, getattr(O, "threads", 1))
    v, el, cores = res[0]
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "one RK4 step of the %d-patch hierarchy at scale %g (%d interior points), the C++ "
                      "oracle's OpenMP build on %d host threads, %.1f s" % (len(specs), scale, zones, cores, el),
            "serial_1_core": {"value": res[None][0], "seconds": res[None][1]}}


def run_reference(args):
    """The reference arm: the CPU oracle as it stands, its OpenMP build (the
    serial code's point loops on all host cores, bitwise the serial results),
    one RK4 step of a 48^3 sub-box of the TOV workload per bench step."""
    ws, rank, local = _dist()
    if rank != 0:
        return 0
    import oracle
    import synth
    n = 48
    P = synth.ideal_params(bc=1)
    nn = (n, n, n)
    ID = synth.tov_id(n=nn, x0=(-(n // 2) * DX,) * 3, dx=DX, seed=1)
    O = oracle.Oracle(P, threads=0)
    U = O.init_state(ID, nn, DX)
    regs = [U, np.zeros_like(U), np.zeros_like(U), np.zeros_like(U)]
    prim = np.zeros((oracle.NP,) + U.shape[1:])
    st = np.zeros(U.shape[1:], dtype=np.int8)
    for _ in range(args.warmup):
        O.rk4_step(regs, prim, st, nn, DX, 0.4 * DX)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.rk4_step(regs, prim, st, nn, DX, 0.4 * DX)
    el = time.perf_counter() - t0
    value = args.steps * n ** 3 / el
    sample = ("one RK4 step of a %d^3 sub-box of the TOV workload per step (same dx, star centre), oracle's "
              "OpenMP build on %d host threads" % (n, O.threads))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "sample_edge": n, "dx": DX},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_grmhd(args):
    ws, rank, local = _dist()
    import torch
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    _barrier(ws)
    import paper_2510_13965_gb300 as g
    import synth

    P = synth.ideal_params(bc=1)
    if args.les_cm:
        # SGS fluxes on above the error policy's low-density threshold rho_low.
        P["les_c"] = (0.0, 0.0, 0.0, args.les_cm)
        P["les_rho_min"] = P["rho_low"]
    edge = args.edge
    dx = 40.0 / edge
    ID = torch.as_tensor(_workload_id(seed=1 + rank, edge=edge), device="cuda")
    pt = g.Patches(P, [dict(n=(edge,) * 3, dx=dx, x0=(X0,) * 3)])
    pt.init_state(0, ID)
    del ID
    dt = 0.4 * dx
    # Block size per kernel kind from the library's timed candidates (64, 128,
    # 256); it leaves U^n as it is apart from con2prim corrections.
    chosen = (128, 128, 128) if args.no_autotune else pt.autotune(dt, reps=2)
    for _ in range(max(args.warmup, 3)):
        pt.step(dt)
    pt.synchronize()
    rc = pt.sync_status()
    if rc != 0:
        raise SystemExit("warm-up failed: status %d" % rc)

    fp64_peak, peak_shape = g.fp64_peak_tflops()
    fp64_add = g.fp64_add_rate()

    # ---- timed region: K RK4 steps, kernels bracketed by CUDA events ----------
    clocks = Clocks(local) if rank == 0 else None
    pt.profile(True)
    launches0 = pt.launch_count()
    s = pt.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    _barrier(ws)
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(args.steps):
        pt.step(dt)
    e1.record(s)
    torch.cuda.synchronize()
    _barrier(ws)
    ms = e0.elapsed_time(e1)
    launches = pt.launch_count() - launches0
    prof = pt.profile_read()
    pt.profile(False)
    clk = clocks.stop() if clocks else None
    ms_max = _max_over_ranks(ws, ms)
    rc = pt.sync_status()
    if rc != 0:
        raise SystemExit("timed steps failed: status %d" % rc)
    zones = edge ** 3
    value = _whole_job_rate(ws, args.steps, zones, ms_max)

    # ---- end to end: state from pinned host memory, step, state back --------
    host_in = pt.U[0][0].detach().to("cpu").pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    nbytes = host_in.numel() * host_in.element_size()
    # One untimed pass first: the first copies into freshly pinned pages are
    # several times slower than the steady state (measured 15 against 3.2 ms
    # device-to-host for the 616 MB state).
    with torch.cuda.stream(s):
        pt.U[0][0].copy_(host_in, non_blocking=True)
    pt.step(dt)
    with torch.cuda.stream(s):
        host_out.copy_(pt.U[0][0], non_blocking=True)
    s.synchronize()
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.e2e_steps)]
    t0 = time.perf_counter()
    for k in range(args.e2e_steps):
        with torch.cuda.stream(s):
            ev[k][0].record(s)
            pt.U[0][0].copy_(host_in, non_blocking=True)
            ev[k][1].record(s)
        pt.step(dt)
        with torch.cuda.stream(s):
            ev[k][2].record(s)
            host_out.copy_(pt.U[0][0], non_blocking=True)
            ev[k][3].record(s)
        s.synchronize()
    e2e_s = (time.perf_counter() - t0) / args.e2e_steps
    e2e_s = _max_over_ranks(ws, e2e_s)
    h2d_ms = sum(e[0].elapsed_time(e[1]) for e in ev) / args.e2e_steps
    d2h_ms = sum(e[2].elapsed_time(e[3]) for e in ev) / args.e2e_steps
    e2e = {"value": ws * zones / e2e_s, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
           "ms_per_step": 1e3 * e2e_s, "h2d_ms": h2d_ms, "d2h_ms": d2h_ms}

    if rank != 0:
        return 0
    rhs_ms, rhs_n = prof["rhs"]
    avg_rhs_ms = rhs_ms / max(rhs_n, 1)
    flops = (RHS_FLOPS_PER_POINT + RK_FLOPS_PER_POINT) * zones
    achieved = flops / (avg_rhs_ms / 1e3) / 1e12
    tot = sum(v[0] for v in prof.values()) or 1.0
    traffic = RHS_TRAFFIC_BYTES_PER_POINT * zones if RHS_TRAFFIC_BYTES_PER_POINT else None
    executed = RHS_EXECUTED_FLOPS_PER_POINT * zones / (avg_rhs_ms / 1e3) / 1e12
    roofline = {"bound": "alu", "kernel": "k_rhs (CCZ4 + MHD RHS + RK epilogue)", "achieved": achieved,
                "peak": fp64_peak, "unit": "TFLOP/s", "frac": achieved / fp64_peak, "traffic": traffic,
                "peak_source": "measured: FP64 FMA throughput probe (grmhd_dfma_probe), best launch over "
                               "blocks/SM x chains/thread shapes (best %d x %d)" % peak_shape,
                "peak_derived": FP64_PEAK_TFLOPS, "flops_per_point": RHS_FLOPS_PER_POINT + RK_FLOPS_PER_POINT,
                "executed_flops_per_point": RHS_EXECUTED_FLOPS_PER_POINT, "achieved_executed": executed,
                "frac_executed": executed / fp64_peak,
                # FP64 instruction issue: k_rhs's FP64 instructions per second
                # against the faster of the probes' FMA and addition rates.
                "fp64_inst_per_point": RHS_FP64_INST_PER_POINT,
                "fp64_probe_inst_per_s": {"fma": fp64_peak * 1e12 / 2, "add": fp64_add},
                "frac_fp64_issue": RHS_FP64_INST_PER_POINT * zones / (avg_rhs_ms / 1e3) /
                                   max(fp64_peak * 1e12 / 2, fp64_add)}
    # The other substep kernels against the same FP64 instruction rate.
    probe_rate = max(fp64_peak * 1e12 / 2, fp64_add)
    other = {}
    for kind, name, per, units in (("iflux", "k_iflux", IFLUX_FP64_INST_PER_IFACE, (edge + 1) * edge * edge),
                                   ("c2p", "k_c2p", C2P_FP64_INST_PER_POINT, (edge + 6) ** 3)):
        kms, kn = prof.get(kind, (0.0, 0))
        if kn:
            rate = per * units / (kms / kn / 1e3)
            other[name] = {"ms_per_launch": kms / kn, "launches": kn, "fp64_inst_per_unit": per,
                           "units_per_launch": units, "fp64_inst_per_s": rate, "frac_fp64_issue": rate / probe_rate}
    roofline["other_kernels"] = other
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": (WORKLOAD if edge == N_EDGE else "tov_magnetised_%d^3_rk4_step" % edge) +
                       ("_les_cm%g" % args.les_cm if args.les_cm else ""),
                       "n": [edge] * 3, "dx": dx, "domain": "[-20,20]^3",
                       "step": "one RK4 step (4 fused substeps)", "parallelism": "replicas" if ws > 1 else "1 GPU",
                       "block_sizes": {"c2p": chosen[0], "iflux": chosen[1], "rhs": chosen[2]},
                       "schedule": _schedule_summary(pt),
                       "l2": "inputs larger than L2 (616 MB per RK register)"},
            "substeps_per_s": 4 * args.steps * ws / (ms_max / 1e3),
            "kernel_ms_per_step": {k: v[0] / args.steps for k, v in prof.items() if v[1]},
            "kernel_share": {k: v[0] / tot for k, v in prof.items() if v[1]},
            "roofline": roofline, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk}
    del pt, host_in, host_out
    torch.cuda.empty_cache()
    if ws == 1 and not args.no_c2p:
        # The metric's second half: con2prim solves/s, plain vs NN-seeded, on
        # the isolated workload (2^24 states, tabulated EOS), same GPU.
        c = _c2p_measure(args, min(args.steps, 5))
        line["con2prim"] = {
            "workload": c["config"]["workload"], "unit": "con2prim solves/s",
            "plain": c["plain"]["solves_per_s"], "nn_seeded": c["seeded"]["solves_per_s"],
            "speedup_nn_seeded_vs_plain": c["speedup_seeded_vs_plain"], "delta": c["seeded"]["delta"],
            "evaluations_per_state": {"plain": c["plain"]["evaluations_per_state"],
                                      "nn_seeded": c["seeded"]["evaluations_per_state"]},
            "inference_ms": c["seeded"]["inference_ms"], "training_ms": c["training"]["ms"],
            "same_status": c["seeded_vs_plain"]["same_status"],
            "max_rel_rho_diff": c["seeded_vs_plain"]["max_rel_rho_diff"], "clocks": c["clocks"]}
        line["gpu_launches_con2prim"] = c["gpu_launches"]
    if ws == 1 and not args.no_configs and edge == N_EDGE:
        # The other configurations on the same GPU: 256 uneven patches (plain
        # per-patch vs batched vs batched NN-seeded) and the 366-patch star
        # hierarchy (batched vs plain per-patch vs batched NN-seeded), each
        # variant one RK4 step per bench step replayed from a CUDA graph.
        torch.cuda.empty_cache()
        line["batched"] = _batched_measure(args, min(args.steps, 5))
        torch.cuda.empty_cache()
        h, st = _amr_measure(args, min(args.steps, 3), seeded=True, per_patch=True)
        del st
        line["hierarchy"] = h
        torch.cuda.empty_cache()
    if ws == 1 and not args.no_cpu_baseline and edge == N_EDGE:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)
    return 0


def _batched_measure(args, K):
    """Config 2: 256 uneven patches (edges in {16,24,32,48,64} per axis, 5
    levels, frozen ghosts).  Each variant advances the same initial state by
    one RK4 step per bench step, replayed from a CUDA graph:
      plain per-patch: one launch per patch and kernel kind, bracketed con2prim;
      batched: one launch per kernel kind over all patches (autotuned blocks);
      batched NN-seeded: the batched form with the learned con2prim seeder."""
    import torch
    import paper_2510_13965_gb300 as g
    import synth

    P = synth.ideal_params(bc=2)
    specs = synth.batched_specs(npatch=256, seed=2)
    _, norm = synth.config0_id(n=(32, 32, 32), seed=0, return_norm=True)
    zones = int(sum(np.prod(s["n"]) for s in specs))
    dt = 0.4 * min(s["dx"] for s in specs)
    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    batched = g.Patches(P, specs, stream=stream)
    for p_, s_ in enumerate(specs):
        batched.init_state(p_, torch.as_tensor(synth.batched_id(s_, seed=0, norm=norm), device="cuda"))
    batched.synchronize()
    gen_s = time.perf_counter() - t0
    init = [u[0].clone() for u in batched.U]

    def timed(fn, steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    def reset(pt):
        for p_ in range(len(specs)):
            pt.U[p_][0].copy_(init[p_])
        torch.cuda.synchronize()

    for _ in range(max(args.warmup, 3)):
        batched.step(dt)
    reset(batched)
    chosen = batched.autotune(dt, reps=2)
    clocks = Clocks(0)
    ms = {}
    launches = {}
    for name, per_patch in (("plain_per_patch_graph", True), ("batched_graph", False)):
        batched.set_per_patch(per_patch)
        batched.capture_graph(1, dt)
        reset(batched)
        batched.graph_launch()
        reset(batched)
        l0 = batched.launch_count()
        ms[name] = timed(batched.graph_launch, K)
        launches[name] = (batched.launch_count() - l0) // K
    batched.set_per_patch(False)
    rc = batched.sync_status()
    seeded = _batched_seeded(args, g, P, batched, reset, timed, dt, K, ms["plain_per_patch_graph"])
    if seeded is not None:
        ms["batched_graph_nn_seeded"] = seeded["ms_per_step"]
    clk = clocks.stop()
    out = {"workload": "batched_256_uneven_patches_5_levels_rk4_step", "unit": UNIT,
           "patches": len(specs), "interior_points": zones, "edges": list(synth.EDGES), "levels": 5,
           "ghosts": "frozen", "l2": "inputs larger than L2", "steps": K,
           "zone_updates_per_s": {k: zones / (v / 1e3) for k, v in ms.items()},
           "ms_per_step": ms, "launches_per_step": launches,
           "speedup_batched_vs_plain_per_patch": ms["plain_per_patch_graph"] / ms["batched_graph"],
           "autotuned_block_sizes": list(chosen), "schedule": _schedule_summary(batched), "status": rc,
           "setup_s": gen_s, "clocks": clk}
    if seeded is not None:
        out["speedup_batched_nn_seeded_vs_plain_per_patch"] = ms["plain_per_patch_graph"] / seeded["ms_per_step"]
        out["nn_seeded"] = seeded
    return out


def run_batched(args):
    """Config 2 on its own line (see _batched_measure)."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    b = _batched_measure(args, args.steps)
    line = {"metric": METRIC, "value": b["zone_updates_per_s"]["batched_graph"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": b["ms_per_step"]["batched_graph"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": b["workload"], "patches": b["patches"], "interior_points": b["interior_points"],
                       "l2": b["l2"]},
            "batched": b, "gpu_launches": int(b["launches_per_step"]["batched_graph"] * args.steps),
            "clocks": b["clocks"]}
    print(json.dumps(line), flush=True)
    return 0


def _ideal_seeder(g, P, n, epochs, seed=13):
    """A con2prim seeder for the ideal-gas Fourier workload, trained on the GPU
    on n flat-metric pairs the method makes itself: primitives spanning the
    workload's states (rho in [3e-4, 3e-3], W <= 1.03, eps log-uniform in
    [1e-3, 0.3] taken from the sample's temperature column, b^2/rho in
    [1e-4, 2]), their conserved states by the library's prim2con and the
    plain con2prim roots as labels."""
    import torch
    import synth
    st = synth.c2p_states(n, seed=seed, rho=(3e-4, 3e-3), W=(1.0, 1.03), T=(1e-3, 0.3), ye=(0.1, 0.1),
                          b2rho=(1e-4, 2.0))
    prim = torch.zeros((n, 10), dtype=torch.float64)
    prim[:, 0] = torch.from_numpy(st["rho"])
    prim[:, 1] = torch.from_numpy(st["T"])
    prim[:, 7] = torch.from_numpy(st["ye"])
    prim[:, 3:6] = torch.from_numpy(st["v"])
    cons = g.prim2con_flat(P, prim.cuda(), torch.from_numpy(st["B"]).cuda())
    _, status, _, roots, _ = g.c2p_flat_seeded(P, cons, None)
    keep = status >= 0
    f = g.seeder_features(cons)[keep].contiguous()
    t = g.seeder_targets(cons, roots)[keep].contiguous()
    S = g.Seeder(seed=1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    hist = S.train(f, t, batch=4096, epochs=epochs, lr=3e-3, lr_final=3e-5)
    e1.record()
    torch.cuda.synchronize()
    return S, e0.elapsed_time(e1), float(hist[-1])


def _batched_seeded(args, g, P, batched, reset, timed, dt, K, ms_plain):
    """The batched, graph-captured step with NN-seeded con2prim against the
    plain per-patch, bracketed-start form; the primitives of one con2prim of
    the initial state, seeded and plain, are compared point by point."""
    import torch
    S, train_ms, loss = _ideal_seeder(g, P, args.train_pairs, args.train_epochs)
    reset(batched)
    batched.set_seeder(None)
    plain_stats = batched.con2prim(0, stats=True)
    prim_plain = [p.clone() for p in batched.prim]
    st_plain = [s.clone() for s in batched.status]
    reset(batched)
    batched.set_seeder(S, args.amr_delta)
    seeded_stats = batched.con2prim(0, stats=True)
    rel_rho, dv, same = 0.0, 0.0, True
    for a, b, sa, sb in zip(prim_plain, batched.prim, st_plain, batched.status):
        rel_rho = max(rel_rho, float(((a[0] - b[0]).abs() / a[0].abs().clamp_min(1e-300)).max()))
        dv = max(dv, float((a[3:6] * a[6:7] - b[3:6] * b[6:7]).abs().max()))
        same = same and bool(torch.equal(sa, sb))
    del prim_plain, st_plain
    for _ in range(2):
        batched.step(dt)
    reset(batched)
    batched.capture_graph(1, dt)
    ms = timed(batched.graph_launch, K)
    rc = batched.sync_status()
    batched.set_seeder(None)
    return {"ms_per_step": ms, "delta": args.amr_delta, "status": rc, "training_ms": train_ms,
            "train_pairs": args.train_pairs, "final_loss": loss,
            "c2p_iterations_per_point": {"plain": plain_stats["iterations"] / max(plain_stats["points"], 1),
                                         "nn_seeded": seeded_stats["iterations"] / max(seeded_stats["points"], 1)},
            "seeded_vs_plain_c2p": {"max_rel_rho_diff": rel_rho, "max_abs_Wv_diff": dv, "same_status": same},
            "speedup_vs_plain_per_patch": ms_plain / ms}


def _c2p_cons(g, P, T, n, seed):
    """Conserved states of the isolated con2prim workload, made on the GPU from
    seeded primitives (rho, T, Ye, v, B) by the library's prim2con."""
    import torch
    import synth
    st = synth.c2p_states(n, seed=seed)
    prim = torch.zeros((n, 10), dtype=torch.float64)
    prim[:, 0] = torch.from_numpy(st["rho"])
    prim[:, 7] = torch.from_numpy(st["ye"])
    prim[:, 8] = torch.from_numpy(st["T"])
    prim[:, 3:6] = torch.from_numpy(st["v"])
    B = torch.from_numpy(st["B"]).cuda()
    prim = prim.cuda()
    del st
    cons = g.prim2con_flat(P, prim, B, table=T)
    del prim, B
    return cons


def run_c2p(args):
    """con2prim in isolation: 2^24 states, synthetic 256 x 128 x 64 table; the
    seeder trained on 2^20 pairs (seed 13) made on the GPU; plain brackets
    against network seeds (inference included in the seeded time)."""
    line = _c2p_measure(args, args.steps)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_c2p()
    print(json.dumps(line), flush=True)
    return 0


def _c2p_measure(args, K):
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2510_13965_gb300 as g
    import synth

    table = synth.make_table()
    P = synth.table_params(table)
    T = g.Table(table)
    n = args.c2p_states
    s = torch.cuda.current_stream()
    t0 = time.perf_counter()
    cons = _c2p_cons(g, P, T, n, seed=3)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0

    # ---- training pairs and training -------------------------------------
    ntr = args.train_pairs
    ctr = _c2p_cons(g, P, T, ntr, seed=13)
    _, st, _, roots, _ = g.c2p_flat_seeded(P, ctr, None, table=T)
    keep = st >= 0
    f = g.seeder_features(ctr)[keep].contiguous()
    t = g.seeder_targets(ctr, roots)[keep].contiguous()
    del ctr, roots
    S = g.Seeder(seed=1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    hist = S.train(f, t, batch=4096, epochs=args.train_epochs, lr=3e-3, lr_final=3e-5)
    e1.record(s)
    torch.cuda.synchronize()
    train_ms = e0.elapsed_time(e1)
    hist = hist.cpu().numpy()

    # ---- bracket half-width from a validation slice ----------------------
    nval = min(n, 1 << 20)
    cv = cons[:nval]
    sv = S.infer(cv)
    _, _, it_plain_v, _, _ = g.c2p_flat_seeded(P, cv, None, table=T)
    sweep = {}

    def _ms(fn, k=3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fn()
        torch.cuda.synchronize()
        a.record(s)
        for _ in range(k):
            fn()
        b.record(s)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / k

    plain_ms_v = _ms(lambda: g.c2p_flat_seeded(P, cv, None, table=T))
    for d in (3e-3, 1e-2, 3e-2, 1e-1):
        _, _, itv, _, sdv = g.c2p_flat_seeded(P, cv, sv, d, table=T)
        sweep[d] = (float(itv.double().mean()), float(((sdv & 2) > 0).double().mean()),
                    _ms(lambda: g.c2p_flat_seeded(P, cv, sv, d, table=T)))
    delta = min(sweep, key=lambda d: sweep[d][2])  # fastest, not fewest evaluations
    del sv, cv

    # ---- timed: plain and seeded over all n states -------------------------
    out_p = [torch.empty((n, 10), dtype=torch.float64, device="cuda"), torch.empty(n, dtype=torch.int8, device="cuda"),
             torch.empty(n, dtype=torch.int32, device="cuda")]
    out_s = [torch.empty_like(x) for x in out_p] + [torch.empty(n, dtype=torch.int8, device="cuda")]
    seeds = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    L = g.load()
    Pp = g.make_params(P)
    import ctypes

    def plain():
        rc = L.grmhd_c2p_flat_seeded(ctypes.byref(Pp), T.ref, n, g._vp(cons), None, 0.0, g._vp(out_p[0]),
                                     g._vp(out_p[1]), g._vp(out_p[2]), None, None, ctypes.c_void_p(s.cuda_stream))
        assert rc == 0

    def seeded():
        rc = L.grmhd_seeder_infer(S.h, n, g._vp(cons), g._vp(seeds), ctypes.c_void_p(s.cuda_stream))
        rc |= L.grmhd_c2p_flat_seeded(ctypes.byref(Pp), T.ref, n, g._vp(cons), g._vp(seeds), delta, g._vp(out_s[0]),
                                      g._vp(out_s[1]), g._vp(out_s[2]), None, g._vp(out_s[3]),
                                      ctypes.c_void_p(s.cuda_stream))
        assert rc == 0

    def infer_only():
        assert L.grmhd_seeder_infer(S.h, n, g._vp(cons), g._vp(seeds), ctypes.c_void_p(s.cuda_stream)) == 0

    def timed(fn, k):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(s)
        for _ in range(k):
            fn()
        b.record(s)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / k

    for _ in range(max(args.warmup, 3)):
        plain()
        seeded()
    clocks = Clocks(0)
    ms_plain = timed(plain, K)
    ms_seeded = timed(seeded, K)
    ms_infer = timed(infer_only, K)
    clk = clocks.stop()
    torch.cuda.synchronize()
    st_p, st_s = out_p[1], out_s[1]
    same_status = bool(torch.equal(st_p, st_s))
    ok = (st_p == 0) & (st_s == 0)
    rel_rho = float(((out_s[0][:, 0] - out_p[0][:, 0]).abs() / out_p[0][:, 0]).masked_fill(~ok, 0).max())
    ev_plain = float(out_p[2].double().mean())
    ev_seeded = float(out_s[2].double().mean())
    line = {"metric": METRIC, "value": n / (ms_seeded / 1e3), "unit": "con2prim solves/s", "n_gpus": 1, "steps": K,
            "warmup": max(args.warmup, 3), "ms_per_step": ms_seeded, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 (network bf16/fp32)", "data": "synthetic",
            "config": {"workload": "con2prim_2^24_states_table_256x128x64" if n == 1 << 24 else
                       "con2prim_%d_states_table_256x128x64" % n, "states": n, "metric": "flat",
                       "train_pairs": ntr, "train_seed": 13, "state_seed": 3,
                       "l2": "inputs larger than L2 (1.34 GB of conserved states)"},
            "plain": {"solves_per_s": n / (ms_plain / 1e3), "ms": ms_plain, "evaluations_per_state": ev_plain},
            "seeded": {"solves_per_s": n / (ms_seeded / 1e3), "ms": ms_seeded, "inference_ms": ms_infer,
                       "evaluations_per_state": ev_seeded, "delta": delta,
                       "mu_seed_bracket_used": float(((out_s[3] & 2) > 0).double().mean()),
                       "mu_plus_not_solved": float(((out_s[3] & 4) > 0).double().mean())},
            "speedup_seeded_vs_plain": ms_plain / ms_seeded,
            "delta_sweep_on_2^20_states": {str(k): {"evaluations": v[0], "mu_seeded": v[1], "ms": v[2]}
                                           for k, v in sweep.items()},
            "plain_on_sweep_slice": {"evaluations": float(it_plain_v.double().mean()), "ms": plain_ms_v},
            "training": {"ms": train_ms, "pairs": int(f.shape[0]), "epochs": args.train_epochs, "batch": 4096,
                         "loss_first_epoch": float(hist[0]), "loss_last_epoch": float(hist[-1])},
            "seeded_vs_plain": {"same_status": same_status, "max_rel_rho_diff": rel_rho},
            "gpu_launches": 4 * K, "clocks": clk, "setup_s": gen_s}
    return line


def _hierarchy_pairs(g, P, T, pt, n, seed):
    """Conserved flat-metric states for training a seeder on a hierarchy's own
    fluid: n points drawn uniformly from those whose last con2prim solved
    without correction (status 0), their (rho, T, Ye, v^i) and the field
    B^i = Bbar^i chi^(3/2) (undensitized with det gt = 1) put into a flat
    metric by the library's prim2con.  The flat states keep the points'
    density, temperature and composition; W and b^2 move by the conformal
    factor, well inside the spread of the set."""
    import torch
    dev = pt.status[0].device
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    counts = [int((st == 0).sum()) for st in pt.status]
    total = sum(counts)
    if total == 0:
        raise SystemExit("no solved points to train the seeder on")
    take = [n * c // total for c in counts]
    take[counts.index(max(counts))] += n - sum(take)
    prims, Bs = [], []
    for q, k in enumerate(take):
        if k <= 0:
            continue
        idx = torch.nonzero((pt.status[q] == 0).reshape(-1)).squeeze(1)
        idx = idx[torch.randint(idx.numel(), (k,), generator=gen, device=dev)]
        pr = pt.prim[q].reshape(g.NP, -1)[:, idx]
        U = pt.U[q][0].reshape(g.NF, -1)[:, idx]
        prims.append(pr.T)
        Bs.append((U[28:31] * U[12:13] ** 1.5).T)
    prim = torch.cat(prims).contiguous()
    B = torch.cat(Bs).contiguous()
    return g.prim2con_flat(P, prim, B, table=T)


def _amr_measure(args, K, seeded=False, per_patch=False):
    """Config 4: the magnetised TOV star with the synthetic tabulated EOS on a
    fixed 5-level hierarchy (level 0 one 128^3 patch, levels 1-3 160^3 cubes in
    uneven blocks, level 4 a 256^3 cube of 64^3 blocks; 366 patches, ~69 GB of
    device state), advanced without sub-cycling: every substep fills the
    hierarchy's ghosts level by level, then runs con2prim, fluxes and the
    right-hand side; each step ends with the restriction.  One bench step = one
    RK4 step of every level, replayed from a CUDA graph.  Variants, each timed
    from the same state saved after the warm-up: batched (one launch per kernel
    kind over all patches), plain per-patch (one launch per patch and kernel
    kind), batched NN-seeded.  Returns (result, state for further runs)."""
    import torch
    import paper_2510_13965_gb300 as g
    import synth

    table = synth.make_table()
    P = synth.table_params(table, bc=3)
    if args.les_cm:
        # LES gradient SGS model on the table star (numerical pressure
        # derivatives), SGS flux above the error policy's rho_low.
        P["les_c"] = (0.0, 0.0, 0.0, args.les_cm)
        P["les_rho_min"] = P["rho_low"]
    T = g.Table(table)
    specs = synth.amr_tov_layout(scale=args.amr_scale)
    prof = synth.tov_profile()
    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    pt = g.Patches(P, specs, table=T, stream=stream)
    for q, s_ in enumerate(specs):
        ID = synth.tov_id(n=s_["n"], x0=s_["x0"], dx=s_["dx"], seed=4000 + q, table=table,
                          rho_atmo=P["rho_atmo"], profile=prof)
        pt.init_state(q, torch.as_tensor(ID, device="cuda"))
        pt.synchronize()
    pt.restrict(0)
    pt.synchronize()
    setup_s = time.perf_counter() - t0
    zones = int(sum(np.prod(s_["n"]) for s_ in specs))
    dt = 0.25 * min(s_["dx"] for s_ in specs)
    for _ in range(max(args.warmup, 3)):
        pt.step(dt)
    pt.synchronize()
    rc = pt.sync_status()
    if rc != 0:
        raise SystemExit("warm-up failed: status %d" % rc)
    chosen = pt.autotune(dt, reps=1)
    # Every variant restarts from this state (the interface fluxes cost more
    # as the atmosphere picks up motion, so the variants advance the same states).
    snap = [u[0].clone() for u in pt.U] if (seeded or per_patch) else None

    def restore():
        for u, u0 in zip(pt.U, snap):
            u[0].copy_(u0)
        torch.cuda.synchronize()

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed_graph():
        l0 = pt.launch_count()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(K):
            pt.graph_launch()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / K, (pt.launch_count() - l0) // K

    pt.capture_graph(1, dt)
    clocks = Clocks(0)
    ms, launches = timed_graph()
    clk = clocks.stop()
    rc = pt.sync_status()
    # One eager, profiled step for the per-kernel split.
    pt.profile(True)
    pt.step(dt)
    pt.synchronize()
    prof_k = pt.profile_read()
    pt.profile(False)
    tot = sum(v[0] for v in prof_k.values()) or 1.0
    out = {"workload": "tov_table_eos_5_level_hierarchy_%d_patches_rk4_step" % len(specs) +
                       ("_les_cm%g" % args.les_cm if args.les_cm else ""),
           "unit": UNIT, "scale": args.amr_scale, "patches": len(specs), "interior_points": zones,
           "finest_dx": min(s_["dx"] for s_ in specs), "dt": dt, "subcycling": "none",
           "eos": "synthetic table 256x128x64", "l2": "inputs larger than L2", "steps": K,
           "autotuned_block_sizes": list(chosen), "schedule": _schedule_summary(pt),
           "value": zones / (ms / 1e3), "ms_per_step": ms, "launches_per_step": launches,
           "kernel_ms_per_step": {k: v[0] for k, v in prof_k.items() if v[1]},
           "kernel_share": {k: v[0] / tot for k, v in prof_k.items() if v[1]},
           "status": rc, "clocks": clk, "setup_s": setup_s}
    if per_patch:
        restore()
        pt.set_per_patch(True)
        pt.capture_graph(1, dt)
        restore()
        ms_p, launches_p = timed_graph()
        pt.set_per_patch(False)
        out["plain_per_patch"] = {"value": zones / (ms_p / 1e3), "ms_per_step": ms_p, "launches_per_step": launches_p,
                                  "status": pt.sync_status()}
        out["speedup_batched_vs_plain_per_patch"] = ms_p / ms
    if seeded:
        # The same steps with NN-seeded con2prim.  The network is trained on
        # the GPU on 2^20 flat-metric pairs the method makes from this star's
        # own solved points (see _hierarchy_pairs); with the network of the
        # isolated con2prim workload (hot, relativistic states) the seeded
        # step was slower than the plain one.
        cons = _hierarchy_pairs(g, P, T, pt, args.train_pairs, seed=13)
        _, st_, _, roots, _ = g.c2p_flat_seeded(P, cons, None, table=T)
        keep = st_ >= 0
        f = g.seeder_features(cons)[keep].contiguous()
        t = g.seeder_targets(cons, roots)[keep].contiguous()
        del cons, roots
        S = g.Seeder(seed=1)
        S.train(f, t, batch=4096, epochs=args.train_epochs, lr=3e-3, lr_final=3e-5)
        del f, t
        restore()
        pt.set_seeder(None)
        it_plain = pt.con2prim(0, stats=True)
        pt.set_seeder(S, args.amr_delta)
        it_seeded = pt.con2prim(0, stats=True)
        pt.capture_graph(1, dt)
        restore()
        ms_s, launches_s = timed_graph()
        pt.profile(True)
        pt.step(dt)
        pt.synchronize()
        prof_s = pt.profile_read()
        pt.profile(False)
        out["nn_seeded"] = {"value": zones / (ms_s / 1e3), "ms_per_step": ms_s, "delta": args.amr_delta,
                            "launches_per_step": launches_s,
                            "kernel_ms_per_step": {k: v[0] for k, v in prof_s.items() if v[1]},
                            "c2p_iterations_per_point": {
                                "plain": it_plain["iterations"] / max(it_plain["points"], 1),
                                "nn_seeded": it_seeded["iterations"] / max(it_seeded["points"], 1)},
                            "train_pairs": "%d flat-metric pairs from the hierarchy's solved points (seed 13)"
                                           % args.train_pairs,
                            "status": pt.sync_status(), "speedup_vs_plain": ms / ms_s}
        if per_patch:
            out["speedup_batched_nn_seeded_vs_plain_per_patch"] = out["plain_per_patch"]["ms_per_step"] / ms_s
        pt.set_seeder(None)
    del snap
    state = dict(pt=pt, specs=specs, dt=dt, stream=stream, ms=ms, e0=e0, e1=e1)
    return out, state


def run_amr(args):
    """Config 4 on its own line (see _amr_measure), with optional sub-cycled
    timing (--amr-subcycle) and a run of the configuration's length (--amr-run)."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    out, state = _amr_measure(args, args.steps, seeded=args.amr_seeded, per_patch=args.amr_per_patch)
    pt, specs, dt, stream, ms = state["pt"], state["specs"], state["dt"], state["stream"], state["ms"]
    e0, e1 = state["e0"], state["e1"]
    zones = out["interior_points"]
    levels = {}
    for s_ in specs:
        levels.setdefault(s_["level"], [0, 0])
        levels[s_["level"]][0] += 1
        levels[s_["level"]][1] += int(np.prod(s_["n"]))
    subcycled = None
    if args.amr_subcycle:
        # Sub-cycling (Sec. IV C, BOR): level l steps dt0 / 2^l with
        # dt0 = 2^L dt, so every level keeps the synchronous run's Courant
        # factor on its own grid; one bench step = one level-0 step, the same
        # physical time as 2^L synchronous steps.
        pt.set_seeder(None)  # the plain con2prim of the synchronous timing
        nlev = max(levels) + 1
        dt0 = dt * 2 ** (nlev - 1)
        pt.set_subcycling(True)
        pt.step(dt0)
        pt.capture_graph(1, dt0)
        l0 = pt.launch_count()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            pt.graph_launch()
        e1.record(stream)
        torch.cuda.synchronize()
        ms_c = e0.elapsed_time(e1) / args.steps
        lc = pt.launch_count() - l0
        pt.profile(True)
        pt.step(dt0)
        pt.synchronize()
        prof_c = pt.profile_read()
        pt.profile(False)
        updates = sum(v[1] * 2 ** k for k, v in levels.items())
        sync_time_rate = dt / (ms / 1e3)
        subcycled = {"unit": "simulated time per second (code units)",
                     "value": dt0 / (ms_c / 1e3), "synchronous": sync_time_rate,
                     "speedup_vs_synchronous": (dt0 / (ms_c / 1e3)) / sync_time_rate,
                     "ms_per_level0_step": ms_c, "dt0": dt0,
                     "zone_updates_per_s": updates / (ms_c / 1e3), "zone_updates_per_level0_step": updates,
                     "kernel_ms_per_step": {k: v[0] for k, v in prof_c.items() if v[1]},
                     "gpu_launches": int(lc), "status": pt.sync_status()}
        pt.set_subcycling(False)
    run = None
    if args.amr_run > 0:
        # The configuration's run length from the state the timing left: the
        # star's central rest-mass density (the finest level's point at the
        # origin) before and after, and the device status.
        nlev = max(levels) + 1
        pc, ijk = None, None
        for q, s_ in enumerate(specs):
            if s_["level"] != nlev - 1:
                continue
            idx = [int(round(-s_["x0"][a] / s_["dx"])) for a in range(3)]
            if all(0 <= idx[a] < s_["n"][a] for a in range(3)):
                pc, ijk = q, idx
                break
        pt.set_seeder(None)
        pt.con2prim(0)
        pt.synchronize()
        rho0 = float(pt.prim[pc][0, ijk[2] + 3, ijk[1] + 3, ijk[0] + 3])
        sub = bool(args.amr_subcycle)
        per = 2 ** (nlev - 1) if sub else 1
        nstep = max(1, args.amr_run // per)
        pt.set_subcycling(sub)
        pt.capture_graph(1, dt * per)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(nstep):
            pt.graph_launch()
        e1.record(stream)
        torch.cuda.synchronize()
        run_s = e0.elapsed_time(e1) / 1e3
        pt.set_subcycling(False)
        pt.con2prim(0)
        pt.synchronize()
        rho1 = float(pt.prim[pc][0, ijk[2] + 3, ijk[1] + 3, ijk[0] + 3])
        run = {"finest_steps": nstep * per, "subcycled": sub, "simulated_time": nstep * per * dt, "seconds": run_s,
               "rho_c": [rho0, rho1], "rho_c_drift": rho1 / rho0 - 1.0, "status": pt.sync_status()}
    line = {"metric": METRIC, "value": out["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": out["workload"], "scale": args.amr_scale, "patches": len(specs),
                       "interior_points": zones,
                       "levels": {str(k): {"patches": v[0], "points": v[1]} for k, v in sorted(levels.items())},
                       "finest_dx": out["finest_dx"], "dt": dt, "subcycling": "none", "eos": out["eos"],
                       "l2": out["l2"]},
            "hierarchy": out, "gpu_launches": int(out["launches_per_step"] * args.steps), "status": out["status"],
            "clocks": out["clocks"], "setup_s": out["setup_s"]}
    if subcycled is not None:
        line["subcycled"] = subcycled
    if run is not None:
        line["run"] = run
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_amr()
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = _args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "c2p":
        return run_c2p(args)
    if args.workload == "amr":
        return run_amr(args)
    return run_grmhd(args)


if __name__ == "__main__":
    sys.exit(main())
