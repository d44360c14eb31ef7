"""Python binding of libgrmhd.so, the GB300 GRMHD substep library.

Argument marshalling only: every step of the substep runs in the library's
CUDA kernels.  PyTorch provides device memory and a CUDA stream.  There is no
CPU fallback: importing works anywhere, but every call that touches the
library raises if libgrmhd.so cannot be loaded or no CUDA device is present.
Names follow include/grmhd.h.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgrmhd.so")

NF, NP, NID, NG = 32, 10, 26, 3
OK = 0
STATUS = {0: "OK", -1: "ERR_ARG", -2: "ERR_CUDA", -3: "ERR_C2P_FATAL", -4: "ERR_TIMEOUT", -5: "ERR_NONFINITE",
          -6: "ERR_NOMEM", -7: "ERR_SIZE"}

_P_DOUBLES = ["kappa_z", "kappa_c", "kappa_2", "eta", "sigma_ko", "c_b", "kappa_b", "gamma_th", "K_atmo",
              "rho_atmo", "rho_min", "rho_low", "rho_max", "alpha_bh", "W_max", "eps_max", "ye_min", "ye_max",
              "ye_atmo", "T_atmo", "h0", "c2p_xtol"]
_P_INTS = ["eos_kind", "bc", "max_iter", "rk"]


class Params(ctypes.Structure):
    _fields_ = ([(n, ctypes.c_double) for n in _P_DOUBLES] + [(n, ctypes.c_int) for n in _P_INTS] +
                [("npoly", ctypes.c_int), ("reserved2", ctypes.c_int), ("K_poly", ctypes.c_double),
                 ("rho_poly", ctypes.c_double * 3), ("gamma_poly", ctypes.c_double * 4),
                 ("les_c", ctypes.c_double * 4), ("les_rho_min", ctypes.c_double)])


class EosTable(ctypes.Structure):
    _fields_ = [("nr", ctypes.c_int), ("nt", ctypes.c_int), ("ny", ctypes.c_int), ("reserved", ctypes.c_int),
                ("lr0", ctypes.c_double), ("dlr", ctypes.c_double), ("lt0", ctypes.c_double), ("dlt", ctypes.c_double),
                ("ye0", ctypes.c_double), ("dye", ctypes.c_double),
                ("p", ctypes.c_void_p), ("eps", ctypes.c_void_p), ("cs2", ctypes.c_void_p)]


class PatchDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("px", ctypes.c_int), ("level", ctypes.c_int), ("reserved", ctypes.c_int),
                ("x0", ctypes.c_double * 3), ("dx", ctypes.c_double), ("U", ctypes.c_void_p * 4),
                ("prim", ctypes.c_void_p), ("status", ctypes.c_void_p)]


class C2PStats(ctypes.Structure):
    _fields_ = [("points", ctypes.c_longlong), ("iterations", ctypes.c_longlong), ("corrected", ctypes.c_longlong),
                ("failed", ctypes.c_longlong)]


class TrainCfg(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_int), ("epochs", ctypes.c_int), ("lr", ctypes.c_float),
                ("lr_final", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("fit_norm", ctypes.c_int)]


class GrmhdError(RuntimeError):
    pass


_lib = None

_SIGS = {
    "grmhd_abi_version": (ctypes.c_int, []),
    "grmhd_init_patches": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p]),
    "grmhd_init_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "grmhd_ghost_fill": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "grmhd_con2prim": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "grmhd_rhs_eval": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "grmhd_rk_update": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p]),
    "grmhd_rhs_substep": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_double]),
    "grmhd_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    "grmhd_restrict": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "grmhd_set_subcycling": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "grmhd_set_seeder": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double]),
    "grmhd_capture_graph": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_double]),
    "grmhd_graph_launch": (ctypes.c_int, [ctypes.c_void_p]),
    "grmhd_sync_status": (ctypes.c_int, [ctypes.c_void_p]),
    "grmhd_profile": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "grmhd_set_block_sizes": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "grmhd_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_void_p]),
    "grmhd_profile_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "grmhd_launch_count": (ctypes.c_longlong, [ctypes.c_void_p]),
    "grmhd_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "grmhd_destroy": (None, [ctypes.c_void_p]),
    "grmhd_prim2con_flat": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "grmhd_c2p_flat": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "grmhd_rhs_eval_static": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "grmhd_set_per_patch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "grmhd_shard_partition": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "grmhd_shard_plan": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong]),
    "grmhd_init_shard": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                        ctypes.c_void_p]),
    "grmhd_shard_ghost0": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "grmhd_shard_pack": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_longlong,
                                        ctypes.c_void_p]),
    "grmhd_shard_unpack": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_longlong,
                                          ctypes.c_void_p]),
    "grmhd_set_schedule": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "grmhd_get_schedule": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "grmhd_seeder_hold_products": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "grmhd_dfma_probe": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_longlong, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p]),
    "grmhd_seeder_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_ulonglong]),
    "grmhd_seeder_set_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "grmhd_seeder_get_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "grmhd_seeder_features": (ctypes.c_int, [ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "grmhd_seeder_targets": (ctypes.c_int, [ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p]),
    "grmhd_seeder_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p]),
    "grmhd_seeder_grad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "grmhd_seeder_adam": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_float,
                                         ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_void_p]),
    "grmhd_seeder_train": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "grmhd_seeder_infer": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p]),
    "grmhd_seeder_destroy": (None, [ctypes.c_void_p]),
    "grmhd_seeder_status": (ctypes.c_int, [ctypes.c_void_p]),
    "grmhd_c2p_flat_seeded": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
}


def load(path=LIB_PATH):
    """Load libgrmhd.so (raises GrmhdError if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise GrmhdError("libgrmhd.so not built (run __graft_entry__.build()): %s" % path)
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def make_params(d):
    p = Params()
    for n in _P_DOUBLES:
        setattr(p, n, float(d.get(n, 0.0)))
    for n in _P_INTS:
        setattr(p, n, int(d.get(n, 0)))
    p.npoly = int(d.get("npoly", 0))
    p.K_poly = float(d.get("K_poly", 0.0))
    for name, n in (("rho_poly", 3), ("gamma_poly", 4), ("les_c", 4)):
        vals = tuple(d.get(name, ()))
        if len(vals) > n:
            raise ValueError(f"{name} holds at most {n} values")
        for i, v in enumerate(vals):
            getattr(p, name)[i] = float(v)
    p.les_rho_min = float(d.get("les_rho_min", 0.0))
    return p


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise GrmhdError("no CUDA device: the GRMHD library has no CPU path")
    return torch


class Table:
    """EOS table resident in device memory (numpy node arrays from synth.make_table)."""

    def __init__(self, t, device="cuda"):
        torch = _torch()
        self.arrays = [torch.as_tensor(np.ascontiguousarray(t[k]), dtype=torch.float64, device=device)
                       for k in ("p", "eps", "cs2")]
        self.s = EosTable(t["nr"], t["nt"], t["ny"], 0, t["lr0"], t["dlr"], t["lt0"], t["dlt"], t["ye0"], t["dye"],
                          *[a.data_ptr() for a in self.arrays])

    @property
    def ref(self):
        return ctypes.byref(self.s)


def _check(rc, ctx=None, what=""):
    if rc != OK:
        msg = ""
        if ctx:
            m = load().grmhd_last_error(ctx)
            msg = m.decode() if m else ""
        raise GrmhdError("%s failed: %s (%d) %s" % (what, STATUS.get(rc, "?"), rc, msg))


class Patches:
    """A set of patches with device-resident RK registers and a library context.

    specs: list of dicts with n (3 ints), dx, x0 (3 floats), optional level.
    Allocates U (4 registers of [32, n2+6, n1+6, px]), prim, status per patch
    with torch on `device`, and works on its own CUDA stream.
    """

    def __init__(self, params, specs, table=None, device="cuda", pad=1, stream=None):
        torch = _torch()
        self.torch = torch
        L = load()
        self.L = L
        self.params = make_params(params)
        self.table = table
        self.stream = stream if stream is not None else torch.cuda.Stream(device=device)
        self.device = device
        self.specs = []
        self.U, self.prim, self.status = [], [], []
        descs = (PatchDesc * len(specs))()
        for i, s in enumerate(specs):
            n = tuple(int(v) for v in s["n"])
            px = n[0] + 2 * NG
            px = (px + pad - 1) // pad * pad
            shp = (n[2] + 2 * NG, n[1] + 2 * NG, px)
            regs = [torch.zeros((NF,) + shp, dtype=torch.float64, device=device) for _ in range(4)]
            prim = torch.zeros((NP,) + shp, dtype=torch.float64, device=device)
            st = torch.zeros(shp, dtype=torch.int8, device=device)
            self.U.append(regs)
            self.prim.append(prim)
            self.status.append(st)
            d = descs[i]
            d.n[:] = list(n)
            d.px = px
            d.level = int(s.get("level", 0))
            d.x0[:] = [float(v) for v in s.get("x0", (0.0, 0.0, 0.0))]
            d.dx = float(s["dx"])
            for r in range(4):
                d.U[r] = regs[r].data_ptr()
            d.prim = prim.data_ptr()
            d.status = st.data_ptr()
            self.specs.append(dict(n=n, px=px, dx=float(s["dx"]), shape=shp))
        self.descs = descs
        torch.cuda.current_stream().synchronize()
        ctx = ctypes.c_void_p()
        rc = L.grmhd_init_patches(ctypes.byref(ctx), ctypes.byref(self.params), len(specs), descs,
                                  table.ref if table is not None else None, ctypes.c_void_p(self.stream.cuda_stream))
        _check(rc, None, "grmhd_init_patches")
        self.ctx = ctx

    def __del__(self):
        try:
            if getattr(self, "ctx", None):
                self.stream.synchronize()
                self.L.grmhd_destroy(self.ctx)
                self.ctx = None
        except Exception:
            pass

    def _enter(self):
        self.stream.wait_stream(self.torch.cuda.current_stream())

    def _leave(self):
        # The caller's stream waits for the work just enqueued, so it may read
        # the registers, primitives and status arrays without synchronize().
        self.torch.cuda.current_stream().wait_stream(self.stream)

    def synchronize(self):
        self.stream.synchronize()

    def init_state(self, patch, id_tensor):
        self._enter()
        assert id_tensor.dtype == self.torch.float64 and id_tensor.is_contiguous()
        assert tuple(id_tensor.shape) == (NID,) + self.specs[patch]["shape"]
        # The library reads id_tensor on its own stream: keep the caching
        # allocator from handing its memory to another tensor before that.
        id_tensor.record_stream(self.stream)
        _check(self.L.grmhd_init_state(self.ctx, patch, ctypes.c_void_p(id_tensor.data_ptr())), self.ctx,
               "grmhd_init_state")
        self._leave()

    def ghost_fill(self, reg):
        self._enter()
        _check(self.L.grmhd_ghost_fill(self.ctx, reg), self.ctx, "grmhd_ghost_fill")
        self._leave()

    def con2prim(self, reg, stats=False):
        self._enter()
        s = C2PStats()
        _check(self.L.grmhd_con2prim(self.ctx, reg, ctypes.byref(s) if stats else None), self.ctx, "grmhd_con2prim")
        self._leave()
        return dict(points=s.points, iterations=s.iterations, corrected=s.corrected, failed=s.failed) if stats else None

    def rhs_eval(self, reg, out=None):
        """Right-hand side of register reg into per-patch arrays (ghost entries
        stay zero).  The arrays are zero-filled on the caller's current stream,
        so the library's stream waits for that stream only after they are
        allocated; the caller's stream in turn waits for the library's."""
        torch = self.torch
        if out is None:
            out = [torch.zeros((NF,) + sp["shape"], dtype=torch.float64, device=self.device) for sp in self.specs]
        self._enter()
        for t in out:
            t.record_stream(self.stream)
        arr = (ctypes.c_void_p * len(out))(*[t.data_ptr() for t in out])
        _check(self.L.grmhd_rhs_eval(self.ctx, reg, arr), self.ctx, "grmhd_rhs_eval")
        torch.cuda.current_stream().wait_stream(self.stream)
        return out

    def rk_update(self, stage, dt, rhs):
        self._enter()
        for t in rhs:
            t.record_stream(self.stream)
        arr = (ctypes.c_void_p * len(rhs))(*[t.data_ptr() for t in rhs])
        _check(self.L.grmhd_rk_update(self.ctx, stage, float(dt), arr), self.ctx, "grmhd_rk_update")
        self._leave()

    def rhs_substep(self, stage, dt):
        self._enter()
        _check(self.L.grmhd_rhs_substep(self.ctx, stage, float(dt)), self.ctx, "grmhd_rhs_substep")
        self._leave()

    def set_seeder(self, seeder, delta=1e-2):
        """Seed every con2prim of this context with the network (None: plain brackets)."""
        self._seeder = seeder  # keep it alive while the context uses it
        rc = self.L.grmhd_set_seeder(self.ctx, seeder.h if seeder is not None else None, float(delta))
        _check(rc, self.ctx, "grmhd_set_seeder")

    def restrict(self, reg=0):
        self._enter()
        _check(self.L.grmhd_restrict(self.ctx, reg), self.ctx, "grmhd_restrict")
        self._leave()

    def set_subcycling(self, on=True):
        """Sub-cycling in time on a hierarchy (bc 3): step(dt0) then advances
        level l by 2^l steps of dt0 / 2^l (BOR ghosts from the dense output)."""
        self._enter()
        _check(self.L.grmhd_set_subcycling(self.ctx, 1 if on else 0), self.ctx, "grmhd_set_subcycling")

    def step(self, dt):
        self._enter()
        _check(self.L.grmhd_step(self.ctx, float(dt)), self.ctx, "grmhd_step")
        self._leave()

    def capture_graph(self, nsteps, dt):
        self.synchronize()
        _check(self.L.grmhd_capture_graph(self.ctx, int(nsteps), float(dt)), self.ctx, "grmhd_capture_graph")

    def graph_launch(self):
        self._enter()
        _check(self.L.grmhd_graph_launch(self.ctx), self.ctx, "grmhd_graph_launch")
        self._leave()

    def sync_status(self):
        return self.L.grmhd_sync_status(self.ctx)

    KERNEL_KINDS = ("ghost", "c2p", "iflux", "rhs", "rk", "init", "seed", "dense", "les")

    def set_per_patch(self, on=True):
        """One launch per patch and kernel kind (the plain per-patch form) instead of one per kernel kind."""
        _check(self.L.grmhd_set_per_patch(self.ctx, 1 if on else 0), self.ctx, "grmhd_set_per_patch")

    def set_block_sizes(self, bs_c2p, bs_iflux, bs_rhs):
        _check(self.L.grmhd_set_block_sizes(self.ctx, bs_c2p, bs_iflux, bs_rhs), self.ctx, "grmhd_set_block_sizes")

    def set_schedule(self, shapes=None, pers=None):
        """Tile shape per patch and kernel kind (list of (c2p, iflux, rhs) per
        patch, 0..4) and persistent flags (c2p, iflux, rhs = 0)."""
        sh = None if shapes is None else (ctypes.c_int * (3 * len(self.specs)))(*[int(v) for t in shapes for v in t])
        pe = None if pers is None else (ctypes.c_int * 3)(*[int(v) for v in pers])
        _check(self.L.grmhd_set_schedule(self.ctx, sh, pe), self.ctx, "grmhd_set_schedule")

    def get_schedule(self):
        """(shapes per patch [(c2p, iflux, rhs)], persistent flags (c2p, iflux, rhs))."""
        sh = (ctypes.c_int * (3 * len(self.specs)))()
        pe = (ctypes.c_int * 3)()
        _check(self.L.grmhd_get_schedule(self.ctx, sh, pe), self.ctx, "grmhd_get_schedule")
        return [tuple(sh[3 * i:3 * i + 3]) for i in range(len(self.specs))], tuple(pe)

    def autotune(self, dt, reps=2):
        """Block sizes, tile shapes per patch-size class and persistent launches
        from timed trials on these patches; returns the block sizes (c2p, iflux, rhs)."""
        self._enter()
        ch = (ctypes.c_int * 3)()
        _check(self.L.grmhd_autotune(self.ctx, float(dt), int(reps), ch), self.ctx, "grmhd_autotune")
        return tuple(ch)

    def profile(self, on=True):
        _check(self.L.grmhd_profile(self.ctx, 1 if on else 0), self.ctx, "grmhd_profile")

    def profile_read(self):
        """Summed CUDA-event milliseconds and launch counts per kernel kind since profile(True)."""
        k = len(self.KERNEL_KINDS)
        ms = (ctypes.c_double * k)()
        cnt = (ctypes.c_longlong * k)()
        _check(self.L.grmhd_profile_read(self.ctx, ms, cnt, k), self.ctx, "grmhd_profile_read")
        return {n: (ms[i], cnt[i]) for i, n in enumerate(self.KERNEL_KINDS)}

    def launch_count(self):
        return self.L.grmhd_launch_count(self.ctx)


def prim2con_flat(params, prim, B, table=None, stream=None):
    """Conserved (n, 10) from primitives (n, 10) and B (n, 3), device tensors."""
    torch = _torch()
    L = load()
    n = prim.shape[0]
    cons = torch.empty((n, 10), dtype=torch.float64, device=prim.device)
    P = make_params(params)
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = L.grmhd_prim2con_flat(ctypes.byref(P), table.ref if table is not None else None, n,
                               ctypes.c_void_p(prim.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                               ctypes.c_void_p(cons.data_ptr()), ctypes.c_void_p(s.cuda_stream))
    _check(rc, None, "grmhd_prim2con_flat")
    return cons


def _fp64_probe(shapes, iters, reps, add):
    torch = _torch()
    L = load()
    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    sink = torch.zeros(nsm * 8, dtype=torch.float64, device="cuda")
    n = ctypes.c_longlong(0)
    s = torch.cuda.current_stream()
    best, best_shape = 0.0, None
    for bps, ch in shapes:
        for r in range(reps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            rc = L.grmhd_dfma_probe(int(bps), -int(ch) if add else int(ch), int(iters * 8 // ch), _vp(sink),
                                    ctypes.byref(n), ctypes.c_void_p(s.cuda_stream))
            e1.record(s)
            _check(rc, None, "grmhd_dfma_probe")
            torch.cuda.synchronize()
            rate = n.value / (e0.elapsed_time(e1) / 1e3)
            if r and rate > best:
                best, best_shape = rate, (bps, ch)
    return best, best_shape


PROBE_SHAPES = ((2, 8), (4, 8), (8, 8), (4, 16), (8, 4), (2, 16))


def fp64_peak_tflops(iters=4000, reps=3, shapes=PROBE_SHAPES):
    """Measured FP64 throughput of this GPU (TFLOP/s, 2 flops per FMA): the
    library's FMA probe over a few launch shapes (blocks per SM, chains per
    thread), each launch timed with CUDA events on the current stream after
    one untimed launch; the best rate seen.  Returns (TFLOP/s, best shape)."""
    rate, shape = _fp64_probe(shapes, iters, reps, False)
    return 2.0 * rate / 1e12, shape


def fp64_add_rate(iters=4000, reps=3, shapes=PROBE_SHAPES):
    """Measured FP64 addition rate (thread instructions per second), the
    same way with addition chains."""
    return _fp64_probe(shapes, iters, reps, True)[0]


def c2p_flat(params, cons, table=None, iters=False, stream=None, out=None):
    """con2prim of (n, 10) conserved states, flat metric; returns prim, status[, iters]."""
    torch = _torch()
    L = load()
    n = cons.shape[0]
    if out is None:
        prim = torch.empty((n, NP), dtype=torch.float64, device=cons.device)
        status = torch.empty((n,), dtype=torch.int8, device=cons.device)
        it = torch.empty((n,), dtype=torch.int32, device=cons.device) if iters else None
    else:
        prim, status, it = out
    P = make_params(params)
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = L.grmhd_c2p_flat(ctypes.byref(P), table.ref if table is not None else None, n,
                          ctypes.c_void_p(cons.data_ptr()), ctypes.c_void_p(prim.data_ptr()),
                          ctypes.c_void_p(status.data_ptr()),
                          ctypes.c_void_p(it.data_ptr()) if it is not None else None, ctypes.c_void_p(s.cuda_stream))
    _check(rc, None, "grmhd_c2p_flat")
    return (prim, status, it) if iters else (prim, status)


def _vp(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(torch, stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def c2p_flat_seeded(params, cons, seeds=None, delta=1e-2, table=None, stream=None):
    """Flat-metric con2prim with optional seeds (n, 3); returns
    (prim, status, iters, roots, seeded) as device tensors."""
    torch = _torch()
    L = load()
    n = cons.shape[0]
    dev = cons.device
    prim = torch.empty((n, NP), dtype=torch.float64, device=dev)
    status = torch.empty((n,), dtype=torch.int8, device=dev)
    it = torch.empty((n,), dtype=torch.int32, device=dev)
    roots = torch.empty((n, 3), dtype=torch.float64, device=dev)
    sd = torch.empty((n,), dtype=torch.int8, device=dev)
    P = make_params(params)
    rc = L.grmhd_c2p_flat_seeded(ctypes.byref(P), table.ref if table is not None else None, n, _vp(cons),
                                 _vp(seeds), float(delta), _vp(prim), _vp(status), _vp(it), _vp(roots), _vp(sd),
                                 _stream(torch, stream))
    _check(rc, None, "grmhd_c2p_flat_seeded")
    return prim, status, it, roots, sd


class Seeder:
    """The learned con2prim seeder (weights, Adam state and scratch on the device)."""

    NPARAMS = 9091
    NNORM = 22

    def __init__(self, seed=0):
        self._torch = _torch()
        L = load()
        h = ctypes.c_void_p()
        _check(L.grmhd_seeder_create(ctypes.byref(h), int(seed)), None, "grmhd_seeder_create")
        self.h = h

    def __del__(self):
        if getattr(self, "h", None):
            load().grmhd_seeder_destroy(self.h)
            self.h = None

    def set_params(self, params=None, norm=None):
        p = np.ascontiguousarray(params, dtype=np.float32) if params is not None else None
        m = np.ascontiguousarray(norm, dtype=np.float32) if norm is not None else None
        rc = load().grmhd_seeder_set_params(self.h, p.ctypes.data if p is not None else None,
                                            m.ctypes.data if m is not None else None)
        _check(rc, None, "grmhd_seeder_set_params")

    def get_params(self):
        p = np.zeros(self.NPARAMS, dtype=np.float32)
        m = np.zeros(self.NNORM, dtype=np.float32)
        _check(load().grmhd_seeder_get_params(self.h, p.ctypes.data, m.ctypes.data), None, "grmhd_seeder_get_params")
        return p, m

    def forward(self, f, stream=None):
        torch = self._torch
        t = torch.empty((f.shape[0], 3), dtype=torch.float32, device=f.device)
        rc = load().grmhd_seeder_forward(self.h, f.shape[0], _vp(f), _vp(t), _stream(torch, stream))
        _check(rc, None, "grmhd_seeder_forward")
        return t

    def grad(self, f, t, stream=None):
        torch = self._torch
        g = torch.empty((self.NPARAMS,), dtype=torch.float32, device=f.device)
        loss = torch.empty((1,), dtype=torch.float64, device=f.device)
        rc = load().grmhd_seeder_grad(self.h, f.shape[0], _vp(f), _vp(t), _vp(g), _vp(loss), _stream(torch, stream))
        _check(rc, None, "grmhd_seeder_grad")
        return loss, g

    def adam(self, grad, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        rc = load().grmhd_seeder_adam(self.h, _vp(grad), int(step), lr, beta1, beta2, eps,
                                      _stream(self._torch, stream))
        _check(rc, None, "grmhd_seeder_adam")

    def train(self, f, t, batch=4096, epochs=10, lr=3e-3, lr_final=3e-5, beta1=0.9, beta2=0.999, eps=1e-8,
              fit_norm=True, stream=None):
        """Trains on (f, t); returns the per-epoch mean losses (device float64 tensor)."""
        torch = self._torch
        hist = torch.zeros((epochs,), dtype=torch.float64, device=f.device)
        cfg = TrainCfg(batch, epochs, lr, lr_final, beta1, beta2, eps, 1 if fit_norm else 0)
        rc = load().grmhd_seeder_train(self.h, f.shape[0], _vp(f), _vp(t), ctypes.byref(cfg), _vp(hist),
                                       _stream(torch, stream))
        _check(rc, None, "grmhd_seeder_train")
        return hist

    def hold_products(self, polls):
        """Test hook: with polls > 0 the inference kernels issue no tensor-core
        products and every bounded wait for one gives up after `polls` polls."""
        _check(load().grmhd_seeder_hold_products(self.h, int(polls)), None, "grmhd_seeder_hold_products")

    def status(self):
        """0, or raises when an inference kernel timed out waiting for its tensor-core products."""
        _check(load().grmhd_seeder_status(self.h), None, "grmhd_seeder_status")
        return 0

    def infer(self, cons, stream=None):
        """Seeds (n, 3) = (mu_+, mu, W) for flat-metric conserved states (n, 10)."""
        torch = self._torch
        s = torch.empty((cons.shape[0], 3), dtype=torch.float64, device=cons.device)
        rc = load().grmhd_seeder_infer(self.h, cons.shape[0], _vp(cons), _vp(s), _stream(torch, stream))
        _check(rc, None, "grmhd_seeder_infer")
        return s


def seeder_features(cons, stream=None):
    torch = _torch()
    f = torch.empty((cons.shape[0], 8), dtype=torch.float32, device=cons.device)
    _check(load().grmhd_seeder_features(cons.shape[0], _vp(cons), _vp(f), _stream(torch, stream)), None,
           "grmhd_seeder_features")
    return f


def seeder_targets(cons, roots, stream=None):
    torch = _torch()
    t = torch.empty((roots.shape[0], 3), dtype=torch.float32, device=roots.device)
    _check(load().grmhd_seeder_targets(roots.shape[0], _vp(cons), _vp(roots), _vp(t), _stream(torch, stream)), None,
           "grmhd_seeder_targets")
    return t


# ---- sharding a hierarchy across ranks --------------------------------------

def _geometry_descs(specs):
    """Patch descriptors carrying geometry only (no arrays)."""
    d = (PatchDesc * len(specs))()
    for i, s in enumerate(specs):
        n = tuple(int(v) for v in s["n"])
        d[i].n[:] = list(n)
        d[i].px = n[0] + 2 * NG
        d[i].level = int(s.get("level", 0))
        d[i].x0[:] = [float(v) for v in s.get("x0", (0.0, 0.0, 0.0))]
        d[i].dx = float(s["dx"])
    return d


def shard_partition(specs, nranks):
    """Owner rank of every patch (Morton order, balanced by interior points)."""
    d = _geometry_descs(specs)
    owner = (ctypes.c_int * len(specs))()
    _check(load().grmhd_shard_partition(len(specs), d, int(nranks), owner), None, "grmhd_shard_partition")
    return [int(v) for v in owner]


SHARD_LISTS = ("gsend", "grecv", "rsend", "rrecv")


def shard_plan(specs, owner, nranks, rank):
    """(role per patch, lists) for one rank: lists[q][name] is an int32 array
    (m, 2) of (patch, offset) points for peer q, name in SHARD_LISTS (ghost
    phase send / receive, restriction send / receive)."""
    import numpy as np
    L = load()
    n = len(specs)
    d = _geometry_descs(specs)
    own = (ctypes.c_int * n)(*owner)
    role = (ctypes.c_int * n)()
    counts = (ctypes.c_longlong * (4 * nranks))()
    _check(L.grmhd_shard_plan(n, d, own, nranks, rank, role, counts, None, 0), None, "grmhd_shard_plan")
    total = 2 * sum(counts)
    buf = np.zeros(max(total, 1), dtype=np.int32)
    _check(L.grmhd_shard_plan(n, d, own, nranks, rank, role, counts, ctypes.c_void_p(buf.ctypes.data), total), None,
           "grmhd_shard_plan")
    lists, o = [], 0
    for q in range(nranks):
        lq = {}
        for k, name in enumerate(SHARD_LISTS):
            m = counts[4 * q + k]
            lq[name] = buf[o:o + 2 * m].reshape(m, 2).copy()
            o += 2 * m
        lists.append(lq)
    return [int(v) for v in role], lists


def exchange_buffers(send, recv, rank, group=None, tag=0):
    """Point-to-point exchange of packed buffers: send[q] goes to rank q and
    recv[q] is filled from rank q (torch tensors; q == rank is a local copy).
    Works with any torch.distributed backend (NCCL for device tensors, gloo
    for host tensors)."""
    import torch.distributed as dist
    ops = []
    for q, t in recv.items():
        if q != rank and t.numel():
            ops.append(dist.irecv(t, src=q, group=group, tag=tag))
    for q, t in send.items():
        if q != rank and t.numel():
            ops.append(dist.isend(t, dst=q, group=group, tag=tag))
    if rank in send and send[rank].numel():
        recv[rank].copy_(send[rank])
    for op in ops:
        op.wait()


class ShardedHierarchy:
    """This rank's part of a mesh-refinement hierarchy (bc 3) sharded across
    ranks (one GPU each; see grmhd_init_shard): arrays for its own patches and
    for the mirrors its ghost fill reads, and one exchange of source points per
    substep (and one per step for the restriction) through torch.distributed.
    Every rank must call step() with the same dt."""

    def __init__(self, params, specs, rank, nranks, table=None, device="cuda", group=None, stream=None):
        torch = _torch()
        import numpy as np
        self.torch, self.rank, self.nranks, self.group = torch, rank, nranks, group
        self.L = L = load()
        self.params = make_params(params)
        self.rk3 = int(params.get("rk", 0)) == 1
        self.owner = shard_partition(specs, nranks)
        self.role, lists = shard_plan(specs, self.owner, nranks, rank)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=device)
        self.device = device
        self.specs = []
        self.U = [None] * len(specs)
        self.prim = [None] * len(specs)
        self.status = [None] * len(specs)
        descs = _geometry_descs(specs)
        dummy_p = torch.zeros(8, dtype=torch.float64, device=device)
        dummy_s = torch.zeros(8, dtype=torch.int8, device=device)
        self._dummy = (dummy_p, dummy_s)
        for i, s in enumerate(specs):
            n = tuple(int(v) for v in s["n"])
            shp = (n[2] + 2 * NG, n[1] + 2 * NG, n[0] + 2 * NG)
            self.specs.append(dict(n=n, px=n[0] + 2 * NG, dx=float(s["dx"]), shape=shp))
            if self.role[i] == 0:
                continue
            regs = [torch.zeros((NF,) + shp, dtype=torch.float64, device=device) for _ in range(4)]
            self.U[i] = regs
            for r in range(4):
                descs[i].U[r] = regs[r].data_ptr()
            if self.role[i] == 1:
                self.prim[i] = torch.zeros((NP,) + shp, dtype=torch.float64, device=device)
                self.status[i] = torch.zeros(shp, dtype=torch.int8, device=device)
                descs[i].prim = self.prim[i].data_ptr()
                descs[i].status = self.status[i].data_ptr()
            else:  # a mirror is never converted or evolved
                descs[i].prim = dummy_p.data_ptr()
                descs[i].status = dummy_s.data_ptr()
        self.descs = descs
        torch.cuda.current_stream().synchronize()
        own = (ctypes.c_int * len(specs))(*self.owner)
        ctx = ctypes.c_void_p()
        _check(L.grmhd_init_shard(ctypes.byref(ctx), ctypes.byref(self.params), len(specs), descs, own, nranks, rank,
                                  table.ref if table is not None else None, ctypes.c_void_p(self.stream.cuda_stream)),
               None, "grmhd_init_shard")
        self.ctx = ctx
        self._table = table
        self.lists = [{k: torch.as_tensor(np.ascontiguousarray(v), device=device) for k, v in lq.items()}
                      for lq in lists]
        self.points_exchanged = {k: int(sum(lq[k].shape[0] for lq in lists)) for k in SHARD_LISTS}

    def __del__(self):
        try:
            if getattr(self, "ctx", None):
                self.stream.synchronize()
                self.L.grmhd_destroy(self.ctx)
                self.ctx = None
        except Exception:
            pass

    def init_state(self, patch, id_tensor):
        self.stream.wait_stream(self.torch.cuda.current_stream())
        id_tensor.record_stream(self.stream)
        _check(self.L.grmhd_init_state(self.ctx, patch, ctypes.c_void_p(id_tensor.data_ptr())), self.ctx,
               "grmhd_init_state")
        self.torch.cuda.current_stream().wait_stream(self.stream)

    def ghost0(self, reg):
        """Level-0 outer ghosts of register reg (on the level-0 patch's rank)."""
        self.stream.wait_stream(self.torch.cuda.current_stream())
        _check(self.L.grmhd_shard_ghost0(self.ctx, reg), self.ctx, "grmhd_shard_ghost0")

    def pack(self, reg, phase):
        """Send buffers {peer: [32, m] tensor} of register reg for phase "g"
        (ghost sources) or "r" (restriction sources)."""
        torch = self.torch
        name = phase + "send"
        send = {}
        self.stream.wait_stream(torch.cuda.current_stream())
        for q in range(self.nranks):
            ps = self.lists[q][name]
            send[q] = torch.empty((NF, ps.shape[0]), dtype=torch.float64, device=self.device)
            if ps.shape[0]:
                _check(self.L.grmhd_shard_pack(self.ctx, reg, ctypes.c_void_p(ps.data_ptr()), ps.shape[0],
                                               ctypes.c_void_p(send[q].data_ptr())), self.ctx, "grmhd_shard_pack")
        torch.cuda.current_stream().wait_stream(self.stream)
        return send

    def recv_buffers(self, phase):
        name = phase + "recv"
        return {q: self.torch.empty((NF, self.lists[q][name].shape[0]), dtype=self.torch.float64, device=self.device)
                for q in range(self.nranks)}

    def unpack(self, reg, phase, recv):
        """Scatter the received buffers into the mirrors (register reg)."""
        torch = self.torch
        name = phase + "recv"
        self.stream.wait_stream(torch.cuda.current_stream())
        for q in range(self.nranks):
            pr = self.lists[q][name]
            if pr.shape[0]:
                _check(self.L.grmhd_shard_unpack(self.ctx, reg, ctypes.c_void_p(pr.data_ptr()), pr.shape[0],
                                                 ctypes.c_void_p(recv[q].data_ptr())), self.ctx, "grmhd_shard_unpack")
            recv[q].record_stream(self.stream)

    def substep(self, stage, dt):
        _check(self.L.grmhd_rhs_substep(self.ctx, stage, float(dt)), self.ctx, "grmhd_rhs_substep")

    def restrict(self):
        _check(self.L.grmhd_restrict(self.ctx, 0), self.ctx, "grmhd_restrict")
        self.torch.cuda.current_stream().wait_stream(self.stream)

    def stage_registers(self):
        return (0, 1, 2) if self.rk3 else (0, 1, 2, 1)

    def step(self, dt):
        """One RK step of this rank's patches (the exchange protocol of
        grmhd_init_shard), exchanging through torch.distributed."""
        for s, reg in enumerate(self.stage_registers()):
            self.ghost0(reg)
            recv = self.recv_buffers("g")
            exchange_buffers(self.pack(reg, "g"), recv, self.rank, self.group, tag=1)
            self.unpack(reg, "g", recv)
            self.substep(s, dt)
        recv = self.recv_buffers("r")
        exchange_buffers(self.pack(0, "r"), recv, self.rank, self.group, tag=2)
        self.unpack(0, "r", recv)
        self.restrict()

    def synchronize(self):
        self.stream.synchronize()

    def sync_status(self):
        return self.L.grmhd_sync_status(self.ctx)
