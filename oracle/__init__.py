"""ctypes wrapper of the CPU oracle (test infrastructure only).

The oracle is a plain, serial FP64 restatement of the paper's GRMHD substep.
Only the tests, the smoke check and the benchmark's CPU-baseline leg use it;
the product (the CUDA library and its binding) never imports this package.
Arrays are numpy float64, C-contiguous, field-major (nf, n2+6, n1+6, px).

Parity unpinned: kappa_2 and the damping, gauge and cleaning constants (see
oracle.hpp): parameter values that no closed form in the paper fixes.
"""
import ctypes
import os

import numpy as np

from . import build as _build

NF, NST, NP = 32, 22, 10
NID = 26

_P_DOUBLES = ["kappa_z", "kappa_c", "kappa_2", "eta", "sigma_ko", "c_b", "kappa_b", "gamma_th", "K_atmo",
              "rho_atmo", "rho_min", "rho_low", "rho_max", "alpha_bh", "W_max", "eps_max", "ye_min", "ye_max",
              "ye_atmo", "T_atmo", "h0", "c2p_xtol"]
_P_INTS = ["eos_kind", "bc", "max_iter", "rk"]


class Params(ctypes.Structure):
    _fields_ = ([(n, ctypes.c_double) for n in _P_DOUBLES] + [(n, ctypes.c_int) for n in _P_INTS] +
                [("npoly", ctypes.c_int), ("pad2_", ctypes.c_int), ("K_poly", ctypes.c_double),
                 ("rho_poly", ctypes.c_double * 3), ("gamma_poly", ctypes.c_double * 4),
                 ("les_c", ctypes.c_double * 4), ("les_rho_min", ctypes.c_double)])


class EosTable(ctypes.Structure):
    _fields_ = [("nr", ctypes.c_int), ("nt", ctypes.c_int), ("ny", ctypes.c_int), ("pad_", ctypes.c_int),
                ("lr0", ctypes.c_double), ("dlr", ctypes.c_double), ("lt0", ctypes.c_double),
                ("dlt", ctypes.c_double), ("ye0", ctypes.c_double), ("dye", ctypes.c_double),
                ("p", ctypes.c_void_p), ("eps", ctypes.c_void_p), ("cs2", ctypes.c_void_p)]


def make_params(d):
    p = Params()
    for n in _P_DOUBLES:
        setattr(p, n, float(d.get(n, 0.0)))
    for n in _P_INTS:
        setattr(p, n, int(d.get(n, 0)))
    p.npoly = int(d.get("npoly", 0))
    p.K_poly = float(d.get("K_poly", 0.0))
    for i, v in enumerate(d.get("rho_poly", ())):
        p.rho_poly[i] = float(v)
    for i, v in enumerate(d.get("gamma_poly", ())):
        p.gamma_poly[i] = float(v)
    for i, v in enumerate(d.get("les_c", ())):
        p.les_c[i] = float(v)
    p.les_rho_min = float(d.get("les_rho_min", 0.0))
    return p


class _Table:
    """Keeps the numpy node arrays alive while the C struct points at them."""

    def __init__(self, t):
        self.arrays = [np.ascontiguousarray(t[k], dtype=np.float64) for k in ("p", "eps", "cs2")]
        self.s = EosTable(t["nr"], t["nt"], t["ny"], 0, t["lr0"], t["dlr"], t["lt0"], t["dlt"], t["ye0"], t["dye"],
                          *[a.ctypes.data for a in self.arrays])


def make_table(t):
    return None if t is None else _Table(t)


_libs = {}


def lib(flops=False, omp=False):
    """The plain serial build, the flop-counting build (flops) or the OpenMP
    build of the same sources (omp: point loops on several host threads,
    bitwise the serial build's results)."""
    assert not (flops and omp)
    name = "liboracle_flops.so" if flops else ("liboracle_omp.so" if omp else "liboracle.so")
    if name not in _libs:
        _build.build()
        L = ctypes.CDLL(os.path.join(os.path.dirname(os.path.abspath(__file__)), name))
        d, i, l, vp = ctypes.c_double, ctypes.c_int, ctypes.c_long, ctypes.c_void_p
        sig = {
            "oracle_flop_counter": (ctypes.c_longlong, [i]),
            "oracle_set_threads": (i, [i]),
            "oracle_ghost_fill": (i, [vp, vp, i, vp, i]),
            "oracle_init_state": (i, [vp, vp, vp, i, d, vp, vp]),
            "oracle_con2prim_patch": (i, [vp, vp, vp, i, vp, vp, vp, vp]),
            "oracle_rhs_patch": (i, [vp, vp, vp, i, d, vp, vp, vp]),
            "oracle_rhs_points": (i, [vp, vp, vp, i, d, vp, vp, i, vp, vp]),
            "oracle_geom_point": (i, [vp, vp, i, d, vp, vp, i, i, i, vp, vp, vp, vp]),
            "oracle_substep": (i, [vp, vp, vp, i, d, i, d, vp, vp, vp, vp, vp, vp]),
            "oracle_rk4_step": (i, [vp, vp, vp, i, d, d, vp, vp, vp, vp, vp, vp]),
            "oracle_substep_counted": (i, [vp, vp, vp, i, d, i, d, vp, vp, vp, vp, vp, vp, vp]),
            "oracle_c2p_point": (i, [vp, vp, vp, vp, d, d, vp, vp, vp]),
            "oracle_c2p_flat": (i, [vp, vp, l, vp, vp, vp, vp]),
            "oracle_c2p_flat_ext": (i, [vp, vp, l, vp, vp, vp, vp, vp, d, vp, vp]),
            "oracle_c2p_master_scan": (d, [vp, vp, vp, l, vp]),
            "oracle_mlp_nparams": (i, []),
            "oracle_mlp_forward": (i, [vp, l, vp, vp, i]),
            "oracle_mlp_grad": (d, [vp, l, vp, vp, vp, i]),
            "oracle_adam": (i, [vp, vp, vp, vp, l, d, d, d, d, i]),
            "oracle_seeder_features": (i, [l, vp, vp]),
            "oracle_hier_ghost_fill": (i, [vp, i, vp, vp, vp]),
            "oracle_hier_ghost_fill_from": (i, [vp, i, vp, vp, vp, i]),
            "oracle_hier_restrict": (i, [i, vp, vp, vp]),
            "oracle_hier_rk4_step": (i, [vp, vp, i, vp, vp, d, vp, vp, vp, vp, vp, vp]),
            "oracle_eos_derivs": (i, [vp, vp, d, d, d, vp]),
            "oracle_les_flux_points": (i, [vp, vp, vp, i, d, vp, vp, i, vp, i, vp]),
            "oracle_hier_rk4_step_mask": (i, [vp, vp, i, vp, vp, d, vp, vp, vp, vp, vp, vp, i]),
            "oracle_hier_subcycle_step": (i, [vp, vp, i, vp, vp, d, vp, vp, vp, vp, vp, vp]),
            "oracle_dense_derivs": (None, [i, vp, vp]),
            "oracle_bor_coeffs": (None, [i, i, i, i, vp]),
            "oracle_seeder_targets": (i, [l, vp, vp, vp]),
            "oracle_prim2con_point": (i, [vp, vp, vp, vp]),
            "oracle_eos_from_eps": (i, [vp, vp, d, d, d, vp]),
            "oracle_eos_from_T": (i, [vp, vp, d, d, d, vp]),
            "oracle_fd_d1": (d, [vp, d]),
            "oracle_fd_d2": (d, [vp, d]),
            "oracle_fd_d11": (d, [vp, l, d]),
            "oracle_fd_up": (d, [vp, d, d]),
            "oracle_fd_ko": (d, [vp, d, d]),
            "oracle_mp5": (d, [vp]),
            "oracle_minmod4": (d, [d, d, d, d]),
            "oracle_fast_speeds": (i, [d, d, d, d, d, d, vp, vp]),
            "oracle_flux_point": (i, [vp, vp, vp, i, vp, vp]),
            "oracle_matter_point": (i, [vp, vp, vp, vp, vp]),
        }
        for fn, (res, args) in sig.items():
            f = getattr(L, fn)
            f.restype = res
            f.argtypes = args
        _libs[name] = L
    return _libs[name]


def _p(a):
    return a.ctypes.data if a is not None else None


def _ref(x):
    return ctypes.byref(x) if x is not None else None


def _chk(a, dtype=np.float64):
    assert a.dtype == dtype and a.flags["C_CONTIGUOUS"]
    return a


def _n3(n):
    return (ctypes.c_int * 3)(*[int(v) for v in n])


class Oracle:
    """Oracle bound to one parameter set (and optional EOS table)."""

    def __init__(self, params, table=None, flops=False, threads=None):
        """threads: None for the serial build; n >= 1 for the OpenMP build on
        n host threads (0: the OpenMP default)."""
        self.L = lib(flops, omp=threads is not None)
        if threads is not None:
            self.threads = self.L.oracle_set_threads(int(threads))
        self.P = make_params(params)
        self.T = make_table(table)
        self.Tp = _ref(self.T.s) if self.T is not None else None

    # ---- patch operations --------------------------------------------------
    def ghost_fill(self, U, n):
        _chk(U)
        self.L.oracle_ghost_fill(_ref(self.P), _n3(n), U.shape[-1], _p(U), U.shape[0])

    def init_state(self, ID, n, dx):
        _chk(ID)
        U = np.zeros((NF,) + ID.shape[1:])
        self.L.oracle_init_state(_ref(self.P), self.Tp, _n3(n), ID.shape[-1], dx, _p(ID), _p(U))
        return U

    def con2prim_patch(self, U, n):
        _chk(U)
        prim = np.zeros((NP,) + U.shape[1:])
        status = np.zeros(U.shape[1:], dtype=np.int8)
        its = ctypes.c_long(0)
        worst = self.L.oracle_con2prim_patch(_ref(self.P), self.Tp, _n3(n), U.shape[-1], _p(U), _p(prim),
                                             _p(status), ctypes.byref(its))
        return prim, status, worst, its.value

    def rhs_patch(self, U, prim, n, dx):
        rhs = np.zeros_like(U)
        self.L.oracle_rhs_patch(_ref(self.P), self.Tp, _n3(n), U.shape[-1], dx, _p(_chk(U)), _p(_chk(prim)), _p(rhs))
        return rhs

    def rhs_points(self, U, prim, n, dx, ijk):
        ijk = np.ascontiguousarray(ijk, dtype=np.int32)
        out = np.zeros((ijk.shape[0], NF))
        self.L.oracle_rhs_points(_ref(self.P), self.Tp, _n3(n), U.shape[-1], dx, _p(_chk(U)), _p(_chk(prim)),
                                 ijk.shape[0], _p(ijk), _p(out))
        return out

    def geom_point(self, U, prim, n, dx, i, j, k):
        R = np.zeros(6)
        Rtr = np.zeros(1)
        Gt = np.zeros(3)
        Z = np.zeros(3)
        self.L.oracle_geom_point(_ref(self.P), _n3(n), U.shape[-1], dx, _p(_chk(U)), _p(_chk(prim)), i, j, k,
                                 _p(R), _p(Rtr), _p(Gt), _p(Z))
        return R, Rtr[0], Gt, Z

    def substep(self, regs, prim, status, n, dx, stage, dt):
        Un, Ua, Ub, acc = regs
        return self.L.oracle_substep(_ref(self.P), self.Tp, _n3(n), Un.shape[-1], dx, stage, dt, _p(Un), _p(Ua),
                                     _p(Ub), _p(acc), _p(prim), _p(status))

    def substep_counted(self, regs, prim, status, n, dx, stage, dt):
        """Substep plus flop counts [con2prim, pointwise fluxes, interface fluxes, local RHS, RK]."""
        Un, Ua, Ub, acc = regs
        c = np.zeros(5, dtype=np.int64)
        self.L.oracle_substep_counted(_ref(self.P), self.Tp, _n3(n), Un.shape[-1], dx, stage, dt, _p(Un), _p(Ua),
                                      _p(Ub), _p(acc), _p(prim), _p(status), _p(c))
        return c

    def rk4_step(self, regs, prim, status, n, dx, dt):
        Un, Ua, Ub, acc = regs
        return self.L.oracle_rk4_step(_ref(self.P), self.Tp, _n3(n), Un.shape[-1], dx, dt, _p(Un), _p(Ua),
                                      _p(Ub), _p(acc), _p(prim), _p(status))

    # ---- pointwise ---------------------------------------------------------
    def c2p_point(self, cons_bar, gt, chi, alpha):
        cb = np.ascontiguousarray(cons_bar, dtype=np.float64)
        g = np.ascontiguousarray(gt, dtype=np.float64)
        prim = np.zeros(NP)
        co = np.zeros(10)
        it = ctypes.c_int(0)
        st = self.L.oracle_c2p_point(_ref(self.P), self.Tp, _p(cb), _p(g), chi, alpha, _p(prim), _p(co),
                                     ctypes.byref(it))
        return st, prim, co, it.value

    def c2p_flat(self, cons):
        cons = np.ascontiguousarray(cons, dtype=np.float64)
        n = cons.shape[0]
        prim = np.zeros((n, NP))
        status = np.zeros(n, dtype=np.int8)
        iters = np.zeros(n, dtype=np.int32)
        self.L.oracle_c2p_flat(_ref(self.P), self.Tp, n, _p(cons), _p(prim), _p(status), _p(iters))
        return prim, status, iters

    def c2p_flat_ext(self, cons, seeds=None, delta=0.0):
        """Flat-metric con2prim with optional seeds (n, 3): prim, status, iters, roots (n, 3), seeded mask."""
        cons = np.ascontiguousarray(cons, dtype=np.float64)
        n = cons.shape[0]
        prim = np.zeros((n, NP))
        status = np.zeros(n, dtype=np.int8)
        iters = np.zeros(n, dtype=np.int32)
        roots = np.zeros((n, 3))
        seeded = np.zeros(n, dtype=np.int8)
        sd = None if seeds is None else np.ascontiguousarray(seeds, dtype=np.float64)
        self.L.oracle_c2p_flat_ext(_ref(self.P), self.Tp, n, _p(cons), _p(prim), _p(status), _p(iters), _p(sd),
                                   float(delta), _p(roots), _p(seeded))
        return prim, status, iters, roots, seeded

    def c2p_master_scan(self, cons, n):
        """Master function of one flat-metric state (10,) at mu_+ k / n,
        k = 1..n: returns (mu_+, f (n,)); mu_+ = 0 for a state below rho_min."""
        cons = np.ascontiguousarray(cons, dtype=np.float64)
        f = np.zeros(n)
        mu_plus = self.L.oracle_c2p_master_scan(_ref(self.P), self.Tp, _p(cons), int(n), _p(f))
        return mu_plus, f

    def eos_derivs(self, rho, eps, ye):
        """(dp/drho|eps, dp/deps|rho, dp/dYe) of the EOS at one state."""
        out = np.zeros(3)
        if self.L.oracle_eos_derivs(_ref(self.P), self.Tp, float(rho), float(eps), float(ye), _p(out)):
            raise ValueError("no pressure derivatives for this EOS")
        return out

    def les_flux_points(self, U, prim, n, dx, ijk, d):
        """LES SGS flux vectors along d at points ijk ([m][3] ints): [m][10]."""
        n3 = _n3(n)
        U = _chk(U)
        prim = _chk(prim)
        pts = np.ascontiguousarray(ijk, dtype=np.int32)
        out = np.zeros((pts.shape[0], 10))
        rc = self.L.oracle_les_flux_points(_ref(self.P), self.Tp, n3, U.shape[-1], dx, _p(U), _p(prim), pts.shape[0],
                                           _p(pts), int(d), _p(out))
        if rc:
            raise ValueError("LES terms need the EOS's pressure derivatives (a table kind needs its table)")
        return out

    def eos_from_eps(self, rho, eps, ye):
        out = np.zeros(4)
        self.L.oracle_eos_from_eps(_ref(self.P), self.Tp, rho, eps, ye, _p(out))
        return out  # p, eps, T, cs2

    def eos_from_T(self, rho, T, ye):
        out = np.zeros(4)
        self.L.oracle_eos_from_T(_ref(self.P), self.Tp, rho, T, ye, _p(out))
        return out

    def flux_point(self, U32, prim, d):
        U32 = np.ascontiguousarray(U32, dtype=np.float64)
        prim = np.ascontiguousarray(prim, dtype=np.float64)
        F = np.zeros(10)
        lam = np.zeros(1)
        self.L.oracle_flux_point(_ref(self.P), _p(U32), _p(prim), d, _p(F), _p(lam))
        return F, lam[0]

    def flops(self, reset=True):
        return self.L.oracle_flop_counter(1 if reset else 0)


def prim2con_point(prim, B, gdd):
    pr = np.ascontiguousarray(prim, dtype=np.float64)
    b = np.ascontiguousarray(B, dtype=np.float64)
    g = np.ascontiguousarray(gdd, dtype=np.float64)
    out = np.zeros(9)
    lib().oracle_prim2con_point(_p(pr), _p(b), _p(g), _p(out))
    return out


def matter_point(U32, prim):
    U32 = np.ascontiguousarray(U32, dtype=np.float64)
    prim = np.ascontiguousarray(prim, dtype=np.float64)
    E = np.zeros(1)
    S = np.zeros(3)
    Sij = np.zeros(6)
    lib().oracle_matter_point(_p(U32), _p(prim), _p(E), _p(S), _p(Sij))
    return E[0], S, Sij


def fast_speeds(alpha, betad, gudd, vd, v2, a2):
    lp, lm = ctypes.c_double(), ctypes.c_double()
    lib().oracle_fast_speeds(alpha, betad, gudd, vd, v2, a2, ctypes.byref(lp), ctypes.byref(lm))
    return lp.value, lm.value


def fd(kind, u, *args):
    u = np.ascontiguousarray(u, dtype=np.float64)
    f = getattr(lib(), "oracle_fd_" + kind)
    c = u.size // 2
    ptr = u.ctypes.data + 8 * c
    return f(ptr, *args)


def fd_d11(u2d, dx):
    """D_y(D_x u) at the centre of a 5x5 (or larger, odd) 2-D array u[y, x]."""
    u = np.ascontiguousarray(u2d, dtype=np.float64)
    cy, cx = u.shape[0] // 2, u.shape[1] // 2
    ptr = u.ctypes.data + 8 * (cy * u.shape[1] + cx)
    return lib().oracle_fd_d11(ptr, u.shape[1], dx)


def mlp_forward(params, x, bf16=True):
    p = np.ascontiguousarray(params, dtype=np.float32)
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.zeros((x.shape[0], 3))
    lib().oracle_mlp_forward(_p(p), x.shape[0], _p(x), _p(y), 1 if bf16 else 0)
    return y


def mlp_grad(params, x, t, bf16=True):
    """(loss, grad) of the mean-squared error; grad has the parameter layout."""
    p = np.ascontiguousarray(params, dtype=np.float32)
    x = np.ascontiguousarray(x, dtype=np.float32)
    t = np.ascontiguousarray(t, dtype=np.float32)
    g = np.zeros(p.size)
    loss = lib().oracle_mlp_grad(_p(p), x.shape[0], _p(x), _p(t), _p(g), 1 if bf16 else 0)
    return loss, g


def adam(w, m, v, g, lr, b1, b2, eps, t):
    w, m, v = (np.ascontiguousarray(a, dtype=np.float64) for a in (w, m, v))
    g = np.ascontiguousarray(g, dtype=np.float64)
    lib().oracle_adam(_p(w), _p(m), _p(v), _p(g), w.size, lr, b1, b2, eps, t)
    return w, m, v


MLP_NPARAMS = 9091


def seeder_features(cons):
    """Seeder features [n][8] (float64) of flat-metric conserved states [n][10]."""
    c = np.ascontiguousarray(cons, dtype=np.float64)
    f = np.zeros((c.shape[0], 8))
    lib().oracle_seeder_features(c.shape[0], _p(c), _p(f))
    return f


def seeder_targets(cons, roots):
    """Seeder targets [n][3] (float64) of states [n][10] from roots [n][3] = (mu_+, mu, W)."""
    c = np.ascontiguousarray(cons, dtype=np.float64)
    r = np.ascontiguousarray(roots, dtype=np.float64)
    t = np.zeros((r.shape[0], 3))
    lib().oracle_seeder_targets(r.shape[0], _p(c), _p(r), _p(t))
    return t


def dense_derivs(rk, k):
    """(D_1, D_2, D_3, J): D_m = dt^m d^m U/dt^m at t^n from one step's k_j = dt f
    (dense output, Sec. III A), J = 4 (k3 - k2) ~ dt^3 f_U U'' (RK4; 0 for SSP-RK3)."""
    kk = np.zeros(4)
    kk[:len(k)] = k
    D = np.zeros(4)
    lib().oracle_dense_derivs(int(rk), _p(kk), _p(D))
    return D


def bor_coeffs(rk, msub, R, s):
    """Coefficients of (U^n, D_1, D_2, D_3, J) in the BOR stage value of stage s of fine step msub of R."""
    c = np.zeros(5)
    lib().oracle_bor_coeffs(int(rk), int(msub), int(R), int(s), _p(c))
    return c


def mp5(f5):
    f = np.ascontiguousarray(f5, dtype=np.float64)
    return lib().oracle_mp5(_p(f))


def minmod4(a, b, c, d):
    return lib().oracle_minmod4(a, b, c, d)


class Hierarchy:
    """A fixed mesh-refinement hierarchy of patches held by the oracle.

    specs: list of dicts with n (3 ints), level, o (3 ints: origin index on the
    level's grid, which starts at the level-0 origin) and dx.  Arrays per patch
    and register: float64 (NF, n2+6, n1+6, px) with px = n0 + 6.
    """

    def __init__(self, oracle, specs):
        self.O = oracle
        self.specs = specs
        np_ = len(specs)
        self.meta = np.zeros((np_, 8), dtype=np.int32)
        for q, s in enumerate(specs):
            n = s["n"]
            self.meta[q] = [n[0], n[1], n[2], n[0] + 6, s["level"], s["o"][0], s["o"][1], s["o"][2]]
        self.dx = np.array([s["dx"] for s in specs], dtype=np.float64)
        self.U = [[np.zeros((NF, s["n"][2] + 6, s["n"][1] + 6, s["n"][0] + 6)) for s in specs] for _ in range(4)]
        self.prim = [np.zeros((NP,) + self.U[0][q].shape[1:]) for q in range(np_)]
        self.status = [np.zeros(self.U[0][q].shape[1:], dtype=np.int8) for q in range(np_)]

    def _ptrs(self, arrs):
        return (ctypes.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])

    def init_state(self, q, ID):
        self.U[0][q][...] = self.O.init_state(np.ascontiguousarray(ID), self.specs[q]["n"], self.specs[q]["dx"])

    def ghost_fill(self, reg=0, lmin=0):
        """Ghost fill of the hierarchy; lmin >= 1 starts at that level and
        leaves the level-0 patch's outer ghosts untouched."""
        return self.O.L.oracle_hier_ghost_fill_from(_ref(self.O.P), len(self.specs), _p(self.meta), _p(self.dx),
                                                   self._ptrs(self.U[reg]), int(lmin))

    def restrict(self, reg=0):
        return self.O.L.oracle_hier_restrict(len(self.specs), _p(self.meta), _p(self.dx), self._ptrs(self.U[reg]))

    def subcycle_step(self, dt0):
        """One level-0 step of dt0 with sub-cycling (level l: 2^l steps of dt0 / 2^l)."""
        return self.O.L.oracle_hier_subcycle_step(_ref(self.O.P), self.O.Tp, len(self.specs), _p(self.meta),
                                                 _p(self.dx), dt0, self._ptrs(self.U[0]), self._ptrs(self.U[1]),
                                                 self._ptrs(self.U[2]), self._ptrs(self.U[3]),
                                                 self._ptrs(self.prim), self._ptrs(self.status))

    def rk4_step(self, dt, rmask=-1):
        """One step of dt on every level; afterwards level l >= 1 is restricted
        into l - 1 when bit l of rmask is set (default: all levels)."""
        return self.O.L.oracle_hier_rk4_step_mask(_ref(self.O.P), self.O.Tp, len(self.specs), _p(self.meta),
                                                 _p(self.dx), dt, self._ptrs(self.U[0]), self._ptrs(self.U[1]),
                                                 self._ptrs(self.U[2]), self._ptrs(self.U[3]), self._ptrs(self.prim),
                                                 self._ptrs(self.status), int(rmask))
