"""Analytic initial data: Fourier-mode perturbations of flat space and a TOV star.

Fourier data (the smooth periodic workload, 32^3 on [0,1)^3):
  gamma_ij = delta_ij + sum of 8 modes A sin(2 pi k.x + phi), A = 1e-4, per component;
  K_ij = same form; alpha = 1; beta = 0;
  rho = 1e-3 (1 + 0.1 m(x)), m an 8-mode sum normalised to max |m| = 1;
  P = 100 rho^2 (Gamma = 2 ideal gas, eps = P / rho);
  v^i from three mode sums scaled to max |v| = 0.1;
  Bbar = curl A_vec (analytic), A_vec three mode sums, scaled so max b^2/rho = 1;
  Ye = 0.1.
TOV star: K = 100, Gamma = 2, rho_c = 1.28e-3, isotropic coordinates, a
low-density atmosphere of 1e-10, optional 1 % random pressure perturbation
and a poloidal field from A_phi = A_b max(p - 0.04 p_max, 0).
"""
import numpy as np

from .eos_table import M_B, model, radiation_constant
from scipy.integrate import solve_ivp
from scipy.interpolate import CubicSpline

from .configs import NID, grid_coords, patch_shape


def _modes(rng, nmodes=8):
    """Random wave vectors in {-2..2}^3 \\ {0} and phases."""
    ks = []
    while len(ks) < nmodes:
        k = rng.integers(-2, 3, size=3)
        if np.any(k != 0):
            ks.append(k)
    return np.array(ks, dtype=np.float64), rng.uniform(0.0, 2.0 * np.pi, size=nmodes)


def _mode_sum(x, y, z, ks, ph, amp=1.0):
    out = np.zeros(np.broadcast_shapes(x.shape, y.shape, z.shape))
    for k, p in zip(ks, ph):
        out += amp * np.sin(2.0 * np.pi * (k[0] * x + k[1] * y + k[2] * z) + p)
    return out


def _mode_grad(x, y, z, ks, ph):
    """Analytic gradient of the unit-amplitude mode sum."""
    g = [np.zeros(np.broadcast_shapes(x.shape, y.shape, z.shape)) for _ in range(3)]
    for k, p in zip(ks, ph):
        c = 2.0 * np.pi * np.cos(2.0 * np.pi * (k[0] * x + k[1] * y + k[2] * z) + p)
        for a in range(3):
            g[a] += k[a] * c
    return g


def _sym_det(g):
    return (g[0] * (g[3] * g[5] - g[4] * g[4]) - g[1] * (g[1] * g[5] - g[4] * g[2])
            + g[2] * (g[1] * g[4] - g[3] * g[2]))


def _lower(g, v):
    S = ((0, 1, 2), (1, 3, 4), (2, 4, 5))
    return [sum(g[S[i][j]] * v[j] for j in range(3)) for i in range(3)]


def config0_id(n=(32, 32, 32), seed=0, pad=1, amp=1e-4, dx=None, x0=(0.0, 0.0, 0.0), norm=None, return_norm=False):
    """Fourier-mode initial data on the periodic unit cube (dx = 1/n0 unless given).

    The density, velocity and field amplitudes are normalised on the patch's own
    points unless `norm` (as returned with return_norm=True) fixes them, which
    keeps one global field across patches of different size and resolution."""
    n = tuple(int(v) for v in n)
    if dx is None:
        dx = 1.0 / n[0]
    rng = np.random.default_rng(np.random.PCG64(seed))
    z, y, x = grid_coords(n, x0, dx, pad)
    shp = patch_shape(n, pad)
    ID = np.zeros((NID,) + shp)
    full = lambda a: np.broadcast_to(a, shp)
    diag = (0, 3, 5)
    for c in range(6):
        ks, ph = _modes(rng)
        ID[c] = full((1.0 if c in diag else 0.0) + _mode_sum(x, y, z, ks, ph, amp))
    for c in range(6):
        ks, ph = _modes(rng)
        ID[6 + c] = full(_mode_sum(x, y, z, ks, ph, amp))
    ID[12] = 1.0
    # Density.
    ks, ph = _modes(rng)
    m = full(_mode_sum(x, y, z, ks, ph))
    m_max = norm["m_max"] if norm else np.max(np.abs(m))
    m = m / m_max
    rho = 1e-3 * (1.0 + 0.1 * m)
    ID[16] = rho
    ID[17] = 100.0 * rho  # eps = P / ((Gamma - 1) rho) with P = 100 rho^2, Gamma = 2
    # Velocity.
    v = []
    for a in range(3):
        ks, ph = _modes(rng)
        v.append(full(_mode_sum(x, y, z, ks, ph)))
    vmag = np.sqrt(v[0] ** 2 + v[1] ** 2 + v[2] ** 2)
    sc = norm["v_scale"] if norm else 0.1 / np.max(vmag)
    for a in range(3):
        ID[18 + a] = v[a] * sc
    # Magnetic field: Bbar = curl A (densitized, analytically divergence free).
    grads = []
    for a in range(3):
        ks, ph = _modes(rng)
        grads.append([full(gc) for gc in _mode_grad(x, y, z, ks, ph)])
    Bbar = [grads[2][1] - grads[1][2], grads[0][2] - grads[2][0], grads[1][0] - grads[0][1]]
    g = [ID[c] for c in range(6)]
    sg = np.sqrt(_sym_det(g))
    B = [b / sg for b in Bbar]
    vv = [ID[18 + a] for a in range(3)]
    vd = _lower(g, vv)
    Bd = _lower(g, B)
    v2 = sum(vv[a] * vd[a] for a in range(3))
    B2 = sum(B[a] * Bd[a] for a in range(3))
    Bv = sum(B[a] * vd[a] for a in range(3))
    b2 = B2 * (1.0 - v2) + Bv ** 2
    s = norm["b_scale"] if norm else np.sqrt(1.0 / np.max(b2 / rho))
    for a in range(3):
        ID[21 + a] = B[a] * s
    ID[24] = 0.1
    if return_norm:
        return np.ascontiguousarray(ID), dict(m_max=m_max, v_scale=sc, b_scale=s)
    return np.ascontiguousarray(ID)


EDGES = (16, 24, 32, 48, 64)


def batched_specs(npatch=256, seed=2, levels=5, edges=EDGES, dx0=1.0 / 32):
    """Uneven patches: each axis edge uniform over `edges`, level uniform in
    0..levels-1 with dx = dx0 / 2^level, origin uniform in [0, 1)^3."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    out = []
    for _ in range(npatch):
        n = tuple(int(v) for v in rng.choice(edges, size=3))
        lev = int(rng.integers(0, levels))
        out.append(dict(n=n, level=lev, dx=dx0 / 2 ** lev, x0=tuple(float(v) for v in rng.uniform(0.0, 1.0, 3))))
    return out


def batched_id(spec, seed=0, norm=None):
    """Initial data of one batched patch: the periodic Fourier field of seed
    `seed` sampled on the patch's points (ghosts from the same field)."""
    if norm is None:
        _, norm = config0_id(n=(32, 32, 32), seed=seed, return_norm=True)
    return config0_id(n=spec["n"], seed=seed, dx=spec["dx"], x0=spec["x0"], norm=norm)


# ---------------------------------------------------------------------------
# TOV star in isotropic coordinates.

def tov_profile(K=100.0, Gamma=2.0, rho_c=1.28e-3):
    """Solve the TOV equations (areal radius r) and return splines in isotropic radius rb.

    Returns a dict with M, R (areal), Rb (isotropic surface radius) and splines
    rho(rb), p(rb), dp/drb(rb), psi(rb), alpha(rb) valid for rb <= Rb.
    """
    def eos(p):
        p = max(p, 0.0)
        rho = (p / K) ** (1.0 / Gamma)
        eps = p / ((Gamma - 1.0) * rho) if rho > 0 else 0.0
        return rho, eps

    def rhs(r, u):
        m, p, nu, lnrb = u
        rho, eps = eos(p)
        e = rho * (1.0 + eps)
        dm = 4.0 * np.pi * r * r * e
        f = (m + 4.0 * np.pi * r ** 3 * p) / (r * (r - 2.0 * m))
        dp = -(e + p) * f
        dnu = f
        dlnrb = 1.0 / (r * np.sqrt(1.0 - 2.0 * m / r))
        return [dm, dp, dnu, dlnrb]

    p_c = K * rho_c ** Gamma
    r0 = 1e-6
    e_c = rho_c * (1.0 + p_c / ((Gamma - 1.0) * rho_c))
    m0 = 4.0 / 3.0 * np.pi * r0 ** 3 * e_c
    ev = lambda r, u: u[1] - 1e-14 * p_c
    ev.terminal = True
    ev.direction = -1
    sol = solve_ivp(rhs, (r0, 50.0), [m0, p_c, 0.0, np.log(r0)], method="DOP853", rtol=1e-12, atol=1e-20,
                    events=ev, dense_output=True, max_step=0.01)
    R = sol.t_events[0][0]
    M = sol.y_events[0][0][0]
    r = np.concatenate([[0.0], np.linspace(r0, R, 20001)])
    u = sol.sol(r[1:])
    m, p, nu, lnrb = u
    # Match the exterior isotropic Schwarzschild solution at the surface.
    Rb = 0.5 * (R - M + np.sqrt(R * (R - 2.0 * M)))
    lnrb = lnrb - lnrb[-1] + np.log(Rb)
    rb = np.concatenate([[0.0], np.exp(lnrb)])
    alpha_R = np.sqrt(1.0 - 2.0 * M / R)
    nu = nu - nu[-1] + np.log(alpha_R)
    p = np.concatenate([[p_c], np.maximum(p, 0.0)])
    alpha = np.concatenate([[np.exp(nu[0])], np.exp(nu)])
    m = np.concatenate([[0.0], m])
    rr = r.copy()
    psi = np.sqrt(np.where(rb > 0, rr / np.where(rb > 0, rb, 1.0), 1.0))
    psi[0] = psi[1]
    rho = (p / K) ** (1.0 / Gamma)
    # dp/drb = dp/dr * dr/drb, dr/drb = r sqrt(1 - 2m/r) / rb.
    e = rho * (1.0 + p / np.where(rho > 0, (Gamma - 1.0) * rho, 1.0))
    with np.errstate(divide="ignore", invalid="ignore"):
        f = np.where(rr > 0, (m + 4.0 * np.pi * rr ** 3 * p) / (rr * (rr - 2.0 * m)), 0.0)
        drdrb = np.where(rb > 0, rr * np.sqrt(np.maximum(1.0 - 2.0 * m / np.where(rr > 0, rr, 1.0), 0.0))
                         / np.where(rb > 0, rb, 1.0), 1.0)
    dpdrb = -(e + p) * f * drdrb
    keep = np.concatenate([[True], np.diff(rb) > 0])
    mk = lambda a: CubicSpline(rb[keep], a[keep])
    return dict(M=M, R=R, Rb=Rb, p_c=p_c, rho=mk(rho), p=mk(p), dpdrb=mk(dpdrb), psi=mk(psi),
                alpha=mk(alpha), K=K, Gamma=Gamma)


def _table_temperature(rho, p, ye, table, iters=48):
    """T [MeV] at which the synthetic table model gives pressure p at (rho, ye):
    bisection in log T over the table's range (clamped to its ends)."""
    a_r = radiation_constant()

    def pres(T):  # the model's pressure alone
        return rho * (T / M_B) * (1.0 + ye) + a_r * T ** 4 / 3.0

    lo = np.full(rho.shape, table["lt0"])
    hi = np.full(rho.shape, table["lt0"] + table["dlt"] * (table["nt"] - 1))
    p_lo = pres(10.0 ** lo)
    p_hi = pres(10.0 ** hi)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        pm = pres(10.0 ** mid)
        up = pm < p
        lo = np.where(up, mid, lo)
        hi = np.where(up, hi, mid)
    lt = np.where(p <= p_lo, table["lt0"], np.where(p >= p_hi, hi, 0.5 * (lo + hi)))
    return 10.0 ** lt


def tov_id(n=(128, 128, 128), x0=(-20.0, -20.0, -20.0), dx=0.3125, seed=1, perturb=True, bfield=True,
           pad=1, rho_atmo=1e-10, profile=None, ye=0.1, table=None, heat=1.0):
    """Static TOV star on a vertex-centred patch (ghosts included).  With a
    synthetic table, the temperature (field 25) is set so the table model's
    pressure equals the polytropic one (eps then follows from the table).
    heat > 1 scales the specific internal energy of the polytrope (a heated
    star: for EOS models whose cold part is stiffer than the polytrope's the
    data then stay above their cold energy)."""
    n = tuple(int(v) for v in n)
    prof = profile if profile is not None else tov_profile()
    K, Gamma, M, Rb = prof["K"], prof["Gamma"], prof["M"], prof["Rb"]
    z, y, x = grid_coords(n, x0, dx, pad)
    shp = patch_shape(n, pad)
    x, y, z = (np.broadcast_to(a, shp) for a in (x, y, z))
    rb = np.sqrt(x * x + y * y + z * z)
    inside = rb < Rb
    rbi = np.where(inside, rb, 0.0)
    psi = np.where(inside, prof["psi"](rbi), 1.0 + M / (2.0 * np.maximum(rb, 1e-300)))
    alpha = np.where(inside, prof["alpha"](rbi),
                     (1.0 - M / (2.0 * np.maximum(rb, 1e-300))) / (1.0 + M / (2.0 * np.maximum(rb, 1e-300))))
    p = np.where(inside, np.maximum(prof["p"](rbi), 0.0), 0.0)
    rho = np.where(p > 0, (p / K) ** (1.0 / Gamma), 0.0)
    rho = np.maximum(rho, rho_atmo)
    p_smooth = p.copy()
    p = K * rho ** Gamma
    if perturb:
        rng = np.random.default_rng(np.random.PCG64(seed))
        xi = rng.uniform(-1.0, 1.0, size=shp)
        p = np.where(rho > 100.0 * rho_atmo, p * (1.0 + 0.01 * xi), p)
    eps = heat * p / ((Gamma - 1.0) * rho)
    ID = np.zeros((NID,) + shp)
    if table is not None:
        ID[25] = _table_temperature(rho, p, ye, table)
        eps = model(rho, ID[25], ye)[1]
    psi4 = psi ** 4
    ID[0] = psi4
    ID[3] = psi4
    ID[5] = psi4
    ID[12] = alpha
    ID[16] = rho
    ID[17] = eps
    ID[24] = ye
    if bfield:
        p_max = prof["p_c"]
        p_cut = 0.04 * p_max
        A = np.maximum(p_smooth - p_cut, 0.0)
        dA = np.where((p_smooth > p_cut) & inside, prof["dpdrb"](rbi), 0.0)
        rs = np.maximum(rb, 1e-300)
        Bbx = -x * dA * z / rs
        Bby = -y * dA * z / rs
        Bbz = 2.0 * A + dA * (x * x + y * y) / rs
        sg = psi ** 6
        B = [Bbx / sg, Bby / sg, Bbz / sg]
        b2 = psi4 * (B[0] ** 2 + B[1] ** 2 + B[2] ** 2)
        mx = np.max(b2)
        s = np.sqrt(2.0 * 1e-3 * p_max / mx) if mx > 0 else 0.0
        for a in range(3):
            ID[21 + a] = B[a] * s
    return np.ascontiguousarray(ID)
