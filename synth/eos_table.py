"""Synthetic tabulated EOS: ideal nucleon gas plus radiation, sampled on nodes.

Nodes: log10 rho in [-14, -2] (code units, G = c = Msun = 1), log10 T in
[-3, 3] (MeV), Ye in [0.03, 0.6]; 256 x 128 x 64 by default, rho fastest.
With theta = T / m_b (m_b = 939.565 MeV):
    p   = rho theta (1 + Ye) + a_r T^4 / 3
    eps = 1.5 theta (1 + Ye) + a_r T^4 / rho
    c_s^2 = (dp/drho|_eps + p / rho^2 dp/deps|_rho) / (1 + eps + p / rho)
a_r is the photon radiation constant pi^2 / 15 / (hbar c)^3 in MeV^-3 fm^-3
converted to code units of mass density: 1 MeV fm^-3 = 1.602176634e33 erg cm^-3,
divided by c^2 to g cm^-3 and by the code density unit c^6 / (G (G Msun)^2)
(CODATA c and G, IAU nominal G Msun).
"""
import numpy as np

HBARC = 197.3269804            # MeV fm
MEV_ERG = 1.602176634e-6       # erg
C_CGS = 2.99792458e10          # cm / s
G_CGS = 6.67430e-8             # cm^3 g^-1 s^-2
GM_SUN = 1.3271244e26          # cm^3 s^-2
M_B = 939.565                  # MeV


def code_density_unit():
    """g cm^-3 per code unit of mass density."""
    return C_CGS ** 6 / (G_CGS * GM_SUN ** 2)


def radiation_constant():
    """a_r such that the radiation energy density is a_r T^4 (code units, T in MeV)."""
    mev_fm3_in_gcc = MEV_ERG * 1e39 / C_CGS ** 2
    return (np.pi ** 2 / 15.0) / HBARC ** 3 * mev_fm3_in_gcc / code_density_unit()


def model(rho, T, ye, a_r=None):
    """Analytic p, eps, c_s^2 of the ideal nucleon gas + radiation model."""
    if a_r is None:
        a_r = radiation_constant()
    th = T / M_B
    p = rho * th * (1.0 + ye) + a_r * T ** 4 / 3.0
    eps = 1.5 * th * (1.0 + ye) + a_r * T ** 4 / rho
    p_rho_T = th * (1.0 + ye)
    p_T = rho * (1.0 + ye) / M_B + 4.0 * a_r * T ** 3 / 3.0
    e_T = 1.5 * (1.0 + ye) / M_B + 4.0 * a_r * T ** 3 / rho
    e_rho_T = -a_r * T ** 4 / rho ** 2
    p_eps = p_T / e_T
    p_rho_eps = p_rho_T - p_T * e_rho_T / e_T
    h = 1.0 + eps + p / rho
    cs2 = (p_rho_eps + p / rho ** 2 * p_eps) / h
    return p, eps, cs2


def make_table(nr=256, nt=128, ny=64, lr=(-14.0, -2.0), lt=(-3.0, 3.0), ye=(0.03, 0.6)):
    """Node values (p, eps, cs2 arrays of shape (ny, nt, nr)) and grid description."""
    lrs = np.linspace(lr[0], lr[1], nr)
    lts = np.linspace(lt[0], lt[1], nt)
    yes = np.linspace(ye[0], ye[1], ny)
    Y, Tl, R = np.meshgrid(yes, lts, lrs, indexing="ij")
    rho = 10.0 ** R
    T = 10.0 ** Tl
    p, eps, cs2 = model(rho, T, Y)
    h0 = float(np.min(1.0 + eps + p / rho))
    return dict(
        nr=nr, nt=nt, ny=ny,
        lr0=lr[0], dlr=(lr[1] - lr[0]) / (nr - 1), lr_max=lr[1],
        lt0=lt[0], dlt=(lt[1] - lt[0]) / (nt - 1), lt_max=lt[1],
        ye0=ye[0], dye=(ye[1] - ye[0]) / (ny - 1), ye_max=ye[1],
        p=np.ascontiguousarray(p), eps=np.ascontiguousarray(eps), cs2=np.ascontiguousarray(cs2),
        h0=h0, a_r=radiation_constant(),
    )
