"""Parameter sets and grid geometry for the synthetic workloads.

Constants the paper leaves open are fixed here (damping and gauge constants,
divergence-cleaning speed and damping, error-policy thresholds, Brent stop
rule); each value is listed with its reason in the design notes.
"""
import numpy as np

NG = 3     # ghost width (KO / upwind stencils and the 6-point MP5 interface stencil)
NID = 26   # initial-data fields

# Ideal-gas runs: Gamma = 2, atmosphere polytrope K = 100.
_COMMON = dict(
    kappa_z=0.5, kappa_c=0.05, kappa_2=0.0, eta=1.4, sigma_ko=0.1,
    c_b=1.0, kappa_b=1.0,
    alpha_bh=0.2, W_max=50.0,
    ye_min=0.03, ye_max=0.6,
    c2p_xtol=1e-300, max_iter=200,
)


def ideal_params(bc=0, **over):
    """Parameters of the ideal-gas configurations (bc 0 periodic, 1 extrapolation)."""
    p = dict(_COMMON)
    p.update(
        gamma_th=2.0, K_atmo=100.0,
        rho_atmo=1e-10, rho_min=1.1e-10, rho_low=1e-8, rho_max=1.0,
        eps_max=1e6, T_atmo=0.0, h0=1.0,
        ye_atmo=0.1,  # Ye is a passive scalar for the ideal gas: the fluid's own value
        eos_kind=0, bc=bc,
    )
    p.update(over)
    return p


def table_params(table, bc=0, **over):
    """Parameters of the tabulated-EOS configurations; h0 is the table's enthalpy bound."""
    p = dict(_COMMON)
    p.update(
        gamma_th=2.0, K_atmo=100.0,
        rho_atmo=1e-13, rho_min=1.1e-13, rho_low=1e-11, rho_max=10.0 ** table["lr_max"],
        eps_max=0.0, T_atmo=10.0 ** table["lt0"], h0=table["h0"],
        ye_atmo=0.315,  # midpoint of the Ye range (no beta-equilibrium data)
        eos_kind=1, bc=bc,
    )
    p.update(over)
    return p


def patch_shape(n, pad=1):
    """Ghosted array extents (pz, py, px) of an n = (n0, n1, n2) patch; px padded to `pad`."""
    n0, n1, n2 = n
    px = n0 + 2 * NG
    px = (px + pad - 1) // pad * pad
    return (n2 + 2 * NG, n1 + 2 * NG, px)


def grid_coords(n, x0, dx, pad=1):
    """Coordinates (z, y, x) broadcastable arrays of a vertex-centred patch incl. ghosts.

    Point i (i = -3 .. n+2) sits at x0 + i dx; padded x entries repeat the last point.
    """
    pz, py, px = patch_shape(n, pad)
    ax = []
    for a, m in enumerate((px, py, pz)):
        idx = np.arange(m) - NG
        if a == 0:
            idx = np.minimum(idx, n[0] + NG - 1)
        ax.append(x0[a] + idx * dx)
    x = ax[0][None, None, :]
    y = ax[1][None, :, None]
    z = ax[2][:, None, None]
    return z, y, x


def hybrid_params(bc=0, **over):
    """Hybrid-EOS parameters (eos_kind 2): a synthetic three-piece cold
    polytrope (K_0 = 100, Gamma = 2, 2.3, 2.6 with pieces divided at rho =
    5e-4 and 1.1e-3, so a 1.28e-3 star centre lies in the stiffest piece) plus a
    Gamma_th = 1.8 thermal part; causal (c_s^2 < 1) up to rho ~ 4e-3 at
    eps = 1.5 eps_cold.  Not a fit to any nuclear EOS."""
    p = ideal_params(bc=bc)
    p.update(eos_kind=2, gamma_th=1.8, npoly=3, K_poly=100.0, rho_poly=(5e-4, 1.1e-3, 0.0),
             gamma_poly=(2.0, 2.3, 2.6, 0.0), eps_max=1e6, h0=1.0)
    p.update(over)
    return p
