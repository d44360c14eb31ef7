"""Independent ADM reference quantities for the CCZ4 pins (test helper).

Fields are given as sympy expressions of (x, y, z); sympy supplies exact first
and second partial derivatives, and everything else (inverse metric,
Christoffel symbols, Ricci tensor, covariant derivatives, the ADM evolution
equations) is assembled numerically with the textbook formulas of the
standard 3+1 (ADM) system, which do not use the conformal decomposition.
"""
import itertools

import numpy as np
import sympy as sp

X = sp.symbols("x y z", real=True)
SYM = ((0, 1, 2), (1, 3, 4), (2, 4, 5))
PAIRS = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]


def lam(expr):
    return sp.lambdify(X, expr, "numpy")


class Field:
    """Value, gradient and Hessian of a scalar sympy expression, evaluated on arrays."""

    def __init__(self, expr):
        self.f = lam(expr)
        self.d = [lam(sp.diff(expr, a)) for a in X]
        self.dd = [[lam(sp.diff(expr, a, b)) for b in X] for a in X]

    def eval(self, x, y, z):
        shp = np.broadcast_shapes(np.shape(x), np.shape(y), np.shape(z))
        b = lambda v: np.broadcast_to(np.asarray(v, dtype=float), shp)
        return (b(self.f(x, y, z)), np.array([b(g(x, y, z)) for g in self.d]),
                np.array([[b(h(x, y, z)) for h in row] for row in self.dd]))


def sym_full(g6):
    return np.array([[g6[SYM[i][j]] for j in range(3)] for i in range(3)])


class ADM:
    """ADM data (gamma_ij, K_ij, alpha, beta^i) from sympy expressions at given points."""

    def __init__(self, g6, K6, alpha, beta, x, y, z):
        G = [Field(e).eval(x, y, z) for e in g6]
        Kf = [Field(e).eval(x, y, z) for e in K6]
        A = Field(alpha).eval(x, y, z)
        B = [Field(e).eval(x, y, z) for e in beta]
        # Move the point axes last: g[i, j, ...], dg[k, i, j, ...], ddg[k, l, i, j, ...]
        self.g = np.array([[G[SYM[i][j]][0] for j in range(3)] for i in range(3)])
        self.dg = np.array([[[G[SYM[i][j]][1][k] for j in range(3)] for i in range(3)] for k in range(3)])
        self.ddg = np.array([[[[G[SYM[i][j]][2][k][l] for j in range(3)] for i in range(3)] for l in range(3)]
                             for k in range(3)])
        self.K = np.array([[Kf[SYM[i][j]][0] for j in range(3)] for i in range(3)])
        self.dK = np.array([[[Kf[SYM[i][j]][1][k] for j in range(3)] for i in range(3)] for k in range(3)])
        self.al, self.dal, self.ddal = A
        self.be = np.array([b[0] for b in B])
        self.dbe = np.array([[B[i][1][k] for i in range(3)] for k in range(3)])  # dbe[k, i] = d_k beta^i
        self.ddbe = np.array([[[B[i][2][k][l] for i in range(3)] for l in range(3)] for k in range(3)])
        self._derived()

    def _derived(self):
        g, dg, ddg = self.g, self.dg, self.ddg
        gi = np.moveaxis(np.linalg.inv(np.moveaxis(g, (0, 1), (-2, -1))), (-2, -1), (0, 1))
        self.gu = gi
        # d_k g^{ij} = -g^{ia} d_k g_ab g^{bj}
        dgi = -np.einsum("ia...,kab...,bj...->kij...", gi, dg, gi)
        # Christoffel Gam[k, i, j] = 1/2 g^{kl} (d_i g_lj + d_j g_li - d_l g_ij)
        low = 0.5 * (np.einsum("ilj...->lij...", dg) + np.einsum("jli...->lij...", dg) - dg)  # low[l,i,j]
        self.Gam = np.einsum("kl...,lij...->kij...", gi, low)
        # d_m Gam[k,i,j]; d_m low[l,i,j] = 1/2 (d_m d_i g_lj + d_m d_j g_li - d_m d_l g_ij)
        dd = ddg  # dd[m, n, a, b] = d_m d_n g_ab
        dlow = np.zeros((3, 3, 3, 3) + g.shape[2:])
        for m, l, i, j in itertools.product(range(3), repeat=4):
            dlow[m, l, i, j] = 0.5 * (dd[m, i, l, j] + dd[m, j, l, i] - dd[m, l, i, j])
        self.dGam = np.einsum("mkl...,lij...->mkij...", dgi, low) + np.einsum("kl...,mlij...->mkij...", gi, dlow)
        Gm, dG = self.Gam, self.dGam
        # R_ij = d_k Gam^k_ij - d_j Gam^k_ik + Gam^k_kl Gam^l_ij - Gam^k_jl Gam^l_ik
        self.Ric = (np.einsum("kkij...->ij...", dG) - np.einsum("jkik...->ij...", dG)
                    + np.einsum("kkl...,lij...->ij...", Gm, Gm) - np.einsum("kjl...,lik...->ij...", Gm, Gm))
        self.R = np.einsum("ij...,ij...->...", gi, self.Ric)
        # D_i D_j alpha
        self.DDa = self.ddal - np.einsum("kij...,k...->ij...", Gm, self.dal)
        K = self.K
        self.trK = np.einsum("ij...,ij...->...", gi, K)
        Kmix = np.einsum("ik...,kj...->ij...", gi, K)  # K^i_j
        Kuu = np.einsum("ik...,jl...,kl...->ij...", gi, gi, K)
        self.KK = np.einsum("ij...,ij...->...", Kuu, K)
        self.H = self.R + self.trK ** 2 - self.KK
        # beta_i and its covariant derivative D_i beta_j
        bl = np.einsum("ij...,j...->i...", g, self.be)
        dbl = np.einsum("kij...,j...->ki...", dg, self.be) + np.einsum("ij...,kj...->ki...", g, self.dbe)
        Db = dbl - np.einsum("kij...,k...->ij...", Gm, bl)  # Db[i,j] = D_i beta_j
        self.Db = Db
        # ADM evolution (vacuum)
        self.dt_g = -2.0 * self.al * K + Db + np.swapaxes(Db, 0, 1)
        lieK = (np.einsum("k...,kij...->ij...", self.be, self.dK) + np.einsum("ik...,jk...->ij...", K, self.dbe)
                + np.einsum("kj...,ik...->ij...", K, self.dbe))
        KKm = np.einsum("ik...,kj...->ij...", K, Kmix)
        self.dt_K = -self.DDa + self.al * (self.Ric - 2.0 * KKm + self.trK * K) + lieK
        # Conformal quantities
        det = np.linalg.det(np.moveaxis(g, (0, 1), (-2, -1)))
        self.chi = det ** (-1.0 / 3.0)
        dchi = -(1.0 / 3.0) * self.chi * np.einsum("ij...,kij...->k...", gi, dg)
        self.gt = self.chi * g
        dgt = np.einsum("k...,ij...->kij...", dchi, g) + self.chi * dg
        gtu = gi / self.chi
        # Gt^i = gt^{ij} gt^{kl} d_l gt_jk
        self.Gt = np.einsum("ij...,kl...,ljk...->i...", gtu, gtu, dgt)
        # Time derivatives of the CCZ4 variables implied by the ADM equations.
        dt_chi = -(self.chi / 3.0) * np.einsum("ij...,ij...->...", gi, self.dt_g)
        self.dt_chi = dt_chi
        self.dt_gt = dt_chi * g + self.chi * self.dt_g
        self.dt_trK = np.einsum("ij...,ij...->...", gi, self.dt_K) - np.einsum("ij...,ij...->...", Kuu, self.dt_g)
        self.dt_At = (dt_chi * K + self.chi * self.dt_K
                      - (self.dt_gt * self.trK + self.gt * self.dt_trK) / 3.0)

    def id_array(self):
        """Initial-data array layout of the synthetic inputs (vacuum)."""
        shp = self.g.shape[2:]
        ID = np.zeros((26,) + shp)
        for n, (i, j) in enumerate(PAIRS):
            ID[n] = self.g[i, j]
            ID[6 + n] = self.K[i, j]
        ID[12] = self.al
        ID[13:16] = self.be
        return ID


def six(T):
    return np.array([T[i, j] for (i, j) in PAIRS])
