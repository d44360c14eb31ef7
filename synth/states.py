"""Random primitive states for con2prim in isolation (flat metric).

rho log-uniform in [1e-10, 1e-2], W uniform in [1, 10] with an isotropic
velocity direction, T log-uniform in [1e-2, 1e2] MeV, Ye uniform in
[0.05, 0.5], B with an isotropic direction and a magnitude such that
b^2 / rho is log-uniform in [1e-4, 10], where b^2 = B^2 / W^2 + (B.v)^2.
"""
import numpy as np


def _unit(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def c2p_states(n, seed=3, rho=(1e-10, 1e-2), W=(1.0, 10.0), T=(1e-2, 1e2), ye=(0.05, 0.5), b2rho=(1e-4, 10.0)):
    """Returns dict of float64 arrays: rho, T, ye (n,), v (n, 3), B (n, 3)."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    lr = rng.uniform(np.log10(rho[0]), np.log10(rho[1]), n)
    Wv = rng.uniform(W[0], W[1], n)
    lt = rng.uniform(np.log10(T[0]), np.log10(T[1]), n)
    yv = rng.uniform(ye[0], ye[1], n)
    lb = rng.uniform(np.log10(b2rho[0]), np.log10(b2rho[1]), n)
    nv = _unit(rng, n)
    nb = _unit(rng, n)
    r = 10.0 ** lr
    vmag = np.sqrt(1.0 - 1.0 / Wv ** 2)
    v = nv * vmag[:, None]
    b2 = (10.0 ** lb) * r
    nbv = np.sum(nb * v, axis=1)
    s = np.sqrt(b2 / (1.0 / Wv ** 2 + nbv ** 2))
    B = nb * s[:, None]
    return dict(rho=r, T=10.0 ** lt, ye=yv, v=np.ascontiguousarray(v), B=np.ascontiguousarray(B))
