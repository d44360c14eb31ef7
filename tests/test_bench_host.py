"""Host-side helpers of bench.py that need no GPU.

The hierarchy's seeder is trained on flat-metric pairs drawn from the star's
own solved points; the sampler must draw only points whose last con2prim
solved without correction (status 0), spread over the patches in proportion
to their solved points, and undensitize B^i with chi^(3/2) (det gt = 1).
"""
import os
import sys
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _FakePatches:
    """Patch arrays as the library's binding holds them, on the CPU."""

    def __init__(self, shapes, seed=0):
        rng = torch.Generator().manual_seed(seed)
        self.status, self.prim, self.U = [], [], []
        for q, shp in enumerate(shapes):
            st = torch.randint(-1, 3, shp, generator=rng).to(torch.int8)
            if q == 2:
                st[:] = 1  # an all-atmosphere patch contributes nothing
            self.status.append(st)
            pr = torch.rand((10,) + shp, generator=rng, dtype=torch.float64)
            pr[0] = torch.where(st == 0, pr[0] + 1.0, -pr[0])  # rho > 1 marks a solved point
            self.prim.append(pr)
            self.U.append([torch.rand((32,) + shp, generator=rng, dtype=torch.float64) + 0.5])


def test_hierarchy_pairs_sample_solved_points_only():
    shapes = [(10, 10, 10), (8, 9, 12), (6, 6, 6), (12, 7, 9)]
    pt = _FakePatches(shapes)
    g = types.SimpleNamespace(NP=10, NF=32, prim2con_flat=lambda P, prim, B, table=None: (prim, B))
    n = 4000
    prim, B = bench._hierarchy_pairs(g, None, None, pt, n, seed=13)
    assert prim.shape == (n, 10) and B.shape == (n, 3)
    assert prim.is_contiguous() and B.is_contiguous()
    assert bool((prim[:, 0] > 1.0).all())  # every sample is a status-0 point
    # The same seed draws the same set.
    prim2, B2 = bench._hierarchy_pairs(g, None, None, pt, n, seed=13)
    assert torch.equal(prim, prim2) and torch.equal(B, B2)
    # Each sample's B is Bbar chi^(3/2) at the point its primitives come from.
    for q, st in enumerate(pt.status):
        ok = (st == 0).reshape(-1)
        if not bool(ok.any()):
            continue
        pr = pt.prim[q].reshape(10, -1)[:, ok].T
        U = pt.U[q][0].reshape(32, -1)[:, ok]
        Bq = (U[28:31] * U[12:13] ** 1.5).T
        # match rows by the (unique) random density
        rows = {float(r[0]): i for i, r in enumerate(pr)}
        hit = [i for i in range(n) if float(prim[i, 0]) in rows]
        for i in hit[:50]:
            assert torch.equal(B[i], Bq[rows[float(prim[i, 0])]])
    # Shares follow the patches' solved-point counts (all-atmosphere patch: none).
    counts = np.array([int((st == 0).sum()) for st in pt.status], dtype=float)
    got = []
    for q, st in enumerate(pt.status):
        ok = (st == 0).reshape(-1)
        vals = set(pt.prim[q].reshape(10, -1)[0, ok].tolist())
        got.append(sum(float(r) in vals for r in prim[:, 0]))
    assert got[2] == 0
    # floor per patch, the remainder (fewer than one per patch) to the largest
    assert np.all(np.abs(np.array(got) - n * counts / counts.sum()) <= len(shapes))
