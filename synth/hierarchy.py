"""Patch layouts of fixed mesh-refinement hierarchies (geometry only).

A hierarchy is a list of patch specs: n (interior points per axis), level,
o (origin index on the level's grid, which starts at the level-0 origin X0
with spacing dx0 / 2^level), and the derived dx and x0 = X0 + o dx.  Level 0
is a single patch.
"""
import numpy as np


def spec(n, level, o, dx0, X0):
    dx = dx0 / 2 ** level
    return dict(n=tuple(int(v) for v in n), level=int(level), o=tuple(int(v) for v in o), dx=dx,
                x0=tuple(float(X0[a]) + o[a] * dx for a in range(3)))


def small_hierarchy(dx0=1.0, X0=(-12.0, -12.0, -12.0), n0=24):
    """Three levels, five patches of uneven shapes: a 24^3 level-0 patch, two
    level-1 patches that share a face, and two level-2 patches, one of which
    straddles the two level-1 patches."""
    return [
        spec((n0, n0, n0), 0, (0, 0, 0), dx0, X0),
        spec((12, 12, 12), 1, (12, 12, 12), dx0, X0),
        spec((10, 12, 12), 1, (24, 12, 12), dx0, X0),
        spec((16, 12, 12), 2, (30, 28, 28), dx0, X0),
        spec((8, 8, 10), 2, (50, 28, 30), dx0, X0),
    ]


def nested_cubes(n0, dx0, X0, fine, edges=(16, 24, 32, 48, 64), seed=4):
    """Level 0: one n0^3 patch at X0.  fine: list of (level, start, size[,
    edges]) with start and size in points of that level's grid (same on every
    axis); each such cube is split into blocks whose edges are drawn per axis
    from edges (seeded), the last block of a row taking what remains."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    out = [spec((n0,) * 3, 0, (0, 0, 0), dx0, X0)]
    for entry in fine:
        level, start, size = entry[:3]
        lev_edges = entry[3] if len(entry) > 3 else edges
        cuts = []
        for _ in range(3):
            c, pos = [], 0
            while pos < size:
                e = int(rng.choice(lev_edges))
                e = min(e, size - pos)
                if size - pos - e and size - pos - e < 8:  # no sliver blocks
                    e = size - pos
                c.append((pos, e))
                pos += e
            cuts.append(c)
        for (oz, ez) in cuts[2]:
            for (oy, ey) in cuts[1]:
                for (ox, ex) in cuts[0]:
                    out.append(spec((ex, ey, ez), level, (start + ox, start + oy, start + oz), dx0, X0))
    return out


def amr_tov_layout(scale=1.0, levels=5, seed=4):
    """The magnetised-star hierarchy.  At scale 1: level 0 one 128^3 patch on
    [-80, 80)^3 (dx0 = 1.25), levels 1..levels-2 cubes of 160 points centred
    on the origin and split into blocks with edges from {24, 32, 48}, and the
    finest level a cube of 256 points in 64^3 blocks (dx0 / 16 = 0.078 on
    [-10, 10)).  A smaller scale shrinks every point count by it and widens
    dx0 by 1/scale, so the finest level still spans [-10, 10)."""
    n0 = int(round(128 * scale))
    fine_size = 8 * int(round(20 * scale))
    finest = 8 * int(round(32 * scale))
    dx0 = 1.25 / scale
    half = n0 * dx0 / 2.0
    X0 = (-half,) * 3
    fine = []
    for l in range(1, levels):
        size = finest if l == levels - 1 else fine_size
        centre = int(round(half / (dx0 / 2 ** l)))
        start = centre - size // 2
        fine.append((l, start, size, (64,) if l == levels - 1 else (24, 32, 48)))
    return nested_cubes(n0, dx0, X0, fine, seed=seed)


def subcycle_hierarchy(dx0=1.0 / 24, X0=(0.0, 0.0, 0.0), n0=24):
    """Three properly nested levels for sub-cycling: a 24^3 level-0 patch,
    level 1 a 24^3 cube (level-1 points 12..35) in four uneven patches, level 2
    a 16^3 cube (level-2 points 32..47) in two patches.  Every fine ghost
    point's prolongation stencil lies inside the interiors of the next coarser
    level (or the level-0 patch's ghosts)."""
    out = [spec((n0, n0, n0), 0, (0, 0, 0), dx0, X0)]
    for (ox, ex) in ((0, 16), (16, 8)):
        for (oy, ey) in ((0, 8), (8, 16)):
            out.append(spec((ex, ey, 24), 1, (12 + ox, 12 + oy, 12), dx0, X0))
    for (ox, ex) in ((0, 8), (8, 8)):
        out.append(spec((ex, 16, 16), 2, (32 + ox, 32, 32), dx0, X0))
    return out
