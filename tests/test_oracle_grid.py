"""Pins of the oracle's grid builder against facts outside itself (no GPU)."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import grid as OG
from tests.conftest import golden_path

R = O.R_EARTH


@pytest.fixture(scope="module", params=[0, 1, 2, 3])
def grid(request):
    return O.build_grid(2, request.param)


def test_counts_euler_and_degrees(grid):
    L = grid.levels
    assert grid.nc == 20 * 4 ** L
    assert grid.ne == 30 * 4 ** L
    assert grid.nv == 10 * 4 ** L + 2
    assert grid.nv - grid.ne + grid.nc == 2                      # Euler characteristic of the sphere
    assert 2 * grid.ne == 3 * grid.nc                            # edges count as 1.5 per cell (Table 2)
    hist = np.bincount(grid.vdeg)
    assert hist[5] == 12 and hist[6] == grid.nv - 12 and hist.sum() == grid.nv   # 12 pentagons


def test_table2_cell_counts():
    rows = {}
    for line in open(golden_path("table2_grids.txt")):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        rows[f[0]] = f[1:]
    # the count formula the builder satisfies (test above) reproduces the printed sizes
    for name in ("R2B8", "R2B11"):
        bis, cells_e8, dx_km, _ = rows[name]
        nc = 20 * 4 ** (int(bis) + 1)
        assert round(nc / 1e8, 2) == float(cells_e8)
        dx = math.sqrt(4 * math.pi * R * R / nc) / 1e3            # sqrt of the mean cell area
        assert abs(dx - float(dx_km)) / float(dx_km) < 0.02
    assert (20 * 4 ** 12) // (20 * 4 ** 9) == int(rows["ratio"][0])
    # and the builder itself at a small size agrees with the same count formula
    g = O.build_grid(2, 4)
    assert g.nc == 20 * 4 ** 5


def test_icosahedron_closed_form():
    v, f = OG.icosahedron()
    assert np.allclose(np.linalg.norm(v, axis=1), 1.0, rtol=0, atol=1e-15)
    # every face edge of a regular icosahedron subtends atan(2)
    for a, b in ((0, 1), (1, 2), (0, 2)):
        ang = np.arccos(np.clip(np.sum(v[f[:, a]] * v[f[:, b]], axis=1), -1, 1))
        assert np.allclose(ang, math.atan(2.0), rtol=0, atol=1e-12)
    # counter-clockwise seen from outside: a.(b x c) > 0
    assert np.all(np.einsum("ij,ij->i", v[f[:, 0]], np.cross(v[f[:, 1]], v[f[:, 2]])) > 0)
    # each of the 30 edges is shared by exactly two faces with opposite directions
    directed = {(f[i, s], f[i, (s + 1) % 3]) for i in range(20) for s in range(3)}
    assert len(directed) == 60
    assert all((b, a) in directed for a, b in directed)


def test_numbering_by_explicit_loops():
    """G-3/G-4 restated as a first-sight scan over (cell, slot) in ascending order."""
    g = O.build_grid(2, 0)
    tri = OG.refine(g.levels)
    seen_v, c2v = {}, np.zeros((g.nc, 3), dtype=np.int64)
    for c in range(g.nc):
        for s in range(3):
            key = tuple(float(x) + 0.0 for x in tri[c, s])
            if key not in seen_v:
                seen_v[key] = len(seen_v)
            c2v[c, s] = seen_v[key]
    assert np.array_equal(c2v, g.c2v)
    seen_e, c2e, e2c = {}, np.zeros((g.nc, 3), dtype=np.int64), {}
    for c in range(g.nc):
        for s in range(3):
            a, b = c2v[c, s], c2v[c, (s + 1) % 3]
            key = (min(a, b), max(a, b))
            if key not in seen_e:
                seen_e[key] = len(seen_e)
                e2c[seen_e[key]] = [c, None, (a, b)]
            else:
                e2c[seen_e[key]][1] = c
            c2e[c, s] = seen_e[key]
    assert np.array_equal(c2e, g.c2e)
    for e in range(g.ne):
        c1, c2, (a, b) = e2c[e]
        assert (g.e2c[e, 0], g.e2c[e, 1]) == (c1, c2)
        assert (g.e2v[e, 0], g.e2v[e, 1]) == (a, b)


def test_orientation(grid):
    g = grid
    c1, c2 = g.e2c[:, 0], g.e2c[:, 1]
    assert np.all(c1 < c2)
    # the edge runs v1 -> v2 in c1 and v2 -> v1 in c2 (consistent CCW orientation)
    for side, want in ((c1, (0, 1)), (c2, (1, 0))):
        cv = g.c2v[side]
        ok = np.zeros(g.ne, dtype=bool)
        for s in range(3):
            ok |= (cv[:, s] == g.e2v[:, want[0]]) & (cv[:, (s + 1) % 3] == g.e2v[:, want[1]])
        assert ok.all()
    assert np.all(np.sum(g.n_e * (g.x_c[c2] - g.x_c[c1]), axis=1) > 0)          # n from c1 to c2
    assert np.all(np.sum(g.t_e * (g.x_v[g.e2v[:, 1]] - g.x_v[g.e2v[:, 0]]), axis=1) > 0)
    assert np.allclose(np.sum(g.n_e * g.x_e, axis=1), 0.0, atol=1e-15)
    # (n, t, r) right-handed
    assert np.allclose(np.cross(g.n_e, g.t_e), g.x_e, atol=1e-15)


def test_vertex_lists_ccw(grid):
    g = grid
    for v in range(g.nv):
        d = g.vdeg[v]
        es = g.v2e[v, :d]
        assert es[0] == es.min()
        assert len(set(es)) == d
        for j in range(d):
            cj = g.v2c[v, j]
            assert es[j] in g.c2e[cj] and es[(j + 1) % d] in g.c2e[cj]
            # direction to the far end of edge j, then of edge j+1: counter-clockwise turn
            far = [g.e2v[e, 1] if g.e2v[e, 0] == v else g.e2v[e, 0] for e in (es[j], es[(j + 1) % d])]
            d0 = g.x_v[far[0]] - g.x_v[v]
            d1 = g.x_v[far[1]] - g.x_v[v]
            assert np.dot(np.cross(d0, d1), g.x_v[v]) > 0
        if d == 5:
            assert g.v2e[v, 5] == g.v2e[v, 0] and g.s_ve[v, 5] == 0.0


def test_areas_tile_the_sphere(grid):
    g = grid
    total = 4 * math.pi * R * R
    assert abs(g.A_c.sum() / total - 1) < 1e-12
    assert abs(g.A_v.sum() / total - 1) < 1e-12
    assert np.all(g.A_c > 0) and np.all(g.A_v > 0)


def test_weights_normalised(grid):
    g = grid
    assert np.allclose(g.kin_w.sum(axis=1), 1.0, rtol=0, atol=1e-15)
    assert np.all(g.kin_w > 0)
    # c2e slot s joins corners s and s+1
    for s in range(3):
        e = g.c2e[:, s]
        a, b = g.c2v[:, s], g.c2v[:, (s + 1) % 3]
        assert np.all(np.minimum(a, b) == np.minimum(g.e2v[e, 0], g.e2v[e, 1]))
        assert np.all(np.maximum(a, b) == np.maximum(g.e2v[e, 0], g.e2v[e, 1]))
