"""Icosahedral triangular C-grid for the oracle (test infrastructure, FP64, plain numpy).

TEST INFRASTRUCTURE ONLY. Nothing in the product library imports this module; only
tests/, bench.py's CPU-baseline leg and __graft_entry__.smoke() may use it.

What the paper fixes: ICON computes on an icosahedral-triangular C grid with a dual
of hexagons and 12 pentagons (Sec. "Current State of the Art"; Sec. "Separation of
Concerns", index reuse), the cell count of the R2B8 (10 km) and R2B11 (1.25 km)
grids and the edge/cell ratio of 1.5 (Table 2). Everything else below is the
builder's reading, written out so that it can be checked by eye:

G-1  Icosahedron: vertex 0 is the north pole, vertices 1..5 lie at latitude
     +atan(1/2) and longitude 72 i degrees, vertices 6..10 at latitude -atan(1/2)
     and longitude 36 + 72 i degrees, vertex 11 is the south pole. The 20 root
     faces are: 5 northern (0, 1+i, 1+(i+1)%5); for each i the equatorial pair
     (1+i, 6+i, 1+(i+1)%5) and (1+(i+1)%5, 6+i, 6+(i+1)%5); 5 southern
     (11, 6+(i+1)%5, 6+i). Each is counter-clockwise seen from outside.
G-2  RnBk with n = 2 is k+1 bisections. A triangle (a, b, c) is split with
     m_ab = normalize(a + b) etc. into children (a, m_ab, m_ca), (m_ab, b, m_bc),
     (m_ca, m_bc, c), (m_bc, m_ca, m_ab). Cell id = root face * 4^L + base-4
     child digits (a hierarchical Morton order).
G-3  Vertex id: ascending order of (lowest incident cell id, corner slot in it).
     Here vertices are identified across cells by exact equality of their
     computed positions: a shared midpoint is computed from the same two parent
     points in every cell that has it, and a + b == b + a bit for bit.
G-4  Edge id: ascending order of (lowest incident cell id, local edge slot), slot
     s joining corner s to corner (s+1)%3. The edge's (v1, v2) is that CCW order
     in its lowest cell c1; c2 is the other cell.
G-5  Geometry on the unit sphere, scaled by R (lengths) and R^2 (areas):
     cell centre = normalize((b-a) x (c-a)); edge midpoint = normalize(v1+v2);
     normal n = normalize(v2 x v1) (points from c1 to c2); tangent t = x_e x n
     (points from v1 to v2); l_e = R arc(v1, v2); d_e = R arc(x_c1, x_c2);
     cell area = R^2 * spherical excess (Van Oosterom-Strackee); dual area =
     sum of the spherical triangles (x_v, x_c(j), x_c(j+1)); f_e = 2 Omega z(x_e).
G-6  s_ce = +1 if c is c1(e) else -1; s_ve = -1 if v is v1(e), +1 if v is v2(e).
     Vertex lists run counter-clockwise from the lowest incident edge id; v2c[j]
     is the cell between v2e[j] and v2e[j+1]. Pentagons repeat entry 0 in slot 5
     with weight 0.
O4   vt_e = 1/2 (u_c1 + u_c2) . t_e with the Perot cell vector
     u_c = (1/A_c) sum_e s_ce l_e vn_e (x_e - x_c) R, folded into 5 weights
     (own edge, the two other edges of c1, the two other edges of c2).
O5   kappa_ce proportional to l_e * R arc(x_c, x_e), normalised to sum 1.
D    Least-squares vertex vector: argmin sum_j (u . n_j - vn_j)^2 over the
     incident edges, u in the tangent plane at x_v, as 3-vector weights.
"""
import numpy as np

R_EARTH = 6.371229e6     # m
OMEGA = 7.29212e-5       # 1/s

# table ids (order shared with nothing; the C library documents its own ids)
INT_TABLES = ("c2v", "c2e", "e2c", "e2v", "v2e", "v2c", "vdeg", "e2vt", "e2q")


def _normalize(v):
    return v / np.sqrt(np.sum(v * v, axis=-1, keepdims=True))


def _arc(a, b):
    """Great-circle angle between unit vectors (rows), atan2 form."""
    cr = np.cross(a, b)
    return np.arctan2(np.sqrt(np.sum(cr * cr, axis=-1)), np.sum(a * b, axis=-1))


def _excess(a, b, c):
    """Spherical excess of the triangle (a, b, c): tan(E/2) = |a.(b x c)| / (1 + a.b + b.c + c.a)."""
    num = np.abs(np.sum(a * np.cross(b, c), axis=-1))
    den = 1.0 + np.sum(a * b, axis=-1) + np.sum(b * c, axis=-1) + np.sum(c * a, axis=-1)
    return 2.0 * np.arctan2(num, den)


def icosahedron():
    """Root vertices (12, 3) and faces (20, 3) of G-1."""
    v = np.zeros((12, 3))
    v[0] = (0.0, 0.0, 1.0)
    lat = np.arctan(0.5)
    for i in range(5):
        ln = 2.0 * np.pi * i / 5.0
        ls = 2.0 * np.pi * (i + 0.5) / 5.0
        v[1 + i] = (np.cos(lat) * np.cos(ln), np.cos(lat) * np.sin(ln), np.sin(lat))
        v[6 + i] = (np.cos(lat) * np.cos(ls), np.cos(lat) * np.sin(ls), -np.sin(lat))
    v[11] = (0.0, 0.0, -1.0)
    f = []
    for i in range(5):
        f.append((0, 1 + i, 1 + (i + 1) % 5))
    for i in range(5):
        f.append((1 + i, 6 + i, 1 + (i + 1) % 5))
        f.append((1 + (i + 1) % 5, 6 + i, 6 + (i + 1) % 5))
    for i in range(5):
        f.append((11, 6 + (i + 1) % 5, 6 + i))
    return v, np.array(f, dtype=np.int64)


def refine(levels):
    """Corner positions (Nc, 3, 3) of all cells after `levels` bisections, in cell-id order (G-2)."""
    rv, rf = icosahedron()
    tri = rv[rf]                                   # (20, 3, 3)
    for _ in range(levels):
        a, b, c = tri[:, 0], tri[:, 1], tri[:, 2]
        mab = _normalize(a + b)
        mbc = _normalize(b + c)
        mca = _normalize(c + a)
        kids = np.stack([
            np.stack([a, mab, mca], axis=1),
            np.stack([mab, b, mbc], axis=1),
            np.stack([mca, mbc, c], axis=1),
            np.stack([mbc, mca, mab], axis=1)], axis=1)   # (n, 4, 3, 3)
        tri = kids.reshape(-1, 3, 3)
    return tri


class Grid:
    """All tables and FP64 geometry of one RnBk grid (attributes are numpy arrays)."""


def build_grid(root, bisections):
    """Build the grid R{root}B{bisections}. Only root 2 is defined (G-2)."""
    if root != 2:
        raise ValueError("only root 2 grids are defined")
    if bisections < 0:
        raise ValueError("bisections must be >= 0")
    L = bisections + 1
    tri = refine(L)
    nc = tri.shape[0]
    g = Grid()
    g.root, g.bisections, g.levels = root, bisections, L

    # ---- G-3 vertices: dedupe corners by exact position; id order = first (cell, slot)
    pts = tri.reshape(-1, 3) + 0.0                 # +0.0 turns -0.0 into 0.0
    _, first, inv = np.unique(pts, axis=0, return_index=True, return_inverse=True)
    inv = inv.reshape(-1)
    order = np.argsort(first, kind="stable")
    vid_of_u = np.empty(len(first), dtype=np.int64)
    vid_of_u[order] = np.arange(len(first))
    c2v = vid_of_u[inv].reshape(nc, 3)
    nv = len(first)
    x_v = pts[first[order]]

    # ---- G-4 edges: dedupe (min, max) vertex pairs; id order = first (cell, slot)
    s0 = c2v
    s1 = np.roll(c2v, -1, axis=1)                  # corner (s+1)%3
    pairs = np.stack([np.minimum(s0, s1), np.maximum(s0, s1)], axis=-1).reshape(-1, 2)
    _, efirst, einv = np.unique(pairs, axis=0, return_index=True, return_inverse=True)
    einv = einv.reshape(-1)
    eorder = np.argsort(efirst, kind="stable")
    eid_of_u = np.empty(len(efirst), dtype=np.int64)
    eid_of_u[eorder] = np.arange(len(efirst))
    c2e = eid_of_u[einv].reshape(nc, 3)
    ne = len(efirst)
    rep = efirst[eorder]                          # flat (cell*3 + slot) of each edge's rep
    c1 = rep // 3
    slot = rep % 3
    e2v = np.stack([c2v[c1, slot], c2v[c1, (slot + 1) % 3]], axis=1)
    # second cell: the occurrence that is not the representative
    occ_cell = np.repeat(np.arange(nc), 3)
    e_of_occ = c2e.reshape(-1)
    c2 = np.full(ne, -1, dtype=np.int64)
    nonrep = np.ones(3 * nc, dtype=bool)
    nonrep[rep] = False
    c2[e_of_occ[nonrep]] = occ_cell[nonrep]
    e2c = np.stack([c1, c2], axis=1)

    # ---- geometry (unit sphere)
    a, b, c = x_v[c2v[:, 0]], x_v[c2v[:, 1]], x_v[c2v[:, 2]]
    x_c = _normalize(np.cross(b - a, c - a))
    v1, v2 = x_v[e2v[:, 0]], x_v[e2v[:, 1]]
    x_e = _normalize(v1 + v2)
    n_e = _normalize(np.cross(v2, v1))
    t_e = np.cross(x_e, n_e)
    R = R_EARTH
    l_e = R * _arc(v1, v2)
    d_e = R * _arc(x_c[c1], x_c[c2])
    A_c = R * R * _excess(a, b, c)
    f_e = 2.0 * OMEGA * x_e[:, 2]

    # ---- G-6 vertex lists: CCW by angle in the tangent plane, from the lowest edge id
    ends = np.concatenate([e2v[:, 0], e2v[:, 1]])
    other = np.concatenate([e2v[:, 1], e2v[:, 0]])
    eidx = np.concatenate([np.arange(ne), np.arange(ne)])
    xv = x_v[ends]
    ref = np.where(np.abs(xv[:, 2:3]) < 0.9, np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))
    b1 = _normalize(np.cross(ref, xv))
    b2 = np.cross(xv, b1)                          # (b1, b2, r) right-handed: b1 -> b2 is CCW
    d = x_v[other] - xv
    ang = np.arctan2(np.sum(d * b2, axis=1), np.sum(d * b1, axis=1))
    srt = np.lexsort((ang, ends))
    ends_s, e_s = ends[srt], eidx[srt]
    vdeg = np.bincount(ends, minlength=nv)
    start = np.concatenate([[0], np.cumsum(vdeg)[:-1]])
    v2e = np.zeros((nv, 6), dtype=np.int64)
    for v_deg in (5, 6):
        vs = np.nonzero(vdeg == v_deg)[0]
        lst = e_s[start[vs][:, None] + np.arange(v_deg)[None, :]]
        shift = np.argmin(lst, axis=1)
        rolled = np.take_along_axis(lst, (shift[:, None] + np.arange(v_deg)[None, :]) % v_deg, axis=1)
        v2e[vs, :v_deg] = rolled
        if v_deg == 5:
            v2e[vs, 5] = rolled[:, 0]
    assert np.all(ends_s[start] == np.arange(nv))
    # cell between v2e[j] and v2e[j+1]: the common cell of the two edges
    v2c = np.zeros((nv, 6), dtype=np.int64)
    for j in range(6):
        ea = v2e[:, j]
        eb = np.where(vdeg == 5, v2e[:, (j + 1) % 5 if j < 5 else 1], v2e[:, (j + 1) % 6])
        ca, cb = e2c[ea], e2c[eb]
        common = np.where((ca[:, 0] == cb[:, 0]) | (ca[:, 0] == cb[:, 1]), ca[:, 0], ca[:, 1])
        v2c[:, j] = common
    v2c[vdeg == 5, 5] = v2c[vdeg == 5, 0]

    # dual areas
    A_v = np.zeros(nv)
    for j in range(6):
        jn = np.where(vdeg == 5, (j + 1) % 5, (j + 1) % 6)
        cn = v2c[np.arange(nv), jn]
        contrib = _excess(x_v, x_c[v2c[:, j]], x_c[cn])
        A_v += np.where((vdeg == 6) | (j < 5), contrib, 0.0)
    A_v *= R * R

    # signs
    s_ce = np.where(e2c[c2e, 0] == np.arange(nc)[:, None], 1.0, -1.0)
    s_ve = np.where(e2v[v2e, 0] == np.arange(nv)[:, None], -1.0, 1.0)
    s_ve[vdeg == 5, 5] = 0.0

    # O4 vt stencil and weights: own edge, then the two other edges of c1 and of c2
    e2vt = np.zeros((ne, 5), dtype=np.int64)
    vt_w = np.zeros((ne, 5))
    eids = np.arange(ne)
    e2vt[:, 0] = eids
    for col, cs in ((1, c1), (3, c2)):
        edges = c2e[cs]                                       # (ne, 3), c2e slot order
        coef = (0.5 * s_ce[cs] * l_e[edges] * R
                * np.sum((x_e[edges] - x_c[cs][:, None, :]) * t_e[:, None, :], axis=2)
                / A_c[cs][:, None])
        own = edges == eids[:, None]
        vt_w[:, 0] += np.sum(np.where(own, coef, 0.0), axis=1)
        e2vt[:, col:col + 2] = edges[~own].reshape(ne, 2)
        vt_w[:, col:col + 2] = coef[~own].reshape(ne, 2)

    # O5 kinetic-energy weights
    h_ce = R * _arc(np.repeat(x_c, 3, axis=0), x_e[c2e].reshape(-1, 3)).reshape(nc, 3)
    kin_w = l_e[c2e] * h_ce
    kin_w = kin_w / np.sum(kin_w, axis=1, keepdims=True)

    # quad vertices (v1, v2, v3 opposite in c1, v4 opposite in c2) and L34
    def opposite(cells):
        cv = c2v[cells]
        m = (cv != e2v[:, 0:1]) & (cv != e2v[:, 1:2])
        return cv[m]
    e2q = np.stack([e2v[:, 0], e2v[:, 1], opposite(c1), opposite(c2)], axis=1)
    L34 = R * _arc(x_v[e2q[:, 2]], x_v[e2q[:, 3]])

    # least-squares vertex reconstruction weights (3-vectors), zero for padding
    ref = np.where(np.abs(x_v[:, 2:3]) < 0.9, np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))
    e1 = _normalize(np.cross(ref, x_v))
    e2 = np.cross(x_v, e1)
    nj = n_e[v2e]                                  # (nv, 6, 3)
    valid = np.ones((nv, 6))
    valid[vdeg == 5, 5] = 0.0
    p1 = np.sum(nj * e1[:, None, :], axis=2) * valid
    p2 = np.sum(nj * e2[:, None, :], axis=2) * valid
    m11, m12, m22 = np.sum(p1 * p1, 1), np.sum(p1 * p2, 1), np.sum(p2 * p2, 1)
    det = m11 * m22 - m12 * m12
    i11, i12, i22 = m22 / det, -m12 / det, m11 / det
    q1 = i11[:, None] * p1 + i12[:, None] * p2      # component along e1 of each weight
    q2 = i12[:, None] * p1 + i22[:, None] * p2
    lsq_w = q1[:, :, None] * e1[:, None, :] + q2[:, :, None] * e2[:, None, :]

    g.nc, g.ne, g.nv = nc, ne, nv
    g.c2v, g.c2e, g.e2c, g.e2v = c2v, c2e, e2c, e2v
    g.v2e, g.v2c, g.vdeg, g.e2vt, g.e2q = v2e, v2c, vdeg, e2vt, e2q
    g.x_v, g.x_c, g.x_e, g.n_e, g.t_e = x_v, x_c, x_e, n_e, t_e
    g.l_e, g.d_e, g.A_c, g.A_v, g.f_e = l_e, d_e, A_c, A_v, f_e
    g.s_ce, g.s_ve, g.vt_w, g.kin_w, g.lsq_w, g.L34 = s_ce, s_ve, vt_w, kin_w, lsq_w, L34
    g.corners = tri
    return g
