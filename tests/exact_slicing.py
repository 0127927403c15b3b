"""Exact rational integral of a linear density over (simplex intersect axis-aligned box).

An independent reference used only to pin the oracle: it shares neither algorithm nor code with
``oracle/oracle.c`` (which clips simplices into sub-simplices in floating point).

Method (slicing + Simpson). Let f(z) be the integral of rho over the cross-section of the
simplex and the box at height z (a 2D polygon clip in 3D, a 1D interval clip in 2D). Between
consecutive "events" -- heights of simplex vertices, heights at which a simplex edge crosses a
side plane of the box, heights at which a simplex facet contains a vertical box edge, and the
box's own bottom/top -- the clipped cross-section keeps its combinatorial type and all its
vertices move linearly in z, so f is a polynomial of degree <= 3 there. Simpson's rule is exact
for cubics, so summing (b-a)/6 (f(a) + 4 f(mid) + f(b)) over the event intervals gives the exact
integral. All arithmetic is in ``fractions.Fraction``.
"""
from __future__ import annotations

from fractions import Fraction as F
import functools
from itertools import combinations


def _solve3(m, r):
    """Solve the 3x3 rational system m x = r by Cramer's rule."""
    def det(a):
        return (a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1])
                - a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0])
                + a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]))
    d = det(m)
    out = []
    for c in range(3):
        mc = [[(r[i] if j == c else m[i][j]) for j in range(3)] for i in range(3)]
        out.append(det(mc) / d)
    return out


def _linear_rho(verts, rho):
    """(c, g) with rho(x) = c + g.x matching the vertex values (D+1 vertices in D dims)."""
    d = len(verts[0])
    if d == 3:
        m = [[verts[i][a] - verts[0][a] for a in range(3)] for i in (1, 2, 3)]
        r = [rho[i] - rho[0] for i in (1, 2, 3)]
        g = _solve3(m, r)
    else:
        a = [[verts[i][k] - verts[0][k] for k in range(2)] for i in (1, 2)]
        r = [rho[i] - rho[0] for i in (1, 2)]
        det = a[0][0] * a[1][1] - a[0][1] * a[1][0]
        g = [(r[0] * a[1][1] - a[0][1] * r[1]) / det, (a[0][0] * r[1] - r[0] * a[1][0]) / det]
    c = rho[0] - sum(g[k] * verts[0][k] for k in range(d))
    return c, g


def _clip_poly(poly, axis, bound, keep_ge):
    """Sutherland-Hodgman clip of a 2D polygon (list of (x, y)) by x_axis >= bound or <= bound."""
    out = []
    n = len(poly)
    for i in range(n):
        p, q = poly[i], poly[(i + 1) % n]
        dp = (p[axis] - bound) if keep_ge else (bound - p[axis])
        dq = (q[axis] - bound) if keep_ge else (bound - q[axis])
        if dp >= 0:
            out.append(p)
        if (dp >= 0) != (dq >= 0):
            t = dp / (dp - dq)
            out.append((p[0] + t * (q[0] - p[0]), p[1] + t * (q[1] - p[1])))
    return out


def _section3(verts, z):
    """Convex cross-section polygon of a tetrahedron at height z (counter-clockwise)."""
    pts = [(v[0], v[1]) for v in verts if v[2] == z]
    for i, j in combinations(range(4), 2):
        a, b = verts[i], verts[j]
        if (a[2] - z) * (b[2] - z) < 0:
            t = (z - a[2]) / (b[2] - a[2])
            pts.append((a[0] + t * (b[0] - a[0]), a[1] + t * (b[1] - a[1])))
    uniq = list(dict.fromkeys(pts))
    if len(uniq) < 3:
        return []
    cx = sum(p[0] for p in uniq) / len(uniq)
    cy = sum(p[1] for p in uniq) / len(uniq)

    # exact angular sort around the centroid: half-plane then cross product
    def half(p):
        dx, dy = p[0] - cx, p[1] - cy
        return 0 if (dy > 0 or (dy == 0 and dx > 0)) else 1

    def cmp(p, q):
        hp, hq = half(p), half(q)
        if hp != hq:
            return hp - hq
        cr = (p[0] - cx) * (q[1] - cy) - (p[1] - cy) * (q[0] - cx)
        return -1 if cr > 0 else (1 if cr < 0 else 0)

    return sorted(uniq, key=functools.cmp_to_key(cmp))


def _poly_mass(poly, c, g, z):
    """Integral of c + g.(x, y, z) over the polygon at height z (fan triangulation)."""
    if len(poly) < 3:
        return F(0)
    tot = F(0)
    p0 = poly[0]
    for i in range(1, len(poly) - 1):
        p1, p2 = poly[i], poly[i + 1]
        area = abs((p1[0] - p0[0]) * (p2[1] - p0[1]) - (p1[1] - p0[1]) * (p2[0] - p0[0])) / 2
        mx = (p0[0] + p1[0] + p2[0]) / 3
        my = (p0[1] + p1[1] + p2[1]) / 3
        tot += area * (c + g[0] * mx + g[1] * my + g[2] * z)
    return tot


def _f3(verts, c, g, box, z):
    poly = _section3(verts, z)
    for axis in (0, 1):
        if not poly:
            break
        poly = _clip_poly(poly, axis, box[axis][0], True)
        if poly:
            poly = _clip_poly(poly, axis, box[axis][1], False)
    return _poly_mass(poly, c, g, z)


def mass3(verts, rho, box):
    """Exact integral over tet(verts) intersect box; verts: 4 triples of Fractions, rho: 4 Fractions,
    box: ((x0, x1), (y0, y1), (z0, z1))."""
    c, g = _linear_rho(verts, rho)
    events = {box[2][0], box[2][1]}
    events.update(v[2] for v in verts)
    for i, j in combinations(range(4), 2):
        a, b = verts[i], verts[j]
        for axis in (0, 1):
            if a[axis] != b[axis]:
                for bound in box[axis]:
                    t = (bound - a[axis]) / (b[axis] - a[axis])
                    if 0 <= t <= 1:
                        events.add(a[2] + t * (b[2] - a[2]))
    for tri in combinations(range(4), 3):
        p, q, r = (verts[k] for k in tri)
        u = [q[k] - p[k] for k in range(3)]
        w = [r[k] - p[k] for k in range(3)]
        n = [u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]]
        if n[2] != 0:
            for x in box[0]:
                for y in box[1]:
                    events.add(p[2] - (n[0] * (x - p[0]) + n[1] * (y - p[1])) / n[2])
    zlo = max(box[2][0], min(v[2] for v in verts))
    zhi = min(box[2][1], max(v[2] for v in verts))
    if zhi <= zlo:
        return F(0)
    zs = sorted(e for e in events if zlo <= e <= zhi)
    tot = F(0)
    for a, b in zip(zs[:-1], zs[1:]):
        if b == a:
            continue
        m = (a + b) / 2
        tot += (b - a) / 6 * (_f3(verts, c, g, box, a) + 4 * _f3(verts, c, g, box, m) + _f3(verts, c, g, box, b))
    return tot


def _f2(verts, c, g, box, y):
    xs = []
    for i, j in combinations(range(3), 2):
        a, b = verts[i], verts[j]
        if a[1] == y:
            xs.append(a[0])
        if b[1] == y:
            xs.append(b[0])
        if (a[1] - y) * (b[1] - y) < 0:
            t = (y - a[1]) / (b[1] - a[1])
            xs.append(a[0] + t * (b[0] - a[0]))
    if len(xs) < 2:
        return F(0)
    lo = max(min(xs), box[0][0])
    hi = min(max(xs), box[0][1])
    if hi <= lo:
        return F(0)
    return (hi - lo) * (c + g[0] * (lo + hi) / 2 + g[1] * y)


def mass2(verts, rho, box):
    """Exact integral over triangle(verts) intersect box ((x0, x1), (y0, y1))."""
    c, g = _linear_rho(verts, rho)
    events = {box[1][0], box[1][1]}
    events.update(v[1] for v in verts)
    for i, j in combinations(range(3), 2):
        a, b = verts[i], verts[j]
        if a[0] != b[0]:
            for bound in box[0]:
                t = (bound - a[0]) / (b[0] - a[0])
                if 0 <= t <= 1:
                    events.add(a[1] + t * (b[1] - a[1]))
    ylo = max(box[1][0], min(v[1] for v in verts))
    yhi = min(box[1][1], max(v[1] for v in verts))
    if yhi <= ylo:
        return F(0)
    ys = sorted(e for e in events if ylo <= e <= yhi)
    tot = F(0)
    for a, b in zip(ys[:-1], ys[1:]):
        if b == a:
            continue
        m = (a + b) / 2
        tot += (b - a) / 6 * (_f2(verts, c, g, box, a) + 4 * _f2(verts, c, g, box, m) + _f2(verts, c, g, box, b))
    return tot
