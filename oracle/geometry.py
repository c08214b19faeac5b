"""Beam geometry and natural-neighbour weights (FP64, plain Python/NumPy).

Paper passages followed:
  * aperture beams {h : Psi(h) != 0}, |q| lambda <= alpha (Sec. 2.1 "Grid,
    probe and specimen"), PRISM subsampling h_y = 0 mod f_y, h_x = 0 mod f_x
    (Algorithm 2, build step; Sec. 2.2.2 "Beam subsampling");
  * detector beams |q| <= theta_det / lambda, PRISM-subsampled (Algorithm 4,
    first step) -- by the probe's f, or along one axis by 1 for qEELS, whose
    resolved axis must be sampled at f = 1 (Sec. 2.2.6);
  * the cube's complete output basis: every beam inside the detector disc,
    no subsampling (Sec. 2.2.6);
  * hex-ring parents: the DC beam plus n_radial rings with n_angular (1 + i)
    samples on ring i, snapped to the nearest beam and deduplicated
    (Sec. 2.2.3 "Parent selection"; Algorithm 3 build step);
  * Sibson natural-neighbour weights w_{p,b} >= 0, sum_p w = 1, local support
    (Eq. nnw; Sibson 1981), computed on signed-frequency coordinates q.

Readings where the paper is silent:
  * beams are ordered by (h_y, h_x) ascending; the aperture edge is
    inclusive with a relative slack of 1e-12;
  * ring radii r_i = R (i + 1) / n_radial, R = max |q| over the retained
    beams; angles theta_k = 2 pi k / (n_angular (1 + i)) from +q_x towards
    +q_y; ties when snapping go to the lowest (h_y, h_x); duplicates keep the
    first occurrence in the order DC, ring 0, ring 1, ...;
  * a query on or outside the parents' convex hull (where Sibson weights are
    undefined) takes the linear weights of the two end points of the nearest
    hull edge -- the limit of Sibson interpolation on the hull.  (Parity
    unpinned against the paper: a project reading; pinned only by the
    linear-precision property it preserves.)
"""
import math
import numpy as np

from .physics import signed_index

APERTURE_SLACK = 1e-12
SNAP_TIE_REL = 1e-9


# --------------------------------------------------------------------------
# beams

def disc_beams(ny, nx, ly, lx, lam, angle, fy=1, fx=1):
    """Integer beam indices h (rows (h_y, h_x)) with |q| lambda <= angle and
    h = 0 mod f, ordered by (h_y, h_x) ascending."""
    hy = np.sort(signed_index(ny))
    hx = np.sort(signed_index(nx))
    HY, HX = np.meshgrid(hy, hx, indexing="ij")
    q = np.sqrt((HY / ly) ** 2 + (HX / lx) ** 2)
    keep = (q * lam <= angle * (1.0 + APERTURE_SLACK)) & (HY % fy == 0) & (HX % fx == 0)
    return np.stack([HY[keep], HX[keep]], axis=1).astype(np.int64)


def aperture_function(h, ly, lx, lam, defocus=0.0, cs=0.0):
    """Psi(h) = exp(-i chi(q)), chi = pi lambda df |q|^2 + (pi/2) Cs lambda^3 |q|^4
    inside the aperture (Sec. 2.1; aberration sign convention is a reading)."""
    q2 = (h[:, 0] / ly) ** 2 + (h[:, 1] / lx) ** 2
    chi = np.pi * lam * defocus * q2 + 0.5 * np.pi * cs * lam ** 3 * q2 ** 2
    return np.exp(-1j * chi)


def beam_q(h, ly, lx):
    return np.stack([h[:, 0] / ly, h[:, 1] / lx], axis=1).astype(np.float64)


# --------------------------------------------------------------------------
# hex-ring parents

def hex_ring_parents(h, ly, lx, nrad, nang):
    """Indices (into the beam list h) of the hex-ring parent beams."""
    q = beam_q(h, ly, lx)
    radius = float(np.max(np.sqrt(np.sum(q ** 2, axis=1)))) if len(q) else 0.0
    targets = [(0.0, 0.0)]
    for i in range(nrad):
        r = radius * (i + 1) / nrad
        n = nang * (1 + i)
        for k in range(n):
            th = 2.0 * math.pi * k / n
            targets.append((r * math.sin(th), r * math.cos(th)))
    chosen = []
    for ty, tx in targets:
        d2 = (q[:, 0] - ty) ** 2 + (q[:, 1] - tx) ** 2
        m = float(np.min(d2))
        cand = np.nonzero(d2 <= m * (1.0 + SNAP_TIE_REL))[0]
        best = min(cand, key=lambda j: (h[j, 0], h[j, 1]))
        if best not in chosen:
            chosen.append(int(best))
    return np.array(chosen, dtype=np.int64)


# --------------------------------------------------------------------------
# convex polygons

def _clip(poly, a0, a1, c):
    """Part of convex polygon `poly` with a0*y + a1*x <= c (Sutherland-Hodgman)."""
    out = []
    n = len(poly)
    for i in range(n):
        py, px = poly[i]
        qy, qx = poly[(i + 1) % n]
        fp = a0 * py + a1 * px - c
        fq = a0 * qy + a1 * qx - c
        if fp <= 0.0:
            out.append((py, px))
        if (fp < 0.0 < fq) or (fq < 0.0 < fp):
            t = fp / (fp - fq)
            out.append((py + t * (qy - py), px + t * (qx - px)))
    return out


def _area(poly):
    n = len(poly)
    if n < 3:
        return 0.0
    s = 0.0
    for i in range(n):
        y0, x0 = poly[i]
        y1, x1 = poly[(i + 1) % n]
        s += x0 * y1 - x1 * y0
    return 0.5 * abs(s)


def _cross_int(o, a, b):
    return (a[0] - o[0]) * (b[1] - o[1]) - (a[1] - o[1]) * (b[0] - o[0])


def convex_hull_int(pts):
    """Convex hull of integer points, counter-clockwise in (y, x) with cross
    defined as above, keeping points that lie on hull edges."""
    P = sorted(set((int(a), int(b)) for a, b in pts))
    if len(P) <= 2:
        return P
    lower, upper = [], []
    for p in P:
        while len(lower) >= 2 and _cross_int(lower[-2], lower[-1], p) < 0:
            lower.pop()
        lower.append(p)
    for p in reversed(P):
        while len(upper) >= 2 and _cross_int(upper[-2], upper[-1], p) < 0:
            upper.pop()
        upper.append(p)
    hull = lower[:-1] + upper[:-1]
    # collinear input degenerates to a doubled segment: keep unique order
    seen, out = set(), []
    for p in hull:
        if p not in seen:
            seen.add(p)
            out.append(p)
    return out


# --------------------------------------------------------------------------
# Sibson weights

def _hull_edges(hull_pts):
    """Edges (position pairs in the hull list) of the hull polygon; when
    every parent lies on one line the hull is a segment, whose edges are
    only the pieces between consecutive parents (no closing edge back over
    the whole segment)."""
    n = len(hull_pts)
    collinear = all(_cross_int(hull_pts[0], hull_pts[1], hull_pts[i]) == 0 for i in range(2, n))
    if collinear:
        return [(e, e + 1) for e in range(n - 1)]
    return [(e, (e + 1) % n) for e in range(n)]


def _edge_weights(hull_idx, hull_q, edges, qb):
    """Linear weights on the hull edge nearest to qb (physical metric)."""
    best = None
    for e0, e1 in edges:
        a = hull_q[e0]
        b = hull_q[e1]
        d = b - a
        dd = float(d @ d)
        t = 0.0 if dd == 0.0 else float(np.clip((qb - a) @ d / dd, 0.0, 1.0))
        p = a + t * d
        dist = float((qb - p) @ (qb - p))
        if best is None or dist < best[0] - 1e-300:
            best = (dist, e0, e1, t)
    _, e0, e1, t = best
    return {hull_idx[e0]: 1.0 - t, hull_idx[e1]: t}


def _strictly_inside(hull_pts, hb):
    n = len(hull_pts)
    if n < 3:
        return False
    # hull orientation: sign of the polygon's signed area (integer arithmetic)
    s = 0
    for i in range(n):
        s += _cross_int((0, 0), hull_pts[i], hull_pts[(i + 1) % n])
    orient = 1 if s > 0 else -1
    for i in range(n):
        c = _cross_int(hull_pts[i], hull_pts[(i + 1) % n], hb)
        if c * orient <= 0:
            return False
    return True


def _voronoi_cell(rel, box):
    """Cell of the origin against points `rel` (relative coordinates)."""
    poly = [(-box, -box), (-box, box), (box, box), (box, -box)]
    for py, px in rel:
        poly = _clip(poly, 2.0 * py, 2.0 * px, py * py + px * px)
        if not poly:
            break
    return poly


def sibson_weights(parent_h, query_h, ly, lx):
    """Weight matrix w [n_query, n_parent] (Eq. nnw): w[b, p] is the area of
    the query's new Voronoi cell (in Vor(parents + query)) stolen from
    parent p's cell, divided by the new cell's area."""
    parent_h = np.asarray(parent_h, dtype=np.int64)
    query_h = np.asarray(query_h, dtype=np.int64)
    nq, npar = len(query_h), len(parent_h)
    W = np.zeros((nq, npar), dtype=np.float64)
    if npar == 0:
        return W
    pq = beam_q(parent_h, ly, lx)
    lut = {(int(a), int(b)): i for i, (a, b) in enumerate(parent_h)}
    hull_pts = convex_hull_int(parent_h)
    hull_idx = [lut[p] for p in hull_pts]
    hull_q = pq[hull_idx]
    edges = _hull_edges(hull_pts) if len(hull_pts) >= 2 else []
    for b in range(nq):
        hb = (int(query_h[b, 0]), int(query_h[b, 1]))
        if hb in lut:
            W[b, lut[hb]] = 1.0
            continue
        qb = np.array([hb[0] / ly, hb[1] / lx])
        if npar == 1:
            W[b, 0] = 1.0
            continue
        if not _strictly_inside(hull_pts, hb):
            for p, w in _edge_weights(hull_idx, hull_q, edges, qb).items():
                W[b, p] += w
            continue
        rel = pq - qb
        dist = np.sqrt(np.sum(rel ** 2, axis=1))
        order = np.argsort(dist, kind="stable")
        box = 4.0 * float(dist.max())
        while True:
            cell = _voronoi_cell(rel[order], box)
            rmax = max(max(abs(y), abs(x)) for y, x in cell)
            if rmax < box * (1.0 - 1e-9):
                break
            box *= 4.0
        a_new = _area(cell)
        r_new = max(math.hypot(y, x) for y, x in cell)
        cand = [int(j) for j in order if dist[j] <= 2.0 * r_new + dist[order[0]] + 1e-12 * r_new]
        for p in cand:
            py, px = rel[p]
            piece = cell
            for j in cand:
                if j == p:
                    continue
                ry, rx = rel[j]
                piece = _clip(piece, 2.0 * (ry - py), 2.0 * (rx - px),
                              (ry * ry + rx * rx) - (py * py + px * px))
                if not piece:
                    break
            W[b, p] = _area(piece) / a_new
    return W


# --------------------------------------------------------------------------
# bundled geometry for a configuration

def cube_basis(cfg, lam):
    """The cube's output beams, (h_y, h_x) ascending: every beam with
    |q| lambda <= theta_det (no subsampling), or, when the configuration
    asks for a box of cube_ky x cube_kx k-pixels, the beams with
    -ky/2 <= h_y < ky/2 and -kx/2 <= h_x < kx/2 (a detector of that many
    pixels at the grid's own k-sampling)."""
    ky, kx = int(getattr(cfg, "cube_ky", 0)), int(getattr(cfg, "cube_kx", 0))
    if ky > 0 and kx > 0:
        hy = np.arange(-(ky // 2), ky - ky // 2)
        hx = np.arange(-(kx // 2), kx - kx // 2)
        HY, HX = np.meshgrid(hy, hx, indexing="ij")
        return np.stack([HY.ravel(), HX.ravel()], axis=1).astype(np.int64)
    return disc_beams(cfg.ny, cfg.nx, cfg.ly, cfg.lx, lam, cfg.theta_det)


def detector_subsampling(cfg):
    """(dfy, dfx): the subsampling of the detector beams (h = 0 mod df); a
    configuration without dfy/dfx, or with 0, takes the probe's (fy, fx)
    (Algorithm 4, first step: the output beams PRISM-subsampled)."""
    dfy = getattr(cfg, "dfy", 0) or cfg.fy
    dfx = getattr(cfg, "dfx", 0) or cfg.fx
    return int(dfy), int(dfx)


class Geometry:
    """All host geometry of one configuration (Algorithm 5, build steps)."""

    def __init__(self, cfg, lam, parents_override=None):
        self.cfg = cfg
        self.lam = lam
        ny, nx, ly, lx = cfg.ny, cfg.nx, cfg.ly, cfg.lx
        # full aperture (for the probe normalisation) and retained beams
        self.h_full = disc_beams(ny, nx, ly, lx, lam, cfg.alpha)
        self.h_beam = disc_beams(ny, nx, ly, lx, lam, cfg.alpha, cfg.fy, cfg.fx)
        # detector beams: subsampled by (dfy, dfx), 0 meaning the probe's f
        # (qEELS resolves one axis at 1 there, Sec. 2.2.6)
        self.dfy, self.dfx = detector_subsampling(cfg)
        self.h_det = disc_beams(ny, nx, ly, lx, lam, cfg.theta_det, self.dfy, self.dfx)
        # the 4D cube's complete output basis: every beam inside the detector
        # disc, unsubsampled (Sec. 2.2.6: S2 cannot be reduced for the cube),
        # or a box of k-pixels
        self.h_cube = cube_basis(cfg, lam)
        self.psi_full = aperture_function(self.h_full, ly, lx, lam, cfg.defocus, cfg.cs)
        self.psi_beam = aperture_function(self.h_beam, ly, lx, lam, cfg.defocus, cfg.cs)
        if parents_override is None:
            self.p1 = hex_ring_parents(self.h_beam, ly, lx, cfg.nrad1, cfg.nang1)
            self.p2 = hex_ring_parents(self.h_det, ly, lx, cfg.nrad2, cfg.nang2)
        else:
            self.p1, self.p2 = parents_override
        self.h_p1 = self.h_beam[self.p1]
        self.h_p2 = self.h_det[self.p2]
        self.w1 = sibson_weights(self.h_p1, self.h_beam, ly, lx)
        self.w2 = sibson_weights(self.h_p2, self.h_det, ly, lx)

    @property
    def B(self):
        return len(self.h_beam)

    @property
    def n_det(self):
        return len(self.h_det)
