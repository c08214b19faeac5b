"""Pins of the oracle's beam geometry and Sibson weights (CPU only)."""
import math
import os

import numpy as np
import pytest

from oracle import geometry as G, physics as ph
from conftest import read_golden


def test_hex_ring_counts(golden_dir):
    """Pin 8: 1 + 3 n (n+1) parents -- 61 at n_radial = 4 as the paper prints
    -- on a dense aperture (no two samples snap to one beam)."""
    lam = ph.wavelength(100e3)
    h = G.disc_beams(512, 512, 200.0, 200.0, lam, 0.030)
    for nrad, nang, count in read_golden(os.path.join(golden_dir, "hex_ring_counts.txt")):
        p = G.hex_ring_parents(h, 200.0, 200.0, int(nrad), int(nang))
        assert len(p) == int(count)
        assert len(set(p.tolist())) == len(p)
        assert p[0] == int(np.nonzero((h[:, 0] == 0) & (h[:, 1] == 0))[0][0])


def test_subsampled_beam_sets():
    """Aperture / detector beam counts of the 128^2, 10 A, 200 keV cell:
    the 20 mrad disc holds 193 beams, 45 of them with h = 0 mod 2; the
    40 mrad detector holds 193 beams with h = 0 mod 2 (lattice-point counts
    of discs of radius 7.98 and 3.99 grid steps)."""
    lam = ph.wavelength(200e3)
    full = G.disc_beams(128, 128, 10.0, 10.0, lam, 0.020)
    sub = G.disc_beams(128, 128, 10.0, 10.0, lam, 0.020, 2, 2)
    det = G.disc_beams(128, 128, 10.0, 10.0, lam, 0.040, 2, 2)
    # count lattice points with |k| <= r independently
    def lattice(r):
        n = int(math.floor(r))
        return sum(1 for a in range(-n, n + 1) for b in range(-n, n + 1) if a * a + b * b <= r * r)
    r1 = 0.020 / lam * 10.0
    assert len(full) == lattice(r1) == 193
    assert len(sub) == lattice(r1 / 2) == 45
    assert len(det) == lattice(2 * r1 / 2) == 193
    assert np.all(sub % 2 == 0)


def _random_parents(rng, n, span=9):
    pts = set()
    while len(pts) < n:
        pts.add((int(rng.integers(-span, span + 1)), int(rng.integers(-span, span + 1))))
    return np.array(sorted(pts), dtype=np.int64)


def _interior_queries(parents, span=9):
    hull = G.convex_hull_int(parents)
    lut = {tuple(p) for p in parents.tolist()}
    out = []
    for a in range(-span, span + 1):
        for b in range(-span, span + 1):
            if (a, b) not in lut and G._strictly_inside(hull, (a, b)):
                out.append((a, b))
    return np.array(out, dtype=np.int64)


@pytest.mark.parametrize("seed,ly,lx", [(0, 10.0, 10.0), (1, 7.0, 13.0), (2, 40.0, 40.0)])
def test_sibson_properties(seed, ly, lx):
    """Pin 7: w >= 0, sum_p w = 1, linear precision sum_p w_p q_p = q_b for
    interior queries, and w = e_p at the parents (Eq. nnw)."""
    rng = np.random.default_rng(seed)
    par = _random_parents(rng, 14)
    qs = _interior_queries(par)
    assert len(qs) > 10
    W = G.sibson_weights(par, qs, ly, lx)
    assert np.all(W >= -1e-15)
    assert np.max(np.abs(W.sum(1) - 1.0)) < 1e-12
    pq = G.beam_q(par, ly, lx)
    assert np.max(np.abs(W @ pq - G.beam_q(qs, ly, lx))) < 1e-12 * np.max(np.abs(pq))
    Wp = G.sibson_weights(par, par, ly, lx)
    assert np.array_equal(Wp, np.eye(len(par)))


def test_sibson_regular_hexagon_centre():
    """Pin 7: the centre of a regular hexagon takes 1/6 from each vertex.
    Integer points (0,+-2), (+-1,+-1) are a regular hexagon when
    L_y = L_x / sqrt(3)."""
    par = np.array([(0, 2), (0, -2), (1, 1), (1, -1), (-1, 1), (-1, -1)])
    W = G.sibson_weights(par, np.array([(0, 0)]), 10.0 / math.sqrt(3.0), 10.0)
    assert np.max(np.abs(W - 1.0 / 6.0)) < 1e-13


def _raster_sibson(pq, qb, res=700):
    """Brute force: sample a square around qb; samples nearer to qb than to
    every parent belong to the new cell; each is credited to its nearest
    parent.  The square grows until the cell does not touch its border."""
    d = np.sqrt(np.sum((pq - qb) ** 2, axis=1))
    R = float(np.min(d))
    while True:
        t = (np.arange(res) + 0.5) / res * 2 * R - R
        Y, X = np.meshgrid(t + qb[0], t + qb[1], indexing="ij")
        pts = np.stack([Y.ravel(), X.ravel()], 1)
        dq = np.sum((pts - qb) ** 2, 1)
        dp = ((pts[:, None, :] - pq[None]) ** 2).sum(-1)
        inside = (dq < dp.min(1)).reshape(res, res)
        if not (inside[0].any() or inside[-1].any() or inside[:, 0].any() or inside[:, -1].any()):
            break
        R *= 1.5
    owner = np.argmin(dp[inside.ravel()], axis=1)
    w = np.bincount(owner, minlength=len(pq)).astype(float)
    return w / w.sum()


@pytest.mark.parametrize("seed", [3, 4, 5])
def test_sibson_against_raster(seed):
    """Pin 7: polygon-clipping weights agree with a brute-force raster
    estimate of the stolen areas to 2e-3."""
    rng = np.random.default_rng(seed)
    par = _random_parents(rng, 12, span=6)
    qs = _interior_queries(par, span=6)
    pick = qs[rng.choice(len(qs), size=min(4, len(qs)), replace=False)]
    W = G.sibson_weights(par, pick, 9.0, 11.0)
    pq = G.beam_q(par, 9.0, 11.0)
    for i, qb in enumerate(G.beam_q(pick, 9.0, 11.0)):
        wr = _raster_sibson(pq, qb)
        assert np.max(np.abs(W[i] - wr)) < 2e-3


def test_hull_rule_linear_on_edges():
    """Hull-boundary reading: a query on a hull edge takes the two end
    points' linear weights; outside queries project to the nearest edge."""
    par = np.array([(0, 0), (0, 4), (4, 0), (4, 4), (2, 2)])
    W = G.sibson_weights(par, np.array([(0, 1), (1, 4), (-2, 2)]), 10.0, 10.0)
    assert np.allclose(W[0], [0.75, 0.25, 0, 0, 0], atol=1e-15)
    assert np.allclose(W[1], [0, 0.75, 0, 0.25, 0], atol=1e-15)
    assert np.allclose(W[2], [0.5, 0.5, 0, 0, 0], atol=1e-15)


def test_hull_rule_on_a_collinear_parent_set():
    """Parents all on one line (a ring of two samples): the hull is a
    segment, and a query on it or off it takes the linear weights of the
    two consecutive parents around its projection -- never of the segment's
    far end (reading of the hull rule for a degenerate hull)."""
    parents = np.array([[0, 0], [0, 5], [0, -5]])
    queries = np.array([[0, 3], [0, 4], [0, -2], [2, 1], [-1, 7]])
    W = G.sibson_weights(parents, queries, 7.5, 7.5)
    np.testing.assert_allclose(W[0], [0.4, 0.6, 0.0], atol=1e-15)
    np.testing.assert_allclose(W[1], [0.2, 0.8, 0.0], atol=1e-15)
    np.testing.assert_allclose(W[2], [0.6, 0.0, 0.4], atol=1e-15)
    np.testing.assert_allclose(W[3], [0.8, 0.2, 0.0], atol=1e-15)
    np.testing.assert_allclose(W[4], [0.0, 1.0, 0.0], atol=1e-15)
