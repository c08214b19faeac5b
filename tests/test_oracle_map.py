"""Map-level pins of the oracle (Algorithms 1, 4, 5), CPU only."""
import numpy as np
import pytest

import synth
from oracle import bip, geometry as G, physics as ph


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def c1():
    cfg = synth.config1()
    sp = synth.make_specimen(cfg)
    pr = bip.make_problem(sp)
    return sp, pr, bip.exact_map(pr)


def test_alg4_equals_conventional_multislice():
    """Pin 4: at f = 1 with a window covering the grid, the dual-matrix map
    (Algorithm 4) equals per-probe conventional multislice (Algorithm 1),
    the paper's ground truth -- this fixes the coupling equation, the plane
    convention, S2's construction and the probe normalisation."""
    cfg = synth.tiny_config()
    sp = synth.make_specimen(cfg)
    pr = bip.make_problem(sp)
    assert len(pr.ion) == 4 and pr.cfg.win == pr.cfg.ny
    a4 = bip.exact_map(pr).map
    a1 = bip.conventional_map(pr)
    assert rel(a4, a1) < 1e-11


def test_alg4_equals_conventional_thicker():
    """Pin 4 with sites in two different planes and a thicker cell."""
    cfg = synth.tiny_config(nz=5, ion_slices=(1, 4), ion_cells=(0, 1))
    sp = synth.make_specimen(cfg)
    pr = bip.make_problem(sp)
    assert len(set(pr.plane.tolist())) == 3
    assert rel(bip.exact_map(pr).map, bip.conventional_map(pr)) < 1e-11


def test_full_detector_unitarity():
    """Pin 6: with every grid beam on the detector (f = 1, full window) the
    map is sum_{tau,n} ||H_n psi(., rho)||^2 by unitarity of F M
    (Eq. loc-unitary); needs no S2."""
    cfg = synth.tiny_config(theta_det=10.0)
    sp = synth.make_specimen(cfg)
    pr = bip.make_problem(sp)
    assert pr.geo.n_det == cfg.ny * cfg.nx
    m = bip.exact_map(pr).map
    expect = np.zeros(len(pr.scans))
    for p, rho in enumerate(pr.scans):
        for k in range(len(pr.ion)):
            psi = bip.elastic_probe_at(pr, rho, int(pr.plane[k]))
            for Hn in bip.full_grid_H(pr, k):
                expect[p] += np.sum(np.abs(Hn * psi) ** 2)
    assert rel(m, expect) < 1e-12


@pytest.mark.parametrize("mode", ["magnitude", "complex"])
def test_full_parent_limit(c1, mode):
    """Pin 5: every beam its own parent (w = I) reduces Algorithm 5 to the
    exact dual-matrix map term by term (Eq. part-exact), in both
    reconstruction modes (magnitude preservation is exact there)."""
    sp, pr, ex = c1
    geo = G.Geometry(pr.cfg, pr.lam, parents_override=(np.arange(pr.geo.B), np.arange(pr.geo.n_det)))
    assert np.array_equal(geo.w1, np.eye(geo.B))
    prf = bip.make_problem(sp, geometry=geo)
    m = bip.bip_map(prf, mode=mode).map
    assert rel(m, ex.map) < 1e-13


@pytest.mark.parametrize("mode", ["magnitude", "complex"])
def test_zero_thickness_envelopes_interpolate_exactly(mode):
    """With dz = 0 every de-tilted parent column equals the same field
    (prod_j T_j), for S1 and S2 alike, so any convex weights reproduce the
    exact map at any parent count.  A wrong de-tilt/re-tilt sign or a
    misplaced carrier breaks this."""
    cfg = synth.config1().replace(dz=0.0)
    sp = synth.make_specimen(cfg)
    pr = bip.make_problem(sp)
    assert len(pr.geo.p1) < pr.geo.B and len(pr.geo.p2) < pr.geo.n_det
    ex = bip.exact_map(pr).map
    assert rel(bip.bip_map(pr, mode=mode).map, ex) < 1e-12


def test_parent_sweep_converges(c1):
    """Pin 14: with magnitude preservation the map error against the exact
    map falls as n_radial grows (Sec. 3 "Accuracy vs. parent counts")."""
    sp, pr, ex = c1
    errs = []
    for nr in (1, 2, 3):
        p = bip.make_problem(sp, nrad1=nr, nrad2=nr)
        errs.append(rel(bip.bip_map(p).map, ex.map))
    assert errs[0] > errs[1] > errs[2]
    assert errs[0] < 5e-3


def test_magnitude_preservation_restores_amplitude(c1):
    """Pin 11: |sum_p w S_p| <= sum_p w |S_p| pointwise (Sec. 2.2.3), and the
    naive complex average loses map intensity that magnitude preservation
    restores."""
    sp, pr, ex = c1
    cfg, geo = pr.cfg, pr.geo
    W1 = bip.s1_windows(pr, geo.h_p1)
    U = np.tensordot(geo.w1, W1[0], axes=(1, 0))
    A = np.tensordot(geo.w1, np.abs(W1[0]), axes=(1, 0))
    assert np.all(np.abs(U) <= A * (1 + 1e-12))
    mag = bip.bip_map(pr, mode="magnitude").map
    cpx = bip.bip_map(pr, mode="complex").map
    assert cpx.sum() < mag.sum()
    assert abs(mag.sum() - ex.map.sum()) < abs(cpx.sum() - ex.map.sum())


def test_naive_mode_equals_beamlet_synthesis(c1):
    """Pin 10: in complex mode the probe the window reconstruction delivers,
    sum_b c_b(rho) S1^b(r), equals the beamlet-basis synthesis
    sum_p psi_hat_p(r, rho) S^dt_p(r) with psi_hat_p the inverse transform
    of w_{p,b} Psi(h_b) e^{-2 pi i h_b.rho/N} (Eq. part-probe / part-basis)."""
    sp, pr, ex = c1
    cfg, geo = pr.cfg, pr.geo
    k = 1
    iy, ix = pr.window_index(k)
    W1 = bip.s1_windows(pr, geo.h_p1)[k]
    S1w = bip.reconstruct(W1, geo.w1, geo.h_beam, iy, ix, cfg.ny, cfg.nx, +1, "complex")
    rhos = pr.scans[[0, 37, 200]]
    C = bip.illumination(pr, geo.h_beam, geo.psi_beam, rhos)
    norm = np.sqrt(cfg.ny * cfg.nx * np.sum(np.abs(geo.psi_full) ** 2))
    for j, rho in enumerate(rhos):
        via_recon = np.tensordot(C[:, j], S1w, axes=(0, 0))
        via_beamlets = np.zeros_like(via_recon)
        for p in range(len(geo.p1)):
            spec = np.zeros((cfg.ny, cfg.nx), complex)
            ramp = np.exp(-2j * np.pi * (geo.h_beam[:, 0] * rho[0] / cfg.ny + geo.h_beam[:, 1] * rho[1] / cfg.nx))
            spec[geo.h_beam[:, 0] % cfg.ny, geo.h_beam[:, 1] % cfg.nx] = geo.w1[:, p] * geo.psi_beam * ramp
            psi_hat = np.fft.ifft2(spec) * cfg.ny * cfg.nx * cfg.fy * cfg.fx / norm
            via_beamlets += psi_hat[iy[:, None], ix[None, :]] * W1[p]
        assert np.max(np.abs(via_recon - via_beamlets)) < 1e-12 * np.max(np.abs(via_recon))


def test_linear_envelopes_reproduced(c1):
    """Sibson linear precision through the window reconstruction: parents
    whose de-tilted windows are affine in q_p give U_b affine in q_b for
    every beam inside (or on) the parents' hull."""
    sp, pr, ex = c1
    cfg, geo = pr.cfg, pr.geo
    rng = np.random.default_rng(7)
    w = cfg.win
    a0, ay, ax = (rng.standard_normal((w, w)) + 1j * rng.standard_normal((w, w)) for _ in range(3))
    qp = G.beam_q(geo.h_p1, cfg.ly, cfg.lx)
    dt = a0[None] + ay[None] * qp[:, 0, None, None] + ax[None] * qp[:, 1, None, None]
    iy, ix = pr.window_index(0)
    S = bip.reconstruct(dt, geo.w1, geo.h_beam, iy, ix, cfg.ny, cfg.nx, +1, "complex")
    S = S * bip.window_phase(geo.h_beam, iy, ix, cfg.ny, cfg.nx, -1)
    hull = G.convex_hull_int(geo.h_p1)
    qb = G.beam_q(geo.h_beam, cfg.ly, cfg.lx)
    n_in = 0
    for b, hb in enumerate(geo.h_beam.tolist()):
        if G._strictly_inside(hull, tuple(hb)) or tuple(hb) in {tuple(x) for x in geo.h_p1.tolist()}:
            n_in += 1
            want = a0 + ay * qb[b, 0] + ax * qb[b, 1]
            assert np.max(np.abs(S[b] - want)) < 1e-12 * np.max(np.abs(want))
    assert n_in >= 20


def test_translation_covariance(c1):
    """Pin 12: shifting specimen, sites and scans by whole pixels leaves the
    map unchanged (rho enters only as a phase ramp, Eq. probe)."""
    sp, pr, ex = c1
    cfg = sp.cfg
    sy, sx = 5, -9
    dy, dx = cfg.ly / cfg.ny, cfg.lx / cfg.nx
    atoms = sp.atoms.copy()
    atoms[:, 0] += sy * dy
    atoms[:, 1] += sx * dx
    V = np.roll(sp.V, (sy, sx), axis=(1, 2))
    scans = sp.scans + np.array([sy, sx])
    shifted = bip.Problem(cfg, atoms, sp.nch, V, sp.H, scans)
    assert rel(bip.bip_map(shifted).map, bip.bip_map(pr).map) < 1e-12


def test_subsampling_scale_consistency(c1):
    """PRISM subsampling (Sec. 2.2.2) with the f_y f_x rescale on both the
    probe and detector sides: the f = 2 exact map, corrected for the
    coarser aperture's beam count (45 beams vs 193/4), matches the f = 1
    exact map on scans within 16 px of each site to ~1%.  A missing or
    doubled f_y f_x factor on either side would be off by 4x."""
    sp, pr, ex = c1
    pr1 = bip.make_problem(sp, fy=1, fx=1)
    e1 = bip.exact_map(pr1)
    geo = pr.geo
    corr = len(geo.h_full) / (pr.cfg.fy * pr.cfg.fx * len(geo.h_beam))
    for k in range(len(pr.ion)):
        near = np.all(np.abs(pr.scans - pr.tau_px[k]) < 16, axis=1)
        assert rel(corr * ex.partials[k][near], e1.partials[k][near]) < 0.03


def test_subsampling_scale_consistency_f3():
    """The same reading at f = 3 on a grid that is not a power of two (96^2,
    three cells of 32 px): the f = 3 exact map, corrected for the aperture's
    beam count (9 beams vs 109/9), matches the f = 1 exact map near each
    site within 6% (the 9-beam aperture samples the disc coarsely).  A
    missing or doubled f_y f_x on either side would be off by 9x.  The
    partitioned map stays within 1e-4 of the exact one there."""
    cfg = synth.config1().replace(name="f3", ny=96, nx=96, ly=7.5, lx=7.5, cells_y=3, cells_x=3, fy=3, fx=3,
                                  win=32, ion_cells=(1, 2), ion_slices=(1, 3), scan_y=(36.0, 3.0, 10),
                                  scan_x=(36.0, 3.0, 10))
    sp = synth.make_specimen(cfg)
    pr = bip.make_problem(sp)
    ex = bip.exact_map(pr)
    e1 = bip.exact_map(bip.make_problem(sp, fy=1, fx=1))
    geo = pr.geo
    assert len(geo.h_beam) == 9
    corr = len(geo.h_full) / (pr.cfg.fy * pr.cfg.fx * len(geo.h_beam))
    for k in range(len(pr.ion)):
        near = np.all(np.abs(pr.scans - pr.tau_px[k]) < 10, axis=1)
        assert near.sum() >= 25
        assert rel(corr * ex.partials[k][near], e1.partials[k][near]) < 0.06
    assert rel(bip.bip_map(pr).map, ex.map) < 1e-4


# ---------------------------------------------------------------------------
# per-beam terms (the cube's and qEELS's own pins: test_oracle_outputs.py)

def test_cube_alg4_equals_conventional_per_beam():
    """Pin 4 beam by beam: at f = 1 with a window covering the grid, the
    dual-matrix cube equals per-probe conventional multislice resolved over
    the detector beams -- this fixes which S2 row is which detector beam."""
    cfg = synth.tiny_config(nz=5, ion_slices=(1, 4), ion_cells=(0, 1))
    sp = synth.make_specimen(cfg)
    pr = bip.make_problem(sp)
    a4 = bip.exact_cube(pr)
    a1 = bip.conventional_cube(pr)
    assert a4.shape == (len(pr.scans), pr.geo.n_det)
    assert rel(a4, a1) < 1e-11
    # the detector sum of either is the map
    assert rel(a1.sum(axis=1), bip.conventional_map(pr)) < 1e-13


def test_golden_config1_map_is_the_oracles():
    """tests/golden/config1_map.txt (the benchmark's precision reference)
    holds exactly what the oracle computes for config 1 today."""
    import os
    here = os.path.dirname(os.path.abspath(__file__))
    stored = np.loadtxt(os.path.join(here, "golden", "config1_map.txt"))
    sp = synth.make_specimen(synth.config1())
    m = bip.bip_map(bip.make_problem(sp)).map
    assert stored.shape == m.shape
    assert np.max(np.abs(stored - m)) <= 1e-15 * np.max(np.abs(m))


def test_site_windows_restrict_the_coupling_sum(c1):
    """Eq. coupling sums over each site's own crop window Omega_tau: sites
    whose windows are smaller than the context's (w_k x w_k from
    floor(t + 1/2) - w_k/2) give exactly the map of the full windows with
    H_n zero outside each site's block -- which pins the sub-window's origin
    and the restriction of the sum -- and a visibly different map from the
    full windows with the full H (the truncation of H matters here)."""
    sp, pr, _ = c1
    site_win = [32, 64, 16, 48]
    parts, _, padded = synth.site_window_inputs(sp, site_win)
    own = bip.bip_map(bip.make_problem(sp, site_win=site_win, H=parts))
    pad = bip.bip_map(bip.make_problem(sp, H=padded))
    assert rel(own.map, pad.map) < 1e-12
    assert rel(own.partials, pad.partials) < 1e-12
    full = bip.bip_map(pr)
    assert rel(own.map, full.map) > 1e-4
    # a site whose window is the context's is untouched
    assert rel(own.partials[1], full.partials[1]) < 1e-12
    with pytest.raises(ValueError):
        bip.make_problem(sp, site_win=[32, 64, 16, 32], H=parts)
