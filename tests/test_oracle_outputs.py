"""Pins of the oracle's output modes (Sec. 2.2.6) and of the locality result
(Sec. 2.3.1, Eq. loc-source ... onatom), CPU only.

The 4D cube keeps every output beam, so S2 is not reduced: S1 partitioned,
the exit exact on the complete (unsubsampled) basis.  Algorithm 3 computes
exactly that by brute force -- per scan, per site and channel, a multislice
of the inelastic wave to the exit surface -- and is the cube's pin.  qEELS
partitions S2 with the resolved axis sampled at f = 1.  The locality result
says the cube's error is set by the probe on the site's window alone."""
import numpy as np
import pytest

import synth
from oracle import bip, physics as ph
from oracle.geometry import Geometry


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def small_cell(**kw):
    """4x4 cells on a 64^2 grid (10 A), three slices, the central four atoms
    of slice 1 ionized, a 32-px window (5 A) -- smaller than the grid, so
    the window and the crop matter."""
    base = dict(ny=64, nx=64, ly=10.0, lx=10.0, cells_y=4, cells_x=4, win=32, nz=3,
                ion_slices=(1, 2), ion_cells=(1, 3), scan_y=(24.0, 8.0, 3), scan_x=(24.0, 8.0, 3))
    base.update(kw)
    return synth.tiny_config(**base)


def problem(cfg, geometry=None):
    return bip.make_problem(synth.make_specimen(cfg), geometry=geometry)


def full_parents(pr):
    geo = Geometry(pr.cfg, pr.lam, parents_override=(np.arange(pr.geo.B), np.arange(pr.geo.n_det)))
    return bip.make_problem(synth.make_specimen(pr.cfg), geometry=geo)


def analytic_H(pr, k):
    """Site k's transition potentials phi_m on the whole grid (minimum-image
    offsets), tail included -- the synthetic inputs sample them on the
    window only."""
    cfg = pr.cfg
    dy, dx = cfg.ly / cfg.ny, cfg.lx / cfg.nx
    out = []
    for ax, (n, d) in enumerate(((cfg.ny, dy), (cfg.nx, dx))):
        u = np.arange(n) - pr.tau_px[k, ax]
        out.append((u - n * np.floor((u + 0.5 * n) / n)) * d)
    ddy, ddx = out[0][:, None], out[1][None, :]
    env = np.exp(-(ddy ** 2 + ddx ** 2) / (2.0 * cfg.phi_sigma ** 2))
    return np.stack([env * ((ddx + 1j * m * ddy) / cfg.phi_r0) ** abs(m) for m in cfg.channels])


# ---------------------------------------------------------------------------
# the 4D cube

@pytest.mark.parametrize("kw", [dict(), dict(fy=2, fx=2, scan_y=(20.0, 6.0, 4), scan_x=(20.0, 6.0, 4)),
                                dict(recon="complex", nz=4, ion_slices=(1, 4, 2))],
                         ids=["f1", "f2-crop", "complex-two-planes"])
def test_cube_is_algorithm3_brute_force(kw):
    """The cube through the unpartitioned S2 columns (reciprocity) equals
    Algorithm 3 run literally: the partitioned probe on the whole grid,
    every inelastic wave taken to the exit by multislice, |F_u|^2 read at
    every beam of the complete basis.  A wrong S2 sign, a subsampled or
    partitioned exit, or a missing re-tilt fails it."""
    pr = problem(small_cell(**kw))
    assert len(pr.geo.h_cube) > pr.geo.n_det or pr.cfg.fy == 1
    cube = bip.bip_cube(pr)
    assert cube.shape == (len(pr.scans), len(pr.geo.h_cube))
    assert rel(cube, bip.alg3_cube(pr)) < 1e-12


def test_cube_on_a_box_of_k_pixels():
    """The cube's basis as a box of k-pixels (16 x 12 around the zero beam,
    the shape of a pixelated detector) instead of the detector disc: still
    Algorithm 3 by brute force, beam by beam."""
    pr = problem(small_cell(cube_ky=16, cube_kx=12))
    h = pr.geo.h_cube
    assert h.shape == (192, 2)
    assert h[:, 0].min() == -8 and h[:, 0].max() == 7 and h[:, 1].min() == -6 and h[:, 1].max() == 5
    assert rel(bip.bip_cube(pr), bip.alg3_cube(pr)) < 1e-12


def test_cube_full_parent_limit_is_exact_prism():
    """Every aperture beam its own parent: the cube is exact PRISM's
    (Algorithm 2 with the exact exit), and at f = 1 that is conventional
    multislice (Algorithm 1) beam by beam."""
    pr = problem(small_cell())
    prf = full_parents(pr)
    ex = bip.exact_cube(pr)
    assert rel(bip.bip_cube(prf), ex) < 1e-12
    assert rel(ex, bip.conventional_cube(pr)) < 1e-11


def test_cube_complete_basis_needs_unreduced_s2():
    """The complete basis has f_y f_x times the map's subsampled detector
    beams; its detector sum approximates the map (which rescales the coarse
    sum by f_y f_x) to the S2 reconstruction and Poisson-summation error,
    not exactly."""
    cfg = synth.config1()
    pr = problem(cfg)
    n_full = len(pr.geo.h_cube)
    assert n_full == 793 and pr.geo.n_det == 193
    cube = bip.bip_cube(pr)
    m = bip.bip_map(pr).map
    assert np.all(cube >= 0.0)
    assert 1e-7 < rel(cube.sum(axis=1), m) < 1e-3


# ---------------------------------------------------------------------------
# qEELS

def test_qeels_needs_the_resolved_axis_at_f1():
    pr = problem(synth.config1())            # detector beams subsampled by 2 on both axes
    for axis in (0, 1):
        with pytest.raises(ValueError, match="f = 1"):
            bip.bip_qeels(pr, axis)


@pytest.mark.parametrize("axis", [0, 1])
def test_qeels_bins_partition_the_map(axis):
    """With the resolved axis at f = 1 the bins are the distinct beam
    components along it and their sum is the map of the same detector set
    (exactly: the bins partition the beams), the invariant the paper
    reports."""
    cfg = synth.config1().replace(**({"dfy": 1} if axis == 0 else {"dfx": 1}))
    pr = problem(cfg)
    h = pr.geo.h_det[:, axis]
    bins, q = bip.bip_qeels(pr, axis)
    assert np.all(np.diff(bins) > 0) and set(bins.tolist()) == set(h.tolist())
    assert np.any(bins % 2 != 0)                       # resolved at f = 1
    assert np.all(pr.geo.h_det[:, 1 - axis] % 2 == 0)  # the other axis subsampled
    assert rel(q.sum(axis=1), bip.bip_map(pr).map) < 1e-13


def test_qeels_full_parents_against_exact_beams():
    """Full detector parents: qEELS is the exact per-beam intensity binned,
    times the perpendicular subsampling (the detector-side reading);
    against the complete basis binned, that reading holds to 1e-4 here."""
    cfg = synth.config1().replace(dfx=1)
    pr = problem(cfg)
    prf = full_parents(pr)
    bins, q = bip.bip_qeels(prf, 1)
    hd = pr.geo.h_det[:, 1]
    ex = bip.exact_cube(pr, det_h=pr.geo.h_det) * cfg.fy
    assert rel(q, np.stack([ex[:, hd == b].sum(axis=1) for b in bins], axis=1)) < 1e-12
    full = bip.exact_cube(pr)
    hc = pr.geo.h_cube[:, 1]
    assert rel(q, np.stack([full[:, hc == b].sum(axis=1) for b in bins], axis=1)) < 1e-4


def test_qeels_f1_is_conventional_multislice_binned():
    """At f = 1, full parents, qEELS is Algorithm 1 resolved over the
    detector beams and binned -- ground truth for the binning itself."""
    pr = full_parents(problem(small_cell()))
    for axis in (0, 1):
        bins, q = bip.bip_qeels(pr, axis)
        conv = bip.conventional_cube(pr, det_h=pr.geo.h_det)
        h = pr.geo.h_det[:, axis]
        assert rel(q, np.stack([conv[:, h == b].sum(axis=1) for b in bins], axis=1)) < 1e-11


# ---------------------------------------------------------------------------
# the locality result (pin 9 iii)

def _hybrid(pr):
    """Probe partitioned on the windows of the plane's sites and exact
    (PRISM, every beam propagated) everywhere else."""
    def probe(scans, plane):
        pp = bip.partitioned_probe(pr, scans, plane)
        out = bip.prism_probe(pr, scans, plane)
        for k in np.nonzero(pr.plane == plane)[0]:
            iy, ix = pr.window_index(k)
            out[:, iy[:, None], ix[None, :]] = pp[:, iy[:, None], ix[None, :]]
        return out
    return probe


def test_locality_hybrid_probe_equals_partitioned():
    """Pin 9 (iii): the cube of a probe that is partitioned on the window
    and exact elsewhere equals the fully partitioned cube, up to the tail of
    H_n outside the window (Eq. loc-source: only the window's probe error
    reaches the inelastic source).  Brute force (Algorithm 3) with H_n
    evaluated on the whole grid, its tail included."""
    pr = problem(small_cell(nrad1=1))
    hf = lambda k: analytic_H(pr, k)
    part = bip.alg3_cube(pr, h_full=hf)
    hyb = bip.alg3_cube(pr, h_full=hf, probe=_hybrid(pr))
    exact = bip.alg3_cube(pr, h_full=hf, probe=lambda sc, pl: bip.prism_probe(pr, sc, pl))
    d_hyb, d_exact = rel(hyb, part), rel(exact, part)
    # the tail of H outside the 5 A window is a few 1e-5 of its peak
    tails = []
    for k in range(len(pr.ion)):
        iy, ix = pr.window_index(k)
        h = analytic_H(pr, k)
        inside = np.abs(h[:, iy[:, None], ix[None, :]]).max()
        h[:, iy[:, None], ix[None, :]] = 0.0
        tails.append(np.abs(h).max() / inside)
    assert max(tails) < 5e-5
    assert d_hyb < 1e-8
    assert d_exact > 1e3 * d_hyb


@pytest.mark.parametrize("mode", ["magnitude", "complex"])
def test_locality_bound_and_on_atom_error(mode):
    """Eq. loc-bound and loc-unitary for every scan, site and channel: the
    exit amplitude error over the complete basis, ||F_u M (H_n dpsi)||,
    equals ||H_n dpsi|| and is at most max|H_n| ||dpsi||_window; the cube's
    error against exact PRISM falls with the on-atom error (Eq. onatom) as
    parents are added, staying proportional to it."""
    errs, eps_mean = [], []
    for nr in (1, 2, 3):
        pr = problem(small_cell(nrad1=nr, recon=mode))
        for plane in sorted(set(pr.plane.tolist())):
            pp = bip.partitioned_probe(pr, pr.scans, plane)
            pe = bip.prism_probe(pr, pr.scans, plane)
            for k in np.nonzero(pr.plane == plane)[0]:
                iy, ix = pr.window_index(k)
                dwin = np.sqrt(np.sum(np.abs(pp - pe)[:, iy[:, None], ix[None, :]] ** 2, axis=(1, 2)))
                for Hn in bip.full_grid_H(pr, k):
                    src = Hn[None] * (pp - pe)
                    amp = ph.unitary_dft(bip.exit_operator(pr, src, plane))
                    lhs = np.sqrt(np.sum(np.abs(amp) ** 2, axis=(1, 2)))
                    norm_src = np.sqrt(np.sum(np.abs(src) ** 2, axis=(1, 2)))
                    assert np.all(np.abs(lhs - norm_src) <= 1e-12 * norm_src)
                    assert np.all(norm_src <= np.abs(Hn).max() * dwin * (1 + 1e-12))
        part = bip.alg3_cube(pr)
        exact = bip.alg3_cube(pr, probe=lambda sc, pl, pr=pr: bip.prism_probe(pr, sc, pl))
        errs.append(rel(part, exact))
        eps_mean.append(np.mean([bip.on_atom_error(pr, k, pr.scans, mode) for k in range(len(pr.ion))]))
    assert errs[0] > errs[1] > errs[2] > 0.0
    assert eps_mean[0] > eps_mean[1] > eps_mean[2] > 0.0
    ratio = np.array(errs) / np.array(eps_mean)
    assert ratio.max() / ratio.min() < 3.0, (errs, eps_mean)


def test_on_atom_error_zero_at_full_parents():
    pr = full_parents(problem(small_cell()))
    for k in range(len(pr.ion)):
        assert np.max(bip.on_atom_error(pr, k, pr.scans)) < 1e-12
