"""Pins of the oracle's forward physics (CPU only)."""
import math
import os

import numpy as np
import pytest

import synth
from oracle import bip, physics as ph
from conftest import read_golden


def test_constants_match_textbook(golden_dir):
    for e0, lam, sig in read_golden(os.path.join(golden_dir, "electron_constants.txt")):
        assert abs(ph.wavelength(e0) - lam) / lam < 2e-4
        assert abs(ph.interaction_constant(e0) - sig) / sig < 2e-4


def test_signed_index_layout():
    assert ph.signed_index(8).tolist() == [0, 1, 2, 3, -4, -3, -2, -1]
    assert ph.signed_index(5).tolist() == [0, 1, 2, -2, -1]


def test_norm_conservation_real_potential():
    """Pin 1: T is unimodular and P has |P| = 1, so a step with real V keeps
    the norm (unitary steps, Sec. 2.3.1) -- over 100 slices to 1e-12."""
    rng = np.random.default_rng(1)
    ny = nx = 64
    lam = ph.wavelength(200e3)
    sig = ph.interaction_constant(200e3)
    P = ph.propagator(ny, nx, 8.0, 8.0, lam, 2.0)
    psi = rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))
    n0 = np.linalg.norm(psi)
    for j in range(100):
        V = 40.0 * rng.random((ny, nx))
        psi = ph.step(psi, ph.transmission(V, sig), P)
    assert abs(np.linalg.norm(psi) - n0) / n0 < 1e-12


def test_free_space_plane_wave_closed_form():
    """Pin 2: with V = 0 a plane wave h is an eigenfunction of the step;
    after n steps it has gained exp(-i pi lambda n dz |q_h|^2), with
    q_h = (h_y/L_y, h_x/L_x) -- the sign, lambda and the index-to-frequency
    map all enter.  Expected phases are computed here from the numbers."""
    ny, nx, ly, lx, dz = 32, 48, 6.0, 9.0, 1.5
    e0 = 300e3
    lam = 12398.419843320026 / math.sqrt(e0 * (2 * 510998.95 + e0))
    P = ph.propagator(ny, nx, ly, lx, ph.wavelength(e0), dz)
    T = np.ones((ny, nx))
    for h in [(3, -2), (-16, 23), (0, -24), (15, 1)]:
        pw = ph.plane_wave(h, ny, nx, +1)
        psi = pw.copy()
        n = 7
        for _ in range(n):
            psi = ph.step(psi, T, P)
        q2 = (h[0] / ly) ** 2 + (h[1] / lx) ** 2
        expect = np.exp(-1j * math.pi * lam * n * dz * q2) * pw
        assert np.max(np.abs(psi - expect)) < 1e-13


def test_free_space_focus_of_defocused_probe():
    """The propagator sign makes a probe with aperture phase
    exp(+i pi lambda z |q|^2) (defocus -z) focus after propagating z: its
    peak intensity grows to the in-focus value."""
    cfg = synth.tiny_config(ny=64, nx=64, ly=10.0, lx=10.0, nz=1, dz=150.0)
    sp = synth.make_specimen(cfg)
    sp.V[:] = 0.0
    pr0 = bip.make_problem(sp)
    focused = bip.exact_probe(pr0, (32.0, 32.0))
    pr1 = bip.make_problem(sp, defocus=-150.0)
    defoc = bip.exact_probe(pr1, (32.0, 32.0))
    prop = ph.step(defoc, np.ones_like(defoc.real), pr1.P)
    assert np.max(np.abs(prop - focused)) < 1e-12
    assert np.max(np.abs(defoc)) < 0.9 * np.max(np.abs(focused))


def test_probe_unit_norm_and_periodicity():
    """Pin 13: at f = 1 the probe has unit norm (normalisation reading); at
    f > 1 the synthesised probe is N/f periodic (Sec. 2.2.2) and keeps a
    near-unit norm inside one period."""
    cfg = synth.config1()
    sp = synth.make_specimen(cfg, with_potential=False)
    sp.V = np.zeros((cfg.nz, cfg.ny, cfg.nx))
    pr1 = bip.make_problem(sp, fy=1, fx=1)
    psi = bip.exact_probe(pr1, (64.0, 64.0))
    assert abs(np.linalg.norm(psi) - 1.0) < 1e-13
    pr2 = bip.make_problem(sp)
    geo = pr2.geo
    C = bip.illumination(pr2, geo.h_beam, geo.psi_beam, np.array([[64.0, 64.0]]))[:, 0]
    spec = np.zeros((cfg.ny, cfg.nx), complex)
    spec[geo.h_beam[:, 0] % cfg.ny, geo.h_beam[:, 1] % cfg.nx] = C
    psi_f = np.fft.ifft2(spec) * cfg.ny * cfg.nx
    per = cfg.ny // cfg.fy
    assert np.max(np.abs(psi_f - np.roll(psi_f, per, axis=0))) < 1e-13
    assert np.max(np.abs(psi_f - np.roll(psi_f, per, axis=1))) < 1e-13
    win = psi_f[32:96, 32:96]
    assert abs(np.linalg.norm(win) - 1.0) < 0.05


def _tiny_problem(**kw):
    cfg = synth.tiny_config(**kw)
    sp = synth.make_specimen(cfg)
    return bip.make_problem(sp), sp


def test_s2_reciprocity():
    """Pin 3: sum_r S2^d(r) w(r) = [F_u M_{i->exit} w]_{h_d} for random w,
    every detector beam and several planes (Eq. s2)."""
    pr, _ = _tiny_problem(nz=4)
    cfg, geo = pr.cfg, pr.geo
    rng = np.random.default_rng(3)
    for plane in (0, 2, 3):
        w = rng.standard_normal((cfg.ny, cfg.nx)) + 1j * rng.standard_normal((cfg.ny, cfg.nx))
        S2 = bip.s2_full(pr, geo.h_det, plane)
        lhs = np.sum(S2 * w[None], axis=(1, 2))
        E = ph.unitary_dft(bip.exit_operator(pr, w, plane))
        rhs = E[geo.h_det[:, 0] % cfg.ny, geo.h_det[:, 1] % cfg.nx]
        assert np.max(np.abs(lhs - rhs)) < 1e-12 * max(1.0, np.max(np.abs(rhs)))


def test_exit_operator_unitary_locality():
    """Pin 9 (i)-(ii): ||F_u M_{i->exit}(H dpsi)|| = ||H dpsi|| (Eq. loc-unitary)
    and ||H dpsi|| <= max|H| ||dpsi||_window (Eq. loc-bound)."""
    pr, _ = _tiny_problem(win=16)
    cfg = pr.cfg
    rng = np.random.default_rng(4)
    dpsi = rng.standard_normal((cfg.ny, cfg.nx)) + 1j * rng.standard_normal((cfg.ny, cfg.nx))
    Hf = bip.full_grid_H(pr, 0)
    iy, ix = pr.window_index(0)
    for Hn in Hf:
        src = Hn * dpsi
        out = ph.unitary_dft(bip.exit_operator(pr, src, int(pr.plane[0])))
        assert abs(np.linalg.norm(out) - np.linalg.norm(src)) < 1e-12 * np.linalg.norm(src)
        onwin = np.linalg.norm(dpsi[iy[:, None], ix[None, :]])
        assert np.linalg.norm(src) <= np.max(np.abs(Hn)) * onwin * (1 + 1e-12)
