"""Pins of the oracle's hand-written reverse pass (oracle/grad.py) by
central finite differences of its own forward map (step 1e-4), which share
none of the reverse-pass code: occupancy, transition amplitude (real and
imaginary part), defocus, Cs, and directional derivatives along seeded
random fields for the slice potentials and the transition potentials H.
Both reconstruction forms; several planes, f = 2 crop windows smaller than
the grid, non-zero defocus and Cs so that the probe phase is not flat."""
import numpy as np
import pytest

import synth
from oracle import bip as obip
from oracle import grad as og

H_STEP = 1e-4


def small_case(recon="magnitude"):
    cfg = synth.config1().replace(name="grad", ny=64, nx=64, ly=5.0, lx=5.0, nz=4, cells_y=2, cells_x=2, win=32,
                                  fy=2, fx=2, ion_slices=(1, 3), ion_cells=(0, 1), defocus=30.0, cs=2.0e5,
                                  recon=recon, scan_y=(10.0, 6.0, 4), scan_x=(12.0, 5.0, 4))
    sp = synth.make_specimen(cfg)
    pr = obip.make_problem(sp)
    rng = np.random.default_rng(5)
    par = og.Params(pr)
    par.occ = 1.0 + 0.2 * rng.standard_normal(len(pr.ion))
    par.amp = (1.0 + 0.2 * rng.standard_normal(par.amp.shape)) * np.exp(0.3j * rng.standard_normal(par.amp.shape))
    I0 = og.forward(pr, par)
    target = I0 * (1.0 + 0.1 * rng.standard_normal(I0.shape))
    return pr, par, target


@pytest.fixture(scope="module", params=["magnitude", "complex"])
def case(request):
    pr, par, target = small_case(request.param)
    L, g = og.gradients(pr, par, target)
    return pr, par, target, L, g


def central(pr, par, target, setter, h=H_STEP):
    p1, p2 = par.copy(), par.copy()
    setter(p1, +h)
    setter(p2, -h)
    return (og.loss(pr, p1, target) - og.loss(pr, p2, target)) / (2.0 * h)


def close(fd, an, rtol):
    assert abs(fd - an) <= rtol * max(abs(fd), abs(an)), (fd, an)


def test_forward_at_defaults_is_the_map(case):
    pr, *_ = case
    ref = obip.bip_map(pr).map
    assert np.max(np.abs(og.forward(pr, og.Params(pr)) - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_loss_value(case):
    pr, par, target, L, _ = case
    assert L == pytest.approx(og.loss(pr, par, target), rel=1e-14)
    assert L > 0.0


def test_occupancy(case):
    pr, par, target, _, g = case
    for k in range(len(pr.ion)):
        def s(p, d, k=k):
            p.occ[k] += d
        close(central(pr, par, target, s), g["occ"][k], 1e-8)


def test_amplitude(case):
    pr, par, target, _, g = case
    for k, n in ((0, 0), (1, 2)):
        def sr(p, d, k=k, n=n):
            p.amp[k, n] += d

        def si(p, d, k=k, n=n):
            p.amp[k, n] += 1j * d
        close(central(pr, par, target, sr), g["amp"][k, n].real, 1e-6)
        close(central(pr, par, target, si), g["amp"][k, n].imag, 1e-6)


def test_defocus_and_cs(case):
    pr, par, target, _, g = case

    def sd(p, d):
        p.defocus += d

    def sc(p, d):
        p.cs += d
    close(central(pr, par, target, sd), g["defocus"], 1e-7)
    # Cs (2e5 A) moves the phase by lam^3 q^4 per A: a larger step keeps the
    # difference above rounding
    close(central(pr, par, target, sc, h=10.0), g["cs"], 1e-6)


def test_slice_potentials_directional(case):
    """d/de L(V + e D) = sum gV D for random D, slice by slice (the S1
    sweep reaches planes 0..1, the S2 sweep planes 1..3).  D has the scale
    of the potential itself (30 V A per pixel, the atoms' peak), so that the
    1e-4 step moves the loss well above FP64 rounding."""
    pr, par, target, _, g = case
    rng = np.random.default_rng(11)
    for j in range(pr.cfg.nz):
        D = np.zeros_like(par.V)
        D[j] = pr.cfg.atom_peak * rng.standard_normal(D[j].shape)

        def s(p, d, D=D):
            p.V += d * D
        close(central(pr, par, target, s), float(np.sum(g["V"] * D)), 1e-6)


def test_transition_potentials_directional(case):
    """d/de L(H_k + e E) = Re sum conj(gH_k) E for a random complex E."""
    pr, par, target, _, g = case
    rng = np.random.default_rng(13)
    for k in range(len(pr.ion)):
        E = rng.standard_normal(pr.H[k].shape) + 1j * rng.standard_normal(pr.H[k].shape)
        H0 = pr.H[k].copy()

        def L_at(e):
            pr.H[k] = H0 + e * E
            try:
                return og.loss(pr, par, target)
            finally:
                pr.H[k] = H0
        fd = (L_at(H_STEP) - L_at(-H_STEP)) / (2.0 * H_STEP)
        close(fd, float(np.real(np.sum(np.conj(g["H"][k]) * E))), 1e-6)


def test_linear_loss_occupancy_is_partials(case):
    """For a given dL/dI the occupancy gradient is sum_rho dL/dI I_tau."""
    pr, par, _, _, _ = case
    rng = np.random.default_rng(2)
    gI = rng.standard_normal(len(pr.scans))
    _, g = og.gradients(pr, par, dL_dI=gI)
    _, fw = og.forward(pr, par, keep=True)
    assert np.allclose(g["occ"], fw["partials"] @ gI, rtol=1e-13, atol=0.0)


def test_site_windows_reverse_pass():
    """The reverse pass with the sites' own crop windows (a 16-px window
    inside the context's 32 px, the other site at 32 px): the slice-potential
    and transition-potential derivatives against central differences, and
    the H derivative shaped like each site's own window."""
    cfg = synth.config1().replace(name="grad_win", ny=64, nx=64, ly=5.0, lx=5.0, nz=4, cells_y=2, cells_x=2,
                                  win=32, fy=2, fx=2, ion_slices=(1, 3), ion_cells=(0, 1), defocus=30.0, cs=2.0e5,
                                  scan_y=(10.0, 6.0, 4), scan_x=(12.0, 5.0, 4))
    sp = synth.make_specimen(cfg)
    site_win = [16, 32]
    parts, _, _ = synth.site_window_inputs(sp, site_win)
    pr = obip.make_problem(sp, site_win=site_win, H=parts)
    rng = np.random.default_rng(21)
    par = og.Params(pr)
    par.occ = 1.0 + 0.2 * rng.standard_normal(len(pr.ion))
    I0 = og.forward(pr, par)
    target = I0 * (1.0 + 0.1 * rng.standard_normal(I0.shape))
    _, g = og.gradients(pr, par, target)
    assert [h.shape[1] for h in g["H"]] == site_win
    for j in (1, 2):
        D = np.zeros_like(par.V)
        D[j] = cfg.atom_peak * rng.standard_normal(D[j].shape)

        def s(p, d, D=D):
            p.V += d * D
        close(central(pr, par, target, s), float(np.sum(g["V"] * D)), 1e-6)
    for k in range(len(pr.ion)):
        E = rng.standard_normal(pr.H[k].shape) + 1j * rng.standard_normal(pr.H[k].shape)
        H0 = pr.H[k].copy()

        def L_at(e):
            pr.H[k] = H0 + e * E
            try:
                return og.loss(pr, par, target)
            finally:
                pr.H[k] = H0
        fd = (L_at(H_STEP) - L_at(-H_STEP)) / (2.0 * H_STEP)
        close(fd, float(np.real(np.sum(np.conj(g["H"][k]) * E))), 1e-6)
