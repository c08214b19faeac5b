"""Forward-physics primitives (paper Sec. 2.1, "Grid, probe and specimen").

Grid: pixel r = (r_y, r_x), corner origin, physical position r_y L_y / N_y.
Beams: signed integer index h in [-N/2, N/2) per axis, spatial frequency
q = (h_y / L_y, h_x / L_x).  The DFT used for propagation is numpy's
(unnormalised forward, 1/G inverse); the detector transform is the unitary
DFT F_u = G^{-1/2} * fft2.
"""
import numpy as np
import scipy.fft as sfft

# library FFT (pocketfft); threads only change speed, not the definition
_WORKERS = -1

M0C2_EV = 510998.95          # electron rest energy (CODATA 2018), eV
HC_EV_A = 12398.419843320026  # h*c (CODATA 2018), eV*Angstrom


def wavelength(e0: float) -> float:
    """Relativistic electron wavelength in Angstrom for beam energy e0 (eV).
    The paper uses lambda without a formula (Eq. propagator); this is the
    standard relativistic form."""
    return HC_EV_A / np.sqrt(e0 * (2.0 * M0C2_EV + e0))


def interaction_constant(e0: float) -> float:
    """sigma in rad/(V*Angstrom) (Sec. 2.1, T_j = exp(i sigma V_j)); the
    standard relativistic interaction constant."""
    lam = wavelength(e0)
    return (2.0 * np.pi / (lam * e0)) * (M0C2_EV + e0) / (2.0 * M0C2_EV + e0)


def signed_index(n: int) -> np.ndarray:
    """Signed DFT index of each corner-origin bin: 0..n/2-1, -n/2..-1."""
    k = np.arange(n)
    return np.where(k < (n + 1) // 2, k, k - n)


def frequencies(ny: int, nx: int, ly: float, lx: float):
    """(q_y, q_x) grids in 1/Angstrom on the corner-origin DFT layout."""
    qy = signed_index(ny) / ly
    qx = signed_index(nx) / lx
    return np.meshgrid(qy, qx, indexing="ij")


def propagator(ny, nx, ly, lx, lam, dz) -> np.ndarray:
    """Fresnel transfer function P(q) = exp(-i pi lambda dz |q|^2)
    (Eq. propagator)."""
    qy, qx = frequencies(ny, nx, ly, lx)
    return np.exp(-1j * np.pi * lam * dz * (qy ** 2 + qx ** 2))


def transmission(V: np.ndarray, sigma: float) -> np.ndarray:
    """T_j = exp(i sigma V_j) (Sec. 2.1)."""
    return np.exp(1j * sigma * V)


def propagate(psi: np.ndarray, P: np.ndarray) -> np.ndarray:
    """Fresnel operator: F^{-1}[P * F psi] over the last two axes (Eq. propagator)."""
    f = sfft.fft2(psi, axes=(-2, -1), workers=_WORKERS)
    return sfft.ifft2(P * f, axes=(-2, -1), workers=_WORKERS)


def step(psi: np.ndarray, T: np.ndarray, P: np.ndarray) -> np.ndarray:
    """One multislice step: transmit then propagate, psi -> P (T psi) (Sec. 2.1)."""
    return propagate(T * psi, P)


def unitary_dft(x: np.ndarray) -> np.ndarray:
    """Detector transform F_u = G^{-1/2} * DFT, unitary on the grid."""
    g = x.shape[-1] * x.shape[-2]
    return sfft.fft2(x, axes=(-2, -1), workers=_WORKERS) / np.sqrt(g)


def plane_wave(h, ny: int, nx: int, sign: int = +1) -> np.ndarray:
    """exp(sign * 2 pi i h . r / N) on the grid (unit modulus; Algorithm 2:
    S_b = F^{-1}[delta_h] read with no 1/G factor)."""
    ry = np.arange(ny)[:, None]
    rx = np.arange(nx)[None, :]
    # reduce h.r modulo N in integers so the phase argument stays exact
    ph = np.mod(int(h[0]) * ry, ny) / ny + np.mod(int(h[1]) * rx, nx) / nx
    return np.exp(sign * 2j * np.pi * ph)
