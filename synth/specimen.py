"""Synthetic specimens: Gaussian atoms on an orthorhombic lattice.

Recipe (shared by every workload):
  * one atom per cell per slice at the cell centre ((c + 1/2) a on each axis)
    plus a uniform jitter in [-j, j) per axis, drawn from SplitMix64 in the
    order slice -> c_y -> c_x -> (y, x);
  * projected potential of each atom: peak * exp(-d^2 / (2 s^2)) [V*A],
    d the minimum-image distance, sampled at pixel corners r = (i dy, j dx),
    truncated at 10 s (the neglected tail is below 1e-21 of the peak);
  * ionized sites: the atoms whose slice lies in ion_slices = (s0, s1[,
    stride]) -- s0 <= s < s1, every stride-th slice from s0 -- and whose cell
    lies in ion_cells on both axes, each with the channels m in `channels`;
  * transition potential of channel m, sampled on the atom's window:
    phi_m(d) = exp(-|d|^2 / (2 sp^2)) * ((d_x + i m d_y) / r0)^|m|,
    d the physical offset of the window pixel from the atom;
  * scans: a raster (y outer, x inner) of pixel positions.

The window of a site at pixel position t (= position / pixel size) is the
win x win block of pixels starting at floor(t + 1/2) - win/2 on each axis,
wrapped periodically; H is passed to the library on exactly that block.
"""
from dataclasses import dataclass
import math
import numpy as np

from .prng import SplitMix64
from .configs import Config


def window_origin(t_px: float, win: int) -> int:
    """First (unwrapped) pixel index of the window of a site at pixel t_px."""
    return int(math.floor(t_px + 0.5)) - win // 2


@dataclass
class Specimen:
    cfg: Config
    atoms: np.ndarray        # [n_atoms, 3] float64: y (A), x (A), slice
    nch: np.ndarray          # [n_atoms] int32: channels per atom (0: not ionized)
    V: np.ndarray            # [nz, ny, nx] float64 projected potential (V*A)
    H: np.ndarray            # [n_channels_total, win, win] complex128
    scans: np.ndarray        # [P, 2] float64 scan positions (pixels, y then x)

    @property
    def ionized(self) -> np.ndarray:
        return np.nonzero(self.nch > 0)[0]


def _atoms(cfg: Config):
    rng = SplitMix64(cfg.seed)
    rows = []
    for s in range(cfg.nz):
        for cy in range(cfg.cells_y):
            for cx in range(cfg.cells_x):
                jy = rng.symmetric(cfg.jitter)
                jx = rng.symmetric(cfg.jitter)
                rows.append(((cy + 0.5) * cfg.cell_a + jy,
                             (cx + 0.5) * cfg.cell_a + jx, float(s)))
    return np.array(rows, dtype=np.float64)


def _potential(cfg: Config, atoms: np.ndarray) -> np.ndarray:
    dy, dx = cfg.ly / cfg.ny, cfg.lx / cfg.nx
    V = np.zeros((cfg.nz, cfg.ny, cfg.nx), dtype=np.float64)
    rc = 10.0 * cfg.atom_sigma
    hy = min(int(math.ceil(rc / dy)), cfg.ny // 2 - 1)
    hx = min(int(math.ceil(rc / dx)), cfg.nx // 2 - 1)
    two_s2 = 2.0 * cfg.atom_sigma ** 2
    for y, x, s in atoms:
        iy0 = int(math.floor(y / dy))
        ix0 = int(math.floor(x / dx))
        iy = np.arange(iy0 - hy, iy0 + hy + 2)
        ix = np.arange(ix0 - hx, ix0 + hx + 2)
        ddy = iy * dy - y
        ddx = ix * dx - x
        g = cfg.atom_peak * np.exp(-(ddy[:, None] ** 2 + ddx[None, :] ** 2) / two_s2)
        V[int(s)][np.ix_(iy % cfg.ny, ix % cfg.nx)] += g
    return V


def _ionized_mask(cfg: Config, n_atoms: int) -> np.ndarray:
    nch = np.zeros(n_atoms, dtype=np.int32)
    stride = cfg.ion_slices[2] if len(cfg.ion_slices) > 2 else 1
    k = 0
    for s in range(cfg.nz):
        for cy in range(cfg.cells_y):
            for cx in range(cfg.cells_x):
                if (cfg.ion_slices[0] <= s < cfg.ion_slices[1] and (s - cfg.ion_slices[0]) % stride == 0
                        and cfg.ion_cells[0] <= cy < cfg.ion_cells[1]
                        and cfg.ion_cells[0] <= cx < cfg.ion_cells[1]):
                    nch[k] = len(cfg.channels)
                k += 1
    return nch


def _transition(cfg: Config, atoms: np.ndarray, nch: np.ndarray) -> np.ndarray:
    dy, dx = cfg.ly / cfg.ny, cfg.lx / cfg.nx
    w = cfg.win
    out = []
    u = np.arange(w)
    for a in np.nonzero(nch > 0)[0]:
        y, x = atoms[a, 0], atoms[a, 1]
        oy = window_origin(y / dy, w)
        ox = window_origin(x / dx, w)
        ddy = ((oy + u) * dy - y)[:, None]
        ddx = ((ox + u) * dx - x)[None, :]
        env = np.exp(-(ddy ** 2 + ddx ** 2) / (2.0 * cfg.phi_sigma ** 2))
        for m in cfg.channels:
            poly = ((ddx + 1j * m * ddy) / cfg.phi_r0) ** abs(m)
            out.append(env * poly)
    if not out:
        return np.zeros((0, w, w), dtype=np.complex128)
    return np.stack(out).astype(np.complex128)


def scan_raster(sy, sx) -> np.ndarray:
    ys = sy[0] + sy[1] * np.arange(sy[2])
    xs = sx[0] + sx[1] * np.arange(sx[2])
    g = np.stack(np.meshgrid(ys, xs, indexing="ij"), axis=-1)
    return g.reshape(-1, 2).astype(np.float64)


def make_specimen(cfg: Config, with_potential: bool = True) -> Specimen:
    atoms = _atoms(cfg)
    nch = _ionized_mask(cfg, len(atoms))
    V = _potential(cfg, atoms) if with_potential else None
    H = _transition(cfg, atoms, nch)
    scans = scan_raster(cfg.scan_y, cfg.scan_x)
    return Specimen(cfg=cfg, atoms=atoms, nch=nch, V=V, H=H, scans=scans)


def site_window_inputs(sp: Specimen, site_win):
    """Transition potentials of the ionized sites on windows of their own:
    site k keeps the central w_k x w_k block of its samples (the same sample
    points: window_origin(t, w_k) is (win - w_k) / 2 past window_origin(t,
    win)).  Returns (per-site arrays [nch_k, w_k, w_k], their flat
    concatenation in site order, and H on the full windows with zeros
    outside each site's block)."""
    win = sp.cfg.win
    nch = sp.nch[sp.nch > 0]
    site_win = np.asarray(site_win, dtype=np.int64)
    if site_win.shape != nch.shape:
        raise ValueError("one window per ionized site")
    off = np.concatenate([[0], np.cumsum(nch)])
    parts, padded = [], np.zeros_like(sp.H)
    for k, w in enumerate(site_win.tolist()):
        o = (win - w) // 2
        h = sp.H[off[k]:off[k + 1], o:o + w, o:o + w]
        parts.append(h.copy())
        padded[off[k]:off[k + 1], o:o + w, o:o + w] = h
    flat = np.concatenate([p.reshape(-1) for p in parts]) if parts else np.zeros(0, dtype=sp.H.dtype)
    return parts, flat, padded
