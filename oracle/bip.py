"""BiP-PRISM core-loss elemental map, FP64, step by step (Algorithm 5), with
the exact dual-matrix map (Algorithm 4) and conventional multislice
(Algorithm 1) it is checked against.

Passages followed, in the order the method takes them:
  * S1 build: unit plane waves of the parent beams advanced by
    transmit-then-propagate to each ionization plane (Eq. smatrix-advance,
    Algorithm 2 "AdvanceTo", Algorithm 5 first step);
  * S2 build: conjugate detector plane waves back-propagated from the exit
    surface by the transposed multislice (Eq. s2).  Reading of the garbled
    wording: S2^d = M_{i->exit}^T (G^{-1/2} e^{-2 pi i h_d.r/N}), applied as
    P, T_{N-1}, P, T_{N-2}, ..., P, T_i (P is even, T symmetric), so that
    sum_r S2^d(r) w(r) = [F_u M_{i->exit} w]_{h_d} with the unitary DFT F_u.
    It is built directly at every plane by one backward sweep (no peeling);
  * window crop: a win x win pixel block starting at floor(tau/dx + 1/2) -
    win/2 on each axis, wrapped periodically (Sec. 2.3.1; size and centring
    are a reading);
  * de-tilt (Eq. part-basis): S1 parents are multiplied by e^{-2 pi i h_p.r/N};
    S2 parents carry the conjugate carrier e^{-2 pi i h_p.r/N} and are
    de-tilted by e^{+2 pi i h_p.r/N} (reading: de-tilting removes the
    carrier, Sec. 2.2.3), then re-tilted by the opposite factor;
  * reconstruction on the window (Eq. window-recon) with the magnitude-
    preserving form (Eq. magpreserve) or the plain complex average; where
    the complex sum is exactly zero its phase is taken as 1 (reading);
  * coupling M^{(n)}_{d,b} = sum_{r in window} S2^d H_n S1^b (Eq. coupling);
  * illumination c_b(rho) = f_y f_x Psi(h_b) / sqrt(G sum_all |Psi|^2)
    e^{-2 pi i h_b.rho/N} (Eq. probe, Sec. 2.2.2 rescale; the unit-norm
    probe normalisation is a reading);
  * a_d(rho) = sum_b M_{d,b} c_b(rho); I(rho) = f_y f_x sum_tau sum_n sum_d
    |a_d|^2 (Eq. map-sum) over the scans inside the site's 1/f crop window
    (Sec. 2.2.4); crop reading: the minimum-image offset rho - tau (pixels)
    lies in [-N/(2f), N/(2f)) on both axes.  Sum over sites in FP64 with
    exactly rounded summation (math.fsum).

Output modes (Sec. 2.2.6):
  * 4D cube: S1 partitioned, the exit exact on the complete output basis --
    every beam inside the detector disc, unsubsampled -- through the
    unpartitioned S2 columns (the reciprocity form of Algorithm 3's exit
    multislice); no detector-side factor.  Algorithm 3 itself is here too,
    by brute force (alg3_cube), with the full-grid partitioned probe;
  * qEELS: the map's per-beam terms binned along one axis, with S2
    partitioned on detector beams sampled at f = 1 along the resolved axis
    (dfy or dfx = 1); the factor is the perpendicular subsampling.

Parity unpinned (project readings with no paper value to check against):
  * the detector-side factor (dfy dfx, by default f_y f_x) at f > 1
    (absolute map scale only);
  * the hull-boundary rule of the weights (see geometry.py).
"""
import math
import numpy as np

from . import physics as ph
from .geometry import Geometry


class Problem:
    """Inputs of one map evaluation, prepared in FP64."""

    def __init__(self, cfg, atoms, nch, V, H, scans, geometry=None, site_win=None):
        """site_win: the window of each ionized site (default: cfg.win for
        all); H: [sum nch, win, win] when every site has cfg.win, else a list
        with one [nch_k, w_k, w_k] array per ionized site."""
        self.cfg = cfg
        self.lam = ph.wavelength(cfg.e0)
        self.sigma = ph.interaction_constant(cfg.e0)
        self.geo = geometry if geometry is not None else Geometry(cfg, self.lam)
        self.P = ph.propagator(cfg.ny, cfg.nx, cfg.ly, cfg.lx, self.lam, cfg.dz)
        self.V = V
        self.ion = np.nonzero(np.asarray(nch) > 0)[0]
        dy, dx = cfg.ly / cfg.ny, cfg.lx / cfg.nx
        self.tau_px = np.stack([atoms[self.ion, 0] / dy, atoms[self.ion, 1] / dx], axis=1)
        self.plane = atoms[self.ion, 2].astype(np.int64)
        self.nch = np.asarray(nch)[self.ion].astype(np.int64)
        n = len(self.ion)
        self.win = (np.full(n, cfg.win, dtype=np.int64) if site_win is None
                    else np.asarray(site_win, dtype=np.int64).reshape(n))
        if isinstance(H, (list, tuple)):
            self.H = [np.asarray(h) for h in H]
        else:
            off = np.concatenate([[0], np.cumsum(self.nch)])
            self.H = [H[off[k]:off[k + 1]] for k in range(n)]
        for k in range(n):
            w = int(self.win[k])
            if self.H[k].shape != (self.nch[k], w, w):
                raise ValueError(f"site {k}: H has shape {self.H[k].shape}, want {(int(self.nch[k]), w, w)}")
        self.scans = np.asarray(scans, dtype=np.float64)

    # ---- transmission of slice j
    def T(self, j):
        return ph.transmission(self.V[j], self.sigma)

    # ---- window geometry of ionized site k: w_k x w_k pixels from
    # floor(tau/dx + 1/2) - w_k/2 on each axis, wrapped
    def window_index(self, k):
        w = int(self.win[k])
        oy = int(math.floor(self.tau_px[k, 0] + 0.5)) - w // 2
        ox = int(math.floor(self.tau_px[k, 1] + 0.5)) - w // 2
        iy = np.mod(oy + np.arange(w), self.cfg.ny)
        ix = np.mod(ox + np.arange(w), self.cfg.nx)
        return iy, ix


def window_phase(h, iy, ix, ny, nx, sign):
    """exp(sign 2 pi i h.r/N) on the window pixels r = (iy, ix) for each beam
    h; returns [n_beams, w, w].  h.r is reduced modulo N in integers."""
    h = np.asarray(h, dtype=np.int64)
    py = np.mod(h[:, 0:1] * iy[None, :], ny) / ny            # [nb, w]
    px = np.mod(h[:, 1:2] * ix[None, :], nx) / nx            # [nb, w]
    return np.exp(sign * 2j * np.pi * (py[:, :, None] + px[:, None, :]))


# --------------------------------------------------------------------------
# scattering-matrix builds (window stashes at every ionization plane)

def s1_windows(prob: Problem, h_cols, detilt=True):
    """Windows of S1 columns at each site's plane: unit plane waves
    e^{2 pi i h.r/N} advanced by psi -> P(T_j psi) for j < i.  With detilt,
    multiplied by e^{-2 pi i h.r/N} on the window (Eq. part-basis)."""
    cfg = prob.cfg
    h_cols = np.asarray(h_cols, dtype=np.int64)
    psi = np.stack([ph.plane_wave(h, cfg.ny, cfg.nx, +1) for h in h_cols])
    out = [None] * len(prob.ion)
    cur = 0
    for i in sorted(set(prob.plane.tolist())):
        while cur < i:
            psi = ph.step(psi, prob.T(cur), prob.P)
            cur += 1
        for k in np.nonzero(prob.plane == i)[0]:
            iy, ix = prob.window_index(k)
            win = psi[:, iy[:, None], ix[None, :]]
            if detilt:
                win = win * window_phase(h_cols, iy, ix, cfg.ny, cfg.nx, -1)
            out[k] = win
    return out


def s2_windows(prob: Problem, h_cols, detilt=True):
    """Windows of S2 columns at each site's plane: G^{-1/2} e^{-2 pi i h.r/N}
    taken through x -> T_j (P x) for j = N_Z-1 down to i (Eq. s2, reading
    above).  With detilt, multiplied by e^{+2 pi i h.r/N} on the window."""
    cfg = prob.cfg
    g = cfg.ny * cfg.nx
    h_cols = np.asarray(h_cols, dtype=np.int64)
    x = np.stack([ph.plane_wave(h, cfg.ny, cfg.nx, -1) for h in h_cols]) / math.sqrt(g)
    out = [None] * len(prob.ion)
    planes = set(prob.plane.tolist())
    if not planes:
        return out
    for j in range(cfg.nz - 1, min(planes) - 1, -1):
        x = prob.T(j) * ph.propagate(x, prob.P)
        if j in planes:
            for k in np.nonzero(prob.plane == j)[0]:
                iy, ix = prob.window_index(k)
                win = x[:, iy[:, None], ix[None, :]]
                if detilt:
                    win = win * window_phase(h_cols, iy, ix, cfg.ny, cfg.nx, +1)
                out[k] = win
    return out


def s2_full(prob: Problem, h_cols, plane):
    """S2 columns on the full grid at one plane (used by the reciprocity check)."""
    cfg = prob.cfg
    g = cfg.ny * cfg.nx
    x = np.stack([ph.plane_wave(h, cfg.ny, cfg.nx, -1) for h in np.asarray(h_cols)]) / math.sqrt(g)
    for j in range(cfg.nz - 1, plane - 1, -1):
        x = prob.T(j) * ph.propagate(x, prob.P)
    return x


def exit_operator(prob: Problem, w, plane):
    """M_{i->exit} w: transmit-and-propagate through slices i..N_Z-1."""
    for j in range(plane, prob.cfg.nz):
        w = ph.step(w, prob.T(j), prob.P)
    return w


# --------------------------------------------------------------------------
# reconstruction, coupling, map

def reconstruct(dt, W, h_targets, iy, ix, ny, nx, sign, mode="magnitude"):
    """Eq. window-recon with Eq. magpreserve: U_b = sum_p w_{b,p} dt_p;
    magnitude mode S_b = (sum_p w_{b,p} |dt_p|) U_b / |U_b|; then re-tilt by
    exp(sign 2 pi i h_b.r/N).  dt: [Bp, w, w]; W: [n_targets, Bp]."""
    U = np.tensordot(W, dt, axes=(1, 0))
    if mode == "magnitude":
        A = np.tensordot(W, np.abs(dt), axes=(1, 0))
        mag = np.abs(U)
        safe = np.where(mag > 0.0, mag, 1.0)
        S = np.where(mag > 0.0, A * (U / safe), A)
    elif mode == "complex":
        S = U
    else:
        raise ValueError(mode)
    return S * window_phase(h_targets, iy, ix, ny, nx, sign)


def coupling(S2w, Hk, S1w):
    """M^{(n)}_{d,b} = sum_r S2^d(r) H_n(r) S1^b(r) over the window
    (Eq. coupling).  S2w [n_det,w,w], Hk [nch,w,w], S1w [B,w,w] ->
    [nch, n_det, B]."""
    nd, B = S2w.shape[0], S1w.shape[0]
    A = S2w.reshape(nd, -1)
    Bm = S1w.reshape(B, -1).T
    return np.stack([A @ (h.reshape(-1, 1) * Bm) for h in Hk])


def detector_factor(prob: Problem):
    """The detector-side factor of the map: (dfy dfx), the subsampling of
    the detector beams (reading: a coarse detector sum is 1/(dfy dfx) of the
    full one for an exit wave confined to the alias-free window, Poisson
    summation mirroring the probe-side PRISM rescale, Sec. 2.2.2)."""
    return prob.geo.dfy * prob.geo.dfx


def illumination(prob: Problem, h_beam, psi_beam, scans):
    """c_b(rho) [B, P] (Eq. probe with the PRISM f_y f_x rescale)."""
    cfg = prob.cfg
    g = cfg.ny * cfg.nx
    norm = math.sqrt(g * float(np.sum(np.abs(prob.geo.psi_full) ** 2)))
    fyfx = cfg.fy * cfg.fx
    phase = (np.outer(h_beam[:, 0], scans[:, 0]) / cfg.ny
             + np.outer(h_beam[:, 1], scans[:, 1]) / cfg.nx)
    return (fyfx * psi_beam / norm)[:, None] * np.exp(-2j * np.pi * phase)


def crop_mask(prob: Problem, k, scans):
    """Scans inside site k's 1/f window (Sec. 2.2.4 crop mask; reading:
    minimum-image offset in [-N/(2f), N/(2f)) on both axes)."""
    cfg = prob.cfg
    ok = np.ones(len(scans), dtype=bool)
    for ax, (n, f) in enumerate(((cfg.ny, cfg.fy), (cfg.nx, cfg.fx))):
        d = scans[:, ax] - prob.tau_px[k, ax]
        d = d - n * np.floor((d + 0.5 * n) / n)
        half = 0.5 * n / f
        ok &= (d >= -half) & (d < half)
    return ok


def site_map(M, C, mask, fyfx):
    """I_tau(rho) = f_y f_x sum_n sum_d |sum_b M_{d,b} c_b(rho)|^2 on the
    masked scans, zero elsewhere (Algorithm 4 last two steps, Eq. map-sum)."""
    out = np.zeros(C.shape[1], dtype=np.float64)
    if not np.any(mask):
        return out
    Cm = C[:, mask]
    acc = np.zeros(Cm.shape[1], dtype=np.float64)
    for Mn in M:
        a = Mn @ Cm
        acc += np.sum(a.real ** 2 + a.imag ** 2, axis=0)
    out[mask] = fyfx * acc
    return out


def site_cube(M, C, mask, fyfx):
    """Momentum-resolved contribution of one site, [P, n_det]: per detector
    beam d, f_y f_x sum_n |sum_b M_{d,b} c_b(rho)|^2 on the masked scans,
    zero elsewhere -- the terms of Eq. map-sum before the detector sum (the
    energy-filtered 4D cube of Sec. 2.2.6)."""
    out = np.zeros((C.shape[1], M[0].shape[0]), dtype=np.float64)
    if not np.any(mask):
        return out
    Cm = C[:, mask]
    acc = np.zeros((M[0].shape[0], Cm.shape[1]), dtype=np.float64)
    for Mn in M:
        a = Mn @ Cm
        acc += a.real ** 2 + a.imag ** 2
    out[mask] = fyfx * acc.T
    return out


def sum_sites(partials):
    """Exactly rounded FP64 sum over sites for every scan."""
    partials = np.asarray(partials, dtype=np.float64)
    if partials.ndim == 1 or partials.shape[0] == 0:
        return np.zeros(partials.shape[-1]) if partials.shape[0] == 0 else partials
    return np.array([math.fsum(partials[:, p]) for p in range(partials.shape[1])])


class MapResult:
    def __init__(self, total, partials, stages=None):
        self.map = total
        self.partials = partials
        self.stages = stages or {}


def bip_map(prob: Problem, scans=None, mode=None, keep_stages=False, sites=None):
    """Algorithm 5: BiP-PRISM map with both matrices partitioned."""
    cfg, geo = prob.cfg, prob.geo
    mode = mode or cfg.recon
    scans = prob.scans if scans is None else np.asarray(scans, dtype=np.float64)
    W1 = s1_windows(prob, geo.h_p1, detilt=True)
    W2 = s2_windows(prob, geo.h_p2, detilt=True)
    C = illumination(prob, geo.h_beam, geo.psi_beam, scans)
    fyfx = detector_factor(prob)
    sites = range(len(prob.ion)) if sites is None else sites
    partials, stages = [], {}
    for k in sites:
        iy, ix = prob.window_index(k)
        S1w = reconstruct(W1[k], geo.w1, geo.h_beam, iy, ix, cfg.ny, cfg.nx, +1, mode)
        S2w = reconstruct(W2[k], geo.w2, geo.h_det, iy, ix, cfg.ny, cfg.nx, -1, mode)
        M = coupling(S2w, prob.H[k], S1w)
        part = site_map(M, C, crop_mask(prob, k, scans), fyfx)
        partials.append(part)
        if keep_stages:
            stages[k] = dict(stash1=W1[k], stash2=W2[k], S1w=S1w, S2w=S2w, M=M)
    partials = np.array(partials).reshape(len(partials), len(scans))
    return MapResult(sum_sites(partials), partials, stages)


def per_beam(prob: Problem, scans=None, mode=None):
    """Algorithm 5's terms with the detector sum left open, on the context's
    (partitioned, subsampled) detector beams: [P, n_det] with entries
    (dfy dfx) sum_tau sum_n |a_d|^2 -- the momentum-resolved intensities
    qEELS bins (Sec. 2.2.6).  Summed over d this is the map."""
    cfg, geo = prob.cfg, prob.geo
    mode = mode or cfg.recon
    scans = prob.scans if scans is None else np.asarray(scans, dtype=np.float64)
    W1 = s1_windows(prob, geo.h_p1, detilt=True)
    W2 = s2_windows(prob, geo.h_p2, detilt=True)
    C = illumination(prob, geo.h_beam, geo.psi_beam, scans)
    out = np.zeros((len(scans), geo.n_det), dtype=np.float64)
    for k in range(len(prob.ion)):
        iy, ix = prob.window_index(k)
        S1w = reconstruct(W1[k], geo.w1, geo.h_beam, iy, ix, cfg.ny, cfg.nx, +1, mode)
        S2w = reconstruct(W2[k], geo.w2, geo.h_det, iy, ix, cfg.ny, cfg.nx, -1, mode)
        M = coupling(S2w, prob.H[k], S1w)
        out += site_cube(M, C, crop_mask(prob, k, scans), detector_factor(prob))
    return out


def qeels_bins(prob: Problem, axis):
    """Bin values h_par (ascending) of the resolved axis and each detector
    beam's bin, for axis 0 (q_y resolved) or 1 (q_x resolved)."""
    h = np.asarray(prob.geo.h_det)[:, axis]
    bins = np.unique(h)
    return bins, np.searchsorted(bins, h)


def bip_qeels(prob: Problem, axis, scans=None, mode=None):
    """Momentum-resolved qEELS (Sec. 2.2.6): one diffraction axis resolved,
    the perpendicular one summed, I(q_par, rho) = (df_perp) sum over the
    detector beams with that h_par of sum_tau sum_n |a_d|^2.  S2 stays
    partitioned (its detector basis is rebuilt from parents whatever the
    binning), which the paper allows only with the resolved axis sampled at
    f = 1: a geometry whose detector beams are subsampled along `axis` is
    refused.  Returns (bins, [P, n_bins])."""
    d_axis = prob.geo.dfy if axis == 0 else prob.geo.dfx
    if axis not in (0, 1):
        raise ValueError("axis must be 0 (q_y) or 1 (q_x)")
    if d_axis != 1:
        raise ValueError("qEELS needs the resolved axis sampled at f = 1 (dfy or dfx = 1)")
    cube = per_beam(prob, scans, mode)
    bins, bin_of = qeels_bins(prob, axis)
    out = np.zeros((cube.shape[0], len(bins)), dtype=np.float64)
    for i in range(len(bins)):
        out[:, i] = cube[:, bin_of == i].sum(axis=1)
    return bins, out


def bip_cube(prob: Problem, scans=None, mode=None):
    """Energy-filtered 4D cube (Sec. 2.2.6, Algorithm 3): S1 partitioned and
    rebuilt on each window (Eq. window-recon, magpreserve), the exit side
    exact on the complete output basis -- every beam inside the detector disc
    at the grid's own sampling (geo.h_cube), S2 neither partitioned nor
    subsampled, since the cube keeps every output beam.  The exit amplitude
    of each beam is taken through the unpartitioned S2 column (Eq. s2, the
    reciprocity form of Algorithm 3's exit multislice):
      cube[rho][q] = sum_tau sum_n |sum_b M_{q,b} c_b(rho)|^2,
      M_{q,b} = sum_{r in window} S2^q(r) H_n(r) S~1^b(r),
    over the sites whose crop mask holds rho; no detector-side factor (the
    basis is not subsampled).  Returns [P, n_cube], beams in geo.h_cube
    order."""
    cfg, geo = prob.cfg, prob.geo
    mode = mode or cfg.recon
    scans = prob.scans if scans is None else np.asarray(scans, dtype=np.float64)
    W1 = s1_windows(prob, geo.h_p1, detilt=True)
    W2 = s2_windows(prob, geo.h_cube, detilt=False)
    C = illumination(prob, geo.h_beam, geo.psi_beam, scans)
    out = np.zeros((len(scans), len(geo.h_cube)), dtype=np.float64)
    for k in range(len(prob.ion)):
        iy, ix = prob.window_index(k)
        S1w = reconstruct(W1[k], geo.w1, geo.h_beam, iy, ix, cfg.ny, cfg.nx, +1, mode)
        M = coupling(W2[k], prob.H[k], S1w)
        out += site_cube(M, C, crop_mask(prob, k, scans), 1)
    return out


def exact_cube(prob: Problem, scans=None, det_h=None):
    """The cube's exact reference (Algorithm 2 with the exit exact): every
    retained aperture beam propagated (no parents, no weights), S2 exact at
    the beams det_h (default: the complete output basis geo.h_cube), the
    crop mask as in the map, no detector-side factor; [P, len(det_h)]."""
    cfg, geo = prob.cfg, prob.geo
    scans = prob.scans if scans is None else np.asarray(scans, dtype=np.float64)
    det_h = geo.h_cube if det_h is None else np.asarray(det_h)
    W1 = s1_windows(prob, geo.h_beam, detilt=False)
    W2 = s2_windows(prob, det_h, detilt=False)
    C = illumination(prob, geo.h_beam, geo.psi_beam, scans)
    out = np.zeros((len(scans), len(det_h)), dtype=np.float64)
    for k in range(len(prob.ion)):
        M = coupling(W2[k], prob.H[k], W1[k])
        out += site_cube(M, C, crop_mask(prob, k, scans), 1)
    return out


def exact_map(prob: Problem, scans=None, keep_stages=False):
    """Algorithm 4: exact dual-matrix map (every retained beam and detector
    beam propagated; no weights, no de-tilt)."""
    cfg, geo = prob.cfg, prob.geo
    scans = prob.scans if scans is None else np.asarray(scans, dtype=np.float64)
    W1 = s1_windows(prob, geo.h_beam, detilt=False)
    W2 = s2_windows(prob, geo.h_det, detilt=False)
    C = illumination(prob, geo.h_beam, geo.psi_beam, scans)
    fyfx = detector_factor(prob)
    partials, stages = [], {}
    for k in range(len(prob.ion)):
        M = coupling(W2[k], prob.H[k], W1[k])
        partials.append(site_map(M, C, crop_mask(prob, k, scans), fyfx))
        if keep_stages:
            stages[k] = dict(S1w=W1[k], S2w=W2[k], M=M)
    partials = np.array(partials).reshape(len(partials), len(scans))
    return MapResult(sum_sites(partials), partials, stages)


# --------------------------------------------------------------------------
# Algorithm 1: conventional transition-potential multislice (ground truth)

def full_grid_H(prob: Problem, k):
    """Site k's transition potentials placed on the full grid at its window."""
    cfg = prob.cfg
    iy, ix = prob.window_index(k)
    out = np.zeros((prob.nch[k], cfg.ny, cfg.nx), dtype=np.complex128)
    out[:, iy[:, None], ix[None, :]] = prob.H[k]
    return out


def exact_probe(prob: Problem, rho):
    """psi_0(r, rho) = sum_b c_b e^{-2 pi i h_b.rho/N} e^{2 pi i h_b.r/N} over
    the full aperture (Eq. probe), unit norm."""
    cfg, geo = prob.cfg, prob.geo
    g = cfg.ny * cfg.nx
    norm = math.sqrt(g * float(np.sum(np.abs(geo.psi_full) ** 2)))
    spec = np.zeros((cfg.ny, cfg.nx), dtype=np.complex128)
    ph_rho = np.exp(-2j * np.pi * (geo.h_full[:, 0] * rho[0] / cfg.ny
                                   + geo.h_full[:, 1] * rho[1] / cfg.nx))
    spec[geo.h_full[:, 0] % cfg.ny, geo.h_full[:, 1] % cfg.nx] = geo.psi_full / norm * ph_rho
    return np.fft.ifft2(spec) * g


def conventional_map(prob: Problem, scans=None, det_h=None):
    """Algorithm 1: per scan, multislice the probe; at each slice with sites
    spawn H_n psi, take it to the exit, add |F_u .|^2 over the detector
    beams (all beams with |q| <= theta/lambda unless det_h is given)."""
    cfg, geo = prob.cfg, prob.geo
    scans = prob.scans if scans is None else np.asarray(scans, dtype=np.float64)
    if det_h is None:
        from .geometry import disc_beams
        det_h = disc_beams(cfg.ny, cfg.nx, cfg.ly, cfg.lx, prob.lam, cfg.theta_det)
    dsel = (det_h[:, 0] % cfg.ny, det_h[:, 1] % cfg.nx)
    Hfull = {k: full_grid_H(prob, k) for k in range(len(prob.ion))}
    out = np.zeros(len(scans))
    for p, rho in enumerate(scans):
        psi = exact_probe(prob, rho)
        acc = []
        for i in range(cfg.nz):
            for k in np.nonzero(prob.plane == i)[0]:
                for Hn in Hfull[k]:
                    e = exit_operator(prob, Hn * psi, i)
                    a = ph.unitary_dft(e)[dsel]
                    acc.append(float(np.sum(np.abs(a) ** 2)))
            psi = ph.step(psi, prob.T(i), prob.P)
        out[p] = math.fsum(acc)
    return out


def conventional_cube(prob: Problem, scans=None, det_h=None):
    """Algorithm 1 per detector beam: [P, n_det] intensities |F_u .|^2 at the
    detector beams det_h (default: the cube's complete output basis, in
    order) summed over sites and channels."""
    cfg, geo = prob.cfg, prob.geo
    scans = prob.scans if scans is None else np.asarray(scans, dtype=np.float64)
    det_h = geo.h_cube if det_h is None else det_h
    dsel = (det_h[:, 0] % cfg.ny, det_h[:, 1] % cfg.nx)
    Hfull = {k: full_grid_H(prob, k) for k in range(len(prob.ion))}
    out = np.zeros((len(scans), len(det_h)))
    for p, rho in enumerate(scans):
        psi = exact_probe(prob, rho)
        for i in range(cfg.nz):
            for k in np.nonzero(prob.plane == i)[0]:
                for Hn in Hfull[k]:
                    e = exit_operator(prob, Hn * psi, i)
                    a = ph.unitary_dft(e)[dsel]
                    out[p] += np.abs(a) ** 2
            psi = ph.step(psi, prob.T(i), prob.P)
    return out


# --------------------------------------------------------------------------
# Algorithm 3 (partitioned S1, exit by multislice) and its probes, on the
# full grid: the brute-force form the cube and the locality result are
# checked with

def s1_columns(prob: Problem, h_cols, plane):
    """S1 columns on the full grid at `plane`: unit plane waves
    e^{2 pi i h.r/N} advanced by psi -> P(T_j psi) for j < plane
    (Eq. smatrix-advance), [n_cols, ny, nx]."""
    cfg = prob.cfg
    psi = np.stack([ph.plane_wave(h, cfg.ny, cfg.nx, +1) for h in np.asarray(h_cols, dtype=np.int64)])
    for j in range(plane):
        psi = ph.step(psi, prob.T(j), prob.P)
    return psi


def prism_probe(prob: Problem, scans, plane):
    """Eq. prism-probe: psi(r, rho) = sum_b c_b(rho) S_b(r) with every
    retained aperture beam propagated (Algorithm 2), [P, ny, nx]."""
    geo = prob.geo
    cols = s1_columns(prob, geo.h_beam, plane)
    C = illumination(prob, geo.h_beam, geo.psi_beam, np.asarray(scans, dtype=np.float64))
    return np.tensordot(C.T, cols, axes=(1, 0))


def partitioned_probe(prob: Problem, scans, plane, mode=None):
    """Algorithm 3's probe at `plane`, [P, ny, nx]: the parent columns
    advanced and de-tilted (Eq. part-basis), every aperture beam's column
    rebuilt from them by Eq. window-recon -- with Eq. magpreserve in the
    magnitude mode -- taken over the whole grid instead of a window, then
    psi(r, rho) = sum_b c_b(rho) S~_b(r) (Eq. prism-probe)."""
    cfg, geo = prob.cfg, prob.geo
    mode = mode or cfg.recon
    iy, ix = np.arange(cfg.ny), np.arange(cfg.nx)
    dt = s1_columns(prob, geo.h_p1, plane) * window_phase(geo.h_p1, iy, ix, cfg.ny, cfg.nx, -1)
    S1 = reconstruct(dt, geo.w1, geo.h_beam, iy, ix, cfg.ny, cfg.nx, +1, mode)
    C = illumination(prob, geo.h_beam, geo.psi_beam, np.asarray(scans, dtype=np.float64))
    return np.tensordot(C.T, S1, axes=(1, 0))


def alg3_cube(prob: Problem, scans=None, det_h=None, probe=None, h_full=None):
    """Algorithm 3 by brute force, [P, len(det_h)]: at each site's plane the
    probe of every scan (partitioned_probe unless `probe(scans, plane)` is
    given), each channel's inelastic wave H_n psi taken to the exit by
    multislice (M_{i->exit}) and |F_u .|^2 read at the beams det_h (default:
    the complete output basis geo.h_cube), summed over channels and over the
    sites whose crop mask holds the scan.  `h_full(k)` gives site k's
    channels on the whole grid (default: the window samples, zero
    elsewhere)."""
    cfg, geo = prob.cfg, prob.geo
    scans = prob.scans if scans is None else np.asarray(scans, dtype=np.float64)
    det_h = geo.h_cube if det_h is None else np.asarray(det_h)
    dsel = (det_h[:, 0] % cfg.ny, det_h[:, 1] % cfg.nx)
    if probe is None:
        probe = lambda sc, plane: partitioned_probe(prob, sc, plane)
    if h_full is None:
        h_full = lambda k: full_grid_H(prob, k)
    out = np.zeros((len(scans), len(det_h)), dtype=np.float64)
    for plane in sorted(set(prob.plane.tolist())):
        psi = probe(scans, plane)
        for k in np.nonzero(prob.plane == plane)[0]:
            sel = np.nonzero(crop_mask(prob, k, scans))[0]
            if len(sel) == 0:
                continue
            for Hn in h_full(k):
                e = exit_operator(prob, Hn[None] * psi[sel], plane)
                out[sel] += np.abs(ph.unitary_dft(e)[:, dsel[0], dsel[1]]) ** 2
    return out


def on_atom_error(prob: Problem, k, scans, mode=None):
    """Eq. onatom for site k at every scan: ||psi_p - psi||_Omega /
    ||psi||_Omega on the site's window, psi_p the partitioned probe
    (Algorithm 3) and psi the exact PRISM probe (Eq. prism-probe) at the
    site's plane."""
    plane = int(prob.plane[k])
    iy, ix = prob.window_index(k)
    pp = partitioned_probe(prob, scans, plane, mode)[:, iy[:, None], ix[None, :]]
    pe = prism_probe(prob, scans, plane)[:, iy[:, None], ix[None, :]]
    num = np.sqrt(np.sum(np.abs(pp - pe) ** 2, axis=(1, 2)))
    return num / np.sqrt(np.sum(np.abs(pe) ** 2, axis=(1, 2)))


def elastic_probe_at(prob: Problem, rho, plane):
    """Exact elastic probe arriving at slice `plane` (Algorithm 1 inner loop)."""
    psi = exact_probe(prob, rho)
    for j in range(plane):
        psi = ph.step(psi, prob.T(j), prob.P)
    return psi


def make_problem(spec, geometry=None, site_win=None, H=None, **cfg_overrides):
    """Problem of a synthetic specimen; site_win and H (per-site arrays)
    replace the uniform windows and the specimen's H when given."""
    cfg = spec.cfg.replace(**cfg_overrides) if cfg_overrides else spec.cfg
    return Problem(cfg, spec.atoms, spec.nch, spec.V, spec.H if H is None else H, spec.scans, geometry, site_win)
