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

Parity unpinned (project readings with no paper value to check against):
  * the detector-side factor f_y f_x at f > 1 (absolute map scale only);
  * the hull-boundary rule of the weights (see geometry.py).
"""
import math
import numpy as np

from . import physics as ph
from .geometry import Geometry


class Problem:
    """Inputs of one map evaluation, prepared in FP64."""

    def __init__(self, cfg, atoms, nch, V, H, scans, geometry=None):
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
        off = np.concatenate([[0], np.cumsum(self.nch)])
        self.H = [H[off[k]:off[k + 1]] for k in range(len(self.ion))]
        self.scans = np.asarray(scans, dtype=np.float64)

    # ---- transmission of slice j
    def T(self, j):
        return ph.transmission(self.V[j], self.sigma)

    # ---- window geometry of ionized site k
    def window_index(self, k):
        w = self.cfg.win
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
    fyfx = cfg.fy * cfg.fx
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


def bip_cube(prob: Problem, scans=None, mode=None):
    """Algorithm 5 with the detector sum left open: the 4D cube [P, n_det]
    (detector beams in geometry order), sites added in order in FP64."""
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
        out += site_cube(M, C, crop_mask(prob, k, scans), cfg.fy * cfg.fx)
    return out


def qeels(prob: Problem, cube, axis):
    """Momentum-resolved output (qEELS): the cube summed over the detector
    beams that share their component along `axis` (0: h_y, 1: h_x) -- one
    resolved axis q_par, the perpendicular one summed.  Returns the bin
    values h_par (ascending) and [P, n_bins] (Sec. 2.2.6 outputs)."""
    h = np.asarray(prob.geo.h_det)[:, axis]
    bins = np.unique(h)
    out = np.zeros((cube.shape[0], len(bins)), dtype=np.float64)
    for i, q in enumerate(bins):
        out[:, i] = cube[:, h == q].sum(axis=1)
    return bins, out


def exact_cube(prob: Problem, scans=None):
    """Algorithm 4 with the detector sum left open, [P, n_det]."""
    cfg, geo = prob.cfg, prob.geo
    scans = prob.scans if scans is None else np.asarray(scans, dtype=np.float64)
    W1 = s1_windows(prob, geo.h_beam, detilt=False)
    W2 = s2_windows(prob, geo.h_det, detilt=False)
    C = illumination(prob, geo.h_beam, geo.psi_beam, scans)
    out = np.zeros((len(scans), geo.n_det), dtype=np.float64)
    for k in range(len(prob.ion)):
        M = coupling(W2[k], prob.H[k], W1[k])
        out += site_cube(M, C, crop_mask(prob, k, scans), cfg.fy * cfg.fx)
    return out


def exact_map(prob: Problem, scans=None, keep_stages=False):
    """Algorithm 4: exact dual-matrix map (every retained beam and detector
    beam propagated; no weights, no de-tilt)."""
    cfg, geo = prob.cfg, prob.geo
    scans = prob.scans if scans is None else np.asarray(scans, dtype=np.float64)
    W1 = s1_windows(prob, geo.h_beam, detilt=False)
    W2 = s2_windows(prob, geo.h_det, detilt=False)
    C = illumination(prob, geo.h_beam, geo.psi_beam, scans)
    fyfx = cfg.fy * cfg.fx
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
    detector beams det_h (default: the geometry's detector beams, in order)
    summed over sites and channels."""
    cfg, geo = prob.cfg, prob.geo
    scans = prob.scans if scans is None else np.asarray(scans, dtype=np.float64)
    det_h = geo.h_det if det_h is None else det_h
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


def elastic_probe_at(prob: Problem, rho, plane):
    """Exact elastic probe arriving at slice `plane` (Algorithm 1 inner loop)."""
    psi = exact_probe(prob, rho)
    for j in range(plane):
        psi = ph.step(psi, prob.T(j), prob.P)
    return psi


def make_problem(spec, geometry=None, **cfg_overrides):
    cfg = spec.cfg.replace(**cfg_overrides) if cfg_overrides else spec.cfg
    return Problem(cfg, spec.atoms, spec.nch, spec.V, spec.H, spec.scans, geometry)
