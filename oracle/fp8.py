"""FP8 (E4M3) form of the coupling contraction, FP64 model.

TEST INFRASTRUCTURE ONLY (see the package header).

The precision study of the contraction runs its operands in 8-bit floating
point with one scale per operand tile and FP32 accumulation.  Here the
operand tiles are the 64 x 64 reconstructed windows themselves: one row of
the coupling operands is one beam's (and, on the S1 side, one channel's)
window, K = the window pixels (Eq. coupling), so a per-window scale is
constant along the contracted index and comes out of the sum.

Scale rule (a reading; the paper fixes no FP8 scheme).  The scale of a row
must be known before the row is written, so it is an a-priori bound of the
row's largest element rather than its measured maximum:
  * a reconstructed window is a convex combination of its parents, with
    non-negative weights summing to one (Eq. nnw), in both forms of Eq.
    window-recon / Eq. magpreserve, so |S^t(r)| <= sum_p w_tp m_p with
    m_p = max_r |dt_p(r)| over the site's window;
  * on the S1 side the row is H_n S1^b, bounded by max_r |H_n| times that;
  * bound = kappa * (that sum), kappa = 1 + 2^-6 (headroom for the rounding
    of the weights and magnitudes on the way), and the row is stored as
    q = e4m3(Re v * 448 / bound) + i e4m3(Im v * 448 / bound), 448 being the
    largest finite E4M3 value.

e4m3_round is the OCP 8-bit E4M3 format (1 sign, 4 exponent bits with bias
7, 3 mantissa bits; subnormals; no infinities; 448 the largest finite
value): nearest value, ties to even mantissa, saturating at +-448.
"""
import numpy as np

from . import bip

E4M3_MAX = 448.0
KAPPA = 1.0 + 2.0 ** -6


def e4m3_round(x):
    """Nearest E4M3 value of each element of the real array x (ties to the
    even mantissa), saturated to [-448, 448]."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    _, e = np.frexp(np.where(a > 0.0, a, 1.0))     # a = m 2^e, m in [0.5, 1)
    # binade exponent floor(log2 a), clamped at the smallest normal 2^-6 so
    # that subnormals share its spacing 2^-9
    eb = np.maximum(e - 1, -6)
    spacing = np.ldexp(1.0, eb - 3)
    q = np.round(a / spacing) * spacing              # np.round: ties to even
    q = np.minimum(q, E4M3_MAX)
    return np.where(a > 0.0, np.copysign(q, x), 0.0 * x)


def quantize_rows(V, bound):
    """Rows of V [rows, ...] complex, each stored as E4M3 with the scale
    bound/448 of its row; returns the values the contraction sees."""
    V = np.asarray(V, dtype=np.complex128)
    bound = np.asarray(bound, dtype=np.float64)
    shape = (-1,) + (1,) * (V.ndim - 1)
    inv = np.where(bound > 0.0, E4M3_MAX / np.where(bound > 0.0, bound, 1.0), 0.0).reshape(shape)
    s = (bound / E4M3_MAX).reshape(shape)
    return s * (e4m3_round(V.real * inv) + 1j * e4m3_round(V.imag * inv))


def row_bounds(W, dt):
    """kappa sum_p w_tp max_r |dt_p(r)| for every target t (W [n_t, Bp],
    dt [Bp, w, w] the site's de-tilted parent windows)."""
    m = np.abs(dt).reshape(dt.shape[0], -1).max(axis=1)
    return KAPPA * (np.asarray(W, dtype=np.float64) @ m)


def site_coupling_fp8(S2w, Hk, S1w, W2, dt2, W1, dt1):
    """M^{(n)} of Eq. coupling with both operands stored as scaled E4M3
    (rows: S2^d, and H_n S1^b per channel); the sum over the window in
    FP64.  Returns [nch, n_det, B]."""
    qS2 = quantize_rows(S2w, row_bounds(W2, dt2))
    b1 = row_bounds(W1, dt1)
    nd, B = S2w.shape[0], S1w.shape[0]
    A = qS2.reshape(nd, -1)
    out = []
    for h in Hk:
        hmax = float(np.max(np.abs(h)))
        X = quantize_rows(h[None, :, :] * S1w, hmax * b1)
        out.append(A @ X.reshape(B, -1).T)
    return np.stack(out)


def _fp8_sites(prob, scans, mode, per_site):
    """per_site(M, C, mask, fyfx) for every site, with the FP8 coupling."""
    cfg, geo = prob.cfg, prob.geo
    mode = mode or cfg.recon
    W1 = bip.s1_windows(prob, geo.h_p1, detilt=True)
    W2 = bip.s2_windows(prob, geo.h_p2, detilt=True)
    C = bip.illumination(prob, geo.h_beam, geo.psi_beam, scans)
    out = []
    for k in range(len(prob.ion)):
        iy, ix = prob.window_index(k)
        S1w = bip.reconstruct(W1[k], geo.w1, geo.h_beam, iy, ix, cfg.ny, cfg.nx, +1, mode)
        S2w = bip.reconstruct(W2[k], geo.w2, geo.h_det, iy, ix, cfg.ny, cfg.nx, -1, mode)
        M = site_coupling_fp8(S2w, prob.H[k], S1w, geo.w2, W2[k], geo.w1, W1[k])
        out.append(per_site(M, C, bip.crop_mask(prob, k, scans), bip.detector_factor(prob)))
    return out


def bip_map_fp8(prob, scans=None, mode=None):
    """Algorithm 5 with the coupling operands in scaled E4M3 (everything
    else as in bip.bip_map, FP64)."""
    scans = prob.scans if scans is None else np.asarray(scans, dtype=np.float64)
    partials = _fp8_sites(prob, scans, mode, bip.site_map)
    partials = np.array(partials).reshape(len(partials), len(scans))
    return bip.MapResult(bip.sum_sites(partials), partials)


def per_beam_fp8(prob, scans=None, mode=None):
    """The per-detector-beam intensities qEELS bins (bip.per_beam) with the
    FP8 coupling, [P, n_det]."""
    scans = prob.scans if scans is None else np.asarray(scans, dtype=np.float64)
    out = np.zeros((len(scans), prob.geo.n_det), dtype=np.float64)
    for c in _fp8_sites(prob, scans, mode, bip.site_cube):
        out += c
    return out
