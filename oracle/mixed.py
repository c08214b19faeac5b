"""The mixed-precision path's roundings, FP64 model.

TEST INFRASTRUCTURE ONLY (see the package header).

The mixed path keeps the method's arithmetic and rounds values at fixed
points.  This module applies those roundings to the oracle's FP64 steps,
with every sum exact, so that the effect of each rounding on the map can be
read off on the CPU:
  * the parents' de-tilted window values (re, im) and their magnitudes, as
    they enter the reconstruction sums (Eq. window-recon, Eq. magpreserve):
    FP16 (`parents="fp16"`, the path as built) or BF16 (`parents="bf16"`);
  * the reconstructed windows as they are written for the coupling, the
    rows S2^d and H_n S1^b: BF16;
  * the coupling result M^(n) (Eq. coupling): BF16, before the Gram product
    and the scan contraction (Algorithm 4's last steps, Eq. map-sum).

Rounding: to the nearest representable value, ties to the even significand.
BF16 keeps 8 significant bits over FP32's exponent range; FP16 (IEEE
binary16) keeps 11, with subnormals below 2^-14 (spacing 2^-24) and 65504
its largest finite value.
"""
import numpy as np

from . import bip

FP16_MAX = 65504.0


def _round_bits(x, bits, emin):
    """Nearest value with `bits` significant bits (ties to even), binades
    below 2^emin sharing that binade's spacing (gradual underflow)."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    _, e = np.frexp(np.where(a > 0.0, a, 1.0))      # a = m 2^e, m in [0.5, 1)
    eb = np.maximum(e - 1, emin)                     # binade exponent floor(log2 a)
    spacing = np.ldexp(1.0, eb - (bits - 1))
    q = np.round(a / spacing) * spacing              # np.round: ties to even
    return np.where(a > 0.0, np.copysign(q, x), 0.0 * x)


def bf16_round(x):
    """Nearest BF16 value of each element (finite inputs in FP32's range)."""
    return _round_bits(x, 8, -126)


def fp16_round(x):
    """Nearest FP16 value of each element; |x| must stay below the overflow
    threshold (the model does not produce infinities)."""
    q = _round_bits(x, 11, -14)
    if np.any(np.abs(q) > FP16_MAX):
        raise OverflowError("value outside the FP16 range")
    return q


def _complex(f, z):
    z = np.asarray(z, dtype=np.complex128)
    return f(z.real) + 1j * f(z.imag)


def reconstruct_mixed(dt, W, h_targets, iy, ix, ny, nx, sign, mode, parents="fp16"):
    """bip.reconstruct with the parent values and magnitudes rounded as the
    mixed path's reconstruction reads them (W exact: it is stored as hi + lo
    to FP32 accuracy)."""
    r = fp16_round if parents == "fp16" else bf16_round
    U = np.tensordot(W, _complex(r, dt), axes=(1, 0))
    if mode == "magnitude":
        A = np.tensordot(W, r(np.abs(dt)), axes=(1, 0))
        mag = np.abs(U)
        safe = np.where(mag > 0.0, mag, 1.0)
        S = np.where(mag > 0.0, A * (U / safe), A)
    elif mode == "complex":
        S = U
    else:
        raise ValueError(mode)
    return S * bip.window_phase(h_targets, iy, ix, ny, nx, sign)


def site_coupling_mixed(S2w, Hk, S1w):
    """M^{(n)} of Eq. coupling from BF16 operand rows (S2^d and H_n S1^b),
    the window sum exact, the result rounded to BF16.  [nch, n_det, B]."""
    nd, B = S2w.shape[0], S1w.shape[0]
    A = _complex(bf16_round, S2w).reshape(nd, -1)
    out = []
    for h in Hk:
        X = _complex(bf16_round, h[None, :, :] * S1w).reshape(B, -1)
        out.append(_complex(bf16_round, A @ X.T))
    return np.stack(out)


def bip_map_mixed(prob, scans=None, mode=None, parents="fp16"):
    """Algorithm 5 with the mixed path's roundings (everything else as in
    bip.bip_map, FP64)."""
    cfg, geo = prob.cfg, prob.geo
    mode = mode or cfg.recon
    scans = prob.scans if scans is None else np.asarray(scans, dtype=np.float64)
    W1 = bip.s1_windows(prob, geo.h_p1, detilt=True)
    W2 = bip.s2_windows(prob, geo.h_p2, detilt=True)
    C = bip.illumination(prob, geo.h_beam, geo.psi_beam, scans)
    partials = []
    for k in range(len(prob.ion)):
        iy, ix = prob.window_index(k)
        S1w = reconstruct_mixed(W1[k], geo.w1, geo.h_beam, iy, ix, cfg.ny, cfg.nx, +1, mode, parents)
        S2w = reconstruct_mixed(W2[k], geo.w2, geo.h_det, iy, ix, cfg.ny, cfg.nx, -1, mode, parents)
        M = site_coupling_mixed(S2w, prob.H[k], S1w)
        partials.append(bip.site_map(M, C, bip.crop_mask(prob, k, scans), bip.detector_factor(prob)))
    partials = np.array(partials).reshape(len(partials), len(scans))
    return bip.MapResult(bip.sum_sites(partials), partials)
