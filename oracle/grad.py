"""Gradients of a map loss through Algorithm 5, FP64 reverse mode by hand.

TEST INFRASTRUCTURE ONLY (see the package header).

The scattering matrices the method builds are a forward model (Sec. 5
names simulation-constrained reconstruction as a use); these are the
derivatives of a scalar loss of the map with respect to the model's inputs:
  * per-site occupancy o_tau:           I = sum_tau o_tau I_tau (Eq. map-sum);
  * per-channel transition amplitude a: H_{tau,n} -> a_{tau,n} H_{tau,n}
                                        (Eq. coupling), and H itself;
  * probe defocus and Cs:               Psi(h) = exp(-i chi(q)),
                                        chi = pi lam df |q|^2 + pi/2 Cs lam^3 |q|^4
                                        (Eq. probe; the sign is the reading
                                        of geometry.aperture_function);
  * slice potentials V_j:               T_j = exp(i sigma V_j) in both the
                                        S1 sweep (Eq. smatrix-advance) and the
                                        S2 sweep (Eq. s2).
The loss is L = sum_rho (I(rho) - target(rho))^2 unless dL/dI is given.

Conventions.  For a complex variable z the adjoint is zbar = dL/dz* (so
that dL = 2 Re sum conj(zbar) dz); a complex parameter's gradient is
reported as dL/dRe z + i dL/dIm z = 2 zbar.  Steps, in reverse order:
  map -> I_tau:  dL/do_tau = sum_rho g I_tau,  g = dL/dI;
  I_tau = f c^H Q c with Q = sum_n M_n^H M_n, f = f_y f_x:
                 Mbar_n = M_n R,  R = f sum_{rho in crop} o_tau g c c^H;
                 the aberration derivative of theta: dL/dtheta =
                 -2 sum_b chi'_b Im D_b, D_b = sum_tau (Q_tau R_tau)_bb;
  M_n = S2^T diag(H_n) S1:
                 Hbar_n(r) = sum_b conj S1_b(r) T_n(b, r),
                 T_n(b, r) = sum_d Mbar_n(d, b) conj S2_d(r);
                 S1bar_b(r) = sum_n conj H_n(r) T_n(b, r);
                 S2bar_d(r) = sum_n conj H_n(r) sum_b Mbar_n(d, b) conj S1_b(r);
  S = phi A U/|U| (Eq. magpreserve, U = sum_p w dt_p, A = sum_p w |dt_p|):
                 Ebar = Sbar conj(phi), dL/dA = 2 Re(conj(Ebar) u),
                 Ubar = -(A/|U|) Im(conj(Ebar) u) i u  (u = U/|U|),
                 dtbar_p = sum_t w_tp (Ubar_t + dL/dA_t dt_p / (2 |dt_p|));
  de-tilt / window crop: scattered back to the grid at the site's plane;
  S1 sweep psi_{j+1} = Prop(T_j psi_j), backwards over j:
                 ubar = Prop^H(psibar_{j+1}), dL/dV_j -= 2 sigma Im(conj(ubar) T_j psi_j),
                 psibar_j = conj(T_j) ubar + (injections at plane j);
  S2 sweep x_j = T_j Prop(x_{j+1}), forwards over j:
                 xbar_j = (injections) + Prop^H(conj(T_{j-1}) xbar_{j-1}),
                 dL/dV_j -= 2 sigma Im(conj(xbar_j) x_j).
Prop = F^-1 P F is normal, Prop^H = F^-1 conj(P) F.  Where |U| or |dt_p| is
zero the (measure-zero) non-differentiable terms are taken as 0.

Every derivative is pinned by central finite differences of `loss`
(tests/test_oracle_grad.py)."""
import math
import numpy as np

from . import bip
from . import physics as ph
from .geometry import aperture_function, beam_q


class Params:
    """Differentiable inputs: occ [n_ion], amp [n_ion, nch] complex,
    defocus and cs (Angstrom), V [nz, ny, nx] (V Angstrom)."""

    def __init__(self, prob, occ=None, amp=None, defocus=None, cs=None, V=None):
        n = len(prob.ion)
        nch = max((len(h) for h in prob.H), default=0)
        self.occ = np.ones(n) if occ is None else np.asarray(occ, dtype=np.float64)
        self.amp = np.ones((n, nch), dtype=np.complex128) if amp is None else np.asarray(amp, dtype=np.complex128)
        self.defocus = prob.cfg.defocus if defocus is None else float(defocus)
        self.cs = prob.cfg.cs if cs is None else float(cs)
        self.V = np.array(prob.V if V is None else V, dtype=np.float64)

    def copy(self):
        p = Params.__new__(Params)
        p.occ, p.amp, p.V = self.occ.copy(), self.amp.copy(), self.V.copy()
        p.defocus, p.cs = self.defocus, self.cs
        return p


def _coef(prob, defocus, cs):
    """c_b(rho) coefficients f_y f_x Psi(h_b) / sqrt(G sum |Psi|^2) and the
    phase derivatives chi'_b with respect to defocus and Cs."""
    cfg, geo = prob.cfg, prob.geo
    psi_full = aperture_function(geo.h_full, cfg.ly, cfg.lx, prob.lam, defocus, cs)
    psi_beam = aperture_function(geo.h_beam, cfg.ly, cfg.lx, prob.lam, defocus, cs)
    norm = math.sqrt(cfg.ny * cfg.nx * float(np.sum(np.abs(psi_full) ** 2)))
    q = beam_q(geo.h_beam, cfg.ly, cfg.lx)
    q2 = q[:, 0] ** 2 + q[:, 1] ** 2
    dchi = {"defocus": np.pi * prob.lam * q2, "cs": 0.5 * np.pi * prob.lam ** 3 * q2 ** 2}
    return cfg.fy * cfg.fx * psi_beam / norm, dchi


def _scan_phase(prob, scans):
    cfg, geo = prob.cfg, prob.geo
    ph_ = (np.outer(geo.h_beam[:, 0], scans[:, 0]) / cfg.ny + np.outer(geo.h_beam[:, 1], scans[:, 1]) / cfg.nx)
    return np.exp(-2j * np.pi * ph_)                                   # [B, P]


def _sweeps(prob, V):
    """Full-grid states of both sweeps: psi[j] (S1, j = 0..max plane) and
    x[j] (S2, j = min plane..N_Z; x[N_Z] the start)."""
    cfg, geo = prob.cfg, prob.geo
    sigma = prob.sigma
    T = [ph.transmission(V[j], sigma) for j in range(cfg.nz)]
    jmax, jmin = int(prob.plane.max()), int(prob.plane.min())
    psi = [np.stack([ph.plane_wave(h, cfg.ny, cfg.nx, +1) for h in geo.h_p1])]
    for j in range(jmax):
        psi.append(ph.step(psi[-1], T[j], prob.P))
    g = cfg.ny * cfg.nx
    x = {cfg.nz: np.stack([ph.plane_wave(h, cfg.ny, cfg.nx, -1) for h in geo.h_p2]) / math.sqrt(g)}
    for j in range(cfg.nz - 1, jmin - 1, -1):
        x[j] = T[j] * ph.propagate(x[j + 1], prob.P)
    return T, psi, x


def _recon_parts(dt, W, h_t, iy, ix, ny, nx, sign, mode):
    U = np.tensordot(W, dt, axes=(1, 0))
    phi = bip.window_phase(h_t, iy, ix, ny, nx, sign)
    if mode == "magnitude":
        A = np.tensordot(W, np.abs(dt), axes=(1, 0))
        m = np.abs(U)
        u = np.where(m > 0.0, U / np.where(m > 0.0, m, 1.0), 1.0)
        return A * u * phi, (U, A, m, u, phi)
    return U * phi, (U, None, None, None, phi)


def _recon_adjoint(Sbar, dt, W, parts, mode):
    U, A, m, u, phi = parts
    Ebar = Sbar * np.conj(phi)
    if mode != "magnitude":
        return np.tensordot(W.T, Ebar, axes=(1, 0))
    dA = 2.0 * np.real(np.conj(Ebar) * u)
    safe = np.where(m > 0.0, m, 1.0)
    Ubar = np.where(m > 0.0, -(A / safe) * np.imag(np.conj(Ebar) * u) * 1j * u, 0.0)
    adt = np.abs(dt)
    unit = np.where(adt > 0.0, dt / np.where(adt > 0.0, adt, 1.0), 0.0)
    return np.tensordot(W.T, Ubar, axes=(1, 0)) + 0.5 * np.tensordot(W.T, dA, axes=(1, 0)) * unit


def forward(prob, params, scans=None, mode=None, keep=False):
    """The map I(rho) of Algorithm 5 under params (FP64); with keep, the
    intermediates the reverse pass needs."""
    cfg, geo = prob.cfg, prob.geo
    mode = mode or cfg.recon
    scans = prob.scans if scans is None else np.asarray(scans, dtype=np.float64)
    T, psi, x = _sweeps(prob, params.V)
    coef, dchi = _coef(prob, params.defocus, params.cs)
    E = _scan_phase(prob, scans)
    C = coef[:, None] * E
    fyfx = bip.detector_factor(prob)
    sites, partials = [], []
    for k in range(len(prob.ion)):
        iy, ix = prob.window_index(k)
        i = int(prob.plane[k])
        dt1 = psi[i][:, iy[:, None], ix[None, :]] * bip.window_phase(geo.h_p1, iy, ix, cfg.ny, cfg.nx, -1)
        dt2 = x[i][:, iy[:, None], ix[None, :]] * bip.window_phase(geo.h_p2, iy, ix, cfg.ny, cfg.nx, +1)
        S1, p1 = _recon_parts(dt1, geo.w1, geo.h_beam, iy, ix, cfg.ny, cfg.nx, +1, mode)
        S2, p2 = _recon_parts(dt2, geo.w2, geo.h_det, iy, ix, cfg.ny, cfg.nx, -1, mode)
        Heff = params.amp[k, :len(prob.H[k]), None, None] * prob.H[k]
        M = bip.coupling(S2, Heff, S1)
        mask = bip.crop_mask(prob, k, scans)
        part = bip.site_map(M, C, mask, fyfx)
        partials.append(part)
        if keep:
            sites.append(dict(iy=iy, ix=ix, i=i, dt1=dt1, dt2=dt2, S1=S1, S2=S2, p1=p1, p2=p2, Heff=Heff, M=M,
                              mask=mask))
    partials = np.array(partials).reshape(len(partials), len(scans))
    total = np.einsum("k,kp->p", params.occ, partials)
    if not keep:
        return total
    return total, dict(T=T, psi=psi, x=x, coef=coef, dchi=dchi, C=C, sites=sites, partials=partials, mode=mode)


def loss(prob, params, target, scans=None, mode=None):
    """L = sum_rho (I(rho) - target(rho))^2."""
    I = forward(prob, params, scans, mode)
    return float(np.sum((I - target) ** 2))


def gradients(prob, params, target=None, scans=None, mode=None, dL_dI=None, want_V=True):
    """dL/d(occ, amp, H, defocus, cs, V) by the reverse pass in the module
    header (without want_V, the sweeps' reverse pass is skipped and "V" is
    absent).  Returns (L or None, dict); complex entries are dL/dRe + i dL/dIm."""
    cfg, geo = prob.cfg, prob.geo
    scans = prob.scans if scans is None else np.asarray(scans, dtype=np.float64)
    I, fw = forward(prob, params, scans, mode, keep=True)
    mode = fw["mode"]
    if dL_dI is None:
        g = 2.0 * (I - target)
        L = float(np.sum((I - target) ** 2))
    else:
        g = np.asarray(dL_dI, dtype=np.float64)
        L = None
    fyfx = bip.detector_factor(prob)
    C = fw["C"]
    n_ion = len(prob.ion)
    out = {"occ": fw["partials"] @ g, "amp": np.zeros_like(params.amp), "H": [], "defocus": 0.0, "cs": 0.0}
    D = np.zeros(geo.B, dtype=np.complex128)
    inj1 = {}      # psibar at S1 planes
    inj2 = {}      # xbar at S2 planes
    for k in range(n_ion):
        s = fw["sites"][k]
        mask = s["mask"]
        Hk = prob.H[k]
        nch = len(Hk)
        if not np.any(mask):
            out["H"].append(np.zeros_like(Hk))
            continue
        Cm = C[:, mask]
        gm = params.occ[k] * g[mask]
        R = fyfx * (Cm * gm[None, :]) @ Cm.conj().T                   # [B, B]
        M = s["M"]
        Q = sum(Mn.conj().T @ Mn for Mn in M)
        D += np.einsum("bc,cb->b", Q, R)
        S1 = s["S1"].reshape(geo.B, -1)
        S2 = s["S2"].reshape(geo.n_det, -1)
        Hbar = np.zeros((nch, S1.shape[1]), dtype=np.complex128)
        S1bar = np.zeros_like(S1)
        S2bar = np.zeros_like(S2)
        Heff = s["Heff"].reshape(nch, -1)
        for n in range(nch):
            Mbar = M[n] @ R                                             # [n_det, B]
            Tn = Mbar.T @ np.conj(S2)                                   # [B, K]
            Hbar[n] = np.sum(np.conj(S1) * Tn, axis=0)
            S1bar += np.conj(Heff[n])[None, :] * Tn
            S2bar += np.conj(Heff[n])[None, :] * (Mbar @ np.conj(S1))
        w = int(prob.win[k])                                            # the site's window
        out["amp"][k, :nch] = 2.0 * np.sum(Hbar * np.conj(Hk.reshape(nch, -1)), axis=1)
        out["H"].append((2.0 * np.conj(params.amp[k, :nch, None]) * Hbar).reshape(nch, w, w))
        if not want_V:
            continue
        # back through the reconstructions and the window crops
        dt1bar = _recon_adjoint(S1bar.reshape(geo.B, w, w), s["dt1"], geo.w1, s["p1"], mode)
        dt2bar = _recon_adjoint(S2bar.reshape(geo.n_det, w, w), s["dt2"], geo.w2, s["p2"], mode)
        iy, ix, i = s["iy"], s["ix"], s["i"]
        g1 = dt1bar * bip.window_phase(geo.h_p1, iy, ix, cfg.ny, cfg.nx, +1)
        g2 = dt2bar * bip.window_phase(geo.h_p2, iy, ix, cfg.ny, cfg.nx, -1)
        for inj, gw, nb in ((inj1, g1, len(geo.h_p1)), (inj2, g2, len(geo.h_p2))):
            if i not in inj:
                inj[i] = np.zeros((nb, cfg.ny, cfg.nx), dtype=np.complex128)
            yy, xx = np.meshgrid(iy, ix, indexing="ij")
            for p in range(nb):
                np.add.at(inj[i][p], (yy, xx), gw[p])
    for name in ("defocus", "cs"):
        out[name] = float(-2.0 * np.sum(fw["dchi"][name] * np.imag(D)))
    if not want_V:
        return L, out
    # slice potentials: the two sweeps backwards
    sigma = prob.sigma
    T, psi, x = fw["T"], fw["psi"], fw["x"]
    gV = np.zeros_like(params.V)
    P = prob.P
    jmax, jmin = len(psi) - 1, min(x)
    lam = inj1.get(jmax, np.zeros_like(psi[jmax]))
    for j in range(jmax - 1, -1, -1):
        ubar = ph.propagate(lam, np.conj(P))
        u = T[j] * psi[j]
        gV[j] -= 2.0 * sigma * np.sum(np.imag(np.conj(ubar) * u), axis=0)
        lam = np.conj(T[j]) * ubar + inj1.get(j, 0.0)
    xbar = None
    for j in range(jmin, cfg.nz):
        cur = inj2.get(j, np.zeros_like(x[j]))
        if xbar is not None:
            cur = cur + ph.propagate(np.conj(T[j - 1]) * xbar, np.conj(P))
        gV[j] -= 2.0 * sigma * np.sum(np.imag(np.conj(cur) * x[j]), axis=0)
        xbar = cur
    out["V"] = gV
    return L, out
