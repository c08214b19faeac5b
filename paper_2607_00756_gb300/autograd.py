"""torch.autograd bridge: the core-loss map as a differentiable function of
the transition potentials H, the site occupancies and the probe defocus
and Cs.  The forward and the reverse pass both run in libbip.so
(bip_coreloss_map and bip_coreloss_grad); this module only passes tensors.

Transition amplitudes a (per site and channel) enter as H -> a H; write
that product in PyTorch before the call and autograd carries the gradient
to a through dL/dH."""
import numpy as np
import torch

from . import capi


class _CorelossMap(torch.autograd.Function):
    @staticmethod
    def forward(fctx, bip, scans, H, occ, defocus, cs):
        bip.set_aberrations(float(defocus), float(cs))
        bip.set_occupancy(occ.detach().cpu().numpy())
        out = bip.map(H, scans)
        fctx.bip, fctx.scans = bip, scans
        fctx.save_for_backward(H, occ, defocus, cs)
        return out

    @staticmethod
    def backward(fctx, grad_out):
        H, occ, defocus, cs = fctx.saved_tensors
        bip = fctx.bip
        # the state of the forward pass
        bip.set_aberrations(float(defocus), float(cs))
        bip.set_occupancy(occ.detach().cpu().numpy())
        need_h, need_occ = fctx.needs_input_grad[2], fctx.needs_input_grad[3]
        need_ab = fctx.needs_input_grad[4] or fctx.needs_input_grad[5]
        g = bip.grad(H, fctx.scans, grad_out.to(torch.float64).contiguous(), occ=need_occ, h=need_h, aberr=need_ab)
        dH = g.get("H")
        docc = g["occ"].to(occ.dtype).to(occ.device) if need_occ else None
        ddf = torch.tensor(g["defocus"], dtype=defocus.dtype, device=defocus.device) if need_ab else None
        dcs = torch.tensor(g["cs"], dtype=cs.dtype, device=cs.device) if need_ab else None
        return None, None, dH, docc, ddf, dcs


def coreloss_map(bip, H, scans, occ=None, defocus=None, cs=None):
    """The map I(rho) [P] float64 for a built BipContext, differentiable in
    H (complex64, [sum nch, win, win]), occ ([n_sites]) and the scalar
    tensors defocus and cs (Angstrom)."""
    scans = np.asarray(scans, dtype=np.float64)
    dev = H.device
    if occ is None:
        occ = torch.ones(bip.n_sites, dtype=torch.float64, device=dev)
    if defocus is None:
        defocus = torch.tensor(float(bip.cfg.defocus), dtype=torch.float64)
    if cs is None:
        cs = torch.tensor(float(bip.cfg.cs), dtype=torch.float64)
    return _CorelossMap.apply(bip, scans, H, occ, defocus, cs)
