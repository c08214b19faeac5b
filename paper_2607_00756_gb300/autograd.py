"""torch.autograd bridge: the core-loss map as a differentiable function of
the slice potentials V, the transition potentials H, the site occupancies
and the probe defocus and Cs.  The forward and the reverse pass both run in
libbip.so (bip_build_s1/s2 + bip_coreloss_map, bip_coreloss_grad); this
module only passes tensors.

Transition amplitudes a (per site and channel) enter as H -> a H; write
that product in PyTorch before the call and autograd carries the gradient
to a through dL/dH."""
import numpy as np
import torch


class _CorelossMap(torch.autograd.Function):
    @staticmethod
    def forward(fctx, bip, scans, atoms, nch, V, H, occ, defocus, cs):
        if V is not None:
            bip.build(V, atoms, nch)
        bip.set_aberrations(float(defocus), float(cs))
        bip.set_occupancy(occ.detach().cpu().numpy())
        out = bip.map(H, scans)
        fctx.bip, fctx.scans, fctx.atoms, fctx.nch = bip, scans, atoms, nch
        fctx.has_V = V is not None
        fctx.save_for_backward(V if V is not None else torch.empty(0), H, occ, defocus, cs)
        return out

    @staticmethod
    def backward(fctx, grad_out):
        V, H, occ, defocus, cs = fctx.saved_tensors
        bip = fctx.bip
        # the state of the forward pass
        if fctx.has_V:
            bip.build(V, fctx.atoms, fctx.nch)
        bip.set_aberrations(float(defocus), float(cs))
        bip.set_occupancy(occ.detach().cpu().numpy())
        need_V = fctx.has_V and fctx.needs_input_grad[4]
        need_h, need_occ = fctx.needs_input_grad[5], fctx.needs_input_grad[6]
        need_ab = fctx.needs_input_grad[7] or fctx.needs_input_grad[8]
        g = bip.grad(H, fctx.scans, grad_out.to(torch.float64).contiguous(), occ=need_occ, h=need_h, aberr=need_ab,
                     V=V.detach().contiguous() if need_V else None)
        dV = g.get("V")
        dH = g.get("H")
        docc = g["occ"].to(occ.dtype).to(occ.device) if need_occ else None
        ddf = torch.tensor(g["defocus"], dtype=defocus.dtype, device=defocus.device) if need_ab else None
        dcs = torch.tensor(g["cs"], dtype=cs.dtype, device=cs.device) if need_ab else None
        return None, None, None, None, dV, dH, docc, ddf, dcs


def coreloss_map(bip, H, scans, occ=None, defocus=None, cs=None, V=None, atoms=None, nch=None):
    """The map I(rho) [P] float64 for a BipContext, differentiable in H
    (complex64, [sum nch, win, win]), occ ([n_sites]), the scalar tensors
    defocus and cs (Angstrom) and, when V ([nz, ny, nx] float32) is given
    with the atoms, the slice potentials (the matrices are then built from V
    inside the call); without V the context's last build is used."""
    scans = np.asarray(scans, dtype=np.float64)
    dev = H.device
    if V is not None and (atoms is None or nch is None):
        raise ValueError("V needs the atoms and their channel counts")
    if V is not None and bip.n_sites == 0:
        bip.build(V.detach(), atoms, nch)
    if occ is None:
        occ = torch.ones(bip.n_sites, dtype=torch.float64, device=dev)
    if defocus is None:
        defocus = torch.tensor(float(bip.cfg.defocus), dtype=torch.float64)
    if cs is None:
        cs = torch.tensor(float(bip.cfg.cs), dtype=torch.float64)
    return _CorelossMap.apply(bip, scans, atoms, nch, V, H, occ, defocus, cs)
