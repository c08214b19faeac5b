"""Convenience wrapper over the C ABI: owns a bip_ctx and allocates the
output tensors with PyTorch.  Marshalling only -- every step runs in
libbip.so."""
import numpy as np
import torch

from . import capi


class BipContext:
    def __init__(self, cfg, prec=None, recon=None):
        self.cfg = cfg
        self._struct = capi.make_config(cfg, prec=prec, recon=recon)
        self.ctx = capi.bip_create(self._struct)
        self.B, self.n_det, self.Bp1, self.Bp2, _ = capi.bip_query(self.ctx)
        self._geo = None
        self._atoms = None
        self.n_sites = 0

    @property
    def geometry(self):
        if self._geo is None:
            self._geo = capi.bip_get_geometry(self.ctx)
        return self._geo

    def set_precision(self, prec):
        capi.bip_set_precision(self.ctx, prec)

    def build(self, V, atoms, nch, stream=None):
        """S1 and S2 builds (both window stashes) from a device V, the two
        sweeps side by side (bip_build)."""
        self._atoms = capi.make_atoms(atoms, nch)
        self._nch_max = int(np.max(nch))
        capi.bip_build(self.ctx, V, self._atoms, stream)
        self.n_sites = capi.bip_query(self.ctx)[4]

    def _config_values(self):
        c = capi.bip_get_config(self.ctx)
        return np.array([float(getattr(c, name)) for name, _ in capi.BipConfig._fields_])

    def save_builds(self, path, stream=None):
        """Writes both window stashes, the sites and the configuration to
        `path` (.npz), for map-only reruns in another process."""
        stashes = {}
        for which in (1, 2):
            host = np.empty(capi.stash_shape(self.ctx, which), dtype=np.complex64)
            capi.bip_export_stash(self.ctx, which, host, stream)
            stashes[f"s{which}"] = host
        atoms = np.ctypeslib.as_array(self._atoms)
        np.savez(path, config=self._config_values(), y=atoms["y"], x=atoms["x"], slice=atoms["slice"], nch=atoms["nch"], **stashes)

    def load_builds(self, path, stream=None):
        """Restores what save_builds wrote; the file's configuration must be
        this context's (else ValueError, nothing restored)."""
        with np.load(path) as f:
            if not np.array_equal(f["config"], self._config_values()):
                raise ValueError("the builds in this file were made with another configuration")
            atoms = np.stack([f["y"], f["x"], f["slice"].astype(np.float64)], axis=1)
            nch = f["nch"]
            self._atoms = capi.make_atoms(atoms, nch)
            self._nch_max = int(np.max(nch))
            for which in (1, 2):
                capi.bip_import_stash(self.ctx, which, self._atoms, np.ascontiguousarray(f[f"s{which}"]), stream)
        self.n_sites = capi.bip_query(self.ctx)[4]

    def set_check_finite(self, on):
        capi.bip_set_check_finite(self.ctx, on)

    def build_s1(self, V, atoms, nch, stream=None):
        self._atoms = capi.make_atoms(atoms, nch)
        capi.bip_build_s1(self.ctx, V, self._atoms, stream)
        self.n_sites = capi.bip_query(self.ctx)[4]

    def build_s2(self, V, atoms, nch, stream=None):
        self._atoms = capi.make_atoms(atoms, nch)
        capi.bip_build_s2(self.ctx, V, self._atoms, stream)
        self.n_sites = capi.bip_query(self.ctx)[4]

    def map(self, H, scans, out=None, stream=None):
        scans = np.asarray(scans, dtype=np.float64)
        if out is None:
            out = torch.empty(len(scans), dtype=torch.float64, device=H.device)
        return capi.bip_coreloss_map(self.ctx, H, scans, out, stream)

    @property
    def cube_beams(self):
        """The cube's complete output basis, [n_cube, 2] (h_y, h_x)."""
        return capi.bip_cube_beams(self.ctx)

    def cube(self, V, H, scans, out=None, stream=None):
        """The 4D cube [P, n_cube] on the complete output basis (S1
        partitioned, the exit exact; needs the S1 build and the potential V
        it was built from)."""
        scans = np.asarray(scans, dtype=np.float64)
        if out is None:
            out = torch.empty((len(scans), len(self.cube_beams)), dtype=torch.float32, device=H.device)
        return capi.bip_coreloss_cube(self.ctx, V, H, scans, out, stream)

    def set_cube_memory(self, nbytes):
        """Device bytes the cube may take per batch of exact S2 columns (0: half
        the free memory, at most 96 GB)."""
        capi.bip_set_cube_memory(self.ctx, nbytes)

    def qeels(self, H, scans, axis, out=None, stream=None):
        """Momentum-resolved output: (bin h values, [P, n_bins]) resolved along
        axis 0 (q_y; the context needs dfy = 1) or 1 (q_x; dfx = 1); its sum
        over the bins is the map."""
        scans = np.asarray(scans, dtype=np.float64)
        bins = capi.bip_qeels_bins(self.ctx, axis)
        if out is None:
            out = torch.empty((len(scans), len(bins)), dtype=torch.float32, device=H.device)
        return bins, capi.bip_coreloss_qeels(self.ctx, H, scans, axis, out, stream)

    def sites(self, H, scans, out=None, stream=None):
        scans = np.asarray(scans, dtype=np.float64)
        if out is None:
            out = torch.empty((self.n_sites, len(scans)), dtype=torch.float32, device=H.device)
        return capi.bip_coreloss_sites(self.ctx, H, scans, out, stream)

    def stash(self, which, site, device="cuda"):
        n = self.Bp1 if which == 1 else self.Bp2
        w = self.cfg.win
        out = torch.empty((n, w, w), dtype=torch.complex64, device=device)
        return capi.bip_copy_stash(self.ctx, which, site, out)

    def windows(self, site, device="cuda"):
        w = self.cfg.win
        s1 = torch.empty((self.B, w, w), dtype=torch.complex64, device=device)
        s2 = torch.empty((self.n_det, w, w), dtype=torch.complex64, device=device)
        return capi.bip_site_windows(self.ctx, site, s1, s2)

    def coupling(self, H, site, device="cuda"):
        """M^(n) of one site, [nch_max, n_det, B] complex64, in the context's
        precision."""
        nch = int(max(1, getattr(self, "_nch_max", 0)))
        out = torch.empty((nch, self.n_det, self.B), dtype=torch.complex64, device=device)
        return capi.bip_site_coupling(self.ctx, H, site, out)

    def set_order(self, order):
        """Scan contraction: 0 (default) Gram matrix, 1 beam order, 2 probe
        order (mixed precision, up to 2048 scans)."""
        capi.bip_set_order(self.ctx, order)

    def autotune(self, H, scans, out=None, stream=None):
        """Time launch choices on this map and keep the fastest: returns
        (sites per batch, coupling tile width (0: built-in), contraction order,
        ms per map)."""
        scans = np.asarray(scans, dtype=np.float64)
        if out is None:
            out = torch.empty(len(scans), dtype=torch.float64, device=H.device)
        return capi.bip_autotune(self.ctx, H, scans, out, stream)

    def set_raster_eval(self, on):
        """Separable scan-polynomial evaluation on raster scan lists (default
        on); off: Horner's rule per scan."""
        capi.bip_set_raster_eval(self.ctx, on)

    def set_launch(self, sites_per_batch=0, coupling_tile=0):
        capi.bip_set_launch(self.ctx, sites_per_batch, coupling_tile)

    def set_occupancy(self, occ):
        """Per-site occupancies weighting the site sum (None: all 1)."""
        capi.bip_set_occupancy(self.ctx, None if occ is None else np.asarray(occ, dtype=np.float64))

    def set_site_windows(self, win, stream=None):
        """Per-site windows (multiples of 16 up to the context's win; 0 or None:
        the context's win) for the following maps; H then holds each site's
        channels on its own window, flattened in site order."""
        capi.bip_set_site_windows(self.ctx, None if win is None else np.asarray(win, dtype=np.int32), stream)

    def set_aberrations(self, defocus, cs, stream=None):
        """Probe defocus and Cs (Angstrom) for the next map."""
        capi.bip_set_aberrations(self.ctx, defocus, cs, stream)

    def grad(self, H, scans, dL_dI, occ=True, h=True, aberr=True, V=None, stream=None):
        """Reverse pass of a scalar loss of the map, given dL/dI on the scans:
        {"occ": [n_sites] float64, "H": H's shape complex64 (dL/dRe + i dL/dIm),
        "defocus", "cs": floats, "V": [nz, ny, nx] float32 when V (the
        potential the matrices were built from) is given}, each only when
        asked for."""
        scans = np.asarray(scans, dtype=np.float64)
        d_occ = torch.empty(self.n_sites, dtype=torch.float64, device=H.device) if occ else None
        d_H = torch.empty_like(H) if h else None
        d_V = torch.empty_like(V) if V is not None else None
        ab = capi.bip_coreloss_grad(self.ctx, H, scans, dL_dI.contiguous(), d_occ, d_H, aberr, V, d_V, stream)
        out = {}
        if d_V is not None:
            out["V"] = d_V
        if occ:
            out["occ"] = d_occ
        if h:
            out["H"] = d_H
        if aberr:
            out["defocus"], out["cs"] = ab
        return out

    def close(self):
        if self.ctx:
            capi.bip_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
