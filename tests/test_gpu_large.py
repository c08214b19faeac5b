"""GPU parity on the largest grids the library accepts (1024 pixels on an
axis) and on 512-pixel rows (the half-warp row pass): the register FFTs of
the row and column passes, the windows and tables at those sizes, in FP32
and mixed precision, against the oracle's map on a few scans around the
sites and, in FP32, the stashed parent windows."""
import numpy as np
import pytest

import synth
from oracle import bip as obip

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def large_case(ny, nx):
    """32 x 32 (or 32 x 8) cells of 2.5 A at 0.078 A pixels, three slices,
    300 keV, 20 mrad, f = 8 on a 1024 axis and 4 on a 256 one (the 64-px
    window inside the 1/f period),
    a 30 mrad detector, three ionized atoms of the middle slice (one near
    the cell edge, its window wrapping), 5 x 4 scans around them."""
    cy, cx = ny // 32, nx // 32
    cfg = synth.config1().replace(
        name=f"grid{ny}x{nx}", ny=ny, nx=nx, ly=2.5 * cy, lx=2.5 * cx, cells_y=cy, cells_x=cx,
        nz=3, e0=300e3, alpha=0.020, theta_det=0.030, fy=8 if ny >= 512 else 4, fx=8 if nx >= 512 else 4,
        ion_slices=(1, 2), ion_cells=(0, 0))
    sp = synth.make_specimen(cfg)
    nch = np.zeros_like(sp.nch)
    ncell = cy * cx
    pick = [ncell + (cy // 2) * cx + cx // 2, ncell + (cy // 2) * cx + cx // 2 + 1, ncell + 0]
    nch[pick] = 3
    H = np.concatenate([synth.specimen._transition(cfg, sp.atoms, np.where(np.arange(len(nch)) == a, 3, 0))
                        for a in sorted(pick)])
    ys = sp.atoms[pick[0], 0] / (cfg.ly / ny) + np.array([-7.0, -2.0, 0.5, 3.0, 9.0])
    xs = sp.atoms[pick[0], 1] / (cfg.lx / nx) + np.array([-6.0, 0.0, 2.5, 8.0])
    scans = np.stack(np.meshgrid(ys, xs, indexing="ij"), axis=-1).reshape(-1, 2)
    return cfg, synth.Specimen(cfg=cfg, atoms=sp.atoms, nch=nch, V=sp.V, H=H, scans=scans)


@pytest.mark.parametrize("shape", [(1024, 1024), (1024, 256), (256, 1024), (512, 512), (256, 512)],
                         ids=lambda s: f"{s[0]}x{s[1]}")
def test_map_on_1024_grids(shape):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2607_00756_gb300 import build
    build.build()
    from paper_2607_00756_gb300.context import BipContext
    cfg, sp = large_case(*shape)
    pr = obip.make_problem(sp)
    assert len(pr.ion) == 3
    want = obip.bip_map(pr, keep_stages=True)
    dev = torch.device("cuda:0")
    V = torch.tensor(sp.V, dtype=torch.float32, device=dev)
    H = torch.tensor(sp.H, dtype=torch.complex64, device=dev)
    for prec, tol in (("fp32", 1e-4), ("mixed", 1e-3)):
        ctx = BipContext(cfg, prec=prec)
        try:
            ctx.build(V, sp.atoms, sp.nch)
            m = ctx.map(H, sp.scans).cpu().numpy()
            parts = ctx.sites(H, sp.scans).cpu().numpy()
            assert rel(m, want.map) < tol, prec
            assert rel(parts, want.partials) < tol, prec
            if prec == "fp32":
                # the stashed parent windows straight from the 1024-point passes
                for k in range(3):
                    for which, key in ((1, "stash1"), (2, "stash2")):
                        got = ctx.stash(which, k).cpu().numpy()
                        ref = want.stages[k][key]
                        assert np.max(np.abs(got - ref)) < 2e-5 * np.max(np.abs(ref)), (k, which)
        finally:
            ctx.close()
