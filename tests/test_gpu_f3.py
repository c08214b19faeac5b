"""GPU parity on grids of 3 x 2^k pixels with PRISM interpolation factor
f = 3 (the register FFTs' radix-3 layer): stashed parent windows straight
from the multislice, maps in FP32 and mixed precision, a cube and qEELS,
against the FP64 oracle."""
import numpy as np
import pytest

import synth
from oracle import bip as obip

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def f3_case(ny, nx, **kw):
    """Gaussian-atom crystal at 0.078 A pixels on an ny x nx grid (cells of
    2.5 A), five slices, 200 keV, 20 mrad, f = 3 (the 64-px window inside
    the 1/f period), the four central atoms of slice 2 ionized, 7 x 6 scans
    around them (sub-pixel positions included)."""
    cy, cx = ny // 32, nx // 32
    c0 = min(cy, cx) // 2 - 1                      # ionized cells c0, c0 + 1 on both axes
    mid = (c0 + 1) * 2.5 / (2.5 / 32)              # their centre in pixels
    cfg = synth.config1().replace(
        name=f"f3_{ny}x{nx}", ny=ny, nx=nx, ly=2.5 * cy, lx=2.5 * cx, cells_y=cy, cells_x=cx, fy=3, fx=3,
        ion_cells=(c0, c0 + 2), ion_slices=(2, 3),
        scan_y=(mid - 9.5, 3.0, 7), scan_x=(mid - 8.25, 3.5, 6), **kw)
    return cfg, synth.make_specimen(cfg)


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2607_00756_gb300 import build
    build.build()
    from paper_2607_00756_gb300.context import BipContext
    return BipContext


@pytest.mark.parametrize("shape", [(192, 192), (384, 192), (384, 384)], ids=lambda s: f"{s[0]}x{s[1]}")
def test_map_f3(lib, shape):
    cfg, sp = f3_case(*shape)
    pr = obip.make_problem(sp)
    assert len(pr.ion) >= 4 and pr.geo.B > 0
    want = obip.bip_map(pr, keep_stages=True)
    dev = torch.device("cuda:0")
    V = torch.tensor(sp.V, dtype=torch.float32, device=dev)
    H = torch.tensor(sp.H, dtype=torch.complex64, device=dev)
    for prec, tol in (("fp32", 1e-4), ("mixed", 1e-3)):
        ctx = lib(cfg, prec=prec)
        try:
            ctx.build(V, sp.atoms, sp.nch)
            if prec == "fp32":
                for k in range(len(pr.ion)):
                    for which, key in ((1, "stash1"), (2, "stash2")):
                        got = ctx.stash(which, k).cpu().numpy()
                        ref = want.stages[k][key]
                        assert np.max(np.abs(got - ref)) < 2e-5 * np.max(np.abs(ref)), (k, which)
            m = ctx.map(H, sp.scans).cpu().numpy()
            assert rel(m, want.map) < tol, prec
        finally:
            ctx.close()


def test_cube_and_qeels_f3(lib):
    """192^2, f = 3: the cube on a 16 x 16 box of k-pixels, and qEELS along
    q_x with the detector beams at f = 1 along x."""
    cfg, sp = f3_case(192, 192, cube_ky=16, cube_kx=16, dfx=1)
    pr = obip.make_problem(sp)
    dev = torch.device("cuda:0")
    V = torch.tensor(sp.V, dtype=torch.float32, device=dev)
    H = torch.tensor(sp.H, dtype=torch.complex64, device=dev)
    ctx = lib(cfg, prec="fp32")
    try:
        ctx.build(V, sp.atoms, sp.nch)
        cube = ctx.cube(V, H, sp.scans).cpu().numpy()
        assert rel(cube, obip.bip_cube(pr)) < 1e-4
        bins, q = ctx.qeels(H, sp.scans, 1)
        bw, want = obip.bip_qeels(pr, 1)
        assert np.array_equal(bins, bw)
        assert rel(q.cpu().numpy(), want) < 1e-4
    finally:
        ctx.close()


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_grad_on_3m_grids(lib, prec):
    """The reverse pass on 192^2, f = 3 -- dL/dV through the adjoint sweeps,
    whose row passes take the radix-3 layer too, and dL/dH -- against the
    oracle's reverse pass (pinned by central differences), 1e-4."""
    from oracle import grad as og
    cfg, sp = f3_case(192, 192)
    pr = obip.make_problem(sp)
    rng = np.random.default_rng(11)
    par = og.Params(pr)
    par.occ = 1.0 + 0.2 * rng.standard_normal(len(pr.ion))
    I0 = og.forward(pr, par)
    gI = 2.0 * (I0 - I0 * (1.0 + 0.1 * rng.standard_normal(I0.shape)))
    _, want = og.gradients(pr, par, dL_dI=gI)
    dev = torch.device("cuda:0")
    V = torch.tensor(sp.V, dtype=torch.float32, device=dev)
    H = torch.tensor(sp.H, dtype=torch.complex64, device=dev)
    ctx = lib(cfg, prec=prec)
    try:
        ctx.build(V, sp.atoms, sp.nch)
        ctx.set_occupancy(par.occ)
        got = ctx.grad(H, sp.scans, torch.tensor(gI, device=dev), occ=False, aberr=False, V=V)
        assert np.linalg.norm(want["V"]) > 0
        assert rel(got["V"].cpu().numpy(), want["V"]) < 1e-4
        wH = np.concatenate([h.reshape(len(h), cfg.win, cfg.win) for h in want["H"]])
        assert rel(got["H"].cpu().numpy(), wH) < 1e-4
    finally:
        ctx.close()
