"""GPU parity of the reverse pass (bip_coreloss_grad and the torch.autograd
bridge) against the oracle's hand-written reverse pass (oracle/grad.py,
itself pinned by finite differences): occupancies, transition potentials H
(and through them the transition amplitudes), probe defocus and Cs, and the
slice potentials V (through the reconstruction and both sweeps, with the
sweeps' forward states recomputed from checkpoints).  The
same dL/dI (from the oracle's forward map) drives both sides.  Tolerance:
rel <= 1e-4 for every derivative computed by the reverse pass's own
contractions (FP32 SIMT in an FP32 context, split BF16 on tcgen05 in a
mixed one); the occupancy gradient of a mixed context is the exact
reduction of its BF16 partials, which meet the mixed bar (1e-3)."""
import numpy as np
import pytest

import synth
from oracle import bip as obip
from oracle import grad as og

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2607_00756_gb300 import build
    build.build()
    from paper_2607_00756_gb300.context import BipContext
    return BipContext


def small_case(recon="magnitude"):
    cfg = synth.config1().replace(name="grad", ny=64, nx=64, ly=5.0, lx=5.0, nz=4, cells_y=2, cells_x=2, win=32,
                                  fy=2, fx=2, ion_slices=(1, 3), ion_cells=(0, 1), defocus=30.0, cs=2.0e5,
                                  recon=recon, scan_y=(10.0, 6.0, 4), scan_x=(12.0, 5.0, 4))
    sp = synth.make_specimen(cfg)
    pr = obip.make_problem(sp)
    rng = np.random.default_rng(5)
    par = og.Params(pr)
    par.occ = 1.0 + 0.2 * rng.standard_normal(len(pr.ion))
    I0 = og.forward(pr, par)
    target = I0 * (1.0 + 0.1 * rng.standard_normal(I0.shape))
    return cfg, sp, pr, par, target


def config1_case():
    cfg = synth.config1().replace(defocus=-40.0, cs=1.0e5)
    sp = synth.make_specimen(cfg)
    pr = obip.make_problem(sp)
    rng = np.random.default_rng(8)
    par = og.Params(pr)
    par.occ = 1.0 + 0.3 * rng.standard_normal(len(pr.ion))
    I0 = og.forward(pr, par)
    target = I0 * (1.0 + 0.1 * rng.standard_normal(I0.shape))
    return cfg, sp, pr, par, target


def _gpu(lib, cfg, sp, prec="fp32"):
    dev = torch.device("cuda:0")
    ctx = lib(cfg, prec=prec)
    ctx.build(torch.tensor(sp.V, dtype=torch.float32, device=dev), sp.atoms, sp.nch)
    H = torch.tensor(sp.H, dtype=torch.complex64, device=dev)
    return ctx, H


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
@pytest.mark.parametrize("which", ["small_magnitude", "small_complex", "config1"])
def test_grad_matches_oracle(lib, which, prec):
    """FP32 context: every contraction FP32 SIMT; mixed context: the reverse
    pass's contractions on tcgen05 in split BF16 (same 1e-4 bar), the map
    and the occupancy gradient's partials in the context's precision."""
    if which == "config1":
        cfg, sp, pr, par, target = config1_case()
    else:
        cfg, sp, pr, par, target = small_case(which.split("_")[1])
    I = og.forward(pr, par)
    gI = 2.0 * (I - target)
    _, want = og.gradients(pr, par, dL_dI=gI, want_V=False)
    ctx, H = _gpu(lib, cfg, sp, prec=prec)
    ctx.set_occupancy(par.occ)
    got = ctx.grad(H, sp.scans, torch.tensor(gI, device=H.device))
    torch.cuda.synchronize()
    if prec == "fp32":
        assert rel(ctx.map(H, sp.scans).cpu().numpy(), I) < 1e-4
        assert rel(got["occ"].cpu().numpy(), want["occ"]) < 1e-4
    else:
        # the occupancy gradient is the exact reduction of the context's own
        # (BF16) partials; their accuracy is the forward map's, tested on the
        # workloads in test_gpu_map.py
        parts = ctx.sites(H, sp.scans).cpu().numpy().astype(np.float64)
        assert rel(got["occ"].cpu().numpy(), parts @ gI) < 1e-9
    gH = got["H"].cpu().numpy()
    wH = np.concatenate([h.reshape(len(h), cfg.win, cfg.win) for h in want["H"]])
    assert gH.shape == wH.shape
    assert rel(gH, wH) < 1e-4, rel(gH, wH)
    for name in ("defocus", "cs"):
        assert got[name] == pytest.approx(want[name], rel=1e-4), (name, got[name], want[name])
    ctx.close()


def test_grad_occupancy_mixed_context(lib):
    """A mixed-precision context: the occupancy gradient comes from its own
    (BF16-contraction) partials, within 1e-3."""
    cfg, sp, pr, par, target = config1_case()
    I = og.forward(pr, par)
    gI = 2.0 * (I - target)
    _, want = og.gradients(pr, par, dL_dI=gI, want_V=False)
    ctx, H = _gpu(lib, cfg, sp, prec="mixed")
    ctx.set_occupancy(par.occ)
    got = ctx.grad(H, sp.scans, torch.tensor(gI, device=H.device), h=False, aberr=False)
    assert rel(got["occ"].cpu().numpy(), want["occ"]) < 1e-3
    ctx.close()


def test_autograd_loss_backward(lib):
    """loss = sum (map - target)^2 through torch.autograd, with transition
    amplitudes a (H -> a H written in PyTorch): occupancy, amplitude, defocus
    and Cs gradients against the oracle's."""
    from paper_2607_00756_gb300.autograd import coreloss_map
    cfg, sp, pr, par, target = small_case()
    rng = np.random.default_rng(21)
    par.amp = (1.0 + 0.2 * rng.standard_normal(par.amp.shape)) * np.exp(0.3j * rng.standard_normal(par.amp.shape))
    L_want, want = og.gradients(pr, par, target, want_V=False)
    ctx, H0 = _gpu(lib, cfg, sp)
    dev = H0.device
    nsite, nch = par.amp.shape
    amp = torch.tensor(par.amp.astype(np.complex64), device=dev, requires_grad=True)
    occ = torch.tensor(par.occ, dtype=torch.float64, device=dev, requires_grad=True)
    df = torch.tensor(cfg.defocus, dtype=torch.float64, requires_grad=True)
    cs = torch.tensor(cfg.cs, dtype=torch.float64, requires_grad=True)
    H = (amp.reshape(nsite * nch, 1, 1) * H0).contiguous()
    m = coreloss_map(ctx, H, sp.scans, occ=occ, defocus=df, cs=cs)
    loss = ((m - torch.tensor(target, device=dev)) ** 2).sum()
    loss.backward()
    assert float(loss.detach()) == pytest.approx(L_want, rel=1e-4)
    assert rel(occ.grad.cpu().numpy(), want["occ"]) < 1e-4
    assert rel(amp.grad.cpu().numpy(), want["amp"]) < 1e-4
    assert float(df.grad) == pytest.approx(want["defocus"], rel=1e-4)
    assert float(cs.grad) == pytest.approx(want["cs"], rel=1e-4)
    ctx.close()


@pytest.fixture(scope="module")
def config5_case():
    """The differentiation workload (256^2 grid, 40 slices, 64 sites, 32x32
    scans) with a seeded target, and the oracle's reverse pass on it."""
    cfg = synth.config5().replace(defocus=25.0, cs=5.0e5)
    sp = synth.make_specimen(cfg)
    pr = obip.make_problem(sp)
    rng = np.random.default_rng(55)
    par = og.Params(pr)
    I = og.forward(pr, par)
    target = I * (1.0 + 0.05 * rng.standard_normal(I.shape))
    gI = 2.0 * (I - target)
    _, want = og.gradients(pr, par, dL_dI=gI)
    return cfg, sp, gI, want


@pytest.mark.slow
@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_grad_config5(lib, config5_case, prec):
    """Occupancy, H, defocus and Cs gradients of every site against the
    oracle (mixed: the occupancy gradient is the exact reduction of the
    BF16 map's own partials)."""
    cfg, sp, gI, want = config5_case
    ctx, H = _gpu(lib, cfg, sp, prec=prec)
    got = ctx.grad(H, sp.scans, torch.tensor(gI, device=H.device))
    if prec == "fp32":
        assert rel(got["occ"].cpu().numpy(), want["occ"]) < 1e-4
    else:
        parts = ctx.sites(H, sp.scans).cpu().numpy().astype(np.float64)
        assert rel(got["occ"].cpu().numpy(), parts @ gI) < 1e-9
    wH = np.concatenate([h.reshape(len(h), cfg.win, cfg.win) for h in want["H"]])
    assert rel(got["H"].cpu().numpy(), wH) < 1e-4
    for name in ("defocus", "cs"):
        assert got[name] == pytest.approx(want[name], rel=1e-4), (name, got[name], want[name])
    ctx.close()


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
@pytest.mark.parametrize("which", ["small_magnitude", "small_complex", "config1"])
def test_grad_V_matches_oracle(lib, which, prec):
    if which == "config1":
        cfg, sp, pr, par, target = config1_case()
    else:
        cfg, sp, pr, par, target = small_case(which.split("_")[1])
    I = og.forward(pr, par)
    gI = 2.0 * (I - target)
    _, want = og.gradients(pr, par, dL_dI=gI)
    ctx, H = _gpu(lib, cfg, sp, prec=prec)
    ctx.set_occupancy(par.occ)
    V = torch.tensor(sp.V, dtype=torch.float32, device=H.device)
    got = ctx.grad(H, sp.scans, torch.tensor(gI, device=H.device), occ=False, h=False, aberr=False, V=V)
    gV = got["V"].cpu().numpy()
    assert gV.shape == want["V"].shape
    assert np.linalg.norm(want["V"]) > 0
    assert rel(gV, want["V"]) < 1e-4, rel(gV, want["V"])
    ctx.close()


def test_autograd_V(lib):
    """loss.backward() with V a leaf: the matrices are built from V inside
    the call and V.grad matches the oracle."""
    from paper_2607_00756_gb300.autograd import coreloss_map
    cfg, sp, pr, par, target = small_case()
    L_want, want = og.gradients(pr, par, target)
    dev = torch.device("cuda:0")
    ctx = lib(cfg, prec="fp32")
    V = torch.tensor(sp.V, dtype=torch.float32, device=dev, requires_grad=True)
    H = torch.tensor(sp.H, dtype=torch.complex64, device=dev)
    occ = torch.tensor(par.occ, dtype=torch.float64, device=dev)
    m = coreloss_map(ctx, H, sp.scans, occ=occ, V=V, atoms=sp.atoms, nch=sp.nch)
    loss = ((m - torch.tensor(target, device=dev)) ** 2).sum()
    loss.backward()
    assert float(loss.detach()) == pytest.approx(L_want, rel=1e-4)
    assert rel(V.grad.cpu().numpy(), want["V"]) < 1e-4
    ctx.close()


@pytest.mark.slow
@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_grad_V_config5(lib, config5_case, prec):
    """The slice-potential derivative on the differentiation workload: 40
    slices, sites at planes 8..32, so both sweeps run through several
    checkpoint segments."""
    cfg, sp, gI, want = config5_case
    ctx, H = _gpu(lib, cfg, sp, prec=prec)
    V = torch.tensor(sp.V, dtype=torch.float32, device=H.device)
    got = ctx.grad(H, sp.scans, torch.tensor(gI, device=H.device), occ=False, h=False, aberr=False, V=V)
    assert rel(got["V"].cpu().numpy(), want["V"]) < 1e-4
    ctx.close()
