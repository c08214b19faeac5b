"""Batched evaluation under a CUDA graph and the launch autotuner.

Specimens of uneven size -- grids 64x128 to 256^2, 4 to 12 slices, f = 1, 2
and 4, one, three and nine channels, FP32, mixed and FP8 contexts -- are
captured into one CUDA graph; every replay must reproduce the eager maps
bit for bit, and each map matches the oracle within its precision's
tolerance.  The autotuner must return valid choices whose map equals the
built-in choice's (the site arithmetic and the site-sum order do not depend
on the launch shape)."""
import numpy as np
import pytest

import synth
from oracle import bip as obip

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2607_00756_gb300 import build
    build.build()
    from paper_2607_00756_gb300.context import BipContext
    return BipContext


def specimens():
    c1 = synth.config1()
    return [
        (c1, "mixed", 1e-3),
        (c1.replace(name="nine", seed=3, channels=tuple(range(-4, 5))), "fp32", 1e-4),
        (synth.config1().replace(name="aniso", ny=64, nx=128, ly=7.5, lx=10.0, cells_y=3, cells_x=4, fy=1, fx=2,
                                 win=32, ion_cells=(1, 3), ion_slices=(1, 4), channels=(0,),
                                 scan_y=(10.3, 3.5, 9), scan_x=(20.7, 6.25, 7)), "mixed", 1e-3),
        (synth.config1().replace(name="wide", ny=256, nx=256, ly=20.0, lx=20.0, nz=12, cells_y=8, cells_x=8,
                                 fy=4, fx=4, ion_cells=(3, 5), ion_slices=(3, 12, 4), seed=7,
                                 scan_y=(100.0, 4.0, 12), scan_x=(100.0, 4.0, 12)), "fp8", None),
    ]


def test_graph_replay_matches_eager_and_oracle(lib):
    from paper_2607_00756_gb300.graphs import GraphedMaps
    dev = torch.device("cuda:0")
    items, eager, refs, tols = [], [], [], []
    for cfg, prec, tol in specimens():
        sp = synth.make_specimen(cfg)
        ctx = lib(cfg, prec=prec)
        ctx.build(torch.tensor(sp.V, dtype=torch.float32, device=dev), sp.atoms, sp.nch)
        H = torch.tensor(sp.H, dtype=torch.complex64, device=dev)
        eager.append(ctx.map(H, sp.scans).cpu().numpy())
        items.append((ctx, H, sp.scans))
        refs.append(obip.bip_map(obip.make_problem(sp)).map)
        tols.append(tol)
    for conc in (False, True):
        g = GraphedMaps(items, concurrent=conc)
        for _ in range(3):
            outs = g.replay()
            torch.cuda.synchronize()
            g.check()
            for o, e in zip(outs, eager):
                assert np.array_equal(o.cpu().numpy(), e), conc
    for e, r, tol in zip(eager, refs, tols):
        # the FP8 context: within 3% (its E4M3 rounding), the others their bars
        assert rel(e, r) < (tol if tol is not None else 3e-2)


@pytest.mark.parametrize("prec", ["mixed", "fp32"])
def test_autotune_keeps_the_map(lib, prec):
    cfg = synth.config1()
    sp = synth.make_specimen(cfg)
    dev = torch.device("cuda:0")
    ctx = lib(cfg, prec=prec)
    ctx.build(torch.tensor(sp.V, dtype=torch.float32, device=dev), sp.atoms, sp.nch)
    H = torch.tensor(sp.H, dtype=torch.complex64, device=dev)
    m0 = ctx.map(H, sp.scans).cpu().numpy()
    sb, cw, order, ms = ctx.autotune(H, sp.scans)
    assert 1 <= sb <= 32 and (cw == 0 or (cw % 16 == 0 and cw <= 256)) and ms > 0.0
    assert order in (0, 1, 2) and (prec != "fp32" or order == 0) and (prec == "mixed" or order != 2)
    m1 = ctx.map(H, sp.scans).cpu().numpy()
    # the Gram route repeats the map exactly; the beam and probe orders
    # (another summation) within the mixed path's bar
    assert rel(m1, m0) < (1e-6 if order == 0 else 1e-3)
    ctx.set_order(0)
    # any explicit choice gives the same map too
    ctx.set_launch(1, 128 if prec != "fp32" else 0)
    assert rel(ctx.map(H, sp.scans).cpu().numpy(), m0) < 1e-6
    ctx.close()



def _order_case(which):
    """Workloads of the contraction-order tests: config 1; the edge-case
    specimen (every plane, wrapping windows, 21 sites with one or three
    channels, a ragged scan line); an anisotropic grid; config 1 with six
    channels per site (two passes of the cube kernel's four accumulators),
    with all its scans or with 40 of them."""
    if which == "edge":
        from test_gpu_map import _edge_specimen
        return _edge_specimen()
    if which == "aniso":
        cfg = synth.config1().replace(name="aniso", ny=64, nx=128, ly=7.5, lx=10.0, cells_y=3, cells_x=4, fy=1,
                                      fx=2, win=32, ion_cells=(1, 3), ion_slices=(1, 4),
                                      scan_y=(10.3, 3.5, 9), scan_x=(20.7, 6.25, 7))
        return cfg, synth.make_specimen(cfg)
    cfg = synth.config1()
    sp = synth.make_specimen(cfg)
    if which.startswith("six_channels"):
        keep = np.nonzero(sp.nch > 0)[0]
        h3 = sp.H.reshape(len(keep), 3, cfg.win, cfg.win)
        h6 = np.concatenate([h3, 0.5j * h3[:, ::-1]], axis=1).reshape(-1, cfg.win, cfg.win)
        nch = sp.nch.copy()
        nch[keep] = 6
        # few scans: the probe order then puts (scan, channel) pairs in the
        # cube kernel's columns instead of one accumulator per channel
        scans = sp.scans[100:140] if which.endswith("few_scans") else sp.scans
        sp = synth.Specimen(cfg=cfg, atoms=sp.atoms, nch=nch, V=sp.V, H=h6, scans=scans)
    return cfg, sp


def _order_check(lib, which, prec, order):
    cfg, sp = _order_case(which)
    ref = obip.bip_map(obip.make_problem(sp))
    dev = torch.device("cuda:0")
    ctx = lib(cfg, prec=prec)
    ctx.build(torch.tensor(sp.V, dtype=torch.float32, device=dev), sp.atoms, sp.nch)
    H = torch.tensor(sp.H, dtype=torch.complex64, device=dev)
    m_gram = ctx.map(H, sp.scans).cpu().numpy()
    ctx.set_order(order)
    m = ctx.map(H, sp.scans).cpu().numpy()
    parts = ctx.sites(H, sp.scans).cpu().numpy()
    assert rel(m, ref.map) < 1e-3
    assert rel(parts, ref.partials) < 1e-3
    assert rel(m, m_gram) < 1e-3
    pr = obip.make_problem(sp)
    for k in range(len(pr.ion)):
        assert np.all(parts[k][~obip.crop_mask(pr, k, sp.scans)] == 0.0)
    # fixed summation order (no atomics): a second map is bit-identical
    assert np.array_equal(ctx.map(H, sp.scans).cpu().numpy(), m)
    ctx.close()


@pytest.mark.parametrize("which", ["config1", "edge", "aniso"])
@pytest.mark.parametrize("prec", ["mixed", "split_bf16"])
def test_beam_order_map(lib, which, prec):
    """The map in beam order (|M c|^2 per detector beam on tcgen05, the
    detector sum in the epilogue) against the oracle and the Gram route."""
    _order_check(lib, which, prec, 1)


@pytest.mark.parametrize("which", ["config1", "edge", "aniso", "six_channels", "six_channels_few_scans"])
def test_probe_order_map(lib, which):
    """The map in probe order (the windowed probes Psi = C^T S1 of every
    scan, then |S2^T (H_n x Psi)|^2 summed over d and n on tcgen05) against
    the oracle and the Gram route, mixed precision.  The edge case (101
    scans, three channels) and the six-channel case with 40 scans take the
    (scan, channel)-column form of the last contraction; the others one
    accumulator per channel."""
    _order_check(lib, which, "mixed", 2)


def test_probe_order_limits(lib):
    """The probe order is refused outside its domain, before any launch:
    other precisions at set time, more than 2048 scans at map time."""
    from paper_2607_00756_gb300.capi import BipError
    cfg = synth.config1()
    sp = synth.make_specimen(cfg)
    dev = torch.device("cuda:0")
    ctx = lib(cfg, prec="split_bf16")
    with pytest.raises(BipError):
        ctx.set_order(2)
    ctx.close()
    ctx = lib(cfg, prec="mixed")
    ctx.build(torch.tensor(sp.V, dtype=torch.float32, device=dev), sp.atoms, sp.nch)
    H = torch.tensor(sp.H, dtype=torch.complex64, device=dev)
    ctx.set_order(2)
    scans = np.tile(sp.scans, (2049 // len(sp.scans) + 1, 1))[:2049]
    with pytest.raises(BipError):
        ctx.map(H, scans)
    ctx.set_order(0)
    m = ctx.map(H, scans).cpu().numpy()
    assert np.all(np.isfinite(m))
    ctx.close()
