"""Sites with windows of their own (Eq. coupling summed over each site's
crop window Omega_tau, the window following the support of its H_n: sites
of several edges batched in one map).  Maps of config 1 and of a 12-site
mix with windows from 16 to 64 pixels against the FP64 oracle in every
precision; the same map as the context's windows with H zero outside each
site's block; the windows cleared again giving the uniform map back bit
for bit; the beam and probe orders and qEELS on such sites; and the paths
that take only the context's window refusing; the cube and the reverse
pass on such sites."""
import numpy as np
import pytest

import synth
from oracle import bip as obip

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = {"fp32": 1e-4, "split_bf16": 1e-4, "mixed": 1e-3, "fp8": 3e-2}


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


def case(kind):
    """(config, specimen, per-site windows): config 1's four sites, or
    twelve sites on three slices with windows 64, 48, 32, 16 in turn."""
    if kind == "config1":
        cfg = synth.config1()
        sp = synth.make_specimen(cfg)
        return cfg, sp, [32, 64, 16, 48]
    cfg = synth.config1().replace(name="mix", ion_slices=(1, 4), seed=5)
    sp = synth.make_specimen(cfg)
    n = int((sp.nch > 0).sum())
    return cfg, sp, [(64, 48, 32, 16)[k % 4] for k in range(n)]


_refs = {}


def oracle_own(kind):
    if kind not in _refs:
        cfg, sp, w = case(kind)
        parts, _, _ = synth.site_window_inputs(sp, w)
        _refs[kind] = obip.bip_map(obip.make_problem(sp, site_win=w, H=parts))
    return _refs[kind]


def built(lib, cfg, sp, prec):
    dev = torch.device("cuda:0")
    ctx = lib(cfg, prec=prec)
    ctx.build(torch.tensor(sp.V, dtype=torch.float32, device=dev), sp.atoms, sp.nch)
    return ctx


@pytest.mark.parametrize("kind", ["config1", "mix"])
@pytest.mark.parametrize("prec", ["fp32", "split_bf16", "mixed", "fp8"])
def test_own_windows_map(lib, kind, prec):
    cfg, sp, w = case(kind)
    ref = oracle_own(kind)
    _, flat, _ = synth.site_window_inputs(sp, w)
    ctx = built(lib, cfg, sp, prec)
    ctx.set_site_windows(w)
    H = torch.tensor(flat, dtype=torch.complex64, device="cuda:0")
    m = ctx.map(H, sp.scans).cpu().numpy()
    assert rel(m, ref.map) < TOL[prec]
    parts = ctx.sites(H, sp.scans).cpu().numpy()
    assert rel(parts, ref.partials) < TOL[prec]
    # smaller batches (never across a window size) give the same map
    ctx.set_launch(2, 0)
    m2 = ctx.map(H, sp.scans).cpu().numpy()
    assert rel(m2, m) < (1e-6 if prec in ("fp32", "split_bf16") else TOL[prec])
    # a second map is bit-identical (fixed order, no atomics)
    assert np.array_equal(ctx.map(H, sp.scans).cpu().numpy(), m2)
    ctx.close()


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_own_windows_equal_zero_padded_context_windows(lib, prec):
    """Own windows against the context's windows with H_n zero outside each
    site's block (the same sum, Eq. coupling), then the windows cleared."""
    cfg, sp, w = case("mix")
    _, flat, padded = synth.site_window_inputs(sp, w)
    dev = torch.device("cuda:0")
    ctx = built(lib, cfg, sp, prec)
    H_full = torch.tensor(sp.H, dtype=torch.complex64, device=dev)
    m_full = ctx.map(H_full, sp.scans).cpu().numpy()
    m_pad = ctx.map(torch.tensor(padded, dtype=torch.complex64, device=dev), sp.scans).cpu().numpy()
    ctx.set_site_windows(w)
    m_own = ctx.map(torch.tensor(flat, dtype=torch.complex64, device=dev), sp.scans).cpu().numpy()
    assert rel(m_own, m_pad) < (1e-5 if prec == "fp32" else 1e-3)
    assert rel(m_own, m_full) > 1e-4          # the windows do change the map
    ctx.set_site_windows(None)
    assert np.array_equal(ctx.map(H_full, sp.scans).cpu().numpy(), m_full)
    # windows equal to the context's are the uniform case
    ctx.set_site_windows([cfg.win] * len(w))
    assert np.array_equal(ctx.map(H_full, sp.scans).cpu().numpy(), m_full)
    ctx.close()


def test_own_windows_autotune_keeps_the_map(lib):
    cfg, sp, w = case("mix")
    _, flat, _ = synth.site_window_inputs(sp, w)
    ctx = built(lib, cfg, sp, "mixed")
    ctx.set_site_windows(w)
    H = torch.tensor(flat, dtype=torch.complex64, device="cuda:0")
    m0 = ctx.map(H, sp.scans).cpu().numpy()
    sb, cw, order, ms = ctx.autotune(H, sp.scans)
    assert order in (0, 1, 2) and ms > 0.0
    # the Gram order repeats the map exactly; the others within the mixed bar
    assert rel(ctx.map(H, sp.scans).cpu().numpy(), m0) < (1e-6 if order == 0 else 1e-3)
    ctx.close()


def test_own_windows_refusals(lib):
    from paper_2607_00756_gb300.capi import BipError
    cfg, sp, w = case("config1")
    _, flat, _ = synth.site_window_inputs(sp, w)
    dev = torch.device("cuda:0")
    V = torch.tensor(sp.V, dtype=torch.float32, device=dev)
    ctx = built(lib, cfg, sp, "mixed")
    for bad in ([17, 64, 16, 48], [32, 80, 16, 48], [32, 64, 0, -16]):
        with pytest.raises(BipError):
            ctx.set_site_windows(bad)
    ctx.set_site_windows(w)
    H = torch.tensor(flat, dtype=torch.complex64, device=dev)
    with pytest.raises(BipError):
        ctx.windows(0)
    assert np.all(np.isfinite(ctx.map(H, sp.scans).cpu().numpy()))
    ctx.close()


@pytest.mark.parametrize("order", [1, 2])
def test_own_windows_beam_and_probe_orders(lib, order):
    """The beam order (|M c|^2 per detector beam) and the probe order
    (S2^T (H_n x S1 c)) on sites with their own windows: batches of one
    window size each, against the oracle and the Gram order."""
    cfg, sp, w = case("mix")
    ref = oracle_own("mix")
    _, flat, _ = synth.site_window_inputs(sp, w)
    ctx = built(lib, cfg, sp, "mixed")
    ctx.set_site_windows(w)
    H = torch.tensor(flat, dtype=torch.complex64, device="cuda:0")
    m_gram = ctx.map(H, sp.scans).cpu().numpy()
    ctx.set_order(order)
    m = ctx.map(H, sp.scans).cpu().numpy()
    assert rel(m, ref.map) < 1e-3
    assert rel(m, m_gram) < 1e-3
    assert rel(ctx.sites(H, sp.scans).cpu().numpy(), ref.partials) < 1e-3
    assert np.array_equal(ctx.map(H, sp.scans).cpu().numpy(), m)
    ctx.close()


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_own_windows_qeels(lib, prec):
    """qEELS (resolved axis at f = 1) with the sites' own windows against the
    oracle's; the bins summed give the map."""
    cfg0, sp0, w = case("mix")
    cfg = cfg0.replace(dfx=1)
    sp = synth.make_specimen(cfg)
    parts, flat, _ = synth.site_window_inputs(sp, w)
    pr = obip.make_problem(sp, site_win=w, H=parts)
    hb_want, want = obip.bip_qeels(pr, 1)
    ctx = built(lib, cfg, sp, prec)
    ctx.set_site_windows(w)
    H = torch.tensor(flat, dtype=torch.complex64, device="cuda:0")
    hb, q = ctx.qeels(H, sp.scans, 1)
    assert np.array_equal(hb, hb_want)
    q = q.cpu().numpy()
    tol = 1e-4 if prec == "fp32" else 1e-3
    assert rel(q, want) < tol
    assert rel(q.astype(np.float64).sum(axis=1), ctx.map(H, sp.scans).cpu().numpy()) < tol
    ctx.close()


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-4), ("mixed", 1e-3)])
@pytest.mark.parametrize("order", ["raster", "shuffled"])
def test_own_windows_cube(lib, prec, tol, order):
    """The exact cube (Algorithm 3) with the sites' own windows: S1's side
    rebuilt and the exact S2 windows re-tilted on each site's block, the
    batches of one window size each -- on the raster scans (the separated
    per-beam contraction) and shuffled (the per-scan one) -- against the
    oracle's cube with the same windows."""
    cfg, sp, w = case("config1")
    parts, flat, _ = synth.site_window_inputs(sp, w)
    pr = obip.make_problem(sp, site_win=w, H=parts)
    want = obip.bip_cube(pr)
    scans = sp.scans
    if order == "shuffled":
        perm = np.random.default_rng(4).permutation(len(scans))
        scans, want = scans[perm], want[perm]
    dev = torch.device("cuda:0")
    V = torch.tensor(sp.V, dtype=torch.float32, device=dev)
    ctx = built(lib, cfg, sp, prec)
    ctx.set_site_windows(w)
    H = torch.tensor(flat, dtype=torch.complex64, device=dev)
    cube = ctx.cube(V, H, scans).cpu().numpy()
    assert cube.shape == want.shape
    assert rel(cube, want) < tol
    ctx.close()


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_own_windows_reverse_pass(lib, prec):
    """The reverse pass on sites with their own windows (config 1, windows
    32, 64, 16, 48): dL/dV through the reconstruction adjoint of each site's
    block and both adjoint sweeps, dL/dH on each site's window, against the
    oracle's reverse pass (pinned by central differences), 1e-4."""
    from oracle import grad as og
    cfg, sp, w = case("config1")
    parts, flat, _ = synth.site_window_inputs(sp, w)
    pr = obip.make_problem(sp, site_win=w, H=parts)
    rng = np.random.default_rng(8)
    par = og.Params(pr)
    par.occ = 1.0 + 0.3 * rng.standard_normal(len(pr.ion))
    I0 = og.forward(pr, par)
    gI = 2.0 * (I0 - I0 * (1.0 + 0.1 * rng.standard_normal(I0.shape)))
    _, want = og.gradients(pr, par, dL_dI=gI)
    dev = torch.device("cuda:0")
    V = torch.tensor(sp.V, dtype=torch.float32, device=dev)
    ctx = built(lib, cfg, sp, prec)
    ctx.set_site_windows(w)
    ctx.set_occupancy(par.occ)
    H = torch.tensor(flat, dtype=torch.complex64, device=dev)
    got = ctx.grad(H, sp.scans, torch.tensor(gI, device=dev), occ=False, aberr=False, V=V)
    assert rel(got["V"].cpu().numpy(), want["V"]) < 1e-4
    wH = np.concatenate([h.reshape(-1) for h in want["H"]])
    assert rel(got["H"].cpu().numpy(), wH) < 1e-4
    ctx.close()


def test_own_windows_under_a_graph(lib):
    """A context whose sites have their own windows inside a CUDA graph of
    several specimens (one stream each): every replay equals the eager maps
    bit for bit, and the windows' map matches the oracle."""
    from paper_2607_00756_gb300.graphs import GraphedMaps
    dev = torch.device("cuda:0")
    cfg, sp, w = case("mix")
    _, flat, _ = synth.site_window_inputs(sp, w)
    a = built(lib, cfg, sp, "mixed")
    a.set_site_windows(w)
    Ha = torch.tensor(flat, dtype=torch.complex64, device=dev)
    cfg1, sp1, _ = case("config1")
    b = built(lib, cfg1, sp1, "fp32")
    Hb = torch.tensor(sp1.H, dtype=torch.complex64, device=dev)
    eager = [a.map(Ha, sp.scans).cpu().numpy(), b.map(Hb, sp1.scans).cpu().numpy()]
    g = GraphedMaps([(a, Ha, sp.scans), (b, Hb, sp1.scans)], concurrent=True)
    for _ in range(3):
        outs = g.replay()
        torch.cuda.synchronize()
        g.check()
        for o, e in zip(outs, eager):
            assert np.array_equal(o.cpu().numpy(), e)
    assert rel(eager[0], oracle_own("mix").map) < 1e-3
    a.close()
    b.close()


def test_own_windows_on_a_3m_grid(lib):
    """Own windows on a 192^2 grid at f = 3 (the radix-3 multislice and the
    modular table indices), FP32 and mixed, against the oracle."""
    cfg = synth.config1().replace(name="f3win", ny=192, nx=192, ly=15.0, lx=15.0, cells_y=6, cells_x=6, fy=3,
                                  fx=3, ion_cells=(2, 4), ion_slices=(2, 3), scan_y=(90.5, 3.0, 7),
                                  scan_x=(91.75, 3.5, 6))
    sp = synth.make_specimen(cfg)
    w = [48, 64, 32, 16]
    parts, flat, _ = synth.site_window_inputs(sp, w)
    ref = obip.bip_map(obip.make_problem(sp, site_win=w, H=parts))
    for prec, tol in (("fp32", 1e-4), ("mixed", 1e-3)):
        ctx = built(lib, cfg, sp, prec)
        ctx.set_site_windows(w)
        H = torch.tensor(flat, dtype=torch.complex64, device="cuda:0")
        assert rel(ctx.map(H, sp.scans).cpu().numpy(), ref.map) < tol
        ctx.close()


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-4), ("mixed", 1e-3), ("split_bf16", 1e-4)])
def test_two_edges_in_one_map(lib, prec, tol):
    """Two edges in one specimen: alternate sites keep nine channels
    (m = -4..4) on the 64-px window, the others one channel (m = 0) on a
    32-px window of their own -- uneven channel counts and windows in the
    same batches -- against the oracle."""
    cfg = synth.config1().replace(name="two_edges", channels=tuple(range(-4, 5)))
    sp = synth.make_specimen(cfg)
    ion = np.nonzero(sp.nch > 0)[0]
    nch = sp.nch.copy()
    parts, w = [], []
    for k, a in enumerate(ion.tolist()):
        h = sp.H[9 * k:9 * (k + 1)]
        if k % 2:
            nch[a] = 1
            parts.append(h[4:5, 16:48, 16:48].copy())
            w.append(32)
        else:
            parts.append(h.copy())
            w.append(64)
    sp2 = synth.Specimen(cfg=cfg, atoms=sp.atoms, nch=nch, V=sp.V, H=sp.H, scans=sp.scans)
    ref = obip.bip_map(obip.make_problem(sp2, site_win=w, H=parts))
    ctx = built(lib, cfg, sp2, prec)
    ctx.set_site_windows(w)
    H = torch.tensor(np.concatenate([p.reshape(-1) for p in parts]), dtype=torch.complex64, device="cuda:0")
    assert rel(ctx.map(H, sp.scans).cpu().numpy(), ref.map) < tol
    assert rel(ctx.sites(H, sp.scans).cpu().numpy(), ref.partials) < tol
    ctx.close()
