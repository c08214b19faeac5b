"""A reduced form of the batched workload (specimens of uneven size under
one CUDA graph, autotuned launches): four specimens -- 192^2 and 384^2 at
f = 3, 256^2 at f = 2, 512^2 at f = 4 -- with 20 to 30 slices, one, three
or nine transition channels and 24 to 48 ionized sites each.  Every map is
computed under one graph with a stream per specimen after each context was
autotuned; sampled sites' contributions are checked against the FP64
oracle, the maps against the FP64 sums of the contributions, and one
specimen's cube on a box of k-pixels against the oracle's."""
import numpy as np
import pytest

import synth
from oracle import bip as obip

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def mix():
    """(config, precision) of the four specimens (300 keV, 25 mrad, 40 mrad
    detector, 0.078 A pixels, 64-px windows)."""
    base = synth.config2().replace(oracle_scan_y=None, oracle_scan_x=None)
    out = []
    for name, n, f, nz, ch, cells, prec in (("c4a", 192, 3, 20, (-1, 0, 1), (1, 4), "mixed"),
                                            ("c4b", 256, 2, 24, (0,), (2, 5), "fp32"),
                                            ("c4c", 384, 3, 30, tuple(range(-4, 5)), (4, 7), "mixed"),
                                            ("c4d", 512, 4, 24, (-1, 0, 1), (6, 9), "split_bf16")):
        cells_n = n // 32
        mid = (cells[0] + 1.5) * 32.0
        out.append((base.replace(name=name, ny=n, nx=n, ly=n / 12.8, lx=n / 12.8, cells_y=cells_n, cells_x=cells_n,
                                 nz=nz, fy=f, fx=f, nrad1=2, nrad2=2, channels=ch, ion_cells=cells,
                                 ion_slices=(nz // 4, nz, nz // 4), seed=len(out) + 11,
                                 scan_y=(mid - 14.5, 3.0, 10), scan_x=(mid - 13.25, 3.0, 10)), prec))
    return out


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2607_00756_gb300 import build
    build.build()
    from paper_2607_00756_gb300.context import BipContext
    return BipContext


def test_config4_mix_under_one_graph(lib):
    from paper_2607_00756_gb300.graphs import GraphedMaps
    dev = torch.device("cuda:0")
    items, specs, parts = [], [], []
    for cfg, prec in mix():
        sp = synth.make_specimen(cfg)
        n_sites = int((sp.nch > 0).sum())
        assert 27 <= n_sites <= 36
        ctx = lib(cfg, prec=prec)
        ctx.build(torch.tensor(sp.V, dtype=torch.float32, device=dev), sp.atoms, sp.nch)
        H = torch.tensor(sp.H, dtype=torch.complex64, device=dev)
        ctx.autotune(H, sp.scans)
        parts.append(ctx.sites(H, sp.scans).cpu().numpy())
        items.append((ctx, H, sp.scans))
        specs.append((cfg, sp, prec))
    g = GraphedMaps(items, concurrent=True)
    outs = [o.cpu().numpy() for o in g.replay()]
    torch.cuda.synchronize()
    g.check()
    for (cfg, sp, prec), m, pt in zip(specs, outs, parts):
        # the map is the FP64 sum of the contributions
        assert rel(m, pt.astype(np.float64).sum(axis=0)) < 1e-6, cfg.name
        # sampled sites against the oracle: the first, a middle and the last
        pr = obip.make_problem(sp)
        k = [0, len(pr.ion) // 2, len(pr.ion) - 1]
        want = obip.bip_map(pr, sites=k).partials
        tol = 1e-4 if prec == "fp32" else 1e-3
        assert rel(pt[k], want) < tol, (cfg.name, rel(pt[k], want))
    for ctx, _, _ in items:
        ctx.close()


def test_config4_cube_on_a_box(lib):
    """The 192^2 f = 3 specimen's cube on a 24 x 24 box of k-pixels (the
    batched workload's pixelated detector, reduced), first six sites."""
    cfg, prec = mix()[0]
    cfg = cfg.replace(cube_ky=24, cube_kx=24)
    sp = synth.make_specimen(cfg)
    ion = np.nonzero(sp.nch > 0)[0]
    nch = np.zeros_like(sp.nch)
    nch[ion[:6]] = sp.nch[ion[:6]]
    sp = synth.Specimen(cfg=cfg, atoms=sp.atoms, nch=nch, V=sp.V, H=sp.H[:6 * len(cfg.channels)], scans=sp.scans)
    dev = torch.device("cuda:0")
    V = torch.tensor(sp.V, dtype=torch.float32, device=dev)
    ctx = lib(cfg, prec=prec)
    try:
        ctx.build_s1(V, sp.atoms, sp.nch)
        cube = ctx.cube(V, torch.tensor(sp.H, dtype=torch.complex64, device=dev), sp.scans).cpu().numpy()
        assert cube.shape == (len(sp.scans), 576)
        assert rel(cube, obip.bip_cube(obip.make_problem(sp))) < 1e-3
    finally:
        ctx.close()
