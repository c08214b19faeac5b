"""Parity at the full paper-like size (512x512 grid, 100 slices, 1600
ionized sites x 3 channels, 128x128 scans), in the launch configuration the
benchmark times: every site built and mapped through the C ABI in one
context.  The FP64 oracle cannot run every site, so it evaluates sampled
sites -- one in the first slice, one in the middle and one in the last, so
the S1 and S2 sweeps are checked over their whole depth -- on every 8th scan
of each axis (16x16 probes).  Properties that hold at any size are checked
on the whole output: the map is the FP64 sum of the per-site
contributions, each contribution is zero outside its crop mask, and the
mixed-precision map lies within 1e-3 relative L2 of the FP32 map (the FP8
map within 3%).
Tolerances: rel L2 <= 1e-4 for FP32, <= 1e-3 for the mixed path."""
import numpy as np
import pytest

import synth
from oracle import bip as obip
from synth.specimen import scan_raster

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module")
def full():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2607_00756_gb300 import build
    build.build()
    from paper_2607_00756_gb300.context import BipContext
    cfg = synth.config2()
    sp = synth.make_specimen(cfg)
    dev = torch.device("cuda:0")
    V = torch.tensor(sp.V, dtype=torch.float32, device=dev)
    H = torch.tensor(sp.H, dtype=torch.complex64, device=dev)
    out = {}
    for prec in ("mixed", "fp8", "fp32"):
        ctx = BipContext(cfg, prec=prec)
        ctx.build(V, sp.atoms, sp.nch)
        m = ctx.map(H, sp.scans).cpu().numpy()
        parts = ctx.sites(H, sp.scans).cpu().numpy()
        ctx.close()
        out[prec] = (m, parts)
    torch.cuda.synchronize()
    return cfg, sp, out


def _sampled_sites(sp):
    ion = sp.ionized
    planes = sp.atoms[ion, 2].astype(int)
    pick = []
    for target in (planes.min(), (planes.min() + planes.max()) // 2, planes.max()):
        cand = ion[planes == target]
        pick.append(int(cand[len(cand) // 2]))
    return sorted(pick)


@pytest.fixture(scope="module")
def oracle_sample(full):
    """The oracle on the sampled sites (the others switched off) and the
    16x16 oracle scans, which are a subset of the full 128x128 raster."""
    cfg, sp, _ = full
    pick = _sampled_sites(sp)
    ion = list(sp.ionized)
    per = len(cfg.channels)
    nch = np.zeros_like(sp.nch)
    nch[pick] = sp.nch[pick]
    H = np.concatenate([sp.H[ion.index(a) * per:(ion.index(a) + 1) * per] for a in pick])
    sub = synth.Specimen(cfg=cfg, atoms=sp.atoms, nch=nch, V=sp.V, H=H, scans=sp.scans)
    oscans = scan_raster(cfg.oracle_scan_y, cfg.oracle_scan_x)
    # positions of the oracle scans in the full raster
    key = {(float(y), float(x)): i for i, (y, x) in enumerate(sp.scans)}
    idx = np.array([key[(float(y), float(x))] for y, x in oscans])
    ref = obip.bip_map(obip.make_problem(sub), scans=oscans)
    rows = [ion.index(a) for a in pick]
    return pick, rows, idx, ref


@pytest.mark.parametrize("prec,tol", [("mixed", 1e-3), ("fp32", 1e-4)])
def test_fullsize_sampled_sites_match_oracle(full, oracle_sample, prec, tol):
    cfg, sp, out = full
    pick, rows, idx, ref = oracle_sample
    _, parts = out[prec]
    planes = sp.atoms[pick, 2].astype(int)
    assert planes.min() == 0 and planes.max() == cfg.nz - 1
    for j, r in enumerate(rows):
        got = parts[r, idx]
        want = ref.partials[j]
        assert np.linalg.norm(want) > 0
        assert rel(got, want) < tol, (prec, pick[j], rel(got, want))


def test_fullsize_map_is_the_site_sum(full):
    """Any size: the map is the FP64 sum of the per-site contributions."""
    _, _, out = full
    for prec in ("mixed", "fp8", "fp32"):
        m, parts = out[prec]
        want = parts.astype(np.float64).sum(axis=0)
        assert np.max(np.abs(m - want)) <= 1e-9 * np.max(np.abs(want)), prec


def test_fullsize_zero_outside_crop(full):
    """Any size: each contribution vanishes outside its site's crop mask."""
    cfg, sp, out = full
    pr = obip.make_problem(synth.Specimen(cfg=cfg, atoms=sp.atoms, nch=sp.nch, V=None, H=sp.H, scans=sp.scans))
    rng = np.random.default_rng(7)
    for k in rng.choice(len(sp.ionized), size=16, replace=False):
        outside = ~obip.crop_mask(pr, k, sp.scans)
        for prec in ("mixed", "fp8", "fp32"):
            assert np.all(out[prec][1][k][outside] == 0.0)


def test_fullsize_mixed_within_1e3_of_fp32(full):
    """The benchmark's accuracy condition: the mixed map within 1e-3
    relative L2 of the FP32 map on the whole 128x128 raster."""
    _, _, out = full
    assert rel(out["mixed"][0], out["fp32"][0]) < 1e-3


def test_fullsize_fp8_near_fp32(full):
    """The FP8 coupling's map on the whole raster: within 3% relative L2 of
    the FP32 map (about four times the E4M3 model's 0.7% at config 1; the
    figure is reported by the benchmark), and not equal to it."""
    _, _, out = full
    e = rel(out["fp8"][0], out["fp32"][0])
    assert 1e-5 < e < 3e-2, e
