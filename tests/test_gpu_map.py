"""GPU parity of the CUDA path against the FP64 oracle, stage by stage and
end to end, through the C ABI.  Tolerances: rel L2 <= 1e-4 for the FP32
path (and for the stashed / reconstructed windows, 2e-5 max-relative), the
figures fixed for this method's FP32 maps."""
import numpy as np
import pytest

import synth
from oracle import bip as obip

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


def gpu_run(BipContext, cfg, sp, prec="fp32", recon=None, scans=None):
    dev = torch.device("cuda:0")
    V = torch.tensor(sp.V, dtype=torch.float32, device=dev)
    H = torch.tensor(sp.H, dtype=torch.complex64, device=dev)
    ctx = BipContext(cfg, prec=prec, recon=recon)
    ctx.build(V, sp.atoms, sp.nch)
    scans = sp.scans if scans is None else scans
    m = ctx.map(H, scans).cpu().numpy()
    parts = ctx.sites(H, scans).cpu().numpy()
    torch.cuda.synchronize()
    return ctx, m, parts, H


@pytest.fixture(scope="module")
def c1(lib):
    cfg = synth.config1()
    sp = synth.make_specimen(cfg)
    pr = obip.make_problem(sp)
    ref = obip.bip_map(pr, keep_stages=True)
    return cfg, sp, pr, ref


def test_stash_parity(lib, c1):
    """Stashed de-tilted parent windows of S1 and S2 (Eq. smatrix-advance,
    Eq. s2, Eq. part-basis) against the oracle, every site."""
    cfg, sp, pr, ref = c1
    ctx, *_ = gpu_run(lib, cfg, sp)
    for k in range(len(pr.ion)):
        for which, key in ((1, "stash1"), (2, "stash2")):
            got = ctx.stash(which, k).cpu().numpy()
            want = ref.stages[k][key]
            assert got.shape == want.shape
            assert np.max(np.abs(got - want)) < 2e-5 * np.max(np.abs(want)), (k, which)


@pytest.mark.parametrize("recon", ["magnitude", "complex"])
def test_window_reconstruction_parity(lib, c1, recon):
    """Reconstructed windows S1^b and S2^d (Eq. window-recon, magpreserve)."""
    cfg, sp, pr, ref = c1
    cref = ref if recon == "magnitude" else obip.bip_map(pr, mode="complex", keep_stages=True)
    ctx, *_ = gpu_run(lib, cfg, sp, recon=recon)
    for k in range(len(pr.ion)):
        s1, s2 = ctx.windows(k)
        s1, s2 = s1.cpu().numpy(), s2.cpu().numpy()
        w1, w2 = cref.stages[k]["S1w"], cref.stages[k]["S2w"]
        assert np.max(np.abs(s1 - w1)) < 2e-5 * np.max(np.abs(w1))
        assert np.max(np.abs(s2 - w2)) < 2e-5 * np.max(np.abs(w2))


def test_map_fp32_config1(lib, c1):
    """The FP32 map and its per-site contributions (Algorithm 5)."""
    cfg, sp, pr, ref = c1
    _, m, parts, _ = gpu_run(lib, cfg, sp)
    assert rel(m, ref.map) < 1e-4
    for k in range(len(pr.ion)):
        assert rel(parts[k], ref.partials[k]) < 1e-4
    # zero outside the crop mask, exactly
    for k in range(len(pr.ion)):
        outside = ~obip.crop_mask(pr, k, pr.scans)
        assert np.all(parts[k][outside] == 0.0)


def test_map_complex_mode(lib, c1):
    cfg, sp, pr, ref = c1
    want = obip.bip_map(pr, mode="complex").map
    _, m, _, _ = gpu_run(lib, cfg, sp, recon="complex")
    assert rel(m, want) < 1e-4


def _edge_specimen():
    """Sites in every plane (first and last included), windows that wrap
    around the grid, 21 sites (not a multiple of the site batch), one or
    three channels per site, and a ragged scan list that wraps the cell."""
    cfg = synth.config1().replace(name="edge", ion_slices=(0, 5), ion_cells=(0, 4))
    sp = synth.make_specimen(cfg)
    keep = np.nonzero(sp.nch > 0)[0]
    rng = np.random.default_rng(5)
    pick = np.sort(rng.choice(keep, size=21, replace=False))
    nch = np.zeros_like(sp.nch)
    nch[pick] = 3
    nch[pick[::4]] = 1
    # H rows for the chosen sites in order; one-channel sites keep m = 0
    H_all = sp.H.reshape(len(keep), 3, cfg.win, cfg.win)
    rows = []
    for a in pick:
        h = H_all[np.searchsorted(keep, a)]
        rows.extend([h[1]] if nch[a] == 1 else list(h))
    scans = np.stack([np.linspace(-20.0, 140.0, 101), np.linspace(130.0, -5.0, 101)], axis=1)
    return cfg, synth.Specimen(cfg=cfg, atoms=sp.atoms, nch=nch, V=sp.V, H=np.stack(rows), scans=scans)


def test_map_edge_cases(lib):
    cfg, sp = _edge_specimen()
    pr = obip.make_problem(sp)
    assert set(pr.plane.tolist()) == {0, 1, 2, 3, 4}
    assert np.any(pr.tau_px < cfg.win / 2) and len(pr.ion) == 21
    ref = obip.bip_map(pr)
    _, m, parts, _ = gpu_run(lib, cfg, sp)
    assert rel(m, ref.map) < 1e-4
    assert rel(parts, ref.partials) < 1e-4


def test_single_scan_single_site(lib):
    cfg = synth.config1().replace(ion_cells=(2, 3))
    sp = synth.make_specimen(cfg)
    sp.scans = np.array([[80.0, 78.0]])
    pr = obip.make_problem(sp)
    assert len(pr.ion) == 1
    ref = obip.bip_map(pr)
    _, m, _, _ = gpu_run(lib, cfg, sp)
    assert abs(m[0] - ref.map[0]) < 1e-4 * abs(ref.map[0])


def test_anisotropic_grid(lib):
    """ny != nx, L_y != L_x, f_y != f_x, a window of 32 and sub-pixel scans."""
    cfg = synth.config1().replace(name="aniso", ny=64, nx=128, ly=7.5, lx=10.0, cells_y=3, cells_x=4,
                                  fy=1, fx=2, win=32, ion_cells=(1, 3), ion_slices=(1, 4),
                                  scan_y=(10.3, 3.5, 9), scan_x=(20.7, 6.25, 7))
    sp = synth.make_specimen(cfg)
    pr = obip.make_problem(sp)
    ref = obip.bip_map(pr)
    _, m, _, _ = gpu_run(lib, cfg, sp)
    assert rel(m, ref.map) < 1e-4


# ---------------------------------------------------------------------------
# split-BF16 tensor-core path (tcgen05): rel L2 <= 1e-3 for maps

@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("split_bf16", 1e-4), ("mixed", 1e-2)])
def test_coupling_parity(lib, c1, prec, tol):
    """Coupling matrices M^(n) (Eq. coupling) of every site, both precisions."""
    cfg, sp, pr, ref = c1
    ctx, _, _, H = gpu_run(lib, cfg, sp, prec=prec)
    for k in range(len(pr.ion)):
        got = ctx.coupling(H, k).cpu().numpy()
        want = ref.stages[k]["M"]
        assert got.shape == want.shape
        assert rel(got, want) < tol, (prec, k, rel(got, want))


@pytest.mark.parametrize("prec", ["split_bf16", "mixed"])
def test_map_split_bf16_config1(lib, c1, prec):
    """Config 3: config 1 with the contraction in split-BF16 (hi + lo), and
    the mixed mode (BF16 coupling and Gram, split-BF16 quadratic form)."""
    cfg, sp, pr, ref = c1
    _, m, parts, _ = gpu_run(lib, cfg, sp, prec=prec)
    assert rel(m, ref.map) < 1e-3
    assert rel(parts, ref.partials) < 1e-3
    for k in range(len(pr.ion)):
        assert np.all(parts[k][~obip.crop_mask(pr, k, pr.scans)] == 0.0)


@pytest.mark.parametrize("prec", ["split_bf16", "mixed"])
def test_map_split_bf16_edge_cases(lib, prec):
    cfg, sp = _edge_specimen()
    pr = obip.make_problem(sp)
    ref = obip.bip_map(pr)
    _, m, parts, _ = gpu_run(lib, cfg, sp, prec=prec)
    assert rel(m, ref.map) < 1e-3
    assert rel(parts, ref.partials) < 1e-3


@pytest.mark.parametrize("prec", ["split_bf16", "mixed"])
def test_map_split_bf16_anisotropic(lib, prec):
    cfg = synth.config1().replace(name="aniso", ny=64, nx=128, ly=7.5, lx=10.0, cells_y=3, cells_x=4,
                                  fy=1, fx=2, win=32, ion_cells=(1, 3), ion_slices=(1, 4),
                                  scan_y=(10.3, 3.5, 9), scan_x=(20.7, 6.25, 7))
    sp = synth.make_specimen(cfg)
    ref = obip.bip_map(obip.make_problem(sp))
    _, m, _, _ = gpu_run(lib, cfg, sp, prec=prec)
    assert rel(m, ref.map) < 1e-3


# ---------------------------------------------------------------------------
# the 4D cube and qEELS (Sec. 2.2.6)

def _cube(ctx, sp, H, **kw):
    V = torch.tensor(sp.V, dtype=torch.float32, device=H.device)
    return ctx.cube(V, H, sp.scans, **kw).cpu().numpy()


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-4), ("split_bf16", 1e-3), ("mixed", 1e-3)])
def test_cube_config1(lib, c1, prec, tol):
    """The cube on the complete output basis (S1 partitioned, the exit
    exact; 793 beams at config 1 against the map's 193) against the
    oracle's, which is pinned to Algorithm 3 by brute force; zero outside
    every crop mask; bit-identical on a second run (no atomics)."""
    cfg, sp, pr, ref = c1
    want = obip.bip_cube(pr)
    ctx, m, _, H = gpu_run(lib, cfg, sp, prec=prec)
    assert np.array_equal(ctx.cube_beams, pr.geo.h_cube)
    cube = _cube(ctx, sp, H)
    assert cube.shape == want.shape == (len(sp.scans), 793)
    assert rel(cube, want) < tol
    outside = np.ones(len(sp.scans), bool)
    for k in range(len(pr.ion)):
        outside &= ~obip.crop_mask(pr, k, pr.scans)
    assert np.all(cube[outside] == 0.0)
    assert np.array_equal(_cube(ctx, sp, H), cube)


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-4), ("split_bf16", 1e-4), ("mixed", 1e-3)])
def test_cube_raster_and_any_scan_order_agree(lib, c1, prec, tol):
    """On a raster scan list the cube's per-beam contraction runs separated
    over the beam lattice (two short sums per site, FP32); the same scans
    shuffled are no raster and take the per-scan contraction.  Both against
    the oracle, and row for row against each other."""
    cfg, sp, pr, ref = c1
    want = obip.bip_cube(pr)
    ctx, m, _, H = gpu_run(lib, cfg, sp, prec=prec)
    cube_r = _cube(ctx, sp, H)
    assert rel(cube_r, want) < tol
    perm = np.random.default_rng(3).permutation(len(sp.scans))
    V = torch.tensor(sp.V, dtype=torch.float32, device=H.device)
    cube_p = ctx.cube(V, H, sp.scans[perm]).cpu().numpy()
    assert rel(cube_p, want[perm]) < tol
    assert rel(cube_p, cube_r[perm]) < tol


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-4), ("mixed", 1e-3)])
def test_cube_edge_cases(lib, prec, tol):
    """Sites in every plane, windows wrapping the grid, one- and
    three-channel sites, a ragged wrapped scan list (FP32: SIMT per-beam
    contraction; mixed: the tcgen05 cube kernel over 64-scan tiles)."""
    cfg, sp = _edge_specimen()
    pr = obip.make_problem(sp)
    want = obip.bip_cube(pr)
    ctx, m, _, H = gpu_run(lib, cfg, sp, prec=prec)
    cube = _cube(ctx, sp, H)
    assert rel(cube, want) < tol
    assert np.array_equal(_cube(ctx, sp, H), cube)


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-4), ("mixed", 1e-3)])
def test_cube_on_a_box_of_k_pixels(lib, prec, tol):
    """A 40 x 24 box of k-pixels as the cube's basis (a pixelated detector
    of that shape; 960 beams, beyond the 40 mrad disc along y) against the
    oracle's cube on the same basis."""
    cfg = synth.config1().replace(cube_ky=40, cube_kx=24)
    sp = synth.make_specimen(cfg)
    pr = obip.make_problem(sp)
    ctx, m, _, H = gpu_run(lib, cfg, sp, prec=prec)
    assert np.array_equal(ctx.cube_beams, pr.geo.h_cube) and len(pr.geo.h_cube) == 960
    assert rel(_cube(ctx, sp, H), obip.bip_cube(pr)) < tol
    ctx.close()


@pytest.mark.parametrize("prec", ["fp32", "split_bf16"])
def test_cube_in_beam_batches(lib, c1, prec):
    """A memory limit that splits the complete basis into several backward
    sweeps (13 batches of 64 beams at config 1) gives the cube of one sweep."""
    cfg, sp, pr, ref = c1
    ctx, m, _, H = gpu_run(lib, cfg, sp, prec=prec)
    one = _cube(ctx, sp, H)
    per_beam = (len(pr.ion) * cfg.win * cfg.win + cfg.ny * cfg.nx) * 8
    ctx.set_cube_memory(64 * per_beam + 1)
    many = _cube(ctx, sp, H)
    assert rel(many, one) < 1e-6
    assert rel(many, obip.bip_cube(pr)) < (1e-4 if prec == "fp32" else 1e-3)


def test_cube_refuses_fp8_and_a_missing_build(lib, c1):
    from paper_2607_00756_gb300.capi import BipError, STATUS
    cfg, sp, pr, ref = c1
    dev = torch.device("cuda:0")
    H = torch.tensor(sp.H, dtype=torch.complex64, device=dev)
    V = torch.tensor(sp.V, dtype=torch.float32, device=dev)
    ctx = lib(cfg, prec="mixed")
    with pytest.raises(BipError) as e:
        ctx.cube(V, H, sp.scans)
    assert STATUS[e.value.status] == "BIP_ERR_INVALID_ARG"
    ctx.close()
    ctx, *_ = gpu_run(lib, cfg, sp, prec="fp8")
    with pytest.raises(BipError) as e:
        ctx.cube(V, H, sp.scans)
    assert STATUS[e.value.status] == "BIP_ERR_UNSUPPORTED"
    ctx.close()


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
@pytest.mark.parametrize("axis", [0, 1])
def test_qeels_config1(lib, axis, prec):
    """qEELS with the resolved axis sampled at f = 1 (S2 partitioned on
    that detector set) against the oracle's; the bins summed give the
    library's map of the same context."""
    cfg = synth.config1().replace(**({"dfy": 1} if axis == 0 else {"dfx": 1}))
    sp = synth.make_specimen(cfg)
    pr = obip.make_problem(sp)
    hb_want, want = obip.bip_qeels(pr, axis)
    ctx, m, _, H = gpu_run(lib, cfg, sp, prec=prec)
    assert ctx.n_det == pr.geo.n_det
    hb, q = ctx.qeels(H, sp.scans, axis)
    assert np.array_equal(hb, hb_want)
    q = q.cpu().numpy()
    tol = 1e-4 if prec == "fp32" else 1e-3
    assert rel(q, want) < tol
    assert rel(q.astype(np.float64).sum(axis=1), m) < tol
    assert rel(m, obip.bip_map(pr).map) < tol


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_qeels_raster_and_any_scan_order_agree(lib, prec):
    """qEELS on the raster scans (the per-beam terms by the separated
    contraction) and on the same scans shuffled (the cube kernel): each
    against the oracle and against each other row for row."""
    cfg = synth.config1().replace(dfx=1)
    sp = synth.make_specimen(cfg)
    pr = obip.make_problem(sp)
    _, want = obip.bip_qeels(pr, 1)
    ctx, m, _, H = gpu_run(lib, cfg, sp, prec=prec)
    _, q_r = ctx.qeels(H, sp.scans, 1)
    perm = np.random.default_rng(6).permutation(len(sp.scans))
    _, q_p = ctx.qeels(H, sp.scans[perm], 1)
    q_r, q_p = q_r.cpu().numpy(), q_p.cpu().numpy()
    tol = 1e-4 if prec == "fp32" else 1e-3
    assert rel(q_r, want) < tol
    assert rel(q_p, want[perm]) < tol
    assert rel(q_p, q_r[perm]) < tol


def test_qeels_refuses_a_subsampled_axis(lib, c1):
    from paper_2607_00756_gb300.capi import BipError, STATUS
    cfg, sp, pr, ref = c1
    ctx, m, _, H = gpu_run(lib, cfg, sp)
    for axis in (0, 1):
        with pytest.raises(BipError) as e:
            ctx.qeels(H, sp.scans, axis)
        assert STATUS[e.value.status] == "BIP_ERR_INVALID_ARG"


# ---------------------------------------------------------------------------
# FP8 (E4M3) coupling with per-window scales (config 3's FP8 form)

def _fp8_model(pr):
    from oracle import fp8
    return fp8.bip_map_fp8(pr)


def test_map_fp8_config1(lib, c1):
    """The FP8 map against the FP64 map and against the oracle's FP8 model
    (E4M3 operands with the same per-window scale rule, contracted in FP64).
    The GPU's error may exceed the model's only by what its BF16
    reconstruction and Gram add on top (<= 1e-3, the mixed path's bound):
    bounded here by twice the model's error plus 1e-3.  Its distance to
    the model comes from E4M3 codes that differ by one step where the two
    pre-quantization values (BF16- vs FP64-reconstructed) straddle a
    rounding boundary, and stays below the model's own error."""
    cfg, sp, pr, ref = c1
    model = _fp8_model(pr)
    e_model = rel(model.map, ref.map)
    _, m, parts, _ = gpu_run(lib, cfg, sp, prec="fp8")
    e_gpu = rel(m, ref.map)
    assert 0.0 < e_gpu < 2.0 * e_model + 1e-3, (e_gpu, e_model)
    assert rel(m, model.map) < e_model, (rel(m, model.map), e_model)
    assert rel(parts, model.partials) < 2.0 * e_model
    for k in range(len(pr.ion)):
        assert np.all(parts[k][~obip.crop_mask(pr, k, pr.scans)] == 0.0)


def test_coupling_fp8_config1(lib, c1):
    """M^(n) of every site from the FP8 coupling against the oracle's FP8
    model of the same contraction and against the FP64 coupling."""
    from oracle import fp8
    cfg, sp, pr, ref = c1
    geo = pr.geo
    ctx, _, _, H = gpu_run(lib, cfg, sp, prec="fp8")
    for k in range(len(pr.ion)):
        st = ref.stages[k]
        want8 = fp8.site_coupling_fp8(st["S2w"], pr.H[k], st["S1w"], geo.w2, st["stash2"], geo.w1, st["stash1"])
        e_model = rel(want8, st["M"])
        got = ctx.coupling(H, k).cpu().numpy()
        assert got.shape == st["M"].shape
        assert rel(got, st["M"]) < 2.0 * e_model + 1e-3, (k, rel(got, st["M"]), e_model)
        assert rel(got, want8) < e_model, (k, rel(got, want8), e_model)


def test_map_fp8_edge_cases(lib):
    cfg, sp = _edge_specimen()
    pr = obip.make_problem(sp)
    ref = obip.bip_map(pr)
    e_model = rel(_fp8_model(pr).map, ref.map)
    _, m, parts, _ = gpu_run(lib, cfg, sp, prec="fp8")
    assert rel(m, ref.map) < 2.0 * e_model + 1e-3
    for k in range(len(pr.ion)):
        assert np.all(parts[k][~obip.crop_mask(pr, k, pr.scans)] == 0.0)


def test_map_fp8_anisotropic(lib):
    """32x32 windows (K = 1024), f_y != f_x, a non-square grid."""
    cfg = synth.config1().replace(name="aniso", ny=64, nx=128, ly=7.5, lx=10.0, cells_y=3, cells_x=4,
                                  fy=1, fx=2, win=32, ion_cells=(1, 3), ion_slices=(1, 4),
                                  scan_y=(10.3, 3.5, 9), scan_x=(20.7, 6.25, 7))
    sp = synth.make_specimen(cfg)
    pr = obip.make_problem(sp)
    ref = obip.bip_map(pr)
    e_model = rel(_fp8_model(pr).map, ref.map)
    _, m, _, _ = gpu_run(lib, cfg, sp, prec="fp8")
    assert rel(m, ref.map) < 2.0 * e_model + 1e-3


def test_qeels_fp8_config1(lib):
    """qEELS through the FP8 coupling against the FP64 qEELS, bounded like
    the map by twice the FP8 model's own error (per detector beam); its
    bins sum to the FP8 map."""
    from oracle import fp8
    cfg = synth.config1().replace(dfx=1)
    sp = synth.make_specimen(cfg)
    pr = obip.make_problem(sp)
    bins, want = obip.bip_qeels(pr, 1)
    pb = fp8.per_beam_fp8(pr)
    hd = pr.geo.h_det[:, 1]
    model = np.stack([pb[:, hd == b].sum(axis=1) for b in bins], axis=1)
    e_model = rel(model, want)
    ctx, m, _, H = gpu_run(lib, cfg, sp, prec="fp8")
    _, q = ctx.qeels(H, sp.scans, 1)
    q = q.cpu().numpy()
    assert rel(q, want) < 2.0 * e_model + 1e-3, (rel(q, want), e_model)
    assert rel(q.astype(np.float64).sum(axis=1), m) < 1e-4


# ---------------------------------------------------------------------------
# the two evaluations of the scan polynomial

@pytest.mark.parametrize("which", ["config1", "aniso"])
@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_raster_and_horner_evaluations_agree(lib, which, prec):
    """A raster scan list takes the separable evaluation; switched off, the
    same scans go through Horner's rule per scan.  Both are the same
    polynomial (FP32 sums in different orders), and both match the oracle."""
    if which == "config1":
        cfg = synth.config1()
    else:
        cfg = synth.config1().replace(name="aniso", ny=64, nx=128, ly=7.5, lx=10.0, cells_y=3, cells_x=4, fy=1,
                                      fx=2, win=32, ion_cells=(1, 3), ion_slices=(1, 4),
                                      scan_y=(10.3, 3.5, 9), scan_x=(20.7, 6.25, 7))
    sp = synth.make_specimen(cfg)
    ref = obip.bip_map(obip.make_problem(sp))
    dev = torch.device("cuda:0")
    ctx = lib(cfg, prec=prec)
    ctx.build(torch.tensor(sp.V, dtype=torch.float32, device=dev), sp.atoms, sp.nch)
    H = torch.tensor(sp.H, dtype=torch.complex64, device=dev)
    m_r = ctx.map(H, sp.scans).cpu().numpy()
    p_r = ctx.sites(H, sp.scans).cpu().numpy()
    ctx.set_raster_eval(False)
    m_h = ctx.map(H, sp.scans).cpu().numpy()
    p_h = ctx.sites(H, sp.scans).cpu().numpy()
    assert rel(m_r, m_h) < 1e-5
    assert rel(p_r, p_h) < 1e-5
    assert np.array_equal(p_r == 0.0, p_h == 0.0)            # the same crop masks
    tol = 1e-4 if prec == "fp32" else 1e-3
    assert rel(m_r, ref.map) < tol and rel(m_h, ref.map) < tol
    ctx.close()


@pytest.mark.parametrize("prec", ["fp32", "split_bf16", "mixed"])
def test_map_unchanged_after_cube_and_grad(lib, c1, prec):
    """The cube and the reverse pass share a context with the map without
    disturbing it: the map after both is the map before, bit for bit (the
    workspaces' zero padding survives the other layouts)."""
    cfg, sp, pr, ref = c1
    ctx, m0, _, H = gpu_run(lib, cfg, sp, prec=prec)
    V = torch.tensor(sp.V, dtype=torch.float32, device=H.device)
    ctx.cube(V, H, sp.scans)
    ctx.grad(H, sp.scans, torch.ones(len(sp.scans), dtype=torch.float64, device=H.device), V=V)
    m1 = ctx.map(H, sp.scans).cpu().numpy()
    assert np.array_equal(m1, m0)
    ctx.close()
