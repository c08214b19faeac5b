"""C-ABI library checks that need no GPU: it builds, loads, exports every
declared entry point, and its host geometry (FP64 beams, parents, Sibson
weights) agrees with the oracle's independent implementation."""
import ctypes
import os
import re

import numpy as np
import pytest

import synth
from oracle import geometry as G, physics as ph

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def capi():
    from paper_2607_00756_gb300 import build
    build.build()
    from paper_2607_00756_gb300 import capi as c
    return c


def declared_functions():
    text = open(os.path.join(ROOT, "include", "bip.h")).read()
    return sorted(set(re.findall(r"^\s*(?:bip_status|const char\*)\s+(bip_\w+)\s*\(", text, re.M)))


def test_exports_every_declared_symbol(capi):
    names = declared_functions()
    assert len(names) >= 14
    lib = ctypes.CDLL(capi.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n


def _cfgs():
    c1 = synth.config1()
    return [c1, synth.config2(), synth.tiny_config(ny=64, nx=64, win=64),
            c1.replace(name="aniso", ny=64, nx=128, ly=6.0, lx=10.0, fy=1, fx=2, win=32),
            c1.replace(name="rings", nrad1=3, nrad2=4, nang1=5, nang2=7),
            c1.replace(name="aberrated", defocus=-35.0, cs=1e4),
            c1.replace(name="qeels_x", dfx=1), c1.replace(name="qeels_y", dfy=1, nrad2=3),
            c1.replace(name="cube_box", cube_ky=32, cube_kx=20),
            c1.replace(name="f3_384", ny=384, nx=384, ly=30.0, lx=30.0, fy=3, fx=3),
            c1.replace(name="f3_aniso", ny=768, nx=192, ly=60.0, lx=15.0, fy=3, fx=3, nrad2=3, dfx=1)]


@pytest.mark.parametrize("cfg", _cfgs(), ids=lambda c: c.name)
def test_geometry_matches_oracle(capi, cfg):
    ctx = capi.bip_create(capi.make_config(cfg))
    try:
        g = capi.bip_get_geometry(ctx)
        og = G.Geometry(cfg, ph.wavelength(cfg.e0))
        assert np.array_equal(g["h_beam"], og.h_beam)
        assert np.array_equal(g["h_det"], og.h_det)
        assert np.array_equal(g["p1"], og.p1)
        assert np.array_equal(g["p2"], og.p2)
        assert np.max(np.abs(g["w1"] - og.w1)) < 1e-12
        assert np.max(np.abs(g["w2"] - og.w2)) < 1e-12
        assert np.array_equal(capi.bip_cube_beams(ctx), og.h_cube)
    finally:
        capi.bip_destroy(ctx)


def test_config2_sizes(capi):
    """300 keV, 25 mrad, 40 A, f = 4: 505 retained beams of 8093, 1305
    detector beams in 40 mrad, 61 parents each at n_radial = 4."""
    ctx = capi.bip_create(capi.make_config(synth.config2()))
    try:
        assert capi.bip_query(ctx) == (505, 1305, 61, 61, 0)
    finally:
        capi.bip_destroy(ctx)


@pytest.mark.parametrize("change,status", [
    (dict(ny=96), "BIP_ERR_SHAPE"),
    (dict(ny=1536, ly=120.0), "BIP_ERR_SHAPE"),
    (dict(ny=320), "BIP_ERR_SHAPE"),
    (dict(nx=2048), "BIP_ERR_SHAPE"),
    (dict(win=40), "BIP_ERR_SHAPE"),
    (dict(win=128), "BIP_ERR_SHAPE"),
    (dict(fy=3), "BIP_ERR_SHAPE"),
    (dict(alpha=0.2), "BIP_ERR_SHAPE"),
    (dict(nz=0), "BIP_ERR_INVALID_ARG"),
    (dict(e0=-1.0), "BIP_ERR_INVALID_ARG"),
    (dict(nang1=0), "BIP_ERR_INVALID_ARG"),
    (dict(dfx=3), "BIP_ERR_SHAPE"),
    (dict(cube_ky=256, cube_kx=16), "BIP_ERR_SHAPE"),
    (dict(cube_ky=16), "BIP_ERR_SHAPE"),
    (dict(dfy=-1), "BIP_ERR_SHAPE"),
])
def test_create_rejects_bad_config(capi, change, status):
    cfg = synth.config1().replace(**change)
    with pytest.raises(capi.BipError) as e:
        capi.bip_create(capi.make_config(cfg))
    assert capi.STATUS[e.value.status] == status


def test_calls_out_of_order_return_errors(capi):
    ctx = capi.bip_create(capi.make_config(synth.config1()))
    try:
        lib = capi.lib()
        scans = np.zeros((4, 2))
        sp = scans.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        dummy = ctypes.c_void_p(16)
        assert lib.bip_coreloss_map(ctx, dummy, sp, 4, dummy, None) == 1
        assert "bip_build_s1" in capi.bip_last_error(ctx)
        assert lib.bip_copy_stash(ctx, 1, 0, dummy, None) == 1
        assert lib.bip_set_precision(ctx, 7) == 1
        assert lib.bip_build_s1(ctx, None, None, 0, None) == 1
        atoms = capi.make_atoms(np.array([[1.0, 1.0, 9.0]]), np.array([3]))
        assert lib.bip_build_s1(ctx, dummy, atoms, 1, None) == 1      # slice 9 >= nz
        assert "slice" in capi.bip_last_error(ctx)
        atoms = capi.make_atoms(np.array([[1.0, 1.0, 0.0]]), np.array([0]))
        assert lib.bip_build_s1(ctx, dummy, atoms, 1, None) == 1      # nothing ionized
        # the combined build checks the same arguments before any device work
        assert lib.bip_build(None, dummy, atoms, 1, None) == 1
        assert lib.bip_build(ctx, None, atoms, 1, None) == 1          # V is null
        assert lib.bip_build(ctx, dummy, atoms, 1, None) == 1         # nothing ionized
        assert "ionized" in capi.bip_last_error(ctx)
        atoms = capi.make_atoms(np.array([[1.0, 1.0, 9.0]]), np.array([3]))
        assert lib.bip_build(ctx, dummy, atoms, 1, None) == 1         # slice 9 >= nz
        assert "slice" in capi.bip_last_error(ctx)
        assert capi.bip_query(ctx)[4] == 0                            # nothing built
    finally:
        capi.bip_destroy(ctx)
    assert capi.lib().bip_last_error(None) == b"null context"
    assert capi.lib().bip_destroy(None) == 1


def test_qeels_bins_host(capi):
    """The qEELS bins: the distinct detector-beam components along the axis,
    ascending; another axis is an argument error."""
    cfg = synth.config1()
    ctx = capi.bip_create(capi.make_config(cfg))
    try:
        geo = capi.bip_get_geometry(ctx)
        for axis in (0, 1):
            h = capi.bip_qeels_bins(ctx, axis)
            assert np.array_equal(h, np.unique(geo["h_det"][:, axis]))
        with pytest.raises(capi.BipError):
            capi.bip_qeels_bins(ctx, 2)
    finally:
        capi.bip_destroy(ctx)


def test_model_and_launch_controls_host(capi):
    """Argument checks of the model-parameter, launch-control and reverse-pass
    entry points, all before any GPU work (the calls fail or succeed on the
    host alone)."""
    ctx = capi.bip_create(capi.make_config(synth.config1()))
    try:
        lib = capi.lib()
        D = ctypes.c_double
        # occupancies need built sites; NULL restores the unit weights
        occ = (D * 4)(1.0, 1.0, 1.0, 1.0)
        assert lib.bip_set_occupancy(ctx, occ) == 1
        assert "build" in capi.bip_last_error(ctx)
        assert lib.bip_set_occupancy(ctx, None) == 0
        # per-site windows need built sites too
        w = (ctypes.c_int32 * 4)(32, 64, 16, 48)
        assert lib.bip_set_site_windows(ctx, w, None) == 1
        assert "build" in capi.bip_last_error(ctx)
        assert lib.bip_set_site_windows(None, w, None) == 1
        # aberrations: finite values only
        assert lib.bip_set_aberrations(ctx, D(float("nan")), D(0.0), None) == 1
        assert lib.bip_set_aberrations(ctx, D(25.0), D(1.0e5), None) == 0
        # launch shapes: tile widths multiples of 16 up to 256, no negatives
        assert lib.bip_set_launch(ctx, 0, 17) == 1
        assert lib.bip_set_launch(ctx, -1, 0) == 1
        assert lib.bip_set_launch(ctx, 0, 272) == 1
        assert lib.bip_set_launch(ctx, 19, 224) == 0
        assert lib.bip_set_launch(ctx, 0, 0) == 0
        assert lib.bip_set_capture_safe(ctx, 1) == 0 and lib.bip_set_capture_safe(ctx, 0) == 0
        assert lib.bip_set_raster_eval(ctx, 0) == 0 and lib.bip_set_raster_eval(ctx, 1) == 0
        assert lib.bip_check_errors(ctx, None) == 0
        # the reverse pass and the autotuner need the builds first
        scans = np.zeros((4, 2))
        sp = scans.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        dummy = ctypes.c_void_p(16)
        assert lib.bip_coreloss_grad(ctx, None, dummy, sp, 4, dummy, dummy, None, None, None, None) == 1
        assert "bip_build_s1" in capi.bip_last_error(ctx)
        assert lib.bip_autotune(ctx, dummy, sp, 4, dummy, None, None, None, None, None) == 1
        assert lib.bip_set_order(ctx, 3) == 1 and lib.bip_set_order(ctx, -1) == 1
        assert lib.bip_set_order(ctx, 1) == 0 and lib.bip_set_order(ctx, 0) == 0
        # the probe order: mixed precision only
        assert lib.bip_set_order(ctx, 2) == (0 if synth.config1().prec == "mixed" else 6)
        mixed = capi.bip_create(capi.make_config(synth.config1(), prec="mixed"))
        try:
            assert lib.bip_set_order(mixed, 2) == 0 and lib.bip_set_order(mixed, 0) == 0
        finally:
            capi.bip_destroy(mixed)
    finally:
        capi.bip_destroy(ctx)
    assert capi.lib().bip_set_launch(None, 0, 0) == 1
    assert capi.lib().bip_set_occupancy(None, None) == 1


def test_product_never_imports_the_oracle():
    """The library package, its C/CUDA sources and the input generators
    reference nothing under oracle/: the product path runs only in
    libbip.so, and the oracle is test infrastructure."""
    import ast
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for sub in ("paper_2607_00756_gb300", "synth"):
        for dirpath, _, files in os.walk(os.path.join(root, sub)):
            for f in files:
                path = os.path.join(dirpath, f)
                if f.endswith(".py"):
                    tree = ast.parse(open(path).read())
                    for node in ast.walk(tree):
                        if isinstance(node, ast.Import):
                            assert not any(a.name.split(".")[0] == "oracle" for a in node.names), path
                        elif isinstance(node, ast.ImportFrom):
                            assert (node.module or "").split(".")[0] != "oracle", path
                elif f.endswith((".cu", ".cuh", ".cpp", ".h")):
                    assert "oracle/" not in open(path).read(), path


def test_noalloc_wrapper_refuses_wrong_stash_shape(capi):
    """The allocation-free S1 build writes n_sites x Bp1 x win x win values
    into the caller's stash, which the C entry point cannot size-check; the
    binding refuses any other shape before anything is launched."""
    torch = pytest.importorskip("torch")
    cfg = synth.config1()
    ctx = capi.bip_create(capi.make_config(cfg))
    try:
        atoms = capi.make_atoms(np.array([[5.0, 5.0, 2.0], [6.0, 6.0, 2.0], [1.0, 1.0, 0.0]]),
                                np.array([3, 1, 0]))
        bp1 = capi.bip_query(ctx)[2]
        assert capi.noalloc_stash_shape(ctx, atoms) == (2, bp1, cfg.win, cfg.win)
        assert capi.bip_get_config(ctx).win == cfg.win
        V = torch.zeros((cfg.nz, cfg.ny, cfg.nx), dtype=torch.float32)
        for shape in [(1, bp1, cfg.win, cfg.win), (2, bp1 - 1, cfg.win, cfg.win), (2, bp1, 32, 32),
                      (2 * bp1 * cfg.win * cfg.win,)]:
            small = torch.empty(shape, dtype=torch.complex64)
            with pytest.raises(ValueError, match="stash must have shape"):
                capi.bip_build_s1_noalloc(ctx, V, atoms, small)
        # the right shape passes the size check and then meets the device check
        ok = torch.empty((2, bp1, cfg.win, cfg.win), dtype=torch.complex64)
        with pytest.raises(ValueError, match="CUDA tensor"):
            capi.bip_build_s1_noalloc(ctx, V, atoms, ok)
    finally:
        capi.bip_destroy(ctx)


def test_geometry_random_rings_match_oracle(capi):
    """The library's Sibson weights (Delaunay triangulation, Watson's
    circumcentre construction) against the oracle's (half-plane clipping of
    Voronoi cells) on seeded random geometries: ring counts 0..5 with 1..8
    samples (collinear and tiny parent sets included), anisotropic cells,
    f = 1 or 2, several apertures and detector discs."""
    rng = np.random.default_rng(7)
    checked = 0
    for _ in range(30):
        cfg = synth.config1().replace(
            ny=int(rng.choice([64, 128])), nx=int(rng.choice([64, 128])),
            ly=float(rng.choice([5.0, 7.5, 10.0, 12.3])), lx=float(rng.choice([5.0, 7.5, 10.0, 13.7])),
            fy=int(rng.choice([1, 2])), fx=int(rng.choice([1, 2])), win=16,
            nrad1=int(rng.integers(0, 6)), nang1=int(rng.integers(1, 9)),
            nrad2=int(rng.integers(0, 6)), nang2=int(rng.integers(1, 9)),
            alpha=float(rng.choice([0.01, 0.02, 0.03])), theta_det=float(rng.choice([0.02, 0.04])))
        try:
            ctx = capi.bip_create(capi.make_config(cfg))
        except capi.BipError:
            continue          # a disc beyond the grid's band
        try:
            g = capi.bip_get_geometry(ctx)
        finally:
            capi.bip_destroy(ctx)
        og = G.Geometry(cfg, ph.wavelength(cfg.e0))
        assert np.array_equal(g["p1"], og.p1) and np.array_equal(g["p2"], og.p2)
        assert np.max(np.abs(g["w1"] - og.w1)) < 1e-12
        assert np.max(np.abs(g["w2"] - og.w2)) < 1e-12
        checked += 1
    assert checked >= 20


def test_geometry_many_parents_is_fast(capi):
    """n_radial = 12 (443 and 469 parents at config 2's sizes): the host
    geometry stays well under a second and agrees with the oracle."""
    import time
    cfg = synth.config2().replace(nrad1=12, nrad2=12)
    t0 = time.perf_counter()
    ctx = capi.bip_create(capi.make_config(cfg))
    dt = time.perf_counter() - t0
    try:
        assert capi.bip_query(ctx)[2:4] == (443, 469)
        g = capi.bip_get_geometry(ctx)
    finally:
        capi.bip_destroy(ctx)
    assert dt < 1.0
    og = G.Geometry(cfg, ph.wavelength(cfg.e0))
    assert np.max(np.abs(g["w1"] - og.w1)) < 1e-12
    assert np.max(np.abs(g["w2"] - og.w2)) < 1e-12


def test_injected_allocation_failure_is_oom_before_any_device_work(capi):
    """The first device allocation of a build made to fail: both builds
    return BIP_ERR_OOM (before anything reaches the device), nothing stays
    allocated, and the injection is off again afterwards."""
    cfg = synth.config1()
    live0, _ = capi.bip_debug_allocs()
    ctx = capi.bip_create(capi.make_config(cfg))
    try:
        atoms = capi.make_atoms(np.array([[5.0, 5.0, 2.0]]), np.array([3]))
        lib = capi.lib()
        dummy = ctypes.c_void_p(256)
        for fn in (lib.bip_build_s1, lib.bip_build_s2):
            capi.bip_debug_fail_alloc(1)
            assert fn(ctx, dummy, atoms, 1, None) == 3                  # BIP_ERR_OOM
            assert "cudaErrorMemoryAllocation" in capi.bip_last_error(ctx) or "memory" in capi.bip_last_error(ctx)
            assert capi.bip_debug_allocs() == (live0, 1)
        assert lib.bip_set_wait_limit(ctx, -5) == 1
        assert lib.bip_set_wait_limit(ctx, 1000) == 0
    finally:
        capi.bip_debug_fail_alloc(0)
        capi.bip_destroy(ctx)
    assert capi.bip_debug_allocs()[0] == live0
    assert capi.lib().bip_debug_fail_alloc(-1) == 1
