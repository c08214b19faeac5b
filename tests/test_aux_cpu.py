"""Auxiliary subsystems that need no GPU: the on-disk geometry cache (its
hits, misses and the files it rejects), the NVTX ranges a tracing tool
sees, and the host-side checks of the stash export / import, the finite
check and the memory statistics."""
import ctypes
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import nvtx_tool
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def capi():
    from paper_2607_00756_gb300 import build
    build.build()
    from paper_2607_00756_gb300 import capi as c
    return c


@pytest.fixture
def cache_dir(capi, tmp_path):
    d = tmp_path / "geometry-cache"
    d.mkdir()
    capi.bip_set_geometry_cache(str(d))
    yield d
    capi.bip_set_geometry_cache(None)


def _geometry(capi, cfg):
    ctx = capi.bip_create(capi.make_config(cfg))
    try:
        g = capi.bip_get_geometry(ctx)
        g["cube"] = capi.bip_cube_beams(ctx)
        g["sizes"] = np.array(capi.bip_query(ctx)[:4])
        return g
    finally:
        capi.bip_destroy(ctx)


def _same(a, b):
    return all(np.array_equal(a[k], b[k]) for k in a)


def _stats_since(capi, s0):
    return tuple(x - y for x, y in zip(capi.bip_geometry_cache_stats(), s0))


def test_geometry_cache_miss_then_hit(capi, cache_dir):
    cfg = synth.config1().replace(nrad1=3, nrad2=3, defocus=-20.0)
    capi.bip_set_geometry_cache(None)
    want = _geometry(capi, cfg)                      # computed without the cache
    capi.bip_set_geometry_cache(str(cache_dir))
    s0 = capi.bip_geometry_cache_stats()
    first = _geometry(capi, cfg)
    assert _stats_since(capi, s0) == (0, 1, 0)
    files = os.listdir(cache_dir)
    assert len(files) == 1 and files[0].startswith("bip-geometry-") and files[0].endswith(".bin")
    second = _geometry(capi, cfg)
    assert _stats_since(capi, s0) == (1, 1, 0)
    assert _same(first, want) and _same(second, want)
    # another geometry (defocus enters Psi, the rings the weights) gets its own file
    _geometry(capi, cfg.replace(defocus=-25.0))
    _geometry(capi, cfg.replace(nrad2=2))
    assert _stats_since(capi, s0) == (1, 3, 0)
    assert len(os.listdir(cache_dir)) == 3
    # fields the geometry does not read (slices, window, precision) share the file
    _geometry(capi, cfg.replace(nz=9, win=32, prec="mixed"))
    assert _stats_since(capi, s0) == (2, 3, 0)


@pytest.mark.parametrize("damage", ["flip", "truncate", "empty", "other_key"])
def test_geometry_cache_rejects_damaged_files(capi, cache_dir, damage):
    cfg = synth.config1()
    want = _geometry(capi, cfg)
    path = cache_dir / os.listdir(cache_dir)[0]
    data = bytearray(path.read_bytes())
    if damage == "flip":
        data[len(data) // 2] ^= 0x10                 # one bit inside the weights
    elif damage == "truncate":
        data = data[: len(data) - 9]
    elif damage == "empty":
        data = bytearray()
    else:
        # a valid file of another geometry under this geometry's name
        other = cfg.replace(nrad1=3)
        _geometry(capi, other)
        names = sorted(os.listdir(cache_dir), key=lambda n: (cache_dir / n).stat().st_mtime)
        data = bytearray((cache_dir / names[-1]).read_bytes())
    path.write_bytes(bytes(data))
    s0 = capi.bip_geometry_cache_stats()
    got = _geometry(capi, cfg)
    assert _stats_since(capi, s0) == (0, 1, 1)      # rejected, recomputed, rewritten
    assert _same(got, want)
    again = _geometry(capi, cfg)
    assert _stats_since(capi, s0) == (1, 1, 1)
    assert _same(again, want)


def test_geometry_cache_unwritable_directory_only_costs_the_rebuild(capi, tmp_path):
    missing = tmp_path / "does-not-exist"
    capi.bip_set_geometry_cache(str(missing))
    try:
        s0 = capi.bip_geometry_cache_stats()
        g = _geometry(capi, synth.config1())
        assert _stats_since(capi, s0) == (0, 1, 0)
        assert not missing.exists()
    finally:
        capi.bip_set_geometry_cache(None)
    assert _same(g, _geometry(capi, synth.config1()))


def test_geometry_cache_from_environment(capi, tmp_path):
    """BIP_GEOMETRY_CACHE names the directory until the call sets one."""
    d = tmp_path / "env-cache"
    d.mkdir()
    code = textwrap.dedent(f"""
        import sys
        sys.path.insert(0, {ROOT!r})
        from paper_2607_00756_gb300 import capi
        import synth
        for _ in range(2):
            ctx = capi.bip_create(capi.make_config(synth.config1()))
            capi.bip_destroy(ctx)
        print(*capi.bip_geometry_cache_stats())
    """)
    env = dict(os.environ, BIP_GEOMETRY_CACHE=str(d))
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    assert out.stdout.split() == ["1", "1", "0"]
    assert len(os.listdir(d)) == 1


def test_nvtx_ranges_reach_a_tool(capi, tmp_path):
    """A tracing tool attached through NVTX's injection interface sees one
    balanced range per public call (the stage ranges need launches, so a
    GPU)."""
    so = nvtx_tool.compile_tool(tmp_path)
    record = tmp_path / "ranges.txt"
    code = textwrap.dedent(f"""
        import sys
        sys.path.insert(0, {ROOT!r})
        from paper_2607_00756_gb300 import capi
        import synth
        ctx = capi.bip_create(capi.make_config(synth.config1()))
        capi.bip_destroy(ctx)
    """)
    env = dict(os.environ, NVTX_INJECTION64_PATH=str(so), NVTX_RECORD=str(record))
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    lines = record.read_text().splitlines()
    assert lines == ["push bip_create", "pop"]


def test_stash_and_check_calls_host_side(capi):
    """Argument checks of the stash export / import (sizes are checked
    against the site list before anything is copied) and of the finite
    check and memory statistics, which need no device work."""
    cfg = synth.config1()
    ctx = capi.bip_create(capi.make_config(cfg))
    lib = capi.lib()
    try:
        atoms = capi.make_atoms(np.array([[5.0, 5.0, 2.0], [2.5, 7.5, 1.0]]), np.array([3, 1]))
        host = np.zeros(16, np.complex64)
        ptr = host.ctypes.data_as(ctypes.c_void_p)
        assert lib.bip_export_stash(ctx, 1, ptr, host.nbytes, None) == 1        # nothing built
        assert lib.bip_export_stash(ctx, 3, ptr, host.nbytes, None) == 1
        assert lib.bip_import_stash(ctx, 0, atoms, 2, ptr, host.nbytes, None) == 1
        assert lib.bip_import_stash(ctx, 1, atoms, 2, None, host.nbytes, None) == 1
        # 2 sites x Bp1 parents x 64 x 64 x 8 bytes, not 128 bytes
        B, nd, bp1, bp2, _ = capi.bip_query(ctx)
        assert lib.bip_import_stash(ctx, 1, atoms, 2, ptr, host.nbytes, None) == 2
        assert str(2 * bp1 * cfg.win * cfg.win * 8) in capi.bip_last_error(ctx)
        assert lib.bip_import_stash(ctx, 2, atoms, 2, ptr, -1, None) == 2
        assert capi.bip_query(ctx)[4] == 0                                       # nothing changed
        assert capi.stash_shape(ctx, 1) == (0, bp1, cfg.win, cfg.win)
        assert lib.bip_set_check_finite(ctx, 1) == 0
        assert lib.bip_set_check_finite(None, 1) == 1
        live, peak = capi.bip_mem_stats()
        assert live >= 0 and peak >= live
        with pytest.raises(ValueError):
            capi.bip_import_stash(ctx, 1, atoms, np.zeros(4, np.complex128))
    finally:
        capi.bip_destroy(ctx)


def test_load_builds_refuses_another_configuration(capi, tmp_path):
    """A saved build is tied to its configuration: loading it into a context
    of another configuration raises before anything is restored."""
    torch = pytest.importorskip("torch")
    from paper_2607_00756_gb300.context import BipContext
    a = BipContext(synth.config1())
    b = BipContext(synth.config1().replace(nrad1=3))
    try:
        path = tmp_path / "builds.npz"
        np.savez(path, config=a._config_values(), y=np.zeros(1), x=np.zeros(1), slice=np.zeros(1, np.int32),
                 nch=np.ones(1, np.int32), s1=np.zeros((1, 1, 1, 1), np.complex64),
                 s2=np.zeros((1, 1, 1, 1), np.complex64))
        with pytest.raises(ValueError, match="another configuration"):
            b.load_builds(path)
        assert capi.bip_query(b.ctx)[4] == 0
    finally:
        a.close()
        b.close()


def test_geometry_cache_concurrent_creates(capi, cache_dir):
    """Contexts created from several threads at once (ctypes releases the
    interpreter lock during the call) with the cache on: every geometry is
    right, the cache ends with one valid file, no temporary file is left."""
    import threading
    cfg = synth.config1().replace(nrad1=3, nrad2=3)
    capi.bip_set_geometry_cache(None)
    want = _geometry(capi, cfg)
    capi.bip_set_geometry_cache(str(cache_dir))
    got, errors = [], []

    def worker():
        try:
            for _ in range(3):
                got.append(_geometry(capi, cfg))
        except Exception as e:                  # noqa: BLE001 -- reported below
            errors.append(e)

    threads = [threading.Thread(target=worker) for _ in range(6)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert not errors
    assert len(got) == 18 and all(_same(g, want) for g in got)
    files = os.listdir(cache_dir)
    assert len(files) == 1 and files[0].endswith(".bin"), files
    s0 = capi.bip_geometry_cache_stats()
    assert _same(_geometry(capi, cfg), want)
    assert _stats_since(capi, s0) == (1, 0, 0)
