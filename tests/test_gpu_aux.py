"""Auxiliary subsystems on the GPU, through the C ABI: builds saved and
restored for map-only reruns (bit-identical maps, qEELS and gradients), the
optional scan of outputs for NaN / Inf, and the library's device-memory
accounting."""
import numpy as np
import pytest

import synth
from oracle import bip as obip

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2607_00756_gb300 import build
    build.build()
    from paper_2607_00756_gb300 import capi
    from paper_2607_00756_gb300.context import BipContext
    return capi, BipContext


def _inputs(cfg, sp):
    dev = torch.device("cuda:0")
    return (torch.tensor(sp.V, dtype=torch.float32, device=dev),
            torch.tensor(sp.H, dtype=torch.complex64, device=dev))


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_saved_builds_rerun_the_map_exactly(lib, tmp_path, prec):
    """A map, the per-site contributions and qEELS from builds restored in
    a fresh context -- through a file and through device tensors -- are
    bit-identical to those of the context that built them, and the map
    matches the oracle."""
    capi, BipContext = lib
    cfg = synth.config1().replace(dfx=1)          # qEELS along q_x needs dfx = 1
    sp = synth.make_specimen(cfg)
    V, H = _inputs(cfg, sp)
    a = BipContext(cfg, prec=prec)
    try:
        a.build(V, sp.atoms, sp.nch)
        m0 = a.map(H, sp.scans).cpu().numpy()
        p0 = a.sites(H, sp.scans).cpu().numpy()
        q0 = a.qeels(H, sp.scans, 1)[1].cpu().numpy()
        path = tmp_path / "builds.npz"
        a.save_builds(path)
        dev = {w: torch.empty(capi.stash_shape(a.ctx, w), dtype=torch.complex64, device="cuda")
               for w in (1, 2)}
        for w in (1, 2):
            capi.bip_export_stash(a.ctx, w, dev[w])
        torch.cuda.synchronize()
    finally:
        a.close()

    b = BipContext(cfg, prec=prec)
    try:
        b.load_builds(path)
        assert b.n_sites == len(sp.nch[sp.nch > 0])
        m1 = b.map(H, sp.scans).cpu().numpy()
        p1 = b.sites(H, sp.scans).cpu().numpy()
        q1 = b.qeels(H, sp.scans, 1)[1].cpu().numpy()
    finally:
        b.close()
    assert np.array_equal(m0, m1) and np.array_equal(p0, p1) and np.array_equal(q0, q1)

    c = BipContext(cfg, prec=prec)
    try:
        atoms = capi.make_atoms(sp.atoms, sp.nch)
        c._atoms = atoms
        for w in (1, 2):
            capi.bip_import_stash(c.ctx, w, atoms, dev[w])
        m2 = c.map(H, sp.scans).cpu().numpy()
    finally:
        c.close()
    assert np.array_equal(m0, m2)

    ref = obip.bip_map(obip.make_problem(sp)).map
    tol = 1e-4 if prec == "fp32" else 1e-3
    assert np.linalg.norm(m0 - ref) / np.linalg.norm(ref) < tol


def test_saved_builds_give_the_same_gradient(lib, tmp_path):
    """The reverse pass (including the adjoint sweeps for dL/dV) after
    restored builds equals the one after the builds themselves."""
    capi, BipContext = lib
    cfg = synth.config1()
    sp = synth.make_specimen(cfg)
    V, H = _inputs(cfg, sp)
    g = torch.tensor(np.random.default_rng(3).standard_normal(len(sp.scans)), dtype=torch.float64, device="cuda")
    out = []
    for restored in (False, True):
        ctx = BipContext(cfg, prec="fp32")
        try:
            if restored:
                ctx.load_builds(tmp_path / "b.npz")
            else:
                ctx.build(V, sp.atoms, sp.nch)
                ctx.save_builds(tmp_path / "b.npz")
            r = ctx.grad(H, sp.scans, g, V=V)
            out.append({k: (v.cpu().numpy() if hasattr(v, "cpu") else np.asarray(v)) for k, v in r.items()})
        finally:
            ctx.close()
    assert out[0].keys() == out[1].keys() and "V" in out[0]
    for k in out[0]:
        assert np.array_equal(out[0][k], out[1][k]), k


def test_finite_check_reports_nan_outputs(lib):
    """With the check on, a NaN in one site's transition potential makes the
    map and the per-site call return BIP_ERR_NUMERIC (the outputs still
    written); with it off the call succeeds and the NaN is in the map; a
    clean H passes the check."""
    capi, BipContext = lib
    cfg = synth.config1()
    sp = synth.make_specimen(cfg)
    V, H = _inputs(cfg, sp)
    bad = H.clone()
    bad.view(-1)[5] = complex(float("nan"), 0.0)
    ctx = BipContext(cfg, prec="mixed")
    try:
        ctx.build(V, sp.atoms, sp.nch)
        clean = ctx.map(H, sp.scans).cpu().numpy()
        m = ctx.map(bad, sp.scans).cpu().numpy()
        assert np.isnan(m).any()
        ctx.set_check_finite(True)
        assert np.array_equal(ctx.map(H, sp.scans).cpu().numpy(), clean)
        out = torch.empty(len(sp.scans), dtype=torch.float64, device="cuda")
        with pytest.raises(capi.BipError) as e:
            capi.bip_coreloss_map(ctx.ctx, bad, sp.scans, out)
        assert e.value.status == 7 and "NaN or infinite" in str(e.value)
        assert np.isnan(out.cpu().numpy()).any()
        with pytest.raises(capi.BipError) as e:
            ctx.sites(bad, sp.scans)
        assert e.value.status == 7
        ctx.set_check_finite(False)
        assert np.array_equal(ctx.map(H, sp.scans).cpu().numpy(), clean)
    finally:
        ctx.close()


def test_memory_accounting(lib):
    """bip_mem_stats follows the contexts' workspaces: a build and a map
    raise the live bytes by at least the two stashes, destroying the
    context gives them back, and the peak covers them."""
    capi, BipContext = lib
    cfg = synth.config1()
    sp = synth.make_specimen(cfg)
    V, H = _inputs(cfg, sp)
    live0, _ = capi.bip_mem_stats(reset_peak=True)
    ctx = BipContext(cfg, prec="mixed")
    try:
        ctx.build(V, sp.atoms, sp.nch)
        ctx.map(H, sp.scans)
        torch.cuda.synchronize()
        live1, peak1 = capi.bip_mem_stats()
        n_sites, win = int((sp.nch > 0).sum()), cfg.win
        stashes = n_sites * (ctx.Bp1 + ctx.Bp2) * win * win * 8
        assert live1 - live0 >= stashes
        assert peak1 >= live1
    finally:
        ctx.close()
    live2, peak2 = capi.bip_mem_stats()
    assert live2 == live0 and peak2 >= peak1


def test_nvtx_stage_ranges(lib, tmp_path):
    """Under an attached NVTX tool, a build and a map show their public
    calls and, nested inside them, one range per stage launch."""
    import os
    import subprocess
    import sys
    import textwrap
    import nvtx_tool
    so = nvtx_tool.compile_tool(str(tmp_path))
    record = tmp_path / "ranges.txt"
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = textwrap.dedent(f"""
        import sys
        sys.path.insert(0, {root!r})
        import torch
        import synth
        from paper_2607_00756_gb300.context import BipContext
        cfg = synth.config1()
        sp = synth.make_specimen(cfg)
        V = torch.tensor(sp.V, dtype=torch.float32, device="cuda")
        H = torch.tensor(sp.H, dtype=torch.complex64, device="cuda")
        ctx = BipContext(cfg, prec="mixed")
        ctx.build(V, sp.atoms, sp.nch)
        ctx.map(H, sp.scans)
        torch.cuda.synchronize()
        ctx.close()
    """)
    env = dict(os.environ, NVTX_INJECTION64_PATH=so, NVTX_RECORD=str(record))
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr
    lines = record.read_text().splitlines()
    assert nvtx_tool.nesting_ok(lines)
    names = [ln[5:] for ln in lines if ln.startswith("push ")]
    for n in ("bip_create", "bip_build", "bip_coreloss_map", "bip:transmission",
              "bip:ms_row", "bip:ms_col", "bip:reconstruct", "bip:coupling", "bip:gram", "bip:quadform",
              "bip:reduce"):
        assert n in names, n
    # stage ranges open only inside a public call's range
    depth, top = 0, []
    for ln in lines:
        if ln.startswith("push "):
            if ln[5:].startswith("bip:"):
                assert depth >= 1 and top[-1].startswith("bip_"), ln
            top.append(ln[5:])
            depth += 1
        else:
            top.pop()
            depth -= 1


@pytest.mark.parametrize("grid", [128, 512])
def test_combined_build_equals_separate_builds(lib, grid):
    """bip_build (S2's sweep on the context's side stream, beside S1's)
    leaves stashes bit-identical to bip_build_s1 followed by bip_build_s2,
    and the same map; a second combined build on the same context too."""
    capi, BipContext = lib
    if grid == 128:
        cfg = synth.config1().replace(ion_slices=(0, 5), ion_cells=(0, 3))   # sites in every plane
    else:
        cfg = synth.config1().replace(name="grid512", ny=512, nx=512, ly=40.0, lx=40.0, cells_y=16, cells_x=16,
                                      nz=6, e0=300e3, alpha=0.020, theta_det=0.030, fy=8, fx=8,
                                      ion_slices=(1, 5), ion_cells=(7, 9))
    sp = synth.make_specimen(cfg)
    V, H = _inputs(cfg, sp)
    atoms = capi.make_atoms(sp.atoms, sp.nch)
    out = {}
    for mode in ("separate", "combined"):
        ctx = BipContext(cfg, prec="mixed")
        try:
            if mode == "separate":
                capi.bip_build_s1(ctx.ctx, V, atoms)
                capi.bip_build_s2(ctx.ctx, V, atoms)
                ctx.n_sites = capi.bip_query(ctx.ctx)[4]
                ctx._atoms = atoms
            else:
                ctx.build(V, sp.atoms, sp.nch)
                ctx.build(V, sp.atoms, sp.nch)
            st = []
            for w in (1, 2):
                t = torch.empty(capi.stash_shape(ctx.ctx, w), dtype=torch.complex64, device="cuda")
                capi.bip_export_stash(ctx.ctx, w, t)
                st.append(t)
            m = ctx.map(H, sp.scans)
            torch.cuda.synchronize()
            out[mode] = (st, m.cpu().numpy())
        finally:
            ctx.close()
    (s_a, m_a), (s_b, m_b) = out["separate"], out["combined"]
    assert s_a[0].shape[0] >= 2
    assert torch.equal(s_a[0], s_b[0]) and torch.equal(s_a[1], s_b[1])
    assert np.array_equal(m_a, m_b)
