"""Failure detection on the GPU without a GPU fault: a device wait that
gives up (a give-up limit so short that the first wait on an unfinished
copy or product runs out) must come back as BIP_ERR_TIMEOUT with the
context still usable; an allocation that fails (injected on the host) must
come back as BIP_ERR_OOM at every allocation of the pipeline, leak nothing
and leave the context usable."""
import numpy as np
import pytest

import synth
from oracle import bip as obip

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2607_00756_gb300 import build
    build.build()
    from paper_2607_00756_gb300 import capi
    from paper_2607_00756_gb300.context import BipContext
    cfg = synth.config1()
    sp = synth.make_specimen(cfg)
    want = obip.bip_map(obip.make_problem(sp)).map
    dev = torch.device("cuda:0")
    V = torch.tensor(sp.V, dtype=torch.float32, device=dev)
    H = torch.tensor(sp.H, dtype=torch.complex64, device=dev)
    return capi, BipContext, cfg, sp, want, V, H


@pytest.mark.parametrize("order", [0, 1])
def test_wait_gives_up_as_timeout_and_context_recovers(env, order):
    """Mixed path (tcgen05 reconstruction, coupling, Gram; order 1: the
    cube kernel's beam order) with a 1 ns give-up limit: the call returns
    BIP_ERR_TIMEOUT; the same context with the default limit, and a fresh
    one, then give the right map."""
    capi, BipContext, cfg, sp, want, V, H = env
    ctx = BipContext(cfg, prec="mixed")
    try:
        ctx.build(V, sp.atoms, sp.nch)
        ctx.set_order(order)
        capi.bip_set_wait_limit(ctx.ctx, 1)
        with pytest.raises(capi.BipError) as e:
            ctx.map(H, sp.scans)
        assert capi.STATUS[e.value.status] == "BIP_ERR_TIMEOUT"
        assert "device timeout" in str(e.value)
        capi.bip_set_wait_limit(ctx.ctx, 0)
        m = ctx.map(H, sp.scans).cpu().numpy()
        assert rel(m, want) < 1e-3
    finally:
        ctx.close()
    ctx = BipContext(cfg, prec="mixed")
    try:
        ctx.build(V, sp.atoms, sp.nch)
        assert rel(ctx.map(H, sp.scans).cpu().numpy(), want) < 1e-3
    finally:
        ctx.close()


def test_wait_limit_rejects_negative(env):
    capi, BipContext, cfg, *_ = env
    ctx = BipContext(cfg)
    try:
        with pytest.raises(capi.BipError):
            capi.bip_set_wait_limit(ctx.ctx, -1)
    finally:
        ctx.close()


def _pipeline(ctx, env):
    capi, BipContext, cfg, sp, want, V, H = env
    ctx.build(V, sp.atoms, sp.nch)
    m = ctx.map(H, sp.scans)
    ctx.cube(V, H, sp.scans)
    g = torch.ones(len(sp.scans), dtype=torch.float64, device=H.device)
    ctx.grad(H, sp.scans, g, V=V)
    torch.cuda.synchronize()
    return m.cpu().numpy()


@pytest.mark.parametrize("prec", ["mixed", "fp32"])
def test_every_allocation_failure_is_oom_and_leaks_nothing(env, prec):
    """Builds, map, cube and reverse pass: the k-th device allocation made
    to fail, for every k the pipeline makes, returns BIP_ERR_OOM; after
    bip_destroy the library holds no more allocations than before; the
    failed context, retried without the injection, gives the right map."""
    capi, BipContext, cfg, sp, want, V, H = env
    live0, _ = capi.bip_debug_allocs()
    capi.bip_debug_fail_alloc(0)
    ctx = BipContext(cfg, prec=prec)
    _pipeline(ctx, env)
    _, n_allocs = capi.bip_debug_allocs()
    ctx.close()
    assert capi.bip_debug_allocs()[0] == live0
    assert n_allocs >= 10
    try:
        for k in range(1, n_allocs + 1):
            ctx = BipContext(cfg, prec=prec)
            try:
                capi.bip_debug_fail_alloc(k)
                with pytest.raises(capi.BipError) as e:
                    _pipeline(ctx, env)
                assert capi.STATUS[e.value.status] == "BIP_ERR_OOM", (k, str(e.value))
                if k in (1, n_allocs // 2, n_allocs):
                    capi.bip_debug_fail_alloc(0)
                    m = _pipeline(ctx, env)
                    assert rel(m, want) < (1e-4 if prec == "fp32" else 1e-3), k
            finally:
                ctx.close()
            assert capi.bip_debug_allocs()[0] == live0, k
    finally:
        capi.bip_debug_fail_alloc(0)
