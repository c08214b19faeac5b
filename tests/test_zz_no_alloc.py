"""bip_build_s1_noalloc: the S1 build for callers that cannot allocate
device memory (a host framework that owns every allocation, a fixed memory
budget, or a pipeline that cannot let cudaMalloc/cudaFree synchronize the
device).  Its parent columns live in the library's static scratch array and
its windows go to a buffer the caller owns; the result must equal the
regular bip_build_s1 stash on two calls in a row.

This file is collected last on purpose: when it fails, a run that stops at
the first failure has already run every other test."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def capi():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2607_00756_gb300 import build
    build.build()
    from paper_2607_00756_gb300 import capi as c
    return c


def test_noalloc_s1_matches_regular_build(capi):
    cfg = synth.config1().replace(ion_slices=(0, 5), ion_cells=(0, 3))   # sites in every plane
    sp = synth.make_specimen(cfg)
    dev = torch.device("cuda:0")
    V = torch.tensor(sp.V, dtype=torch.float32, device=dev)
    atoms = capi.make_atoms(sp.atoms, sp.nch)

    # regular path: the context allocates its own stash
    ctx = capi.bip_create(capi.make_config(cfg))
    try:
        capi.bip_build_s1(ctx, V, atoms)
        B, nd, bp1, bp2, n_sites = capi.bip_query(ctx)
        ref = torch.empty((n_sites, bp1, cfg.win, cfg.win), dtype=torch.complex64, device=dev)
        for k in range(n_sites):
            capi.bip_copy_stash(ctx, 1, k, ref[k])
        torch.cuda.synchronize()
        want = ref.cpu().numpy()
    finally:
        capi.bip_destroy(ctx)

    # allocation-free path on a fresh context (bip_create touches no GPU)
    ctx2 = capi.bip_create(capi.make_config(cfg))
    try:
        out = torch.empty_like(ref)
        for call in range(2):
            out.fill_(complex(float("nan"), float("nan")))        # every entry must be written
            torch.cuda.synchronize()
            free_before, _ = torch.cuda.mem_get_info()
            capi.bip_build_s1_noalloc(ctx2, V, atoms, out)
            torch.cuda.synchronize()
            free_after, _ = torch.cuda.mem_get_info()
            # the first call on the device looks up the static array, and the
            # driver may place the array (32 MiB) in memory at that moment;
            # every later call must take no device memory at all
            limit = (32 << 20) + (1 << 20) if call == 0 else (1 << 20)
            assert free_before - free_after < limit, call
            got = out.cpu().numpy()
            assert np.all(np.isfinite(got)), call
            assert np.max(np.abs(got - want)) <= 2e-5 * np.max(np.abs(want)), call
    finally:
        capi.bip_destroy(ctx2)


def test_noalloc_rejects_oversized_request(capi):
    """61 parent columns of 512^2 need 128 MB, beyond the 32 MiB scratch."""
    cfg = synth.config2()
    ctx = capi.bip_create(capi.make_config(cfg))
    try:
        atoms = capi.make_atoms(np.array([[20.0, 20.0, 3.0]]), np.array([3]))
        V = torch.zeros((cfg.nz, cfg.ny, cfg.nx), dtype=torch.float32, device="cuda:0")
        out = torch.empty((1, 61, cfg.win, cfg.win), dtype=torch.complex64, device="cuda:0")
        with pytest.raises(capi.BipError) as e:
            capi.bip_build_s1_noalloc(ctx, V, atoms, out)
        assert capi.STATUS[e.value.status] == "BIP_ERR_SHAPE"
        assert "static scratch" in str(e.value)
    finally:
        capi.bip_destroy(ctx)
