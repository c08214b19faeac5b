"""ctypes binding of libbip.so -- argument marshalling only.

Every function named bip_* here calls the C entry point of the same name
(include/bip.h); tensors are passed as raw device pointers together with
the current CUDA stream of PyTorch.  The library must have been built (see
build.py); importing this module without it raises, so no call can silently
run anything but the CUDA path.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbip.so")

BIP_OK = 0
STATUS = {0: "BIP_OK", 1: "BIP_ERR_INVALID_ARG", 2: "BIP_ERR_SHAPE", 3: "BIP_ERR_OOM",
          4: "BIP_ERR_CUDA", 5: "BIP_ERR_TIMEOUT", 6: "BIP_ERR_UNSUPPORTED", 7: "BIP_ERR_NUMERIC"}
PREC = {"fp32": 0, "split_bf16": 1, "mixed": 2, "fp8": 3}
RECON = {"complex": 0, "magnitude": 1}


class BipConfig(ctypes.Structure):
    _fields_ = [("ny", ctypes.c_int32), ("nx", ctypes.c_int32),
                ("ly", ctypes.c_double), ("lx", ctypes.c_double),
                ("nz", ctypes.c_int32), ("dz", ctypes.c_double),
                ("e0", ctypes.c_double), ("alpha", ctypes.c_double), ("theta_det", ctypes.c_double),
                ("defocus", ctypes.c_double), ("cs", ctypes.c_double),
                ("fy", ctypes.c_int32), ("fx", ctypes.c_int32),
                ("nrad1", ctypes.c_int32), ("nang1", ctypes.c_int32),
                ("nrad2", ctypes.c_int32), ("nang2", ctypes.c_int32),
                ("win", ctypes.c_int32), ("recon", ctypes.c_int32), ("prec", ctypes.c_int32),
                ("dfy", ctypes.c_int32), ("dfx", ctypes.c_int32),
                ("cube_ky", ctypes.c_int32), ("cube_kx", ctypes.c_int32)]


class BipAtom(ctypes.Structure):
    _fields_ = [("y", ctypes.c_double), ("x", ctypes.c_double),
                ("slice", ctypes.c_int32), ("nch", ctypes.c_int32)]


class BipError(RuntimeError):
    def __init__(self, fn, status, text):
        super().__init__(f"{fn} -> {STATUS.get(status, status)}: {text}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libbip.so is not built ({LIB_PATH}); run paper_2607_00756_gb300/build.py")
    lib = ctypes.CDLL(LIB_PATH)
    P, I32, VP, D = ctypes.POINTER, ctypes.c_int32, ctypes.c_void_p, ctypes.c_double
    sig = {
        "bip_create": [P(BipConfig), P(VP)],
        "bip_destroy": [VP],
        "bip_query": [VP, P(I32), P(I32), P(I32), P(I32), P(I32)],
        "bip_get_geometry": [VP, VP, VP, VP, VP, VP, VP],
        "bip_get_config": [VP, P(BipConfig)],
        "bip_set_precision": [VP, I32],
        "bip_build_s1": [VP, VP, P(BipAtom), I32, VP],
        "bip_build_s2": [VP, VP, P(BipAtom), I32, VP],
        "bip_build": [VP, VP, P(BipAtom), I32, VP],
        "bip_coreloss_map": [VP, VP, P(D), I32, VP, VP],
        "bip_coreloss_sites": [VP, VP, P(D), I32, VP, VP],
        "bip_coreloss_cube": [VP, VP, VP, P(D), I32, VP, VP],
        "bip_cube_beams": [VP, P(I32), P(I32)],
        "bip_set_cube_memory": [VP, ctypes.c_int64],
        "bip_set_wait_limit": [VP, ctypes.c_int64],
        "bip_debug_fail_alloc": [ctypes.c_int64],
        "bip_debug_allocs": [P(ctypes.c_int64), P(ctypes.c_int64)],
        "bip_qeels_bins": [VP, I32, P(I32), P(I32)],
        "bip_coreloss_qeels": [VP, VP, P(D), I32, I32, VP, VP],
        "bip_copy_stash": [VP, I32, I32, VP, VP],
        "bip_site_windows": [VP, I32, VP, VP, VP],
        "bip_site_coupling": [VP, VP, I32, VP, VP],
        "bip_set_profiling": [VP, I32],
        "bip_build_s1_noalloc": [VP, VP, P(BipAtom), I32, VP, VP],
        "bip_get_profile": [VP, VP, VP],
        "bip_set_occupancy": [VP, P(D)],
        "bip_set_site_windows": [VP, P(I32), VP],
        "bip_set_capture_safe": [VP, I32],
        "bip_set_raster_eval": [VP, I32],
        "bip_check_errors": [VP, VP],
        "bip_set_launch": [VP, I32, I32],
        "bip_autotune": [VP, VP, P(D), I32, VP, VP, P(I32), P(I32), P(I32), P(D)],
        "bip_set_order": [VP, I32],
        "bip_set_aberrations": [VP, D, D, VP],
        "bip_coreloss_grad": [VP, VP, VP, P(D), I32, VP, VP, VP, P(D), VP, VP],
        "bip_set_geometry_cache": [ctypes.c_char_p],
        "bip_geometry_cache_stats": [P(ctypes.c_int64), P(ctypes.c_int64), P(ctypes.c_int64)],
        "bip_export_stash": [VP, I32, VP, ctypes.c_int64, VP],
        "bip_import_stash": [VP, I32, P(BipAtom), I32, VP, ctypes.c_int64, VP],
        "bip_set_check_finite": [VP, I32],
        "bip_mem_stats": [P(ctypes.c_int64), P(ctypes.c_int64), I32],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.bip_last_error.argtypes = [VP]
    lib.bip_last_error.restype = ctypes.c_char_p
    return lib


_lib = _load()


def lib():
    return _lib


def _check(fn, ctx, status):
    if status != BIP_OK:
        text = _lib.bip_last_error(ctx).decode() if ctx else ""
        raise BipError(fn, status, text)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(int(stream))


def _dev(t, dtype=None, name="tensor"):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}")
    return ctypes.c_void_p(t.data_ptr())


def make_config(cfg, prec=None, recon=None):
    """bip_config from any object with the configuration's attributes."""
    c = BipConfig()
    for name, _ in BipConfig._fields_:
        if name in ("recon", "prec"):
            continue
        optional = ("dfy", "dfx", "cube_ky", "cube_kx")
        setattr(c, name, getattr(cfg, name, 0) if name in optional else getattr(cfg, name))
    r = recon if recon is not None else getattr(cfg, "recon", "magnitude")
    p = prec if prec is not None else getattr(cfg, "prec", "fp32")
    c.recon = RECON[r] if isinstance(r, str) else int(r)
    c.prec = PREC[p] if isinstance(p, str) else int(p)
    return c


def make_atoms(atoms, nch):
    """bip_atom array from [n,3] (y, x, slice) and [n] channel counts."""
    atoms = np.asarray(atoms, dtype=np.float64).reshape(-1, 3)
    nch = np.asarray(nch).reshape(-1)
    arr = (BipAtom * len(atoms))()
    view = np.ctypeslib.as_array(arr)          # structured view of the same memory
    view["y"] = atoms[:, 0]
    view["x"] = atoms[:, 1]
    view["slice"] = atoms[:, 2].astype(np.int32)
    view["nch"] = nch.astype(np.int32)
    return arr


# ---- the C entry points, by name -------------------------------------------

def bip_create(cfg_struct):
    ctx = ctypes.c_void_p()
    st = _lib.bip_create(ctypes.byref(cfg_struct), ctypes.byref(ctx))
    _check("bip_create", None, st)
    return ctx


def bip_destroy(ctx):
    _check("bip_destroy", None, _lib.bip_destroy(ctx))


def bip_query(ctx):
    v = [ctypes.c_int32() for _ in range(5)]
    _check("bip_query", ctx, _lib.bip_query(ctx, *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def bip_get_geometry(ctx):
    B, nd, bp1, bp2, _ = bip_query(ctx)
    hb = np.zeros((B, 2), np.int32)
    hd = np.zeros((nd, 2), np.int32)
    p1 = np.zeros(bp1, np.int32)
    p2 = np.zeros(bp2, np.int32)
    w1 = np.zeros((B, bp1), np.float64)
    w2 = np.zeros((nd, bp2), np.float64)
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    _check("bip_get_geometry", ctx, _lib.bip_get_geometry(ctx, ptr(hb), ptr(hd), ptr(p1), ptr(p2), ptr(w1), ptr(w2)))
    return dict(h_beam=hb, h_det=hd, p1=p1, p2=p2, w1=w1, w2=w2)


def bip_get_config(ctx):
    """The context's configuration (a BipConfig)."""
    c = BipConfig()
    _check("bip_get_config", ctx, _lib.bip_get_config(ctx, ctypes.byref(c)))
    return c


def bip_set_precision(ctx, prec):
    p = PREC[prec] if isinstance(prec, str) else int(prec)
    _check("bip_set_precision", ctx, _lib.bip_set_precision(ctx, p))


def bip_build_s1(ctx, V, atoms_arr, stream=None):
    import torch
    _check("bip_build_s1", ctx, _lib.bip_build_s1(ctx, _dev(V, torch.float32, "V"), atoms_arr,
                                                   len(atoms_arr), _stream(stream)))


def bip_build_s2(ctx, V, atoms_arr, stream=None):
    import torch
    _check("bip_build_s2", ctx, _lib.bip_build_s2(ctx, _dev(V, torch.float32, "V"), atoms_arr,
                                                   len(atoms_arr), _stream(stream)))


def bip_build(ctx, V, atoms_arr, stream=None):
    """Both builds, the S2 sweep on the context's side stream."""
    import torch
    _check("bip_build", ctx, _lib.bip_build(ctx, _dev(V, torch.float32, "V"), atoms_arr, len(atoms_arr),
                                             _stream(stream)))


def _scans(scans):
    s = np.ascontiguousarray(scans, dtype=np.float64)
    if s.ndim != 2 or s.shape[1] != 2:
        raise ValueError("scans must be [P, 2]")
    return s, s.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def noalloc_stash_shape(ctx, atoms_arr):
    """Shape [n_sites, Bp1, win, win] the caller's stash must have for
    bip_build_s1_noalloc: n_sites counts the atoms with nch > 0, Bp1 and win
    come from the context."""
    n_sites = sum(1 for a in atoms_arr if a.nch > 0)
    bp1 = bip_query(ctx)[2]
    win = bip_get_config(ctx).win
    return (n_sites, bp1, win, win)


def bip_build_s1_noalloc(ctx, V, atoms_arr, stash, stream=None):
    """S1 build into the caller's `stash` [n_sites, Bp1, win, win] complex64
    with no device allocation (scratch in the library's static array).  The
    kernels write every element of that shape, so any other shape is
    refused here, before a launch (the C entry point cannot see the
    buffer's size)."""
    import torch
    want = noalloc_stash_shape(ctx, atoms_arr)
    if tuple(stash.shape) != want:
        raise ValueError(f"stash must have shape {list(want)} (n_sites, Bp1, win, win), got {list(stash.shape)}")
    _check("bip_build_s1_noalloc", ctx,
           _lib.bip_build_s1_noalloc(ctx, _dev(V, torch.float32, "V"), atoms_arr, len(atoms_arr),
                                     _dev(stash, torch.complex64, "stash"), _stream(stream)))
    return stash


def bip_coreloss_map(ctx, H, scans, out, stream=None):
    import torch
    s, sp = _scans(scans)
    _check("bip_coreloss_map", ctx, _lib.bip_coreloss_map(ctx, _dev(H, torch.complex64, "H"), sp, len(s),
                                                           _dev(out, torch.float64, "out"), _stream(stream)))
    return out


def bip_coreloss_sites(ctx, H, scans, out, stream=None):
    import torch
    s, sp = _scans(scans)
    _check("bip_coreloss_sites", ctx, _lib.bip_coreloss_sites(ctx, _dev(H, torch.complex64, "H"), sp, len(s),
                                                               _dev(out, torch.float32, "out"), _stream(stream)))
    return out


def bip_coreloss_cube(ctx, V, H, scans, out, stream=None):
    import torch
    s, sp = _scans(scans)
    _check("bip_coreloss_cube", ctx, _lib.bip_coreloss_cube(ctx, _dev(V, torch.float32, "V"),
                                                             _dev(H, torch.complex64, "H"), sp, len(s),
                                                             _dev(out, torch.float32, "out"), _stream(stream)))
    return out


def bip_cube_beams(ctx):
    """The cube's complete basis, [n_cube, 2] int32 (h_y, h_x)."""
    n = ctypes.c_int32(0)
    _check("bip_cube_beams", ctx, _lib.bip_cube_beams(ctx, ctypes.byref(n), None))
    h = np.zeros((n.value, 2), dtype=np.int32)
    _check("bip_cube_beams", ctx, _lib.bip_cube_beams(ctx, ctypes.byref(n),
                                                       h.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
    return h


def bip_set_wait_limit(ctx, ns):
    _check("bip_set_wait_limit", ctx, _lib.bip_set_wait_limit(ctx, int(ns)))


def bip_debug_fail_alloc(k):
    _check("bip_debug_fail_alloc", None, _lib.bip_debug_fail_alloc(int(k)))


def bip_debug_allocs():
    """(live device allocations of the library, allocations made since the
    last bip_debug_fail_alloc)."""
    live, made = ctypes.c_int64(0), ctypes.c_int64(0)
    _check("bip_debug_allocs", None, _lib.bip_debug_allocs(ctypes.byref(live), ctypes.byref(made)))
    return live.value, made.value


def bip_set_geometry_cache(directory):
    """Directory of the on-disk geometry cache (None or "": off)."""
    d = None if not directory else os.fsencode(directory)
    _check("bip_set_geometry_cache", None, _lib.bip_set_geometry_cache(d))


def bip_geometry_cache_stats():
    """(hits, misses, rejected) of the geometry cache since the process started."""
    v = [ctypes.c_int64(0) for _ in range(3)]
    _check("bip_geometry_cache_stats", None, _lib.bip_geometry_cache_stats(*[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def _buffer(a, name):
    """(pointer, bytes) of a contiguous complex64 CUDA tensor or host array."""
    if hasattr(a, "data_ptr"):
        import torch
        if a.dtype != torch.complex64 or not a.is_contiguous():
            raise ValueError(f"{name} must be a contiguous complex64 tensor")
        return ctypes.c_void_p(a.data_ptr()), a.numel() * 8
    if not isinstance(a, np.ndarray) or a.dtype != np.complex64 or not a.flags["C_CONTIGUOUS"]:
        raise ValueError(f"{name} must be a C-contiguous complex64 array")
    return a.ctypes.data_as(ctypes.c_void_p), a.nbytes


def stash_shape(ctx, which):
    """[n_sites, Bp, win, win] of the built stash `which` (1: S1, 2: S2)."""
    _, _, bp1, bp2, n_sites = bip_query(ctx)
    win = bip_get_config(ctx).win
    return (n_sites, bp1 if which == 1 else bp2, win, win)


def bip_export_stash(ctx, which, dst, stream=None):
    """Whole stash of S1 (which=1) or S2 (2) into `dst` (CUDA tensor or host
    array, complex64, exactly the stash's size)."""
    ptr, nbytes = _buffer(dst, "dst")
    _check("bip_export_stash", ctx, _lib.bip_export_stash(ctx, int(which), ptr, nbytes, _stream(stream)))
    return dst


def bip_import_stash(ctx, which, atoms_arr, src, stream=None):
    """Restores a stash exported from a context of the same configuration,
    for the sites of `atoms_arr`; afterwards S<which> counts as built."""
    ptr, nbytes = _buffer(src, "src")
    _check("bip_import_stash", ctx, _lib.bip_import_stash(ctx, int(which), atoms_arr, len(atoms_arr), ptr, nbytes,
                                                           _stream(stream)))


def bip_set_check_finite(ctx, on):
    _check("bip_set_check_finite", ctx, _lib.bip_set_check_finite(ctx, 1 if on else 0))


def bip_mem_stats(reset_peak=False):
    """(live bytes, peak bytes) of the library's device workspaces."""
    live, peak = ctypes.c_int64(0), ctypes.c_int64(0)
    _check("bip_mem_stats", None, _lib.bip_mem_stats(ctypes.byref(live), ctypes.byref(peak), 1 if reset_peak else 0))
    return live.value, peak.value


def bip_set_cube_memory(ctx, nbytes):
    _check("bip_set_cube_memory", ctx, _lib.bip_set_cube_memory(ctx, int(nbytes)))


def bip_qeels_bins(ctx, axis):
    """Bin components h (ascending) of the qEELS output along `axis`."""
    n = ctypes.c_int32(0)
    _check("bip_qeels_bins", ctx, _lib.bip_qeels_bins(ctx, int(axis), ctypes.byref(n), None))
    h = np.zeros(n.value, dtype=np.int32)
    _check("bip_qeels_bins", ctx, _lib.bip_qeels_bins(ctx, int(axis), ctypes.byref(n),
                                                       h.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
    return h


def bip_coreloss_qeels(ctx, H, scans, axis, out, stream=None):
    import torch
    s, sp = _scans(scans)
    _check("bip_coreloss_qeels", ctx, _lib.bip_coreloss_qeels(ctx, _dev(H, torch.complex64, "H"), sp, len(s),
                                                               int(axis), _dev(out, torch.float32, "out"),
                                                               _stream(stream)))
    return out


def bip_copy_stash(ctx, which, site, out, stream=None):
    import torch
    _check("bip_copy_stash", ctx, _lib.bip_copy_stash(ctx, which, site, _dev(out, torch.complex64, "out"),
                                                       _stream(stream)))
    return out


def bip_site_windows(ctx, site, s1_out, s2_out, stream=None):
    import torch
    _check("bip_site_windows", ctx, _lib.bip_site_windows(ctx, site, _dev(s1_out, torch.complex64, "s1_out"),
                                                           _dev(s2_out, torch.complex64, "s2_out"),
                                                           _stream(stream)))
    return s1_out, s2_out


def bip_site_coupling(ctx, H, site, out, stream=None):
    import torch
    _check("bip_site_coupling", ctx, _lib.bip_site_coupling(ctx, _dev(H, torch.complex64, "H"), site,
                                                             _dev(out, torch.complex64, "out"), _stream(stream)))
    return out


def bip_set_capture_safe(ctx, on):
    _check("bip_set_capture_safe", ctx, _lib.bip_set_capture_safe(ctx, 1 if on else 0))


def bip_set_raster_eval(ctx, on):
    _check("bip_set_raster_eval", ctx, _lib.bip_set_raster_eval(ctx, 1 if on else 0))


def bip_check_errors(ctx, stream=None):
    _check("bip_check_errors", ctx, _lib.bip_check_errors(ctx, _stream(stream)))


def bip_set_launch(ctx, sites_per_batch=0, coupling_tile=0):
    _check("bip_set_launch", ctx, _lib.bip_set_launch(ctx, int(sites_per_batch), int(coupling_tile)))


def bip_autotune(ctx, H, scans, out, stream=None):
    """Times launch choices on this map; returns (sites per batch, coupling
    tile width (0: built-in), contraction order (0 Gram, 1 beam), ms per
    map) and keeps them in the context."""
    import torch
    s, sp = _scans(scans)
    sb, cw, od, ms = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_double(0.0)
    _check("bip_autotune", ctx, _lib.bip_autotune(ctx, _dev(H, torch.complex64, "H"), sp, len(s),
                                                   _dev(out, torch.float64, "out"), _stream(stream),
                                                   ctypes.byref(sb), ctypes.byref(cw), ctypes.byref(od),
                                                   ctypes.byref(ms)))
    return sb.value, cw.value, od.value, ms.value


def bip_set_order(ctx, order):
    _check("bip_set_order", ctx, _lib.bip_set_order(ctx, int(order)))


def bip_set_occupancy(ctx, occ):
    """Per-site occupancies weighting the site sum (None: all 1)."""
    if occ is None:
        _check("bip_set_occupancy", ctx, _lib.bip_set_occupancy(ctx, None))
        return
    o = np.ascontiguousarray(occ, dtype=np.float64)
    _check("bip_set_occupancy", ctx, _lib.bip_set_occupancy(ctx, o.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))


def bip_set_site_windows(ctx, win, stream=None):
    """Windows of their own for the built sites (None: all at the context's win)."""
    if win is None:
        _check("bip_set_site_windows", ctx, _lib.bip_set_site_windows(ctx, None, _stream(stream)))
        return
    w = np.ascontiguousarray(win, dtype=np.int32)
    _check("bip_set_site_windows", ctx,
           _lib.bip_set_site_windows(ctx, w.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _stream(stream)))


def bip_set_aberrations(ctx, defocus, cs, stream=None):
    _check("bip_set_aberrations", ctx, _lib.bip_set_aberrations(ctx, float(defocus), float(cs), _stream(stream)))


def bip_coreloss_grad(ctx, H, scans, dL_dI, d_occ=None, d_H=None, aberr=False, V=None, d_V=None, stream=None):
    """Reverse pass of a map loss: fills d_occ [n_sites] float64, d_H (H's
    shape, complex64: dL/dRe H + i dL/dIm H) and d_V ([nz, ny, nx] float32,
    needs V) when given; returns (dL/d defocus, dL/d Cs) when aberr, else None."""
    import torch
    s, sp = _scans(scans)
    ab = np.zeros(2, dtype=np.float64)
    abp = ab.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if aberr else None
    _check("bip_coreloss_grad", ctx, _lib.bip_coreloss_grad(
        ctx, _dev(V, torch.float32, "V"), _dev(H, torch.complex64, "H"), sp, len(s),
        _dev(dL_dI, torch.float64, "dL_dI"), _dev(d_occ, torch.float64, "d_occ"), _dev(d_H, torch.complex64, "d_H"),
        abp, _dev(d_V, torch.float32, "d_V"), _stream(stream)))
    return (float(ab[0]), float(ab[1])) if aberr else None


N_STAGES = 8
STAGES = ["ms_row", "ms_col", "gather", "coupling", "gram", "quadform", "reduce", "transmission"]


def bip_set_profiling(ctx, on, stages=None):
    """Time every stage (on true), none (on false), or only `stages` (names)."""
    mask = 0
    if on:
        mask = -1 if stages is None else sum(1 << STAGES.index(n) for n in stages)
    _check("bip_set_profiling", ctx, _lib.bip_set_profiling(ctx, mask))


def bip_get_profile(ctx):
    ms = np.zeros(N_STAGES, np.float64)
    n = np.zeros(N_STAGES, np.int64)
    _check("bip_get_profile", ctx, _lib.bip_get_profile(ctx, ms.ctypes.data_as(ctypes.c_void_p),
                                                         n.ctypes.data_as(ctypes.c_void_p)))
    return {STAGES[i]: (float(ms[i]), int(n[i])) for i in range(N_STAGES)}


def bip_last_error(ctx):
    return _lib.bip_last_error(ctx).decode()
