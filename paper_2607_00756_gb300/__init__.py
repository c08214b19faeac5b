"""GB300 (sm_103a) BiP-PRISM core-loss map library.

The compute lives in libbip.so (C ABI, include/bip.h), built by
`paper_2607_00756_gb300.build.build()`.  `capi` is the ctypes binding with
the C names; `context.BipContext` is a small convenience wrapper over it.
Neither falls back to anything else when the library is missing.
"""

__all__ = ["build", "capi", "context"]
