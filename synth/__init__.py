"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This package holds no arithmetic of the BiP-PRISM method itself: it only
produces specimens (atom sites, projected potentials), transition-potential
samples on the per-atom windows, and scan lists, from a counter-based PRNG
(SplitMix64).  The paper's own workloads (FePt, SrTiO3, LAO/STO with GPAW or
hydrogenic transition potentials) are not available; these Gaussian-atom
crystals stand in for them with the same shape regime.
"""
from .prng import SplitMix64
from .configs import (Config, config1, config2, config3, config5, tiny_config, CONFIGS, config_to_json,
                      config_from_json, load_config)
from .specimen import Specimen, make_specimen, window_origin, site_window_inputs

__all__ = [
    "SplitMix64", "Config", "config1", "config2", "config3", "config5", "tiny_config",
    "CONFIGS", "config_to_json", "config_from_json", "load_config", "Specimen", "make_specimen", "window_origin", "site_window_inputs",
]
