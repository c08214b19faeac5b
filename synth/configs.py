"""Workload configurations (synthetic Gaussian-atom crystals).

Lengths in Angstrom, angles in rad, energies in eV, potentials in V*Angstrom.
Slices are indexed from 0; "the third slice" of a five-slice cell is index 2.
"""
import json
from dataclasses import asdict, dataclass, field, fields, replace
from typing import Tuple


@dataclass(frozen=True)
class Config:
    name: str
    # simulation grid and optics (the fields of the C-ABI bip_config)
    ny: int
    nx: int
    ly: float
    lx: float
    nz: int
    dz: float
    e0: float
    alpha: float
    theta_det: float
    defocus: float = 0.0
    cs: float = 0.0
    fy: int = 1
    fx: int = 1
    # detector-side subsampling of the beams S2 carries (0: fy, fx); qEELS
    # along x wants dfx = 1, along y dfy = 1
    dfy: int = 0
    dfx: int = 0
    # the 4D cube's output basis: 0, 0 -- every beam inside the detector
    # disc; else a box of cube_ky x cube_kx k-pixels centred on the zero beam
    cube_ky: int = 0
    cube_kx: int = 0
    nrad1: int = 2
    nang1: int = 6
    nrad2: int = 2
    nang2: int = 6
    win: int = 64
    recon: str = "magnitude"        # "magnitude" | "complex"
    prec: str = "fp32"              # "fp32" | "split_bf16"
    # specimen: one atom per cell per slice, at the cell centre plus jitter
    cells_y: int = 4
    cells_x: int = 4
    cell_a: float = 2.5
    atom_peak: float = 30.0
    atom_sigma: float = 0.3
    jitter: float = 0.05
    seed: int = 0
    # ionization: (slice range [s0, s1), cell range [c0, c1) on both axes)
    ion_slices: Tuple[int, ...] = (2, 3)        # (first, end[, stride])
    ion_cells: Tuple[int, int] = (1, 3)
    channels: Tuple[int, ...] = (-1, 0, 1)
    phi_sigma: float = 0.5
    phi_r0: float = 0.5
    # scan raster in pixels: (first, step, count) on each axis
    scan_y: Tuple[float, float, int] = (34.0, 4.0, 16)
    scan_x: Tuple[float, float, int] = (34.0, 4.0, 16)
    # subsampled raster on which the oracle is evaluated at full size
    oracle_scan_y: Tuple[float, float, int] = None
    oracle_scan_x: Tuple[float, float, int] = None

    def replace(self, **kw) -> "Config":
        return replace(self, **kw)

    @property
    def n_scans(self) -> int:
        return self.scan_y[2] * self.scan_x[2]


def config1() -> Config:
    """Plain BiP-PRISM, 4x4 cells of 2.5 A, 128^2 grid, 5 slices of 2 A,
    200 keV, 20 mrad, f=2, four atoms of slice index 2 ionized with three
    channels, 16x16 scans over the central 5x5 A, 0-40 mrad detector."""
    return Config(
        name="config1", ny=128, nx=128, ly=10.0, lx=10.0, nz=5, dz=2.0,
        e0=200e3, alpha=0.020, theta_det=0.040, fy=2, fx=2,
        nrad1=2, nrad2=2, win=64, cells_y=4, cells_x=4,
        ion_slices=(2, 3), ion_cells=(1, 3),
        scan_y=(34.0, 4.0, 16), scan_x=(34.0, 4.0, 16),
        oracle_scan_y=(34.0, 4.0, 16), oracle_scan_x=(34.0, 4.0, 16))


def config2() -> Config:
    """Paper-like scale: 16x16 cells (40x40 A), 512^2 grid, 100 slices of
    2 A, 300 keV, 25 mrad, f=4, every atom of the central 10x10 A ionized at
    every depth (1600 sites, three channels), 128x128 scans at 1 px over the
    central 10x10 A; the oracle is evaluated on every 8th scan (16x16)."""
    return Config(
        name="config2", ny=512, nx=512, ly=40.0, lx=40.0, nz=100, dz=2.0,
        e0=300e3, alpha=0.025, theta_det=0.040, fy=4, fx=4,
        nrad1=4, nrad2=4, win=64, cells_y=16, cells_x=16,
        ion_slices=(0, 100), ion_cells=(6, 10),
        scan_y=(192.0, 1.0, 128), scan_x=(192.0, 1.0, 128),
        oracle_scan_y=(196.0, 8.0, 16), oracle_scan_x=(196.0, 8.0, 16))


def config3() -> Config:
    """Config 1 with the contraction in split-BF16 (hi+lo), FP32 accumulate."""
    return config1().replace(name="config3", prec="split_bf16")


def config5() -> Config:
    """Differentiation workload: 8x8 cells (20x20 A), 256^2 grid, 40 slices of
    2 A, 200 keV, 20 mrad, f=2; 64 ionized sites (the central 4x4 cells at
    four depths) with three channels; 32x32 scans at 2 px over the central
    8x8 A.  The loss is the L2 distance of the map to a seeded perturbed
    target."""
    return Config(
        name="config5", ny=256, nx=256, ly=20.0, lx=20.0, nz=40, dz=2.0,
        e0=200e3, alpha=0.020, theta_det=0.040, fy=2, fx=2,
        nrad1=2, nrad2=2, win=64, cells_y=8, cells_x=8,
        ion_slices=(8, 40, 8), ion_cells=(2, 6),
        scan_y=(96.0, 2.0, 32), scan_x=(96.0, 2.0, 32),
        oracle_scan_y=(96.0, 2.0, 32), oracle_scan_x=(96.0, 2.0, 32))


def tiny_config(**kw) -> Config:
    """A 2x2-cell (5x5 A) specimen on a 32^2 grid with 3 slices, used by the
    brute-force checks; f=1 and a window covering the whole grid."""
    base = Config(
        name="tiny", ny=32, nx=32, ly=5.0, lx=5.0, nz=3, dz=2.0,
        e0=200e3, alpha=0.020, theta_det=0.040, fy=1, fx=1,
        nrad1=2, nrad2=2, win=32, cells_y=2, cells_x=2,
        ion_slices=(1, 2), ion_cells=(0, 2), channels=(-1, 0, 1),
        scan_y=(6.0, 10.0, 3), scan_x=(6.0, 10.0, 3))
    return base.replace(**kw)


CONFIGS = {"config1": config1, "config2": config2, "config3": config3, "config5": config5}


def config_to_json(cfg: Config) -> str:
    """The configuration as JSON (every field; tuples as lists)."""
    return json.dumps(asdict(cfg), indent=1, sort_keys=True)


def config_from_json(text: str) -> Config:
    """A configuration from JSON: the fields config_to_json writes; missing
    optional fields take their defaults, unknown ones are refused."""
    d = json.loads(text)
    known = {f.name: f for f in fields(Config)}
    unknown = sorted(set(d) - set(known))
    if unknown:
        raise ValueError(f"unknown configuration fields: {unknown}")
    for k, v in list(d.items()):
        if isinstance(v, list):
            d[k] = tuple(v)
    return Config(**d)


def load_config(name_or_path: str) -> Config:
    """A named workload (config1, config2, config3, config5) or a JSON file."""
    if name_or_path.endswith(".json"):
        with open(name_or_path) as f:
            return config_from_json(f.read())
    return CONFIGS[name_or_path]()
