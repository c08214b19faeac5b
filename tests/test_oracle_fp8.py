"""Pins of the FP8 (E4M3) model of the coupling contraction.

e4m3_round is checked against PyTorch's own float8_e4m3fn conversion (a
library routine, not the oracle's code) on every code, on the midpoints
between neighbouring codes and on random values, and against the format's
fixed points (saturation, subnormal spacing).  The per-window scale rule is
checked as a bound (no element of a scaled row exceeds 448) on reconstructed
windows, and the FP8 map against the FP64 map: close, but not equal."""
import numpy as np
import pytest

import synth
from oracle import bip as obip
from oracle import fp8

torch = pytest.importorskip("torch")


def torch_e4m3(x):
    return torch.tensor(np.asarray(x, dtype=np.float32)).to(torch.float8_e4m3fn).to(torch.float64).numpy()


def all_codes():
    """Every finite E4M3 value, from PyTorch's decoding of the 256 bytes."""
    v = torch.arange(256, dtype=torch.uint8).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    return np.unique(v[np.isfinite(v)])


def test_codes_are_fixed_points():
    v = all_codes()
    assert len(v) == 253                      # 254 finite codes, +0 and -0 equal
    assert v.max() == 448.0 and v.min() == -448.0
    assert np.array_equal(fp8.e4m3_round(v), v)


def test_midpoints_round_to_even_like_torch():
    v = all_codes()
    pos = v[v >= 0.0]
    mid = 0.5 * (pos[:-1] + pos[1:])
    got = fp8.e4m3_round(mid)
    assert np.array_equal(got, torch_e4m3(mid))
    assert np.array_equal(fp8.e4m3_round(-mid), -got)
    # ties go to the code with an even mantissa (the last bit of the code)
    codes = torch.tensor(got.astype(np.float32)).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.all(codes % 2 == 0)


def test_random_values_match_torch():
    rng = np.random.default_rng(3)
    x = np.concatenate([
        rng.uniform(-448.0, 448.0, 20000),
        np.exp(rng.uniform(np.log(2.0 ** -12), np.log(448.0), 20000)) * rng.choice([-1.0, 1.0], 20000),
    ]).astype(np.float32).astype(np.float64)
    assert np.array_equal(fp8.e4m3_round(x), torch_e4m3(x))


def test_saturation_and_subnormals():
    assert fp8.e4m3_round(1.0e6) == 448.0 and fp8.e4m3_round(-470.0) == -448.0
    assert fp8.e4m3_round(2.0 ** -9) == 2.0 ** -9           # smallest subnormal
    assert fp8.e4m3_round(2.0 ** -10) == 0.0                 # tie to even (zero)
    assert fp8.e4m3_round(3 * 2.0 ** -10) == 2.0 ** -8       # tie 1.5 -> 2 (even)
    # relative error of normal values at most 2^-4
    x = np.linspace(2.0 ** -6, 448.0, 100001)
    assert np.max(np.abs(fp8.e4m3_round(x) - x) / x) <= 2.0 ** -4


@pytest.fixture(scope="module")
def case():
    cfg = synth.config1()
    sp = synth.make_specimen(cfg)
    return obip.make_problem(sp)


def test_row_bounds_hold_on_reconstructed_windows(case):
    pr = case
    cfg, geo = pr.cfg, pr.geo
    W1 = obip.s1_windows(pr, geo.h_p1, detilt=True)
    W2 = obip.s2_windows(pr, geo.h_p2, detilt=True)
    for k in range(len(pr.ion)):
        iy, ix = pr.window_index(k)
        for mode in ("magnitude", "complex"):
            S1 = obip.reconstruct(W1[k], geo.w1, geo.h_beam, iy, ix, cfg.ny, cfg.nx, +1, mode)
            S2 = obip.reconstruct(W2[k], geo.w2, geo.h_det, iy, ix, cfg.ny, cfg.nx, -1, mode)
            b1 = fp8.row_bounds(geo.w1, W1[k])
            b2 = fp8.row_bounds(geo.w2, W2[k])
            assert np.all(np.abs(S1).reshape(len(b1), -1).max(axis=1) * fp8.KAPPA <= b1 * (1 + 1e-12))
            assert np.all(np.abs(S2).reshape(len(b2), -1).max(axis=1) * fp8.KAPPA <= b2 * (1 + 1e-12))
            for h in pr.H[k]:
                X = h[None] * S1
                q = fp8.quantize_rows(X, np.max(np.abs(h)) * b1)
                # stored codes stay inside the finite range, no saturation
                scaled = np.abs(X.real).reshape(len(b1), -1).max(axis=1) * fp8.E4M3_MAX / (np.max(np.abs(h)) * b1)
                assert np.all(scaled < fp8.E4M3_MAX)
                # every element within half a step of its scaled E4M3 grid
                s = (np.max(np.abs(h)) * b1 / fp8.E4M3_MAX)[:, None, None]
                big = np.abs(X.real) / s >= 2.0 ** -6
                assert np.all(np.abs(q.real - X.real)[big] <= 2.0 ** -4 * np.abs(X.real)[big] * (1 + 1e-12))


def test_fp8_map_close_to_but_not_the_fp64_map(case):
    """The FP8 model departs from the FP64 map by the E4M3 rounding of the
    operands: a 3-bit mantissa (relative step 2^-4 at most) averaged over
    the 4096-term window sums.  On config 1 it lands at 0.69%; the pin
    requires (0, 2%)."""
    r = obip.bip_map(case)
    r8 = fp8.bip_map_fp8(case)
    rel = np.linalg.norm(r8.map - r.map) / np.linalg.norm(r.map)
    assert 1e-4 < rel < 2e-2, rel


def test_fp8_per_beam_sums_to_fp8_map(case):
    """The FP8 model's per-beam intensities (what qEELS bins) summed over
    the detector are its map (the same coupling feeds both)."""
    m = fp8.bip_map_fp8(case).map
    c = fp8.per_beam_fp8(case)
    assert c.shape == (len(case.scans), case.geo.n_det)
    assert np.max(np.abs(c.sum(axis=1) - m)) <= 1e-12 * np.max(np.abs(m))
