"""Pins of the mixed path's rounding model (oracle/mixed.py): the BF16 and
FP16 roundings against PyTorch's conversions, and the map-level error
budget the model gives on config 1 -- with the parent values in FP16 (as
built) and in BF16 (the earlier form, whose rounding dominated)."""
import numpy as np
import pytest

import synth
from oracle import bip, mixed

torch = pytest.importorskip("torch")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _torch_round(x, dtype):
    return torch.tensor(x, dtype=torch.float64).to(dtype).to(torch.float64).numpy()


def _cases(rng, lo, hi):
    """Random FP32 values (the GPU rounds FP32 values; PyTorch converts a
    double to these formats through FP32, so FP32 inputs make its result a
    single rounding too)."""
    mag = np.exp(rng.uniform(np.log(lo), np.log(hi), 20000))
    x = mag * rng.choice([-1.0, 1.0], mag.shape)
    return np.concatenate([x, [0.0, 1.0, -1.0, 0.5, 3.0]]).astype(np.float32).astype(np.float64)


def test_bf16_round_matches_torch():
    rng = np.random.default_rng(1)
    x = _cases(rng, 1e-30, 1e30)
    np.testing.assert_array_equal(mixed.bf16_round(x), _torch_round(x, torch.bfloat16))
    # exact midpoints between neighbours go to the even significand
    v = _torch_round(rng.uniform(1.0, 2.0, 2000), torch.bfloat16)
    mid = v + 2.0 ** -8
    np.testing.assert_array_equal(mixed.bf16_round(mid), _torch_round(mid, torch.bfloat16))


def test_fp16_round_matches_torch():
    rng = np.random.default_rng(2)
    x = _cases(rng, 1e-8, 6.0e4)                      # subnormals to near the top
    np.testing.assert_array_equal(mixed.fp16_round(x), _torch_round(x, torch.float16))
    v = _torch_round(rng.uniform(1.0, 2.0, 2000), torch.float16)
    mid = v + 2.0 ** -11
    np.testing.assert_array_equal(mixed.fp16_round(mid), _torch_round(mid, torch.float16))
    with pytest.raises(OverflowError):
        mixed.fp16_round(np.array([7.0e4]))


@pytest.fixture(scope="module")
def c1():
    sp = synth.make_specimen(synth.config1())
    pr = bip.make_problem(sp)
    return pr, bip.bip_map(pr)


def test_mixed_model_error_budget(c1):
    """Config 1: with FP16 parent values the model's map is within 3e-4 of
    the FP64 map; with BF16 parents it is several times further (over
    5e-4), the share the parents' rounding took in the map's error.  The
    same holds on a 40-scan subset, where the BF16-parent model passes the
    mixed path's 1e-3 bar and the FP16 one stays far inside it."""
    pr, ref = c1
    m16 = mixed.bip_map_mixed(pr)
    m8 = mixed.bip_map_mixed(pr, parents="bf16")
    e16, e8 = rel(m16.map, ref.map), rel(m8.map, ref.map)
    assert e16 < 3e-4
    assert e8 > 5e-4 and e8 > 3 * e16
    sub = pr.scans[100:140]
    ref_s = bip.bip_map(pr, scans=sub).map
    assert rel(mixed.bip_map_mixed(pr, scans=sub).map, ref_s) < 3e-4
    assert rel(mixed.bip_map_mixed(pr, scans=sub, parents="bf16").map, ref_s) > 1e-3
