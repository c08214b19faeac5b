"""Host logic of the benchmark that needs no GPU: the workload options
(site subsets, the central scan sub-raster), the raster detection that
decides which evaluation of the scan polynomial the library runs, and the
JSON configuration block."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
import synth  # noqa: E402


def test_workload_scan_side_is_the_central_subraster():
    cfg, full = bench.workload("config1", 0)
    _, sub = bench.workload("config1", 0, scan_side=4)
    n = int(round(np.sqrt(len(full.scans))))
    grid = full.scans.reshape(n, n, 2)
    c = n // 2
    assert sub.scans.shape == (16, 2)
    np.testing.assert_array_equal(sub.scans.reshape(4, 4, 2), grid[c - 2:c + 2, c - 2:c + 2])
    # the rest of the specimen is untouched
    np.testing.assert_array_equal(sub.V, full.V)
    np.testing.assert_array_equal(sub.nch, full.nch)
    assert bench.raster_shape(sub.scans) == (4, 4)


def test_workload_max_sites_keeps_the_first_sites():
    cfg, full = bench.workload("config1", 0)
    _, sp = bench.workload("config1", 0, max_sites=2)
    ion = np.nonzero(full.nch > 0)[0]
    assert np.count_nonzero(sp.nch) == 2
    assert list(np.nonzero(sp.nch > 0)[0]) == list(ion[:2])
    assert sp.H.shape[0] == 2 * len(cfg.channels)


def test_raster_shape():
    y, x = np.meshgrid(np.arange(3.0), np.arange(5.0) * 0.5, indexing="ij")
    sc = np.stack([y.ravel(), x.ravel()], axis=1)
    assert bench.raster_shape(sc) == (3, 5)
    assert bench.raster_shape(sc[:14]) is None          # ragged
    bad = sc.copy()
    bad[7, 1] += 0.25                                   # one column out of line
    assert bench.raster_shape(bad) is None
    assert bench.raster_shape(np.zeros((0, 2))) is None
    # a column of scans is a raster of one column; a diagonal line is not
    column = np.stack([np.linspace(0, 9, 10), np.full(10, 3.0)], axis=1)
    assert bench.raster_shape(column) == (10, 1)
    diagonal = np.stack([np.linspace(0, 9, 10), np.linspace(3, 5, 10)], axis=1)
    assert bench.raster_shape(diagonal) is None


@pytest.mark.parametrize("order", bench.ORDERS)
def test_config_block_names_the_workload_and_order(order):
    cfg, sp = bench.workload("config1", 0, scan_side=4)
    blk = bench.config_block(cfg, sp, order)
    assert blk["order"] == order
    assert blk["scans"] == 16 and "16 scans" in blk["workload"]
    assert blk["sites"] == int((sp.nch > 0).sum())
    assert blk["grid"] == [cfg.ny, cfg.nx] and blk["window"] == cfg.win


def test_crop_counts_bound_the_pairs():
    # every site's crop window holds at most all scans, and at config 1 (a
    # 5 A window per site over a 10 A cell) at least one
    cfg, sp = bench.workload("config1", 0)
    n_sites = int((sp.nch > 0).sum())
    n = bench.crop_counts(cfg, sp)
    assert n_sites <= n <= n_sites * len(sp.scans)
    assert synth.config1().name == cfg.name


@pytest.mark.parametrize("name", sorted(synth.CONFIGS))
def test_config_json_round_trip(name):
    cfg = synth.CONFIGS[name]()
    assert synth.config_from_json(synth.config_to_json(cfg)) == cfg


def test_workload_from_a_json_file(tmp_path):
    """A workload given as a JSON file is the named workload's specimen,
    bit for bit; unknown fields are refused."""
    path = tmp_path / "c1.json"
    path.write_text(synth.config_to_json(synth.config1()))
    cfg_a, a = bench.workload("config1", 0)
    cfg_b, b = bench.workload(str(path), 0)
    assert cfg_a == cfg_b
    for k in ("V", "H", "atoms", "nch", "scans"):
        np.testing.assert_array_equal(getattr(a, k), getattr(b, k))
    bad = tmp_path / "bad.json"
    bad.write_text(synth.config_to_json(synth.config1())[:-2] + ', "grid": 3}')
    with pytest.raises(ValueError, match="unknown configuration fields"):
        synth.load_config(str(bad))
