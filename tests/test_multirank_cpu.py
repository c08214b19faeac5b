"""The multi-rank host logic of the benchmark, run as two gloo ranks on CPU.

Each rank evaluates its own frozen-phonon configuration (the seed of the
synthetic specimen is the rank), with no exchange inside a step; after the
timed steps the job's step time is the largest rank's and the map is the
incoherent average of the ranks' maps (Sec. 2.1: intensities averaged over
frozen-phonon configurations).  Here the per-rank maps come from the FP64
oracle on a small case, and the combined results are checked against the
same quantities computed in one process."""
import os
import socket
import sys
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _small_case(rank):
    """The benchmark's per-rank workload rule on a small configuration."""
    import synth
    cfg = synth.config1().replace(ion_cells=(1, 3), scan_y=(30.0, 16.0, 5), scan_x=(30.0, 16.0, 5))
    if rank:
        cfg = cfg.replace(seed=rank)
    return cfg, synth.make_specimen(cfg)


def _rank_map(rank):
    from oracle import bip as obip
    _, sp = _small_case(rank)
    return obip.bip_map(obip.make_problem(sp)).map


def _worker(rank, world, port, outdir):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        m = torch.tensor(_rank_map(rank), dtype=torch.float64)
        bench.phonon_mean(m, world)
        t = bench.max_over_ranks(10.0 + rank, world)
        np.save(os.path.join(outdir, f"map{rank}.npy"), m.numpy())
        with open(os.path.join(outdir, f"t{rank}.txt"), "w") as f:
            f.write(repr(t))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_average_maps_and_take_max_time():
    world = 2
    with tempfile.TemporaryDirectory() as d:
        ctx = mp.get_context("spawn")
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, world, port, d)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=300)
        assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
        maps = [np.load(os.path.join(d, f"map{r}.npy")) for r in range(world)]
        times = [float(open(os.path.join(d, f"t{r}.txt")).read()) for r in range(world)]
    want = 0.5 * (_rank_map(0) + _rank_map(1))
    # both ranks hold the same average, equal to the average of the two
    # configurations' maps; the configurations differ
    assert np.array_equal(maps[0], maps[1])
    assert np.allclose(maps[0], want, rtol=1e-12, atol=0.0)
    assert not np.allclose(_rank_map(0), _rank_map(1), rtol=1e-6)
    assert times == [11.0, 11.0]
