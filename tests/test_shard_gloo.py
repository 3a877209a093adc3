"""Multi-rank path (CPU, gloo, world_size 2): pairs shard with no data-path
exchange and meet in one final gather.  The per-rank aligner here is the
oracle, since the host logic is what is under test."""
import os
import socket

import numpy as np
import pytest

from paper_2607_15478_gb300 import shard, synth


def test_partition_is_a_balanced_cover():
    rng = np.random.default_rng(3)
    cells = rng.integers(1, 10_000, size=57)
    for world in (1, 2, 3, 8):
        parts = shard.partition_pairs(cells, world)
        flat = sorted(k for p in parts for k in p)
        assert flat == list(range(len(cells)))
        loads = [int(cells[np.array(p, dtype=int)].sum()) for p in parts]
        # LPT: the spread is at most the largest single item
        assert max(loads) - min(loads) <= int(cells.max())
    assert shard.partition_pairs(cells, 4) == shard.partition_pairs(cells, 4)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pairs = [(p.A, p.B) for p in synth.config_batch(2, n_pairs=7, La_range=(40, 160))]
    local = shard.align_share(pairs, rank, world, lambda a, b: oracle.dtw(a, b))
    res = shard.gather_results(local, len(pairs))
    if rank == 0:
        np.save(os.path.join(out_dir, "costs.npy"), np.array([r[1] for r in res]))
        np.save(os.path.join(out_dir, "lens.npy"), np.array([len(r[0]) for r in res]))
    dist.destroy_process_group()


def test_two_ranks_cover_the_batch(tmp_path):
    import torch.multiprocessing as mp

    import oracle
    oracle.build()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn",
                       join=True)
    costs = np.load(tmp_path / "costs.npy")
    lens = np.load(tmp_path / "lens.npy")
    pairs = synth.config_batch(2, n_pairs=7, La_range=(40, 160))
    for k, p in enumerate(pairs):
        path, total = oracle.dtw(p.A, p.B)
        assert costs[k] == total and lens[k] == len(path)
