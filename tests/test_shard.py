"""The multi-rank path split on CPU: two gloo ranks each run the oracle on their
own path range of the same entries, all-gather (count, mean, SE) and merge; the
result must be the single-process oracle run over the union of the ranges
(Sec. 1 and Sec. 7: independent samples; Sec. 5: sample mean and variance)."""
import os

import numpy as np
import pytest

import workloads as W
from paper_1904_12759_gb300 import shard

torch = pytest.importorskip("torch")


def test_path_range_partitions():
    for paths in (0, 1, 7, 1000, 1001):
        for world in (1, 2, 3, 8):
            got = [shard.path_range(r, world, paths) for r in range(world)]
            assert sum(c for _, c in got) == paths
            pos = 0
            for off, c in got:
                assert off == pos
                pos += c
    with pytest.raises(ValueError):
        shard.path_range(2, 2, 10)


def test_merge_single_rank_is_identity():
    m = np.array([1.0, 2.0, -3.0])
    s = np.array([0.1, 0.2, 0.0])
    mm, ss = shard.merge(m[None], s[None], [50])
    assert np.allclose(mm, m, rtol=1e-15) and np.allclose(ss, s, rtol=1e-12)


def _rank(rank, world, port, out_dir):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import walker as OW

    csr = W.erdos_renyi(300, 6, 3)
    v = W.uniform_vector(300, 4, -1.0, 1.0)
    ent = W.random_entries(300, 40, 5)
    paths = 3001
    off, cnt = shard.path_range(rank, world, paths)
    mean, sem, _ = OW.Graph(csr).estimate(v, 0.2, cnt, entries=ent, seed=9, path_offset=off)
    local = torch.tensor(np.stack([mean, sem]), dtype=torch.float64)
    gathered = [torch.zeros_like(local) for _ in range(world)]
    dist.all_gather(gathered, local)
    counts = torch.tensor([cnt], dtype=torch.int64)
    all_counts = [torch.zeros_like(counts) for _ in range(world)]
    dist.all_gather(all_counts, counts)
    if rank == 0:
        g = torch.stack(gathered).numpy()
        mm, ss = shard.merge(g[:, 0], g[:, 1], [int(c) for c in all_counts])
        np.save(os.path.join(out_dir, "merged.npy"), np.stack([mm, ss]))
    dist.destroy_process_group()


def test_two_gloo_ranks_merge_to_single_run(tmp_path):
    import socket

    import torch.multiprocessing as mp
    from oracle import walker as OW

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.start_processes(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    mm, ss = np.load(tmp_path / "merged.npy")
    csr = W.erdos_renyi(300, 6, 3)
    v = W.uniform_vector(300, 4, -1.0, 1.0)
    ent = W.random_entries(300, 40, 5)
    mean, sem, _ = OW.Graph(csr).estimate(v, 0.2, 3001, entries=ent, seed=9)
    scale = np.abs(mean) + sem * np.sqrt(3001)
    assert np.all(np.abs(mm - mean) <= 1e-12 * scale)
    assert np.allclose(ss, sem, rtol=1e-8, atol=1e-14)
