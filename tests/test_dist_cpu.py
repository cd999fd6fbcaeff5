"""World-size-2 runs of the multi-rank plumbing on CPU (gloo).

Two processes split a k-point list with ``partition``, each evaluates its
share of Gamma_nk (the FP64 oracle stands in for the device path here), and
the gathered result must equal the single-process one; the timing reduction
must return the slowest rank's value.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2002_02045_gb300.dist import partition


def test_partition_covers_each_unit_once():
    for n in (0, 1, 7, 216, 3223):
        for world in (1, 2, 3, 8):
            spans = [partition(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            for (a, b), (c, d) in zip(spans, spans[1:]):
                assert b == c
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        partition(5, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    import synthetic as S
    from oracle import eph as O
    from paper_2002_02045_gb300 import dist as D
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m = S.model_c1()
    kidx = np.arange(0, 216, 5)
    a, b = partition(len(kidx), rank, world)
    gam = O.scattering_rates_grid(m, (6, 6, 6), (6, 6, 6), kidx[a:b], 300.0, 0.5, 0.005)
    parts = [None] * world
    dist.all_gather_object(parts, (a, b, gam))
    slow = D.max_over_ranks(1.0 + rank)
    total = D.sum_over_ranks(b - a)
    D.barrier()
    if rank == 0:
        full = np.concatenate([p[2] for p in sorted(parts, key=lambda x: x[0])])
        np.save(os.path.join(out_dir, "gathered.npy"), full)
        np.save(os.path.join(out_dir, "stats.npy"), np.array([slow, total]))
    dist.destroy_process_group()


def test_two_rank_gloo_split_matches_single_process(tmp_path):
    import synthetic as S
    from oracle import eph as O
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    full = np.load(tmp_path / "gathered.npy")
    slow, total = np.load(tmp_path / "stats.npy")
    kidx = np.arange(0, 216, 5)
    ref = O.scattering_rates_grid(S.model_c1(), (6, 6, 6), (6, 6, 6), kidx, 300.0, 0.5, 0.005)
    assert np.array_equal(full, ref)
    assert slow == 2.0 and total == len(kidx)
