"""Multi-rank path on CPU (gloo, world size 2): disjoint event shards, the
step-time max and the histogram sum over ranks reproduce a single-process
oracle run over the union of the shards."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2511_19633_gb300.sharding import max_over_ranks, rank_first_event, sum_histograms

WS, STEPS, PER_STEP = 2, 2, 150


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _hists(O, first, n):
    from tests.golden.make_oracle_hists import NBINS, fill
    st = O.Settings(process=0, sqrt_s=91.2, nmax=64, seed=3)
    r = O.run(st, first, n)
    h, h2 = np.zeros((6, NBINS)), np.zeros((6, NBINS))
    done = r["status"] == 1
    fill(h, h2, r["obs"][done], r["weight"][done], "ee")
    return h, h2


def _worker(rank, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=WS)
    from oracle import oracle as O
    h = torch.zeros((6, 66), dtype=torch.float64)
    h2 = torch.zeros_like(h)
    for k in range(STEPS):
        a, b = _hists(O, rank_first_event(rank, k, PER_STEP, STEPS), PER_STEP)
        h += torch.from_numpy(a)
        h2 += torch.from_numpy(b)
    sum_histograms([h, h2], dist)
    t = max_over_ranks(10.0 + rank, dist)
    if rank == 0:
        torch.save({"h": h, "h2": h2, "t": t}, out)
    dist.barrier()
    dist.destroy_process_group()


def test_shards_are_disjoint_and_cover():
    ids = set()
    for r in range(3):
        for k in range(4):
            f = rank_first_event(r, k, 10, 4)
            block = set(range(f, f + 10))
            assert not (ids & block)
            ids |= block
    assert ids == set(range(120))
    with pytest.raises(ValueError):
        rank_first_event(0, 4, 10, 4)


def test_two_ranks_reproduce_one_process(tmp_path):
    out = str(tmp_path / "r0.pt")
    mp.spawn(_worker, args=(_free_port(), out), nprocs=WS, join=True)
    res = torch.load(out)
    from oracle import oracle as O
    ref, ref2 = _hists(O, 0, WS * STEPS * PER_STEP)
    assert np.allclose(res["h"].numpy(), ref, rtol=1e-12, atol=0)
    assert np.allclose(res["h2"].numpy(), ref2, rtol=1e-12, atol=0)
    assert res["t"] == 11.0
