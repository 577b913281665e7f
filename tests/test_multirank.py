"""Multi-rank host logic on CPU: template shards and the reductions of the benchmark's timing,
with world size 2 over the gloo backend (templates are independent, so a sharded run
exchanges no data)."""
import os
import socket

import numpy as np
import pytest

import oracle
import synth
from paper_2011_06787_b300.shard import reduce_over_ranks, template_shards


def test_shards_cover_all_templates_contiguously():
    bank = synth.online_bank_global(4, 64)
    for world in (1, 2, 3, 4, 7):
        sh = template_shards(bank.offsets, world)
        assert sh[0][0] == 0 and sh[-1][1] == bank.n_templates
        assert all(lo < hi for lo, hi in sh)
        assert all(sh[r][1] == sh[r + 1][0] for r in range(world - 1))
        f = [int(bank.offsets[hi] - bank.offsets[lo]) for lo, hi in sh]
        # each cut sits at the template boundary nearest its target: shares differ from
        # F / world by less than one template's filters on each side
        assert max(abs(x - bank.n_filters / world) for x in f) <= 2 * int(bank.counts().max())


def test_shards_edge_cases():
    off = np.array([0, 1000, 1001, 1002, 1003], dtype=np.int64)  # one heavy template first
    assert template_shards(off, 1) == [(0, 4)]
    assert template_shards(off, 4) == [(0, 1), (1, 2), (2, 3), (3, 4)]
    sh = template_shards(off, 2)
    assert sh == [(0, 1), (1, 4)]
    with pytest.raises(ValueError):
        template_shards(off, 5)
    with pytest.raises(ValueError):
        template_shards(off, 0)


def test_reduce_without_a_process_group_is_the_identity():
    assert reduce_over_ranks([3.0, 4.0], "max") == [3.0, 4.0]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        gbank = synth.online_bank_global(world, 8)
        lo, hi = template_shards(gbank.offsets, world)[rank]
        mine = gbank.subset(range(lo, hi))
        x = synth.white_noise(1, 3, 300, sub=77)
        z, _, _ = oracle.filter_bank(x, mine.offsets, mine.a1, mine.b0, mine.delay)
        # the benchmark's reductions: slowest rank's time, all ranks' work
        t_max = reduce_over_ranks([1.0 + rank], "max")[0]
        work = reduce_over_ranks([mine.n_filters * 3 * 300], "sum")[0]
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), lo=lo, hi=hi, z=z, t_max=t_max, work=work)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_the_bank(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r = [np.load(tmp_path / f"rank{i}.npz") for i in range(world)]
    gbank = synth.online_bank_global(world, 8)
    assert int(r[0]["lo"]) == 0 and int(r[0]["hi"]) == int(r[1]["lo"]) and int(r[1]["hi"]) == gbank.n_templates
    for x in r:
        assert float(x["t_max"]) == 2.0
        assert float(x["work"]) == gbank.n_filters * 3 * 300
    # the shards' outputs, concatenated, are the unsharded bank's outputs
    xs = synth.white_noise(1, 3, 300, sub=77)
    z_all, _, _ = oracle.filter_bank(xs, gbank.offsets, gbank.a1, gbank.b0, gbank.delay)
    np.testing.assert_array_equal(np.concatenate([r[0]["z"], r[1]["z"]]), z_all)
