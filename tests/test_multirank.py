"""Multi-rank host logic on CPU: template shards and the reductions of the benchmark's timing,
with world size 2 over the gloo backend (templates are independent, so a sharded run
exchanges no data)."""
import os
import socket

import numpy as np
import pytest

import oracle
import synth
from paper_2011_06787_b300.shard import bank_max_over_ranks, reduce_over_ranks, template_shards


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


def test_shards_at_bank_boundaries():
    """With bank starts, cuts fall only on bank boundaries (no bank spans two ranks) and still
    balance the filters as well as whole banks allow."""
    g = synth.rng(6, "misc", 1)
    sizes = [40, 3, 77, 12, 60, 5, 31, 50]
    starts = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    bank = synth.random_bank(g, g.integers(100, 1200, sum(sizes)), d_max=100)
    for world in (1, 2, 3, 5, 8):
        sh = template_shards(bank.offsets, world, starts)
        assert sh[0][0] == 0 and sh[-1][1] == bank.n_templates
        assert all(lo in set(starts) for lo, _ in sh) and all(sh[r][1] == sh[r + 1][0] for r in range(world - 1))
        f = [int(bank.offsets[hi] - bank.offsets[lo]) for lo, hi in sh]
        heaviest = max(int(bank.offsets[starts[i] + sizes[i]] - bank.offsets[starts[i]]) for i in range(len(sizes)))
        assert max(abs(x - bank.n_filters / world) for x in f) <= 2 * heaviest
    with pytest.raises(ValueError):
        template_shards(bank.offsets, 9, starts)       # more ranks than banks
    with pytest.raises(ValueError):
        template_shards(bank.offsets, 2, [5, 40])      # must start at template 0


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


def _bank_rank_main(rank, world, port, out_dir):
    """Per-bank selection with whole banks per rank, and the per-sample maximum of one bank
    split over the two ranks through bank_max_over_ranks."""
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        z = synth.complex_gaussian_snr(6, (22, 2, 1024), sub=3)
        sizes = [6, 4, 7, 5]
        starts = np.concatenate([[0], np.cumsum(sizes)[:-1]])
        off = np.arange(23, dtype=np.int64) * 10
        lo, hi = template_shards(off, world, starts)[rank]
        recs = []
        for b, (s0, n_t) in enumerate(zip(starts, sizes)):
            if lo <= s0 < hi:
                for I, t, k, v in oracle.select_candidates(z[s0:s0 + n_t], 0, 1024, 3.0, 256):
                    recs.append((b, I, s0 + t, k, v))
        # one bank of all 22 templates split in the middle: local maxima, then the all-reduce
        cut = 9
        mine = slice(0, cut) if rank == 0 else slice(cut, 22)
        w = z[mine].astype(np.complex64)
        m2 = w.real.astype(np.float32) ** 2 + w.imag.astype(np.float32) ** 2
        tl = np.argmax(m2, axis=0) + (0 if rank == 0 else cut)
        gm, gt = bank_max_over_ranks(m2.max(axis=0), tl)
        np.savez(os.path.join(out_dir, f"bank{rank}.npz"), recs=np.array(recs, dtype=np.float64).reshape(-1, 5),
                 gm=gm, gt=gt)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_keep_banks_whole_and_reduce_a_split_bank(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_bank_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r = [np.load(tmp_path / f"bank{i}.npz") for i in range(world)]
    z = synth.complex_gaussian_snr(6, (22, 2, 1024), sub=3)
    sizes = [6, 4, 7, 5]
    starts = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    want = []
    for b, (s0, n_t) in enumerate(zip(starts, sizes)):
        for I, t, k, v in oracle.select_candidates(z[s0:s0 + n_t], 0, 1024, 3.0, 256):
            want.append((b, I, s0 + t, k, v))
    got = sorted(tuple(x) for x in np.concatenate([r[0]["recs"], r[1]["recs"]]))
    assert len(want) > 10 and got == sorted(tuple(float(v) for v in w) for w in want)
    # the split bank's per-sample maximum and template equal the unsplit ones on both ranks
    w = z.astype(np.complex64)
    m2 = w.real.astype(np.float32) ** 2 + w.imag.astype(np.float32) ** 2
    for x in r:
        np.testing.assert_array_equal(x["gm"], m2.max(axis=0))
        np.testing.assert_array_equal(x["gt"], np.argmax(m2, axis=0))
