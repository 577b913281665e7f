"""Batched multirate banks (row A6): plain per-bank launches, one persistent launch, and the
CUDA-graph replay, against the FP64 oracle's multirate definition and the coherent scan."""
import numpy as np
import pytest

import oracle
import synth
from helpers import assert_coherent_close, cuda_ok

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs CUDA")]

FACTORS = (1, 4, 16)


def _concat(banks):
    offs, a1, b0, d, band = [np.zeros(1, np.int64)], [], [], [], []
    for o, a, b, dd, bb in banks:
        offs.append(offs[-1][-1] + np.asarray(o)[1:])
        a1.append(a)
        b0.append(b)
        d.append(dd)
        band.append(bb)
    return np.concatenate(offs), np.concatenate(a1), np.concatenate(b0), np.concatenate(d), np.concatenate(band)


def _setup(nside=4, sub=1, chunk=512):
    import paper_2011_06787_b300 as sp
    det = synth.detectors(1, 3)
    sigma = synth.noise_weights(1, 3, 0.5, 2.0)
    sky = sp.Sky(*sp.sky_tables(det.pos_m, det.arm_x, det.arm_y, sigma, nside, 2048.0))
    _, G, d_or = oracle.sky_geometry(det, sigma, nside, 2048.0)
    banks = synth.multirate_banks(n_banks=3, t_range=(3, 12), f_range=(20, 80), seed_sub=sub)
    return sp, sky, G, d_or, banks


def _run(sp, sky, banks, mode, n_chunks, chunk=512, shape=None):
    import torch
    b = sp.Batch(3, banks, FACTORS, sky, chunk)
    if shape:
        b.set_shape(*shape)
    T = b.n_templates
    ms = torch.empty((T, chunk), device="cuda")
    am = torch.empty((T, chunk), dtype=torch.int32, device="cuda")
    nl = torch.empty((T, chunk), device="cuda")
    x = torch.empty((3, chunk), device="cuda")
    outs = []
    for c in range(n_chunks):
        x.copy_(torch.from_numpy(synth.multirate_chunk(c, 3, chunk)))
        b.run(x, ms, am, nl, mode=mode)
        outs.append((ms.cpu().numpy().copy(), am.cpu().numpy().copy(), nl.cpu().numpy().copy()))
    torch.cuda.synchronize()
    sp.device_status()
    return [np.concatenate([o[i] for o in outs], axis=1) for i in range(3)]


def _oracle(banks, G, d_or, H, n_chunks, chunk=512):
    off, a1, b0, d, band = _concat(banks)
    x = np.concatenate([synth.multirate_chunk(c, 3, chunk) for c in range(n_chunks)], axis=1)
    z = oracle.multirate_bank(x, off, a1, b0, d, band, FACTORS)
    N = x.shape[1]
    zp = np.concatenate([np.zeros((z.shape[0], 3, 2 * H)), z], axis=2)
    return oracle.coherent(zp, G, d_or, H, N, skymap=True)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_every_path_matches_the_oracle(mode):
    sp, sky, G, d_or, banks = _setup()
    ms, am, nl = _run(sp, sky, banks, mode, 4)
    ms_or, am_or, nl_or, sm_or = _oracle(banks, G, d_or, sky.halo, 4)
    assert_coherent_close(ms, am, nl, ms_or, am_or, nl_or, sm_or)


def test_graph_replay_equals_the_eager_persistent_launch_bit_for_bit():
    sp, sky, G, d_or, banks = _setup(sub=2)
    eager = _run(sp, sky, banks, 1, 3)
    graph = _run(sp, sky, banks, 2, 3)
    for e, g in zip(eager, graph):
        np.testing.assert_array_equal(e, g)


@pytest.mark.parametrize("shape", [(4, 128, 16, 1), (8, 256, 32, 0), (16, 128, 32, 2)])
def test_persistent_shapes_match_the_oracle(shape):
    sp, sky, G, d_or, banks = _setup(sub=3)
    ms, am, nl = _run(sp, sky, banks, 2, 3, shape=shape)
    ms_or, am_or, nl_or, sm_or = _oracle(banks, G, d_or, sky.halo, 3)
    assert_coherent_close(ms, am, nl, ms_or, am_or, nl_or, sm_or)


def test_switching_paths_needs_a_reset():
    import torch
    sp, sky, G, d_or, banks = _setup(sub=4)
    b = sp.Batch(3, banks, FACTORS, sky, 512)
    T = b.n_templates
    ms = torch.empty((T, 512), device="cuda")
    am = torch.empty((T, 512), dtype=torch.int32, device="cuda")
    nl = torch.empty((T, 512), device="cuda")
    x = torch.from_numpy(synth.multirate_chunk(0, 3, 512)).cuda()
    b.run(x, ms, am, nl, mode=2)
    with pytest.raises(sp.SpiirError):
        b.run(x, ms, am, nl, mode=0)
    b.reset()
    b.run(x, ms, am, nl, mode=0)
    first = ms.clone()
    b.reset()
    b.run(x, ms, am, nl, mode=0)
    assert torch.equal(first, ms)


def test_persistent_launch_with_full_blocks_and_short_reduction_blocks():
    sp, sky, G, d_or, _ = _setup(sub=5)
    banks = synth.multirate_banks(n_banks=4, t_range=(60, 90), f_range=(60, 70), seed_sub=6)
    ms, am, nl = _run(sp, sky, banks, 2, 2, shape=(8, 128, 16, 0))
    ms_or, am_or, nl_or, sm_or = _oracle(banks, G, d_or, sky.halo, 2)
    assert_coherent_close(ms, am, nl, ms_or, am_or, nl_or, sm_or)


def test_persistent_filter_launch_time_hook():
    """spiir_batch_filter_time: -1 until armed and until an eager batched chunk ran; then the
    device time of that chunk's persistent filter launch, which graph replays leave unchanged."""
    import torch
    sp, sky, G, d_or, banks = _setup()
    b = sp.Batch(3, banks, FACTORS, sky, 512)
    T = b.n_templates
    ms = torch.empty((T, 512), device="cuda")
    am = torch.empty((T, 512), dtype=torch.int32, device="cuda")
    nl = torch.empty((T, 512), device="cuda")
    x = torch.from_numpy(synth.multirate_chunk(0, 3, 512)).cuda()
    assert b.filter_time() == -1.0          # arms the events
    b.run(x, ms, am, nl, mode=sp.Batch.GRAPH)
    assert b.filter_time() == -1.0          # graph replays are not timed
    b.run(x, ms, am, nl, mode=sp.Batch.BATCHED)
    t1 = b.filter_time()
    assert 0.0 < t1 < 1000.0
    b.run(x, ms, am, nl, mode=sp.Batch.GRAPH)
    assert b.filter_time() == t1
