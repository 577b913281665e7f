"""GPU filter bank (K1) against the FP64 oracle, through the C ABI (Sec. II.B.1, Eq. (zk))."""
import numpy as np
import pytest

import oracle
import synth
from helpers import assert_snr_close, cuda_ok

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs CUDA")]


def _torch():
    import torch
    return torch


def _run_bank(bank, strain, chunks=None, pitch_pad=0):
    """Run a library bank over strain [n_det][n] in the given chunk sizes; returns z [T][n_det][n]."""
    torch = _torch()
    import paper_2011_06787_b300 as sp
    b = sp.Bank(strain.shape[0], bank.offsets, bank.a1, bank.b0, bank.delay)
    n = strain.shape[1]
    chunks = chunks or [n]
    out = []
    pos = 0
    while pos < n:
        c = chunks[len(out) % len(chunks)]
        c = min(c, n - pos)
        x = torch.from_numpy(np.ascontiguousarray(strain[:, pos:pos + c])).cuda()
        z = torch.zeros((bank.n_templates, strain.shape[0], c + pitch_pad), dtype=torch.complex64, device="cuda")
        b.filter_chunk(x, z)
        out.append(z[:, :, :c].cpu().numpy())
        pos += c
    torch.cuda.synchronize()
    import paper_2011_06787_b300 as sp2
    sp2.device_status()
    return np.concatenate(out, axis=2), b


def test_tiny_workload_full_parity():
    w = synth.tiny_workload()
    z, _ = _run_bank(w["bank"], w["strain"])
    z_or, _, _ = oracle.filter_bank(w["strain"], w["bank"].offsets, w["bank"].a1, w["bank"].b0, w["bank"].delay)
    assert_snr_close(z, z_or)


@pytest.mark.parametrize("chunks", [[3000], [1, 7, 512], [2048, 333]])
def test_ragged_tiles_and_chunking(chunks):
    g = synth.rng(0, "misc", 1)
    bank = synth.random_bank(g, [5, 64, 130, 1, 700], d_max=1500)
    x = synth.white_noise(0, 3, 3000, sub=5)
    z, _ = _run_bank(bank, x, chunks=chunks, pitch_pad=3)
    z_or, _, _ = oracle.filter_bank(x, bank.offsets, bank.a1, bank.b0, bank.delay)
    assert_snr_close(z, z_or)


def test_chunking_is_bit_identical_to_one_shot():
    g = synth.rng(0, "misc", 2)
    bank = synth.random_bank(g, [40, 300, 17], d_max=900)
    x = synth.white_noise(0, 2, 2500, sub=6)
    z1, _ = _run_bank(bank, x)
    z2, _ = _run_bank(bank, x, chunks=[1, 7, 512, 2048])
    np.testing.assert_array_equal(z1, z2)


def test_online_subset_parity_two_chunks():
    bank = synth.online_bank(48)
    x = np.concatenate([synth.online_chunk(0), synth.online_chunk(1)], axis=1)
    z, _ = _run_bank(bank, x, chunks=[2048])
    z_or, _, _ = oracle.filter_bank(x, bank.offsets, bank.a1, bank.b0, bank.delay)
    assert_snr_close(z, z_or)


def test_edge_cases_empty_single_and_large_templates():
    g = synth.rng(0, "misc", 3)
    # template 0 empty, 1 has one filter with d = 0, 2 has one with the maximum delay,
    # 3 needs 16 filters per lane (3000 filters)
    counts = [0, 1, 1, 3000]
    bank = synth.random_bank(g, counts, d_max=4000)
    bank.delay[0] = 0
    bank.delay[1] = 4000
    x = synth.white_noise(0, 1, 5000, sub=7)
    z, _ = _run_bank(bank, x, chunks=[4096])
    z_or, _, _ = oracle.filter_bank(x, bank.offsets, bank.a1, bank.b0, bank.delay)
    assert np.all(z[0] == 0)
    assert_snr_close(z[1:], z_or[1:])


def test_maximum_delay_carries_across_chunks():
    """A filter at the largest supported delay (2^20 samples, 512 s at 2048 Hz) answers an
    impulse only many chunks later, as b0 a1^(k - 5 - d), and its template also holds a
    filter of delay 7: the two sit in different delay bins, so the template is cut into two
    pieces whose outputs are added after the launch.  One sample more is rejected."""
    import paper_2011_06787_b300 as sp
    D = 1 << 20
    a = np.array([0.999 * np.exp(0.3j), 0.9 * np.exp(-1.1j)], np.complex64)
    b = np.array([0.5 + 0.2j, 0.25 - 0.1j], np.complex64)
    d = np.array([D, 7], np.int32)
    bank = synth.Bank(np.array([0, 2], np.int64), a, b, d)
    n = D + 6000
    x = np.zeros((1, n), np.float32)
    x[0, 5] = 1.0
    z, bk = _run_bank(bank, x, chunks=[65536])
    assert bk.get_delay_bin() == (8192, 2, 2)
    k = np.arange(n)
    ref = sum(np.where(k >= 5 + dl, complex(bl) * complex(al) ** np.maximum(k - 5 - dl, 0), 0) for al, bl, dl in zip(a, b, d))
    assert np.max(np.abs(z[0, 0] - ref)) <= 1e-5 * np.abs(ref).max()
    assert abs(z[0, 0, 5 + D] - (b[0] + complex(b[1]) * complex(a[1]) ** D)) < 1e-6
    with pytest.raises(sp.SpiirError):
        sp.Bank(1, np.array([0, 1], np.int64), a[:1], b[:1], np.array([D + 1], np.int32))


def test_long_templates_across_delay_bins_match_oracle():
    """Templates whose delays span 160k samples (a 78 s chirp at 2048 Hz) stream in 1 s chunks:
    each is cut into pieces of 8192-sample delay bins, every block stages only its bin's
    window, and the pieces add up to the oracle's SNR.  One template stays within one bin,
    one has no filter in bin 0, one is empty."""
    g = synth.rng(0, "misc", 12)
    counts = [300, 40, 0, 170, 1]
    bank = synth.random_bank(g, counts, d_max=160000)
    bank.delay[300:340] = g.integers(20000, 30000, 40)          # template 1: bins 1 only
    bank.delay[340:510] = g.integers(17000, 160000, 170)        # template 3: no filter in bin 0
    x = synth.white_noise(0, 2, 165000, sub=12)
    z, bk = _run_bank(bank, x, chunks=[2048])
    dbin, blocks, pieces = bk.get_delay_bin()
    assert dbin == 8192 and pieces > len(counts)
    z_or, _, _ = oracle.filter_bank(x, bank.offsets, bank.a1, bank.b0, bank.delay)
    assert np.all(z[2] == 0)
    assert_snr_close(z[[0, 1, 3, 4]], z_or[[0, 1, 3, 4]])


@pytest.mark.parametrize("delay_bin", [0, 1024, 4096, 16384])
def test_delay_bin_width_does_not_change_results(delay_bin):
    """The same bank laid out with whole templates or with pieces of 1024 to 16384-sample bins,
    changed in the middle of the stream (the state carries over), matches the oracle."""
    torch = _torch()
    import paper_2011_06787_b300 as sp
    g = synth.rng(0, "misc", 13)
    bank = synth.random_bank(g, [3, 200, 500, 57, 1, 440], d_max=12000)
    x = synth.white_noise(0, 3, 14000, sub=13)
    b = sp.Bank(3, bank.offsets, bank.a1, bank.b0, bank.delay)
    assert b.get_delay_bin()[0] == 0
    z1 = torch.zeros((6, 3, 9000), dtype=torch.complex64, device="cuda")
    b.filter_chunk(torch.from_numpy(np.ascontiguousarray(x[:, :9000])).cuda(), z1)
    b.set_delay_bin(delay_bin)
    assert b.get_delay_bin()[0] == delay_bin
    z2 = torch.zeros((6, 3, 5000), dtype=torch.complex64, device="cuda")
    b.filter_chunk(torch.from_numpy(np.ascontiguousarray(x[:, 9000:])).cuda(), z2)
    torch.cuda.synchronize()
    sp.device_status()
    z = np.concatenate([z1.cpu().numpy(), z2.cpu().numpy()], axis=2)
    z_or, _, _ = oracle.filter_bank(x, bank.offsets, bank.a1, bank.b0, bank.delay)
    assert_snr_close(z, z_or)
    with pytest.raises(sp.SpiirError):
        b.set_delay_bin(1000)   # not a multiple of 4 in [1024, 2^20]
    assert b.get_delay_bin()[0] == delay_bin


def test_impulse_response_closed_form_on_gpu():
    a = np.array([0.995 * np.exp(0.7j)], np.complex64)
    b = np.array([0.3 - 0.4j], np.complex64)
    bank = synth.Bank(np.array([0, 1], np.int64), a, b, np.array([37], np.int32))
    x = np.zeros((1, 4000), np.float32)
    x[0, 0] = 1.0
    z, _ = _run_bank(bank, x)
    k = np.arange(4000)
    ref = np.where(k >= 37, complex(b[0]) * complex(a[0]) ** np.maximum(k - 37, 0), 0)
    assert np.max(np.abs(z[0, 0] - ref)) <= 1e-5 * np.abs(ref).max()


def test_state_checkpoint_resume_is_bit_identical():
    torch = _torch()
    import paper_2011_06787_b300 as sp
    g = synth.rng(0, "misc", 4)
    bank = synth.random_bank(g, [100, 250, 33], d_max=700)
    x = synth.white_noise(0, 2, 4096, sub=8)
    ref, b1 = _run_bank(bank, x, chunks=[2048])
    # run the first chunk, checkpoint, restore into a fresh bank, run the second
    b2 = sp.Bank(2, bank.offsets, bank.a1, bank.b0, bank.delay)
    z = torch.zeros((3, 2, 2048), dtype=torch.complex64, device="cuda")
    b2.filter_chunk(torch.from_numpy(np.ascontiguousarray(x[:, :2048])).cuda(), z)
    state = b2.get_state()
    assert len(state) == b2.state_bytes()
    b3 = sp.Bank(2, bank.offsets, bank.a1, bank.b0, bank.delay)
    b3.set_state(state)
    z2 = torch.zeros((3, 2, 2048), dtype=torch.complex64, device="cuda")
    b3.filter_chunk(torch.from_numpy(np.ascontiguousarray(x[:, 2048:])).cuda(), z2)
    np.testing.assert_array_equal(z2.cpu().numpy(), ref[:, :, 2048:])
    # the serialised IIR state equals the oracle's state after the first chunk
    _, st_or, hist_or = oracle.filter_bank(x[:, :2048], bank.offsets, bank.a1, bank.b0, bank.delay)
    arr = np.frombuffer(state, dtype=np.float32)
    F = bank.n_filters
    st = arr[: 2 * F * 2].reshape(2, F, 2)
    st = st[..., 0] + 1j * st[..., 1]
    assert np.max(np.abs(st - st_or)) <= 1e-4 * np.abs(st_or).max()
    np.testing.assert_array_equal(arr[2 * F * 2:].reshape(2, -1), hist_or.real.astype(np.float32)[:, -bank.delay.max():])
    with pytest.raises(sp.SpiirError):
        b3.set_state(state[:-4])


def test_reset_restarts_the_stream():
    torch = _torch()
    import paper_2011_06787_b300 as sp
    g = synth.rng(0, "misc", 5)
    bank = synth.random_bank(g, [64, 64], d_max=300)
    x = torch.from_numpy(synth.white_noise(0, 2, 1024, sub=9)).cuda()
    b = sp.Bank(2, bank.offsets, bank.a1, bank.b0, bank.delay)
    z1 = torch.zeros((2, 2, 1024), dtype=torch.complex64, device="cuda")
    z2 = torch.zeros_like(z1)
    b.filter_chunk(x, z1)
    b.reset()
    b.filter_chunk(x, z2)
    assert torch.equal(z1, z2)


def test_online_full_size_sampled_templates():
    """Full 1024-template online bank, one 1 s chunk, as the benchmark launches it; the oracle
    recomputes a sample of templates (templates are independent)."""
    torch = _torch()
    import paper_2011_06787_b300 as sp
    bank = synth.online_bank()
    x = synth.online_chunk(0)
    b = sp.Bank(3, bank.offsets, bank.a1, bank.b0, bank.delay)
    z = torch.zeros((1024, 3, 2048), dtype=torch.complex64, device="cuda")
    b.filter_chunk(torch.from_numpy(x).cuda(), z)
    z = z.cpu().numpy()
    pick = [0, 1, 511, 777, 1023]
    sub = bank.subset(pick)
    z_or, _, _ = oracle.filter_bank(x, sub.offsets, sub.a1, sub.b0, sub.delay)
    assert_snr_close(z[pick], z_or)
    assert np.isfinite(z).all()


@pytest.mark.parametrize("shape", [(4, 128, 16, 512), (8, 128, 32, 1024), (8, 256, 16, 2048), (16, 256, 32, 1024),
                                   (16, 128, 16, 64), (8, 128, 20, 1000), (4, 256, 20, 60), (8, 128, 64, 1024)])
def test_every_launch_shape_matches_oracle(shape):
    torch = _torch()
    import paper_2011_06787_b300 as sp
    g = synth.rng(0, "misc", 6)
    bank = synth.random_bank(g, [3, 200, 500, 57, 1, 440], d_max=3000)
    x = synth.white_noise(0, 3, 3100, sub=10)
    b = sp.Bank(3, bank.offsets, bank.a1, bank.b0, bank.delay)
    # change the shape in the middle of the stream: the state must carry over
    z1 = torch.zeros((6, 3, 1000), dtype=torch.complex64, device="cuda")
    b.filter_chunk(torch.from_numpy(np.ascontiguousarray(x[:, :1000])).cuda(), z1)
    b.set_shape(*shape)
    assert b.get_shape() == shape
    z2 = torch.zeros((6, 3, 2100), dtype=torch.complex64, device="cuda")
    b.filter_chunk(torch.from_numpy(np.ascontiguousarray(x[:, 1000:])).cuda(), z2)
    z = np.concatenate([z1.cpu().numpy(), z2.cpu().numpy()], axis=2)
    z_or, _, _ = oracle.filter_bank(x, bank.offsets, bank.a1, bank.b0, bank.delay)
    assert_snr_close(z, z_or)


def test_shape_rejections_keep_the_bank_usable():
    import paper_2011_06787_b300 as sp
    g = synth.rng(0, "misc", 7)
    bank = synth.random_bank(g, [700], d_max=100)
    b = sp.Bank(1, bank.offsets, bank.a1, bank.b0, bank.delay)
    with pytest.raises(sp.SpiirError):
        b.set_shape(4, 128, 16, 1024)   # 700 filters > 4 x 128
    with pytest.raises(sp.SpiirError):
        b.set_shape(8, 100, 16, 1024)
    assert b.get_shape() == (8, 128, 32, 1024)  # the default for templates of up to 1024 filters


@pytest.mark.parametrize("shape", [(8, 128, 16, 1024), (4, 256, 16, 512), (16, 128, 16, 1024), (8, 128, 20, 1000), (8, 128, 64, 1024)])
def test_full_blocks_with_short_reduction_blocks(shape):
    # templates of 8 lanes fill every warp of every block, so the last warp reduces too
    torch = _torch()
    import paper_2011_06787_b300 as sp
    g = synth.rng(0, "misc", 8)
    S = shape[0]
    bank = synth.random_bank(g, [8 * S] * 40, d_max=700)
    x = synth.white_noise(0, 2, 1500, sub=11)
    b = sp.Bank(2, bank.offsets, bank.a1, bank.b0, bank.delay)
    b.set_shape(*shape)
    z = torch.zeros((40, 2, 1500), dtype=torch.complex64, device="cuda")
    b.filter_chunk(torch.from_numpy(x).cuda(), z)
    torch.cuda.synchronize()
    sp.device_status()
    z_or, _, _ = oracle.filter_bank(x, bank.offsets, bank.a1, bank.b0, bank.delay)
    assert_snr_close(z.cpu().numpy(), z_or)
