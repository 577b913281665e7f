"""GPU coherent scan (K2) and the streaming pipeline against the FP64 oracle, through the C ABI
(Sec. II.C.1 Eq. (llr_form), Eq. (null_def); App. A)."""
import numpy as np
import pytest

import oracle
import synth
from helpers import assert_coherent_close, assert_snr_close, cuda_ok

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs CUDA")]


def _sky(cfg, n_det, nside, sig):
    import paper_2011_06787_b300 as sp
    det = synth.detectors(cfg, n_det)
    sigma = synth.noise_weights(cfg, n_det, *sig)
    tabs = sp.sky_tables(det.pos_m, det.arm_x, det.arm_y, sigma, nside, 2048.0)
    _, G, d_or = oracle.sky_geometry(det, sigma, nside, 2048.0)
    return sp.Sky(*tabs), G, d_or


def _scan(sky, z_pad, n, skymap=False):
    import torch
    T = z_pad.shape[0]
    zt = torch.from_numpy(np.ascontiguousarray(z_pad.astype(np.complex64))).cuda()
    ms = torch.empty((T, n), dtype=torch.float32, device="cuda")
    am = torch.empty((T, n), dtype=torch.int32, device="cuda")
    nl = torch.empty((T, n), dtype=torch.float32, device="cuda")
    mp = torch.empty((T, sky.n_pix, n), dtype=torch.float32, device="cuda") if skymap else None
    sky.scan(zt, n, ms, am, nl, mp)
    torch.cuda.synchronize()
    return ms.cpu().numpy(), am.cpu().numpy(), nl.cpu().numpy(), (mp.cpu().numpy() if skymap else None)


@pytest.mark.parametrize("cfg,n_det,nside,sig,T,n", [
    (0, 2, 4, (1.0, 1.0), 4, 2000),
    (1, 3, 16, (0.5, 2.0), 3, 700),
    (5, 4, 4, (0.7, 1.6), 2, 1100),
])
def test_scan_parity_gaussian_snr(cfg, n_det, nside, sig, T, n):
    sky, G, d_or = _sky(cfg, n_det, nside, sig)
    H = sky.halo
    z = synth.complex_gaussian_snr(cfg, (T, n_det, n + 2 * H + 5))
    ms, am, nl, _ = _scan(sky, z, n)
    ms_or, am_or, nl_or, sm_or = oracle.coherent(z, G, d_or, H, n, skymap=True)
    assert_coherent_close(ms, am, nl, ms_or, am_or, nl_or, sm_or)
    if n_det == 2:
        assert np.all(nl == 0)


def test_skymap_mode_matches_oracle_map():
    sky, G, d_or = _sky(1, 3, 4, (0.5, 2.0))
    H = sky.halo
    n = 777
    z = synth.complex_gaussian_snr(1, (2, 3, n + 2 * H), sub=3)
    ms, am, nl, mp = _scan(sky, z, n, skymap=True)
    _, _, _, sm_or = oracle.coherent(z, G, d_or, H, n, skymap=True)
    # device map is [T][P][n]; oracle map is [T][n][P]
    mp = np.transpose(mp, (0, 2, 1))
    assert np.all(np.abs(mp - sm_or) <= 1e-4 * sm_or.max(axis=-1, keepdims=True))
    np.testing.assert_array_equal(ms, mp.max(axis=-1))


def test_noiseless_injection_found_at_true_pixel():
    sky, G, d_or = _sky(1, 3, 16, (0.5, 2.0))
    H = sky.halo
    n, k0, pstar = 300, 120, 1999
    j = np.arange(-4 * H, n + 4 * H)
    f = np.exp(-0.5 * ((j - k0) / 0.6) ** 2) * np.exp(0.9j * j)
    A = np.array([1.0 + 0.3j, -0.4 + 0.8j])
    amp = G[pstar] @ A
    z = np.zeros((1, 3, n + 2 * H), dtype=np.complex128)
    for I in range(3):
        idx = np.arange(n + 2 * H) - H - d_or[pstar, I]
        z[0, I] = amp[I] * f[idx + 4 * H]
    ms, am, nl, _ = _scan(sky, z, n)
    tot = sum(abs(z[0, I, H + k0 + d_or[pstar, I]]) ** 2 for I in range(3))
    ms_or, am_or, _, _ = oracle.coherent(z.astype(np.complex64), G, d_or, H, n)
    assert am_or[0, k0] == pstar
    assert am[0, k0] == pstar
    assert abs(ms[0, k0] - tot) <= 1e-4 * tot
    assert nl[0, k0] <= 1e-4 * tot


def test_argmax_ties_take_lowest_pixel():
    import paper_2011_06787_b300 as sp
    # four identical pixels
    d = np.zeros((4, 3), np.int32)
    us = np.tile(np.array([[1, 0], [0, 1], [0, 0]], np.float32)[None], (4, 1, 1))
    un = np.tile(np.array([[0], [0], [1]], np.float32)[None], (4, 1, 1))
    sky = sp.Sky(d, us, un)
    z = np.ones((2, 3, 50), np.complex64)
    ms, am, nl, _ = _scan(sky, z, 50)
    assert np.all(am == 0) and np.allclose(ms, 2.0) and np.allclose(nl, 1.0)


@pytest.mark.parametrize("copies", [2, 3])
@pytest.mark.parametrize("shape", [(512, 4, 1), (512, 4, 0), (256, 4, 1), (256, 2, 1), (256, 2, 0)])
def test_exact_ties_across_groups_take_lowest_pixel(copies, shape):
    """Every pixel of the first third (half) has copies whose detector-0 delay is 1 or 2
    samples later, so they sit in other detector-0 groups.  Detector 0 is silent, so each pixel
    and its copies have bit-identical statistics: every sample's maximum is attained in 2 (3)
    groups, and the lowest original index, the original pixel, must win."""
    import paper_2011_06787_b300 as sp
    det = synth.detectors(1, 3)
    sigma = synth.noise_weights(1, 3, 0.5, 2.0)
    d, us, un = sp.sky_tables(det.pos_m, det.arm_x, det.arm_y, sigma, 8, 2048.0)
    _, G, d_or = oracle.sky_geometry(det, sigma, 8, 2048.0)
    m = d.shape[0] // copies
    idx = np.concatenate([np.arange(m)] * copies)
    shift = np.repeat(np.arange(copies), m).astype(np.int32)
    d2, d2_or = d[idx].copy(), d_or[idx].copy()
    d2[:, 0] += shift
    d2_or[:, 0] += shift
    sky = sp.Sky(d2, us[idx], un[idx])
    sky.set_scan_shape(*shape)
    assert sky.get_scan_shape()[:3] == shape
    H, n, T = sky.halo, 1300, 2
    z = synth.complex_gaussian_snr(1, (T, 3, n + 2 * H), sub=71).astype(np.complex64)
    z[:, 0, :] = 0
    ms, am, nl, _ = _scan(sky, z, n)
    ms_or, am_or, nl_or, sm_or = oracle.coherent(z, G[idx], d2_or, H, n, skymap=True)
    assert_coherent_close(ms, am, nl, ms_or, am_or, nl_or, sm_or)
    assert np.all(am < m)
    # where the best original pixel leads the next distinct one clearly, it is the oracle's
    top = np.sort(sm_or[:, :, :m], axis=-1)
    clear = top[..., -1] - top[..., -2] > 1e-4 * top[..., -1]
    assert clear.mean() > 0.5
    np.testing.assert_array_equal(am[clear], am_or[clear])
    # the sky-map instances resolve the ties identically, and the map holds the copies' equal values
    ms2, am2, nl2, mp = _scan(sky, z, n, skymap=True)
    assert np.array_equal(ms2, ms) and np.array_equal(am2, am) and np.array_equal(nl2, nl)
    for c in range(1, copies):
        assert np.array_equal(mp[:, c * m:(c + 1) * m], mp[:, :m])


@pytest.mark.parametrize("shape", [(256, 2, 1), (512, 1, 0), (512, 4, 1), (512, 4, 0), (256, 4, 1)])
@pytest.mark.parametrize("n", [1, 3, 13])
def test_few_output_samples(shape, n):
    """One, three and thirteen output samples: partial thread rows and items, through every
    kind of scan."""
    sky, G, d_or = _sky(1, 3, 8, (0.5, 2.0))
    sky.set_scan_shape(*shape)
    H = sky.halo
    z = synth.complex_gaussian_snr(1, (2, 3, n + 2 * H), sub=110 + n)
    ms, am, nl, _ = _scan(sky, z, n)
    ms_or, am_or, nl_or, sm_or = oracle.coherent(z, G, d_or, H, n, skymap=True)
    assert_coherent_close(ms, am, nl, ms_or, am_or, nl_or, sm_or)


def test_scan_rejects_bad_arguments_and_stays_usable():
    import torch
    import paper_2011_06787_b300 as sp
    sky, G, d_or = _sky(1, 3, 4, (0.5, 2.0))
    H, n, T = sky.halo, 64, 2
    z = synth.complex_gaussian_snr(1, (T, 3, n + 2 * H), sub=120)
    zt = torch.from_numpy(z.astype(np.complex64)).cuda()
    out = [torch.empty((T, n), dtype=dt, device="cuda") for dt in (torch.float32, torch.int32, torch.float32)]
    L = sp.native.lib()
    ptr = lambda t: sp._dev_ptr(t)
    # n < 1, no templates, rows shorter than n + 2 H, NULL outputs
    for T_, n_, pitch in ((T, 0, n + 2 * H), (0, n, n + 2 * H), (T, n, n + 2 * H - 1)):
        rc = L.spiir_coherent_scan(sky._h, ptr(zt), pitch, T_, n_, ptr(out[0]), ptr(out[1]), ptr(out[2]), None, None)
        assert rc != 0
    assert L.spiir_coherent_scan(sky._h, ptr(zt), n + 2 * H, T, n, None, ptr(out[1]), ptr(out[2]), None, None) != 0
    ms, am, nl, _ = _scan(sky, z, n)
    ms_or, am_or, nl_or, sm_or = oracle.coherent(z, G, d_or, H, n, skymap=True)
    assert_coherent_close(ms, am, nl, ms_or, am_or, nl_or, sm_or)


def _pipeline_stream(bank, sky, strain, chunk, host=False):
    import torch
    import paper_2011_06787_b300 as sp
    b = sp.Bank(strain.shape[0], bank.offsets, bank.a1, bank.b0, bank.delay)
    pipe = sp.Pipeline(b, sky, max_chunk=chunk)
    T = bank.n_templates
    outs = []
    for s in range(0, strain.shape[1], chunk):
        x = np.ascontiguousarray(strain[:, s:s + chunk])
        n = x.shape[1]
        if host:
            ms = np.zeros((T, n), np.float32); am = np.zeros((T, n), np.int32); nl = np.zeros((T, n), np.float32)
            pipe.run_host(x, ms, am, nl)
            outs.append((ms, am, nl))
        else:
            ms = torch.empty((T, n), dtype=torch.float32, device="cuda")
            am = torch.empty((T, n), dtype=torch.int32, device="cuda")
            nl = torch.empty((T, n), dtype=torch.float32, device="cuda")
            pipe.run(torch.from_numpy(x).cuda(), ms, am, nl)
            outs.append((ms.cpu().numpy(), am.cpu().numpy(), nl.cpu().numpy()))
    return [np.concatenate([o[i] for o in outs], axis=1) for i in range(3)]


@pytest.mark.parametrize("host", [False, True])
def test_streaming_pipeline_matches_oracle(host):
    sky, G, d_or = _sky(1, 3, 4, (0.5, 2.0))
    H = sky.halo
    bank = synth.online_bank(6)
    strain = np.concatenate([synth.online_chunk(i) for i in range(3)], axis=1)[:, :5000]
    ms, am, nl = _pipeline_stream(bank, sky, strain, 1024, host=host)
    # oracle: whole-stream SNR, H zeros before the stream start (values before it are 0),
    # output j of the stream is geocentric sample j - H
    z_or, _, _ = oracle.filter_bank(strain, bank.offsets, bank.a1, bank.b0, bank.delay)
    N = strain.shape[1]
    zp = np.concatenate([np.zeros((bank.n_templates, 3, 2 * H)), z_or], axis=2)
    ms_or, am_or, nl_or, sm_or = oracle.coherent(zp, G, d_or, H, N, skymap=True)
    assert_coherent_close(ms, am, nl, ms_or, am_or, nl_or, sm_or)


def test_asynchronous_host_steps_match_synchronous_ones():
    """Chunks submitted with host buffers and collected by wait() (outputs copied while the
    next chunk runs) equal the synchronous host-buffer steps bit for bit, also when the two
    kinds of call are interleaved on one pipeline."""
    import torch
    import paper_2011_06787_b300 as sp
    sky, _, _ = _sky(1, 3, 16, (0.5, 2.0))
    sky.set_scan_shape(512, 4, 1)
    bank = synth.online_bank(24)
    n = 1024
    chunks = [np.ascontiguousarray(synth.online_chunk(i)[:, :n]) for i in range(6)]
    T = bank.n_templates

    def bufs():
        return (torch.empty((T, n), dtype=torch.float32).pin_memory().numpy(),
                torch.empty((T, n), dtype=torch.int32).pin_memory().numpy(),
                torch.empty((T, n), dtype=torch.float32).pin_memory().numpy())

    ref = []
    pipe = sp.Pipeline(sp.Bank(3, bank.offsets, bank.a1, bank.b0, bank.delay), sky, max_chunk=n)
    for c in chunks:
        o = bufs()
        pipe.run_host(c, *o)
        ref.append(o)
    pipe2 = sp.Pipeline(sp.Bank(3, bank.offsets, bank.a1, bank.b0, bank.delay), sky, max_chunk=n)
    got = [bufs() for _ in chunks]
    for i in range(3):
        pipe2.submit_host(chunks[i], *got[i])
    pipe2.run_host(chunks[3], *got[3])          # waits for the submitted steps first
    for i in (4, 5):
        pipe2.submit_host(chunks[i], *got[i])
    pipe2.wait()
    for r, g in zip(ref, got):
        for a, b in zip(r, g):
            np.testing.assert_array_equal(a, b)


def test_timed_wait_reports_unfinished_steps_without_blocking():
    """A host-side limit on collecting submitted steps: with several full online chunks queued,
    a 1 ms limit returns before the work is done (the steps keep running), and an unlimited wait
    then collects them; the outputs equal the synchronous path's."""
    import time
    import torch
    import paper_2011_06787_b300 as sp
    sky, _, _ = _sky(1, 3, 16, (0.5, 2.0))
    sky.set_scan_shape(512, 4, 1)
    bank = synth.online_bank()
    chunks = [np.ascontiguousarray(synth.online_chunk(i)) for i in range(4)]
    T, n = bank.n_templates, 2048
    outs = [tuple(torch.empty((T, n), dtype=dt).pin_memory().numpy() for dt in (torch.float32, torch.int32, torch.float32))
            for _ in chunks]
    pipe = sp.Pipeline(sp.Bank(3, bank.offsets, bank.a1, bank.b0, bank.delay), sky, max_chunk=n)
    assert pipe.wait_for(0.0)          # nothing submitted yet
    for c, o in zip(chunks, outs):
        pipe.submit_host(c, *o)
    t0 = time.perf_counter()
    assert not pipe.wait_for(1e-3)     # about 18 ms of GPU work is queued
    assert time.perf_counter() - t0 < 0.5
    assert pipe.wait_for(60.0)
    ref = sp.Pipeline(sp.Bank(3, bank.offsets, bank.a1, bank.b0, bank.delay), sky, max_chunk=n)
    for c, o in zip(chunks, outs):
        r = tuple(np.empty_like(a) for a in o)
        ref.run_host(c, *r)
        for a, b in zip(o, r):
            np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("shape", [(256, 1, 1), (256, 2, 1), (512, 1, 0), (512, 2, 0), (256, 2, 0), (512, 4, 1)])
@pytest.mark.parametrize("n_det", [2, 3])
def test_every_scan_shape_matches_oracle(shape, n_det):
    if shape[1] == 4 and n_det == 2:
        pytest.skip("the tensor-memory scan is for three detectors")
    sky, G, d_or = _sky(1, n_det, 8, (0.5, 2.0))
    sky.set_scan_shape(*shape)
    assert sky.get_scan_shape() == shape + (1,)
    H = sky.halo
    n = 2500
    z = synth.complex_gaussian_snr(1, (3, n_det, n + 2 * H), sub=11)
    ms, am, nl, _ = _scan(sky, z, n)
    ms_or, am_or, nl_or, sm_or = oracle.coherent(z, G, d_or, H, n, skymap=True)
    assert_coherent_close(ms, am, nl, ms_or, am_or, nl_or, sm_or)
    ms2, am2, nl2, mp = _scan(sky, z, n, skymap=True)
    np.testing.assert_array_equal(ms2, ms)
    np.testing.assert_array_equal(am2, am)
    mp = np.transpose(mp, (0, 2, 1))
    assert np.all(np.abs(mp - sm_or) <= 1e-4 * sm_or.max(axis=-1, keepdims=True))


@pytest.mark.parametrize("rate,shape", [(16384.0, (256, 2, 1)), (16384.0, (512, 1, 0)), (8192.0, (256, 1, 1))])
def test_long_delays_take_the_fallback_layouts(rate, shape):
    """Skies sampled at 8 and 16 kHz (|Delta| up to 173 and 346 samples): the tensor-memory scan
    does not apply, and the shared-memory scan stages wider windows (or reads through L1);
    results against the oracle as at 2048 Hz."""
    import paper_2011_06787_b300 as sp
    det = synth.detectors(1, 3)
    sigma = synth.noise_weights(1, 3, 0.5, 2.0)
    tabs = sp.sky_tables(det.pos_m, det.arm_x, det.arm_y, sigma, 4, rate)
    sky = sp.Sky(*tabs)
    _, G, d_or = oracle.sky_geometry(det, sigma, 4, rate)
    H = sky.halo
    assert H == int(np.abs(d_or).max()) and H > 60
    with pytest.raises(sp.SpiirError):
        sky.set_scan_shape(512, 4, 1)
    sky.set_scan_shape(*shape)
    z = synth.complex_gaussian_snr(1, (2, 3, 1300 + 2 * H), sub=40)
    ms, am, nl, _ = _scan(sky, z, 1300)
    ms_or, am_or, nl_or, sm_or = oracle.coherent(z, G, d_or, H, 1300, skymap=True)
    assert_coherent_close(ms, am, nl, ms_or, am_or, nl_or, sm_or)


def test_delays_beyond_the_limit_are_rejected():
    import paper_2011_06787_b300 as sp
    det = synth.detectors(1, 3)
    with pytest.raises(sp.SpiirError):
        sp.Sky(*sp.sky_tables(det.pos_m, det.arm_x, det.arm_y, np.ones(3), 4, 49152.0))   # |Delta| = 1038 > 1024


def test_sky_map_moments_in_gaussian_noise():
    """Statistical invariant on the GPU (App. A): with i.i.d. complex Gaussian SNR of
    E|z_I|^2 = 2 the coherent statistic at a fixed pixel is chi^2 with 4 degrees of freedom,
    mean 4 and variance 8; checked on the sky map of 1.2e6 pixel-samples."""
    sky, G, d_or = _sky(1, 3, 4, (0.5, 2.0))
    H = sky.halo
    T, n = 3, 2048
    z = synth.complex_gaussian_snr(1, (T, 3, n + 2 * H), sub=50)
    _, _, _, mp = _scan(sky, z, n, skymap=True)
    assert mp.size == T * 192 * n
    # 6144 independent samples per pixel: the mean of a chi^2_4 has a standard error of 0.036
    # at most (less after the average over correlated pixels), its variance about 0.2
    assert abs(float(mp.mean()) - 4.0) < 0.1, mp.mean()
    assert abs(float(mp.var()) - 8.0) < 0.8, mp.var()
    # per pixel over samples: every pixel's statistic has the same distribution
    per_pix = mp.mean(axis=(0, 2))
    assert np.all(np.abs(per_pix - 4.0) < 0.35)


def test_general_kernel_for_non_orthonormal_tables():
    import paper_2011_06787_b300 as sp
    sky, G, d_or = _sky(1, 3, 4, (0.5, 2.0))
    det = synth.detectors(1, 3)
    sigma = synth.noise_weights(1, 3, 0.5, 2.0)
    d, us, un = sp.sky_tables(det.pos_m, det.arm_x, det.arm_y, sigma, 4, 2048.0)
    un2 = un * 1.5  # not a unit null vector: the grouped null-vector form does not apply
    sky2 = sp.Sky(d, us, un2)
    assert sky2.get_scan_shape()[3] == 0
    H = sky2.halo
    z = synth.complex_gaussian_snr(1, (2, 3, 600 + 2 * H), sub=12)
    ms, am, nl, _ = _scan(sky2, z, 600)
    ms_or, am_or, nl_or, sm_or = oracle.coherent(z, G, d_or, H, 600, skymap=True)
    # the statistic uses U_s only; the null uses the (scaled) table as given
    assert_coherent_close(ms, am, nl / 2.25, ms_or, am_or, nl_or, sm_or)


def test_all_zero_window_ties_resolve_to_pixel_zero():
    sky, G, d_or = _sky(1, 3, 16, (0.5, 2.0))
    H = sky.halo
    z = np.zeros((2, 3, 1500 + 2 * H), np.complex64)
    z[1, :, 700:] = synth.complex_gaussian_snr(1, (3, z.shape[2] - 700), sub=13)
    ms, am, nl, _ = _scan(sky, z, 1500)
    assert np.all(ms[0] == 0) and np.all(am[0] == 0) and np.all(nl[0] == 0)
    ms_or, am_or, nl_or, sm_or = oracle.coherent(z, G, d_or, H, 1500, skymap=True)
    assert_coherent_close(ms, am, nl, ms_or, am_or, nl_or, sm_or)


@pytest.mark.parametrize("threads", [512, 256])
@pytest.mark.parametrize("nside,T,n,param", [(8, 3, 2500, 1), (16, 2, 1024, 1), (16, 2, 3000, 1), (16, 2, 3000, 0),
                                              (16, 3, 512, 1), (8, 5, 300, 1), (16, 3, 256, 1), (8, 7, 100, 0),
                                              (16, 2, 2048, 1), (8, 5, 1000, 0)])
def test_tensor_memory_scan_matches_oracle_and_shared_memory_scan(threads, nside, T, n, param):
    """The TMEM scan (512 threads with 8 samples per row, or 256 with 16; detector 1 and 2
    windows in tensor memory) against the oracle, and against the shared-memory scan (the two pair the FP32
    arithmetic differently, so they agree to rounding).  n = 2500 and 3000 leave ragged last
    tiles of 1024 (2048) samples; short chunks put 2 or 4 templates in one work item, here with
    template counts that leave the last item partly empty.  param: group and
    offset tables in the kernel parameters (1) or in shared memory (0), with bit-identical
    results."""
    sky, G, d_or = _sky(1, 3, nside, (0.5, 2.0))
    H = sky.halo
    z = synth.complex_gaussian_snr(1, (T, 3, n + 2 * H), sub=21)
    ms_s, am_s, nl_s, _ = _scan(sky, z, n)
    sky.set_scan_shape(threads, 4, param)
    assert sky.get_scan_shape() == (threads, 4, param, 1)
    ms, am, nl, _ = _scan(sky, z, n)
    sky.set_scan_shape(threads, 4, 1 - param)
    ms2, am2, nl2, _ = _scan(sky, z, n)
    assert np.array_equal(ms, ms2) and np.array_equal(am, am2) and np.array_equal(nl, nl2)
    assert np.all(np.abs(ms - ms_s) <= 1e-5 * ms_s.max())
    assert np.mean(am == am_s) > 0.999
    ms_or, am_or, nl_or, sm_or = oracle.coherent(z, G, d_or, H, n, skymap=True)
    assert_coherent_close(ms, am, nl, ms_or, am_or, nl_or, sm_or)


@pytest.mark.parametrize("nside,T,n", [(16, 3, 2048), (8, 4, 700), (16, 5, 300)])
def test_tensor_memory_scan_forms_agree_bit_for_bit(nside, T, n):
    """8 samples per thread row (512 threads) and 16 (256 threads) evaluate every pixel and
    sample with the same arithmetic, so their maxima, argmax and null agree exactly."""
    sky, _, _ = _sky(1, 3, nside, (0.5, 2.0))
    H = sky.halo
    z = synth.complex_gaussian_snr(1, (T, 3, n + 2 * H), sub=90 + n)
    sky.set_scan_shape(512, 4, 1)
    a = _scan(sky, z, n)
    sky.set_scan_shape(256, 4, 1)
    b = _scan(sky, z, n)
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("threads", [512, 256])
def test_tensor_memory_scan_ties_and_sky_map(threads):
    sky, G, d_or = _sky(1, 3, 16, (0.5, 2.0))
    sky.set_scan_shape(threads, 4, 1)
    H = sky.halo
    z = np.zeros((2, 3, 2100 + 2 * H), np.complex64)
    z[1, :, 900:] = synth.complex_gaussian_snr(1, (3, z.shape[2] - 900), sub=14)
    ms, am, nl, _ = _scan(sky, z, 2100)
    assert np.all(ms[0] == 0) and np.all(am[0] == 0) and np.all(nl[0] == 0)
    ms_or, am_or, nl_or, sm_or = oracle.coherent(z, G, d_or, H, 2100, skymap=True)
    assert_coherent_close(ms, am, nl, ms_or, am_or, nl_or, sm_or)
    # with a sky map (n = 2100: vector stores, a ragged last tile)
    ms2, am2, nl2, mp = _scan(sky, z, 2100, skymap=True)
    assert_coherent_close(ms2, am2, nl2, ms_or, am_or, nl_or, sm_or)
    mp = np.transpose(mp, (0, 2, 1))
    assert np.all(np.abs(mp - sm_or) <= 1e-4 * np.maximum(sm_or.max(axis=-1, keepdims=True), 1e-30))


@pytest.mark.parametrize("n,T", [(200, 5), (512, 3)])
@pytest.mark.parametrize("threads", [512, 256])
def test_tensor_memory_sky_map_with_several_templates_per_item(n, T, threads):
    sky, G, d_or = _sky(1, 3, 8, (0.5, 2.0))
    sky.set_scan_shape(threads, 4, 1)
    H = sky.halo
    z = synth.complex_gaussian_snr(1, (T, 3, n + 2 * H), sub=60 + n)
    ms, am, nl, mp = _scan(sky, z, n, skymap=True)
    ms_or, am_or, nl_or, sm_or = oracle.coherent(z, G, d_or, H, n, skymap=True)
    assert_coherent_close(ms, am, nl, ms_or, am_or, nl_or, sm_or)
    mp = np.transpose(mp, (0, 2, 1))
    assert np.all(np.abs(mp - sm_or) <= 1e-4 * np.maximum(sm_or.max(axis=-1, keepdims=True), 1e-30))


def test_tensor_memory_scan_needs_three_detectors():
    import paper_2011_06787_b300 as sp
    sky, _, _ = _sky(0, 2, 4, (1.0, 1.0))
    with pytest.raises(sp.SpiirError):
        sky.set_scan_shape(512, 4, 1)
    assert sky.get_scan_shape()[:2] == (256, 2)


def test_online_full_size_pipeline_sampled_templates():
    """The full online workload (1024 templates, 3 detectors, nside 16) streamed through the
    pipeline in the benchmark's launch configuration (tensor-memory scan, 8 filters x 128
    lanes); the oracle recomputes a sample of templates, which are independent."""
    import torch
    import paper_2011_06787_b300 as sp
    w = synth.online_workload()
    c, det, bank, sigma = w["cfg"], w["det"], w["bank"], w["sigma"]
    sky = sp.Sky(*sp.sky_tables(det.pos_m, det.arm_x, det.arm_y, sigma, c["nside"], 2048.0))
    _, G, d_or = oracle.sky_geometry(det, sigma, c["nside"], 2048.0)
    sky.set_scan_shape(512, 4, 1)
    b = sp.Bank(3, bank.offsets, bank.a1, bank.b0, bank.delay)
    b.set_shape(8, 128, 32, 1024)
    pipe = sp.Pipeline(b, sky, max_chunk=2048)
    T, H = bank.n_templates, sky.halo
    strain = np.concatenate([synth.online_chunk(i) for i in range(2)], axis=1)
    outs = []
    for s in range(0, strain.shape[1], 2048):
        ms = torch.empty((T, 2048), dtype=torch.float32, device="cuda")
        am = torch.empty((T, 2048), dtype=torch.int32, device="cuda")
        nl = torch.empty((T, 2048), dtype=torch.float32, device="cuda")
        pipe.run(torch.from_numpy(np.ascontiguousarray(strain[:, s:s + 2048])).cuda(), ms, am, nl)
        outs.append((ms.cpu().numpy(), am.cpu().numpy(), nl.cpu().numpy()))
    ms, am, nl = [np.concatenate([o[i] for o in outs], axis=1) for i in range(3)]
    assert np.isfinite(ms).all() and np.isfinite(nl).all()
    assert am.min() >= 0 and am.max() < sky.n_pix
    pick = [0, 333, 1023]
    sub = bank.subset(pick)
    z_or, _, _ = oracle.filter_bank(strain, sub.offsets, sub.a1, sub.b0, sub.delay)
    N = strain.shape[1]
    zp = np.concatenate([np.zeros((len(pick), 3, 2 * H)), z_or], axis=2)
    for i, t in enumerate(pick):
        ms_or, am_or, nl_or, sm_or = oracle.coherent(zp[i:i + 1], G, d_or, H, N, skymap=True)
        assert_coherent_close(ms[t:t + 1], am[t:t + 1], nl[t:t + 1], ms_or, am_or, nl_or, sm_or)


@pytest.mark.parametrize("n", [777, 2050])
def test_tensor_memory_sky_map_scalar_tail_and_odd_lengths(n):
    """Sky map from the tensor-memory scan where n is not a multiple of 4 (scalar stores)."""
    sky, G, d_or = _sky(1, 3, 16, (0.5, 2.0))
    sky.set_scan_shape(512, 4, 1)
    H = sky.halo
    z = synth.complex_gaussian_snr(1, (2, 3, n + 2 * H), sub=15)
    ms, am, nl, mp = _scan(sky, z, n, skymap=True)
    ms_or, am_or, nl_or, sm_or = oracle.coherent(z, G, d_or, H, n, skymap=True)
    assert_coherent_close(ms, am, nl, ms_or, am_or, nl_or, sm_or)
    mp = np.transpose(mp, (0, 2, 1))
    assert np.all(np.abs(mp - sm_or) <= 1e-4 * sm_or.max(axis=-1, keepdims=True))


@pytest.mark.parametrize("threads,param", [(512, 1), (256, 1), (512, 0)])
def test_tensor_memory_scan_of_a_sky_in_parts(threads, param):
    """nside 32 (12288 pixels) exceeds one parameter table (6400 pixels): the tensor-memory
    scan runs the sky as consecutive parts, each later part keeping the better of its own and the
    stored (maximum, lowest pixel).  Against the oracle and the shared-memory scan, in argmax and
    sky-map mode."""
    sky, G, d_or = _sky(4, 3, 32, (0.5, 2.0))
    H, T, n = sky.halo, 2, 1300
    z = synth.complex_gaussian_snr(4, (T, 3, n + 2 * H), sub=32)
    ms_s, am_s, nl_s, _ = _scan(sky, z, n)
    sky.set_scan_shape(threads, 4, param)
    assert sky.get_scan_shape() == (threads, 4, param, 1)
    ms, am, nl, _ = _scan(sky, z, n)
    assert np.all(np.abs(ms - ms_s) <= 1e-5 * ms_s.max()) and np.mean(am == am_s) > 0.999
    ms_or, am_or, nl_or, sm_or = oracle.coherent(z, G, d_or, H, n, skymap=True)
    assert_coherent_close(ms, am, nl, ms_or, am_or, nl_or, sm_or)
    ms2, am2, nl2, mp = _scan(sky, z, n, skymap=True)
    assert np.array_equal(ms2, ms) and np.array_equal(am2, am) and np.array_equal(nl2, nl)
    mp = np.transpose(mp, (0, 2, 1))
    assert np.all(np.abs(mp - sm_or) <= 1e-4 * np.maximum(sm_or.max(axis=-1, keepdims=True), 1e-30))


def test_tensor_memory_parts_resolve_exact_ties_and_zero_windows_to_the_lowest_pixel():
    """Three copies of the nside-16 sky (9216 pixels, two parts) whose detector-0 delays are
    0, 1 and 2 samples later, with detector 0 silent: each pixel ties exactly with its copies,
    which sit in other groups and parts, and the original (lowest) index must win; an all-zero
    window ties every pixel and gives pixel 0."""
    import paper_2011_06787_b300 as sp
    det = synth.detectors(1, 3)
    sigma = synth.noise_weights(1, 3, 0.5, 2.0)
    d, us, un = sp.sky_tables(det.pos_m, det.arm_x, det.arm_y, sigma, 16, 2048.0)
    _, G, d_or = oracle.sky_geometry(det, sigma, 16, 2048.0)
    m, copies = d.shape[0], 3
    idx = np.concatenate([np.arange(m)] * copies)
    shift = np.repeat(np.arange(copies), m).astype(np.int32)
    d2, d2_or = d[idx].copy(), d_or[idx].copy()
    d2[:, 0] += shift
    d2_or[:, 0] += shift
    sky = sp.Sky(d2, us[idx], un[idx])
    sky.set_scan_shape(512, 4, 1)
    H, n, T = sky.halo, 1100, 2
    z = synth.complex_gaussian_snr(1, (T, 3, n + 2 * H), sub=72).astype(np.complex64)
    z[:, 0, :] = 0
    z[1, :, :400] = 0                      # template 1 starts with an all-zero window
    ms, am, nl, _ = _scan(sky, z, n)
    ms_or, am_or, nl_or, sm_or = oracle.coherent(z, G[idx], d2_or, H, n, skymap=True)
    assert_coherent_close(ms, am, nl, ms_or, am_or, nl_or, sm_or)
    assert np.all(am < m)
    zero = np.all(sm_or == 0, axis=-1)
    assert zero.any() and np.all(am[zero] == 0) and np.all(ms[zero] == 0)
    top = np.sort(sm_or[:, :, :m], axis=-1)
    clear = top[..., -1] - top[..., -2] > 1e-4 * top[..., -1]
    assert clear.mean() > 0.5
    np.testing.assert_array_equal(am[clear], am_or[clear])
