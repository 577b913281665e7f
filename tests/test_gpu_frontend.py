"""GPU front end (Sec. II.A): 16384 -> 2048 Hz FIR down-sampling and time-domain whitening
(Eq. (whiten)) streamed in segments, against the FP64 oracle on the same FP32 taps."""
import numpy as np
import pytest

import oracle
import synth
from helpers import cuda_ok

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs CUDA")]

TOL = 2e-5  # max |y_gpu - y_oracle| / max |y_oracle|: FP32 sums of a few thousand products


def _psd_ar1(fs, N, phi, s):
    f = np.arange(N // 2 + 1) * fs / N
    return (2.0 * s ** 2 / fs) / np.abs(1.0 - phi * np.exp(-2j * np.pi * f / fs)) ** 2


def _colored(seed, n_det, n, phis):
    """AR(1)-coloured noise per detector at the input rate."""
    e = synth.white_noise(seed, n_det, n).astype(np.float64)
    x = np.zeros_like(e)
    for I, p in enumerate(phis):
        for k in range(1, n):
            x[I, k] = p * x[I, k - 1] + e[I, k]
    return x.astype(np.float32)


def _run(fe, x, segs):
    import torch
    outs, k0 = [], 0
    for c in segs:
        xt = torch.from_numpy(np.ascontiguousarray(x[:, k0: k0 + c])).cuda()
        outs.append(fe.run(xt).cpu().numpy())
        k0 += c
    return np.concatenate(outs, axis=1)


@pytest.mark.parametrize("Ld,M,Lw,segs", [
    (192, 8, 4097, [16384, 16384, 16384]),                   # the paper's rates, 1 s segments, 2 s kernel
    (192, 8, 1025, [8 * 2048, 8 * 1000, 8, 8 * 2040, 8 * 520]),  # ragged segments, one of a single output
    (48, 4, 129, [400, 4, 1204]),                            # other factor, short filters (padded taps)
    (1, 1, 1, [300, 700]),                                   # both filters one tap: the identity (scaled)
])
def test_frontend_matches_oracle(Ld, M, Lw, segs):
    import paper_2011_06787_b300 as sp
    n_det = 3
    n = sum(segs)
    x = _colored(9, n_det, n, (0.95, 0.5, -0.3))
    h = oracle.lowpass_taps(Ld, M, 0.9).astype(np.float32) if Ld > 1 else np.array([1.0], np.float32)
    if Lw > 1:
        w = np.stack([oracle.whitening_kernel(_psd_ar1(2048.0, 2 * (Lw + 1), p, 1.0), 2048.0, Lw)
                      for p in (0.9, 0.4, -0.2)]).astype(np.float32)
    else:
        w = np.array([[0.5], [2.0], [-1.0]], np.float32)
    fe = sp.Frontend(n_det, h, M, w, max(segs))
    y = _run(fe, x, segs)
    y_or, _, _ = oracle.frontend(x, h, M, w)
    assert y.shape == y_or.shape
    err = np.abs(y - y_or).max() / np.abs(y_or).max()
    assert err < TOL, err
    # a reset starts a new stream
    fe.reset()
    y2 = _run(fe, x, segs[:1])
    np.testing.assert_array_equal(y2, y[:, : segs[0] // M])


def test_frontend_whitens_coloured_noise_to_unit_variance():
    """Strain whose 2048 Hz PSD is an AR(1) shape comes out of the whitening stage with unit
    variance and no lag-1 correlation (the decimator passes the band below 920 Hz)."""
    import paper_2011_06787_b300 as sp
    fs16, M = 16384, 8
    n = 8 * fs16
    e = synth.white_noise(10, 1, n // M).astype(np.float64)[0]
    phi, s = 0.8, 3.0
    x2 = np.zeros(n // M)
    for k in range(1, n // M):
        x2[k] = phi * x2[k - 1] + s * e[k]
    # the 2048 Hz stream held at the input rate (each sample repeated), then the GPU path;
    # the reference for the statistics is the whitening of x2 itself on the oracle
    w = oracle.whitening_kernel(_psd_ar1(2048.0, 8192, phi, s), 2048.0, 2049).astype(np.float32)
    fe = sp.Frontend(1, np.array([1.0], np.float32), 1, w[None], n // M)
    y = _run(fe, x2[None].astype(np.float32), [n // M])[0][4096:]
    assert abs(float(y.var()) - 1.0) < 0.03
    assert abs(float(np.mean(y[1:] * y[:-1]) / y.var())) < 0.03


def test_frontend_rejects_bad_segments():
    import torch
    import paper_2011_06787_b300 as sp
    fe = sp.Frontend(2, oracle.lowpass_taps(192, 8, 0.9).astype(np.float32), 8, np.ones((2, 5), np.float32), 1024)
    with pytest.raises(sp.SpiirError):
        fe.run(torch.zeros((2, 100), device="cuda"))      # not a multiple of 8
    with pytest.raises(sp.SpiirError):
        fe.run(torch.zeros((2, 2048), device="cuda"))     # above max_in


def test_raw_strain_to_statistic_in_one_call():
    """spiir_pipeline_run_frontend: 16384 Hz strain of three detectors through the front end,
    the filter bank and the coherent scan per 1 s segment, against the oracle's front end,
    filter bank and scan composed over the same stream."""
    import torch
    import paper_2011_06787_b300 as sp
    from helpers import assert_coherent_close
    n_det, M, Ld, Lw, seg, n_seg = 3, 8, 192, 1025, 16384, 3
    x = _colored(11, n_det, seg * n_seg, (0.9, 0.5, -0.3))
    h = oracle.lowpass_taps(Ld, M, 0.9).astype(np.float32)
    w = np.stack([oracle.whitening_kernel(_psd_ar1(2048.0, 4096, p, 1.0), 2048.0, Lw) for p in (0.8, 0.4, -0.2)]
                 ).astype(np.float32)
    fe = sp.Frontend(n_det, h, M, w, seg)
    det = synth.detectors(11, n_det)
    sigma = synth.noise_weights(11, n_det, 0.5, 2.0)
    bank = synth.random_bank(synth.rng(11, "misc", 1), [30, 200, 77, 410], d_max=1500)
    sky = sp.Sky(*sp.sky_tables(det.pos_m, det.arm_x, det.arm_y, sigma, 4, 2048.0))
    pipe = sp.Pipeline(sp.Bank(n_det, bank.offsets, bank.a1, bank.b0, bank.delay), sky, max_chunk=seg // M)
    T, n, H = bank.n_templates, seg // M, sky.halo
    outs = []
    for s in range(n_seg):
        ms = torch.empty((T, n), device="cuda")
        am = torch.empty((T, n), dtype=torch.int32, device="cuda")
        nl = torch.empty((T, n), device="cuda")
        pipe.run_frontend(fe, torch.from_numpy(np.ascontiguousarray(x[:, s * seg:(s + 1) * seg])).cuda(), ms, am, nl)
        outs.append([v.cpu().numpy() for v in (ms, am, nl)])
    torch.cuda.synchronize()
    sp.device_status()
    y_or, _, _ = oracle.frontend(x, h, M, w)
    z_or, _, _ = oracle.filter_bank(y_or, bank.offsets, bank.a1, bank.b0, bank.delay)
    _, G, d_or = oracle.sky_geometry(det, sigma, 4, 2048.0)
    # output j of segment s is 2048 Hz sample s n + j - H
    zp = np.concatenate([np.zeros((T, n_det, 2 * H)), z_or], axis=2)
    ms_or, am_or, nl_or, sm_or = oracle.coherent(zp, G, d_or, H, n * n_seg, skymap=True)
    ms = np.concatenate([o[0] for o in outs], axis=1)
    am = np.concatenate([o[1] for o in outs], axis=1)
    nl = np.concatenate([o[2] for o in outs], axis=1)
    assert_coherent_close(ms, am, nl, ms_or, am_or, nl_or, sm_or)
    bad = torch.zeros((n_det, 100), device="cuda")                                  # not a multiple of 8
    with pytest.raises(sp.SpiirError):
        pipe.run_frontend(fe, bad, torch.empty((T, n), device="cuda"), torch.empty((T, n), dtype=torch.int32,
                          device="cuda"), torch.empty((T, n), device="cuda"))
