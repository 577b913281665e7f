"""Scale workload at full size: 3 detectors, 60 s of 2048 Hz noise in 1 s chunks, 20 injected
Newtonian chirps (chirp mass 1-3 Msun, network SNR 8-20, isotropic sky), a bank of 4096
chirp templates x 600 IIR filters and a coherent scan over HEALPix nside 32 (12288 pixels)
with the null stream.  Each injection's best template and time on the GPU are recomputed by
the FP64 oracle over a window around the injection: statistic, null and argmax pixel agree
within the parity tolerances, so the sky pixel is recovered within one pixel of the
oracle's.  The batched persistent path (one full-rate band) is checked against the plain
path on the same stream."""
import math

import numpy as np
import pytest

import oracle
import synth
from helpers import assert_coherent_close, cuda_ok

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs CUDA")]

HALF = 256  # half-width of the window around each injection (samples)


def _strain(det, sigma, inj, tmpl_len, tmpl_mc):
    """Unit white noise plus the injections.  Detector I sees the geocentric waveform
    shifted by its integer arrival offset Delta_I (the scan's own convention), weighted by
    sigma_I (F+ h+ + Fx hx); amplitudes are set so that the network SNR over the part a
    template covers is the drawn value."""
    c = synth.SCALE
    N = c["n_chunks"] * c["chunk"]
    x = synth.white_noise(c["index"], 3, N).astype(np.float64)
    for i in range(inj["mc"].size):
        hf = synth.newtonian_chirp(float(inj["mc"][i]))[::-1] * np.exp(1j * inj["phic"][i])
        ci = inj["cosi"][i]
        hp, hc = 0.5 * (1.0 + ci * ci) * hf.real, ci * hf.imag
        nh = inj["nhat"][i:i + 1]
        Fp, Fc = oracle.antenna_patterns(det.arm_x, det.arm_y, nh, float(inj["psi"][i]))
        dl = oracle.arrival_delays(det.pos_m, nh, 2048.0)[0]
        s = sigma[:, None] * (Fp[0][:, None] * hp[None, :] + Fc[0][:, None] * hc[None, :])
        L = min(hf.size, int(tmpl_len[np.argmin(np.abs(tmpl_mc - inj["mc"][i]))]))
        amp = inj["snr"][i] / math.sqrt(float(np.sum(s[:, -L:] ** 2)))
        for I in range(3):
            start = int(inj["tc"][i]) + int(dl[I]) - (hf.size - 1)
            lo = max(0, -start)
            x[I, start + lo: start + hf.size] += amp * s[I, lo:]
    return x.astype(np.float32)


def _angle_deg(a, b):
    return math.degrees(math.acos(max(-1.0, min(1.0, float(np.dot(a, b))))))


def test_scale_injections_recovered_within_one_pixel_of_the_oracle():
    import torch
    import paper_2011_06787_b300 as sp
    c = synth.SCALE
    det = synth.detectors(c["index"], 3)
    sigma = synth.noise_weights(c["index"], 3, *c["sigma"])
    bank, tmpl_mc, tmpl_len = synth.scale_bank()
    inj = synth.scale_injections()
    x = _strain(det, sigma, inj, tmpl_len, tmpl_mc)
    N, n = x.shape[1], c["chunk"]

    sky = sp.Sky(*sp.sky_tables(det.pos_m, det.arm_x, det.arm_y, sigma, c["nside"], 2048.0))
    nhat_pix, G, d_or = oracle.sky_geometry(det, sigma, c["nside"], 2048.0)
    H = sky.halo
    T = bank.n_templates
    # chunks holding each injection's window; output j of chunk k is geocentric k n - H + j
    need = set()
    for tc in inj["tc"]:
        for g in (int(tc) - HALF, int(tc) + HALF - 1):
            need.add((g + H) // n)

    def stream(run):
        kept = {}
        for k in range(N // n):
            outs = run(torch.from_numpy(np.ascontiguousarray(x[:, k * n:(k + 1) * n])).cuda())
            if k in need:
                kept[k] = [o.clone() for o in outs]
        torch.cuda.synchronize()
        return kept

    b = sp.Bank(3, bank.offsets, bank.a1, bank.b0, bank.delay)
    pipe = sp.Pipeline(b, sky, max_chunk=n)
    ms = torch.empty((T, n), dtype=torch.float32, device="cuda")
    am = torch.empty((T, n), dtype=torch.int32, device="cuda")
    nl = torch.empty((T, n), dtype=torch.float32, device="cuda")

    def run_plain(xc):
        pipe.run(xc, ms, am, nl)
        return ms, am, nl

    kept = stream(run_plain)

    def window(kept, tc, t=None):
        g0 = int(tc) - HALF
        cols = [(g + H) // n for g in range(g0, g0 + 2 * HALF)]
        outs = []
        for o in range(3):
            parts = [kept[k][o][:, (g + H) - k * n] for g, k in zip(range(g0, g0 + 2 * HALF), cols)]
            w = torch.stack(parts, dim=1)
            outs.append(w if t is None else w[t])
        return outs

    picks = []
    for i, tc in enumerate(inj["tc"]):
        wms, _, _ = window(kept, tc)
        flat = int(torch.argmax(wms))
        t, k = flat // (2 * HALF), flat % (2 * HALF)
        picks.append((t, k))
        if inj["snr"][i] >= 12.0:
            # a loud injection is found near its time by a template of nearly its chirp mass
            # (the coherent maximum of a long low-mass chirp can sit tens of samples from the
            # coalescence: its correlation envelope is broad and the sky delays absorb part of
            # a time shift)
            assert abs(k - HALF) <= 64, (i, k - HALF)
            assert abs(tmpl_mc[t] - inj["mc"][i]) <= 0.05 * inj["mc"][i], (i, tmpl_mc[t], inj["mc"][i])
            assert float(wms[t, k]) > 0.5 * inj["snr"][i] ** 2

    tsel = sorted({t for t, _ in picks})
    sub = bank.subset(tsel)
    oracle.set_threads(16)
    z_or, _, _ = oracle.filter_bank(x, sub.offsets, sub.a1, sub.b0, sub.delay)
    for i, (tc, (t, k)) in enumerate(zip(inj["tc"], picks)):
        g0 = int(tc) - HALF
        zw = z_or[tsel.index(t)][None, :, g0 - H: g0 + 2 * HALF + H]
        ms_or, am_or, nl_or, sm_or = oracle.coherent(zw, G, d_or, H, 2 * HALF, skymap=True)
        gms, gam, gnl = [w.cpu().numpy()[None] for w in window(kept, tc, t)]
        assert_coherent_close(gms, gam, gnl, ms_or, am_or, nl_or, sm_or)
        # the recovered pixel at the detection is within one pixel of the oracle's
        p_gpu, p_or = int(gam[0, k]), int(am_or[0, k])
        assert _angle_deg(nhat_pix[p_gpu], nhat_pix[p_or]) <= 1.5 * math.degrees(math.sqrt(4 * math.pi / 12288)), i

    # batched persistent path, one full-rate band (M = 1: no decimation, no upsampling lag):
    # the plain path's results
    bt = sp.Batch(3, [(bank.offsets, bank.a1, bank.b0, bank.delay, np.zeros(bank.n_filters, np.int32))], (1,), sky, n)
    bms = torch.empty((T, n), dtype=torch.float32, device="cuda")
    bam = torch.empty((T, n), dtype=torch.int32, device="cuda")
    bnl = torch.empty((T, n), dtype=torch.float32, device="cuda")

    def run_batch(xc):
        bt.run(xc, bms, bam, bnl, mode=2)
        return bms, bam, bnl

    kept_b = stream(run_batch)
    for k in sorted(need):
        p_ms, p_am, _ = kept[k]
        q_ms, q_am, _ = kept_b[k]
        assert torch.all(torch.abs(p_ms - q_ms) <= 1e-5 * torch.abs(p_ms) + 1e-5), k
        assert float((p_am == q_am).float().mean()) > 0.999, k
