"""Candidate-driven streaming search (Sec. II.C.1 - II.C.3) through spiir_search_run: the filter
bank's own output on injected chirps in white noise, per chunk, against the FP64 oracle's
filter bank, selection, coherent statistic at the candidates (zero lag and time shifts) and
xi^2, composed over a plain linear stream.

The oracle's SNR and the GPU's differ at rounding level, so selection decisions whose margin in
the oracle's FP32 |z|^2 is within tolerance (threshold, the largest template of a sample, the
largest sample of a (template, second)) may go either way; every other candidate matches bit
for bit in (detector, template, sample), and |z|^2, statistic, null and xi^2 match within the
parity tolerances."""
import math

import numpy as np
import pytest

import oracle
import synth
from helpers import NULL_TOL, STAT_TOL, TIE_TOL, cuda_ok

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs CUDA")]

MARGIN = 1e-4   # relative margin of a selection decision below which either outcome is valid


def _chirp_bank(mcs, n_filters, f_lo):
    """Chirp templates (synth.chirp_fit of conj(h), time-reversed Newtonian chirp from f_lo),
    b0 scaled so that E|z|^2 = 2 in unit white noise."""
    A, B, D = [], [], []
    for mc in mcs:
        a1, b0, d, _, power = synth.chirp_fit(float(mc), n_filters, f_lo=f_lo)
        A.append(a1)
        B.append(b0 * math.sqrt(2.0 / power))
        D.append(d)
    off = np.arange(len(mcs) + 1, dtype=np.int64) * n_filters
    return synth.Bank(off, np.concatenate(A).astype(np.complex64), np.concatenate(B).astype(np.complex64),
                      np.concatenate(D).astype(np.int32))


def _strain(cfg, det, sigma, N, inj):
    """Unit white noise plus chirps: (mc, f_lo, geocentric coalescence sample, direction, psi,
    network SNR) per injection; detector I sees the chirp at its integer arrival offset."""
    nd = sigma.size
    x = synth.white_noise(cfg, nd, N, sub=77).astype(np.float64)
    for mc, f_lo, tc, nh, psi, snr in inj:
        hf = synth.newtonian_chirp(mc, f_lo=f_lo)[::-1]
        Fp, Fc = oracle.antenna_patterns(det.arm_x, det.arm_y, nh[None], psi)
        dl = oracle.arrival_delays(det.pos_m, nh[None], 2048.0)[0]
        s = sigma[:, None] * (Fp[0][:, None] * hf.real[None, :] + Fc[0][:, None] * hf.imag[None, :])
        amp = snr / math.sqrt(float(np.sum(s ** 2)))
        for I in range(nd):
            start = tc + int(dl[I]) - (hf.size - 1)
            x[I, start: start + hf.size] += amp * s[I]
    return x.astype(np.float32)


def _m2(z):
    """FP32 |z|^2 with each operation rounded, as both sides decide on."""
    z = np.asarray(z).astype(np.complex64)
    re, im = z.real.astype(np.float32), z.imag.astype(np.float32)
    return re * re + im * im


def _ambiguous(zspan, rec, thr, per_second):
    """True when the selection of the record's (detector, template, second) is decided within
    MARGIN in the oracle's values (zspan [T][n_det][n], the oracle SNR of the span): at some
    sample of the second the template is within MARGIN of the largest |z|^2 together with
    another template, or is (near) the largest and within MARGIN of the threshold; or two of
    the template's candidate samples in the second are within MARGIN of each other."""
    I, t, k = rec
    m2 = _m2(zspan[:, I, :])
    thr2 = float(np.float32(thr) * np.float32(thr))
    sec = k // per_second
    blk = m2[:, sec * per_second: min((sec + 1) * per_second, m2.shape[1])].astype(np.float64)
    mx = blk.max(axis=0)
    near_t = (blk[t] >= mx * (1 - MARGIN)) & (mx > thr2 * (1 - MARGIN))
    shared = (blk >= (mx * (1 - MARGIN))[None, :]).sum(axis=0) > 1
    if np.any(near_t & shared) or np.any(near_t & (np.abs(mx - thr2) <= MARGIN * thr2)):
        return True
    own = np.sort(mx[(np.argmax(blk, axis=0) == t) & (mx > thr2)])
    return own.size > 1 and own[-1] - own[-2] <= MARGIN * own[-1]


def _check_point(ms, am, nl, zp, G, d_or, pt, shift):
    """GPU (max, argmax, null) at one point against the oracle: statistic within STAT_TOL; the
    pixel is the oracle's or one within TIE_TOL of the maximum; the null matches at that pixel.
    Returns the pixel the oracle accepts for the GPU's choice."""
    mo, ao, no = oracle.coherent_points(zp, G, d_or, pt[None], shift[None])
    assert abs(ms - mo[0]) <= STAT_TOL * mo[0], (ms, mo[0])
    p = int(am)
    if p != int(ao[0]):
        m1, _, n1 = oracle.coherent_points(zp, G[[p]], d_or[[p]], pt[None], shift[None])
        assert m1[0] >= mo[0] * (1 - TIE_TOL), (p, int(ao[0]))
        no = n1
    assert abs(nl - no[0]) <= NULL_TOL * mo[0]
    return p


def _xi2_oracle(zp, A, Nj, t, r, e, p, d_or, shift):
    n_det = zp.shape[1]
    vals = []
    for J in range(n_det):
        x = e + int(d_or[p, J]) - int(d_or[p, r]) + int(shift[J])
        vals.append(oracle.xi2(zp[t:t + 1, J:J + 1, x - Nj: x + Nj + 1], A[t:t + 1], Nj, 1)[0, 0, 0])
    return float(np.mean(vals))


@pytest.mark.parametrize("case,nd,overlap", [("short", 3, False), ("paper", 3, False), ("short", 2, False),
                                             ("short", 4, False), ("short", 3, True), ("paper", 3, True)])
def test_search_on_injected_chirps_matches_the_oracle(case, nd, overlap):
    """Three detectors with short and with the paper's shifts; two (null stream zero) and four
    detectors (three companions per candidate) with short shifts; the overlapped mode (the span
    of the previous chunk analysed beside the filter bank) with three detectors."""
    import torch
    import paper_2011_06787_b300 as sp
    cfg = 5
    if case == "short":
        T, F, f_lo, n_sh, step, Nj, nside_fg, nside_bg, n_chunks = 12, 120, 80.0, 20, 205, 60, 8, 4, 9
        if nd == 4:
            n_sh, n_chunks = 12, 10
        check_shifts = range(n_sh)
    else:
        T, F, f_lo, n_sh, step, Nj, nside_fg, nside_bg, n_chunks = 8, 100, 90.0, 100, 205, 175, 16, 8, 24
        check_shifts = range(0, n_sh, 9)
    chunk, thr, per_second = 2048, 4.0, 2048
    det = synth.detectors(cfg, nd)
    sigma = synth.noise_weights(cfg, nd, 0.5, 2.0)
    mcs = np.linspace(1.1, 2.2, T)
    bank = _chirp_bank(mcs, F, f_lo)
    N = n_chunks * chunk
    g = synth.rng(cfg, "inject", 9)
    nh = g.standard_normal((2, 3))
    nh /= np.linalg.norm(nh, axis=1, keepdims=True)
    inj = [(float(mcs[3]), f_lo, N - 3 * chunk + 700, nh[0], 0.3, 18.0),
           (float(mcs[T - 2]), f_lo, N - chunk - 900, nh[1], 1.1, 15.0)]
    x = _strain(cfg, det, sigma, N, inj)
    # autocorrelations of the templates' responses (oracle impulse responses), an input of both sides
    u = oracle.impulse_forward(bank.offsets, bank.a1, bank.b0, bank.delay, np.zeros(bank.n_filters, np.complex64),
                               int(bank.delay.max()) + 4096)
    A = oracle.autocorr(u, Nj).astype(np.complex64)

    skf = sp.Sky(*sp.sky_tables(det.pos_m, det.arm_x, det.arm_y, sigma, nside_fg, 2048.0))
    skb = sp.Sky(*sp.sky_tables(det.pos_m, det.arm_x, det.arm_y, sigma, nside_bg, 2048.0))
    _, Gf, df = oracle.sky_geometry(det, sigma, nside_fg, 2048.0)
    _, Gb, db = oracle.sky_geometry(det, sigma, nside_bg, 2048.0)
    b = sp.Bank(nd, bank.offsets, bank.a1, bank.b0, bank.delay)
    At = torch.from_numpy(A).cuda()
    srch = sp.Search(b, skf, skb, At, Nj, chunk, thr, per_second, n_sh, step, max_cand=4096, overlap=overlap)
    L, Hb, La, _ = srch.info()
    H = max(skf.halo, skb.halo)
    lag = chunk if overlap else 0  # the overlapped mode analyses the previous call's span
    assert La == 2 * H + Nj and Hb == n_sh * (nd - 1) * step + 2 * H + Nj and L == Hb + chunk + lag + La
    assert N > L    # the ring wraps around

    # oracle: the whole stream through the FP64 bank, zero before the stream start
    oracle.set_threads(16)
    z_or, _, _ = oracle.filter_bank(x, bank.offsets, bank.a1, bank.b0, bank.delay)
    pad = Hb + La + lag
    zp = np.concatenate([np.zeros((T, nd, pad)), z_or], axis=2)

    n_matched = n_diff = 0
    found = set()
    for c in range(n_chunks):
        xc = torch.from_numpy(np.ascontiguousarray(x[:, c * chunk:(c + 1) * chunk])).cuda()
        S0 = srch.run(xc)
        torch.cuda.synchronize()
        assert S0 == (c + 1) * chunk - chunk - La - lag
        cnt = int(srch.n_cand.item())
        assert cnt <= srch.max_cand
        got = [tuple(r) for r in srch.cand[:cnt].cpu().numpy()]
        e0 = S0 + pad                               # zp entry of span sample 0
        want = oracle.select_candidates(zp, e0, chunk, thr, per_second)
        zspan = zp[:, :, e0:e0 + chunk]
        g_set = {(I, t, k): i for i, (I, t, k, _) in enumerate(got)}
        w_set = {(I, t, k): v for I, t, k, v in want}
        for key in set(g_set) ^ set(w_set):
            assert _ambiguous(zspan, key, thr, per_second), (c, key)
            n_diff += 1
        fg = [v.cpu().numpy() for v in srch.fg]
        bg = [v.cpu().numpy() for v in srch.bg]
        for key, i in g_set.items():
            if key not in w_set:
                continue
            n_matched += 1
            I, t, k = key
            m2g = np.array([got[i][3]], np.int32).view(np.float32)[0]
            assert abs(float(m2g) - w_set[key]) <= 2e-4 * w_set[key], (c, key)
            if S0 + k >= 0:
                for tc_i, (_, _, tc, _, _, _) in enumerate(inj):
                    if abs(S0 + k - tc) <= 64:
                        found.add(tc_i)
            pt = np.array([t, I, e0 + k], np.int64)
            zero = np.zeros(nd, np.int64)
            p = _check_point(fg[0][i], fg[1][i], fg[2][i], zp, Gf, df, pt, zero)
            want_xi = _xi2_oracle(zp, A, Nj, t, I, e0 + k, p, df, zero)
            assert abs(fg[3][i] - want_xi) <= 1e-4 * max(1.0, want_xi), (c, key, fg[3][i], want_xi)
            for si in check_shifts:
                sh = oracle.background_shifts(I, nd, si + 1, step)
                p = _check_point(bg[0][i, si], bg[1][i, si], bg[2][i, si], zp, Gb, db, pt, sh)
                want_xi = _xi2_oracle(zp, A, Nj, t, I, e0 + k, p, db, sh)
                assert abs(bg[3][i, si] - want_xi) <= 1e-4 * max(1.0, want_xi), (c, key, si)
    sp.device_status()
    if nd == 2:
        assert np.all(srch.fg[2].cpu().numpy()[:cnt] == 0)    # no null stream with two detectors
    assert n_matched > 30 and n_diff <= max(3, n_matched // 50), (n_matched, n_diff)
    assert found == {0, 1}      # both injections give candidates near their coalescence


def test_search_rejects_bad_arguments_and_resets():
    import torch
    import paper_2011_06787_b300 as sp
    det = synth.detectors(5, 3)
    sigma = synth.noise_weights(5, 3, 0.5, 2.0)
    sky = sp.Sky(*sp.sky_tables(det.pos_m, det.arm_x, det.arm_y, sigma, 4, 2048.0))
    det2 = synth.detectors(5, 2)
    sky2 = sp.Sky(*sp.sky_tables(det2.pos_m, det2.arm_x, det2.arm_y, sigma[:2], 4, 2048.0))
    bank = synth.random_bank(synth.rng(5, "misc", 1), [20, 30], d_max=300)
    b = sp.Bank(3, bank.offsets, bank.a1, bank.b0, bank.delay)
    A = torch.zeros((2, 2 * 10 + 1), dtype=torch.complex64, device="cuda")
    A[:, 10] = 1.0
    with pytest.raises(sp.SpiirError):
        sp.Search(b, sky, sky2, A, 10, 512)               # detector counts differ
    with pytest.raises(sp.SpiirError):
        sp.Search(b, sky, sky, A, 2000, 512)              # n_lags above 1024
    s = sp.Search(b, sky, sky, A, 10, 512, n_shifts=0, max_cand=64)
    x = torch.from_numpy(synth.white_noise(5, 3, 512, sub=3)).cuda()
    s0 = s.run(x)
    c1 = s.cand.clone(), s.n_cand.clone(), s.fg[0].clone()
    s1 = s.run(x)
    assert s1 == s0 + 512
    s.reset()
    assert s.info()[3] == s0
    assert s.run(x) == s0
    torch.cuda.synchronize()
    assert torch.equal(s.n_cand, c1[1])
    n = int(c1[1].item())
    assert torch.equal(s.cand[:n], c1[0][:n]) and torch.equal(s.fg[0][:n], c1[2][:n])
    with pytest.raises(sp.SpiirError):
        s.run(torch.zeros((3, 100), dtype=torch.float32, device="cuda"))   # rows shorter than a chunk


@pytest.mark.parametrize("overlap", [False, True])
def test_search_candidate_overflow_keeps_the_first_records(overlap):
    """With max_cand below the number of candidates, the first max_cand records and their
    zero-lag, background and xi^2 results are those of a search with room for all of them,
    and the count reports the total."""
    import torch
    import paper_2011_06787_b300 as sp
    det = synth.detectors(5, 3)
    sigma = synth.noise_weights(5, 3, 0.5, 2.0)
    sky = sp.Sky(*sp.sky_tables(det.pos_m, det.arm_x, det.arm_y, sigma, 4, 2048.0))
    bank = synth.random_bank(synth.rng(5, "misc", 2), [20, 30, 25, 18], d_max=300)
    A = torch.zeros((4, 2 * 10 + 1), dtype=torch.complex64, device="cuda")
    A[:, 10] = 1.0
    kw = dict(threshold=0.5, per_second=64, n_shifts=3, shift_step=40, overlap=overlap)
    big = sp.Search(sp.Bank(3, bank.offsets, bank.a1, bank.b0, bank.delay), sky, sky, A, 10, 512, max_cand=4096, **kw)
    small = sp.Search(sp.Bank(3, bank.offsets, bank.a1, bank.b0, bank.delay), sky, sky, A, 10, 512, max_cand=8, **kw)
    for c in range(5):
        x = torch.from_numpy(synth.white_noise(5, 3, 512, sub=40 + c)).cuda()
        assert big.run(x) == small.run(x)
        torch.cuda.synchronize()
        n = int(big.n_cand.item())
        if overlap and c == 0:
            assert n == 0       # the first span lies before the stream start
            continue
        assert n > 8 and int(small.n_cand.item()) == n
        assert torch.equal(small.cand[:8], big.cand[:8])
        for a, b in zip(small.fg, big.fg):
            assert torch.equal(a[:8], b[:8]) or torch.allclose(a[:8], b[:8], equal_nan=True, rtol=0, atol=0)
        for a, b in zip(small.bg, big.bg):
            assert torch.equal(a[:8], b[:8]) or torch.allclose(a[:8], b[:8], equal_nan=True, rtol=0, atol=0)
    sp.device_status()
