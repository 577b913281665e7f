"""GPU candidate selection and the candidate-driven coherent scan with the time-shift
background (Sec. II.C.1, II.C.3) against the oracle, through the C ABI.

Selection is integer work decided in FP32 on both sides: the records must match exactly.
The coherent values at each (candidate, shift) follow the all-sky scan's tolerances; the
argmax must be the oracle's or, on a near tie, a pixel whose oracle statistic is within
TIE_TOL of the maximum."""
import numpy as np
import pytest

import oracle
import synth
from helpers import NULL_TOL, STAT_TOL, TIE_TOL, cuda_ok

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs CUDA")]


def _cuda(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _sky(cfg, n_det, nside, sig=(0.5, 2.0), rate=2048.0):
    import paper_2011_06787_b300 as sp
    det = synth.detectors(cfg, n_det)
    sigma = synth.noise_weights(cfg, n_det, *sig)
    tabs = sp.sky_tables(det.pos_m, det.arm_x, det.arm_y, sigma, nside, rate)
    _, G, d_or = oracle.sky_geometry(det, sigma, nside, rate)
    np.testing.assert_array_equal(np.asarray(tabs[0]).reshape(d_or.shape), d_or)
    return sp.Sky(*tabs), G, d_or


def _select(z, off, n, thr=4.0, per_second=2048, max_cand=65536):
    import torch
    import paper_2011_06787_b300 as sp
    T, nd, _ = z.shape
    sel = sp.Selector(T, nd, n, per_second, max_cand)
    cand, cnt = sel.select(_cuda(z.astype(np.complex64)), off, thr)
    torch.cuda.synchronize()
    assert int(torch.count_nonzero(sel.workspace)) == 0  # the workspace is left zero
    return sel, cand, cnt


def _same_records(got, want):
    assert [(a, b, c) for a, b, c, _ in got] == [(a, b, c) for a, b, c, _ in want]
    assert [v for *_, v in got] == [v for *_, v in want]  # the same FP32 |z|^2, bit for bit


def _oracle_records(cand, cnt, z, off, n, thr, per_second):
    """The oracle's candidates, after checking that the GPU selected exactly these.  The
    oracle's side of every later comparison is built from them (never from GPU output)."""
    import paper_2011_06787_b300 as sp
    want = oracle.select_candidates(z, off, n, thr, per_second)
    _same_records(sp.Selector.records(cand, cnt), want)
    return want


def test_selection_on_constructed_peaks():
    """The oracle pin's constructed case: maxima over templates, exact threshold, ties between
    templates and within a second, both sides of a second boundary."""
    import paper_2011_06787_b300 as sp
    T, nd, n, sec = 4, 2, 4096, 2048
    z = np.zeros((T, nd, n), np.complex128)
    put = lambda t, I, k, v: z.__setitem__((t, I, k), v * np.exp(0.3j * (k % 7)))
    put(1, 0, 100, 5.0); put(1, 0, 300, 7.0)
    put(2, 0, 497, 4.0)
    put(3, 0, 2100, 6.0)
    put(0, 0, 700, 5.0); put(3, 0, 700, 5.5)
    put(0, 0, 900, 6.0); put(2, 0, 900, 6.0)
    put(2, 0, 1000, 5.0); put(2, 0, 1203, 5.0)
    put(1, 1, 2047, 4.5); put(1, 1, 2048, 4.6)
    _, cand, cnt = _select(z, 0, n, 4.0, sec)
    got = sp.Selector.records(cand, cnt)
    _same_records(got, oracle.select_candidates(z.astype(np.complex64), 0, n, 4.0, sec))
    assert [(a, b, c) for a, b, c, _ in got] == [(0, 0, 900), (0, 1, 300), (0, 2, 1000), (0, 3, 700), (0, 3, 2100),
                                                 (1, 1, 2047), (1, 1, 2048)]


def test_selection_ties_across_template_groups():
    """Equal maxima in templates far apart (the selection splits the bank into groups of 32
    templates): the lowest template wins; a larger value later in the bank still wins."""
    import paper_2011_06787_b300 as sp
    T, nd, n, sec = 100, 2, 96, 32
    z = np.zeros((T, nd, n), np.complex128)
    z[70, 0, 10] = z[5, 0, 10] = 6.0 * np.exp(0.4j)
    z[64, 1, 40] = z[33, 1, 40] = 5.0
    z[99, 1, 40] = 5.5
    z[31, 0, 95] = z[32, 0, 95] = z[63, 0, 95] = 4.5j
    _, cand, cnt = _select(z, 0, n, 4.0, sec)
    got = sp.Selector.records(cand, cnt)
    _same_records(got, oracle.select_candidates(z.astype(np.complex64), 0, n, 4.0, sec))
    assert [(a, b, c) for a, b, c, _ in got] == [(0, 5, 10), (0, 31, 95), (1, 99, 40)]


@pytest.mark.parametrize("T,nd,n,off,per_second,thr", [
    (1, 1, 1, 0, 2048, 0.5),          # one sample, one template
    (37, 3, 5000, 13, 2048, 3.0),     # ragged: T below one unrolled pass, n % 32 != 0, last second short
    (200, 2, 3001, 7, 1000, 3.5),     # T above one pass with a tail of templates
    (1024, 3, 2048, 175, 2048, 4.0),  # the online bank at full size, one second
])
def test_selection_matches_oracle_on_gaussian_snr(T, nd, n, off, per_second, thr):
    import paper_2011_06787_b300 as sp
    z = synth.complex_gaussian_snr(2, (T, nd, off + n + 3), sub=T)
    _, cand, cnt = _select(z, off, n, thr, per_second)
    got = sp.Selector.records(cand, cnt)
    want = oracle.select_candidates(z, off, n, thr, per_second)
    _same_records(got, want)
    if T >= 37:
        assert len(want) > 10


def test_selection_overflow_keeps_the_first_records_and_reports_the_count():
    import paper_2011_06787_b300 as sp
    z = synth.complex_gaussian_snr(3, (64, 3, 4096), sub=1)
    want = oracle.select_candidates(z, 0, 4096, 3.0, 512)
    m = len(want) // 3
    _, cand, cnt = _select(z, 0, 4096, 3.0, 512, max_cand=m)
    assert int(cnt.item()) == len(want)
    _same_records(sp.Selector.records(cand, cnt), want[:m])


def test_selection_of_quiet_data_is_empty_and_repeatable():
    import torch
    import paper_2011_06787_b300 as sp
    z = 0.1 * synth.complex_gaussian_snr(3, (16, 2, 3000), sub=2)
    sel, cand, cnt = _select(z, 0, 3000)
    assert int(cnt.item()) == 0
    z[5, 1, 1234] = 9.0
    zt = _cuda(z)
    for _ in range(2):  # the workspace is zero again after each call
        cand, cnt = sel.select(zt, 0, 4.0)
        torch.cuda.synchronize()
        assert sp.Selector.records(cand, cnt) == [(1, 5, 1234, 81.0)]


def test_nan_snr_is_never_a_candidate():
    """A NaN sample neither becomes a candidate nor hides the real maximum of its sample: the
    records equal the oracle's on the same SNR with the NaN samples set to zero."""
    import paper_2011_06787_b300 as sp
    z = synth.complex_gaussian_snr(5, (12, 2, 3000), sub=3)
    z[4, 0, 100] = np.nan
    z[7, 1, 2000:2010] = np.nan + 1j * np.nan
    z[3, 0, 100] = 9.0                     # the real maximum of sample 100 of detector 0
    _, cand, cnt = _select(z, 0, 3000, 3.5, 1024)
    clean = np.where(np.isnan(z), 0, z)
    _same_records(sp.Selector.records(cand, cnt), oracle.select_candidates(clean, 0, 3000, 3.5, 1024))
    assert (0, 3, 100) in [(a, b, c) for a, b, c, _ in sp.Selector.records(cand, cnt)]


def test_selection_rejects_bad_arguments():
    import torch
    import paper_2011_06787_b300 as sp
    sel = sp.Selector(4, 2, 100)
    z = torch.zeros((4, 2, 100), dtype=torch.complex64, device="cuda")
    with pytest.raises(sp.SpiirError):
        sel.select(z, 1)  # entries 1 .. 100 leave the row
    with pytest.raises(sp.SpiirError):
        sel.select(z, 0, float("nan"))


def _points_oracle(z, G, d_or, pts, shifts):
    """Oracle values at the points, and the oracle's (statistic, null) at a given pixel of a
    point."""
    ms, am, nl = oracle.coherent_points(z, G, d_or, pts, shifts)

    def at(i, p):
        m1, _, n1 = oracle.coherent_points(z, G[[p]], d_or[[p]], pts[i:i + 1], shifts[i:i + 1])
        return m1[0], n1[0]
    return ms, am, nl, at


def _assert_points_close(ms, am, nl, ms_or, am_or, nl_or, at):
    """Statistic within STAT_TOL; the GPU's pixel is the oracle's or one whose oracle statistic
    is within TIE_TOL of the maximum (pixels with the same delay pattern tie exactly for two
    detectors); the null matches the oracle's null at the GPU's pixel."""
    ms = np.asarray(ms, np.float64)
    nl = np.asarray(nl, np.float64)
    assert np.all(np.abs(ms - ms_or) <= STAT_TOL * ms_or), np.max(np.abs(ms - ms_or) / ms_or)
    nl_ref = np.array(nl_or, np.float64)
    for i in np.flatnonzero(am != am_or):
        v, nv = at(i, int(am[i]))
        assert v >= ms_or[i] * (1 - TIE_TOL), i
        nl_ref[i] = nv
    assert np.all(np.abs(nl - nl_ref) <= NULL_TOL * ms_or), np.max(np.abs(nl - nl_ref) / ms_or)


def _companion_shifts(r, nd, s, step):
    return oracle.background_shifts(r, nd, s, step)


@pytest.mark.parametrize("n_det,nside,rate", [
    (2, 4, 2048.0), (3, 8, 2048.0), (4, 4, 2048.0),   # chunked kernel
    (3, 4, 8192.0),                                    # windows wider than 192 samples: one block per item
    (3, 32, 2048.0),                                   # table above shared memory: read through L1
])
def test_foreground_points_match_oracle(n_det, nside, rate):
    """Zero-lag statistic at the selected candidates of Gaussian SNR (every detector serves as
    the reference of some candidates)."""
    import torch
    import paper_2011_06787_b300 as sp
    sky, G, d_or = _sky(4, n_det, nside, rate=rate)
    H = sky.halo
    T, n, off = 24, 3000, 2 * H + 3
    z = synth.complex_gaussian_snr(4, (T, n_det, off + n + 2 * H + 1), sub=n_det)
    sel, cand, cnt = _select(z, off, n, 3.5, 1024)
    recs = _oracle_records(cand, cnt, z, off, n, 3.5, 1024)
    assert len(recs) > 20 and {r for r, *_ in recs} == set(range(n_det))
    ms, am, nl = sp.coherent_candidates(sky, _cuda(z), off, cand, cnt, 0, 1, 205)
    torch.cuda.synchronize()
    m = len(recs)
    pts = np.array([[t, r, off + k] for r, t, k, _ in recs], np.int64)
    shifts = np.zeros((m, n_det), np.int64)
    ms_or, am_or, nl_or, at = _points_oracle(z, G, d_or, pts, shifts)
    _assert_points_close(ms[:m, 0].cpu().numpy(), am[:m, 0].cpu().numpy(), nl[:m, 0].cpu().numpy(),
                         ms_or, am_or, nl_or, at)
    if n_det == 2:
        assert np.all(nl[:m].cpu().numpy() == 0)
    # rows past the count are not written
    assert bool(torch.all(torch.isnan(ms[m:])))


@pytest.mark.parametrize("rate", [2048.0, 8192.0])
def test_background_shifts_match_oracle_and_realign_a_shifted_source(rate):
    """A source whose companion data sit s* c step samples early is realigned by time shift s*
    (Sec. II.C.3); every (candidate, shift) matches the oracle, and a shift whose reads would
    leave the buffer gives (NaN, -1, NaN)."""
    import torch
    import paper_2011_06787_b300 as sp
    sky, G, d_or = _sky(1, 3, 4, (1.0, 1.0), rate)
    H = sky.halo
    step, sstar, n_sh, r = 205, 3, 6, 1
    T, n = 4, 2048
    off = 2 * H + (n_sh - 2) * 2 * step  # shifts up to 4 fit for every candidate; 5 only for late ones
    pitch = off + n + 2 * H
    z = (0.05 * synth.complex_gaussian_snr(6, (T, 3, pitch), sub=1)).astype(np.complex128)
    # a direction every detector sees well, and amplitudes with |amp_r| = 8
    pstar, k0 = int(np.argmax(np.linalg.norm(G, axis=2).min(axis=1))), 1500
    amp = G[pstar] @ np.array([3.0 + 1.0j, -2.0 + 2.5j])
    amp *= 8.0 / abs(amp[r])
    sh = _companion_shifts(r, 3, sstar, step)
    for I in range(3):
        z[2, I, off + k0 + d_or[pstar, I] - d_or[pstar, r] + sh[I]] += amp[I]
    # a second, quiet candidate early in the span, where shift 5 reads before entry 0
    z[1, 0, off + 10] += 5.0
    sel, cand, cnt = _select(z, off, n, 4.0, 2048)
    recs = _oracle_records(cand, cnt, z.astype(np.complex64), off, n, 4.0, 2048)
    assert (r, 2, k0) in [(a, b, c) for a, b, c, _ in recs] and (0, 1, 10) in [(a, b, c) for a, b, c, _ in recs]
    ms, am, nl = sp.coherent_candidates(sky, _cuda(z.astype(np.complex64)), off, cand, cnt, 0, n_sh, step)
    torch.cuda.synchronize()
    ms, am, nl = ms.cpu().numpy(), am.cpu().numpy(), nl.cpu().numpy()
    zc = z.astype(np.complex64)
    dmin = {(a, b): int(np.min(d_or[:, b] - d_or[:, a])) for a in range(3) for b in range(3)}
    for c, (rr, t, k, _) in enumerate(recs):
        for s in range(n_sh):
            shv = _companion_shifts(rr, 3, s, step)
            inside = all(off + k + shv[J] + dmin[(rr, J)] >= 0 for J in range(3))
            if not inside:
                assert np.isnan(ms[c, s]) and am[c, s] == -1 and np.isnan(nl[c, s]), (c, s)
                continue
            pts = np.array([[t, rr, off + k]], np.int64)
            mo, ao, no, at = _points_oracle(zc, G, d_or, pts, shv[None])
            _assert_points_close(ms[c, s:s + 1], am[c, s:s + 1], nl[c, s:s + 1], mo, ao, no, at)
    c = [(a, b, kk) for a, b, kk, _ in recs].index((r, 2, k0))
    assert int(np.argmax(ms[c])) == sstar and am[c, sstar] == pstar
    assert np.isnan(ms[[(a, b, kk) for a, b, kk, _ in recs].index((0, 1, 10)), 5])


@pytest.mark.parametrize("n_det,rate,n_sh", [(2, 2048.0, 20), (3, 2048.0, 20), (4, 2048.0, 20), (4, 4096.0, 4)])
def test_background_points_match_oracle_on_gaussian_snr(n_det, rate, n_sh):
    """Every (candidate, shift) of 20 shifts of 41 samples (chunks of 16 or 8 shifts with a
    ragged last chunk; two, three and four detectors; windows wider than the chunked kernel's
    at 4096 Hz for four detectors) against the oracle; shifts reaching before the buffer give
    (NaN, -1, NaN)."""
    import torch
    import paper_2011_06787_b300 as sp
    sky, G, d_or = _sky(7, n_det, 4, rate=rate)
    H = sky.halo
    step, T, n = 41, 6, 1500
    off = 2 * H + (n_sh // 2) * (n_det - 1) * step  # later shifts leave the buffer for early candidates
    z = synth.complex_gaussian_snr(7, (T, n_det, off + n + 2 * H), sub=10 + n_det)
    sel, cand, cnt = _select(z, off, n, 3.3, 512)
    recs = _oracle_records(cand, cnt, z, off, n, 3.3, 512)
    assert len(recs) > 10
    ms, am, nl = sp.coherent_candidates(sky, _cuda(z), off, cand, cnt, 1, n_sh, step)
    torch.cuda.synchronize()
    ms, am, nl = ms.cpu().numpy(), am.cpu().numpy(), nl.cpu().numpy()
    dmin = {(a, b): int(np.min(d_or[:, b] - d_or[:, a])) for a in range(n_det) for b in range(n_det)}
    pts, shifts, rows, n_out = [], [], [], 0
    for c, (rr, t, k, _) in enumerate(recs):
        for si in range(n_sh):
            shv = _companion_shifts(rr, n_det, 1 + si, step)
            if all(off + k + shv[J] + dmin[(rr, J)] >= 0 for J in range(n_det)):
                pts.append([t, rr, off + k])
                shifts.append(shv)
                rows.append((c, si))
            else:
                assert np.isnan(ms[c, si]) and am[c, si] == -1 and np.isnan(nl[c, si]), (c, si)
                n_out += 1
    assert n_out > 0 and len(rows) > 100
    mo, ao, no, at = _points_oracle(z, G, d_or, np.array(pts, np.int64), np.array(shifts, np.int64))
    _assert_points_close(np.array([ms[c, s] for c, s in rows]), np.array([am[c, s] for c, s in rows]),
                         np.array([nl[c, s] for c, s in rows]), mo, ao, no, at)


def test_online_full_size_candidates_and_background():
    """The online workload's selection (1024 templates, 3 detectors, one 2048-sample second),
    the zero-lag scan on the nside-16 sky and the 100-shift background (0.1 s steps) on the
    nside-8 sky, with 20.5 s of SNR history.  Selection is compared in full; the coherent
    values on a sample of candidates, every shift."""
    import torch
    import paper_2011_06787_b300 as sp
    sky16, G16, d16 = _sky(1, 3, 16)
    sky8, G8, d8 = _sky(1, 3, 8)
    H = max(sky16.halo, sky8.halo)
    T, n, step, n_sh = 1024, 2048, 205, 100
    off = n_sh * 2 * step + 2 * H
    pitch = off + n + 2 * H
    z = synth.complex_gaussian_snr(1, (T, 3, pitch), sub=40)
    zt = _cuda(z)
    sel = sp.Selector(T, 3, n, 2048, 8192)
    cand, cnt = sel.select(zt, off, 4.0)
    fg = sp.coherent_candidates(sky16, zt, off, cand, cnt, 0, 1, step)
    bg = sp.coherent_candidates(sky8, zt, off, cand, cnt, 1, n_sh, step)
    torch.cuda.synchronize()
    recs = _oracle_records(cand, cnt, z, off, n, 4.0, 2048)
    assert 300 < len(recs) <= 8192
    pick = list(range(0, len(recs), max(1, len(recs) // 12)))
    for which, (ms, am, nl), G, dd, s0, ns in ((0, fg, G16, d16, 0, 1), (1, bg, G8, d8, 1, n_sh)):
        ms, am, nl = ms.cpu().numpy(), am.cpu().numpy(), nl.cpu().numpy()
        assert np.isfinite(ms[:len(recs)]).all()
        pts, shifts, rows = [], [], []
        for c in pick:
            rr, t, k, _ = recs[c]
            for s in range(ns):
                pts.append([t, rr, off + k])
                shifts.append(_companion_shifts(rr, 3, s0 + s, step))
                rows.append((c, s))
        pts, shifts = np.array(pts, np.int64), np.array(shifts, np.int64)
        mo, ao, no, at = _points_oracle(z, G, dd, pts, shifts)
        g_ms = np.array([ms[c, s] for c, s in rows])
        g_am = np.array([am[c, s] for c, s in rows])
        g_nl = np.array([nl[c, s] for c, s in rows])
        _assert_points_close(g_ms, g_am, g_nl, mo, ao, no, at)


def _responses(T, F, nr, seed):
    g = np.random.default_rng(seed)
    a1 = (g.uniform(0.8, 0.98, (T, F)) * np.exp(1j * g.uniform(0, 2 * np.pi, (T, F)))).astype(np.complex64)
    b0 = ((g.standard_normal((T, F)) + 1j * g.standard_normal((T, F))) / np.sqrt(2 * F)).astype(np.complex64)
    d = g.integers(0, nr // 3, (T, F)).astype(np.int32)
    off = np.arange(T + 1, dtype=np.int64) * F
    return oracle.impulse_forward(off, a1.ravel(), b0.ravel(), d.ravel(), np.zeros(T * F, np.complex64), nr)


# taps per lane 3, 11, 1, 7 and 13 take the register forms (4, 12, 4, 8 and 16 taps per lane),
# 601 taps the general kernel; 9 and 10 shifts leave a ragged last group of 8
@pytest.mark.parametrize("n_det,Nj,n_sh", [(3, 40, 6), (2, 175, 1), (4, 7, 9), (4, 100, 10), (3, 200, 9), (3, 300, 3)])
def test_xi2_at_candidates_matches_oracle(n_det, Nj, n_sh):
    """xi_C^2 at each (candidate, shift) item at the oracle's coherent argmax, against the
    oracle's xi^2 on a one-sample window at each detector's implied time; items whose reads
    leave the buffer are NaN."""
    import torch
    import paper_2011_06787_b300 as sp
    sky, G, d_or = _sky(3, n_det, 4)
    H = sky.halo
    T, n, step = 8, 1200, 37
    off = 2 * H + Nj + (n_sh // 2) * (n_det - 1) * step
    z = synth.complex_gaussian_snr(8, (T, n_det, off + n + 2 * H + Nj + 1), sub=n_det)
    A = oracle.autocorr(_responses(T, 30, 1500, seed=n_det), Nj).astype(np.complex64)
    sel, cand, cnt = _select(z, off, n, 3.2, 400)
    recs = _oracle_records(cand, cnt, z, off, n, 3.2, 400)
    assert len(recs) > 5
    dmin = {(a, b): int(np.min(d_or[:, b] - d_or[:, a])) for a in range(n_det) for b in range(n_det)}
    # the oracle's coherent argmax of every item (NaN items keep -1)
    am = np.full((sel.max_cand, n_sh), -1, np.int32)
    for c, (r, t, k, _) in enumerate(recs):
        for si in range(n_sh):
            shv = oracle.background_shifts(r, n_det, si, step)
            if all(off + k + shv[J] + dmin[(r, J)] >= 0 for J in range(n_det)):
                _, a_or, _ = oracle.coherent_points(z, G, d_or, np.array([[t, r, off + k]], np.int64), shv[None])
                am[c, si] = a_or[0]
    xi, xd = sp.xi2_candidates(sky, _cuda(z), off, _cuda(A), Nj, cand, cnt, _cuda(am), 0, n_sh, step, per_detector=True)
    torch.cuda.synchronize()
    xi, xd = xi.cpu().numpy(), xd.cpu().numpy()
    n_nan = 0
    for c, (r, t, k, _) in enumerate(recs):
        for si in range(n_sh):
            p = int(am[c, si])
            shv = oracle.background_shifts(r, n_det, si, step)
            xs = [off + k + int(d_or[p, J]) - int(d_or[p, r]) + int(shv[J]) for J in range(n_det)] if p >= 0 else []
            if p < 0 or any(x - Nj < 0 for x in xs):
                assert np.isnan(xi[c, si]) and np.isnan(xd[c, si]).all(), (c, si)
                n_nan += 1
                continue
            want = [oracle.xi2(z[t:t + 1, J:J + 1, x - Nj: x + Nj + 1], A[t:t + 1], Nj, 1)[0, 0, 0]
                    for J, x in enumerate(xs)]
            np.testing.assert_allclose(xd[c, si], want, rtol=1e-4, atol=1e-4)
            np.testing.assert_allclose(xi[c, si], np.mean(want), rtol=1e-4, atol=1e-4)
    assert bool(np.all(np.isnan(xi[len(recs):])))
    if n_sh > 1:
        assert n_nan > 0
