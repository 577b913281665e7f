"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: closed forms,
brute force on tiny inputs, special cases that reduce to a textbook result,
statistical invariants or values printed in the paper (tests/golden/).
"""
import math

import numpy as np
import pytest

import oracle
import synth
from conftest import golden_rows


def _rng(seed=0):
    return np.random.default_rng(seed)


# ---------------------------------------------------------------------------------------------
# Filter bank (Sec. II.B.1 Eq. (zk))


def test_single_filter_impulse_response_closed_form():
    # commented closed form beside Eq. (zk): u(t) = b a^(t - t_d) for one filter
    a = 0.95 * np.exp(0.3j)
    b = 0.4 - 0.2j
    d, n = 7, 200
    x = np.zeros((1, n))
    x[0, 0] = 1.0
    z, _, _ = oracle.filter_bank(x, [0, 1], [a], [b], [d])
    k = np.arange(n)
    expect = np.where(k >= d, b * a ** np.maximum(k - d, 0), 0.0)
    np.testing.assert_allclose(z[0, 0], expect, rtol=1e-12, atol=1e-15)


def test_single_filter_initial_state_decays_geometrically():
    a = 0.9 * np.exp(-1.1j)
    s = 0.3 + 0.7j
    n = 50
    z, st, _ = oracle.filter_bank(np.zeros((1, n)), [0, 1], [a], [1.0], [3], state=np.array([[s]]))
    np.testing.assert_allclose(z[0, 0], s * a ** (np.arange(n) + 1), rtol=1e-12)
    np.testing.assert_allclose(st[0, 0], s * a ** n, rtol=1e-12)


def test_complex_exponential_input_geometric_series():
    a = 0.97 * np.exp(0.8j)
    b = -0.3 + 0.5j
    d, n, w = 5, 300, 0.37
    k = np.arange(n)
    x = np.exp(1j * w * k)[None, :]
    z, _, _ = oracle.filter_bank(x, [0, 1], [a], [b], [d])
    r = a * np.exp(-1j * w)
    m = k - d
    expect = np.where(m >= 0, b * np.exp(1j * w * m) * (1 - r ** (np.maximum(m, 0) + 1)) / (1 - r), 0)
    np.testing.assert_allclose(z[0, 0], expect, rtol=1e-11, atol=1e-13)


def test_real_cosine_input_is_sum_of_two_exponentials():
    a = 0.93 * np.exp(-0.4j)
    b = 0.25 + 0.1j
    d, n, w, phi = 11, 256, 1.3, 0.6
    k = np.arange(n)
    x = np.cos(w * k + phi)[None, :]
    z, _, _ = oracle.filter_bank(x, [0, 1], [a], [b], [d])
    m = k - d
    mm = np.maximum(m, 0)

    def S(om):
        r = a * np.exp(-1j * om)
        return (1 - r ** (mm + 1)) / (1 - r)

    expect = 0.5 * b * (np.exp(1j * phi) * np.exp(1j * w * m) * S(w) + np.exp(-1j * phi) * np.exp(-1j * w * m) * S(-w))
    expect = np.where(m >= 0, expect, 0)
    np.testing.assert_allclose(z[0, 0], expect, rtol=1e-11, atol=1e-13)


def test_bank_equals_direct_convolution_with_truncated_impulse_responses():
    g = _rng(1)
    counts = [3, 1, 5]
    bank = synth.random_bank(g, counts, d_max=9)
    n_det, n = 2, 120
    x = g.standard_normal((n_det, n))
    z, _, _ = oracle.filter_bank(x, bank.offsets, bank.a1, bank.b0, bank.delay)
    a1 = bank.a1.astype(np.complex128)
    b0 = bank.b0.astype(np.complex128)
    for t in range(3):
        for I in range(n_det):
            ref = np.zeros(n, dtype=np.complex128)
            for l in range(bank.offsets[t], bank.offsets[t + 1]):
                h = np.zeros(n, dtype=np.complex128)  # impulse response of filter l
                for k in range(bank.delay[l], n):
                    h[k] = b0[l] * a1[l] ** (k - bank.delay[l])
                for k in range(n):
                    ref[k] += sum(h[j] * x[I, k - j] for j in range(k + 1))
            np.testing.assert_allclose(z[t, I], ref, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("chunk", [1, 7, 64, 333])
def test_streaming_in_chunks_equals_one_shot(chunk):
    g = _rng(2)
    bank = synth.random_bank(g, [4, 6], d_max=40)
    x = g.standard_normal((3, 700))
    z1, st1, _ = oracle.filter_bank(x, bank.offsets, bank.a1, bank.b0, bank.delay)
    D = int(bank.delay.max())
    state, hist, parts = None, np.zeros((3, D)), []
    for s in range(0, 700, chunk):
        zc, state, hist = oracle.filter_bank(x[:, s:s + chunk], bank.offsets, bank.a1, bank.b0, bank.delay,
                                             state=state, history=hist)
        parts.append(zc)
    np.testing.assert_array_equal(np.concatenate(parts, axis=2), z1)
    np.testing.assert_array_equal(state, st1)


def test_cost_model_matches_paper_filtering_demand():
    # Sec. II.B.2: 12 flops per filter per sample; 412000 templates x ~350 filters x 2048 Hz
    # x 3 detectors is "about 10.6 TFLOPS".
    assert abs(12 * 350 * 412000 * 2048 * 3 / 1e12 - 10.6) < 0.05


# ---------------------------------------------------------------------------------------------
# Sky grid and geometry


def test_healpix_base_pixels_and_ring_structure():
    rows = golden_rows("healpix_base.txt")
    c1 = oracle.healpix_centres(1)
    assert c1.shape == (12, 3)
    for r in rows:
        if r[0] != "1":
            continue
        p, z, phi = int(r[1]), float(r[2]), float(r[3])
        assert abs(c1[p, 2] - z) < 1e-12
        ph = math.degrees(math.atan2(c1[p, 1], c1[p, 0])) % 360.0
        assert abs(ph - phi) < 1e-9
    c2 = oracle.healpix_centres(2)
    assert c2.shape == (48, 3)
    zs = c2[:, 2]
    start = 0
    for r in rows:
        if r[0] != "2":
            continue
        zr, cnt = float(r[2]), int(r[3])
        np.testing.assert_allclose(zs[start:start + cnt], zr, atol=1e-12)
        start += cnt
    assert start == 48


@pytest.mark.parametrize("nside", [4, 16])
def test_healpix_counts_unit_vectors_and_symmetry(nside):
    c = oracle.healpix_centres(nside)
    assert c.shape == (12 * nside * nside, 3)  # Sec. II.C.1: nside 16 gives the 3072 tiles
    np.testing.assert_allclose(np.linalg.norm(c, axis=1), 1.0, atol=1e-12)
    np.testing.assert_allclose(c.sum(axis=0), 0.0, atol=1e-9)
    # the north polar cap (centres above z = 2/3) holds rings 1..nside-1 with 4i pixels each
    assert np.sum(c[:, 2] > 2.0 / 3.0 + 1e-12) == 2 * nside * (nside - 1)
    # equal-area belt: every belt ring holds 4 nside pixels, at z = 4/3 - 2i/(3 nside)
    zb = np.round(c[np.abs(c[:, 2]) <= 2.0 / 3.0 + 1e-12, 2] * 3 * nside) / (3 * nside)
    vals, cnt = np.unique(zb, return_counts=True)
    assert vals.size == 2 * nside + 1 and np.all(cnt == 4 * nside)


def test_healpix_nside16_tile_spacing_matches_paper():
    # Sec. II.C.1 quotes 1.9 deg from a tile centre to its boundary for 3072 tiles.  For
    # equal-area tiles the typical centre spacing is sqrt(4 pi / 3072) = 3.66 deg, so the
    # typical half-width is 1.83 deg; the worst case is at the poles, where four ring-1
    # tiles meet at a vertex arccos(1 - 1/(3 nside^2)) = 2.92 deg from their centres.
    c = oracle.healpix_centres(16)
    nn = np.degrees(np.arccos(np.clip(np.sort(c @ c.T, axis=1)[:, -2], -1, 1)))
    typical = math.degrees(math.sqrt(4 * math.pi / 3072))
    assert abs(np.median(nn) - typical) < 0.02 * typical
    assert abs(0.5 * typical - 1.9) < 0.1
    pole = math.degrees(math.acos(1 - 1 / (3 * 16 * 16)))
    assert abs(math.degrees(math.acos(c[0, 2])) - pole) < 1e-9
    g = _rng(3)
    v = g.standard_normal((20000, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    ang = np.degrees(np.arccos(np.clip((v @ c.T).max(axis=1), -1, 1)))
    assert ang.max() <= pole + 1e-9 and abs(np.median(ang) - 0.4 * typical) < 0.2


def test_antenna_patterns_textbook_detector_at_pole():
    # L-shaped detector at the north pole, arms along x and y: for psi = 0,
    # F+ = (1 + cos^2 th) cos(2 ph) / 2 and Fx = cos th sin(2 ph).
    g = _rng(4)
    th = g.uniform(0, math.pi, 50)
    ph = g.uniform(0, 2 * math.pi, 50)
    nhat = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], axis=1)
    Fp, Fc = oracle.antenna_patterns(np.array([[1.0, 0, 0]]), np.array([[0, 1.0, 0]]), nhat)
    np.testing.assert_allclose(Fp[:, 0], 0.5 * (1 + np.cos(th) ** 2) * np.cos(2 * ph), atol=1e-12)
    np.testing.assert_allclose(Fc[:, 0], np.cos(th) * np.sin(2 * ph), atol=1e-12)


def test_polarisation_angle_rotates_patterns_by_twice_psi():
    # App. A: (F+, Fx) at angle psi are (G+, Gx) rotated by 2 psi, so F+^2 + Fx^2 is
    # independent of psi; swapping the arms flips the sign of the detector tensor.
    det = synth.detectors(0, 2)
    nhat = oracle.healpix_centres(4)
    Gp, Gc = oracle.antenna_patterns(det.arm_x, det.arm_y, nhat)
    psi = 0.37
    Fp, Fc = oracle.antenna_patterns(det.arm_x, det.arm_y, nhat, psi=psi)
    c, s = math.cos(2 * psi), math.sin(2 * psi)
    np.testing.assert_allclose(Fp, c * Gp + s * Gc, atol=1e-12)
    np.testing.assert_allclose(Fc, -s * Gp + c * Gc, atol=1e-12)
    np.testing.assert_allclose(Fp ** 2 + Fc ** 2, Gp ** 2 + Gc ** 2, atol=1e-12)
    Sp, Sc = oracle.antenna_patterns(det.arm_y, det.arm_x, nhat)
    np.testing.assert_allclose(Sp, -Gp, atol=1e-12)
    np.testing.assert_allclose(Sc, -Gc, atol=1e-12)


def test_arrival_delays_closed_form():
    R = synth.EARTH_RADIUS_M
    pos = np.array([[0, 0, R]])
    nhat = np.array([[0, 0, 1.0], [0, 0, -1.0], [1.0, 0, 0]])
    d = oracle.arrival_delays(pos, nhat, 2048.0)
    v = 2048.0 * R / 299792458.0  # 43.52 samples
    assert d[0, 0] == -round(v) == -44 and d[1, 0] == 44 and d[2, 0] == 0


# ---------------------------------------------------------------------------------------------
# Coherent statistic (Sec. II.C.1 Eq. (llr_form), Eq. (null_def), App. A)


def _random_g(g, P, n_det):
    return g.standard_normal((P, n_det, 2))


def test_two_detectors_statistic_is_total_power_and_null_vanishes():
    g = _rng(5)
    P, n, H = 7, 50, 3
    G = _random_g(g, P, 2)
    delays = g.integers(-H, H + 1, (P, 2)).astype(np.int32)
    z = g.standard_normal((2, 2, n + 2 * H)) + 1j * g.standard_normal((2, 2, n + 2 * H))
    ms, am, nl, sm = oracle.coherent(z, G, delays, H, n, skymap=True)
    for p in range(P):
        w = np.stack([z[:, I, H + np.arange(n) + delays[p, I]] for I in range(2)], axis=2)
        np.testing.assert_allclose(sm[:, :, p], np.sum(np.abs(w) ** 2, axis=2), rtol=1e-12)
    np.testing.assert_allclose(nl, 0.0, atol=1e-10)


def test_projector_form_equals_svd_form_and_explicit_null():
    g = _rng(6)
    P, n, H, n_det = 9, 40, 2, 4
    G = _random_g(g, P, n_det)
    delays = g.integers(-H, H + 1, (P, n_det)).astype(np.int32)
    z = g.standard_normal((1, n_det, n + 2 * H)) + 1j * g.standard_normal((1, n_det, n + 2 * H))
    ms, am, nl, sm = oracle.coherent(z, G, delays, H, n, skymap=True)
    for p in range(P):
        U, s, Vt = np.linalg.svd(G[p])  # Eq. (svd): G = U Lambda V^T, U is n_det x n_det
        w = np.stack([z[0, I, H + np.arange(n) + delays[p, I]] for I in range(n_det)], axis=1)
        sig = np.sum(np.abs(w @ U[:, :2]) ** 2, axis=1)      # |I U^T z|^2
        null = np.sum(np.abs(w @ U[:, 2:]) ** 2, axis=1)     # |I^dagger U^T z|^2 (App. A)
        np.testing.assert_allclose(sm[0, :, p], sig, rtol=1e-11)
        sel = am[0] == p
        np.testing.assert_allclose(nl[0, sel], null[sel], rtol=1e-9, atol=1e-12)
    np.testing.assert_array_equal(ms[0], sm[0].max(axis=1))
    np.testing.assert_array_equal(am[0], sm[0].argmax(axis=1))


def test_statistic_equals_twice_brute_force_maximised_llr():
    g = _rng(7)
    n_det = 3
    G = _random_g(g, 1, n_det)
    z = g.standard_normal((1, n_det, 4)) + 1j * g.standard_normal((1, n_det, 4))
    delays = np.zeros((1, n_det), dtype=np.int32)
    ms, _, _, _ = oracle.coherent(z, G, delays, 0, 4)
    for k in range(4):
        llr = oracle.llr_bruteforce(z[0, :, k], G[0])
        assert abs(ms[0, k] - 2.0 * llr) < 1e-7 * max(1.0, ms[0, k])


def test_noiseless_injection_recovers_pixel_total_power_and_zero_null():
    # Sec. II.C.1: in the true direction the projection keeps all the signal power and the
    # null stream holds none.  z_I = (G_sigma(p*) (A_c + i A_s))_I f(k - Delta_I(p*)).
    det = synth.detectors(1, 3)
    sigma = np.array([0.7, 1.3, 1.9])
    nhat, G, delays = oracle.sky_geometry(det, sigma, 4, 2048.0)
    H = int(np.abs(delays).max())
    g = _rng(8)
    pstar, n, k0 = 77, 64, 30
    j = np.arange(-4 * H, n + 4 * H)
    f = np.exp(-0.5 * ((j - k0) / 0.6) ** 2) * np.exp(0.9j * j)   # narrow pulse at k0
    A = g.standard_normal(2) + 1j * g.standard_normal(2)           # A_c + i A_s
    amp = G[pstar] @ A
    z = np.zeros((1, 3, n + 2 * H), dtype=np.complex128)
    for I in range(3):
        idx = np.arange(n + 2 * H) - H - delays[pstar, I]            # time read by sample index
        z[0, I] = amp[I] * f[idx + 4 * H]
    ms, am, nl, sm = oracle.coherent(z, G, delays, H, n, skymap=True)
    k = np.arange(n)
    w = np.stack([z[0, I, H + k + delays[pstar, I]] for I in range(3)], axis=1)
    tot = np.sum(np.abs(w) ** 2, axis=1)
    np.testing.assert_allclose(sm[0, :, pstar], tot, rtol=1e-10, atol=1e-300)
    assert am[0, k0] == pstar
    assert abs(ms[0, k0] - tot[k0]) < 1e-10 * tot[k0] and abs(nl[0, k0]) < 1e-10 * tot[k0]


def test_gaussian_noise_moments_match_chi2_dof():
    # App. A: rho_C^2 is chi^2 with 4 dof and the null chi^2 with 2 N_d - 4 dof when
    # E|z_I|^2 = 2 (Sec. III.C: mean null^2 is 2 N_d - 4).
    g = _rng(9)
    n_det, P, n = 3, 5, 40000
    G = _random_g(g, P, n_det)
    delays = np.zeros((P, n_det), dtype=np.int32)
    z = g.standard_normal((1, n_det, n)) + 1j * g.standard_normal((1, n_det, n))
    _, _, _, sm = oracle.coherent(z, G, delays, 0, n, skymap=True)
    tot = np.sum(np.abs(z[0]) ** 2, axis=0)
    for p in range(P):
        assert abs(sm[0, :, p].mean() - 4.0) < 0.1
        assert abs((tot - sm[0, :, p]).mean() - (2 * n_det - 4)) < 0.06


def test_argmax_ties_take_lowest_pixel():
    G = np.tile(np.array([[1.0, 0.0], [0.0, 1.0], [1.0, 1.0]])[None], (4, 1, 1))
    delays = np.zeros((4, 3), dtype=np.int32)
    z = np.ones((1, 3, 5), dtype=np.complex128)
    _, am, _, _ = oracle.coherent(z, G, delays, 0, 5)
    assert np.all(am == 0)


def test_printed_event_table_null_identity():
    # Sec. III.C, Table event_tab: the network SNR is the quadrature sum of the individual
    # SNRs.  With |w_I| = rho_I the oracle's rho_C^2 + null^2 must equal sum rho_I^2, and
    # both parts are bounded by it, whatever the sky geometry.
    det = synth.detectors(1, 3)
    nhat, G, delays = oracle.sky_geometry(det, np.ones(3), 4, 2048.0)
    g = _rng(10)
    for name, rl, rh, rv, net, null in golden_rows("event_table.txt"):
        rho = np.array([float(rl), float(rh), float(rv)])
        w = rho * np.exp(1j * g.uniform(0, 2 * np.pi, 3))
        z = w[None, :, None].astype(np.complex128)
        ms, am, nl, _ = oracle.coherent(z, G, np.zeros_like(delays), 0, 1)
        tot = ms[0, 0] + nl[0, 0]
        assert abs(tot - np.sum(rho ** 2)) < 1e-9 * tot
        assert abs(math.sqrt(tot) - float(net)) <= 0.05 + 0.05 * 3 + 1e-9
        assert 0 <= nl[0, 0] <= tot and ms[0, 0] <= tot


# ---------------------------------------------------------------------------------------------
# Impulse response, overlap loss and adjoint


def _tiny_impulse_bank(seed=11):
    g = _rng(seed)
    bank = synth.random_bank(g, [3, 2], d_max=20)
    s0 = (g.standard_normal(5) + 1j * g.standard_normal(5)) * 0.1
    h = g.standard_normal((2, 60)) + 1j * g.standard_normal((2, 60))
    return bank, s0, h


def test_impulse_forward_matches_filter_bank_and_closed_form():
    bank, s0, h = _tiny_impulse_bank()
    n = 60
    u = oracle.impulse_forward(bank.offsets, bank.a1, bank.b0, bank.delay, s0, n)
    x = np.zeros((1, n))
    x[0, 0] = 1.0
    z, _, _ = oracle.filter_bank(x, bank.offsets, bank.a1, bank.b0, bank.delay, state=s0[None, :])
    np.testing.assert_allclose(u, z[:, 0], rtol=1e-12, atol=1e-14)
    k = np.arange(n)
    a = bank.a1.astype(np.complex128)
    b = bank.b0.astype(np.complex128)
    ref = np.zeros((2, n), dtype=np.complex128)
    for t in range(2):
        for l in range(bank.offsets[t], bank.offsets[t + 1]):
            ref[t] += s0[l] * a[l] ** (k + 1) + np.where(k >= bank.delay[l], b[l] * a[l] ** np.maximum(k - bank.delay[l], 0), 0)
    np.testing.assert_allclose(u, ref, rtol=1e-11, atol=1e-13)


def test_overlap_loss_gradient_matches_finite_differences():
    g = _rng(12)
    h = g.standard_normal((1, 30)) + 1j * g.standard_normal((1, 30))
    u = g.standard_normal((1, 30)) + 1j * g.standard_normal((1, 30))
    L, gr = oracle.overlap_loss(h, u)
    eps = 1e-6
    for k in (0, 7, 29):
        for unit in (1.0, 1j):
            up = u.copy(); up[0, k] += eps * unit
            um = u.copy(); um[0, k] -= eps * unit
            fd = (oracle.overlap_loss(h, up)[0][0] - oracle.overlap_loss(h, um)[0][0]) / (2 * eps)
            an = gr[0, k].real if unit == 1.0 else gr[0, k].imag
            assert abs(fd - an) < 1e-8
    assert 0.0 <= L[0] <= 1.0
    # a perfect match up to a constant phase has zero loss
    L0, _ = oracle.overlap_loss(h, 2.5 * np.exp(0.7j) * h)
    assert abs(L0[0]) < 1e-12


def test_adjoint_matches_fp64_finite_differences():
    bank, s0, h = _tiny_impulse_bank(13)
    n = 60
    a1 = bank.a1.astype(np.complex128)
    b0 = bank.b0.astype(np.complex128)

    def loss(a, b, s):
        u = oracle.impulse_forward(bank.offsets, a, b, bank.delay, s, n)
        return oracle.overlap_loss(h, u)[0].sum()

    u = oracle.impulse_forward(bank.offsets, a1, b0, bank.delay, s0, n)
    _, gu = oracle.overlap_loss(h, u)
    ga, gb, gs = oracle.impulse_backward(bank.offsets, a1, b0, bank.delay, s0, gu)
    eps = 1e-6
    for which, base, grad in (("a", a1, ga), ("b", b0, gb), ("s", s0, gs)):
        for l in range(5):
            for unit, part in ((1.0, np.real), (1j, np.imag)):
                vp = base.copy(); vp[l] += eps * unit
                vm = base.copy(); vm[l] -= eps * unit
                args_p = {"a": a1, "b": b0, "s": s0}
                args_m = dict(args_p)
                args_p[which] = vp
                args_m[which] = vm
                fd = (loss(args_p["a"], args_p["b"], args_p["s"]) - loss(args_m["a"], args_m["b"], args_m["s"])) / (2 * eps)
                an = part(grad[l])
                assert abs(fd - an) < 1e-6 * max(1.0, abs(fd)), (which, l, fd, an)


# ---------------------------------------------------------------------------------------------
# Multirate split (not in the paper): identities, and the library routines each step reduces to


def test_fir_has_unit_dc_gain_and_attenuates_above_cutoff():
    for M in (4, 16):
        h = oracle.fir_taps(M)
        assert h.size == 32 and abs(h.sum() - 1.0) < 1e-14
        f = np.linspace(0, 0.5, 2001)
        H = np.abs(np.exp(-2j * np.pi * np.outer(f, np.arange(32))) @ h)
        fc = 0.8 * 0.5 / M
        assert np.all(H[f <= 0.5 * fc] > 0.9)        # passband
        # stopband beyond the Hann main-lobe half-width 2/ntaps past the cutoff
        assert np.all(H[f >= fc + 2.0 / 32] < 0.01)


def test_decimate_identity_dc_and_chunking():
    g = _rng(14)
    x = g.standard_normal((2, 512))
    xb, _ = oracle.decimate(x, 1)
    np.testing.assert_array_equal(xb, x)
    dc, _ = oracle.decimate(np.full((1, 512), 3.0), 16)
    np.testing.assert_allclose(dc[0, 2:], 3.0, rtol=1e-13)
    one, _ = oracle.decimate(x, 4)
    hist, parts = None, []
    for s in range(0, 512, 128):
        p, hist = oracle.decimate(x[:, s:s + 128], 4, history=hist)
        parts.append(p)
    np.testing.assert_allclose(np.concatenate(parts, axis=1), one, rtol=1e-13, atol=1e-13)


def test_linear_upsample_reproduces_ramp_with_one_sample_lag():
    M = 4
    zb = np.arange(10, dtype=np.float64)[None, :] * (1 + 0.5j)
    z, last = oracle.upsample_linear(zb, M)
    k = np.arange(40)
    np.testing.assert_allclose(z[0, M:], (k[M:] / M - 1) * (1 + 0.5j), rtol=1e-14)
    assert last[0] == zb[0, -1]


def _hann_half_sample(n):
    # the window sampled at i + 1/2: the odd samples of the periodic Hann window of length 2n
    import scipy.signal as ss
    return ss.windows.hann(2 * n, sym=False)[1::2]


def test_fir_taps_equal_scipy_sinc_times_half_sample_hann():
    import scipy.signal as ss
    for M in (2, 4, 16):
        # firwin with a boxcar window and no scaling is the ideal low-pass 2 fc sinc(2 fc (i - c))
        box = ss.firwin(32, 0.8 / M, window="boxcar", scale=False)
        ref = box * _hann_half_sample(32)
        np.testing.assert_allclose(oracle.fir_taps(M), ref / ref.sum(), rtol=0, atol=1e-15)


def test_decimate_equals_scipy_upfirdn():
    import scipy.signal as ss
    g = _rng(41)
    x = g.standard_normal((2, 768))
    for M, taps in ((4, None), (16, None), (3, g.standard_normal(7))):
        h = oracle.fir_taps(M) if taps is None else taps
        y, _ = oracle.decimate(x, M, taps)
        ref = ss.upfirdn(h, x, up=1, down=M, axis=-1)[:, : 768 // M]
        np.testing.assert_allclose(y, ref, rtol=0, atol=1e-13)


def test_linear_upsample_equals_numpy_interp():
    g = _rng(42)
    for M in (2, 4, 16):
        zb = g.standard_normal((3, 12)) + 1j * g.standard_normal((3, 12))
        prev = g.standard_normal(3) + 1j * g.standard_normal(3)
        z, last = oracle.upsample_linear(zb, M, prev=prev)
        k = np.arange(12 * M)
        for r in range(3):
            # output k sits at low-rate position k / M - 1 (one low-rate sample of lag), prev at -1
            fp = np.concatenate([[prev[r]], zb[r]])
            xp = np.arange(-1, 12)
            ref = np.interp(k / M - 1, xp, fp.real) + 1j * np.interp(k / M - 1, xp, fp.imag)
            np.testing.assert_allclose(z[r], ref, rtol=0, atol=1e-14)
        np.testing.assert_array_equal(last, zb[:, -1])


def test_multirate_bank_equals_upfirdn_lfilter_interp_per_filter():
    # z_t = sum over the template's filters of: decimate (upfirdn), one-pole IIR on the delayed
    # low-rate input (lfilter), linear upsampling (interp); the bank is linear in its filters
    import scipy.signal as ss
    g = _rng(43)
    n_det, n, factors = 2, 1024, (1, 4, 16)
    x = g.standard_normal((n_det, n))
    offsets = np.array([0, 5, 12])
    F = offsets[-1]
    a1 = g.uniform(0.6, 0.98, F) * np.exp(1j * g.uniform(-2.5, 2.5, F))
    b0 = (g.standard_normal(F) + 1j * g.standard_normal(F)) / np.sqrt(2 * F)
    band = g.integers(0, 3, F)
    delay = np.array([g.integers(0, 40 if factors[b] == 1 else 10) for b in band])
    z = oracle.multirate_bank(x, offsets, a1, b0, delay, band, factors)
    ref = np.zeros((2, n_det, n), dtype=np.complex128)
    for t in range(2):
        for l in range(offsets[t], offsets[t + 1]):
            M = factors[band[l]]
            for I in range(n_det):
                xb = x[I] if M == 1 else ss.upfirdn(oracle.fir_taps(M), x[I], down=M)[: n // M]
                xd = np.concatenate([np.zeros(delay[l]), xb])[: xb.size]
                yb = ss.lfilter([b0[l]], [1.0, -a1[l]], xd.astype(np.complex128))
                if M == 1:
                    ref[t, I] += yb
                else:
                    k = np.arange(n)
                    fp = np.concatenate([[0.0], yb])
                    xp = np.arange(-1, yb.size)
                    ref[t, I] += np.interp(k / M - 1, xp, fp.real) + 1j * np.interp(k / M - 1, xp, fp.imag)
    np.testing.assert_allclose(z, ref, rtol=0, atol=1e-11)


# ---------------------------------------------------------------------------------------------
# Signal-consistency statistic (Sec. II.C.2)


def _random_template(seed, F=6, d_max=40):
    g = np.random.default_rng(seed)
    a1 = (g.uniform(0.7, 0.95, F) * np.exp(1j * g.uniform(0, 2 * np.pi, F))).astype(np.complex64)
    b0 = ((g.standard_normal(F) + 1j * g.standard_normal(F)) / np.sqrt(2 * F)).astype(np.complex64)
    d = g.integers(0, d_max, F).astype(np.int32)
    return a1, b0, d


def _response(a1, b0, d, nr):
    F = a1.size
    return oracle.impulse_forward(np.array([0, F], np.int64), a1, b0, d, np.zeros(F, np.complex64), nr)[0]


def test_autocorr_of_one_filter_is_a_power_of_its_pole():
    """u[k] = b a^k (k >= 0): R[j] = |b|^2 a^j sum_k |a|^2k, so A[j] = a^j and A[-j] = conj(a)^j."""
    a = 0.9 * np.exp(0.7j)
    nr, Nj = 4000, 12
    u = (0.3 - 0.2j) * a ** np.arange(nr)
    A = oracle.autocorr(u[None, :], Nj)[0]
    j = np.arange(Nj + 1)
    np.testing.assert_allclose(A[Nj:], a ** j, rtol=0, atol=1e-12)
    np.testing.assert_allclose(A[:Nj + 1][::-1], np.conj(a) ** j, rtol=0, atol=1e-12)


def test_xi2_vanishes_for_a_window_shaped_like_the_autocorrelation():
    """z[k0 + j] = c A[j] for |j| <= Nj is exactly what the statistic expects: xi^2[k0] = 0,
    while the same window mirrored in time (A[-j]) or conjugated does not vanish."""
    Nj = 9
    a1, b0, d = _random_template(1)
    A = oracle.autocorr(_response(a1, b0, d, 300)[None, :], Nj)[0]
    g = np.random.default_rng(2)
    z = (g.standard_normal(4 * Nj + 1) + 1j * g.standard_normal(4 * Nj + 1))
    k0 = 2 * Nj
    c = 3.0 - 1.5j
    for mod, zero in ((lambda x: x, True), (lambda x: x[::-1], False), (np.conj, False)):
        zz = z.copy()
        zz[k0 - Nj: k0 + Nj + 1] = c * mod(A)
        x = oracle.xi2(zz[None, None, :], A[None, :], Nj, 2 * Nj + 1)[0, 0, Nj]
        assert (x < 1e-24) == zero, x


def test_xi2_of_a_matched_signal_through_the_filter_bank_vanishes():
    """A signal s with s[k0 - m] = conj(u[m]) filtered by the template's own filters gives
    z[k0 + j] = R[j] = z[k0] A[j] exactly (finite sums over the same range): xi^2[k0] = 0."""
    Nj, nr = 10, 400
    a1, b0, d = _random_template(3)
    u = _response(a1, b0, d, nr)
    A = oracle.autocorr(u[None, :], Nj)[0]
    k0 = nr + 50
    x = np.zeros((1, k0 + Nj + 60), np.complex128)
    x[0, k0 - np.arange(nr)] = np.conj(u)
    z, _, _ = oracle.filter_bank(x, np.array([0, a1.size], np.int64), a1, b0, d)
    zr = z[0, 0]
    np.testing.assert_allclose(zr[k0 + np.arange(-Nj, Nj + 1)], zr[k0] * A, rtol=0, atol=1e-12 * abs(zr[k0]))
    xi = oracle.xi2(zr[None, None, k0 - 2 * Nj: k0 + 2 * Nj + 1], A[None, :], Nj, 2 * Nj + 1)[0, 0, Nj]
    assert xi < 1e-20


def test_xi2_has_mean_one_in_white_noise():
    """z = u * x with x unit white noise and sum |u|^2 = 2: E|z[k+j] - z[k] A[j]|^2 = 2 - 2|A[j]|^2
    term by term, so the statistic is a reduced chi-square of mean 1."""
    Nj, nr = 30, 600
    a1, b0, d = _random_template(4, F=8, d_max=200)
    u = _response(a1, b0, d, nr)
    s = np.sqrt(2.0 / np.sum(np.abs(u) ** 2))
    b0 = (b0 * s).astype(np.complex64)
    u = _response(a1, b0, d, nr)
    A = oracle.autocorr(u[None, :], Nj)[0]
    x = synth.white_noise(0, 1, 120000, sub=99).astype(np.float64)
    z, _, _ = oracle.filter_bank(x, np.array([0, a1.size], np.int64), a1, b0, d)
    zs = z[0, 0, 2 * nr:]  # past the start-up transient
    n = zs.size - 2 * Nj
    xi = oracle.xi2(zs[None, None, :], A[None, :], Nj, n)[0, 0]
    assert abs(xi.mean() - 1.0) < 0.03, xi.mean()


def test_network_average_reads_each_detector_at_its_arrival_time():
    """xi_C^2 at (t, k) is the mean over detectors of xi_I^2 at k + Delta_I(argmax)."""
    T, n_det, n, H = 2, 3, 7, 4
    xi = np.arange(T * n_det * (n + 2 * H), dtype=np.float64).reshape(T, n_det, n + 2 * H)
    delays = np.array([[0, 0, 0], [-4, 1, 4], [3, -2, 0]])
    argmax = np.array([[0, 1, 2, 1, 0, 2, 1], [2, 2, 1, 0, 0, 1, 2]])
    out = oracle.xi2_network(xi, delays, argmax, H)
    for t in range(T):
        for k in range(n):
            p = argmax[t, k]
            expect = np.mean([xi[t, I, H + k + delays[p, I]] for I in range(n_det)])
            assert out[t, k] == expect


def test_network_xi2_of_linear_per_detector_values():
    """With xi_I^2 at sample x equal to I + x / 1000, the network value at sample k and pixel p
    is the mean over detectors of I + (k + Delta_I(p)) / 1000: a closed form that fails for a
    wrong halo offset, a wrong delay sign or detector, or a wrong divisor."""
    g = _rng(33)
    T, n_det, n, H, P = 2, 3, 50, 7, 11
    delays = g.integers(-H, H + 1, (P, n_det))
    x = np.arange(n + 2 * H) - H
    xi = np.stack([np.stack([I + x / 1000.0 for I in range(n_det)]) for _ in range(T)])
    am = g.integers(0, P, (T, n))
    got = oracle.xi2_network(xi, delays, am, H)
    k = np.arange(n)
    want = np.mean([[I + (k + delays[am[t], I]) / 1000.0 for I in range(n_det)] for t in range(T)], axis=1)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


# ---------------------------------------------------------------------------------------------
# Candidate selection and the candidate-driven scan (Sec. II.C.1), time-shift background
# (Sec. II.C.3)


def test_candidate_selection_on_constructed_peaks():
    """Largest SNR over the bank per sample, kept when over 4; one candidate per template per
    second (the largest, the earliest among equals); the lowest template among equal maxima."""
    T, nd, n, sec = 4, 2, 4096, 2048
    z = np.zeros((T, nd, n), np.complex128)
    put = lambda t, I, k, v: z.__setitem__((t, I, k), v * np.exp(0.3j * (k % 7)))
    put(1, 0, 100, 5.0); put(1, 0, 300, 7.0)         # same template, same second: only 300
    put(2, 0, 497, 4.0)                               # exactly 4 (phase 0): not over the threshold
    put(3, 0, 2100, 6.0)                              # second 1
    put(0, 0, 700, 5.0); put(3, 0, 700, 5.5)          # template 3 holds the maximum at 700
    put(0, 0, 900, 6.0); put(2, 0, 900, 6.0)          # equal maxima: template 0
    put(2, 0, 1000, 5.0); put(2, 0, 1203, 5.0)        # equal values (same phase) in one second: the earlier
    put(1, 1, 2047, 4.5); put(1, 1, 2048, 4.6)        # either side of the second boundary
    got = oracle.select_candidates(z, 0, n, 4.0, sec)
    expect = [(0, 0, 900, 6.0), (0, 1, 300, 7.0), (0, 2, 1000, 5.0), (0, 3, 700, 5.5), (0, 3, 2100, 6.0),
              (1, 1, 2047, 4.5), (1, 1, 2048, 4.6)]
    assert [(a, b, c) for a, b, c, _ in got] == [(a, b, c) for a, b, c, _ in expect]
    np.testing.assert_allclose([v for *_, v in got], [v * v for *_, v in expect], rtol=1e-6)


def test_candidate_threshold_is_decided_in_fp32():
    """|z| just above 4 in FP64 but 4 after rounding to FP32 is not a candidate; the next FP32
    value above 4 is (the decision is taken on FP32 |z|^2, as on the GPU)."""
    z = np.zeros((1, 1, 8), np.complex128)
    z[0, 0, 2] = 4.0 + 1e-9
    z[0, 0, 5] = float(np.nextafter(np.float32(4.0), np.float32(5.0)))
    got = oracle.select_candidates(z, 0, 8, 4.0, 8)
    assert [(a, b, c) for a, b, c, _ in got] == [(0, 0, 5)]


def test_point_scan_with_two_detectors_is_the_power_at_the_implied_times():
    """N_d = 2 (rank-2 G): the statistic at every pixel is |w_0|^2 + |w_1|^2, w read at the
    reference detector's own sample and the other detector at e + Delta_1(p) - Delta_r(p)."""
    g = _rng(21)
    P, n, H = 11, 80, 4
    G = _random_g(g, P, 2)
    delays = g.integers(-H, H + 1, (P, 2)).astype(np.int32)
    z = g.standard_normal((2, 2, n)) + 1j * g.standard_normal((2, 2, n))
    pts = np.array([[0, 0, 20], [1, 1, 40], [1, 0, 2 * H]], np.int64)
    ms, am, nl = oracle.coherent_points(z, G, delays, pts, np.zeros((3, 2), np.int64))
    for i, (t, r, e) in enumerate(pts):
        power = [sum(abs(z[t, I, e + delays[p, I] - delays[p, r]]) ** 2 for I in range(2)) for p in range(P)]
        assert am[i] == int(np.argmax(power))
        np.testing.assert_allclose(ms[i], max(power), rtol=1e-12)
        assert abs(nl[i]) < 1e-10 * ms[i]


def test_point_scan_recovers_an_injection_from_any_reference_detector():
    """A noiseless source in direction p*: read from any detector's arrival sample, the scan
    keeps the whole power at p* with a vanishing null (Sec. II.C.1)."""
    det = synth.detectors(1, 3)
    sigma = np.array([0.7, 1.3, 1.9])
    nhat, G, delays = oracle.sky_geometry(det, sigma, 4, 2048.0)
    H = int(np.abs(delays).max())
    g = _rng(22)
    pstar, n, k0 = 101, 200, 100
    A = g.standard_normal(2) + 1j * g.standard_normal(2)
    amp = G[pstar] @ A
    z = np.zeros((1, 3, n), np.complex128)
    for I in range(3):
        z[0, I, k0 + delays[pstar, I]] = amp[I]            # geocentric sample k0 arrives at k0 + Delta_I
    tot = float(np.sum(np.abs(amp) ** 2))
    for r in range(3):
        pts = np.array([[0, r, k0 + delays[pstar, r]]], np.int64)
        ms, am, nl = oracle.coherent_points(z, G, delays, pts, np.zeros((1, 3), np.int64))
        assert am[0] == pstar and abs(ms[0] - tot) < 1e-10 * tot and abs(nl[0]) < 1e-10 * tot


def test_background_shift_pairs_the_reference_with_earlier_companion_data():
    """A companion detector holding the signal s c step samples earlier than coincidence is
    realigned by time shift s and by no other (Sec. II.C.3: shifts of at least 0.1 s)."""
    det = synth.detectors(1, 3)
    sigma = np.array([1.0, 1.0, 1.0])
    nhat, G, delays = oracle.sky_geometry(det, sigma, 2, 2048.0)
    H = int(np.abs(delays).max())
    g = _rng(23)
    pstar, step, sstar, r = 20, 205, 3, 1
    n = 2 * H + 3 * 100 * step
    k0 = n - 2 * H - 1
    A = g.standard_normal(2) + 1j * g.standard_normal(2)
    amp = G[pstar] @ A
    sh = oracle.background_shifts(r, 3, sstar, step)
    z = 1e-6 * (g.standard_normal((1, 3, n)) + 1j * g.standard_normal((1, 3, n)))
    for I in range(3):
        z[0, I, k0 + delays[pstar, I] + sh[I]] += amp[I]
    e = k0 + delays[pstar, r]
    pts = np.array([[0, r, e]] * 6, np.int64)
    shifts = np.stack([oracle.background_shifts(r, 3, s, step) for s in range(6)])
    ms, am, nl = oracle.coherent_points(z, G, delays, pts, shifts)
    tot = float(np.sum(np.abs(amp) ** 2))
    assert int(np.argmax(ms)) == sstar and am[sstar] == pstar and abs(ms[sstar] - tot) < 1e-6 * tot
    assert all(ms[s] < 0.9 * tot for s in range(6) if s != sstar)


# ---------------------------------------------------------------------------------------------
# Front end (Sec. II.A): FIR down-sampling and whitening, Eq. (whiten), in the time domain


def test_whitening_kernel_of_a_flat_psd_is_a_scaled_delta():
    """White noise of variance sigma^2 has the one-sided PSD 2 sigma^2 / f_s: its whitening
    filter is 1 / sigma at the centre tap and zero elsewhere."""
    fs, sigma, N = 2048.0, 1.7, 256
    psd = np.full(N // 2 + 1, 2.0 * sigma ** 2 / fs)
    w = oracle.whitening_kernel(psd, fs, 101)
    expect = np.zeros(101)
    expect[50] = 1.0 / sigma
    np.testing.assert_allclose(w, expect, rtol=0, atol=1e-13)


def test_whitening_kernel_is_eq_whiten_in_the_time_domain():
    """Eq. (whiten) on a periodic signal: division by sqrt(S_n) in the frequency domain (numpy
    FFT, with the unit-variance factor sqrt(2 / f_s)) equals circular convolution with the
    unwindowed kernel (the PSD of an AR(1) process is smooth, so the kernel vanishes well before
    half the period)."""
    g = _rng(30)
    fs, N, phi, s = 2048.0, 512, 0.6, 1.3
    f = np.arange(N // 2 + 1) * fs / N
    psd = (2.0 * s ** 2 / fs) / np.abs(1.0 - phi * np.exp(-2j * np.pi * f / fs)) ** 2
    w = oracle.whitening_kernel(psd, fs, N - 1, window=False)
    K = N // 2 - 1
    x = g.standard_normal(N)
    y_fd = np.fft.irfft(np.fft.rfft(x) * np.sqrt(2.0 / (fs * psd)), n=N)
    y_td = np.array([sum(w[m + K] * x[(k - m) % N] for m in range(-K, K + 1)) for k in range(N)])
    np.testing.assert_allclose(y_td, y_fd, rtol=0, atol=1e-10)


def test_whitened_ar1_noise_is_white_with_unit_variance():
    """x[k] = phi x[k-1] + s e[k] has S_n(f) = (2 s^2 / f_s) / |1 - phi e^{-2 pi i f / f_s}|^2;
    the whitening FIR turns it into unit-variance noise with vanishing autocorrelation."""
    g = _rng(31)
    fs, phi, s, n = 2048.0, 0.9, 2.5, 1 << 16
    e = g.standard_normal(n)
    x = np.zeros(n)
    for k in range(1, n):
        x[k] = phi * x[k - 1] + s * e[k]
    N = 4096
    f = np.arange(N // 2 + 1) * fs / N
    psd = (2.0 * s ** 2 / fs) / np.abs(1.0 - phi * np.exp(-2j * np.pi * f / fs)) ** 2
    w = oracle.whitening_kernel(psd, fs, 1025)
    y, _ = oracle.fir(x, w)
    y = y[2048:]
    assert abs(y.var() - 1.0) < 0.03, y.var()
    for lag in range(1, 6):
        r = float(np.mean(y[lag:] * y[:-lag]) / y.var())
        assert abs(r) < 0.02, (lag, r)
    # without whitening the lag-1 correlation is phi
    assert abs(float(np.mean(x[2049:] * x[2048:-1]) / x[2048:].var()) - phi) < 0.02


def test_decimation_low_pass_dc_passband_and_stopband():
    """192-tap low-pass for 16384 -> 2048 Hz: a constant passes with gain 1 once the filter is
    full, a 100 Hz tone keeps its amplitude, a 3 kHz tone (above the output Nyquist frequency)
    is suppressed before it aliases."""
    h = oracle.lowpass_taps(192, 8, 0.9)
    fs, n = 16384.0, 16384
    k = np.arange(n)
    y, _ = oracle.decimate(np.ones((1, n)), 8, h)
    assert np.max(np.abs(y[0, 24:] - 1.0)) < 1e-12
    for f0, lo, hi in ((100.0, 0.995, 1.005), (3000.0, 0.0, 3e-3)):
        y, _ = oracle.decimate(np.cos(2 * np.pi * f0 * k / fs)[None], 8, h)
        amp = math.sqrt(2.0 * float(np.mean(y[0, 64:] ** 2)))
        assert lo <= amp <= hi, (f0, amp)


def test_frontend_streams_identically_across_chunks():
    """Decimation and whitening with histories carried between segments of any length (a
    multiple of the decimation factor) reproduce the whole-stream result."""
    g = _rng(32)
    x = g.standard_normal((2, 8 * 600))
    h = oracle.lowpass_taps(48, 8, 0.9)
    fs, N = 2048.0, 128
    f = np.arange(N // 2 + 1) * fs / N
    psds = [(2.0 / fs) / np.abs(1.0 - p * np.exp(-2j * np.pi * f / fs)) ** 2 for p in (0.3, -0.5)]
    w = np.stack([oracle.whitening_kernel(p, fs, 41) for p in psds])
    y_all, _, _ = oracle.frontend(x, h, 8, w)
    parts, h16, h2, k0 = [], None, None, 0
    for c in (100, 37, 263, 200):
        y, h16, h2 = oracle.frontend(x[:, k0: k0 + 8 * c], h, 8, w, h16, h2)
        parts.append(y)
        k0 += 8 * c
    np.testing.assert_allclose(np.concatenate(parts, axis=1), y_all, rtol=0, atol=1e-12)
    # the decimated stream is x low-passed and subsampled: M = 8 with a one-tap filter is x[8 j]
    y1, _ = oracle.decimate(x, 8, np.array([1.0]))
    np.testing.assert_array_equal(y1, x[:, ::8])
