"""GPU signal-consistency statistic (Sec. II.C.2) against the FP64 oracle: template
autocorrelation, xi_I^2 per sample, and the network average at the coherent argmax."""
import numpy as np
import pytest

import oracle
import synth
from helpers import cuda_ok

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs CUDA")]

XI_TOL = 1e-4  # relative to max(xi^2, 1): FP32 sums of up to 2049 squared differences


def _cuda(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _responses(T, F, nr, seed):
    g = np.random.default_rng(seed)
    a1 = (g.uniform(0.8, 0.98, (T, F)) * np.exp(1j * g.uniform(0, 2 * np.pi, (T, F)))).astype(np.complex64)
    b0 = ((g.standard_normal((T, F)) + 1j * g.standard_normal((T, F))) / np.sqrt(2 * F)).astype(np.complex64)
    d = g.integers(0, nr // 3, (T, F)).astype(np.int32)
    off = np.arange(T + 1, dtype=np.int64) * F
    u = oracle.impulse_forward(off, a1.ravel(), b0.ravel(), d.ravel(), np.zeros(T * F, np.complex64), nr)
    return u.astype(np.complex64)


@pytest.mark.parametrize("Nj", [0, 5, 175])
def test_autocorr_matches_oracle(Nj):
    import paper_2011_06787_b300 as sp
    u = _responses(5, 40, 3000, seed=Nj)
    A = sp.autocorr(_cuda(u), Nj).cpu().numpy()
    A_or = oracle.autocorr(u, Nj)
    assert np.max(np.abs(A - A_or)) < 2e-5
    np.testing.assert_allclose(A[:, Nj], 1.0, atol=1e-6)


@pytest.mark.parametrize("Nj,n", [(3, 700), (4, 1024), (175, 2500), (60, 3000), (5, 1), (175, 1), (2, 9)])
def test_xi2_matches_oracle(Nj, n):
    """Ragged last tiles (n not a multiple of 1024), single and few output samples, and tap
    counts below, at and above one unrolled group of 8."""
    import paper_2011_06787_b300 as sp
    T, nd = 3, 3
    A = oracle.autocorr(_responses(T, 30, 2000, seed=7), Nj).astype(np.complex64)
    z = synth.complex_gaussian_snr(1, (T, nd, n + 2 * Nj + 3), sub=31)
    xi = sp.xi2(_cuda(z), _cuda(A), Nj, n).cpu().numpy()
    xi_or = oracle.xi2(z, A, Nj, n)
    err = np.abs(xi - xi_or) / np.maximum(np.abs(xi_or), 1.0)
    assert err.max() < XI_TOL, err.max()
    if n >= 100:
        assert 0.5 < xi_or.mean() < 2.0


def test_xi2_of_a_template_shaped_window_is_near_zero():
    import paper_2011_06787_b300 as sp
    Nj, n = 175, 1100
    A = oracle.autocorr(_responses(1, 30, 2000, seed=9), Nj).astype(np.complex64)
    z = synth.complex_gaussian_snr(1, (1, 2, n + 2 * Nj), sub=32)
    k0 = 600
    z[0, 0, k0: k0 + 2 * Nj + 1] = (5.0 - 2.0j) * A[0]  # centred on sample k0 (entry Nj + k0)
    xi = sp.xi2(_cuda(z), _cuda(A), Nj, n).cpu().numpy()
    assert xi[0, 0, k0] < 1e-5
    assert xi[0, 1, k0] > 0.2


def test_network_average_on_a_coherent_scan():
    """xi_C^2 gathered at the coherent argmax: the GPU gather and the oracle's gather of the
    oracle's per-detector statistic, both at the oracle's own coherent argmax (the argmax of
    the GPU scan agrees with it almost everywhere; the scan's parity is tested elsewhere)."""
    import torch
    import paper_2011_06787_b300 as sp
    det = synth.detectors(1, 3)
    sigma = synth.noise_weights(1, 3, 0.5, 2.0)
    tabs = sp.sky_tables(det.pos_m, det.arm_x, det.arm_y, sigma, 8, 2048.0)
    sky = sp.Sky(*tabs)
    H, T, n, Nj = sky.halo, 2, 1500, 40
    z = synth.complex_gaussian_snr(1, (T, 3, n + 2 * H + 2 * Nj), sub=33)
    A = oracle.autocorr(_responses(T, 20, 1500, seed=10), Nj).astype(np.complex64)
    # coherent scan on the window [Nj, Nj + n + 2H): entry H + k of its rows is sample k
    zs = np.ascontiguousarray(z[:, :, Nj:])
    ms = torch.empty((T, n), device="cuda")
    am = torch.empty((T, n), dtype=torch.int32, device="cuda")
    nl = torch.empty((T, n), device="cuda")
    sky.scan(_cuda(zs), n, ms, am, nl)
    _, G, d_or = oracle.sky_geometry(det, sigma, 8, 2048.0)
    _, am_or, _, _ = oracle.coherent(zs, G, d_or, H, n)
    assert float(np.mean(am.cpu().numpy() == am_or)) > 0.99
    # xi^2 of samples -H .. n + H - 1 (entry H + k = sample k)
    xi = sp.xi2(_cuda(z), _cuda(A), Nj, n + 2 * H)
    xc = sp.xi2_network(sky, xi, _cuda(am_or.astype(np.int32)), n).cpu().numpy()
    xi_or = oracle.xi2(z, A, Nj, n + 2 * H)
    xc_or = oracle.xi2_network(xi_or, d_or, am_or, H)
    assert np.max(np.abs(xc - xc_or) / np.maximum(xc_or, 1.0)) < XI_TOL


def test_online_full_size_sampled_templates():
    """The online workload's SNR (1024 templates, 3 detectors, one 2048-sample chunk plus
    Nj = 175 samples of history and lookahead) through the GPU filter bank, then xi^2 for all
    templates; the oracle filters the same strain for a sample of templates and computes their
    xi^2.  The two SNRs agree to the filter bank's parity tolerance (1e-4 of the row maximum),
    which xi^2 passes on amplified by about the ratio of |z| to the residuals it sums: 5e-4."""
    import torch
    import paper_2011_06787_b300 as sp
    Nj, n = 175, 2048
    bank = synth.online_bank()
    x = np.concatenate([synth.online_chunk(i) for i in range(3)], axis=1)
    b = sp.Bank(3, bank.offsets, bank.a1, bank.b0, bank.delay)
    z = torch.zeros((1024, 3, x.shape[1]), dtype=torch.complex64, device="cuda")
    b.filter_chunk(torch.from_numpy(np.ascontiguousarray(x)).cuda(), z)
    zw = z[:, :, 2048 - Nj: 2048 + n + Nj].contiguous()
    pick = [0, 512, 1023]
    sub = bank.subset(pick)
    u = oracle.impulse_forward(sub.offsets, sub.a1, sub.b0, sub.delay, np.zeros(sub.n_filters, np.complex64), 6000)
    A_or = oracle.autocorr(u, Nj).astype(np.complex64)
    A = torch.zeros((1024, 2 * Nj + 1), dtype=torch.complex64, device="cuda")
    A[:] = _cuda(A_or[0])
    A[pick] = _cuda(A_or)
    xi = sp.xi2(zw, A, Nj, n).cpu().numpy()
    z_or, _, _ = oracle.filter_bank(x, sub.offsets, sub.a1, sub.b0, sub.delay)
    xi_or = oracle.xi2(z_or[:, :, 2048 - Nj: 2048 + n + Nj], A_or, Nj, n)
    err = np.abs(xi[pick] - xi_or) / np.maximum(np.abs(xi_or), 1.0)
    assert err.max() < 5e-4, err.max()
    assert np.isfinite(xi).all()
