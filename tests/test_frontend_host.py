"""Host helpers of the front end (Sec. II.A) on the CPU: the library's FP64 designs of the
decimation low-pass and of the whitening kernel of Eq. (whiten) against the oracle's, and their
argument checks.  No GPU is used."""
import numpy as np
import pytest

import oracle


def _psd_ar1(fs, N, phi, s):
    f = np.arange(N // 2 + 1) * fs / N
    return (2.0 * s ** 2 / fs) / np.abs(1.0 - phi * np.exp(-2j * np.pi * f / fs)) ** 2


@pytest.mark.parametrize("n,M,cutoff", [(192, 8, 0.9), (32, 4, 0.8), (1, 1, 1.0), (33, 16, 0.5)])
def test_lowpass_matches_oracle(n, M, cutoff):
    import paper_2011_06787_b300 as sp
    h = sp.fir_lowpass(n, M, cutoff)
    ho = oracle.lowpass_taps(n, M, cutoff)
    np.testing.assert_allclose(h, ho.astype(np.float32), rtol=0, atol=2e-7 * np.abs(ho).max())
    assert abs(float(np.sum(h.astype(np.float64))) - 1.0) < 1e-6


@pytest.mark.parametrize("L,N,phi", [(1025, 4096, 0.9), (101, 256, 0.0), (4097, 8192, -0.4), (1, 16, 0.3)])
def test_whitening_kernel_matches_oracle(L, N, phi):
    import paper_2011_06787_b300 as sp
    psd = _psd_ar1(2048.0, N, phi, 1.7)
    w = sp.whitening_kernel(psd, 2048.0, L)
    wo = oracle.whitening_kernel(psd, 2048.0, L)
    np.testing.assert_allclose(w, wo.astype(np.float32), rtol=0, atol=1e-6 * np.abs(wo).max())


def test_host_helpers_reject_bad_arguments():
    import paper_2011_06787_b300 as sp
    psd = _psd_ar1(2048.0, 64, 0.5, 1.0)
    for args in ((psd, 2048.0, 64), (psd, 2048.0, 65), (psd, 0.0, 31)):   # even, too long, rate 0
        with pytest.raises(sp.SpiirError):
            sp.whitening_kernel(*args)
    bad = psd.copy()
    bad[3] = 0.0
    with pytest.raises(sp.SpiirError):
        sp.whitening_kernel(bad, 2048.0, 31)
    for args in ((0, 8, 0.9), (192, 0, 0.9), (192, 8, 0.0), (192, 8, 1.5)):
        with pytest.raises(sp.SpiirError):
            sp.fir_lowpass(*args)
