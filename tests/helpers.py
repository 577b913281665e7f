"""Shared checks for the parity tests (tolerances from the method's accuracy targets)."""
import numpy as np

SNR_TOL = 1e-4      # max_k |z_gpu - z_oracle| <= SNR_TOL * max_k |z_oracle| per (template, detector)
STAT_TOL = 1e-4     # coherent statistic: relative
NULL_TOL = 1e-4     # null stream: absolute, in units of the statistic at that sample
TIE_TOL = 1e-4      # argmax must match exactly when the oracle's top-2 margin exceeds this


def cuda_ok():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def assert_snr_close(z_gpu, z_or, tol=SNR_TOL):
    z_gpu = np.asarray(z_gpu)
    z_or = np.asarray(z_or)
    assert z_gpu.shape == z_or.shape, (z_gpu.shape, z_or.shape)
    err = np.abs(z_gpu.astype(np.complex128) - z_or).max(axis=-1)
    ref = np.abs(z_or).max(axis=-1)
    bad = err > tol * np.maximum(ref, 1e-30)
    assert not bad.any(), f"{bad.sum()} rows exceed tol; worst ratio {np.max(err / np.maximum(ref, 1e-30)):.3e}"


def assert_coherent_close(ms, am, nl, ms_or, am_or, nl_or, skymap_or=None):
    ms = np.asarray(ms, dtype=np.float64)
    nl = np.asarray(nl, dtype=np.float64)
    assert np.all(np.abs(ms - ms_or) <= STAT_TOL * np.abs(ms_or) + 1e-30), \
        f"max_stat rel err {np.max(np.abs(ms - ms_or) / np.maximum(np.abs(ms_or), 1e-30)):.3e}"
    if skymap_or is not None:
        top2 = np.sort(skymap_or, axis=-1)[..., -2] if skymap_or.shape[-1] > 1 else np.zeros_like(ms_or)
        margin = (ms_or - top2) / np.maximum(ms_or, 1e-30)
        clear = margin > TIE_TOL
        assert np.all(am[clear] == am_or[clear]), f"{np.sum(am[clear] != am_or[clear])} clear argmax mismatches"
        # near ties: the chosen pixel must be within tolerance of the maximum
        vals = np.take_along_axis(skymap_or, np.asarray(am)[..., None].astype(np.int64), axis=-1)[..., 0]
        assert np.all(vals >= ms_or * (1 - TIE_TOL) - 1e-30)
        ok = clear | (am == am_or)
        assert np.all(np.abs(nl[ok] - nl_or[ok]) <= NULL_TOL * np.maximum(ms_or[ok], 1e-30) + 1e-30), \
            f"null abs err {np.max(np.abs(nl[ok] - nl_or[ok]) / np.maximum(ms_or[ok], 1e-30)):.3e}"
    else:
        same = am == am_or
        assert same.mean() > 0.999, f"argmax agreement {same.mean():.5f}"
        assert np.all(np.abs(nl[same] - nl_or[same]) <= NULL_TOL * np.maximum(ms_or[same], 1e-30) + 1e-30)
