"""Host-side FP64 sky tables of the library against the oracle's independent geometry
(Sec. II.C.1 look-up tables; App. A Eq. (svd)).  Runs on the CPU."""
import numpy as np
import pytest

import oracle
import paper_2011_06787_b300 as sp
import synth


@pytest.mark.parametrize("cfg,n_det,nside,sig", [(0, 2, 4, (1.0, 1.0)), (1, 3, 16, (0.5, 2.0)), (5, 4, 8, (0.7, 1.6))])
def test_tables_match_oracle_geometry(cfg, n_det, nside, sig):
    det = synth.detectors(cfg, n_det)
    sigma = synth.noise_weights(cfg, n_det, *sig)
    delays, u_sig, u_null = sp.sky_tables(det.pos_m, det.arm_x, det.arm_y, sigma, nside, 2048.0)
    nhat, G, d_or = oracle.sky_geometry(det, sigma, nside, 2048.0)
    # integer arrival offsets: bit-exact
    np.testing.assert_array_equal(delays, d_or)
    assert np.abs(delays).max() <= 44
    P = 12 * nside * nside
    for p in range(P):
        U = np.concatenate([u_sig[p], u_null[p]], axis=1).astype(np.float64) if n_det > 2 else u_sig[p].astype(np.float64)
        # orthonormal columns
        np.testing.assert_allclose(U.T @ U, np.eye(U.shape[1]), atol=3e-7)
        # the signal columns span the column space of G_sigma: same projector as the
        # oracle's normal equations
        Pi_or = G[p] @ np.linalg.solve(G[p].T @ G[p], G[p].T)
        Pi = u_sig[p].astype(np.float64) @ u_sig[p].astype(np.float64).T
        np.testing.assert_allclose(Pi, Pi_or, atol=3e-7)


def test_rank_deficient_pixel_keeps_one_signal_column():
    # two co-located, co-aligned detectors: G_sigma has rank 1 at every pixel
    det = synth.detectors(0, 1)
    pos = np.repeat(det.pos_m, 2, axis=0)
    ax = np.repeat(det.arm_x, 2, axis=0)
    ay = np.repeat(det.arm_y, 2, axis=0)
    delays, u_sig, _ = sp.sky_tables(pos, ax, ay, np.ones(2), 2, 2048.0)
    assert np.all(u_sig[:, :, 1] == 0.0)
    np.testing.assert_allclose(np.linalg.norm(u_sig[:, :, 0], axis=1), 1.0, atol=1e-6)
