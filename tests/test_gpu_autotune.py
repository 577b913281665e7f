"""Launch-shape autotuner: the shapes it keeps come from its candidate lists, tuning leaves the
bank's stream where it was, results after tuning match the FP64 oracle, and the JSON cache
short-cuts a second search."""
import json

import numpy as np
import pytest

import oracle
import synth
from helpers import assert_coherent_close, assert_snr_close, cuda_ok

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs CUDA")]


def test_tune_bank_keeps_the_stream_and_caches(tmp_path):
    import torch
    import paper_2011_06787_b300 as sp
    from paper_2011_06787_b300 import autotune
    autotune._cache.clear()
    g = synth.rng(0, "misc", 31)
    bank = synth.random_bank(g, [180, 40, 420, 77, 260], d_max=900)
    n = 1024
    x = synth.white_noise(0, 2, 3 * n, sub=31)
    b = sp.Bank(2, bank.offsets, bank.a1, bank.b0, bank.delay)
    chunk = [torch.from_numpy(np.ascontiguousarray(x[:, i * n:(i + 1) * n])).cuda() for i in range(3)]
    zs = []
    z = torch.zeros((bank.n_templates, 2, n), dtype=torch.complex64, device="cuda")
    b.filter_chunk(chunk[0], z)
    zs.append(z.cpu().numpy())
    cache = str(tmp_path / "tune.json")
    scratch = torch.zeros_like(z)
    rec = autotune.tune_bank(b, chunk[1], scratch, reps=1, cache_path=cache)
    assert tuple(rec["shape"]) in autotune.BANK_SHAPES and rec["tried"]
    assert tuple(b.get_shape()) == tuple(rec["shape"])
    for i in (1, 2):
        b.filter_chunk(chunk[i], z)
        zs.append(z.cpu().numpy())
    # the timing calls advanced the stream; the tuner restored it, so the three chunks are the
    # oracle's continuous stream
    z_or, _, _ = oracle.filter_bank(x, bank.offsets, bank.a1, bank.b0, bank.delay)
    assert_snr_close(np.concatenate(zs, axis=2), z_or)
    # the record is in the file, and a new search on the same problem is skipped
    key = autotune.bank_key(b, n)
    assert json.load(open(cache))[key]["shape"] == rec["shape"]
    autotune._cache.clear()
    again = autotune.tune_bank(b, chunk[1], scratch, reps=1, cache_path=cache)
    assert again == json.load(open(cache))[key]


def test_tune_scan_keeps_a_valid_shape_and_matches_the_oracle(tmp_path):
    import torch
    import paper_2011_06787_b300 as sp
    from paper_2011_06787_b300 import autotune
    autotune._cache.clear()
    det = synth.detectors(1, 3)
    sigma = synth.noise_weights(1, 3, 0.5, 2.0)
    sky = sp.Sky(*sp.sky_tables(det.pos_m, det.arm_x, det.arm_y, sigma, 8, 2048.0))
    _, G, d_or = oracle.sky_geometry(det, sigma, 8, 2048.0)
    H, T, n = sky.halo, 3, 1500
    z = synth.complex_gaussian_snr(1, (T, 3, n + 2 * H), sub=33).astype(np.complex64)
    zt = torch.from_numpy(z).cuda()
    ms = torch.empty((T, n), dtype=torch.float32, device="cuda")
    am = torch.empty((T, n), dtype=torch.int32, device="cuda")
    nl = torch.empty((T, n), dtype=torch.float32, device="cuda")
    rec = autotune.tune_scan(sky, zt, n, ms, am, nl, reps=1, cache_path=str(tmp_path / "tune.json"))
    tried = {tuple(s) for _, s in rec["tried"]}
    skipped = {tuple(s) for s, _ in rec["skipped"]}
    assert tried | skipped == set(autotune.SCAN_SHAPES) and tuple(rec["shape"]) in tried
    # all four tensor-memory shapes apply to this sky (3 detectors, small halo)
    assert {(512, 4, 1), (256, 4, 1), (512, 4, 0), (256, 4, 0)} <= tried
    assert tuple(sky.get_scan_shape()[:3]) == tuple(rec["shape"])
    sky.scan(zt, n, ms, am, nl)
    torch.cuda.synchronize()
    ms_or, am_or, nl_or, sm_or = oracle.coherent(z, G, d_or, H, n, skymap=True)
    assert_coherent_close(ms.cpu().numpy(), am.cpu().numpy(), nl.cpu().numpy(), ms_or, am_or, nl_or, sm_or)
