"""Launch-shape autotuner for the filter bank and the coherent scan.

Each candidate shape is applied through the C ABI (spiir_bank_set_shape,
spiir_sky_set_scan_shape), timed with CUDA events on the current stream over a few
repetitions of a representative call, and the fastest is kept.  Results are cached in
memory and, optionally, in a JSON file keyed by the problem shape, so that later runs on
the same problem skip the search.
"""
from __future__ import annotations

import json
import os

BANK_SHAPES = [(8, 256, 32, 1024), (8, 128, 32, 1024), (8, 128, 64, 1024), (8, 128, 20, 1000), (4, 256, 16, 1024), (4, 128, 16, 1024),
               (8, 256, 16, 1024), (8, 128, 16, 2048), (16, 256, 32, 1024), (16, 128, 16, 1024)]
SCAN_SHAPES = [(512, 4, 1), (256, 4, 1), (512, 4, 0), (256, 4, 0), (256, 2, 1), (256, 2, 0), (512, 1, 0), (256, 1, 0), (512, 2, 0), (512, 1, 1)]

_cache: dict = {}


def _time_ms(fn, reps):
    import torch
    s = torch.cuda.current_stream()
    fn()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        fn()
    e1.record(s)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def _load(path):
    if path and os.path.exists(path):
        try:
            return json.load(open(path))
        except Exception:
            return {}
    return {}


def _store(path, key, value):
    if not path:
        return
    d = _load(path)
    d[key] = value
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1)
    os.replace(tmp, path)


def bank_key(bank, n):
    return f"bank:det{bank.n_det}:T{bank.n_templates}:F{bank.n_filters}:d{bank.max_delay}:n{n}"


def tune_bank(bank, strain, out, reps=3, shapes=BANK_SHAPES, cache_path=None, verbose=False):
    """Pick the fastest filter-bank shape for this bank and chunk length.  The bank's stream
    state is restored afterwards (the timing calls advance it)."""
    key = bank_key(bank, strain.shape[1])
    hit = _cache.get(key) or _load(cache_path).get(key)
    if hit:
        bank.set_shape(*hit["shape"])
        _cache[key] = hit
        return hit
    state = bank.get_state()
    results = []
    for shp in shapes:
        try:
            bank.set_shape(*shp)
        except Exception:
            continue
        ms = _time_ms(lambda: bank.filter_chunk(strain, out), reps)
        results.append((ms, shp))
        if verbose:
            print(f"bank shape {shp}: {ms:.3f} ms")
    best = min(results)
    bank.set_shape(*best[1])
    bank.set_state(state)
    rec = {"shape": list(best[1]), "ms": best[0], "tried": [[m, list(s)] for m, s in results]}
    _cache[key] = rec
    _store(cache_path, key, rec)
    return rec


def sky_key(sky, T, n):
    return f"sky:det{sky.n_det}:P{sky.n_pix}:H{sky.halo}:T{T}:n{n}"


def tune_scan(sky, snr, n, max_stat, argmax, null_stat, reps=3, shapes=SCAN_SHAPES, cache_path=None, verbose=False):
    key = sky_key(sky, snr.shape[0], n)
    hit = _cache.get(key) or _load(cache_path).get(key)
    if hit:
        sky.set_scan_shape(*hit["shape"])
        _cache[key] = hit
        return hit
    results, skipped = [], []
    for shp in shapes:
        try:
            sky.set_scan_shape(*shp)
        except Exception as e:
            skipped.append([list(shp), str(e)])
            continue
        ms = _time_ms(lambda: sky.scan(snr, n, max_stat, argmax, null_stat), reps)
        results.append((ms, shp))
        if verbose:
            print(f"scan shape {shp}: {ms:.3f} ms")
    best = min(results)
    sky.set_scan_shape(*best[1])
    rec = {"shape": list(best[1]), "ms": best[0], "tried": [[m, list(s)] for m, s in results], "skipped": skipped}
    _cache[key] = rec
    _store(cache_path, key, rec)
    return rec


BATCH_SHAPES = [(8, 128, 32, 0), (8, 256, 32, 0), (8, 128, 16, 0), (8, 128, 32, 1), (16, 128, 32, 0), (4, 128, 16, 0)]


def tune_batch(batch, strain, max_stat, argmax, null_stat, reps=4, shapes=BATCH_SHAPES, verbose=False):
    """Pick the persistent-launch shape of a Batch by timing graph replays of one chunk.  The
    batch is reset afterwards (the timing calls advance its stream state)."""
    results = []
    for shp in shapes:
        try:
            batch.set_shape(*shp)
        except Exception:
            continue
        batch.reset()
        ms = _time_ms(lambda: batch.run(strain, max_stat, argmax, null_stat, mode=2), reps)
        results.append((ms, shp))
        if verbose:
            print(f"batch shape {shp}: {ms:.3f} ms")
    best = min(results)
    batch.set_shape(*best[1])
    batch.reset()
    return {"shape": list(best[1]), "ms": best[0], "tried": [[m, list(s)] for m, s in results]}
