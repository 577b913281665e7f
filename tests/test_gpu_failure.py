"""Failure detection without a GPU fault: a device wait that runs out of iterations is
reported through the sticky status word and leaves the context usable; injected allocation
failures make the create calls fail cleanly and leave the library usable."""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from helpers import assert_snr_close, cuda_ok

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs CUDA")]


def _tiny_filter_check():
    import torch
    import paper_2011_06787_b300 as sp
    w = synth.tiny_workload()
    bank, x = w["bank"], w["strain"][:, :4096]
    b = sp.Bank(2, bank.offsets, bank.a1, bank.b0, bank.delay)
    z = torch.zeros((bank.n_templates, 2, x.shape[1]), dtype=torch.complex64, device="cuda")
    b.filter_chunk(torch.from_numpy(np.ascontiguousarray(x)).cuda(), z)
    z_or, _, _ = oracle.filter_bank(x, bank.offsets, bank.a1, bank.b0, bank.delay)
    assert_snr_close(z.cpu().numpy(), z_or)


def test_bounded_wait_timeout_is_reported_and_the_context_stays_usable():
    import torch
    import paper_2011_06787_b300 as sp
    from paper_2011_06787_b300 import native
    L = native.lib()
    sp.device_status()  # start from a clear word
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    native.check(L.spiir_debug_wait_timeout(1 << 12, st))
    with pytest.raises(sp.SpiirError) as e:
        sp.device_status()
    assert e.value.code == native.ETIMEOUT
    sp.device_status()  # the previous call cleared the word
    _tiny_filter_check()
    sp.device_status()


def _walk_allocation_sites(L, native, sp, build, limit=200):
    """Fail the k-th allocation for k = 1, 2, ... until build() succeeds; every failure must be
    a clean SPIIR_ENOMEM.  Returns the number of allocations build() makes."""
    try:
        for k in range(1, limit):
            L.spiir_debug_fail_alloc_at(k)
            try:
                build()
            except sp.SpiirError as e:
                assert e.code == native.ENOMEM and "injected" in str(e), str(e)
                continue
            return k - 1
        raise AssertionError("build() kept failing")
    finally:
        L.spiir_debug_fail_alloc_at(0)
        L.spiir_debug_fail_allocs(0)


def test_injected_allocation_failures_fail_the_create_calls_cleanly():
    import torch
    import paper_2011_06787_b300 as sp
    from paper_2011_06787_b300 import native
    L = native.lib()
    w = synth.tiny_workload()
    bank, det = w["bank"], w["det"]
    tabs = sp.sky_tables(det.pos_m, det.arm_x, det.arm_y, w["sigma"], 4, 2048.0)
    sky = sp.Sky(*tabs)

    def bank_and_pipeline():
        b = sp.Bank(2, bank.offsets, bank.a1, bank.b0, bank.delay)
        sp.Pipeline(b, sky, max_chunk=1024)

    assert _walk_allocation_sites(L, native, sp, bank_and_pipeline) >= 3
    assert _walk_allocation_sites(L, native, sp, lambda: sp.Sky(*tabs)) >= 2

    det3 = synth.detectors(1, 3)
    sky3 = sp.Sky(*sp.sky_tables(det3.pos_m, det3.arm_x, det3.arm_y, synth.noise_weights(1, 3, 0.5, 2.0), 4, 2048.0))
    banks = synth.multirate_banks(n_banks=2, t_range=(3, 6), f_range=(20, 40), seed_sub=5)

    def batch_and_graph_run():
        bt = sp.Batch(3, banks, (1, 4, 16), sky3, 512)
        T = bt.n_templates
        ms = torch.empty((T, 512), device="cuda")
        am = torch.empty((T, 512), dtype=torch.int32, device="cuda")
        nl = torch.empty((T, 512), device="cuda")
        bt.run(torch.zeros((3, 512), device="cuda"), ms, am, nl, mode=2)
        torch.cuda.synchronize()

    assert _walk_allocation_sites(L, native, sp, batch_and_graph_run) >= 5
    # the next n allocations fail
    L.spiir_debug_fail_allocs(1)
    try:
        with pytest.raises(sp.SpiirError) as e:
            sp.Sky(*tabs)
        assert e.value.code == native.ENOMEM
    finally:
        L.spiir_debug_fail_allocs(0)
    _tiny_filter_check()
    sp.device_status()


@pytest.mark.parametrize("overlap", [False, True])
def test_injected_allocation_failures_fail_the_search_cleanly(overlap):
    """Every allocation of a streaming search's set-up and first chunk (its bank, sky, ring,
    autocorrelations, selection workspace and the sky's lazily built point table) fails
    cleanly when injected, and the library stays usable."""
    import torch
    import paper_2011_06787_b300 as sp
    from paper_2011_06787_b300 import native
    L = native.lib()
    det = synth.detectors(5, 3)
    tabs = sp.sky_tables(det.pos_m, det.arm_x, det.arm_y, synth.noise_weights(5, 3, 0.5, 2.0), 4, 2048.0)
    bank = synth.random_bank(synth.rng(5, "misc", 3), [20, 30, 25], d_max=300)

    def search_and_run():
        sky = sp.Sky(*tabs)
        b = sp.Bank(3, bank.offsets, bank.a1, bank.b0, bank.delay)
        A = torch.zeros((3, 21), dtype=torch.complex64, device="cuda")
        A[:, 10] = 1.0
        s = sp.Search(b, sky, sky, A, 10, 512, n_shifts=2, shift_step=40, max_cand=64, overlap=overlap)
        s.run(torch.zeros((3, 512), device="cuda"))
        torch.cuda.synchronize()

    assert _walk_allocation_sites(L, native, sp, search_and_run) >= 6
    _tiny_filter_check()
    sp.device_status()


def test_injected_failures_in_the_first_asynchronous_step_are_resumable():
    """The second staging set of the asynchronous host-buffer steps is allocated on the first
    submission: failing each of its allocations in turn makes that call fail with SPIIR_ENOMEM,
    and the next call resumes the setup and processes the chunk as the synchronous call does."""
    import torch
    import paper_2011_06787_b300 as sp
    from paper_2011_06787_b300 import native
    L = native.lib()
    w = synth.tiny_workload()
    bank, det = w["bank"], w["det"]
    sky = sp.Sky(*sp.sky_tables(det.pos_m, det.arm_x, det.arm_y, w["sigma"], 4, 2048.0))
    x = np.ascontiguousarray(w["strain"][:, :1024])
    T = bank.n_templates
    pin = lambda dt: torch.empty((T, 1024), dtype=dt).pin_memory().numpy()
    pipe = sp.Pipeline(sp.Bank(2, bank.offsets, bank.a1, bank.b0, bank.delay), sky, max_chunk=1024)
    out = (pin(torch.float32), pin(torch.int32), pin(torch.float32))
    try:
        # each call makes only the allocations still missing: failing the first allocation of
        # the first call, then the second of the next three, walks the four staging allocations
        # (each call completes one more of them before the injected failure)
        for k, site in zip((1, 2, 2, 2), ("strain", "max", "null", "argmax")):
            L.spiir_debug_fail_alloc_at(k)
            with pytest.raises(sp.SpiirError) as e:
                pipe.submit_host(x, *out)
            assert e.value.code == native.ENOMEM
            assert f"for {site} staging" in str(e.value), str(e.value)
        # the four failures hit strain, max, null and argmax staging in that order; without an
        # injected failure the fifth call completes the setup (the argmax staging) and runs
        L.spiir_debug_fail_alloc_at(0)
        pipe.submit_host(x, *out)
        pipe.wait()
    finally:
        L.spiir_debug_fail_alloc_at(0)
    pipe.reset()
    pipe.submit_host(x, *out)
    pipe.wait()
    ref = sp.Pipeline(sp.Bank(2, bank.offsets, bank.a1, bank.b0, bank.delay), sky, max_chunk=1024)
    r = (pin(torch.float32), pin(torch.int32), pin(torch.float32))
    ref.run_host(x, *r)
    for a, b in zip(out, r):
        np.testing.assert_array_equal(a, b)
    sp.device_status()
