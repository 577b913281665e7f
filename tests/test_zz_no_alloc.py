"""The allocation-free filter entry point (spiir_filter_static).

Some callers cannot allocate device memory -- code running where cudaMalloc is forbidden or
would stall, such as a real-time loop, under an allocator that owns all device memory, or in a
process whose footprint is frozen after start-up.  They get one entry point whose scratch lives
in a fixed file-scope device array.  This file is collected last, so that a run stopping at the
first failure has already run every other test.  It calls the entry point through the C ABI
twice in a row, with different problems, and compares each result with the FP64 oracle and
with the allocating path (spiir_bank_create + spiir_filter_chunk on a new bank) within the
tolerance of the other parity tests.  Every call runs with the library's allocation hook armed
to fail, so that a call reaching any allocating routine of the library would return an error.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from helpers import SNR_TOL, assert_snr_close, cuda_ok

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs CUDA")]


def _problem(sub, counts, d_max, n_det, n):
    g = synth.rng(2, "misc", sub)
    bank = synth.random_bank(g, counts, d_max=d_max)
    x = synth.white_noise(2, n_det, n, sub=sub)
    return bank, x


def _static(bank, x):
    import torch
    from paper_2011_06787_b300 import native
    L = native.lib()
    n_det, n = x.shape
    off = np.ascontiguousarray(bank.offsets, np.int64)
    a1 = np.ascontiguousarray(bank.a1, np.complex64).view(np.float32)
    b0 = np.ascontiguousarray(bank.b0, np.complex64).view(np.float32)
    d = np.ascontiguousarray(bank.delay, np.int32)
    xs = torch.from_numpy(x).cuda()
    z = torch.zeros((bank.n_templates, n_det, n), dtype=torch.complex64, device="cuda")
    torch.cuda.synchronize()
    P = ctypes.c_void_p
    L.spiir_debug_fail_allocs(1 << 30)   # any allocation by the library would now fail
    try:
        rc = L.spiir_filter_static(n_det, bank.n_templates, P(off.ctypes.data), P(a1.ctypes.data),
                                   P(b0.ctypes.data), P(d.ctypes.data), P(xs.data_ptr()), n, n,
                                   P(z.data_ptr()), n, P(torch.cuda.current_stream().cuda_stream))
        native.check(rc)
        torch.cuda.synchronize()         # the host arrays are read until the stream passes the call
        native.check(L.spiir_device_status(0))   # no bounded device wait ran out
    finally:
        L.spiir_debug_fail_allocs(0)
    return z.cpu().numpy()


def _allocating(bank, x):
    import torch
    import paper_2011_06787_b300 as sp
    b = sp.Bank(x.shape[0], bank.offsets, bank.a1, bank.b0, bank.delay)
    z = torch.zeros((bank.n_templates, x.shape[0], x.shape[1]), dtype=torch.complex64, device="cuda")
    b.filter_chunk(torch.from_numpy(x).cuda(), z)
    torch.cuda.synchronize()
    return z.cpu().numpy()


def _oracle(bank, x):
    z, _, _ = oracle.filter_bank(x, bank.offsets, bank.a1, bank.b0, bank.delay)
    return z


def test_static_entry_matches_oracle_and_allocating_path_on_two_calls_in_a_row():
    # first call: three detectors, uneven templates (one large enough for 256-lane blocks)
    bank1, x1 = _problem(1, [5, 300, 1, 1500, 64, 0, 777], 3000, 3, 4100)
    # second call: a different, smaller problem; the scratch keeps the first call's contents
    bank2, x2 = _problem(2, [64] * 9 + [33], 500, 2, 1500)
    z1 = _static(bank1, x1)
    z2 = _static(bank2, x2)
    assert_snr_close(z1, _oracle(bank1, x1), SNR_TOL)
    assert_snr_close(z2, _oracle(bank2, x2), SNR_TOL)
    assert_snr_close(z1, _allocating(bank1, x1).astype(np.complex128), SNR_TOL)
    assert_snr_close(z2, _allocating(bank2, x2).astype(np.complex128), SNR_TOL)
    # repeating the first problem after the second gives the same result again
    np.testing.assert_array_equal(_static(bank1, x1), z1)


def test_static_entry_shares_the_reported_status_word():
    """A bounded wait that runs out is reported through spiir_device_status for this entry point
    too: the status word it passes its kernel is the library's one, which the debug hook sets."""
    import torch
    from paper_2011_06787_b300 import native
    L = native.lib()
    bank, x = _problem(4, [40, 17], 200, 2, 700)
    z = _static(bank, x)
    native.check(L.spiir_debug_wait_timeout(1000, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    assert L.spiir_device_status(1) == native.ETIMEOUT
    assert L.spiir_device_status(0) == native.OK
    np.testing.assert_array_equal(_static(bank, x), z)


def test_static_entry_rejects_problems_beyond_its_limits():
    import paper_2011_06787_b300 as sp
    bank, x = _problem(3, [10], 100, 1, 70000)   # more samples than the static limit
    with pytest.raises(sp.SpiirError) as e:
        _static(bank, x)
    assert e.value.code == sp.native.EUNSUPPORTED and "65536" in str(e.value)
