"""B300 (sm_103a) SPIIR hot path: filter bank and coherent sky scan behind a C ABI.

The classes here marshal arguments into the C entry points of libspiir.so
(include/spiir.h); every step of the computation runs in the library's CUDA kernels.
PyTorch supplies device memory and the current CUDA stream.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import native
from .native import SpiirError, check

__all__ = ["Bank", "Sky", "Pipeline", "Batch", "sky_tables", "autocorr", "xi2", "xi2_network", "Selector",
           "coherent_candidates", "xi2_candidates", "Frontend", "fir_lowpass", "whitening_kernel", "SpiirError", "device_status", "version"]


def _stream_ptr(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _host_ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _dev_ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _require_cuda(t, dtype, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")


def version() -> int:
    return native.lib().spiir_version()


def device_status(clear: bool = True) -> None:
    """Raise SpiirError(ETIMEOUT) if a bounded device-side wait gave up since the last check."""
    check(native.lib().spiir_device_status(1 if clear else 0))


class Bank:
    """SPIIR filter bank (Sec. II.B.1, Eq. (zk)); see spiir_bank_create in include/spiir.h.

    offsets [T+1] int64, a1 / b0 [F] complex, delay [F] int32 (host arrays).
    """

    def __init__(self, n_det: int, offsets, a1, b0, delay):
        L = native.lib()
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        a = np.ascontiguousarray(np.asarray(a1, dtype=np.complex64)).view(np.float32)
        b = np.ascontiguousarray(np.asarray(b0, dtype=np.complex64)).view(np.float32)
        d = np.ascontiguousarray(delay, dtype=np.int32)
        h = ctypes.c_void_p()
        check(L.spiir_bank_create(int(n_det), int(off.size - 1), _host_ptr(off), _host_ptr(a), _host_ptr(b),
                                  _host_ptr(d), ctypes.byref(h)))
        self._h = h
        self.n_det = int(n_det)
        self.n_templates = int(off.size - 1)
        self.n_filters = int(off[-1])
        self.max_delay = int(d.max()) if d.size else 0

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            native.lib().spiir_bank_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self, stream=None):
        check(native.lib().spiir_bank_reset(self._h, _stream_ptr(stream)))

    def filter_chunk(self, strain, out, stream=None):
        """strain: float32 CUDA tensor [n_det][n] (row stride = pitch); out: complex64 CUDA tensor
        [T][n_det][>= n] whose first n samples of each row are written."""
        import torch
        _require_cuda(strain, torch.float32, "strain")
        _require_cuda(out, torch.complex64, "out")
        if strain.dim() != 2 or strain.shape[0] != self.n_det or strain.stride(1) != 1:
            raise ValueError("strain must be [n_det][n] with unit stride along time")
        n = strain.shape[1]
        if out.dim() != 3 or out.shape[0] != self.n_templates or out.shape[1] != self.n_det or out.stride(2) != 1 \
                or out.stride(1) != out.stride(0) // self.n_det or out.shape[2] < n:
            raise ValueError("out must be a [T][n_det][pitch] complex64 tensor with contiguous rows")
        check(native.lib().spiir_filter_chunk(self._h, _dev_ptr(strain), strain.stride(0), n, _dev_ptr(out),
                                              out.stride(1), _stream_ptr(stream)))
        return out

    def set_shape(self, filters_per_lane=8, lanes_per_block=128, steps_per_reduce=32, tile=1024):
        """Launch shape of the filter-bank kernel (spiir_bank_set_shape); keeps the stream state."""
        check(native.lib().spiir_bank_set_shape(self._h, int(filters_per_lane), int(lanes_per_block),
                                                int(steps_per_reduce), int(tile)))

    def get_shape(self):
        v = [ctypes.c_int() for _ in range(4)]
        check(native.lib().spiir_bank_get_shape(self._h, *[ctypes.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def set_delay_bin(self, delay_bin: int):
        """Delay-bin width of the block layout (spiir_bank_set_delay_bin); 0 keeps templates whole."""
        check(native.lib().spiir_bank_set_delay_bin(self._h, int(delay_bin)))

    def get_delay_bin(self):
        """(delay-bin width, thread blocks, delay pieces) of the current layout."""
        v = [ctypes.c_int32(), ctypes.c_int(), ctypes.c_int()]
        check(native.lib().spiir_bank_get_delay_bin(self._h, *[ctypes.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def state_bytes(self) -> int:
        n = ctypes.c_size_t()
        check(native.lib().spiir_bank_state_bytes(self._h, ctypes.byref(n)))
        return n.value

    def get_state(self) -> bytes:
        buf = ctypes.create_string_buffer(self.state_bytes())
        check(native.lib().spiir_bank_get_state(self._h, buf, len(buf)))
        return buf.raw

    def set_state(self, state: bytes) -> None:
        buf = ctypes.create_string_buffer(bytes(state), len(state))
        check(native.lib().spiir_bank_set_state(self._h, buf, len(state)))


def sky_tables(det_pos_m, arm_x, arm_y, sigma, nside: int, rate_hz: float):
    """Host FP64 per-pixel tables (delays [P][n_det] int32, u_sig [P][n_det][2], u_null [P][n_det][n_det-2])."""
    pos = np.ascontiguousarray(det_pos_m, dtype=np.float64)
    ax = np.ascontiguousarray(arm_x, dtype=np.float64)
    ay = np.ascontiguousarray(arm_y, dtype=np.float64)
    sg = np.ascontiguousarray(sigma, dtype=np.float64)
    nd = pos.shape[0]
    P = 12 * nside * nside
    delays = np.zeros((P, nd), dtype=np.int32)
    u_sig = np.zeros((P, nd, 2), dtype=np.float32)
    u_null = np.zeros((P, nd, max(nd - 2, 1)), dtype=np.float32)
    check(native.lib().spiir_sky_tables(nd, _host_ptr(pos), _host_ptr(ax), _host_ptr(ay), _host_ptr(sg), int(nside),
                                        float(rate_hz), _host_ptr(delays), _host_ptr(u_sig), _host_ptr(u_null)))
    return delays, u_sig, u_null[:, :, : max(nd - 2, 0)].copy()


class Sky:
    """Per-pixel coherent-scan tables on the device (spiir_sky_create)."""

    def __init__(self, delays, u_sig, u_null):
        L = native.lib()
        d = np.ascontiguousarray(delays, dtype=np.int32)
        us = np.ascontiguousarray(u_sig, dtype=np.float32)
        P, nd = d.shape
        un = np.ascontiguousarray(u_null, dtype=np.float32) if nd > 2 else np.zeros(1, dtype=np.float32)
        h = ctypes.c_void_p()
        check(L.spiir_sky_create(nd, P, _host_ptr(d), _host_ptr(us), _host_ptr(un), ctypes.byref(h)))
        self._h = h
        self.n_det = nd
        self.n_pix = P
        H = ctypes.c_int()
        check(L.spiir_sky_info(h, None, None, ctypes.byref(H)))
        self.halo = H.value

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            native.lib().spiir_sky_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_scan_shape(self, threads=256, pairs=2, table_in_shared=1):
        check(native.lib().spiir_sky_set_scan_shape(self._h, int(threads), int(pairs), int(table_in_shared)))

    def get_scan_shape(self):
        v = [ctypes.c_int() for _ in range(4)]
        check(native.lib().spiir_sky_get_scan_shape(self._h, *[ctypes.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def scan(self, snr, n: int, max_stat, argmax, null_stat, skymap=None, stream=None):
        """snr: complex64 CUDA tensor [T][n_det][pitch], entry H + k = output sample k.
        Outputs: float32 [T][n], int32 [T][n], float32 [T][n], optional float32 [T][P][n]."""
        import torch
        _require_cuda(snr, torch.complex64, "snr")
        T = snr.shape[0]
        for t, dt, nm in ((max_stat, torch.float32, "max_stat"), (argmax, torch.int32, "argmax"),
                          (null_stat, torch.float32, "null_stat")):
            _require_cuda(t, dt, nm)
            if not t.is_contiguous() or t.numel() < T * n:
                raise ValueError(f"{nm} must be contiguous with T*n elements")
        if skymap is not None:
            _require_cuda(skymap, torch.float32, "skymap")
            if not skymap.is_contiguous() or skymap.numel() < T * self.n_pix * n:
                raise ValueError("skymap must be contiguous [T][n_pix][n]")
        if snr.stride(2) != 1 or snr.stride(1) != snr.stride(0) // self.n_det:
            raise ValueError("snr rows must be contiguous [T][n_det][pitch]")
        check(native.lib().spiir_coherent_scan(self._h, _dev_ptr(snr), snr.stride(1), T, int(n), _dev_ptr(max_stat),
                                               _dev_ptr(argmax), _dev_ptr(null_stat),
                                               _dev_ptr(skymap) if skymap is not None else None,
                                               _stream_ptr(stream)))


class Pipeline:
    """Filter bank + SNR history + coherent scan per strain chunk (spiir_pipeline_*)."""

    def __init__(self, bank: Bank, sky: Sky, max_chunk: int):
        h = ctypes.c_void_p()
        check(native.lib().spiir_pipeline_create(bank.handle, sky.handle, int(max_chunk), ctypes.byref(h)))
        self._h = h
        self.bank = bank
        self.sky = sky
        self.max_chunk = int(max_chunk)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            native.lib().spiir_pipeline_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self, stream=None):
        check(native.lib().spiir_pipeline_reset(self._h, _stream_ptr(stream)))

    def run(self, strain, max_stat, argmax, null_stat, skymap=None, stream=None):
        import torch
        _require_cuda(strain, torch.float32, "strain")
        n = strain.shape[1]
        check(native.lib().spiir_pipeline_run(self._h, _dev_ptr(strain), strain.stride(0), n, _dev_ptr(max_stat),
                                              _dev_ptr(argmax), _dev_ptr(null_stat),
                                              _dev_ptr(skymap) if skymap is not None else None,
                                              _stream_ptr(stream)))

    def run_frontend(self, fe, strain, max_stat, argmax, null_stat, skymap=None, stream=None):
        """Raw strain at the front end's input rate, [n_det][n_in] float32 CUDA tensor: front end
        (down-sampling, whitening) then this pipeline's step, n = n_in / M (spiir_pipeline_run_frontend)."""
        import torch
        _require_cuda(strain, torch.float32, "strain")
        check(native.lib().spiir_pipeline_run_frontend(self._h, fe.handle, _dev_ptr(strain), strain.stride(0),
                                                       strain.shape[1], _dev_ptr(max_stat), _dev_ptr(argmax),
                                                       _dev_ptr(null_stat),
                                                       _dev_ptr(skymap) if skymap is not None else None,
                                                       _stream_ptr(stream)))

    def run_host(self, strain: np.ndarray, max_stat: np.ndarray, argmax: np.ndarray, null_stat: np.ndarray,
                 stream=None):
        """Host buffers (ideally page-locked): strain [n_det][n] float32 C-contiguous; outputs [T][n]."""
        for a, dt in ((strain, np.float32), (max_stat, np.float32), (argmax, np.int32), (null_stat, np.float32)):
            if a.dtype != dt or not a.flags.c_contiguous:
                raise ValueError("host buffers must be C-contiguous with the documented dtypes")
        n = strain.shape[1]
        check(native.lib().spiir_pipeline_run_host(self._h, _host_ptr(strain), n, _host_ptr(max_stat),
                                                   _host_ptr(argmax), _host_ptr(null_stat), _stream_ptr(stream)))

    def submit_host(self, strain: np.ndarray, max_stat: np.ndarray, argmax: np.ndarray, null_stat: np.ndarray,
                    stream=None):
        """Enqueue one chunk with host buffers and return; its outputs land in the host buffers
        by the next wait().  The buffers must stay alive and unread until then (page-locked for
        overlap)."""
        for a, dt in ((strain, np.float32), (max_stat, np.float32), (argmax, np.int32), (null_stat, np.float32)):
            if a.dtype != dt or not a.flags.c_contiguous:
                raise ValueError("host buffers must be C-contiguous with the documented dtypes")
        n = strain.shape[1]
        check(native.lib().spiir_pipeline_submit_host(self._h, _host_ptr(strain), n, _host_ptr(max_stat),
                                                      _host_ptr(argmax), _host_ptr(null_stat), _stream_ptr(stream)))

    def wait(self):
        check(native.lib().spiir_pipeline_wait(self._h))

    def wait_for(self, timeout_s: float) -> bool:
        """True once every submitted step is complete; False if timeout_s passed first (the
        steps keep running)."""
        rc = native.lib().spiir_pipeline_wait_for(self._h, float(timeout_s))
        if rc == native.ETIMEOUT:
            return False
        check(rc)
        return True


class Search:
    """Candidate-driven streaming search (spiir_search_*): per chunk, filter bank into an SNR
    ring, candidate selection, zero-lag scan on sky_fg, time-shift background on sky_bg and
    xi_C^2 at the candidates (Sec. II.C.1 - II.C.3).  A [T][2 n_lags + 1] complex64 CUDA tensor
    of the templates' autocorrelations.  Output tensors are allocated once and overwritten by
    every run(); rows past the count keep older values.  overlap=True: each run() analyses the
    span completed by the previous chunk on an internal stream while the new chunk is filtered
    (SPIIR_SEARCH_OVERLAP)."""

    OVERLAP = 1

    def __init__(self, bank: Bank, sky_fg: Sky, sky_bg: Sky, A, n_lags: int, chunk: int, threshold: float = 4.0,
                 per_second: int = 2048, n_shifts: int = 100, shift_step: int = 205, max_cand: int = 16384,
                 overlap: bool = False):
        import torch
        _require_cuda(A, torch.complex64, "A")
        h = ctypes.c_void_p()
        check(native.lib().spiir_search_create(bank.handle, sky_fg.handle, sky_bg.handle, _dev_ptr(A), int(n_lags),
                                               int(chunk), float(threshold), int(per_second), int(n_shifts),
                                               int(shift_step), int(max_cand), self.OVERLAP if overlap else 0,
                                               ctypes.byref(h)))
        self._h = h
        self.bank, self.sky_fg, self.sky_bg = bank, sky_fg, sky_bg
        self.chunk, self.n_shifts, self.max_cand = int(chunk), int(n_shifts), int(max_cand)
        dev = A.device
        m, s = max(1, max_cand), max(1, n_shifts)
        self.cand = torch.zeros((m, 4), dtype=torch.int32, device=dev)
        self.n_cand = torch.zeros(1, dtype=torch.int32, device=dev)
        self.fg = (torch.full((m,), float("nan"), device=dev), torch.full((m,), -1, dtype=torch.int32, device=dev),
                   torch.full((m,), float("nan"), device=dev), torch.full((m,), float("nan"), device=dev))
        self.bg = (torch.full((m, s), float("nan"), device=dev), torch.full((m, s), -1, dtype=torch.int32, device=dev),
                   torch.full((m, s), float("nan"), device=dev), torch.full((m, s), float("nan"), device=dev))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            native.lib().spiir_search_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        """(ring length L, history Hb, lag La, S0 of the next span) in samples."""
        v = [ctypes.c_int64() for _ in range(4)]
        check(native.lib().spiir_search_info(self._h, *[ctypes.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def reset(self, stream=None):
        check(native.lib().spiir_search_reset(self._h, _stream_ptr(stream)))

    def run(self, strain, stream=None):
        """strain [n_det][>= chunk] float32 CUDA tensor.  Returns S0, the stream sample of the
        span's sample 0; the results are in self.cand, self.n_cand, self.fg = (max, argmax,
        null, xi2) [max_cand] and self.bg = the same [max_cand][n_shifts]."""
        import torch
        _require_cuda(strain, torch.float32, "strain")
        s0 = ctypes.c_int64()
        bg = [_dev_ptr(t) for t in self.bg] if self.n_shifts > 0 else [None] * 4
        check(native.lib().spiir_search_run(self._h, _dev_ptr(strain), strain.stride(0), _dev_ptr(self.cand),
                                            _dev_ptr(self.n_cand), *[_dev_ptr(t) for t in self.fg], *bg,
                                            ctypes.byref(s0), _stream_ptr(stream)))
        return s0.value


class Batch:
    """Batched multirate banks (spiir_batch_*).  banks: list of (offsets, a1, b0, delay, band)
    host arrays, one per bank; band_factor: decimation factor of each band."""

    PLAIN, BATCHED, GRAPH = 0, 1, 2

    def __init__(self, n_det: int, banks, band_factor, sky: Sky, chunk: int):
        offs, a1s, b0s, ds, bs, tpb = [np.zeros(1, np.int64)], [], [], [], [], []
        for off, a1, b0, d, band in banks:
            off = np.asarray(off, np.int64)
            offs.append(offs[-1][-1] + off[1:])
            a1s.append(np.asarray(a1, np.complex64))
            b0s.append(np.asarray(b0, np.complex64))
            ds.append(np.asarray(d, np.int32))
            bs.append(np.asarray(band, np.int32))
            tpb.append(off.size - 1)
        off = np.ascontiguousarray(np.concatenate(offs))
        a1 = np.ascontiguousarray(np.concatenate(a1s)).view(np.float32)
        b0 = np.ascontiguousarray(np.concatenate(b0s)).view(np.float32)
        d = np.ascontiguousarray(np.concatenate(ds))
        band = np.ascontiguousarray(np.concatenate(bs))
        tpb = np.ascontiguousarray(tpb, np.int32)
        bf = np.ascontiguousarray(band_factor, np.int32)
        h = ctypes.c_void_p()
        check(native.lib().spiir_batch_create(int(n_det), len(tpb), _host_ptr(tpb), _host_ptr(off), _host_ptr(a1),
                                              _host_ptr(b0), _host_ptr(d), _host_ptr(band), int(bf.size), _host_ptr(bf),
                                              sky.handle, int(chunk), ctypes.byref(h)))
        self._h = h
        self.sky = sky
        self.n_det = int(n_det)
        self.chunk = int(chunk)
        self.n_templates = int(off.size - 1)
        self.templates_per_bank = tpb

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            native.lib().spiir_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        T, F, I = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int()
        check(native.lib().spiir_batch_info(self._h, ctypes.byref(T), ctypes.byref(F), ctypes.byref(I)))
        return T.value, F.value, I.value

    def reset(self, stream=None):
        check(native.lib().spiir_batch_reset(self._h, _stream_ptr(stream)))

    def set_shape(self, filters_per_lane=8, lanes_per_block=128, steps_per_reduce=32, blocks_per_sm=0):
        check(native.lib().spiir_batch_set_shape(self._h, int(filters_per_lane), int(lanes_per_block),
                                                 int(steps_per_reduce), int(blocks_per_sm)))

    def filter_time(self) -> float:
        """Device time (ms) of the last eager batched chunk's persistent filter launch; the
        first call arms the events and returns -1 (spiir_batch_filter_time)."""
        v = ctypes.c_float()
        check(native.lib().spiir_batch_filter_time(self._h, ctypes.byref(v)))
        return float(v.value)

    def run(self, strain, max_stat, argmax, null_stat, mode=GRAPH, stream=None):
        import torch
        _require_cuda(strain, torch.float32, "strain")
        if not strain.is_contiguous() or tuple(strain.shape) != (self.n_det, self.chunk):
            raise ValueError("strain must be a contiguous [n_det][chunk] tensor")
        check(native.lib().spiir_batch_run(self._h, int(mode), _dev_ptr(strain), _dev_ptr(max_stat),
                                           _dev_ptr(argmax), _dev_ptr(null_stat), _stream_ptr(stream)))


# ------------------------------------------------------------------------------------------------
# Signal-consistency statistic (spiir_autocorr, spiir_xi2, spiir_xi2_network)


def autocorr(u, n_lags: int, out=None, stream=None):
    """Template autocorrelation A [T][2 n_lags + 1] (complex64 CUDA tensor) of the responses
    u [T][n_resp] (complex64 CUDA tensor); entry n_lags + j is lag j."""
    import torch
    _require_cuda(u, torch.complex64, "u")
    if u.dim() != 2 or not u.is_contiguous():
        raise ValueError("u must be a contiguous [T][n_resp] tensor")
    T, nr = u.shape
    if out is None:
        out = torch.empty((T, 2 * n_lags + 1), dtype=torch.complex64, device=u.device)
    check(native.lib().spiir_autocorr(T, _dev_ptr(u), nr, int(n_lags), _dev_ptr(out), _stream_ptr(stream)))
    return out


def xi2(snr, A, n_lags: int, n: int, out=None, stream=None):
    """xi_I^2 [T][n_det][n] (float32 CUDA tensor) from snr [T][n_det][pitch] (complex64, entry
    n_lags + k = sample k) and A [T][2 n_lags + 1]."""
    import torch
    _require_cuda(snr, torch.complex64, "snr")
    _require_cuda(A, torch.complex64, "A")
    if snr.dim() != 3 or not snr.is_contiguous() or not A.is_contiguous():
        raise ValueError("snr must be a contiguous [T][n_det][pitch] tensor and A contiguous")
    T, n_det, pitch = snr.shape
    if out is None:
        out = torch.empty((T, n_det, n), dtype=torch.float32, device=snr.device)
    _require_cuda(out, torch.float32, "out")
    check(native.lib().spiir_xi2(T, n_det, _dev_ptr(snr), pitch, _dev_ptr(A), int(n_lags), int(n), _dev_ptr(out),
                                 out.shape[-1], _stream_ptr(stream)))
    return out


def xi2_network(sky, xi, argmax, n: int, out=None, stream=None):
    """xi_C^2 [T][n] from xi [T][n_det][pitch] (entry H + k = sample k, H = sky.halo) and the
    coherent scan's argmax [T][n]."""
    import torch
    _require_cuda(xi, torch.float32, "xi")
    _require_cuda(argmax, torch.int32, "argmax")
    T = xi.shape[0]
    if out is None:
        out = torch.empty((T, n), dtype=torch.float32, device=xi.device)
    check(native.lib().spiir_xi2_network(sky.handle, T, _dev_ptr(xi), xi.shape[-1], _dev_ptr(argmax), int(n),
                                         _dev_ptr(out), _stream_ptr(stream)))
    return out


class Selector:
    """Single-detector candidate selection (Sec. II.C.1) for spans of n samples of a bank of
    n_templates templates: owns the zeroed slot workspace and the record buffers.

    select() returns (cand, n_cand): cand [max_cand][4] int32 (detector, template, sample,
    bits of the FP32 |z|^2), n_cand a one-element int32 tensor holding the number found (above
    max_cand on overflow).  Both stay on the device; nothing is synchronised."""

    def __init__(self, n_templates: int, n_det: int, n: int, per_second: int = 2048, max_cand: int = 65536,
                 device="cuda"):
        import torch
        nb = ctypes.c_size_t()
        check(native.lib().spiir_select_workspace_bytes(n_templates, n_det, int(n), per_second, ctypes.byref(nb)))
        self.n_templates, self.n_det, self.n, self.per_second, self.max_cand = n_templates, n_det, int(n), per_second, max_cand
        self.workspace = torch.zeros(nb.value // 8, dtype=torch.int64, device=device)
        self.cand = torch.zeros((max(max_cand, 1), 4), dtype=torch.int32, device=device)
        self.n_cand = torch.zeros(1, dtype=torch.int32, device=device)

    def select(self, snr, offset: int, threshold: float = 4.0, stream=None):
        import torch
        _require_cuda(snr, torch.complex64, "snr")
        if snr.dim() != 3 or not snr.is_contiguous() or tuple(snr.shape[:2]) != (self.n_templates, self.n_det):
            raise ValueError("snr must be a contiguous [n_templates][n_det][pitch] tensor")
        check(native.lib().spiir_select_candidates(
            self.n_templates, self.n_det, _dev_ptr(snr), snr.shape[-1], int(offset), self.n, float(threshold),
            self.per_second, _dev_ptr(self.workspace), self.workspace.numel() * 8, _dev_ptr(self.cand),
            self.max_cand, _dev_ptr(self.n_cand), _stream_ptr(stream)))
        return self.cand, self.n_cand

    @staticmethod
    def records(cand, n_cand):
        """Host copy of the records as a list of (detector, template, sample, |z|^2), the last the
        FP32 value the selection stored (synchronises)."""
        n = min(int(n_cand.item()), cand.shape[0])
        c = cand[:n].cpu().numpy()
        m2 = c[:, 3].copy().view(np.float32)
        return [(int(a), int(b), int(k), float(v)) for (a, b, k), v in zip(c[:, :3], m2)]


def coherent_candidates(sky, snr, offset: int, cand, n_cand, first_shift: int = 0, n_shifts: int = 1,
                        shift_step: int = 205, out=None, stream=None):
    """Coherent statistic at the candidates (Sec. II.C.1) under time shifts
    first_shift .. first_shift + n_shifts - 1 of shift_step samples per companion detector
    (Sec. II.C.3).  snr [T][n_det][pitch] complex64 with entry offset + k = sample k; cand and
    n_cand as returned by Selector.select.  Returns (max, argmax, null), each
    [max_cand][n_shifts]; rows past the count are left as they were."""
    import torch
    _require_cuda(snr, torch.complex64, "snr")
    _require_cuda(cand, torch.int32, "cand")
    _require_cuda(n_cand, torch.int32, "n_cand")
    if snr.dim() != 3 or not snr.is_contiguous() or not cand.is_contiguous():
        raise ValueError("snr must be a contiguous [T][n_det][pitch] tensor and cand contiguous")
    m = cand.shape[0]
    if out is None:
        out = (torch.full((m, n_shifts), float("nan"), dtype=torch.float32, device=snr.device),
               torch.full((m, n_shifts), -1, dtype=torch.int32, device=snr.device),
               torch.full((m, n_shifts), float("nan"), dtype=torch.float32, device=snr.device))
    ms, am, nl = out
    check(native.lib().spiir_coherent_candidates(
        sky.handle, snr.shape[0], _dev_ptr(snr), snr.shape[-1], int(offset), _dev_ptr(cand), _dev_ptr(n_cand), m,
        int(first_shift), int(n_shifts), int(shift_step), _dev_ptr(ms), _dev_ptr(am), _dev_ptr(nl),
        _stream_ptr(stream)))
    return ms, am, nl


def fir_lowpass(n_taps: int, M: int, cutoff: float) -> np.ndarray:
    """Hann-windowed sinc low-pass for decimation by M (cutoff x the output Nyquist frequency,
    unit DC gain), designed in FP64 by the library; float32 [n_taps]."""
    h = np.empty(n_taps, dtype=np.float32)
    check(native.lib().spiir_fir_lowpass(int(n_taps), int(M), float(cutoff), _host_ptr(h)))
    return h


def whitening_kernel(psd, rate_hz: float, n_taps: int) -> np.ndarray:
    """Whitening FIR of Eq. (whiten) from the one-sided PSD psd[j] at f_j = j rate / N,
    N = 2 (len(psd) - 1): linear phase, odd length, unit-variance output; float32 [n_taps]."""
    psd = np.ascontiguousarray(psd, dtype=np.float64)
    w = np.empty(n_taps, dtype=np.float32)
    check(native.lib().spiir_whitening_kernel(psd.size, _host_ptr(psd), float(rate_hz), int(n_taps), _host_ptr(w)))
    return w


class Frontend:
    """Streaming down-sampling and whitening of n_det strain channels (Sec. II.A): decimation by
    M with the FIR dec_taps, then each detector's whitening FIR white_taps[I]."""

    def __init__(self, n_det: int, dec_taps, M: int, white_taps, max_in: int):
        dec_taps = np.ascontiguousarray(dec_taps, dtype=np.float32)
        white_taps = np.ascontiguousarray(white_taps, dtype=np.float32).reshape(n_det, -1)
        self.n_det, self.M = n_det, M
        h = ctypes.c_void_p()
        check(native.lib().spiir_frontend_create(n_det, M, dec_taps.size, _host_ptr(dec_taps), white_taps.shape[1],
                                                 _host_ptr(white_taps), int(max_in), ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            native.lib().spiir_frontend_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self, stream=None):
        check(native.lib().spiir_frontend_reset(self._h, _stream_ptr(stream)))

    def run(self, strain, out=None, stream=None):
        """strain [n_det][n_in] float32 CUDA tensor (n_in a multiple of M); returns (or fills)
        out [n_det][n_in / M]."""
        import torch
        _require_cuda(strain, torch.float32, "strain")
        if strain.dim() != 2 or strain.shape[0] != self.n_det or strain.stride(1) != 1:
            raise ValueError("strain must be [n_det][n] with unit stride along samples")
        n_in = strain.shape[1]
        if out is None:
            out = torch.empty((self.n_det, n_in // self.M), dtype=torch.float32, device=strain.device)
        _require_cuda(out, torch.float32, "out")
        if out.stride(1) != 1:
            raise ValueError("out must have unit stride along samples")
        check(native.lib().spiir_frontend_run(self._h, _dev_ptr(strain), strain.stride(0), n_in, _dev_ptr(out),
                                              out.stride(0), _stream_ptr(stream)))
        return out


def xi2_candidates(sky, snr, offset: int, A, n_lags: int, cand, n_cand, argmax, first_shift: int = 0,
                   n_shifts: int = 1, shift_step: int = 205, per_detector: bool = False, stream=None):
    """xi_C^2 [max_cand][n_shifts] at the candidates' coherent argmax pixels (argmax as written by
    coherent_candidates), with the same time shifts; also [max_cand][n_shifts][n_det] per detector
    when per_detector.  snr [T][n_det][pitch] complex64 (entry offset + k = sample k), A
    [T][2 n_lags + 1] complex64."""
    import torch
    _require_cuda(snr, torch.complex64, "snr")
    _require_cuda(A, torch.complex64, "A")
    _require_cuda(cand, torch.int32, "cand")
    _require_cuda(argmax, torch.int32, "argmax")
    if snr.dim() != 3 or not snr.is_contiguous() or not A.is_contiguous() or not argmax.is_contiguous():
        raise ValueError("snr [T][n_det][pitch], A and argmax must be contiguous")
    m = cand.shape[0]
    xi = torch.full((m, n_shifts), float("nan"), dtype=torch.float32, device=snr.device)
    xd = torch.full((m, n_shifts, snr.shape[1]), float("nan"), dtype=torch.float32, device=snr.device) \
        if per_detector else None
    check(native.lib().spiir_xi2_candidates(
        sky.handle, snr.shape[0], _dev_ptr(snr), snr.shape[-1], int(offset), _dev_ptr(A), int(n_lags), _dev_ptr(cand),
        _dev_ptr(n_cand), m, int(first_shift), int(n_shifts), int(shift_step), _dev_ptr(argmax), _dev_ptr(xi),
        _dev_ptr(xd) if xd is not None else None, _stream_ptr(stream)))
    return (xi, xd) if per_detector else xi
