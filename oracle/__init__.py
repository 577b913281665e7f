"""FP64 CPU oracle for the SPIIR hot path (arxiv 2011.06787).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg import this package.  The product library never
imports it and shares no code with it; the only common module is ``synth``,
which draws seeded inputs and holds none of the method's arithmetic.

Contents, each a plain restatement of the paper in double precision:

* ``filter_bank``        Sec. II.B.1 Eq. (zk), per-filter reading (C, spiir_oracle.c)
* ``healpix_centres``    HEALPix RING pixel centres (Sec. II.C.1, 3072-tile sky grid;
                         ring geometry of Gorski et al. 2005)
* ``antenna_patterns``   App. A Eq. (strain_sngl): F+ and Fx of each detector, psi = 0
* ``arrival_delays``     integer light-travel offsets of the SNR series (Sec. II.C.1)
* ``g_sigma``            App. A Eq. (svd): noise-weighted antenna matrix
* ``coherent``           Sec. II.C.1 Eq. (llr_form) by the projector Pi = G (G^T G)^-1 G^T,
                         and Eq. (null_def) (C, spiir_oracle.c)
* ``llr_bruteforce``     App. A Eqs. (llr_def), (llr_extend): direct numerical maximisation
                         of the network log likelihood over A_c, A_s
* ``impulse_forward`` / ``impulse_backward``  bank impulse response and its adjoint
* ``overlap_loss``       1 - O with O from Sec. II.B.1 Eq. (overlap) (modulus reading)
* ``fir_taps`` / ``decimate`` / ``upsample_linear`` / ``multirate_bank``
                         multirate split of the bank (not in the paper; its definition is
                         stated in the docstrings below)
* ``autocorr`` / ``xi2`` / ``xi2_network``  Sec. II.C.2: template autocorrelation, xi_I^2 per
                         sample, network average at the coherent argmax
* ``select_candidates`` / ``coherent_points`` / ``background_shifts``  Sec. II.C.1 and II.C.3:
                         single-detector candidates, the coherent statistic at them, time shifts
* ``lowpass_taps`` / ``whitening_kernel`` / ``fir`` / ``frontend``  Sec. II.A: 16384 -> 2048 Hz
                         FIR down-sampling and whitening (Eq. (whiten)) as a time-domain FIR

The multirate split (``fir_taps``, ``decimate``, ``upsample_linear``, ``multirate_bank``) is
defined here, not by the paper.  Its pins are the library routines each step reduces to
(scipy ``firwin`` and the Hann window for the taps, ``upfirdn`` for the decimation, numpy
``interp`` for the upsampling, ``lfilter`` for the one-pole filters of a band) and identities
(M = 1 is the identity, unit DC gain, exact reproduction of ramps).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spiir_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None

C_LIGHT = 299792458.0


def build(force: bool = False) -> str:
    """Compile spiir_oracle.c with gcc (OpenMP over templates)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", _SRC,
                               "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        lib.oracle_filter_bank.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P, P, P, i64, i64, P, P]
        lib.oracle_filter_bank.restype = ctypes.c_int
        lib.oracle_coherent.argtypes = [ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int, P, i64, i64,
                                        i64, P, P, P, P]
        lib.oracle_coherent.restype = ctypes.c_int
        lib.oracle_impulse_forward.argtypes = [ctypes.c_int, P, P, P, P, P, i64, P, P]
        lib.oracle_impulse_forward.restype = None
        lib.oracle_impulse_backward.argtypes = [ctypes.c_int, P, P, P, P, P, i64, P, P, P, P]
        lib.oracle_impulse_backward.restype = ctypes.c_int
        lib.oracle_coherent_points.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P, i64, i64, P, P, P, P, P]
        lib.oracle_coherent_points.restype = ctypes.c_int
        lib.oracle_autocorr.argtypes = [ctypes.c_int, P, i64, ctypes.c_int, P]
        lib.oracle_autocorr.restype = None
        lib.oracle_xi2.argtypes = [ctypes.c_int, ctypes.c_int, P, i64, P, ctypes.c_int, i64, P]
        lib.oracle_xi2.restype = None
        _lib = lib
    return _lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def set_threads(n: int) -> None:
    """Number of OpenMP threads the C oracle uses (must be called before its first use)."""
    os.environ["OMP_NUM_THREADS"] = str(int(n))


# --------------------------------------------------------------------------------------------
# Filter bank: Sec. II.B.1 Eq. (zk), per-filter reading


def filter_bank(x, offsets, a1, b0, delay, state=None, history=None):
    """Run the bank over one stream segment.

    x        [n_det][n] real or complex samples of this segment
    history  [n_det][D] the D samples preceding the segment (zeros at stream start)
    state    [n_det][F] complex y_l[-1] (zeros at stream start); returned updated
    Returns (z [T][n_det][n] complex128, new_state, new_history).
    """
    lib = _load()
    x = np.asarray(x)
    n_det, n = x.shape
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    T = offsets.size - 1
    F = int(offsets[-1])
    a1 = np.ascontiguousarray(a1, dtype=np.complex128)
    b0 = np.ascontiguousarray(b0, dtype=np.complex128)
    delay = np.ascontiguousarray(delay, dtype=np.int32)
    D = int(delay.max()) if F else 0
    if history is None:
        history = np.zeros((n_det, D))
    history = np.asarray(history)
    D = max(D, history.shape[1])
    hist = np.zeros((n_det, D), dtype=np.complex128)
    if history.shape[1]:
        hist[:, D - history.shape[1]:] = history
    xx = np.ascontiguousarray(np.concatenate([hist, x.astype(np.complex128)], axis=1))
    st = np.zeros((n_det, F), dtype=np.complex128) if state is None else \
        np.ascontiguousarray(state, dtype=np.complex128).copy()
    z = np.zeros((T, n_det, n), dtype=np.complex128)
    rc = lib.oracle_filter_bank(n_det, T, _ptr(offsets), _ptr(a1), _ptr(b0), _ptr(delay), _ptr(xx), D, n,
                                _ptr(st), _ptr(z))
    if rc != 0:
        raise ValueError(f"oracle_filter_bank failed ({rc})")
    return z, st, xx[:, -D:] if D else xx[:, :0]


# --------------------------------------------------------------------------------------------
# Sky grid and detector geometry (Sec. II.C.1; App. A)


def healpix_centres(nside: int) -> np.ndarray:
    """Unit vectors of the 12 nside^2 HEALPix pixel centres in RING order.

    Rings are numbered from the north pole.  Ring i (1 <= i <= 4 nside - 1) has
    z = 1 - i^2 / (3 nside^2) in the north polar cap (i < nside), z = 4/3 - 2 i / (3 nside)
    in the equatorial belt (nside <= i <= 3 nside) and the mirror image in the south cap.
    A cap ring at distance i from its pole holds 4 i pixels at phi = (j + 1/2) pi / (2 i),
    j = 0..4i-1; a belt ring holds 4 nside pixels at phi = (j + s/2) pi / (2 nside) with
    s = 1 when i - nside is even and s = 0 otherwise.  Pixels are numbered ring by ring,
    north to south, with increasing phi inside a ring.
    """
    ns = int(nside)
    out = []
    for i in range(1, 4 * ns):
        if i < ns:  # north cap
            z = 1.0 - i * i / (3.0 * ns * ns)
            m = 4 * i
            phis = [(j + 0.5) * math.pi / (2 * i) for j in range(m)]
        elif i <= 3 * ns:  # belt
            z = 4.0 / 3.0 - 2.0 * i / (3.0 * ns)
            s = 1 if (i - ns) % 2 == 0 else 0
            phis = [(j + 0.5 * s) * math.pi / (2 * ns) for j in range(4 * ns)]
        else:  # south cap, ring at distance ii from the south pole
            ii = 4 * ns - i
            z = -(1.0 - ii * ii / (3.0 * ns * ns))
            phis = [(j + 0.5) * math.pi / (2 * ii) for j in range(4 * ii)]
        st = math.sqrt(max(0.0, 1.0 - z * z))
        for ph in phis:
            out.append((st * math.cos(ph), st * math.sin(ph), z))
    return np.asarray(out, dtype=np.float64)


def antenna_patterns(arm_x, arm_y, nhat, psi: float = 0.0):
    """F+ and Fx of each detector for each source direction and polarisation angle psi.

    Detector tensor D = (X X^T - Y Y^T) / 2 from the unit arm vectors.  For a source in
    direction nhat = (sin th cos ph, sin th sin ph, cos th) the polarisation basis is
    e_x = e_theta, e_y = -e_phi (right-handed about the propagation direction -nhat),
    e+ = e_x e_x^T - e_y e_y^T, ex = e_x e_y^T + e_y e_x^T, and F+ = D : e+, Fx = D : ex.
    A polarisation angle psi turns (e_x, e_y) by psi about nhat before the contraction.
    Returns arrays [P][n_det] each.
    """
    arm_x = np.asarray(arm_x, dtype=np.float64)
    arm_y = np.asarray(arm_y, dtype=np.float64)
    nhat = np.asarray(nhat, dtype=np.float64)
    th = np.arccos(np.clip(nhat[:, 2], -1.0, 1.0))
    ph = np.arctan2(nhat[:, 1], nhat[:, 0])
    e_th = np.stack([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)], axis=1)
    e_ph = np.stack([-np.sin(ph), np.cos(ph), np.zeros_like(ph)], axis=1)
    ex = math.cos(psi) * e_th - math.sin(psi) * e_ph
    ey = -math.sin(psi) * e_th - math.cos(psi) * e_ph
    Fp = np.empty((nhat.shape[0], arm_x.shape[0]))
    Fc = np.empty_like(Fp)
    for I in range(arm_x.shape[0]):
        Dt = 0.5 * (np.outer(arm_x[I], arm_x[I]) - np.outer(arm_y[I], arm_y[I]))
        for p in range(nhat.shape[0]):
            ep = np.outer(ex[p], ex[p]) - np.outer(ey[p], ey[p])
            ec = np.outer(ex[p], ey[p]) + np.outer(ey[p], ex[p])
            Fp[p, I] = np.sum(Dt * ep)
            Fc[p, I] = np.sum(Dt * ec)
    return Fp, Fc


def arrival_delays(pos_m, nhat, rate_hz: float) -> np.ndarray:
    """Integer sample offsets Delta_I(p) = round(-rate * nhat . r_I / c), half away from zero.

    A detector displaced towards the source sees the wavefront earlier, so the SNR of
    detector I for geocentric sample k is read at k + Delta_I.  Returns [P][n_det] int32.
    """
    pos_m = np.asarray(pos_m, dtype=np.float64)
    nhat = np.asarray(nhat, dtype=np.float64)
    out = np.empty((nhat.shape[0], pos_m.shape[0]), dtype=np.int32)
    for p in range(nhat.shape[0]):
        for I in range(pos_m.shape[0]):
            v = -rate_hz * float(np.dot(nhat[p], pos_m[I])) / C_LIGHT
            out[p, I] = int(math.floor(abs(v) + 0.5)) * (1 if v >= 0 else -1)
    return out


def g_sigma(Fp, Fc, sigma) -> np.ndarray:
    """App. A Eq. (svd): rows (G+_I sigma_I, Gx_I sigma_I); returns [P][n_det][2]."""
    sigma = np.asarray(sigma, dtype=np.float64)
    return np.stack([Fp * sigma[None, :], Fc * sigma[None, :]], axis=2)


def sky_geometry(det, sigma, nside: int, rate_hz: float):
    """(nhat [P][3], G [P][n_det][2], delays [P][n_det]) for a detector network."""
    nhat = healpix_centres(nside)
    Fp, Fc = antenna_patterns(det.arm_x, det.arm_y, nhat)
    return nhat, g_sigma(Fp, Fc, sigma), arrival_delays(det.pos_m, nhat, rate_hz)


# --------------------------------------------------------------------------------------------
# Coherent statistic: Sec. II.C.1 Eq. (llr_form), Eq. (null_def)


def coherent(z, G, delays, H: int, n: int, skymap: bool = False):
    """Coherent scan of SNR series z [T][n_det][pitch]; output sample k reads z_I[H + k + Delta_I(p)].

    Returns (max_stat [T][n], argmax [T][n] int32, null at argmax [T][n], skymap [T][n][P] or None).
    """
    lib = _load()
    z = np.ascontiguousarray(z, dtype=np.complex128)
    T, n_det, pitch = z.shape
    G = np.ascontiguousarray(G, dtype=np.float64)
    delays = np.ascontiguousarray(delays, dtype=np.int32)
    P = G.shape[0]
    ms = np.zeros((T, n), dtype=np.float64)
    am = np.zeros((T, n), dtype=np.int32)
    nl = np.zeros((T, n), dtype=np.float64)
    sm = np.zeros((T, n, P), dtype=np.float64) if skymap else None
    rc = lib.oracle_coherent(n_det, P, _ptr(G), _ptr(delays), T, _ptr(z), pitch, H, n, _ptr(ms), _ptr(am),
                             _ptr(nl), _ptr(sm))
    if rc != 0:
        raise ValueError(f"oracle_coherent failed ({rc})")
    return ms, am, nl, sm


def llr_bruteforce(w, G):
    """Maximum over A_c, A_s of the network log likelihood ratio, App. A Eq. (llr_extend).

    With the matched-filter outputs of the two quadratures w_c = Re w, w_s = Im w
    (normalised so that (h_x | h_x) = 1 per unit of G), the LLR for amplitudes A_x is
    sum_x [ (G A_x)^T w_x - |G A_x|^2 / 2 ].  It is maximised here numerically
    (Nelder-Mead from the origin, then polished), with no closed form used.
    """
    from scipy.optimize import minimize
    w = np.asarray(w, dtype=np.complex128)
    G = np.asarray(G, dtype=np.float64)
    wc, ws = w.real, w.imag

    def neg(A):
        ac, as_ = A[:2], A[2:]
        gc, gs = G @ ac, G @ as_
        return -((gc @ wc - 0.5 * gc @ gc) + (gs @ ws - 0.5 * gs @ gs))

    best = None
    for start in (np.zeros(4), np.ones(4), -np.ones(4)):
        r = minimize(neg, start, method="Nelder-Mead",
                     options=dict(xatol=1e-12, fatol=1e-14, maxiter=40000, maxfev=40000))
        r = minimize(neg, r.x, method="BFGS", options=dict(gtol=1e-12))
        if best is None or r.fun < best.fun:
            best = r
    return -best.fun


# --------------------------------------------------------------------------------------------
# Impulse response and its adjoint


def impulse_forward(offsets, a1, b0, delay, s0, n: int, return_end: bool = False):
    """u_t[k] = sum_l y_l[k], y_l[-1] = s_l, y_l[k] = a1 y_l[k-1] + b0 [k == d_l]; [T][n] complex128."""
    lib = _load()
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    T = offsets.size - 1
    a1 = np.ascontiguousarray(a1, dtype=np.complex128)
    b0 = np.ascontiguousarray(b0, dtype=np.complex128)
    s0 = np.ascontiguousarray(s0, dtype=np.complex128)
    delay = np.ascontiguousarray(delay, dtype=np.int32)
    u = np.zeros((T, n), dtype=np.complex128)
    yend = np.zeros(a1.shape[0], dtype=np.complex128) if return_end else None
    lib.oracle_impulse_forward(T, _ptr(offsets), _ptr(a1), _ptr(b0), _ptr(delay), _ptr(s0), n, _ptr(u),
                               _ptr(yend))
    return (u, yend) if return_end else u


def impulse_backward(offsets, a1, b0, delay, s0, g):
    """Adjoint of impulse_forward for gradient g = dL/dRe u + i dL/dIm u; returns (g_a1, g_b0, g_s0)."""
    lib = _load()
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    T = offsets.size - 1
    g = np.ascontiguousarray(g, dtype=np.complex128)
    n = g.shape[1]
    a1 = np.ascontiguousarray(a1, dtype=np.complex128)
    b0 = np.ascontiguousarray(b0, dtype=np.complex128)
    s0 = np.ascontiguousarray(s0, dtype=np.complex128)
    delay = np.ascontiguousarray(delay, dtype=np.int32)
    ga = np.zeros_like(a1)
    gb = np.zeros_like(b0)
    gs = np.zeros_like(s0)
    rc = lib.oracle_impulse_backward(T, _ptr(offsets), _ptr(a1), _ptr(b0), _ptr(delay), _ptr(s0), n, _ptr(g),
                                     _ptr(ga), _ptr(gb), _ptr(gs))
    if rc != 0:
        raise MemoryError("oracle_impulse_backward")
    return ga, gb, gs


def overlap_loss(h, u):
    """L = 1 - |sum conj(h) u| / (|h| |u|) per row (Sec. II.B.1 Eq. (overlap), modulus reading).

    Returns (L [T], g [T][n]) with g = dL/dRe u + i dL/dIm u = -O (h / conj(c) - u / |u|^2),
    c = sum conj(h) u.
    """
    h = np.asarray(h, dtype=np.complex128)
    u = np.asarray(u, dtype=np.complex128)
    c = np.sum(np.conj(h) * u, axis=-1)
    nh = np.sqrt(np.sum(np.abs(h) ** 2, axis=-1))
    nu2 = np.sum(np.abs(u) ** 2, axis=-1)
    O = np.abs(c) / (nh * np.sqrt(nu2))
    g = -O[..., None] * (h / np.conj(c)[..., None] - u / nu2[..., None])
    return 1.0 - O, g


# --------------------------------------------------------------------------------------------
# Multirate split (not in the paper): decimate, run band filters, upsample and sum


def fir_taps(M: int, ntaps: int = 32) -> np.ndarray:
    """Causal Hann-windowed sinc low-pass for decimation by M, cutoff 0.8 x output Nyquist,
    unit DC gain.  h[i], i = 0..ntaps-1, centred at (ntaps-1)/2."""
    if M == 1:
        h = np.zeros(ntaps)
        h[0] = 1.0
        return h
    fc = 0.8 * 0.5 / M  # cycles per input sample
    i = np.arange(ntaps, dtype=np.float64)
    c = (ntaps - 1) / 2.0
    arg = 2.0 * fc * (i - c)
    s = np.array([2.0 * fc * (math.sin(math.pi * a) / (math.pi * a) if a != 0 else 1.0) for a in arg])
    win = 0.5 - 0.5 * np.cos(2.0 * math.pi * (i + 0.5) / ntaps)
    h = s * win
    return h / h.sum()


def decimate(x, M: int, taps=None, history=None):
    """x_b[j] = sum_i h[i] x[j M - i] over one segment (len(x) a multiple of M).

    history: the len(h)-1 input samples before the segment (zeros at stream start).
    M = 1 returns x unchanged.  Returns (x_b, new_history)."""
    x = np.asarray(x, dtype=np.float64)
    if M == 1:
        return x.copy(), None
    h = fir_taps(M) if taps is None else np.asarray(taps, dtype=np.float64)
    L = h.size
    hist = np.zeros(x.shape[:-1] + (L - 1,)) if history is None else np.asarray(history, dtype=np.float64)
    xx = np.concatenate([hist, x], axis=-1)
    n = x.shape[-1]
    assert n % M == 0
    out = np.zeros(x.shape[:-1] + (n // M,))
    for j in range(n // M):
        k = j * M + (L - 1)  # index of x[jM] in xx
        for i in range(L):
            out[..., j] += h[i] * xx[..., k - i]
    return out, xx[..., -(L - 1):]


def upsample_linear(zb, M: int, prev=None):
    """z[k] = (1 - w) zb[m - 1] + w zb[m], m = floor(k / M), w = (k mod M) / M, zb[-1] = prev.

    One low-rate sample of lag; M = 1 returns zb.  Returns (z, last low-rate sample)."""
    zb = np.asarray(zb, dtype=np.complex128)
    if M == 1:
        return zb.copy(), None
    p = np.zeros(zb.shape[:-1], dtype=np.complex128) if prev is None else np.asarray(prev, dtype=np.complex128)
    nb = zb.shape[-1]
    out = np.zeros(zb.shape[:-1] + (nb * M,), dtype=np.complex128)
    for k in range(nb * M):
        m, r = divmod(k, M)
        lo = zb[..., m - 1] if m > 0 else p
        out[..., k] = (1.0 - r / M) * lo + (r / M) * zb[..., m]
    return out, zb[..., -1]


def multirate_bank(x, offsets, a1, b0, delay, band, factors):
    """Whole-stream multirate response: z_t = sum_b upsample_M_b( bank_b( decimate_M_b(x) ) ).

    band[l] selects factors[band[l]] for filter l (delays in samples of that band).
    Returns z [T][n_det][n] complex128."""
    x = np.asarray(x, dtype=np.float64)
    n_det, n = x.shape
    offsets = np.asarray(offsets, dtype=np.int64)
    T = offsets.size - 1
    z = np.zeros((T, n_det, n), dtype=np.complex128)
    band = np.asarray(band)
    for b, M in enumerate(factors):
        xb, _ = decimate(x, M)
        sel_off = [0]
        idx = []
        for t in range(T):
            ls = [l for l in range(offsets[t], offsets[t + 1]) if band[l] == b]
            idx.extend(ls)
            sel_off.append(len(idx))
        if not idx:
            continue
        idx = np.asarray(idx)
        zb, _, _ = filter_bank(xb, np.asarray(sel_off), np.asarray(a1)[idx], np.asarray(b0)[idx],
                               np.asarray(delay)[idx])
        up, _ = upsample_linear(zb, M)
        z += up
    return z


# --------------------------------------------------------------------------------------------
# Signal consistency: Sec. II.C.2


def autocorr(u, Nj: int):
    """A[t][Nj + j] = R[j] / R[0], R[j] = sum_k conj(u_t[k]) u_t[k + j], A[-j] = conj(A[j]);
    u [T][nr] complex.  Returns [T][2 Nj + 1] complex128."""
    lib = _load()
    u = np.ascontiguousarray(u, dtype=np.complex128)
    T, nr = u.shape
    A = np.zeros((T, 2 * Nj + 1), dtype=np.complex128)
    lib.oracle_autocorr(T, _ptr(u), nr, int(Nj), _ptr(A))
    return A


def xi2(z, A, Nj: int, n: int):
    """xi^2[t][I][k] = sum_{|j| <= Nj} |z[k + j] - z[k] A[j]|^2 / sum_{|j| <= Nj} (2 - 2 |A[j]|^2)
    for z [T][n_det][pitch] with entry Nj + k = sample k and A [T][2 Nj + 1]."""
    lib = _load()
    z = np.ascontiguousarray(z, dtype=np.complex128)
    A = np.ascontiguousarray(A, dtype=np.complex128)
    T, n_det, pitch = z.shape
    if pitch < n + 2 * Nj:
        raise ValueError("z holds fewer than n + 2 Nj samples")
    out = np.zeros((T, n_det, n), dtype=np.float64)
    lib.oracle_xi2(T, n_det, _ptr(z), pitch, _ptr(A), int(Nj), n, _ptr(out))
    return out


def xi2_network(xi, delays, argmax, H: int):
    """xi_C^2[t][k] = (1 / N_d) sum_I xi_I^2 at the detector's sample k + Delta_I(p), p the
    argmax pixel of (t, k) (Sec. II.C.2); xi [T][n_det][pitch] with entry H + k = sample k."""
    xi = np.asarray(xi, dtype=np.float64)
    delays = np.asarray(delays)
    argmax = np.asarray(argmax)
    T, n_det, _ = xi.shape
    n = argmax.shape[1]
    out = np.zeros((T, n), dtype=np.float64)
    for t in range(T):
        for k in range(n):
            d = delays[argmax[t, k]]
            out[t, k] = sum(xi[t, I, H + k + d[I]] for I in range(n_det)) / n_det
    return out


# --------------------------------------------------------------------------------------------
# Candidate selection and the candidate-driven scan: Sec. II.C.1; background: Sec. II.C.3


def select_candidates(z, off: int, n: int, threshold: float = 4.0, per_second: int = 2048):
    """Single-detector candidates of one bank (Sec. II.C.1): for every detector and sample, the
    largest |z| over the bank's templates (the lowest template among equals); samples where it
    exceeds the threshold are candidates of that template; a template keeps only its largest
    candidate per second (the earliest among equals).  z [T][n_det][pitch], entry off + k =
    sample k; the n samples are split into seconds of per_second samples from sample 0.

    Every comparison is made on |z|^2 in FP32, re*re + im*im with each operation rounded, against
    threshold^2 rounded the same way (the values the GPU decides on; equal values are equal on
    both sides).  Returns a list of (detector, template, sample, |z|^2) sorted by detector, then
    template, then second; |z|^2 is that FP32 value."""
    z = np.asarray(z)
    T, n_det, _ = z.shape
    thr2 = np.float32(threshold) * np.float32(threshold)
    out = []
    for I in range(n_det):
        w = z[:, I, off: off + n].astype(np.complex64)
        re, im = w.real.astype(np.float32), w.imag.astype(np.float32)
        m2 = re * re + im * im                          # [T][n] float32
        best_t = np.argmax(m2, axis=0)                  # first (lowest) template among equals
        best = m2[best_t, np.arange(n)]
        kept = {}                                       # (template, second) -> sample
        for k in np.flatnonzero(best > thr2):           # ascending: the earliest stays on ties
            key = (int(best_t[k]), int(k) // per_second)
            if key not in kept or best[k] > best[kept[key]]:
                kept[key] = int(k)
        for (t, _), k in sorted(kept.items()):
            out.append((I, t, k, float(best[k])))
    return out


def coherent_points(z, G, delays, pts, shifts):
    """Coherent statistic at points (template, reference detector, buffer entry of its sample)
    with per-detector extra offsets; see oracle_coherent_points.  Returns (max, argmax, null)."""
    lib = _load()
    z = np.ascontiguousarray(z, dtype=np.complex128)
    G = np.ascontiguousarray(G, dtype=np.float64)
    delays = np.ascontiguousarray(delays, dtype=np.int32)
    pts = np.ascontiguousarray(pts, dtype=np.int64).reshape(-1, 3)
    shifts = np.ascontiguousarray(shifts, dtype=np.int64).reshape(pts.shape[0], -1)
    T, n_det, pitch = z.shape
    m = pts.shape[0]
    ms = np.zeros(m)
    am = np.zeros(m, dtype=np.int32)
    nl = np.zeros(m)
    rc = lib.oracle_coherent_points(n_det, G.shape[0], _ptr(G), _ptr(delays), _ptr(z), pitch, m, _ptr(pts),
                                    _ptr(shifts), _ptr(ms), _ptr(am), _ptr(nl))
    if rc != 0:
        raise ValueError(f"oracle_coherent_points failed ({rc})")
    return ms, am, nl


def background_shifts(ref: int, n_det: int, s: int, step: int):
    """Offsets of time shift s (Sec. II.C.3): the reference detector is unshifted and the c-th
    other detector (c = 1, 2, ...) is read s c step samples earlier."""
    out = np.zeros(n_det, dtype=np.int64)
    c = 0
    for J in range(n_det):
        if J != ref:
            c += 1
            out[J] = -s * c * step
    return out


# --------------------------------------------------------------------------------------------
# Front end (Sec. II.A): FIR down-sampling 16384 -> 2048 Hz and whitening, Eq. (whiten), in the
# time domain


def lowpass_taps(ntaps: int, M: int, cutoff: float) -> np.ndarray:
    """Causal Hann-windowed sinc low-pass for decimation by M: cutoff at cutoff x the output
    Nyquist frequency (cycles per input sample fc = cutoff / (2 M)), unit DC gain.
    h[i], i = 0..ntaps-1, centred at (ntaps - 1) / 2."""
    fc = cutoff * 0.5 / M
    c = (ntaps - 1) / 2.0
    h = np.zeros(ntaps)
    for i in range(ntaps):
        a = 2.0 * fc * (i - c)
        sinc = math.sin(math.pi * a) / (math.pi * a) if a != 0 else 1.0
        h[i] = 2.0 * fc * sinc * (0.5 - 0.5 * math.cos(2.0 * math.pi * (i + 0.5) / ntaps))
    return h / h.sum()


def whitening_kernel(psd, rate_hz: float, ntaps: int, window: bool = True) -> np.ndarray:
    """Time-domain whitening filter of Eq. (whiten): the zero-phase response
    A(f) = sqrt(2 / (f_s S_n(f))) (unit-variance output for noise of one-sided PSD S_n), as a
    causal linear-phase FIR of odd length L = 2K + 1 with delay K.

    psd[j] is S_n at f_j = j f_s / N, j = 0 .. N/2 (N = 2 (len(psd) - 1)); L < N.  The
    impulse response of A on the N-point grid is
        a[m] = (1/N) [A_0 + (-1)^m A_{N/2} + 2 sum_{j=1}^{N/2-1} A_j cos(2 pi j m / N)],
    and w[i] = win[i] a[i - K] with the Hann window win[i] = 1/2 - 1/2 cos(2 pi (i+1) / (L+1))
    (win[K] = 1; window=False keeps a[i - K] unwindowed)."""
    psd = np.asarray(psd, dtype=np.float64)
    N = 2 * (psd.size - 1)
    if ntaps % 2 != 1 or ntaps >= N:
        raise ValueError("ntaps must be odd and below 2 (len(psd) - 1)")
    A = np.sqrt(2.0 / (rate_hz * psd))
    K = ntaps // 2
    w = np.zeros(ntaps)
    for i in range(ntaps):
        m = i - K
        acc = A[0] + (-1.0) ** (m % 2) * A[N // 2]
        for j in range(1, N // 2):
            acc += 2.0 * A[j] * math.cos(2.0 * math.pi * j * m / N)
        win = 0.5 - 0.5 * math.cos(2.0 * math.pi * (i + 1) / (ntaps + 1)) if window else 1.0
        w[i] = win * acc / N
    return w


def fir(x, h, history=None):
    """Causal FIR y[k] = sum_j h[j] x[k - j] over one segment of each row of x (FP64).
    history: the len(h) - 1 samples before the segment (zeros at stream start).
    Returns (y, new_history)."""
    x = np.asarray(x, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    L = h.size
    hist = np.zeros(x.shape[:-1] + (L - 1,)) if history is None else np.asarray(history, dtype=np.float64)
    xx = np.concatenate([hist, x], axis=-1)
    n = x.shape[-1]
    y = np.convolve(xx, h)[L - 1: L - 1 + n] if x.ndim == 1 else \
        np.stack([np.convolve(r, h)[L - 1: L - 1 + n] for r in xx])
    return y, xx[..., xx.shape[-1] - (L - 1):]


def frontend(x16, dec_taps, M: int, white_taps, hist16=None, hist2=None):
    """Front end of one segment (Sec. II.A): each detector's strain at the input rate is
    low-passed and decimated by M (decimate: x_2[j] = sum_i h[i] x[j M - i]), then whitened by
    its own causal FIR (fir with white_taps[I]).  Returns (y [n_det][n / M], hist16, hist2),
    the histories to pass with the next segment."""
    x16 = np.asarray(x16, dtype=np.float64)
    x2, h16 = decimate(x16, M, dec_taps, hist16)
    white_taps = np.asarray(white_taps, dtype=np.float64)
    ys, hs = [], []
    for I in range(x16.shape[0]):
        y, h = fir(x2[I], white_taps[I], None if hist2 is None else hist2[I])
        ys.append(y)
        hs.append(h)
    return np.stack(ys), h16, np.stack(hs)
