"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module draws random numbers and builds input arrays; it holds none of the
SPIIR arithmetic (no filtering, no antenna patterns, no delays, no coherent
statistic).  Every draw is made in FP64 by NumPy's PCG64 and then rounded to
FP32 where the hot path takes FP32; the FP32 values are the canonical inputs
for both the CUDA path and the FP64 oracle.

Workloads (the paper's O2 data and LVC template banks are not available, so
these synthetic recipes stand in for them):

* ``tiny``      2 detectors, 32768 samples of white noise at 2048 Hz, one bank
                of 4 templates x 64 filters, HEALPix nside 4, unit noise weights.
* ``online``    3 detectors, 2048 Hz noise in 1 s chunks, 1024 templates with
                200..900 filters each, delays up to 2 s, nside 16, noise
                weights uniform in [0.5, 2].
* ``multirate`` 8 banks of uneven size over bands at 2048/512/128 Hz.
* ``chirp``     Newtonian complex chirps used as targets for the adjoint.

Filter coefficients follow one recipe: |a1| uniform in [0.9, 0.999] with a
uniform phase, b0 complex normal (unit variance) scaled by 1/sqrt(F), integer
delay uniform in [0, d_max].
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 20110678
EARTH_RADIUS_M = 6371.0e3

# stream identifiers: one independent PCG64 stream per purpose
_STREAMS = {"detectors": 1, "noise": 2, "bank": 3, "sigma": 4, "snr": 5, "chirp": 6,
            "bands": 7, "inject": 8, "misc": 9}


def rng(config_index: int, purpose: str, sub: int = 0) -> np.random.Generator:
    """Independent generator for (workload, purpose, sub-stream)."""
    ss = np.random.SeedSequence([SEED_BASE + int(config_index), _STREAMS[purpose], int(sub)])
    return np.random.Generator(np.random.PCG64(ss))


@dataclasses.dataclass
class Detectors:
    pos_m: np.ndarray    # [n_det][3] fp64, Earth-fixed position (m)
    arm_x: np.ndarray    # [n_det][3] fp64, unit vector of arm X
    arm_y: np.ndarray    # [n_det][3] fp64, unit vector of arm Y (orthogonal to X, tangent plane)


def detectors(config_index: int, n_det: int) -> Detectors:
    """Detectors placed uniformly on a 6371 km sphere with seeded arm azimuths.

    Arm X = cos(alpha) e_north + sin(alpha) e_east with alpha uniform; arm Y =
    r_hat x X, so the arms are orthogonal and tangent to the sphere.
    """
    g = rng(config_index, "detectors")
    pos = np.empty((n_det, 3))
    ax = np.empty((n_det, 3))
    ay = np.empty((n_det, 3))
    for i in range(n_det):
        cz = g.uniform(-1.0, 1.0)
        lon = g.uniform(0.0, 2.0 * math.pi)
        sz = math.sqrt(max(0.0, 1.0 - cz * cz))
        rhat = np.array([sz * math.cos(lon), sz * math.sin(lon), cz])
        east = np.array([-math.sin(lon), math.cos(lon), 0.0])
        north = np.cross(rhat, east)
        alpha = g.uniform(0.0, 2.0 * math.pi)
        x = math.cos(alpha) * north + math.sin(alpha) * east
        x /= np.linalg.norm(x)
        y = np.cross(rhat, x)
        y /= np.linalg.norm(y)
        pos[i] = EARTH_RADIUS_M * rhat
        ax[i] = x
        ay[i] = y
    return Detectors(pos, ax, ay)


def white_noise(config_index: int, n_det: int, n: int, sub: int = 0) -> np.ndarray:
    """Unit-variance white Gaussian strain, [n_det][n] float32."""
    g = rng(config_index, "noise", sub)
    return g.standard_normal((n_det, n)).astype(np.float32)


@dataclasses.dataclass
class Bank:
    offsets: np.ndarray  # [T+1] int64, CSR over templates
    a1: np.ndarray       # [F] complex64 feedback coefficient
    b0: np.ndarray       # [F] complex64 feedforward coefficient
    delay: np.ndarray    # [F] int32 integer delay in samples

    @property
    def n_templates(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def n_filters(self) -> int:
        return int(self.offsets[-1])

    def counts(self) -> np.ndarray:
        return np.diff(self.offsets)

    def subset(self, templates) -> "Bank":
        """Bank made of the listed templates (in that order)."""
        idx = []
        off = [0]
        for t in templates:
            lo, hi = int(self.offsets[t]), int(self.offsets[t + 1])
            idx.extend(range(lo, hi))
            off.append(off[-1] + hi - lo)
        idx = np.asarray(idx, dtype=np.int64)
        return Bank(np.asarray(off, dtype=np.int64), self.a1[idx].copy(), self.b0[idx].copy(),
                    self.delay[idx].copy())


def random_bank(g: np.random.Generator, counts, d_max: int, mag=(0.9, 0.999),
                phase=(0.0, 2.0 * math.pi), d_min: int = 0) -> Bank:
    """Bank with the given filter count per template (recipe in the module docstring)."""
    counts = np.asarray(counts, dtype=np.int64)
    off = np.zeros(counts.size + 1, dtype=np.int64)
    np.cumsum(counts, out=off[1:])
    F = int(off[-1])
    r = g.uniform(mag[0], mag[1], F)
    ph = g.uniform(phase[0], phase[1], F)
    a1 = (r * np.exp(1j * ph)).astype(np.complex64)
    scale = np.repeat(1.0 / np.sqrt(np.maximum(counts, 1)), counts)
    b0 = ((g.standard_normal(F) + 1j * g.standard_normal(F)) / math.sqrt(2.0) * scale).astype(np.complex64)
    d = g.integers(d_min, d_max + 1, F).astype(np.int32)
    return Bank(off, a1, b0, d)


def noise_weights(config_index: int, n_det: int, lo: float, hi: float) -> np.ndarray:
    if lo == hi:
        return np.full(n_det, lo, dtype=np.float64)
    return rng(config_index, "sigma").uniform(lo, hi, n_det)


def complex_gaussian_snr(config_index: int, shape, sub: int = 0) -> np.ndarray:
    """i.i.d. complex Gaussian SNR samples with E|z|^2 = 2 (complex64)."""
    g = rng(config_index, "snr", sub)
    return (g.standard_normal(shape) + 1j * g.standard_normal(shape)).astype(np.complex64)


# ----------------------------------------------------------------------------------------------
# workload recipes

TINY = dict(index=0, n_det=2, rate=2048, n=32768, n_templates=4, n_filters=64, d_max=2047,
            nside=4, sigma=(1.0, 1.0))
ONLINE = dict(index=1, n_det=3, rate=2048, chunk=2048, n_chunks=32, n_templates=1024,
              f_range=(200, 900), d_max=4096, nside=16, sigma=(0.5, 2.0))


def tiny_workload():
    c = TINY
    det = detectors(c["index"], c["n_det"])
    strain = white_noise(c["index"], c["n_det"], c["n"])
    bank = random_bank(rng(c["index"], "bank"), [c["n_filters"]] * c["n_templates"], c["d_max"])
    sigma = noise_weights(c["index"], c["n_det"], *c["sigma"])
    return dict(cfg=c, det=det, strain=strain, bank=bank, sigma=sigma)


def online_bank(n_templates: int = ONLINE["n_templates"]) -> Bank:
    c = ONLINE
    g = rng(c["index"], "bank")
    counts = g.integers(c["f_range"][0], c["f_range"][1] + 1, c["n_templates"])
    full = random_bank(g, counts, c["d_max"])
    if n_templates == c["n_templates"]:
        return full
    return full.subset(range(n_templates))


def normalised(bank: Bank, power: float = 2.0) -> Bank:
    """The bank with each template's b0 scaled so that the filters' output powers in unit white
    noise add up to `power`: sum_l |b0_l|^2 / (1 - |a1_l|^2) = power (cross terms between
    filters, which average out over random phases and delays, are left out).  With power 2 the
    SNR of a template has E|z|^2 close to 2, the normalisation the candidate threshold assumes."""
    a2 = np.abs(bank.a1.astype(np.complex128)) ** 2
    b2 = np.abs(bank.b0.astype(np.complex128)) ** 2
    per = np.add.reduceat(b2 / (1.0 - a2), bank.offsets[:-1]) if bank.n_filters else np.zeros(0)
    per = np.where(np.diff(bank.offsets) > 0, per, 1.0)
    scale = np.repeat(np.sqrt(power / per), np.diff(bank.offsets))
    return Bank(bank.offsets.copy(), bank.a1.copy(), (bank.b0 * scale).astype(np.complex64), bank.delay.copy())


def online_bank_global(world: int = 1, per_rank: int = ONLINE["n_templates"]) -> Bank:
    """Bank of world x per_rank online-sized templates for a run sharded by template over
    world GPUs (each rank filters a contiguous slice).  world = 1 gives online_bank(per_rank)."""
    if world == 1:
        return online_bank(per_rank)
    c = ONLINE
    g = rng(c["index"], "bank", world)
    counts = g.integers(c["f_range"][0], c["f_range"][1] + 1, world * per_rank)
    return random_bank(g, counts, c["d_max"])


def online_workload(n_templates: int = ONLINE["n_templates"]):
    c = ONLINE
    det = detectors(c["index"], c["n_det"])
    sigma = noise_weights(c["index"], c["n_det"], *c["sigma"])
    return dict(cfg=c, det=det, bank=online_bank(n_templates), sigma=sigma)


def online_chunk(chunk_index: int) -> np.ndarray:
    """1 s chunk number ``chunk_index`` of the online-sized strain, [3][2048] float32."""
    c = ONLINE
    return white_noise(c["index"], c["n_det"], c["chunk"], sub=1000 + chunk_index)


# ----------------------------------------------------------------------------------------------
# Chirp targets and initial IIR coefficients for the adjoint workload

G_MSUN_S = 4.925490947641267e-06   # G M_sun / c^3 in seconds
CHIRP = dict(index=3, n_templates=256, n_filters=300, rate=2048.0, f_lo=30.0, f_hi=1024.0, mc=(1.0, 3.0))


def newtonian_chirp(mc_msun: float, rate: float = 2048.0, f_lo: float = 30.0, f_hi: float = 1024.0):
    """Leading-order (Newtonian) complex chirp, time-reversed so that sample 0 is the
    high-frequency end.  tau is the time to coalescence, M = G Mc / c^3:
        f(tau) = (1/pi) (5 / (256 tau))^(3/8) M^(-5/8),   phi(tau) = -2 (tau / (5 M))^(5/8),
        amplitude proportional to f^(2/3).
    Sample j is at tau_j = tau(f_hi) + j / rate, up to tau(f_lo).  Returns complex128 h[j]."""
    M = mc_msun * G_MSUN_S
    tau_of_f = lambda f: (5.0 / 256.0) * (math.pi * f) ** (-8.0 / 3.0) * M ** (-5.0 / 3.0)
    t_hi, t_lo = tau_of_f(f_hi), tau_of_f(f_lo)
    n = int(math.floor((t_lo - t_hi) * rate)) + 1
    tau = t_hi + np.arange(n) / rate
    f = (1.0 / math.pi) * (5.0 / (256.0 * tau)) ** (3.0 / 8.0) * M ** (-5.0 / 8.0)
    phi = -2.0 * (tau / (5.0 * M)) ** (5.0 / 8.0)
    amp = (f / f_hi) ** (2.0 / 3.0)
    return amp * np.exp(1j * phi)


def segment_fit(h: np.ndarray, n_filters: int):
    """Per-frequency-segment first-order IIR fit of a complex waveform h[k].

    The phase is approximated linearly on each segment (the SPIIR construction: a = e^(gamma +
    i omega), b = the waveform at the segment start).  Segment lengths follow an equal
    share of the integral of |phi''|^(1/2), so that the quadratic phase error is about the same
    on every segment.  omega is the mean phase slope over the segment and gamma = -1 / length.
    Returns (a1, b0, delay) as complex128, complex128, int32 arrays of n_filters entries."""
    n = h.size
    ph = np.unwrap(np.angle(h))
    d2 = np.abs(np.gradient(np.gradient(ph)))
    w = np.sqrt(d2 + 1e-12)
    cum = np.concatenate([[0.0], np.cumsum(w)])
    edges = np.searchsorted(cum, np.linspace(0.0, cum[-1], n_filters + 1))
    edges = np.clip(edges, 0, n)
    edges[0], edges[-1] = 0, n
    # strictly increasing, at least one sample each: e_i = max(e_i, e_{i-1} + 1)
    k = np.arange(edges.size)
    edges = np.maximum.accumulate(edges - k) + k
    edges = np.minimum(edges, n)
    lo = np.minimum(edges[:-1], n - 1)
    hi = np.maximum(np.minimum(edges[1:], n), lo + 1)
    L = np.maximum(hi - lo, 1)
    omega = np.where(L > 1, (ph[hi - 1] - ph[lo]) / np.maximum(L - 1, 1), ph[np.minimum(lo + 1, n - 1)] - ph[lo])
    a1 = np.exp(-1.0 / L + 1j * omega)
    b0 = h[lo].astype(np.complex128)
    d = lo.astype(np.int32)
    return a1, b0, d


def chirp_workload(n_templates: int = CHIRP["n_templates"], n_filters: int = CHIRP["n_filters"],
                   mc=None, max_len: int = None):
    """Adjoint workload: chirp targets and perturbed IIR fits.

    Chirp masses are uniform in [1, 3] solar masses (or the given list).  The fit
    coefficients are perturbed by +-5%: the decay rate gamma and |b0| by a factor 1 + 0.05 u,
    the phase of b0 by 0.05 pi u, and the frequency omega by 0.05 u (2 pi / length) -- a drift of
    at most 5% of a cycle over the segment -- with u uniform in [-1, 1].  Targets are padded
    with zeros to the longest chirp (or truncated to max_len).  Returns dict with h [T][n]
    complex128, a1, b0 [T][F] complex64, delay [T][F] int32, s0 [T][F] complex64 (zeros), mc."""
    g = rng(CHIRP["index"], "chirp")
    if mc is None:
        mc = g.uniform(CHIRP["mc"][0], CHIRP["mc"][1], n_templates)
    mc = np.asarray(mc, dtype=np.float64)
    hs = [newtonian_chirp(float(m)) for m in mc]
    if max_len is not None:
        hs = [h[:max_len] for h in hs]
    n = max(h.size for h in hs)
    H = np.zeros((len(hs), n), dtype=np.complex128)
    A = np.empty((len(hs), n_filters), dtype=np.complex64)
    B = np.empty_like(A)
    D = np.empty((len(hs), n_filters), dtype=np.int32)
    for t, h in enumerate(hs):
        H[t, : h.size] = h
        a1, b0, d = segment_fit(h, n_filters)
        L = np.diff(np.concatenate([d, [h.size]])).clip(min=1)
        u = g.uniform(-1.0, 1.0, (4, n_filters))
        gam = np.log(np.abs(a1)) * (1.0 + 0.05 * u[0])
        om = np.angle(a1) + 0.05 * u[1] * 2.0 * math.pi / L
        A[t] = np.exp(gam + 1j * om).astype(np.complex64)
        B[t] = (b0 * (1.0 + 0.05 * u[2]) * np.exp(1j * 0.05 * math.pi * u[3])).astype(np.complex64)
        D[t] = d
    return dict(h=H, a1=A, b0=B, delay=D, s0=np.zeros_like(A), mc=mc)


# ----------------------------------------------------------------------------------------------
# Scale workload: 4096 chirp templates x 600 filters, 60 s, 20 injections, nside 32

SCALE = dict(index=4, n_det=3, rate=2048, chunk=2048, n_chunks=60, n_templates=4096, n_filters=600,
             mc=(1.0, 3.0), f_lo=30.0, f_hi=1024.0, nside=32, sigma=(0.5, 2.0),
             n_inj=20, snr=(8.0, 20.0), tc_s=(20.0, 58.0), factors=(1, 4, 16))


def chirp_fit(mc_msun: float, n_filters: int, rate: float = 2048.0, f_lo: float = 30.0, f_hi: float = 1024.0):
    """First-order IIR fit of conj(h), h = newtonian_chirp(mc) (time-reversed, sample j at
    tau_j = tau(f_hi) + j / rate), built from the chirp's closed form so that long templates cost
    O(n_filters): the segment construction of segment_fit with the integral of |phi''|^(1/2)
    taken analytically.  With phi(tau) = -2 (tau / 5M)^(5/8), phi'' is proportional to
    tau^(-11/8), so the integral of |phi''|^(1/2) grows as tau^(5/16) and segment i starts at
    the first sample with tau^(5/16) - tau_hi^(5/16) >= (i / N) (tau_lo^(5/16) - tau_hi^(5/16)).
    On each segment omega is the mean phase slope of conj(h), gamma = -1 / length and b0 the
    value of conj(h) at the segment start.  Returns (a1, b0, delay, n, sum_j |h_j|^2) with
    complex128 coefficients and int32 delays."""
    M = mc_msun * G_MSUN_S
    tau_of_f = lambda f: (5.0 / 256.0) * (math.pi * f) ** (-8.0 / 3.0) * M ** (-5.0 / 3.0)
    t_hi, t_lo = tau_of_f(f_hi), tau_of_f(f_lo)
    n = int(math.floor((t_lo - t_hi) * rate)) + 1
    tau_end = t_hi + (n - 1) / rate
    u = np.linspace(0.0, 1.0, n_filters + 1) * (tau_end ** 0.3125 - t_hi ** 0.3125) + t_hi ** 0.3125
    edges = np.ceil((u ** 3.2 - t_hi) * rate - 1e-9).astype(np.int64)
    edges = np.clip(edges, 0, n)
    edges[0], edges[-1] = 0, n
    k = np.arange(edges.size)
    edges = np.maximum.accumulate(edges - k) + k      # strictly increasing
    edges = np.minimum(edges, n)
    lo = np.minimum(edges[:-1], n - 1)
    hi = np.maximum(np.minimum(edges[1:], n), lo + 1)
    L = np.maximum(hi - lo, 1)
    phase = lambda j: -2.0 * ((t_hi + j / rate) / (5.0 * M)) ** 0.625        # phase of h at sample j
    amp = lambda j: ((t_hi + j / rate) / t_hi) ** (-0.25)                     # (f / f_hi)^(2/3)
    jb = np.where(L > 1, hi - 1, np.minimum(lo + 1, n - 1))
    omega = -(phase(jb.astype(np.float64)) - phase(lo.astype(np.float64))) / np.maximum(jb - lo, 1)
    a1 = np.exp(-1.0 / L + 1j * omega)
    b0 = amp(lo.astype(np.float64)) * np.exp(-1j * phase(lo.astype(np.float64)))
    # sum_j amp_j^2 = sum_j (tau_j / t_hi)^(-1/2) by Euler-Maclaurin (the integrand is smooth)
    g = lambda j: ((t_hi + j / rate) / t_hi) ** (-0.5)
    dg = lambda j: -0.5 * ((t_hi + j / rate) / t_hi) ** (-1.5) / (rate * t_hi)
    e = float(n - 1)
    integral = 2.0 * rate * t_hi * (((t_hi + e / rate) / t_hi) ** 0.5 - 1.0)
    power = integral + 0.5 * (g(0.0) + g(e)) + (dg(e) - dg(0.0)) / 12.0
    return a1, b0, lo.astype(np.int32), n, power


def scale_bank(n_templates: int = SCALE["n_templates"], n_filters: int = SCALE["n_filters"]):
    """Template bank on a uniform chirp-mass grid over [1, 3] Msun.  Template t is the
    first-order IIR fit (chirp_fit) of conj(h_t), h_t the whole time-reversed Newtonian chirp
    from 30 Hz to 1024 Hz (12 s at 3 Msun to 74 s, about 151k samples, at 1 Msun), so that the
    bank's output is the correlation with the chirp; b0 is scaled by sqrt(2 / sum |h_t|^2), which
    makes E|z|^2 = 2 in unit white noise (up to the fit's mismatch).  Returns (Bank, mc [T],
    template lengths [T])."""
    c = SCALE
    mcs = np.linspace(c["mc"][0], c["mc"][1], n_templates)
    A = np.empty((n_templates, n_filters), dtype=np.complex64)
    B = np.empty_like(A)
    D = np.empty((n_templates, n_filters), dtype=np.int32)
    lens = np.empty(n_templates, dtype=np.int64)
    for t, mc in enumerate(mcs):
        a1, b0, d, n, power = chirp_fit(float(mc), n_filters, c["rate"], c["f_lo"], c["f_hi"])
        A[t] = a1.astype(np.complex64)
        B[t] = (b0 * math.sqrt(2.0 / power)).astype(np.complex64)
        D[t] = d
        lens[t] = n
    off = np.arange(n_templates + 1, dtype=np.int64) * n_filters
    return Bank(off, A.ravel(), B.ravel(), D.ravel()), mcs, lens


def scale_bank_multirate(bank: Bank, factors=SCALE["factors"], rate: float = 2048.0, fir_delay: float = 15.5):
    """The scale bank recast over the multirate bands of the batched path (decimation by M_b
    with the 32-tap low-pass, band SNR upsampled linearly with one band sample of lag).  A
    full-rate filter (a, b, d) of frequency f = |arg a| rate / 2 pi goes to the slowest band
    with f <= 0.3 rate / M_b (0.6 of the band's Nyquist frequency) whose rate still gives the
    filter's decay length 1 / |log|a|| at least 2 band samples and whose total lag
    fir_delay + M_b fits in d; there it becomes (a^M, M b a^(l - d), d_b) with
    d_b = floor((d - fir_delay - M) / M) and l = M d_b + M + fir_delay the full-rate lag of the
    band path, so that its response approximates b a^(k - d).  Returns (offsets, a1, b0, delay,
    band) for spiir_batch_create and oracle.multirate_bank."""
    a = bank.a1.astype(np.complex128)
    b = bank.b0.astype(np.complex128)
    d = bank.delay.astype(np.int64)
    f = np.abs(np.angle(a)) * rate / (2.0 * math.pi)
    decay = 1.0 / np.maximum(-np.log(np.abs(a)), 1e-12)
    band = np.zeros(a.size, dtype=np.int32)
    for bi, M in enumerate(factors):
        if M == 1:
            continue
        ok = (f <= 0.3 * rate / M) & (decay >= 2.0 * M) & (d >= fir_delay + M)
        band[ok] = bi      # later (slower) bands override earlier ones
    Mv = np.asarray(factors, dtype=np.int64)[band]
    db = np.where(Mv == 1, d, np.floor((d - fir_delay - Mv) / Mv)).astype(np.int64)
    lag = np.where(Mv == 1, d, Mv * db + Mv + fir_delay)
    loga = np.log(a)
    a_b = np.exp(Mv * loga)
    b_b = np.where(Mv == 1, b, Mv * b * np.exp((lag - d) * loga))
    return (bank.offsets.copy(), a_b.astype(np.complex64), b_b.astype(np.complex64), db.astype(np.int32), band)


def scale_injections(n: int = SCALE["n_inj"]):
    """Injection parameters: chirp mass U[1, 3] Msun; source direction isotropic (unit
    vector); polarisation angle U[0, pi); cos(inclination) U[-1, 1]; coalescence phase
    U[0, 2 pi); geocentric coalescence sample round(2048 x U[20, 58] s); network SNR U[8, 20]."""
    c = SCALE
    g = rng(c["index"], "inject")
    mc = g.uniform(c["mc"][0], c["mc"][1], n)
    cz = g.uniform(-1.0, 1.0, n)
    ph = g.uniform(0.0, 2.0 * math.pi, n)
    sz = np.sqrt(1.0 - cz ** 2)
    nhat = np.stack([sz * np.cos(ph), sz * np.sin(ph), cz], axis=1)
    return dict(mc=mc, nhat=nhat, psi=g.uniform(0.0, math.pi, n), cosi=g.uniform(-1.0, 1.0, n),
                phic=g.uniform(0.0, 2.0 * math.pi, n),
                tc=np.rint(g.uniform(c["tc_s"][0], c["tc_s"][1], n) * c["rate"]).astype(np.int64),
                snr=g.uniform(c["snr"][0], c["snr"][1], n))


# ----------------------------------------------------------------------------------------------
# Multirate batched workload

MULTIRATE = dict(index=2, n_det=3, rate=2048, chunk=512, n_banks=8, t_range=(64, 2048), f_range=(100, 1200),
                 factors=(1, 4, 16), band_p=(0.4, 0.35, 0.25), d_max_s=2.0, nside=16, sigma=(0.5, 2.0))


def multirate_banks(n_banks=None, t_range=None, f_range=None, seed_sub=0):
    """Banks of the batched workload: template counts log-uniform in t_range, filters per
    template uniform in f_range, each filter in band b with probability band_p[b].  In band b
    (decimation M_b) the delay is uniform in [0, 2 s x 2048 / M_b] band samples, |a1| uniform in
    [0.9, 0.999] and arg a1 uniform in [-0.8 pi, 0.8 pi] for decimated bands (inside the
    decimation filter's passband) or [0, 2 pi) at the full rate; b0 complex normal / sqrt(F).
    Returns a list of (offsets, a1, b0, delay, band)."""
    c = MULTIRATE
    n_banks = c["n_banks"] if n_banks is None else n_banks
    t_range = c["t_range"] if t_range is None else t_range
    f_range = c["f_range"] if f_range is None else f_range
    g = rng(c["index"], "bands", seed_sub)
    out = []
    for _ in range(n_banks):
        T = int(round(math.exp(g.uniform(math.log(t_range[0]), math.log(t_range[1])))))
        counts = g.integers(f_range[0], f_range[1] + 1, T)
        off = np.zeros(T + 1, dtype=np.int64)
        np.cumsum(counts, out=off[1:])
        F = int(off[-1])
        band = g.choice(len(c["factors"]), size=F, p=c["band_p"]).astype(np.int32)
        M = np.asarray(c["factors"])[band]
        r = g.uniform(0.9, 0.999, F)
        ph_full = g.uniform(0.0, 2.0 * math.pi, F)
        ph_dec = g.uniform(-0.8 * math.pi, 0.8 * math.pi, F)
        ph = np.where(M == 1, ph_full, ph_dec)
        a1 = (r * np.exp(1j * ph)).astype(np.complex64)
        scale = np.repeat(1.0 / np.sqrt(counts), counts)
        b0 = ((g.standard_normal(F) + 1j * g.standard_normal(F)) / math.sqrt(2.0) * scale).astype(np.complex64)
        dmax = (c["d_max_s"] * c["rate"] / M).astype(np.int64)
        d = np.floor(g.uniform(0.0, 1.0, F) * (dmax + 1)).astype(np.int32)
        out.append((off, a1, b0, d, band))
    return out


def multirate_chunk(chunk_index: int, n_det: int = 3, chunk: int = 512) -> np.ndarray:
    return white_noise(MULTIRATE["index"], n_det, chunk, sub=2000 + chunk_index)
