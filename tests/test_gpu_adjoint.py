"""GPU impulse response and adjoint (K3) against the FP64 oracle and FP64 finite differences."""
import numpy as np
import pytest

import oracle
import synth
from helpers import cuda_ok

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs CUDA")]

ADJ_TOL = 1e-3  # adjoint gradients vs FP64 finite differences, relative


def _cuda(x, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x))
    return (t if dtype is None else t.to(dtype)).cuda()


def _flat_bank(w):
    T, F = w["a1"].shape
    return np.arange(T + 1, dtype=np.int64) * F


def _gpu_forward(a1, b0, s0, d, n, ckpt_every=1024):
    import torch
    from paper_2011_06787_b300.adjoint import impulse_response
    u = impulse_response(_cuda(a1), _cuda(b0), _cuda(s0), _cuda(d), n, ckpt_every)
    torch.cuda.synchronize()
    return u


def test_forward_matches_oracle_with_initial_states():
    w = synth.chirp_workload(4, 300, mc=[1.3, 1.8, 2.4, 2.9], max_len=20000)
    g = np.random.default_rng(1)
    s0 = ((g.standard_normal(w["a1"].shape) + 1j * g.standard_normal(w["a1"].shape)) * 0.01).astype(np.complex64)
    n = w["h"].shape[1]
    u = _gpu_forward(w["a1"], w["b0"], s0, w["delay"], n).cpu().numpy()
    u_or = oracle.impulse_forward(_flat_bank(w), w["a1"].ravel(), w["b0"].ravel(), w["delay"].ravel(), s0.ravel(), n)
    err = np.abs(u - u_or).max(axis=1) / np.abs(u_or).max(axis=1)
    assert np.all(err < 1e-4), err


@pytest.mark.parametrize("ckpt_every", [64, 1024])
def test_backward_matches_oracle_adjoint(ckpt_every):
    import torch
    from paper_2011_06787_b300 import native
    import ctypes
    w = synth.chirp_workload(3, 200, mc=[2.2, 2.6, 3.0], max_len=12000)
    T, F = w["a1"].shape
    n = w["h"].shape[1]
    g = np.random.default_rng(2)
    s0 = ((g.standard_normal((T, F)) + 1j * g.standard_normal((T, F))) * 0.01).astype(np.complex64)
    grad_u = (g.standard_normal((T, n)) + 1j * g.standard_normal((T, n))).astype(np.complex64)
    a1, b0, d, s = _cuda(w["a1"]), _cuda(w["b0"]), _cuda(w["delay"]), _cuda(s0)
    u = torch.empty((T, n), dtype=torch.complex64, device="cuda")
    nck = (n + ckpt_every - 1) // ckpt_every
    ck = torch.empty((nck, T, F), dtype=torch.complex64, device="cuda")
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    L = native.lib()
    native.check(L.spiir_impulse_forward(T, F, P(a1), P(b0), P(d), P(s), n, P(u), ckpt_every, P(ck), st))
    gu = _cuda(grad_u)
    ga, gb, gs = (torch.empty_like(a1) for _ in range(3))
    work = torch.empty((nck + 2, T, F), dtype=torch.complex64, device="cuda")
    native.check(L.spiir_impulse_backward(T, F, P(a1), P(b0), P(d), n, P(gu), ckpt_every, P(ck), P(ga), P(gb), P(gs),
                                          P(work), st))
    torch.cuda.synchronize()
    ga_or, gb_or, gs_or = oracle.impulse_backward(_flat_bank(w), w["a1"].ravel(), w["b0"].ravel(), w["delay"].ravel(),
                                                  s0.ravel(), grad_u)
    for got, ref in ((ga, ga_or), (gb, gb_or), (gs, gs_or)):
        got = got.cpu().numpy().ravel()
        assert np.max(np.abs(got - ref)) <= 1e-4 * np.max(np.abs(ref)), np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    # checkpoints: state before sample j * ckpt_every
    _, yend = oracle.impulse_forward(_flat_bank(w), w["a1"].ravel(), w["b0"].ravel(), w["delay"].ravel(), s0.ravel(),
                                     ckpt_every, return_end=True)
    assert np.max(np.abs(ck[1].cpu().numpy().ravel() - yend)) <= 1e-4 * np.max(np.abs(yend))


def _loss_oracle(w, T8, a1, b0, s0):
    n = w["h"].shape[1]
    off = np.arange(T8 + 1, dtype=np.int64) * a1.shape[1]
    u = oracle.impulse_forward(off, a1.ravel(), b0.ravel(), w["delay"][:T8].ravel(), s0.ravel(), n)
    return oracle.overlap_loss(w["h"][:T8], u)[0].sum()


def test_adjoint_matches_fp64_finite_differences_on_first_8_chirps():
    """Chirp workload (300 filters per template, chirp mass 1..3 Msun): gradient of the summed
    loss 1 - O of the first 8 templates, through the autograd wrapper, against FP64 central
    differences of the oracle's loss along random directions."""
    import torch
    from paper_2011_06787_b300.adjoint import impulse_response, overlap_loss
    oracle.set_threads(16)
    w = synth.chirp_workload(8, 300)
    n = w["h"].shape[1]
    a1 = _cuda(w["a1"]).requires_grad_(True)
    b0 = _cuda(w["b0"]).requires_grad_(True)
    s0 = _cuda(w["s0"]).requires_grad_(True)
    u = impulse_response(a1, b0, s0, _cuda(w["delay"]), n, 1024)
    loss = overlap_loss(_cuda(w["h"], torch.complex64), u).sum()
    loss.backward()
    grads = [x.grad.cpu().numpy().astype(np.complex128) for x in (a1, b0, s0)]
    base = [w["a1"].astype(np.complex128), w["b0"].astype(np.complex128), w["s0"].astype(np.complex128)]
    L0 = _loss_oracle(w, 8, *base)
    assert abs(loss.item() - L0) < 1e-4 * max(L0, 1e-3)
    g = np.random.default_rng(3)
    for trial in range(3):
        dirs = [g.standard_normal(x.shape) + 1j * g.standard_normal(x.shape) for x in base]
        scale = [1e-7, 1e-6, 1e-6]
        dirs = [s * v for s, v in zip(scale, dirs)]
        plus = _loss_oracle(w, 8, *[x + v for x, v in zip(base, dirs)])
        minus = _loss_oracle(w, 8, *[x - v for x, v in zip(base, dirs)])
        fd = (plus - minus) / 2.0
        ad = sum(np.sum((np.conj(gr) * v).real) for gr, v in zip(grads, dirs))
        assert abs(ad - fd) <= ADJ_TOL * abs(fd), (trial, ad, fd)


def test_adjoint_per_parameter_finite_differences_short_bank():
    import torch
    from paper_2011_06787_b300.adjoint import impulse_response, overlap_loss
    w = synth.chirp_workload(2, 12, mc=[2.8, 3.0], max_len=1500)
    n = w["h"].shape[1]
    g = np.random.default_rng(4)
    w["s0"] = ((g.standard_normal(w["a1"].shape) + 1j * g.standard_normal(w["a1"].shape)) * 0.05).astype(np.complex64)
    a1 = _cuda(w["a1"]).requires_grad_(True)
    b0 = _cuda(w["b0"]).requires_grad_(True)
    s0 = _cuda(w["s0"]).requires_grad_(True)
    u = impulse_response(a1, b0, s0, _cuda(w["delay"]), n, 64)
    overlap_loss(_cuda(w["h"], torch.complex64), u).sum().backward()
    base = [w["a1"].astype(np.complex128), w["b0"].astype(np.complex128), w["s0"].astype(np.complex128)]
    for which, t in enumerate((a1, b0, s0)):
        grad = t.grad.cpu().numpy()
        for idx in [(0, 0), (0, 5), (1, 11), (1, 3)]:
            for unit, part in ((1.0, np.real), (1j, np.imag)):
                eps = 1e-7
                p = [x.copy() for x in base]
                m = [x.copy() for x in base]
                p[which][idx] += eps * unit
                m[which][idx] -= eps * unit
                fd = (_loss_oracle(w, 2, *p) - _loss_oracle(w, 2, *m)) / (2 * eps)
                ad = part(grad[idx])
                assert abs(ad - fd) <= ADJ_TOL * max(abs(fd), 1e-3), (which, idx, unit, ad, fd)


def test_checkpoint_interval_does_not_change_gradients():
    import torch
    from paper_2011_06787_b300.adjoint import impulse_response, overlap_loss
    w = synth.chirp_workload(4, 300, mc=[1.0, 1.7, 2.3, 3.0])
    n = w["h"].shape[1]
    out = []
    for ck in (256, 1024):
        a1 = _cuda(w["a1"]).requires_grad_(True)
        b0 = _cuda(w["b0"]).requires_grad_(True)
        s0 = _cuda(w["s0"]).requires_grad_(True)
        u = impulse_response(a1, b0, s0, _cuda(w["delay"]), n, ck)
        overlap_loss(_cuda(w["h"], torch.complex64), u).sum().backward()
        out.append([x.grad.cpu().numpy() for x in (a1, b0, s0)])
    for g1, g2 in zip(*out):
        assert np.max(np.abs(g1 - g2)) <= 1e-5 * np.max(np.abs(g1)) + 1e-12


def test_gradient_descent_improves_the_overlap():
    import torch
    from paper_2011_06787_b300.adjoint import impulse_response, overlap_loss
    w = synth.chirp_workload(4, 300, mc=[1.2, 1.9, 2.5, 2.95], max_len=40000)
    n = w["h"].shape[1]
    h = _cuda(w["h"], torch.complex64)
    a1 = _cuda(w["a1"]).requires_grad_(True)
    b0 = _cuda(w["b0"]).requires_grad_(True)
    s0 = _cuda(w["s0"]).requires_grad_(True)
    d = _cuda(w["delay"])
    opt = torch.optim.Adam([b0], lr=2e-3)
    first = None
    for it in range(30):
        opt.zero_grad()
        loss = overlap_loss(h, impulse_response(a1, b0, s0, d, n, 1024)).sum()
        loss.backward()
        opt.step()
        first = loss.item() if first is None else first
    assert loss.item() < 0.95 * first


@pytest.mark.parametrize("ckpt_every,F", [(32, 64), (96, 64), (4096, 64), (1024, 900), (224, 333)])
def test_forward_without_checkpoints_matches_the_segmented_forward(ckpt_every, F):
    """The segmented forward (FP64 jumps between checkpoints, segments in parallel) against the
    sequential one (no checkpoint buffer) and the oracle; ragged last segments, delays past n,
    non-zero initial states."""
    import torch
    from paper_2011_06787_b300 import native
    import ctypes
    w = synth.chirp_workload(3, F, mc=[2.5, 2.8, 3.0], max_len=5000)
    T, F = w["a1"].shape
    n = 4999
    g = np.random.default_rng(5)
    s0 = ((g.standard_normal((T, F)) + 1j * g.standard_normal((T, F))) * 0.02).astype(np.complex64)
    d = w["delay"].copy()
    d[:, -3:] = n + 100  # impulses that never arrive
    a1, b0, dd, s = _cuda(w["a1"]), _cuda(w["b0"]), _cuda(d), _cuda(s0)
    P = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    L = native.lib()
    u_seq = torch.empty((T, n), dtype=torch.complex64, device="cuda")
    rc = L.spiir_impulse_forward(T, F, P(a1), P(b0), P(dd), P(s), n, P(u_seq), ckpt_every, None, st)
    if F > 864:  # the sequential form's reduction rows exceed shared memory
        assert rc == native.EUNSUPPORTED
        u_seq = None
    else:
        native.check(rc)
    u_seg = torch.empty((T, n), dtype=torch.complex64, device="cuda")
    ck = torch.empty(((n + ckpt_every - 1) // ckpt_every, T, F), dtype=torch.complex64, device="cuda")
    native.check(L.spiir_impulse_forward(T, F, P(a1), P(b0), P(dd), P(s), n, P(u_seg), ckpt_every, P(ck), st))
    torch.cuda.synchronize()
    u_or = oracle.impulse_forward(_flat_bank(w), w["a1"].ravel(), w["b0"].ravel(), d.ravel(), s0.ravel(), n)
    for u in (u_seq, u_seg):
        if u is None:
            continue
        u = u.cpu().numpy()
        err = np.abs(u - u_or).max(axis=1) / np.abs(u_or).max(axis=1)
        assert np.all(err < 1e-4), err
