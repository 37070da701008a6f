"""The learned initial guess (bf16 tensor-core CNN) against the float64
oracle network (oracle/cnn.py), and what the trained network gains for
BiCGSTAB, through the C ABI. Grids whose x side is a multiple of 128 run the
32 -> 32 layers on the tcgen05 tensor cores (accumulator in tensor memory,
rows staged by TMA); the others on the warp-level mma kernels; both are
compared with the oracle."""

import numpy as np
import pytest

import oracle
from oracle import cnn
from synth import fields

pytestmark = pytest.mark.gpu


def _to_lib(ws):
    """oracle weights (Cout, Cin, 3, 3, 3) -> the library's flat [tap][in][out] layout."""
    w1 = np.transpose(ws[0][:, 0], (1, 2, 3, 0)).reshape(27, 32)
    w2 = np.transpose(ws[1], (2, 3, 4, 1, 0)).reshape(27, 32, 32)
    w3 = np.transpose(ws[2], (2, 3, 4, 1, 0)).reshape(27, 32, 32)
    w4 = np.transpose(ws[3][0], (1, 2, 3, 0)).reshape(27, 32)
    return np.concatenate([w1.ravel(), w2.ravel(), w3.ravel(), w4.ravel()]).astype(np.float32)


def _from_lib(flat):
    w1 = flat[:27 * 32].reshape(3, 3, 3, 32)
    w2 = flat[27 * 32:27 * 32 + 27 * 1024].reshape(3, 3, 3, 32, 32)
    w3 = flat[27 * 32 + 27 * 1024:27 * 32 + 2 * 27 * 1024].reshape(3, 3, 3, 32, 32)
    w4 = flat[27 * 32 + 2 * 27 * 1024:].reshape(3, 3, 3, 32)
    return [np.transpose(w1, (3, 0, 1, 2))[:, None].astype(np.float64),
            np.transpose(w2, (4, 3, 0, 1, 2)).astype(np.float64),
            np.transpose(w3, (4, 3, 0, 1, 2)).astype(np.float64),
            np.transpose(w4, (3, 0, 1, 2))[None].astype(np.float64)]


def _pairs(shape, n, gamma, seed0=0):
    ut, ub = [], []
    for i in range(n):
        u = fields.random_velocity_field(shape, seed0 + i, fields.spectrum_3d_kolmogorov)[i % 3]
        ut.append(u)
        ub.append(oracle.filter_field(u, gamma))
    return np.array(ut, dtype=np.float32), np.array(ub, dtype=np.float32)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("shape", [(32, 32, 32), (16, 24, 64), (8, 12, 128), (8, 8, 256), (8, 16, 384)])
def test_forward_matches_oracle(gad, shape):
    import torch
    gamma = 0.1
    A = cnn.output_scale(gamma)
    ws = cnn.init_weights(channels=32, seed=3, scale_last=1.0)
    w = torch.from_numpy(_to_lib(ws)).cuda()
    _, ub = _pairs(shape, 2, gamma)
    u0 = gad.guess_infer(w, torch.from_numpy(ub).cuda(), gamma).cpu().numpy()
    for b in range(2):
        ref, _ = cnn.forward(ws, ub[b].astype(np.float64), A)
        # bfloat16 activations: ~2^-8 relative per layer
        assert _rel(u0[b] - ub[b], ref - ub[b]) < 3e-2, b


def test_tensor_core_wait_times_out_cleanly(gad):
    """The tensor-core convolution's barrier waits are bounded. With the limit
    at 0 every wait gives up at once (each CTA still drains, bounded, the TMA
    loads it has in flight and frees its tensor memory): inference reports
    AD_ERR_TIMEOUT instead of hanging, and the context then infers exactly
    what it inferred before."""
    import torch
    gamma = 0.1
    ws = cnn.init_weights(channels=32, seed=3, scale_last=1.0)
    w = torch.from_numpy(_to_lib(ws)).cuda()
    _, ub = _pairs((8, 8, 128), 1, gamma)
    t = torch.from_numpy(ub).cuda()
    ok = gad.guess_infer(w, t, gamma).cpu().numpy()
    gad.set_wait_limit(0)
    try:
        with pytest.raises(gad.GadError) as e:
            gad.guess_infer(w, t, gamma)
        assert e.value.status == gad.AD_ERR_TIMEOUT
    finally:
        gad.set_wait_limit(1_000_000_000)
    again = gad.guess_infer(w, t, gamma).cpu().numpy()
    np.testing.assert_array_equal(again, ok)


@pytest.mark.parametrize("shape", [(8, 16, 32), (8, 8, 128)])
def test_gradients_match_oracle(gad, shape):
    import torch
    gamma = 0.1
    A = cnn.output_scale(gamma)
    ws = cnn.init_weights(channels=32, seed=4, scale_last=1.0)
    ws[3] *= 0.05                                   # keep u0 near u_bar so the loss is O(1)
    w = torch.from_numpy(_to_lib(ws)).cuda()
    ut, ub = _pairs(shape, 2, gamma, seed0=10)
    loss, grad = gad.guess_grad(w, torch.from_numpy(ub).cuda(), torch.from_numpy(ut).cuda(), gamma)
    gl = _from_lib(grad.cpu().numpy())
    ref_loss, ref = 0.0, [np.zeros_like(x) for x in ws]
    for b in range(2):
        L, gs = cnn.loss_and_grads(ws, ub[b].astype(np.float64), ut[b].astype(np.float64), A)
        ref_loss += L / 2
        ref = [r + g / 2 for r, g in zip(ref, gs)]
    assert abs(loss - ref_loss) < 2e-2 * ref_loss
    for k in range(4):
        a, r = gl[k].ravel(), ref[k].ravel()
        cos = float(np.dot(a, r) / (np.linalg.norm(a) * np.linalg.norm(r)))
        assert cos > 0.98 and _rel(a, r) < 0.15, (k, cos, _rel(a, r))


def test_stencil_start_is_the_explicit_inverse(gad):
    import torch
    gamma, shape = 0.01, (32, 32, 32)
    A = cnn.output_scale(gamma)
    w = gad.guess_init(seed=1, stencil=True)
    ut, ub = _pairs(shape, 1, gamma, seed0=20)
    u0 = gad.guess_infer(w, torch.from_numpy(ub).cuda(), gamma).cpu().numpy()[0]
    x = ub[0].astype(np.float64)
    lap = -6 * x + sum(np.roll(x, s, ax) for ax in range(3) for s in (1, -1))
    ref = x - A * lap
    assert _rel(u0, ref) < 2e-2


def test_trained_guess_gains_over_plain_bicgstab(gad):
    """Training lowers the loss from the stencil start, and BiCGSTAB started
    from the trained guess needs fewer passes than from u_bar on held-out
    fields (gamma = 0.01, tolerance 1e-6)."""
    import torch
    gamma, shape = 0.01, (32, 32, 32)
    ut, ub = _pairs(shape, 72, gamma, seed0=100)
    ubt, utt = torch.from_numpy(ub[:64]).cuda(), torch.from_numpy(ut[:64]).cuda()
    w = gad.guess_init(seed=2, stencil=True)
    l0, _ = gad.guess_grad(w, ubt[:8], utt[:8], gamma)
    hist = gad.guess_train(w, ubt, utt, gamma, epochs=6, batch=8, lr=2e-5, seed=5)
    l1, _ = gad.guess_grad(w, ubt[:8], utt[:8], gamma)
    assert np.all(np.isfinite(hist)) and l1 < l0, (l0, l1, hist)
    held = torch.from_numpy(ub[64:]).cuda()
    u0 = gad.guess_infer(w, held, gamma)
    plain = gad.deconvolve(held, gamma, method="bicgstab", tol=1e-6, maxit=3000, ndim=3)
    learned = gad.deconvolve(held, gamma, method="bicgstab", tol=1e-6, maxit=3000, ndim=3, u0=u0)
    assert np.all(plain.status == gad.AD_OK) and np.all(learned.status == gad.AD_OK)
    assert np.all(learned.history[:, 0] < 0.2)
    assert learned.iterations.mean() < 0.8 * plain.iterations.mean(), (learned.iterations, plain.iterations)
    # both reach the same absolute residual target (normalised by ||u_bar - G u_bar||)
    for b in range(held.shape[0]):
        assert learned.history[b, learned.iterations[b]] <= 1e-6
