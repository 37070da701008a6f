"""Float64 reference of the learned initial guess for BiCGSTAB.
TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper has no learned component; this module fixes what the GPU network
computes (readings of an unstated design):
  * input normalisation: sigma = RMS(u_bar), x0 = u_bar / sigma;
  * four bias-free 3x3x3 convolutions with circular (periodic) padding,
    channels 1 -> C -> C -> C -> 1, ReLU after the first three; bias-free
    ReLU layers make the map positively homogeneous, so the normalisation is
    exact for positive scales;
  * residual output: u0 = u_bar + sigma * A * y with the fixed output scale
    A = (delta/h)^2 = 1/(pi gamma)^2 (the grid-unit size of the delta^2
    Laplacian term of G^{-1} = I - delta^2 Laplacian, Section 4, Eq. df);
  * loss: relative mean-square error ||u0 - u_true||^2 / ||u_true||^2,
    averaged over the samples of a batch;
  * Adam (beta1 = 0.9, beta2 = 0.999, eps = 1e-8).
Arrays are channel-first: activations (C, Z, Y, X), weights (Cout, Cin, 3, 3, 3)
with w[co, ci, a, b, c] multiplying x[ci, z + a - 1, y + b - 1, x + c - 1].
"""

from __future__ import annotations

import numpy as np

TAPS = [(a, b, c) for a in range(3) for b in range(3) for c in range(3)]


def _shift(x, a, b, c):
    """x[..., z + a - 1, y + b - 1, x + c - 1] (periodic)."""
    return np.roll(x, shift=(1 - a, 1 - b, 1 - c), axis=(-3, -2, -1))


def conv3d(x, w):
    """Periodic cross-correlation: y[co] = sum_{ci, taps} w[co, ci, tap] x[ci] shifted by the tap."""
    y = np.zeros((w.shape[0],) + x.shape[1:])
    for (a, b, c) in TAPS:
        y += np.einsum("oi,izyx->ozyx", w[:, :, a, b, c], _shift(x, a, b, c))
    return y


def conv3d_backward(x, w, dy):
    """Gradients of sum(dy * conv3d(x, w)) with respect to x and w."""
    dx = np.zeros_like(x)
    dw = np.zeros_like(w)
    for (a, b, c) in TAPS:
        xs = _shift(x, a, b, c)
        dw[:, :, a, b, c] = np.einsum("ozyx,izyx->oi", dy, xs)
        # d/dx of x[z + a - 1]: move dy by the opposite offset
        dx += np.roll(np.einsum("oi,ozyx->izyx", w[:, :, a, b, c], dy), shift=(a - 1, b - 1, c - 1),
                      axis=(-3, -2, -1))
    return dx, dw


def init_weights(channels=32, seed=0, scale_last=0.1):
    """He-normal initial weights (last layer scaled down so the initial guess
    starts near u_bar)."""
    rng = np.random.default_rng(seed)
    shapes = [(channels, 1), (channels, channels), (channels, channels), (1, channels)]
    ws = []
    for k, (co, ci) in enumerate(shapes):
        std = np.sqrt(2.0 / (27 * ci))
        w = rng.standard_normal((co, ci, 3, 3, 3)) * std
        if k == len(shapes) - 1:
            w *= scale_last
        ws.append(w)
    return ws


def output_scale(gamma):
    """A = (delta/h)^2 = 1/(pi gamma)^2: delta = 1/k_c, k_c = gamma N/2, h = 2 pi/N."""
    return 1.0 / (np.pi * gamma) ** 2


def forward(ws, ubar, ascale=1.0):
    """u0 = u_bar + sigma * A * CNN(u_bar / sigma) and the cache for backward."""
    sigma = float(np.sqrt(np.mean(ubar * ubar)))
    x = (ubar / sigma)[None]
    acts = [x]
    pre = []
    for k, w in enumerate(ws):
        z = conv3d(acts[-1], w)
        pre.append(z)
        acts.append(np.maximum(z, 0.0) if k < len(ws) - 1 else z)
    u0 = ubar + sigma * ascale * acts[-1][0]
    return u0, dict(sigma=sigma, acts=acts, pre=pre)


def loss(u0, utrue):
    """Relative mean-square error of one sample."""
    return float(np.sum((u0 - utrue) ** 2) / np.sum(utrue * utrue))


def loss_and_grads(ws, ubar, utrue, ascale=1.0):
    """Loss of one sample and its gradients with respect to the weights."""
    u0, cache = forward(ws, ubar, ascale)
    L = loss(u0, utrue)
    g = 2.0 * (u0 - utrue) / np.sum(utrue * utrue)      # dL/du0
    dz = (cache["sigma"] * ascale * g)[None]            # dL/dy of the last layer
    grads = [None] * len(ws)
    for k in range(len(ws) - 1, -1, -1):
        dx, dw = conv3d_backward(cache["acts"][k], ws[k], dz)
        grads[k] = dw
        if k > 0:
            dz = dx * (cache["pre"][k - 1] > 0.0)
    return L, grads


class Adam:
    """Adam on a list of arrays."""

    def __init__(self, ws, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = [np.zeros_like(w) for w in ws]
        self.v = [np.zeros_like(w) for w in ws]
        self.t = 0

    def step(self, ws, grads):
        self.t += 1
        out = []
        for i, (w, g) in enumerate(zip(ws, grads)):
            self.m[i] = self.b1 * self.m[i] + (1 - self.b1) * g
            self.v[i] = self.b2 * self.v[i] + (1 - self.b2) * g * g
            mh = self.m[i] / (1 - self.b1 ** self.t)
            vh = self.v[i] / (1 - self.b2 ** self.t)
            out.append(w - self.lr * mh / (np.sqrt(vh) + self.eps))
        return out
