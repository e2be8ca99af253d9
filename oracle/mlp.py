"""FP64 numpy oracle of the neural proxy -- TEST INFRASTRUCTURE.

The proxy P(omega, theta | psi) maps the sun direction and the design
parameters to force and torque (Sec. 3.3); it is fitted by minimising the
empirical L1 risk E |P - (F|tau)| (Sec. 3.3, Alg. 1 NNLoss) with Adam
(Sec. 3.3).  Architecture (a reading of the paper's inconsistent
sizes): 19 inputs -> 4 hidden layers of 256 with SiLU -> 6 linear outputs.

Plain definitions, no fusion:
  h_0 = x;  z_l = W_l h_l + b_l;  h_{l+1} = silu(z_l)  (l = 0..3);
  y = W_4 h_4 + b_4;  silu(z) = z / (1 + exp(-z)).
Loss: L = mean over the batch of sum_j |y_j - t_j|.
Adam (Kingma & Ba 2015): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
  p -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).

`bf16_round` rounds to bfloat16 (round to nearest even) so a test can feed
the oracle the same BF16 operands a tensor-core kernel consumes and round
the hidden activations at the same points."""
from __future__ import annotations

import numpy as np

SIZES = (19, 256, 256, 256, 256, 6)


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def bf16_round(x):
    """Round float64/float32 values to the nearest bfloat16 (ties to even);
    returns float64 holding exactly representable bf16 values."""
    a = np.asarray(x, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = (u + 0x7FFF + lsb) >> 16 << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(a)
    if np.any(nan):
        out[nan] = np.nan
    return out


def init_params(seed=0, sizes=SIZES):
    """He-uniform weights, zero biases (float64): list of (W [out,in], b [out])."""
    rng = np.random.default_rng(seed)
    ps = []
    for i in range(len(sizes) - 1):
        fan_in = sizes[i]
        lim = np.sqrt(6.0 / fan_in)
        W = rng.uniform(-lim, lim, size=(sizes[i + 1], fan_in))
        b = np.zeros(sizes[i + 1])
        ps.append((W, b))
    return ps


def forward(x, params, round_act=False):
    """y [B,6] and the list of pre-activations z_l (for backward)."""
    h = np.asarray(x, np.float64)
    zs, hs = [], [h]
    L = len(params)
    for l, (W, b) in enumerate(params):
        z = h @ W.T + b
        zs.append(z)
        if l < L - 1:
            h = silu(z)
            if round_act:
                h = bf16_round(h)
            hs.append(h)
        else:
            h = z
    return h, zs, hs


def l1_loss_and_grad(x, t, params, round_act=False, round_grad=False):
    """L1 risk and its gradient w.r.t. every (W, b) by reverse mode.

    round_act: hidden activations rounded to bfloat16 in the forward.
    round_grad: the back-propagated dL/dz of each layer is rounded to
    bfloat16 where it enters a matrix product (the weight gradient
    dz^T h and the next layer's dz W), as a BF16 tensor-core step consumes
    it; the bias gradient sums the unrounded dL/dz."""
    y, zs, hs = forward(x, params, round_act=round_act)
    B = y.shape[0]
    loss = np.abs(y - t).sum() / B
    dy = np.sign(y - t) / B
    grads = [None] * len(params)
    g = dy
    for l in range(len(params) - 1, -1, -1):
        W, b = params[l]
        gq = bf16_round(g) if round_grad else g
        gW = gq.T @ hs[l]
        gb = g.sum(axis=0)
        grads[l] = (gW, gb)
        if l > 0:
            g = (gq @ W) * dsilu(zs[l - 1])
    return loss, grads


def input_grad(x, params, wy, round_act=False, round_grad=False):
    """d(sum wy . y)/dx for weights wy [B,6] (the proxy's input gradient).
    round_act / round_grad as in l1_loss_and_grad: the forward's hidden
    activations, and each layer's back-propagated vector where it enters
    the product with W, rounded to bfloat16."""
    y, zs, hs = forward(x, params, round_act=round_act)
    g = np.asarray(wy, np.float64)
    for l in range(len(params) - 1, -1, -1):
        W, _ = params[l]
        gq = bf16_round(g) if round_grad else g
        g = gq @ W
        if l > 0:
            g = g * dsilu(zs[l - 1])
    return g


def adam_step(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step in place; state = dict(t, m, v)."""
    if not state:
        state["t"] = 0
        state["m"] = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
        state["v"] = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
    state["t"] += 1
    t = state["t"]
    out = []
    for i, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
        new = []
        for j, (p, g) in enumerate(((W, gW), (b, gb))):
            m = state["m"][i][j]
            v = state["v"][i][j]
            m[...] = b1 * m + (1 - b1) * g
            v[...] = b2 * v + (1 - b2) * g * g
            mh = m / (1 - b1 ** t)
            vh = v / (1 - b2 ** t)
            p = p - lr * mh / (np.sqrt(vh) + eps)
            new.append(p)
        out.append(tuple(new))
    return out
