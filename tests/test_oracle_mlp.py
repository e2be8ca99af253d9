"""Pins of the FP64 proxy-network oracle (oracle/mlp.py): reverse-mode
gradients against central finite differences, Adam's first step against its
closed form (the bias-corrected update is -lr*sign(g)), SiLU special values,
and bfloat16 rounding (round to nearest even) on hand-worked ties."""
import numpy as np

from oracle import mlp


def _small():
    return mlp.init_params(seed=3, sizes=(19, 16, 16, 16, 16, 6))


def test_silu_special_values():
    assert mlp.silu(0.0) == 0.0 and mlp.dsilu(0.0) == 0.5
    assert abs(mlp.silu(40.0) - 40.0) < 1e-12 and abs(mlp.silu(-40.0)) < 1e-15
    z = np.linspace(-5, 5, 11)
    fd = (mlp.silu(z + 1e-6) - mlp.silu(z - 1e-6)) / 2e-6
    assert np.allclose(fd, mlp.dsilu(z), atol=1e-8)


def test_bf16_round_ties_to_even():
    one = 1.0
    assert mlp.bf16_round(one) == 1.0
    assert mlp.bf16_round(1.0 + 2 ** -8) == 1.0                  # tie -> even mantissa 0
    assert mlp.bf16_round(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6     # tie -> even mantissa 2
    assert mlp.bf16_round(1.0 + 2 ** -7) == 1.0 + 2 ** -7         # representable
    assert mlp.bf16_round(-3.0) == -3.0


def test_loss_gradient_matches_fd():
    rng = np.random.default_rng(0)
    p = _small()
    x = rng.normal(size=(32, 19))
    t = rng.normal(size=(32, 6)) * 10.0  # far from outputs: |y-t| has no kink nearby
    loss, grads = mlp.l1_loss_and_grad(x, t, p)
    h = 1e-6
    for l, (i, j) in [(0, (3, 5)), (2, (7, 1)), (4, (2, 9))]:
        W, b = p[l]
        Wp = W.copy(); Wp[i, j] += h
        Wm = W.copy(); Wm[i, j] -= h
        pp = list(p); pp[l] = (Wp, b)
        pm = list(p); pm[l] = (Wm, b)
        fd = (mlp.l1_loss_and_grad(x, t, pp)[0] - mlp.l1_loss_and_grad(x, t, pm)[0]) / (2 * h)
        assert abs(fd - grads[l][0][i, j]) <= 1e-6 * max(1.0, abs(fd)), (l, fd, grads[l][0][i, j])
    for l in (1, 4):
        W, b = p[l]
        bp = b.copy(); bp[1] += h
        bm = b.copy(); bm[1] -= h
        pp = list(p); pp[l] = (W, bp)
        pm = list(p); pm[l] = (W, bm)
        fd = (mlp.l1_loss_and_grad(x, t, pp)[0] - mlp.l1_loss_and_grad(x, t, pm)[0]) / (2 * h)
        assert abs(fd - grads[l][1][1]) <= 1e-6 * max(1.0, abs(fd))


def test_input_gradient_matches_fd():
    rng = np.random.default_rng(1)
    p = _small()
    x = rng.normal(size=(4, 19))
    wy = rng.normal(size=(4, 6))
    g = mlp.input_grad(x, p, wy)
    h = 1e-6
    for j in (0, 7, 18):
        xp = x.copy(); xp[:, j] += h
        xm = x.copy(); xm[:, j] -= h
        fd = ((mlp.forward(xp, p)[0] - mlp.forward(xm, p)[0]) * wy).sum(axis=1) / (2 * h)
        assert np.allclose(fd, g[:, j], rtol=1e-6, atol=1e-9)


def test_adam_first_step_closed_form():
    p = [(np.array([[1.0, -2.0]]), np.array([0.5]))]
    g = [(np.array([[3.0, -0.25]]), np.array([1e-3]))]
    st = {}
    q = mlp.adam_step(p, g, st, lr=0.01)
    # m_hat = g, v_hat = g^2 after one step -> update = -lr * g / (|g| + eps)
    assert np.allclose(q[0][0], [[1.0 - 0.01, -2.0 + 0.01]], atol=1e-9)
    assert np.allclose(q[0][1], [0.5 - 0.01 * 1e-3 / (1e-3 + 1e-8)], atol=1e-12)


def test_forward_against_a_hand_built_network():
    """The forward pass y = W4 s(W3 s(W2 s(W1 s(W0 x + b0) + b1) + b2) + b3) + b4
    (s = SiLU on the hidden layers only, linear output) on a network wired
    by hand: unit 0 of each hidden layer carries x[2] forward through a
    chain of scalars (weights 2, 0.5, -1, 3 and biases 0.1, -0.2, 0.3, 0.4),
    output 5 reads unit 0 with weight -2 plus bias 0.7, outputs 0..4 read
    nothing and keep their biases; the expected values are the same scalar
    chain written out."""
    import math
    sizes = (19, 256, 256, 256, 256, 6)
    p = [(np.zeros((sizes[i + 1], sizes[i])), np.zeros(sizes[i + 1])) for i in range(5)]
    p[0][0][0, 2], p[0][1][0] = 2.0, 0.1
    p[1][0][0, 0], p[1][1][0] = 0.5, -0.2
    p[2][0][0, 0], p[2][1][0] = -1.0, 0.3
    p[3][0][0, 0], p[3][1][0] = 3.0, 0.4
    p[4][0][5, 0], p[4][1][:] = -2.0, [0.1, 0.2, 0.3, 0.4, 0.5, 0.7]
    s = lambda z: z / (1.0 + math.exp(-z))
    for x2 in (-1.5, 0.0, 0.8):
        x = np.zeros((1, 19)); x[0, 2] = x2; x[0, 7] = 9.0      # input 7 is wired to nothing
        h = s(2.0 * x2 + 0.1)
        h = s(0.5 * h - 0.2)
        h = s(-1.0 * h + 0.3)
        h = s(3.0 * h + 0.4)
        want = [0.1, 0.2, 0.3, 0.4, 0.5, -2.0 * h + 0.7]
        y = mlp.forward(x, p)[0][0]
        assert np.allclose(y, want, rtol=1e-14, atol=1e-15), (x2, y, want)


def test_round_grad_single_layer_closed_form():
    """round_grad on a network with no hidden layer (19 -> 6, linear): the
    only back-propagated vector is dL/dy = sign(y - t)/B.  For B = 3 its
    bfloat16 rounding is bf16(1/3) = 0.333984375 = (1/3)(1 + 2^-9), so the
    weight gradient is the exact one times 3 * 0.333984375 = 1.001953125
    (a rounding applied after the product, or to the inputs, gives another
    factor), and the bias gradient, which sums the unrounded vector, is
    exact.  For B = 4, 1/4 is a bfloat16 and nothing changes."""
    rng = np.random.default_rng(5)
    p = [(rng.normal(size=(6, 19)), rng.normal(size=6))]
    for B, factor in ((3, 1.001953125), (4, 1.0)):
        x = rng.normal(size=(B, 19))
        t = rng.normal(size=(B, 6)) * 10.0
        _, g0 = mlp.l1_loss_and_grad(x, t, p)
        _, g1 = mlp.l1_loss_and_grad(x, t, p, round_grad=True)
        assert np.array_equal(g1[0][1], g0[0][1])
        mag = (np.ones((B, 6)) / B).T @ np.abs(x)      # |dL/dy|^T |x|
        assert np.all(np.abs(g1[0][0] - factor * g0[0][0]) <= 1e-14 * mag), B


def test_round_grad_deviation_is_bounded_by_bf16():
    """round_grad on the full network: every back-propagated vector is
    rounded to bfloat16 (relative error <= 2^-9 per element) where it
    enters a product, so the weight gradients differ from the exact ones by
    at most a few times 2^-9 relative to the products of magnitudes
    |g| |h| summed over the batch, and the bias gradient of the last layer
    (which sums the unrounded dL/dy) is exact.  The deviation is also not
    zero: the rounding is applied."""
    rng = np.random.default_rng(6)
    p = mlp.init_params(seed=4)
    x = rng.normal(size=(48, 19))
    t = rng.normal(size=(48, 6)) * 10.0
    _, g0 = mlp.l1_loss_and_grad(x, t, p)
    _, g1 = mlp.l1_loss_and_grad(x, t, p, round_grad=True)
    assert np.array_equal(g1[4][1], g0[4][1])
    # magnitudes: |dL/dz_l|^T |h_l| along the exact backward
    y, zs, hs = mlp.forward(x, p)
    g = np.sign(y - t) / 48
    for l in range(4, -1, -1):
        mag = np.abs(g).T @ np.abs(hs[l])
        dev = np.abs(g1[l][0] - g0[l][0])
        assert np.all(dev <= (5 - l) * 2.0 ** -8 * mag + 1e-18), l
        assert dev.max() > 0.0, l
        if l > 0:
            g = (g @ p[l][0]) * mlp.dsilu(zs[l - 1])


def test_round_grad_input_gradient():
    """input_grad with round_grad: with wy of bfloat16 values and a network
    whose only layer is linear the rounding changes nothing; on the full
    network the deviation from the exact input gradient stays within the
    BF16 bound and is not zero."""
    rng = np.random.default_rng(8)
    p1 = [(rng.normal(size=(6, 19)), rng.normal(size=6))]
    x = rng.normal(size=(5, 19))
    wy = mlp.bf16_round(rng.normal(size=(5, 6)))
    assert np.array_equal(mlp.input_grad(x, p1, wy, round_grad=True), mlp.input_grad(x, p1, wy))
    p = mlp.init_params(seed=9)
    wy = rng.normal(size=(5, 6))
    g0 = mlp.input_grad(x, p, wy)
    g1 = mlp.input_grad(x, p, wy, round_grad=True)
    # magnitude of the exact chain: |wy| |W4| |s'| |W3| ... |W0|
    _, zs, _ = mlp.forward(x, p)
    m = np.abs(wy)
    for l in range(4, -1, -1):
        m = m @ np.abs(p[l][0])
        if l > 0:
            m = m * np.abs(mlp.dsilu(zs[l - 1]))
    dev = np.abs(g1 - g0)
    assert np.all(dev <= 5 * 2.0 ** -8 * m) and dev.max() > 0.0
