"""GPU parity of the tensor-core proxy network (srp_mlp_*) against the FP64
numpy oracle (oracle/mlp.py) fed the same BF16 operands: weights and inputs
rounded to bfloat16, hidden activations rounded to bfloat16 at the same
points as the kernel.  What remains is FP32 (kernel) vs FP64 (oracle)
accumulation and rare one-ulp BF16 rounding flips of an activation.  Their
RMS effect does not depend on the batch (measured 4.3e-4 rms(y) at 1,000 rows,
4.9e-4 at 58,445) but the largest one grows with the number of rows (6.1e-3
and 1.3e-2 rms(y)).  The forward test therefore bounds the RMS deviation
(3e-3 rms(y)) and the largest one (5e-2 rms(y)); an operand-layout or
descriptor error (wrong row/column pairing) gives O(rms) differences, at
least 20x above either bound."""
import numpy as np
import pytest

from oracle import mlp as omlp

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def flat(params):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params]).astype(np.float32)


def unflat(v):
    out, o = [], 0
    for i in range(5):
        a, b = omlp.SIZES[i], omlp.SIZES[i + 1]
        W = v[o:o + a * b].reshape(b, a); o += a * b
        bb = v[o:o + b]; o += b
        out.append((W.astype(np.float64), bb.astype(np.float64)))
    return out


def inputs(B, seed):
    rng = np.random.default_rng(seed)
    e = rng.normal(size=(B, 3)); e /= np.linalg.norm(e, axis=1, keepdims=True)
    rho = rng.uniform(0, 0.5, size=(B, 14))
    hin = rng.uniform(-1.5, 1.5, size=(B, 2))
    return np.concatenate([e, rho, hin], axis=1).astype(np.float32)


def oracle_bf16(x, p):
    pb = [(omlp.bf16_round(W), b) for W, b in p]
    y, _, _ = omlp.forward(omlp.bf16_round(x), pb, round_act=True)
    return y


@pytest.fixture(scope="module")
def srp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_10712_gb300 as srp
    return srp


# 58,445 rows: three 128-row tiles per CTA of the persistent forward kernel
# on 152 SMs (weights streamed across tiles, next inputs prefetched) and a
# ragged last tile
@pytest.mark.parametrize("B", [1, 129, 1000, 3 * 128 * 152 + 77])
def test_forward_parity(srp, B):
    ctx = srp.Context(0)
    p = omlp.init_params(seed=7)
    p = [(W, np.random.default_rng(l).normal(size=b.shape) * 0.1) for l, (W, b) in enumerate(p)]
    net = srp.MLP(ctx, flat(p))
    x = inputs(B, seed=B)
    y = net.infer(x)
    yo = oracle_bf16(x, unflat(flat(p)))
    rms = np.sqrt(np.mean(yo ** 2))
    err = np.abs(y - yo)
    assert np.sqrt(np.mean(err ** 2)) <= 3e-3 * rms, (np.sqrt(np.mean(err ** 2)), rms)
    assert err.max() <= 5e-2 * rms, (err.max(), rms)
    # element by element within each output's own scale (force and torque
    # components differ in magnitude): a wrong row or column pairing in one
    # tile moves its elements by O(rms) of that output
    col = np.sqrt(np.mean(yo ** 2, axis=0)) + 1e-30
    assert np.all(err <= 5e-2 * col), ("per output", (err / col).max())


def test_params_roundtrip_and_device_mode(srp):
    ctx = srp.Context(0)
    net = srp.MLP(ctx, seed=3)
    p = net.params()
    assert p.shape == (srp.mlp_param_count(),) and np.all(np.isfinite(p))
    x = inputs(300, seed=1)
    yh = net.infer(x)
    dev = torch.device("cuda:0")
    yd = net.infer(torch.from_numpy(x).to(dev))
    torch.cuda.synchronize()
    assert np.array_equal(yd.cpu().numpy(), yh)
    net.set_params(p * 0.5)
    assert np.array_equal(net.params(), (p * 0.5).astype(np.float32))


def _grad_flat(grads):
    return np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])


def _elementwise(g, go, what, el=1e-2, rm=1e-3):
    """Every element within el * rms(go) and the RMS deviation within
    rm * rms(go): a layout or descriptor error confined to one row block or
    one K chunk moves its elements by O(rms) and fails the first bound."""
    scale = np.sqrt(np.mean(go ** 2)) + 1e-30
    dev = np.abs(g - go)
    assert dev.max() <= el * scale, (what, "max", dev.max() / scale)
    assert np.sqrt(np.mean(dev ** 2)) <= rm * scale, (what, "rms", np.sqrt(np.mean(dev ** 2)) / scale)


# 1,000 samples: eight 128-row tiles, the last one ragged, each on a pair of
# CTAs (two-CTA clusters, half the features each); 12,000 samples: 94 tiles,
# one CTA each
@pytest.mark.parametrize("B", [1000, 12000])
def test_training_gradient_parity(srp, B):
    """One L1 gradient on B samples vs the FP64 oracle fed the same BF16 weights and inputs, with
    the hidden activations and every back-propagated dL/dz rounded to BF16
    where the kernel's GEMMs consume them (oracle round_act, round_grad).
    Targets sit 0.2-1.0 away from the oracle's outputs on either side, so
    the sign of y - t (an integer decided by floating point) is the same on
    both sides.  Element by element, per parameter block: |g - g_or| <=
    1e-2 rms(g_or) for every element and 1e-3 rms(g_or) in RMS.  What
    remains is FP32 vs FP64 accumulation and one-ulp BF16 flips where the
    two sides' values straddle a rounding boundary."""
    ctx = srp.Context(0)
    p = omlp.init_params(seed=11)
    p = [(W, np.random.default_rng(40 + l).normal(size=b.shape) * 0.1) for l, (W, b) in enumerate(p)]
    net = srp.MLP(ctx, flat(p))
    x = inputs(B, seed=5)
    pb = [(omlp.bf16_round(W), b) for W, b in unflat(flat(p))]
    xb = omlp.bf16_round(x)
    yo = omlp.forward(xb, pb, round_act=True)[0]
    rng = np.random.default_rng(9)
    t = (yo + rng.choice([-1.0, 1.0], size=yo.shape) * rng.uniform(0.2, 1.0, size=yo.shape)).astype(np.float32)
    loss, g = net.train_step(x, t, lr=0.0, want_grad=True)
    lo, go = omlp.l1_loss_and_grad(xb, t.astype(np.float64), pb, round_act=True, round_grad=True)
    assert abs(loss - lo) <= 1e-4 * lo, (loss, lo)
    go = _grad_flat(go)
    o = 0
    for l in range(5):
        a, b = omlp.SIZES[l], omlp.SIZES[l + 1]
        for n, name in ((a * b, "W"), (b, "b")):
            _elementwise(g[o:o + n], go[o:o + n], (l, name))
            o += n


def test_adam_step_parity(srp):
    ctx = srp.Context(0)
    p = omlp.init_params(seed=12)
    v0 = flat(p)
    net = srp.MLP(ctx, v0)
    x = inputs(512, seed=6)
    t = np.random.default_rng(2).normal(size=(512, 6)).astype(np.float32)
    _, g = net.train_step(x, t, lr=1e-3, want_grad=True)
    v1 = net.params()
    q = omlp.adam_step(unflat(v0), [(gW, gb) for gW, gb in unflat(g)], {}, lr=1e-3)
    vo = np.concatenate([np.concatenate([W.ravel(), b]) for W, b in q])
    assert np.allclose(v1, vo, rtol=1e-5, atol=1e-7)


def test_adam_repacks_both_layouts(srp):
    """The Adam kernel writes each updated weight, rounded to BF16, into the
    forward and the transposed packed layouts: after three steps the network
    infers and back-propagates bit for bit like a fresh network packed from
    its updated parameters."""
    ctx = srp.Context(0)
    net = srp.MLP(ctx, flat(omlp.init_params(seed=13)))
    x = inputs(3000, seed=9)
    t = np.random.default_rng(4).normal(size=(3000, 6)).astype(np.float32)
    for _ in range(3):
        net.train_step(x, t, lr=1e-2, want_loss=False)
    fresh = srp.MLP(ctx, net.params())
    assert np.array_equal(net.infer(x), fresh.infer(x))
    wy = np.random.default_rng(5).normal(size=(3000, 6)).astype(np.float32)
    assert np.array_equal(net.grad_input(x, wy), fresh.grad_input(x, wy))


def test_train_epoch_matches_gathered_steps(srp):
    """srp_mlp_train_epoch (each batch gathered by row number inside the
    training forward, the steps queued by one call) against
    srp_mlp_train_step on the same batches gathered on the host, from the
    same parameters, with the same learning rates: batches of 1,000 rows
    (eight tiles, the last ragged) drawn with repeats from 5,000.  The two
    differ only in the order of the weight gradient's FP32 atomic sums, so
    after three Adam steps (each moving a weight by about lr) almost every
    parameter agrees to 1e-2 lr and the losses to 1e-5; a batch gathered
    from the wrong rows moves most parameters by O(lr)."""
    ctx = srp.Context(0)
    n, batch, steps = 5000, 1000, 3
    rng = np.random.default_rng(31)
    x = inputs(n, seed=21)
    t = rng.normal(size=(n, 6)).astype(np.float32)
    idx = rng.integers(0, n, size=steps * batch).astype(np.int32)
    lrs = np.array([1e-3, 7e-4, 4e-4], np.float32)
    p0 = flat(omlp.init_params(seed=14))
    a, b = srp.MLP(ctx, p0), srp.MLP(ctx, p0)
    dev = torch.device("cuda", 0)
    a.train_epoch(torch.from_numpy(x).to(dev), torch.from_numpy(t).to(dev), torch.from_numpy(idx).to(dev), batch, lrs)
    for s in range(steps):
        rows = idx[s * batch:(s + 1) * batch]
        b.train_step(x[rows], t[rows], float(lrs[s]), want_loss=False)
    pa, pb = a.params(), b.params()
    d = np.abs(pa - pb)
    assert np.mean(d > 1e-2 * lrs[0]) < 1e-3, np.mean(d > 1e-2 * lrs[0])
    assert d.max() <= 2.0 * lrs.sum(), d.max()
    assert np.mean(np.abs(pa - p0) > 0.1 * lrs[0]) > 0.5   # the steps did move the weights
    la, _ = a.train_step(x[:2000], t[:2000], 0.0)
    lb, _ = b.train_step(x[:2000], t[:2000], 0.0)
    assert abs(la - lb) <= 1e-5 * lb, (la, lb)


def test_train_epoch_rejects_rows_outside_the_data_set(srp):
    """A row number outside 0..n-1 is not read: the forward reads a zero row
    in its place and flags it, the next synchronisation reports
    SRP_EDEVICE_LIMIT, and the context trains normally afterwards."""
    ctx = srp.Context(0)
    n, batch = 600, 256
    x = inputs(n, seed=22)
    t = np.random.default_rng(3).normal(size=(n, 6)).astype(np.float32)
    dev = torch.device("cuda", 0)
    xd, td = torch.from_numpy(x).to(dev), torch.from_numpy(t).to(dev)
    net = srp.MLP(ctx, seed=2)
    for bad in (n, -1):
        idx = np.arange(batch, dtype=np.int32)
        idx[77] = bad
        net.train_epoch(xd, td, torch.from_numpy(idx).to(dev), batch, np.array([1e-3], np.float32))
        with pytest.raises(srp.SRPError) as e:
            srp.srp_sync(ctx)
        assert e.value.code == srp.SRP_EDEVICE_LIMIT and "training batch index" in str(e.value)
    net.train_epoch(xd, td, torch.arange(batch, dtype=torch.int32, device=dev), batch, np.array([1e-3], np.float32))
    srp.srp_sync(ctx)
    with pytest.raises(srp.SRPError, match="SRP_EINVAL"):
        net.train_epoch(xd, td, torch.arange(batch, dtype=torch.int32, device=dev), batch,
                        np.array([0.0], np.float32))


def test_training_reduces_loss(srp):
    """Fit a smooth synthetic map (a fixed random 19->6 linear map + tanh):
    200 Adam steps reduce the L1 loss at least 5x."""
    ctx = srp.Context(0)
    net = srp.MLP(ctx, seed=1)
    rng = np.random.default_rng(3)
    A = rng.normal(size=(19, 6))
    x = inputs(8192, seed=7)
    t = np.tanh(x @ A).astype(np.float32)
    l0, _ = net.train_step(x, t, lr=0.0)
    for _ in range(200):
        net.train_step(x, t, lr=2e-3, want_loss=False)
    l1, _ = net.train_step(x, t, lr=0.0)
    assert l1 < l0 / 5, (l0, l1)


@pytest.mark.parametrize("B", [777, 10001])
def test_input_gradient_parity(srp, B):
    """srp_mlp_grad_input vs the FP64 oracle's input gradient with the same
    BF16 weights and inputs, the hidden activations and each back-propagated
    vector (wy included) rounded to BF16 where the kernel's GEMMs consume
    them (round_act, round_grad); row by row, every element within 2e-2 of
    its row's RMS, and the RMS deviation over the batch within 1e-3; host
    and device modes agree bit for bit.  The per-row bound is twice the
    training gradient's: a row's input gradient ends in one dot product per
    element over 256 terms of both signs, so rows whose result cancels to a
    small RMS carry the terms' FP32/BF16 rounding relatively larger (the
    worst of 777 rows measured 1.1e-2).  777 rows run on CTA pairs, 10,001
    rows (79 tiles) on one CTA per tile."""
    ctx = srp.Context(0)
    p = omlp.init_params(seed=21)
    net = srp.MLP(ctx, flat(p))
    x = inputs(B, seed=8)
    wy = np.random.default_rng(3).normal(size=(B, 6)).astype(np.float32)
    gx = net.grad_input(x, wy)
    pb = [(omlp.bf16_round(W), b) for W, b in unflat(flat(p))]
    go = omlp.input_grad(omlp.bf16_round(x), pb, wy.astype(np.float64), round_act=True, round_grad=True)
    row = np.sqrt(np.mean(go ** 2, axis=1, keepdims=True)) + 1e-30
    dev = np.abs(gx - go)
    assert np.all(dev <= 2e-2 * row), ("max per row", (dev / row).max())
    assert np.sqrt(np.mean(dev ** 2)) <= 1e-3 * np.sqrt(np.mean(go ** 2)), np.sqrt(np.mean(dev ** 2))
    dev_ = torch.device("cuda", 0)
    gd = net.grad_input(torch.from_numpy(x).to(dev_), torch.from_numpy(wy).to(dev_))
    torch.cuda.synchronize()
    assert np.array_equal(gd.cpu().numpy(), gx)


def test_save_load_roundtrip(srp, tmp_path):
    ctx = srp.Context(0)
    a = srp.MLP(ctx, seed=4)
    b = srp.MLP(ctx, seed=5)
    f = str(tmp_path / "proxy.bin")
    a.save(f)
    b.load_file(f)
    assert np.array_equal(a.params(), b.params())
    x = inputs(64, seed=1)
    assert np.array_equal(a.infer(x), b.infer(x))
    bad = tmp_path / "bad.bin"
    bad.write_bytes(b"not a parameter file")
    with pytest.raises(srp.SRPError, match="SRP_EINVAL"):
        b.load_file(str(bad))
