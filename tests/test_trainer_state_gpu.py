"""Checkpoint and resume of the proxy's training (srp_mlp_save_state /
srp_mlp_load_state through the C ABI): parameters, Adam moments and the
step count round-trip exactly, and a network resumed from the file takes
the same next Adam step as the one that wrote it."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_state_roundtrip_and_resume(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_10712_gb300 as srp
    ctx = srp.Context(0)
    rng = np.random.default_rng(0)
    x = rng.uniform(-1.0, 1.0, size=(2048, 19)).astype(np.float32)
    t = np.tanh(x @ rng.normal(size=(19, 6))).astype(np.float32)
    lr = 2e-3
    a = srp.MLP(ctx, seed=2)
    for _ in range(5):
        a.train_step(x, t, lr=lr, want_loss=False)
    f1 = str(tmp_path / "a.state")
    a.save_state(f1)
    raw = open(f1, "rb").read()
    assert raw[:8] == b"SRPMLS1\0"
    n, step = np.frombuffer(raw[8:24], np.int64)
    assert n == srp.mlp_param_count() and step == 5 and len(raw) == 24 + 12 * n
    # another network takes over the whole state: saving it again gives the same bytes
    b = srp.MLP(ctx, seed=9)
    b.load_state(f1)
    f2 = str(tmp_path / "b.state")
    b.save_state(f2)
    assert open(f2, "rb").read() == raw
    # the next step: the same loss before it and the same Adam update (up to
    # the FP32 order of the atomically added loss and weight-gradient sums);
    # a state without its moments or step would change the typical update by
    # a sizeable fraction of the learning rate
    la, _ = a.train_step(x, t, lr=lr)
    lb, _ = b.train_step(x, t, lr=lr)
    assert abs(la - lb) <= 1e-4 * abs(la), (la, lb)
    d = np.abs(a.params() - b.params())
    assert np.median(d) <= 1e-2 * lr, (np.median(d), d.max())
    # a file of another kind is refused and leaves the network as it was
    p_before = b.params()
    bad = tmp_path / "bad.state"
    bad.write_bytes(b"SRPMLP1\0" + raw[8:])
    with pytest.raises(srp.SRPError, match="SRP_EINVAL"):
        b.load_state(str(bad))
    assert np.array_equal(b.params(), p_before)
