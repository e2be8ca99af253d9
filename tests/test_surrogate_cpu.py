"""Host logic of the proxy's data pipeline on CPU: design and sun sampling
ranges, the network input encoding, and trace_dataset's chunked calls
(srp_force replaced by a stand-in that records its arguments), so the
design-vector layout, the per-design suns and the counter offsets are
checked without a GPU."""
import math
import types

import numpy as np


def test_sampling_and_encoding():
    from paper_2602_10712_gb300 import surrogate as S
    th = S.sample_designs(4096, seed=3)
    assert th.shape == (4096, 16)
    assert th[:, :14].min() >= 0.0 and th[:, :14].max() <= 0.5
    assert th[:, 14:].min() >= -math.pi / 2 and th[:, 14:].max() <= math.pi / 2
    assert np.array_equal(th, S.sample_designs(4096, seed=3))
    sun = S.sample_suns(4096, seed=4)
    assert np.allclose(np.linalg.norm(sun, axis=1), 1.0)
    x = S.encode(sun, th)
    assert x.dtype == np.float32 and x.shape == (4096, 19)
    assert np.array_equal(x[:, :3], sun.astype(np.float32))
    assert x[:, 3:].min() >= -1.0 and x[:, 3:].max() <= 1.0
    assert np.allclose(x[:, 3:17], 4.0 * th[:, :14] - 1.0, atol=1e-6)
    assert np.allclose(x[:, 17:], th[:, 14:] / (math.pi / 2), atol=1e-6)


def test_trace_dataset_chunks_and_layout(monkeypatch):
    from paper_2602_10712_gb300 import surrogate as S
    import workloads as W
    mesh = W.box_wing_7group()
    calls = []

    def fake_instantiate(verts, vhinge, hinges, angles):
        return np.asarray(angles, np.float64)           # stands for the instantiated design

    def fake_build(ctx, v, tris, group, width):
        return types.SimpleNamespace(angles=v, close=lambda: None)

    def fake_force(ctx, bvhs, rho, sun, com, **kw):
        calls.append(kw)
        D, Sn = sun.shape[0], sun.shape[1]
        assert kw["sun_per_design"] == 1 and rho.shape == (D, 7, 2) and com.shape == (D, 3)
        out = np.zeros((D, Sn, 6))
        for d in range(D):
            # a force that records the design's reflectances, angles and suns
            out[d, :, 0] = rho[d, :, 0].sum()
            out[d, :, 1] = rho[d, :, 1].sum()
            out[d, :, 2] = bvhs[d].angles[0]
            out[d, :, 3:] = sun[d]
        return out

    monkeypatch.setattr(S, "srp_design_instantiate", fake_instantiate)
    monkeypatch.setattr(S, "srp_build_bvh", fake_build)
    monkeypatch.setattr(S, "srp_force", fake_force)
    theta = S.sample_designs(1100, seed=1)
    sun, ft = S.trace_dataset(None, mesh, theta, suns_per_design=3, rays=64, bounces=2, seed=7, sun_seed=8)
    assert sun.shape == (1100, 3, 3) and ft.shape == (1100, 3, 6)
    assert [c["design_base"] for c in calls] == [0, 512, 1024]
    assert all(c["rays_x"] == 64 and c["max_bounces"] == 2 and c["seed"] == 7 for c in calls)
    assert np.allclose(ft[:, 0, 0], theta[:, :7].sum(axis=1), rtol=1e-6)
    assert np.allclose(ft[:, 0, 1], theta[:, 7:14].sum(axis=1), rtol=1e-6)
    assert np.array_equal(ft[:, 0, 2], theta[:, 14])
    assert np.array_equal(ft[:, :, 3:], sun)


def test_fit_resumes_after_a_crash(monkeypatch, tmp_path):
    """Training checkpoints: a run that crashes after two of four epochs and
    is resumed from its checkpoint ends with exactly the state of an
    uninterrupted run (same batches in the same order, same learning
    rates).  The network is a stand-in whose update depends on the batch
    order and the learning rate; the real trainer state (srp_mlp_save_state)
    is checked on the GPU."""
    from paper_2602_10712_gb300 import surrogate as S
    crash = {"at": None}

    class Net:
        def __init__(self, ctx, params=None, seed=0):
            self.w, self.t = 0.0, 0

        def train_step(self, xb, yb, lr, want_loss=True, want_grad=False):
            if crash["at"] is not None and self.t == crash["at"]:
                raise RuntimeError("simulated crash")
            self.w = 0.999 * self.w + lr * float(xb[:, 0].sum() + 2.0 * yb[:, 1].sum() + xb[0, 5])
            if lr > 0:
                self.t += 1
            return (self.w if want_loss else None), None

        def save_state(self, path):
            with open(path, "wb") as f:
                np.save(f, np.array([self.w, self.t]))

        def load_state(self, path):
            with open(path, "rb") as f:
                a = np.load(f)
            self.w, self.t = float(a[0]), int(a[1])

    def data(ctx, mesh, theta, spd, rays, bounces, seed, sun_seed):
        r = np.random.default_rng(seed)
        return S.sample_suns(theta.shape[0] * spd, sun_seed).reshape(-1, spd, 3), r.normal(size=(theta.shape[0], spd, 6))

    monkeypatch.setattr(S, "MLP", Net)
    monkeypatch.setattr(S, "trace_dataset", data)
    kw = dict(n_designs=64, suns_per_design=16, epochs=4, batch=128, lr=1e-2, seed=3, device="cpu")
    ref, info = S.fit(None, None, **kw)
    assert info["steps"] == 32
    prefix = str(tmp_path / "ckpt")
    crash["at"] = 16                       # the first step of the third epoch
    try:
        S.fit(None, None, checkpoint=prefix, **kw)
        raise AssertionError("the stand-in should have crashed")
    except RuntimeError as e:
        assert "simulated crash" in str(e)
    meta = np.load(prefix + ".npz")
    assert int(meta["epoch"]) == 2 and int(meta["step"]) == 16
    crash["at"] = None
    res, info2 = S.fit(None, None, checkpoint=prefix, resume=True, **kw)
    assert info2["steps"] == 32 and res.net.t == 32
    assert res.net.w == ref.net.w
    # without resume the same call starts over (and gives the same result)
    again, _ = S.fit(None, None, checkpoint=prefix, **kw)
    assert again.net.w == ref.net.w


def test_evaluate_falls_back_to_the_tracer_outside_the_domain(monkeypatch):
    """Surrogate.evaluate answers with the proxy inside its training domain
    and with the tracer (instantiate, BVH, srp_force) outside it; the
    tracer receives the row's reflectance layout, hinge angles and sun."""
    from paper_2602_10712_gb300 import surrogate as S
    import workloads as W
    traced = []

    class Net:
        def infer(self, x):
            return np.tile(np.arange(6, dtype=np.float32), (x.shape[0], 1))

    def fake_force(ctx, bvhs, rho, sun, com, **kw):
        traced.append((rho.copy(), sun.copy(), bvhs[0].angles.copy(), kw))
        return np.full((1, 1, 6), -7.0)

    monkeypatch.setattr(S, "srp_design_instantiate", lambda v, vh, hg, ang: np.asarray(ang))
    monkeypatch.setattr(S, "srp_build_bvh", lambda ctx, v, t, g, w: type("B", (), {"angles": v, "close": lambda self: None})())
    monkeypatch.setattr(S, "srp_force", fake_force)
    sur = S.Surrogate(None, Net(), np.zeros(6), np.ones(6))
    theta = S.sample_designs(5, seed=2)
    theta[1, 3] = 0.6                      # a reflectance above the training range
    theta[3, 15] = 2.0                     # a hinge beyond pi/2
    sun = S.sample_suns(5, seed=3)
    assert list(sur.in_domain(theta)) == [True, False, True, False, True]
    ft, tr = sur.evaluate(sun, theta, W.box_wing_7group(), rays=128, bounces=2, seed=4)
    assert list(tr) == [False, True, False, True, False]
    assert np.array_equal(ft[~tr], np.tile(np.arange(6.0), (3, 1)))
    assert np.all(ft[tr] == -7.0) and len(traced) == 2
    for (rho, s, ang, kw), i in zip(traced, (1, 3)):
        assert rho.shape == (1, 7, 2) and np.allclose(rho[0, :, 0], theta[i, :7]) and np.allclose(rho[0, :, 1], theta[i, 7:14])
        assert np.array_equal(s, sun[i:i + 1]) and np.array_equal(ang, theta[i, 14:])
        assert kw["rays_x"] == 128 and kw["max_bounces"] == 2 and kw["seed"] == 4
