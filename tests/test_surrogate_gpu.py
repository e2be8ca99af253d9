"""The proxy trained on tracer data (Sec. 3.3), small scale: it must track
held-out Monte Carlo forces traced with 16x the training rays and answer
far faster than the tracer on the same GPU (what the learned part gains)."""
import time

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_surrogate_fits_and_beats_tracer():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_10712_gb300 as srp
    from paper_2602_10712_gb300 import surrogate as S
    ctx = srp.Context(0)
    mesh = W.box_wing_7group()
    sur, info = S.fit(ctx, mesh, n_designs=1024, suns_per_design=64, rays=128, bounces=3, epochs=40, batch=4096,
                      lr=2e-3, seed=1)
    err = S.force_rms_error(sur, ctx, mesh, n_designs=64, suns_per_design=8, rays=512, bounces=3, seed=5)
    assert err < 0.10, err
    # speed: surrogate evaluations vs tracer evaluations (256^2 rays each)
    dev = torch.device("cuda:0")
    x = torch.from_numpy(S.encode(S.sample_suns(1 << 20, 3), S.sample_designs(1 << 20, 4))).to(dev)
    y = sur.net.infer(x)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(3):
        sur.net.infer(x, y)
    torch.cuda.synchronize()
    nn_rate = 3 * (1 << 20) / (time.perf_counter() - t0)
    th = S.sample_designs(1, 8)
    v = srp.srp_design_instantiate(mesh.verts, mesh.vhinge, mesh.hinges, th[0, 14:])
    b = srp.srp_build_bvh(ctx, v, mesh.tris, mesh.group, 4)
    rho = np.zeros((1, 7, 2), np.float32); rho[0, :, 0] = th[0, :7]; rho[0, :, 1] = th[0, 7:14]
    suns = torch.from_numpy(S.sample_suns(4096, 9)).to(dev)
    r_t = torch.from_numpy(rho).to(dev); c_t = torch.zeros((1, 3), dtype=torch.float64, device=dev)
    srp.srp_force(ctx, [b], r_t, suns, c_t, rays_x=256, max_bounces=3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    srp.srp_force(ctx, [b], r_t, suns, c_t, rays_x=256, max_bounces=3)
    torch.cuda.synchronize()
    mc_rate = 4096 / (time.perf_counter() - t0)
    assert nn_rate >= 100 * mc_rate, (nn_rate, mc_rate)


def test_fit_resumes_on_the_gpu(tmp_path, monkeypatch):
    """fit's GPU path (one srp_mlp_train_epoch call per epoch over a batch
    order drawn on the device from (seed, epoch)) interrupted in its third
    epoch and resumed from its checkpoint ends where an uninterrupted run
    ends: same step count, parameters equal up to the FP32 order of the
    weight gradient's atomic sums.  Under the L1 loss that order can flip
    the sign of a near-zero residual, so the two runs drift apart a little
    over the last steps: the median parameter difference must stay below a
    tenth of the median distance the training moved them (a resumed run
    that replayed another batch order or restarted the learning-rate
    schedule differs by a sizeable fraction of that distance)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_10712_gb300 as srp
    from paper_2602_10712_gb300 import surrogate as S
    ctx = srp.Context(0)
    mesh = W.box_wing_7group()
    kw = dict(n_designs=32, suns_per_design=16, rays=64, bounces=1, epochs=4, batch=128, lr=1e-2, seed=3)
    ref, info = S.fit(ctx, mesh, **kw)
    assert info["steps"] == 16
    calls = {"n": 0}

    class Crashing(srp.MLP):
        def train_epoch(self, *a, **k):
            calls["n"] += 1
            if calls["n"] == 3:
                raise RuntimeError("simulated crash")
            return super().train_epoch(*a, **k)

    prefix = str(tmp_path / "ckpt")
    monkeypatch.setattr(S, "MLP", Crashing)
    with pytest.raises(RuntimeError, match="simulated crash"):
        S.fit(ctx, mesh, checkpoint=prefix, **kw)
    monkeypatch.setattr(S, "MLP", srp.MLP)
    meta = np.load(prefix + ".npz")
    assert int(meta["epoch"]) == 2 and int(meta["step"]) == 8
    res, info2 = S.fit(ctx, mesh, checkpoint=prefix, resume=True, **kw)
    assert info2["steps"] == 16
    d = np.abs(res.net.params() - ref.net.params())
    moved = np.abs(ref.net.params() - S.MLP(ctx, seed=3).params())
    assert np.median(moved) > 0.3 * kw["lr"], np.median(moved)
    assert np.median(d) <= 0.1 * np.median(moved), (np.median(d), np.median(moved))
