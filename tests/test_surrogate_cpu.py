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
