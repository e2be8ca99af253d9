"""Host logic of the autotuner (tune.autotune) on CPU, with srp_force,
srp_build_bvh and the CUDA synchronisation replaced by fakes: the candidate
grid, the chunks per item derived from rays per work unit, whole-grid
versus strided sampling, and the choice of the fastest candidate."""
import types

import pytest

torch = pytest.importorskip("torch")


def _run(monkeypatch, **kw):
    from paper_2602_10712_gb300 import tune
    calls = []

    def fake_force(ctx, bvhs, rho, sun, com, **opts):
        calls.append(dict(opts, n_bvh=len(bvhs), n_sun=int(sun.shape[-2])))
        # pretend width 4, variant 6 and 1024 chunks per item are fastest
        t = 1.0 + 0.1 * (opts["kernel_variant"] != 6) + 0.2 * (opts.get("chunks_per_item") != 1024)
        t += 0.5 * (bvhs[0].w != 4)
        fake_force.clock += t

    fake_force.clock = 0.0
    monkeypatch.setattr(tune, "srp_force", fake_force)
    monkeypatch.setattr(tune, "srp_build_bvh", lambda ctx, v, t, g, w: types.SimpleNamespace(w=w, close=lambda: None))
    monkeypatch.setattr(tune.time, "perf_counter", lambda: fake_force.clock)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    mesh = types.SimpleNamespace(verts=None, tris=None, group=None)
    sun = torch.zeros((64, 3), dtype=torch.float64)
    best, table = tune.autotune(None, [mesh, mesh], torch.zeros((2, 4, 2)), sun, torch.zeros((2, 3)),
                                rays_x=1024, max_bounces=3, sample_suns=8, **kw)
    return best, table, calls


def test_candidates_and_best(monkeypatch):
    best, table, calls = _run(monkeypatch)
    assert len(table) == 2 * 3 * 4                      # widths x variants x rays per unit
    assert best == {"width": 4, "kernel_variant": 6, "chunks_per_item": 1024}
    # whole grids: no ray subset, chunks = ceil(rays per item / rays per unit)
    cpis = sorted({c["chunks_per_item"] for c in calls})
    assert cpis == [0, 64, 256, 1024]                    # 0 = the library's own plan
    assert all("ray_count" not in c for c in calls)
    assert all(c["n_sun"] == 8 and c["n_bvh"] == 2 for c in calls)
    # every candidate is timed after one untimed call, `repeats` times
    assert len(calls) == len(table) * 3


def test_strided_sample(monkeypatch):
    best, table, calls = _run(monkeypatch, sample_rays=16384, rays_per_unit=(0, 4096), widths=(4,),
                              variants=(6,))
    assert len(table) == 2
    stride = 1024 * 1024 // 16384
    assert all(c["ray_stride"] == stride and c["ray_count"] == 16384 and c["ray_offset"] == 0 for c in calls)
    assert sorted({c["chunks_per_item"] for c in calls}) == [0, 4]
