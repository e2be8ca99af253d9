"""srp_force_noalloc: the variant of srp_force for callers that cannot
allocate GPU memory (its partial sums, design table, error word and queue
counter live in fixed arrays inside the library instead of context-owned
scratch).  Checked through the C ABI against srp_force on the same inputs,
on two calls in a row (the second call reuses the arrays the first one left
filled), and on the paths where the two entry points differ: more designs
than one 64-entry design-table launch carries, per-design sun directions,
automatic chunking capped by the fixed array, and full grids whose width is
a multiple of 32 (srp_force skips the batches that cannot meet the scene;
the variant traces them).  This file is collected last."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# the suite's tolerance for two groupings of the same FP32-per-ray sums
RTOL = 1e-6


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _close(a, b, rtol=RTOL):
    """Per item: |dF| <= rtol |F| and |dtau| <= rtol |F| (R = O(1) m here)."""
    a = np.asarray(a).reshape(-1, 6)
    b = np.asarray(b).reshape(-1, 6)
    fn = np.linalg.norm(b[:, :3], axis=1)[:, None] + 1e-300
    return bool(np.all(np.abs(a - b) <= rtol * fn + 1e-15))


def _run_noalloc(srp, bvhs, r_t, s_t, c_t, D, S, dev, **kw):
    out = torch.full((D, S, 6), float("nan"), dtype=torch.float64, device=dev)
    sig = torch.full((D, S, 6), float("nan"), dtype=torch.float64, device=dev)
    st = torch.full((1,), -1, dtype=torch.int32, device=dev)
    srp.srp_force_noalloc(bvhs, r_t, s_t, c_t, out, out_sigma=sig, status=st, **kw)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    return out.cpu().numpy(), sig.cpu().numpy()


def test_noalloc_matches_srp_force_twice():
    _need_gpu()
    import paper_2602_10712_gb300 as srp
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    ctx = srp.Context(0)
    m, rho, _, com = W.config2(4)
    sun = W.fibonacci_directions(6)
    b = srp.srp_build_bvh(ctx, m.verts, m.tris, m.group, 4)
    r_t = torch.from_numpy(rho[None].copy()).to(dev)
    s_t = torch.from_numpy(sun.copy()).to(dev)
    c_t = torch.from_numpy(com[None].copy()).to(dev)
    kw = dict(rays_x=300, rays_y=200, max_bounces=3, seed=5)
    ref = srp.srp_force(ctx, [b], r_t, s_t, c_t, out_sigma=True, **kw)
    torch.cuda.synchronize()
    for call in range(2):
        out, sig = _run_noalloc(srp, [b], r_t, s_t, c_t, 1, 6, dev, **kw)
        assert _close(out, ref[0].cpu().numpy()), call
        assert np.allclose(sig, ref[1].cpu().numpy(), rtol=1e-5, atol=1e-12), call


def test_noalloc_full_grid_multiple_of_32():
    """rays_x % 32 == 0 over the whole grid: both entry points run the
    batch pre-pass (the variant with its tables in its fixed array); the
    sums agree, on two calls in a row."""
    _need_gpu()
    import paper_2602_10712_gb300 as srp
    dev = torch.device("cuda:0")
    ctx = srp.Context(0)
    m, rho, _, com = W.config2(4)
    sun = W.fibonacci_directions(5)
    b = srp.srp_build_bvh(ctx, m.verts, m.tris, m.group, 4)
    r_t = torch.from_numpy(rho[None].copy()).to(dev)
    s_t = torch.from_numpy(sun.copy()).to(dev)
    c_t = torch.from_numpy(com[None].copy()).to(dev)
    kw = dict(rays_x=256, rays_y=192, max_bounces=3, seed=2)
    ref = srp.srp_force(ctx, [b], r_t, s_t, c_t, out_sigma=True, **kw)
    torch.cuda.synchronize()
    for call in range(2):
        out, sig = _run_noalloc(srp, [b], r_t, s_t, c_t, 1, 5, dev, **kw)
        assert _close(out, ref[0].cpu().numpy()), call
        assert np.allclose(sig, ref[1].cpu().numpy(), rtol=1e-5, atol=1e-12), call


def test_noalloc_full_grid_beyond_the_prepass_array():
    """A full 32-aligned grid whose pre-pass tables would not fit the fixed
    16 MiB array (520 suns x 4096 rows: 17 MB): the variant traces every
    ray instead, srp_force skips the empty batches; the sums agree to the
    suite's tolerance, on two calls in a row."""
    _need_gpu()
    import paper_2602_10712_gb300 as srp
    dev = torch.device("cuda:0")
    ctx = srp.Context(0)
    m, rho, _, com = W.config1()
    S = 520
    sun = W.fibonacci_directions(S)
    b = srp.srp_build_bvh(ctx, m.verts, m.tris, m.group, 4)
    r_t = torch.from_numpy(rho[None].copy()).to(dev)
    s_t = torch.from_numpy(sun.copy()).to(dev)
    c_t = torch.from_numpy(com[None].copy()).to(dev)
    kw = dict(rays_x=32, rays_y=4096, max_bounces=1, seed=8)
    assert S * (8 * 4096 + 4) + 128 * S > (16 << 20)
    ref = srp.srp_force(ctx, [b], r_t, s_t, c_t, out_sigma=True, **kw)
    torch.cuda.synchronize()
    for call in range(2):
        out, sig = _run_noalloc(srp, [b], r_t, s_t, c_t, 1, S, dev, **kw)
        assert _close(out, ref[0].cpu().numpy()), call
        assert np.allclose(sig, ref[1].cpu().numpy(), rtol=1e-5, atol=1e-12), call


def _hinged_designs(srp, ctx, n, seed):
    mb = W.box_wing()
    rng = np.random.default_rng(seed)
    bvhs = []
    for _ in range(n):
        ang = rng.uniform(-1.2, 1.2, size=mb.H)
        v = srp.srp_design_instantiate(mb.verts, mb.vhinge, mb.hinges, ang)
        bvhs.append(srp.srp_build_bvh(ctx, v, mb.tris, mb.group, 4))
    return mb, bvhs


def test_noalloc_many_designs_and_sun_per_design():
    """70 designs (two design-table launches, the second partly filled),
    then 2 designs with their own sun directions; chunks_per_item given so
    both entry points cut the rays identically."""
    _need_gpu()
    import paper_2602_10712_gb300 as srp
    dev = torch.device("cuda:0")
    ctx = srp.Context(0)
    D, S = 70, 3
    mb, bvhs = _hinged_designs(srp, ctx, D, 11)
    rho = np.stack([W.random_reflectances(64, seed=d) for d in range(D)]).astype(np.float32)
    com = np.random.default_rng(3).normal(scale=0.1, size=(D, 3))
    sun = W.random_unit_vectors(S, 4)
    r_t = torch.from_numpy(rho).to(dev)
    s_t = torch.from_numpy(sun).to(dev)
    c_t = torch.from_numpy(com).to(dev)
    kw = dict(rays_x=100, rays_y=90, max_bounces=2, seed=9, chunks_per_item=7)
    ref = srp.srp_force(ctx, bvhs, r_t, s_t, c_t, out_sigma=True, **kw)
    torch.cuda.synchronize()
    for call in range(2):
        out, sig = _run_noalloc(srp, bvhs, r_t, s_t, c_t, D, S, dev, **kw)
        assert _close(out, ref[0].cpu().numpy()), call
        assert np.allclose(sig, ref[1].cpu().numpy(), rtol=1e-5, atol=1e-12), call
    # two designs, each with its own three sun directions
    sun2 = W.random_unit_vectors(2 * S, 6).reshape(2, S, 3)
    s2 = torch.from_numpy(np.ascontiguousarray(sun2)).to(dev)
    kw2 = dict(rays_x=128, rays_y=64, max_bounces=3, seed=4, chunks_per_item=5, sun_per_design=1,
               ray_count=128 * 64 - 3)
    ref2 = srp.srp_force(ctx, bvhs[:2], r_t[:2].contiguous(), s2, c_t[:2].contiguous(), out_sigma=True, **kw2)
    torch.cuda.synchronize()
    for call in range(2):
        out, sig = _run_noalloc(srp, bvhs[:2], r_t[:2].contiguous(), s2, c_t[:2].contiguous(), 2, S, dev, **kw2)
        assert _close(out, ref2[0].cpu().numpy()), call
        assert np.allclose(sig, ref2[1].cpu().numpy(), rtol=1e-5, atol=1e-12), call


def test_noalloc_auto_chunks_capped_by_the_array():
    """160 suns x 512^2 rays: srp_force's automatic rule wants 160 x 1024
    chunks, above the 87,381 units of the fixed array, so the variant cuts
    coarser chunks; the sums agree to the suite's tolerance.  An explicit
    chunks_per_item that does not fit is refused."""
    _need_gpu()
    import paper_2602_10712_gb300 as srp
    dev = torch.device("cuda:0")
    ctx = srp.Context(0)
    m, rho, _, com = W.config1()
    b = srp.srp_build_bvh(ctx, m.verts, m.tris, m.group, 4)
    S = 160
    r_t = torch.from_numpy(rho[None].copy()).to(dev)
    s_t = torch.from_numpy(W.fibonacci_directions(S)).to(dev)
    c_t = torch.from_numpy(com[None].copy()).to(dev)
    kw = dict(rays_x=512, rays_y=512, max_bounces=1, seed=1, ray_count=512 * 512 - 1)
    ref = srp.srp_force(ctx, [b], r_t, s_t, c_t, out_sigma=True, **kw)
    torch.cuda.synchronize()
    for call in range(2):
        out, sig = _run_noalloc(srp, [b], r_t, s_t, c_t, 1, S, dev, **kw)
        assert _close(out, ref[0].cpu().numpy()), call
        assert np.allclose(sig, ref[1].cpu().numpy(), rtol=1e-5, atol=1e-12), call
    out = torch.empty((1, S, 6), dtype=torch.float64, device=dev)
    with pytest.raises(srp.SRPError) as e:
        srp.srp_force_noalloc([b], r_t, s_t, c_t, out, chunks_per_item=1000, **kw)
    assert e.value.code == srp.SRP_EINVAL and "capacity" in str(e.value)


def test_noalloc_rejects_oversize():
    _need_gpu()
    import paper_2602_10712_gb300 as srp
    dev = torch.device("cuda:0")
    ctx = srp.Context(0)
    m, rho, _, com = W.config1()
    b = srp.srp_build_bvh(ctx, m.verts, m.tris, m.group, 4)
    r_t = torch.from_numpy(rho[None].copy()).to(dev)
    c_t = torch.from_numpy(com[None].copy()).to(dev)
    big = torch.from_numpy(W.fibonacci_directions(90000)).to(dev)
    out = torch.empty((1, 90000, 6), dtype=torch.float64, device=dev)
    with pytest.raises(srp.SRPError) as e:
        srp.srp_force_noalloc([b], r_t, big, c_t, out, rays_x=64)
    assert e.value.code == srp.SRP_EINVAL and "capacity" in str(e.value)
