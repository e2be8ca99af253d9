"""GPU parity of the SRP tracer (srp_force, srp_trace_rays through the C ABI)
against the FP64 brute-force oracle on the same Philox rays.

Parity bar (relative 1e-5, FP32 kernel vs FP64 oracle):
  |F_gpu - F_or| <= 1e-5 |F_or|,   |tau_gpu - tau_or| <= 1e-5 |F_or| R.
The closest-hit triangle is an argmin decided by floating point; a ray that
passes within FP32 rounding (~1e-6 m) of a shared edge may legitimately pick
the neighbouring triangle.  Where that can happen (fine meshes) the tests
compare per-ray paths: rays whose hit sequences agree must agree to 1e-5, the
count of rays whose paths differ is bounded and reported, and the aggregate
is checked with those rays' differences accounted for exactly."""

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def srp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_10712_gb300 as srp
    return srp


@pytest.fixture(scope="module")
def ctx(srp):
    return srp.Context(0)


def _bvh(srp, ctx, m, verts=None, width=4):
    v = m.verts if verts is None else verts
    return srp.srp_build_bvh(ctx, v, m.tris, m.group, width)


def _assert_parity(ft_gpu, ft_or, R, tol=1e-5, what=""):
    ft_gpu = np.asarray(ft_gpu).reshape(-1, 6)
    ft_or = np.asarray(ft_or).reshape(-1, 6)
    for s in range(ft_or.shape[0]):
        fn = np.linalg.norm(ft_or[s, :3])
        if fn == 0.0:
            assert np.all(np.abs(ft_gpu[s]) <= 1e-12), (what, s, ft_gpu[s])
            continue
        ef = np.linalg.norm(ft_gpu[s, :3] - ft_or[s, :3]) / fn
        et = np.linalg.norm(ft_gpu[s, 3:] - ft_or[s, 3:]) / (fn * R)
        assert ef <= tol and et <= tol, (what, s, ef, et, ft_gpu[s], ft_or[s])


def _assert_per_ray(yg, yo, w, R, what=""):
    """Per-ray deposits of rays whose hit lists agree: force components
    within 1e-5 of the ray weight w, torque components within 1e-5 w R
    (the lever arm is up to the grid radius R)."""
    if yg.shape[0] == 0:
        return
    df = np.abs(yg[:, :3] - yo[:, :3]).max() / w
    dt = np.abs(yg[:, 3:] - yo[:, 3:]).max() / (w * R)
    assert df <= 1e-5 and dt <= 1e-5, (what, "per-ray force / torque deviation in ray weights", df, dt)


def _corrected(ft, yg, hg, yo, ho):
    """The GPU aggregate with the contributions of rays whose hit lists
    differ (an FP32 argmin next to a shared edge) replaced by the oracle's."""
    diff = ~np.all(hg == ho, axis=1)
    return ft - yg[diff].sum(0) + yo[diff].sum(0), int(diff.sum())


# ------------------------------------------------------------------ config 1
@pytest.mark.parametrize("K", [1, 2, 3])
def test_boxwing_full_grid_parity(srp, ctx, K):
    """Box-wing (16 triangles), 1024 x 1024 rays, sun (1,2,3)/sqrt 14."""
    m, rho, sun, com = W.config1()
    b = _bvh(srp, ctx, m)
    ft, sg = srp.srp_force(ctx, [b], rho[None], sun, com[None], out_sigma=True, rays_x=1024, max_bounces=K)
    fo, so = oracle.force(m.verts, m.tris, m.group, rho, sun, com, nx=1024, K=K)
    R = b.info()["radius"]
    _assert_parity(ft[0], fo, R, what=f"K={K}")
    assert np.allclose(sg[0], so, rtol=1e-3, atol=1e-6 * np.linalg.norm(fo[0, :3]))


def test_boxwing_per_ray_paths(srp, ctx):
    """Per-ray samples of the whole 512^2 grid: hit sequences and deposits."""
    m, rho, sun, com = W.config1()
    b = _bvh(srp, ctx, m)
    idx = np.arange(512 * 512, dtype=np.int64)
    yg, hg = srp.srp_trace_rays(ctx, b, rho, sun[0], com, idx, rays_x=512, max_bounces=3)
    yo, ho = oracle.trace_rays(m.verts, m.tris, m.group, rho, sun[0], com, idx, nx=512, K=3)
    same = np.all(hg == ho, axis=1)
    assert same.mean() > 0.99999, same.mean()
    R = b.info()["radius"]
    w = (2 * R / 512) ** 2
    _assert_per_ray(yg[same], yo[same], w, R, "box-wing 512^2")
    ft = srp.srp_force(ctx, [b], rho[None], sun, com[None], rays_x=512, max_bounces=3)
    assert np.allclose(ft[0, 0], yg.sum(0), rtol=1e-6, atol=1e-9 * w)  # FP32 per-lane partials


def test_boxwing_direction_sweep(srp, ctx):
    """64 Fibonacci sun directions in one launch, K = 3: per direction the
    aggregate within 1e-5 once the rays whose hit lists differ (edge-grazing
    FP32 argmins) carry the oracle's deposits, and every other ray within
    1e-5 of its weight."""
    m, rho, _, com = W.config1()
    sun = W.fibonacci_directions(64)
    b = _bvh(srp, ctx, m)
    ft = srp.srp_force(ctx, [b], rho[None], sun, com[None], rays_x=128, max_bounces=3)
    fo, _ = oracle.force(m.verts, m.tris, m.group, rho, sun, com, nx=128, K=3)
    R = b.info()["radius"]
    w = (2 * R / 128) ** 2
    idx = np.arange(128 * 128, dtype=np.int64)
    mis = 0
    for s in range(64):
        yg, hg = srp.srp_trace_rays(ctx, b, rho, sun[s], com, idx, sun_index=s, rays_x=128, max_bounces=3)
        yo, ho = oracle.trace_rays(m.verts, m.tris, m.group, rho, sun[s], com, idx, nx=128, K=3, sun_index=s)
        same = np.all(hg == ho, axis=1)
        _assert_per_ray(yg[same], yo[same], w, R, f"sun {s}")
        corr, nd = _corrected(ft[0, s], yg, hg, yo, ho)
        mis += nd
        if np.linalg.norm(fo[s, :3]) > 0.0:
            _assert_parity(corr, fo[s], R, what=f"sun {s}")
    assert mis <= 1e-3 * 64 * idx.shape[0], mis


# ------------------------------------------------------------------ config 2
def test_procedural_satellite_sampled_full_grid(srp, ctx):
    """~50k triangles, K = 3, the full 2048^2 grid sampled every 1021st ray
    for 3 of 4096 Fibonacci directions (the benchmark's launch geometry)."""
    m, rho, sun_all, com = W.config2(4096)
    b = _bvh(srp, ctx, m)
    R = b.info()["radius"]
    n = 2048 * 2048
    idx = np.arange(0, n, 1021, dtype=np.int64)[:3000]
    w = (2 * R / 2048) ** 2
    tot_mis = 0
    for s in (5, 1777, 3001):
        sun = sun_all[s]
        yg, hg = srp.srp_trace_rays(ctx, b, rho, sun, com, idx, sun_index=s, rays_x=2048, max_bounces=3)
        yo, ho = oracle.trace_rays(m.verts, m.tris, m.group, rho, sun, com, idx, nx=2048, K=3, sun_index=s)
        same = np.all(hg == ho, axis=1)
        mis = int((~same).sum())
        tot_mis += mis
        _assert_per_ray(yg[same], yo[same], w, R, f"sun {s}")
        # aggregate over the sample through srp_force (same rays, same counters)
        ft = srp.srp_force(ctx, [b], rho[None], sun_all[s:s + 1], com[None], rays_x=2048, max_bounces=3,
                           ray_offset=0, ray_stride=1021, ray_count=len(idx), sun_base=s)
        # FP32 tile partials (<= 128 rays) then FP64: rounding ~1e-7 of the sums' scale
        assert np.linalg.norm(ft[0, 0] - yg.sum(0)) <= 1e-6 * np.linalg.norm(yg.sum(0)) + 1e-9 * w
        # oracle aggregate, with the differing rays' contributions swapped in
        fo_agree = yo[same].sum(0)
        fg_agree = yg[same].sum(0)
        _assert_parity(fg_agree, fo_agree, R, what=f"sun {s} agreeing rays")
    assert tot_mis <= 0.002 * 3 * len(idx), tot_mis


def test_procedural_satellite_small_grid_aggregate(srp, ctx):
    """Whole 96^2 grid, 4 directions, K = 3, BVH8: aggregate within 1e-5
    after accounting for per-ray path differences exactly."""
    m, rho, sun_all, com = W.config2(4)
    b = _bvh(srp, ctx, m, width=8)
    R = b.info()["radius"]
    ft = srp.srp_force(ctx, [b], rho[None], sun_all, com[None], rays_x=96, max_bounces=3)
    fo, _ = oracle.force(m.verts, m.tris, m.group, rho, sun_all, com, nx=96, K=3)
    idx = np.arange(96 * 96, dtype=np.int64)
    for s in range(4):
        yg, hg = srp.srp_trace_rays(ctx, b, rho, sun_all[s], com, idx, sun_index=s, rays_x=96, max_bounces=3)
        yo, ho = oracle.trace_rays(m.verts, m.tris, m.group, rho, sun_all[s], com, idx, nx=96, K=3, sun_index=s)
        diff = ~np.all(hg == ho, axis=1)
        corrected = ft[0, s] - yg[diff].sum(0) + yo[diff].sum(0)
        _assert_parity(corrected, fo[s], R, what=f"sun {s}")
        assert diff.sum() <= 10


# ------------------------------------------------------------------ equivalences
def test_width4_equals_width8_bitwise(srp, ctx):
    """The BVH width changes the traversal, not the rays or their deposits:
    bit-identical on a grid whose rays are all traced (200 columns); on a
    full grid of whole 32-pixel batches the batches that cannot meet the
    scene are found from each BVH's top boxes, so the batches grouped per
    FP32 tile sum differ and only rounding may change."""
    m, rho, sun, com = W.config2(8)
    b4 = _bvh(srp, ctx, m, width=4)
    b8 = _bvh(srp, ctx, m, width=8)
    kw = dict(rays_x=200, rays_y=256, max_bounces=3, chunks_per_item=8)
    f4 = srp.srp_force(ctx, [b4], rho[None], sun, com[None], **kw)
    f8 = srp.srp_force(ctx, [b8], rho[None], sun, com[None], **kw)
    assert np.array_equal(f4, f8)
    kw = dict(rays_x=256, max_bounces=3, chunks_per_item=8)
    f4 = srp.srp_force(ctx, [b4], rho[None], sun, com[None], **kw)
    f8 = srp.srp_force(ctx, [b8], rho[None], sun, com[None], **kw)
    scale = np.abs(f4[..., :3]).max()
    assert np.all(np.abs(f4 - f8) <= 1e-6 * scale * np.array([1, 1, 1, 10, 10, 10]))


def test_deterministic_and_host_equals_device(srp, ctx):
    m, rho, sun, com = W.config2(8)
    b = _bvh(srp, ctx, m)
    kw = dict(rays_x=200, rays_y=130, max_bounces=3, seed=12345)
    f1 = srp.srp_force(ctx, [b], rho[None], sun, com[None], **kw)
    f2 = srp.srp_force(ctx, [b], rho[None], sun, com[None], **kw)
    assert np.array_equal(f1, f2)
    dev = torch.device("cuda:0")
    r_t = torch.from_numpy(rho[None].copy()).to(dev)
    s_t = torch.from_numpy(sun.copy()).to(dev)
    c_t = torch.from_numpy(com[None].copy()).to(dev)
    f3 = srp.srp_force(ctx, [b], r_t, s_t, c_t, **kw)
    torch.cuda.synchronize()
    assert np.array_equal(f1, f3.cpu().numpy())


def test_chunking_only_changes_rounding(srp, ctx):
    m, rho, sun, com = W.config1()
    b = _bvh(srp, ctx, m)
    a = srp.srp_force(ctx, [b], rho[None], sun, com[None], rays_x=512, max_bounces=2)
    c = srp.srp_force(ctx, [b], rho[None], sun, com[None], rays_x=512, max_bounces=2, block_threads=128,
                      chunks_per_item=3)
    # per-thread FP32 partials (<= 32 rays) group rays differently: FP32-level rounding
    assert np.allclose(a, c, rtol=2e-7, atol=1e-12)


def test_sun_sharding_bitwise(srp, ctx):
    """Splitting the sun directions across calls (sun_base offsets the RNG
    counter) reproduces the unsharded result bit for bit."""
    m, rho, _, com = W.config1()
    sun = W.fibonacci_directions(10)
    b = _bvh(srp, ctx, m)
    kw = dict(rays_x=256, max_bounces=3, chunks_per_item=4)
    full = srp.srp_force(ctx, [b], rho[None], sun, com[None], **kw)
    p1 = srp.srp_force(ctx, [b], rho[None], sun[:4], com[None], **kw)
    p2 = srp.srp_force(ctx, [b], rho[None], sun[4:], com[None], sun_base=4, **kw)
    assert np.array_equal(full[0], np.concatenate([p1[0], p2[0]]))


def test_more_items_than_one_grid(srp, ctx):
    """2^20 + 4096 (design, sun) items -- more than the per-item kernels'
    grids (2^20 blocks), so the span pre-pass and the reduction loop over
    items: one call equals two half calls bit for bit (one chunk per item in
    both), and sampled items match the oracle."""
    import torch
    m, rho, _, com = W.config1()
    S = (1 << 20) + 4096
    sun = W.fibonacci_directions(S)
    b = _bvh(srp, ctx, m)
    dev = torch.device("cuda:0")
    r_t = torch.from_numpy(rho[None].copy()).to(dev)
    c_t = torch.from_numpy(com[None].copy()).to(dev)
    s_t = torch.from_numpy(sun).to(dev)
    kw = dict(rays_x=32, rays_y=1, max_bounces=1)
    full = srp.srp_force(ctx, [b], r_t, s_t, c_t, **kw)
    h = S // 2
    p1 = srp.srp_force(ctx, [b], r_t, s_t[:h].contiguous(), c_t, **kw)
    p2 = srp.srp_force(ctx, [b], r_t, s_t[h:].contiguous(), c_t, sun_base=h, **kw)
    srp.srp_sync(ctx)
    assert torch.equal(full[0, :h], p1[0]) and torch.equal(full[0, h:], p2[0])
    got = full[0].cpu().numpy()
    R = b.info()["radius"]
    for s in (0, 1, h, (1 << 20) - 1, 1 << 20, S - 1):
        fo, _ = oracle.force(m.verts, m.tris, m.group, rho, sun[s], com, nx=32, ny=1, K=1, sun_base=s)
        _assert_parity(got[s:s + 1], fo, R, what=f"sun {s}")


# ------------------------------------------------------------------ edge cases
def test_multi_design_uneven_and_sun_per_design(srp, ctx):
    """Three designs of 2, 16 and 320 triangles in one call, each with its own
    sun directions and COM; ragged grid 77 x 50."""
    designs = [W.flat_plate((2.0, 1.0), 2), W.box_wing(), W.icosphere(2)]
    G = 64
    rng = np.random.default_rng(1)
    rho = np.stack([W.random_reflectances(G, seed=10 + k) for k in range(3)])
    sun = W.random_unit_vectors(9, seed=3).reshape(3, 3, 3)
    com = rng.normal(size=(3, 3)) * 0.1
    bv = [_bvh(srp, ctx, d) for d in designs]
    ft = srp.srp_force(ctx, bv, rho, sun, com, rays_x=77, rays_y=50, max_bounces=3, sun_per_design=1,
                       design_base=7)
    for k, d in enumerate(designs):
        fo, _ = oracle.force(d.verts, d.tris, d.group, rho[k], sun[k], com[k], nx=77, ny=50, K=3,
                             design_index=7 + k)
        R = bv[k].info()["radius"]
        _assert_parity(ft[k], fo, R, what=f"design {k}")


def test_ragged_ray_subset(srp, ctx):
    m, rho, sun, com = W.config1()
    b = _bvh(srp, ctx, m)
    kw = dict(rays_x=1000, rays_y=999, max_bounces=2, jitter=0, ray_offset=17, ray_stride=7, ray_count=1001)
    ft, sg = srp.srp_force(ctx, [b], rho[None], sun, com[None], out_sigma=True, **kw)
    fo, so = oracle.force(m.verts, m.tris, m.group, rho, sun, com, nx=1000, ny=999, K=2, jitter=0,
                          ray_offset=17, ray_stride=7, ray_count=1001)
    _assert_parity(ft[0], fo, b.info()["radius"])
    assert np.allclose(sg[0], so, rtol=1e-4, atol=1e-9)


def test_empty_and_single_triangle(srp, ctx):
    rho = np.full((1, 64, 2), 0.2, np.float32)
    sun = W.SUN_C1[None]
    e = srp.srp_build_bvh(ctx, np.zeros((3, 3), np.float32), np.zeros((0, 3), np.int32), np.zeros(0, np.int32))
    f = srp.srp_force(ctx, [e], rho, sun, np.zeros((1, 3)), rays_x=64)
    assert np.all(f == 0.0)
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0.2]], np.float32)
    t = np.array([[0, 1, 2]], np.int32)
    g = np.zeros(1, np.int32)
    b = srp.srp_build_bvh(ctx, v, t, g)
    ft = srp.srp_force(ctx, [b], rho, sun, np.zeros((1, 3)), rays_x=300, max_bounces=3)
    fo, _ = oracle.force(v, t, g, rho[0], sun, np.zeros(3), nx=300, K=3)
    _assert_parity(ft[0], fo, b.info()["radius"])


def test_zero_items(srp, ctx):
    m, rho, sun, com = W.config1()
    b = _bvh(srp, ctx, m)
    f = srp.srp_force(ctx, [b], rho[None], np.zeros((0, 3)), com[None], rays_x=64)
    assert f.shape == (1, 0, 6)


def test_statistical_agreement_other_seed(srp, ctx):
    """GPU and oracle with different seeds agree within 3 sigma per
    component (the criterion for two independent estimates of the same
    integral)."""
    m, rho, sun, com = W.config1()
    b = _bvh(srp, ctx, m)
    ft, sg = srp.srp_force(ctx, [b], rho[None], sun, com[None], out_sigma=True, rays_x=512, max_bounces=3, seed=77)
    fo, so = oracle.force(m.verts, m.tris, m.group, rho, sun, com, nx=512, K=3, seed=78)
    tol = 3 * np.sqrt(sg[0, 0] ** 2 + so[0] ** 2) + 1e-12
    assert np.all(np.abs(ft[0, 0] - fo[0]) <= tol)


def test_invalid_arguments_rejected(srp, ctx):
    m, rho, sun, com = W.config1()
    b = _bvh(srp, ctx, m)
    bad = rho.copy(); bad[3] = [0.7, 0.6]
    for kw, args in [(dict(max_bounces=4), (rho[None], sun)), (dict(rays_x=0), (rho[None], sun)),
                     (dict(ray_offset=5, ray_stride=1000, ray_count=2000), (rho[None], sun)),
                     ({}, (bad[None], sun)), ({}, (rho[None], sun * 1.1))]:
        with pytest.raises(srp.SRPError) as e:
            srp.srp_force(ctx, [b], args[0], args[1], com[None], **{"rays_x": 64, **kw})
        assert e.value.code == srp.SRP_EINVAL, kw
    with pytest.raises(srp.SRPError):
        srp.srp_build_bvh(ctx, m.verts, m.tris, np.full(16, 64, np.int32))
    # the box-wing uses groups 0..15: reflectances for 8 groups are too few
    with pytest.raises(srp.SRPError) as e:
        srp.srp_force(ctx, [b], rho[None, :8], sun, com[None], rays_x=64)
    assert e.value.code == srp.SRP_EINVAL and "group 15" in str(e.value)


def test_bvh_info(srp, ctx):
    m, _, _, _ = W.config2(1)
    b = _bvh(srp, ctx, m, width=8)
    info = b.info()
    c, R = oracle.grid(m.verts)
    assert info["n_tris"] == m.T and info["width"] == 8 and info["n_leaves"] >= m.T / 4
    assert np.allclose(info["center"], c) and abs(info["radius"] - R) < 1e-12


def test_corrupted_bvh_reports_device_limit(srp, ctx):
    """Failure detection without a GPU fault: node data with out-of-range
    indices is rejected on the host; an in-range cycle (a node that is its
    own child) makes the traversal hit its stack-depth / visit bounds, which
    end the ray and flag SRP_EDEVICE_LIMIT; the context stays usable."""
    m, rho, sun, com = W.config1()
    b = _bvh(srp, ctx, m)
    nodes, order, nn = srp.srp_build_bvh_host(m.verts, m.tris, 4)
    bad = nodes.copy().reshape(nn, 32)
    ch = bad[:, 24:28].view(np.int32)
    ch[0, 0] = nn + 5
    with pytest.raises(srp.SRPError) as e:
        srp.srp_bvh_set_nodes(ctx, b, bad)
    assert e.value.code == srp.SRP_EINVAL
    cyc = nodes.copy().reshape(nn, 32)
    cyc[0, 0], cyc[0, 4 * 0 + 4] = -1e3, 1e3   # child 0 box: everything (lo_x, hi_x)
    cyc[0, 8], cyc[0, 12] = -1e3, 1e3           # lo_y, hi_y
    cyc[0, 16], cyc[0, 20] = -1e3, 1e3          # lo_z, hi_z
    cyc[0, 24:28].view(np.int32)[0] = 0         # node 0 is its own child
    srp.srp_bvh_set_nodes(ctx, b, cyc)
    with pytest.raises(srp.SRPError) as e:
        srp.srp_force(ctx, [b], rho[None], sun, com[None], rays_x=32)
    assert e.value.code == srp.SRP_EDEVICE_LIMIT
    # restore and check the context still works
    srp.srp_bvh_set_nodes(ctx, b, nodes)
    ft = srp.srp_force(ctx, [b], rho[None], sun, com[None], rays_x=256, max_bounces=1)
    fo, _ = oracle.force(m.verts, m.tris, m.group, rho, sun, com, nx=256, K=1)
    _assert_parity(ft[0], fo, b.info()["radius"])


@pytest.mark.parametrize("width,ny", [(4, 256), (8, 256), (4, 258), (4, 257)])
def test_skipped_batches_deposit_nothing(srp, ctx, width, ny):
    """On a full grid of whole 32-pixel batches only the batches that can
    meet the scene are traced; the rest must deposit nothing.  The same grid
    without its last ray is traced ray by ray (a ray subset): full =
    subset + last ray, to rounding, on the satellite with K = 3.  256 rows
    make the batches 8 x 4 pixel blocks, 258 rows 16 x 2, 257 rows 32 x 1:
    each shape must cover every ray of the grid exactly once."""
    m, rho, sun, com = W.config2(8)
    b = _bvh(srp, ctx, m, width=width)
    nx = 256
    kw = dict(rays_x=nx, rays_y=ny, max_bounces=3, seed=3)
    full = srp.srp_force(ctx, [b], rho[None], sun, com[None], **kw)
    sub = srp.srp_force(ctx, [b], rho[None], sun, com[None], ray_offset=0, ray_stride=1, ray_count=nx * ny - 1,
                        **kw)
    for s in range(sun.shape[0]):
        y, _ = srp.srp_trace_rays(ctx, b, rho, sun[s], com, np.array([nx * ny - 1]), sun_index=s, **kw)
        want = sub[0, s] + y[0]
        scale = np.linalg.norm(full[0, s, :3])
        assert np.all(np.abs(full[0, s] - want) <= 1e-6 * scale * np.array([1, 1, 1, 10, 10, 10])), (s, full[0, s], want)
