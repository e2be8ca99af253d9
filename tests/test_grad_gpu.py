"""GPU parity of the gradient kernels (srp_force_grad through the C ABI and
the autograd wrapper) against the oracle's gradient of the same estimate
(relative 1e-5), which tests/test_oracle_grad.py pins to finite differences
and to the per-plate law."""
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


def _rel(a, b):
    a = np.asarray(a, np.float64); b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("K", [1, 2, 3])
def test_rho_gradient_parity(srp, ctx, K):
    """Box-wing (64 groups, 16 used), 3 suns, 512^2 rays: d_rho vs oracle."""
    m, rho, _, com = W.config1()
    sun = W.fibonacci_directions(3)
    up = np.random.default_rng(K).normal(size=(3, 6))
    b = srp.srp_build_bvh(ctx, m.verts, m.tris, m.group, 4)
    dr, _ = srp.srp_force_grad(ctx, b, rho, sun, com, up, rays_x=512, max_bounces=K, seed=3)
    _, dro, _ = oracle.force_grad(m.verts, m.tris, m.group, rho, sun, com, up, nx=512, K=K, seed=3)
    assert _rel(dr, dro) <= 1e-5, _rel(dr, dro)
    assert np.all(dr[16:] == 0.0)


@pytest.mark.parametrize("K", [1, 2, 3])
def test_hinge_gradient_parity(srp, ctx, K):
    """Hinge angles (0.3, -0.5) on the box-wing, 2 suns.  K = 1: against the
    oracle's analytic derivative (1e-5); K = 2, 3: against its per-path
    central difference of the fixed-visibility path value (1e-4: the GPU's
    FP32 tangents through plane intersections of grazing bounce rays)."""
    m, rho, _, com = W.config1()
    ang = np.array([0.3, -0.5])
    v = srp.srp_design_instantiate(m.verts, m.vhinge, m.hinges, ang)
    th = oracle.tri_hinge(m.tris, m.vhinge)
    sun = np.stack([W.SUN_C1, np.array([0.6, -0.2, 0.77]) / np.linalg.norm([0.6, -0.2, 0.77])])
    up = np.random.default_rng(8).normal(size=(2, 6))
    b = srp.srp_build_bvh(ctx, v, m.tris, m.group, 4)
    dr, dh = srp.srp_force_grad(ctx, b, rho, sun, com, up, tri_hinge=th, hinge_axes=m.hinges, rays_x=512,
                                max_bounces=K, seed=4)
    _, dro, dho = oracle.force_grad(v, m.tris, m.group, rho, sun, com, up, nx=512, K=K, seed=4,
                                    tri_hinge=th, hinge_axes=m.hinges)
    assert _rel(dr, dro) <= 1e-5
    assert np.all(np.abs(dho) > 0.0)
    assert _rel(dh, dho) <= (1e-5 if K == 1 else 1e-4), (dh, dho)


def test_grad_device_mode(srp, ctx):
    m, rho, _, com = W.config1()
    sun = W.fibonacci_directions(2)
    up = np.ones((2, 6))
    b = srp.srp_build_bvh(ctx, m.verts, m.tris, m.group, 8)
    dev = torch.device("cuda:0")
    h = srp.srp_force_grad(ctx, b, rho, sun, com, up, rays_x=256, max_bounces=2)[0]
    d = srp.srp_force_grad(ctx, b, torch.from_numpy(rho).to(dev), torch.from_numpy(sun).to(dev),
                           torch.from_numpy(com).to(dev), torch.from_numpy(up).to(dev), rays_x=256, max_bounces=2)[0]
    torch.cuda.synchronize()
    assert np.allclose(d.cpu().numpy(), h, rtol=1e-6, atol=1e-12)
    th = oracle.tri_hinge(m.tris, m.vhinge)
    hh = srp.srp_force_grad(ctx, b, rho, sun, com, up, tri_hinge=th, hinge_axes=m.hinges, rays_x=256,
                            max_bounces=2)[1]
    hd = srp.srp_force_grad(ctx, b, torch.from_numpy(rho).to(dev), torch.from_numpy(sun).to(dev),
                            torch.from_numpy(com).to(dev), torch.from_numpy(up).to(dev),
                            tri_hinge=torch.from_numpy(th).to(dev), hinge_axes=torch.from_numpy(m.hinges).to(dev),
                            rays_x=256, max_bounces=2)[1]
    torch.cuda.synchronize()
    assert np.allclose(hd.cpu().numpy(), hh, rtol=1e-5, atol=1e-12)


def test_autograd_function(srp, ctx):
    """torch.autograd through the tracer: backward equals srp_force_grad, and
    the rho gradient matches a central difference of the GPU forward (the K=1
    estimate is affine in rho)."""
    m = W.box_wing()
    design = dict(verts=m.verts, tris=m.tris, group=m.group, vhinge=m.vhinge, hinges=m.hinges)
    dev = torch.device("cuda:0")
    rho = torch.from_numpy(W.random_reflectances(64, seed=0)).to(dev).requires_grad_(True)
    ang = torch.tensor([0.2, -0.1], dtype=torch.float64, device=dev, requires_grad=True)
    sun = torch.from_numpy(W.fibonacci_directions(2)).to(dev)
    com = torch.zeros(3, dtype=torch.float64, device=dev)
    opts = dict(rays_x=512, max_bounces=1, seed=2)
    F = srp.SRPForce.apply(ctx, design, rho, ang, sun, com, opts)
    wts = torch.from_numpy(np.random.default_rng(1).normal(size=(2, 6))).to(dev)
    L = (F * wts).sum()
    L.backward()
    g_rho = rho.grad.detach().cpu().numpy().astype(np.float64)
    g_ang = ang.grad.detach().cpu().numpy()
    # central difference in one reflectance through the forward
    h = 0.05
    r0 = rho.detach().clone()
    for (gi, j) in [(3, 0), (13, 1)]:
        rp = r0.clone(); rp[gi, j] += h
        rm = r0.clone(); rm[gi, j] -= h
        Lp = (srp.SRPForce.apply(ctx, design, rp, ang.detach(), sun, com, opts) * wts).sum().item()
        Lm = (srp.SRPForce.apply(ctx, design, rm, ang.detach(), sun, com, opts) * wts).sum().item()
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g_rho[gi, j]) <= 1e-4 * (abs(fd) + 1e-3), (gi, j, fd, g_rho[gi, j])
    # hinge gradient matches the oracle on the instantiated design
    v = oracle.instantiate(m.verts, m.vhinge, m.hinges, [0.2, -0.1])
    _, _, dho = oracle.force_grad(v, m.tris, m.group, r0.cpu().numpy(), sun.cpu().numpy(), np.zeros(3),
                                  wts.cpu().numpy(), nx=512, K=1, seed=2, tri_hinge=oracle.tri_hinge(m.tris, m.vhinge),
                                  hinge_axes=m.hinges)
    assert _rel(g_ang, dho) <= 1e-4, (g_ang, dho)


@pytest.mark.parametrize("K,ny", [(1, 256), (3, 256), (1, 258), (1, 257)])
def test_grad_span_prepass_equals_ray_subsets(srp, ctx, K, ny):
    """A full grid of whole 32-pixel batches traces only the batches that can
    meet the scene (the forward's pre-pass); the same grid given as two ray
    subsets traces every ray.  Both give the gradient of the same estimate:
    reflectance and hinge gradients agree to the FP32 grouping of the
    per-warp sums (1e-5, the suite's bound), on the box-wing with hinges, 4
    suns, 256 columns; 256, 258 and 257 rows give batches of 8 x 4, 16 x 2
    and 32 x 1 pixels."""
    m, rho, _, com = W.config1()
    ang = np.array([0.3, -0.5])
    v = srp.srp_design_instantiate(m.verts, m.vhinge, m.hinges, ang)
    th = oracle.tri_hinge(m.tris, m.vhinge)
    sun = W.fibonacci_directions(4)
    up = np.random.default_rng(12).normal(size=(4, 6))
    b = srp.srp_build_bvh(ctx, v, m.tris, m.group, 4)
    kw = dict(tri_hinge=th, hinge_axes=m.hinges, rays_x=256, rays_y=ny, max_bounces=K, seed=6)
    dr, dh = srp.srp_force_grad(ctx, b, rho, sun, com, up, **kw)
    n = 256 * ny
    a_r, a_h = srp.srp_force_grad(ctx, b, rho, sun, com, up, ray_offset=0, ray_count=n // 2, **kw)
    b_r, b_h = srp.srp_force_grad(ctx, b, rho, sun, com, up, ray_offset=n // 2, ray_count=n // 2, **kw)
    assert np.any(dr != 0.0) and np.all(np.abs(dh) > 0.0)
    assert _rel(dr, a_r + b_r) <= 1e-5, _rel(dr, a_r + b_r)
    assert _rel(dh, a_h + b_h) <= 1e-5, _rel(dh, a_h + b_h)
