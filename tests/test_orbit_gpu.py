"""GPU parity of srp_integrate (RK4 of Sec. 3.4 in FP64, discrete adjoint)
against the FP64 orbit oracle: trajectories, and adjoint gradients against
the oracle's complex-step derivatives of the same discrete map."""
import math

import numpy as np
import pytest

from oracle import mlp as omlp
from oracle import orbit as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SUN = np.array([0.3, 0.5, 0.81]) / np.linalg.norm([0.3, 0.5, 0.81])


@pytest.fixture(scope="module")
def srp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_10712_gb300 as srp
    return srp


def _z0():
    z0 = O.circular_state(26560e3, math.radians(55), 0.2, 0.4)
    q = np.array([0.9, 0.1, -0.3, 0.2]); q /= np.linalg.norm(q)
    z0[6:10] = q
    z0[10:13] = [1e-4, -2e-4, 5e-5]
    return z0


def test_two_body_energy_gpu(srp):
    ctx = srp.Context(0)
    o = srp.orbit_opts(model=srp.SRP_FM_NONE, j2=0.0, dt=60.0, n_steps=1440)
    z0 = O.circular_state(26560e3, math.radians(55))
    z0[3:6] *= 1.05
    r = srp.srp_integrate(ctx, o, z0, np.zeros(1), want_traj=True)
    tr = r["traj"][0]
    E = 0.5 * np.sum(tr[:, 3:6] ** 2, axis=1) - O.MU / np.linalg.norm(tr[:, :3], axis=1)
    assert np.max(np.abs(E / E[0] - 1)) < 1e-9
    zo = O.rk4(O.Model("none", j2=0.0), z0, np.zeros(1), 60.0, 1440)
    assert np.allclose(r["zN"][0], zo, rtol=1e-12, atol=1e-6)


def test_cannonball_trajectory_and_adjoint(srp):
    ctx = srp.Context(0)
    P = 4.56e-6
    o = srp.orbit_opts(model=srp.SRP_FM_CANNONBALL, pressure=P, mass=1000.0, sun=SUN, dt=60.0, n_steps=240,
                       n_theta=1, ckpt_every=16)
    z0 = _z0()
    th = np.array([20.0])
    wN = np.random.default_rng(0).normal(size=13) * np.array([1e-3] * 3 + [1.0] * 3 + [1e3] * 4 + [1e4] * 3)
    r = srp.srp_integrate(ctx, o, z0, th, dL_dzN=wN)
    m = O.Model("cannonball", P=P, mass=1000.0, sun=SUN)
    zo = O.rk4(m, z0, th, 60.0, 240)
    assert np.allclose(r["zN"][0], zo, rtol=1e-12, atol=1e-7)
    gt, gz = O.cs_grad(m, z0, th, 60.0, 240, wN)
    assert abs(r["dL_dtheta"][0, 0] - gt[0]) <= 1e-7 * abs(gt[0]) + 1e-15, (r["dL_dtheta"], gt)
    assert np.allclose(r["dL_dz0"][0], gz, rtol=1e-7, atol=1e-12 * np.abs(gz).max())


def test_proxy_trajectory_and_adjoint(srp):
    """Proxy force model (the tensor-core MLP's FP32 weights, evaluated in
    FP32 inside the integrator): trajectory to 1e-9 relative; dL/dtheta and
    dL/dz0 to 1e-4 relative of the complex-step gradient."""
    ctx = srp.Context(0)
    p = omlp.init_params(seed=4)
    p = [(W, np.random.default_rng(l).normal(size=b.shape) * 0.1) for l, (W, b) in enumerate(p)]
    flat = np.concatenate([np.concatenate([W.ravel(), b]) for W, b in p]).astype(np.float32)
    net = srp.MLP(ctx, flat)
    p32 = []
    o_ = 0
    for i in range(5):
        a, b = omlp.SIZES[i], omlp.SIZES[i + 1]
        p32.append((flat[o_:o_ + a * b].reshape(b, a).astype(np.float64), flat[o_ + a * b:o_ + a * b + b].astype(np.float64)))
        o_ += a * b + b
    scale = np.concatenate([np.ones(3), 4 * np.ones(14), np.ones(2) / (math.pi / 2)]).astype(np.float32)
    offset = np.concatenate([np.zeros(3), -np.ones(14), np.zeros(2)]).astype(np.float32)
    mean = np.array([0.1, -0.2, 0.3, 0.01, 0.02, -0.01], np.float32)
    std = np.array([2.0, 1.5, 3.0, 0.5, 0.4, 0.3], np.float32)
    P = 4.56e-6 * 20.0
    o = srp.orbit_opts(model=srp.SRP_FM_PROXY, pressure=P, mass=500.0, sun=SUN, dt=60.0, n_steps=120, n_theta=16,
                       in_scale=scale, in_offset=offset, out_mean=mean, out_std=std, ckpt_every=12)
    z0 = _z0()
    th = np.random.default_rng(3).uniform(0, 0.5, size=16)
    th[14:] = [0.3, -0.4]
    wN = np.random.default_rng(1).normal(size=13) * np.array([1e-3] * 3 + [1.0] * 3 + [1e3] * 4 + [1e4] * 3)
    r = srp.srp_integrate(ctx, o, z0, th, proxy=net, dL_dzN=wN)
    m = O.Model("proxy", P=P, mass=500.0, sun=SUN, params=p32, scale=scale.astype(np.float64),
                offset=offset.astype(np.float64), mean=mean.astype(np.float64), std=std.astype(np.float64))
    zo = O.rk4(m, z0, th, 60.0, 120)
    assert np.allclose(r["zN"][0], zo, rtol=1e-9, atol=1e-6), (r["zN"][0] - zo)
    gt, gz = O.cs_grad(m, z0, th, 60.0, 120, wN)
    assert np.linalg.norm(r["dL_dtheta"][0] - gt) <= 1e-4 * np.linalg.norm(gt), (r["dL_dtheta"][0], gt)
    assert np.linalg.norm(r["dL_dz0"][0] - gz) <= 1e-4 * np.linalg.norm(gz)


def test_batched_trajectories_independent(srp):
    ctx = srp.Context(0)
    o = srp.orbit_opts(model=srp.SRP_FM_CANNONBALL, pressure=4.56e-6, sun=SUN, dt=30.0, n_steps=100, n_theta=1)
    z0 = np.stack([_z0(), O.circular_state(7000e3, 0.5)])
    th = np.array([[10.0], [3.0]])
    r2 = srp.srp_integrate(ctx, o, z0, th)
    r0 = srp.srp_integrate(ctx, o, z0[:1], th[:1])
    r1 = srp.srp_integrate(ctx, o, z0[1:], th[1:])
    assert np.array_equal(r2["zN"][0], r0["zN"][0]) and np.array_equal(r2["zN"][1], r1["zN"][0])


@pytest.mark.parametrize("per_sm", [2, 3, 9])
def test_trajectories_per_cta_bitwise(srp, per_sm):
    """A CTA integrates 1, 2, 4 or 8 trajectories, chosen from their count
    and the SM count; the per-trajectory arithmetic is the same for every
    batch, so trajectories (and their adjoint gradients) integrated in a
    batch of per_sm x SMs, with a ragged last CTA, equal bit for bit the
    same trajectories integrated one at a time.  Proxy model, 14 steps with
    checkpoints every 5."""
    ctx = srp.Context(0)
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    n = per_sm * n_sm - 1
    net = srp.MLP(ctx, seed=5)
    o = srp.orbit_opts(model=srp.SRP_FM_PROXY, pressure=4.56e-5, mass=800.0, sun=SUN, dt=60.0, n_steps=14,
                       n_theta=16, ckpt_every=5)
    rng = np.random.default_rng(per_sm)
    z0 = np.stack([O.circular_state(rng.uniform(7e6, 4e7), rng.uniform(0, 1.5), rng.uniform(0, 6), rng.uniform(0, 6))
                   for _ in range(n)])
    q = rng.normal(size=(n, 4)); q /= np.linalg.norm(q, axis=1, keepdims=True)
    z0[:, 6:10] = q
    z0[:, 10:13] = rng.normal(size=(n, 3)) * 1e-4
    th = rng.uniform(0, 0.5, size=(n, 16))
    wN = rng.normal(size=(n, 13))
    r = srp.srp_integrate(ctx, o, z0, th, proxy=net, dL_dzN=wN)
    for i in (0, n // 2, n - 1):
        ri = srp.srp_integrate(ctx, o, z0[i:i + 1], th[i:i + 1], proxy=net, dL_dzN=wN[i:i + 1])
        assert np.array_equal(r["zN"][i], ri["zN"][0]), i
        assert np.array_equal(r["dL_dtheta"][i], ri["dL_dtheta"][0]), i
        assert np.array_equal(r["dL_dz0"][i], ri["dL_dz0"][0]), i


def test_design_optimisation_loop(srp):
    """Alg. 1's optimisation: recover the cannonball parameter that produced
    a reference end position (2 h arc) from a start 40% off, with bounds."""
    from paper_2602_10712_gb300.design import optimize_design
    ctx = srp.Context(0)
    o = srp.orbit_opts(model=srp.SRP_FM_CANNONBALL, pressure=4.56e-6 * 100, mass=100.0, sun=SUN, dt=60.0,
                       n_steps=120, n_theta=1)
    z0 = _z0()
    ref = srp.srp_integrate(ctx, o, z0, np.array([30.0]))["zN"][0, :3]
    th, losses = optimize_design(ctx, o, z0, np.array([18.0]), ref, steps=100, lr=1.0, lo=np.array([0.0]),
                                 hi=np.array([100.0]))
    assert losses[-1] < 1e-4 * losses[0], losses[[0, -1]]
    # the loss fell 1e4x: the error of theta fell ~100x from the 12-unit start
    assert abs(th[0] - 30.0) < 0.2


def test_eclipse_and_third_bodies_parity(srp):
    """Cannonball SRP with the cylinder eclipse and Sun/Moon point masses on
    a LEO orbit that passes through the Earth's shadow: trajectory and
    adjoint (dL/dtheta, dL/dz0) against the oracle's RK4 and complex-step
    gradient; the eclipse must change the result."""
    ctx = srp.Context(0)
    P = 4.56e-6 * 50.0
    sun = np.array([1.0, 0.0, 0.0])
    moon = np.array([0.0, 3.844e8, 1.0e7])
    kw = dict(model=srp.SRP_FM_CANNONBALL, pressure=P, mass=100.0, sun=sun, dt=30.0, n_steps=300, n_theta=1,
              ckpt_every=20, gm_sun=1.32712440018e20, sun_dist=1.495978707e11, gm_moon=4.9028e12, moon=moon)
    z0 = O.circular_state(7.0e6, 0.2, u=1.2)
    th = np.array([4.0])
    wN = np.random.default_rng(1).normal(size=13) * np.array([1e-3] * 3 + [1.0] * 3 + [1e3] * 4 + [1e4] * 3)
    r = srp.srp_integrate(ctx, srp.orbit_opts(eclipse=1, **kw), z0, th, dL_dzN=wN)
    m = O.Model("cannonball", P=P, mass=100.0, sun=sun, eclipse=True, gm_sun=1.32712440018e20,
                sun_dist=1.495978707e11, gm_moon=4.9028e12, moon=moon)
    zo, tr = O.rk4(m, z0, th, 30.0, 300, keep=True)
    shadow = [m.in_shadow(z[:3]) for z in tr]
    assert any(shadow) and not all(shadow)
    assert np.allclose(r["zN"][0], zo, rtol=1e-12, atol=1e-6)
    gt, gz = O.cs_grad(m, z0, th, 30.0, 300, wN)
    assert abs(r["dL_dtheta"][0, 0] - gt[0]) <= 1e-7 * abs(gt[0]) + 1e-15, (r["dL_dtheta"], gt)
    assert np.allclose(r["dL_dz0"][0], gz, rtol=1e-7, atol=1e-12 * np.abs(gz).max())
    r0 = srp.srp_integrate(ctx, srp.orbit_opts(eclipse=0, **kw), z0, th)
    assert np.linalg.norm(r0["zN"][0][:3] - r["zN"][0][:3]) > 1.0
    with pytest.raises(srp.SRPError, match="SRP_EINVAL"):
        srp.srp_integrate(ctx, srp.orbit_opts(eclipse=2, **kw), z0, th)


def test_tracer_design_optimisation(srp):
    """Design optimisation through the tracer's own gradient (Adam on 7 x
    (rho_s, rho_d) of the 7-group box-wing, hinges fixed, 16 suns, K = 1):
    recover the reflectances that produced the target forces from a start
    0.15 off; the loss falls by more than 100x and the median error by more
    than 3x."""
    import workloads as W
    from paper_2602_10712_gb300.design import optimize_tracer
    ctx = srp.Context(0)
    m = W.box_wing_7group()
    rng = np.random.default_rng(4)
    rho_true = rng.uniform(0.1, 0.4, size=(7, 2))
    sun = W.fibonacci_directions(16)
    com = np.zeros(3)
    ang = np.array([0.2, -0.3])
    kw = dict(rays_x=256, max_bounces=1, seed=1)
    v = srp.srp_design_instantiate(m.verts, m.vhinge, m.hinges, ang)
    b = srp.srp_build_bvh(ctx, v, m.tris, m.group, 4)
    target = srp.srp_force(ctx, [b], rho_true.astype(np.float32)[None], sun, com[None], **kw)[0]
    rho0 = np.clip(rho_true + rng.choice([-0.15, 0.15], size=rho_true.shape), 0.0, 0.5)
    rho, ang_out, losses = optimize_tracer(ctx, m, rho0, ang, sun, com, target, steps=100, lr=0.01,
                                           hinge_lo=ang, hinge_hi=ang, **kw)
    assert losses[-1] < 1e-2 * losses[0], losses[[0, -1]]
    # most reflectances are recovered; a weakly lit small facet may trade off
    # against the large panels, so the median error is the measure
    assert np.median(np.abs(rho - rho_true)) < np.median(np.abs(rho0 - rho_true)) / 3
