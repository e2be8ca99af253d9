"""Design optimisation through the orbit (Sec. 3.4.3, Alg. 1 Main): find
theta minimising g(z(t1, theta)) = |r(t1) - r_ref|^2 by gradient descent
with the adjoint of the RK4 integration (srp_integrate), clipping theta to
its bounds after every step (Sec. 3.4: parameters with a limited range are
clipped).  Adam (Kingma & Ba) is the step rule.  All integration and
gradients run in the library's kernels."""
from __future__ import annotations

import numpy as np

from . import srp_integrate


def optimize_design(ctx, opts, z0, theta0, r_ref, *, proxy=None, steps=100, lr=0.01, lo=None, hi=None,
                    b1=0.9, b2=0.999, eps=1e-12):
    """Returns (theta, losses [steps+1])."""
    th = np.array(theta0, dtype=np.float64).reshape(1, -1)
    lo = -np.inf if lo is None else np.asarray(lo, np.float64)
    hi = np.inf if hi is None else np.asarray(hi, np.float64)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    losses = []
    z0 = np.asarray(z0, np.float64).reshape(1, 13)
    for it in range(steps + 1):
        r = srp_integrate(ctx, opts, z0, th, proxy=proxy, dL_dzN=np.zeros((1, 13)))
        d = r["zN"][0, :3] - r_ref
        losses.append(float(d @ d))
        if it == steps:
            break
        lam = np.zeros((1, 13))
        lam[0, :3] = 2.0 * d
        g = srp_integrate(ctx, opts, z0, th, proxy=proxy, dL_dzN=lam)["dL_dtheta"]
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        mh = m / (1 - b1 ** (it + 1))
        vh = v / (1 - b2 ** (it + 1))
        th = np.clip(th - lr * mh / (np.sqrt(vh) + eps), lo, hi)
    return th[0], np.array(losses)


def _project_rho(rho):
    """Reflectances back into the admissible set: 0 <= rho_s, rho_d and
    rho_s + rho_d <= 1 (an excess is removed equally from both)."""
    r = np.clip(rho, 0.0, 1.0)
    ex = np.maximum(r.sum(axis=-1) - 1.0, 0.0)
    r = r - 0.5 * ex[..., None]
    return np.clip(r, 0.0, 1.0)


def optimize_tracer(ctx, mesh, rho0, angles0, sun_dir, com, target_ft, *, steps=100, lr=0.01, hinge_lo=-np.pi / 2,
                    hinge_hi=np.pi / 2, b1=0.9, b2=0.999, eps=1e-12, refit=True, **trace_opts):
    """Design optimisation through the tracer itself: Adam on the group
    reflectances (rho [G,2]) and the hinge angles of one design to bring its
    force and torque at the given suns (target_ft [S,6]) to the target,
    L = sum_s |(F,tau)_s - target_s|^2, with the reflectances projected into
    their admissible set and the angles clipped after every step.  Each step
    instantiates the design, brings its BVH up to date (refit=True: the
    first step builds it on the host, later steps refit it on the device to
    the moved vertices; False: a host build every step) and calls srp_force
    and srp_force_grad (upstream 2 (ft - target)); the hinge gradient holds
    the visibility fixed (it is exact while no shadow boundary moves).
    Returns (rho, angles, losses [steps+1])."""
    from . import srp_build_bvh, srp_bvh_refit, srp_design_instantiate, srp_force, srp_force_grad
    rho = _project_rho(np.array(rho0, dtype=np.float64))
    ang = np.array(angles0, dtype=np.float64)
    tri_hinge = np.asarray(mesh.vhinge)[np.asarray(mesh.tris)[:, 0]].astype(np.int32)
    p = np.concatenate([rho.ravel(), ang])
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    losses = []
    tgt = np.asarray(target_ft, np.float64)
    b = None
    for it in range(steps + 1):
        verts = srp_design_instantiate(mesh.verts, mesh.vhinge, mesh.hinges, ang)
        if b is not None and refit:
            srp_bvh_refit(ctx, b, verts, mesh.tris)
        else:
            if b is not None:
                b.close()
            b = srp_build_bvh(ctx, verts, mesh.tris, mesh.group, 4)
        ft = srp_force(ctx, [b], rho.astype(np.float32)[None], sun_dir, com[None], **trace_opts)[0]
        d = ft - tgt
        losses.append(float(np.sum(d * d)))
        if it == steps:
            b.close()
            break
        d_rho, d_h = srp_force_grad(ctx, b, rho.astype(np.float32), sun_dir, com, 2.0 * d, tri_hinge=tri_hinge,
                                    hinge_axes=mesh.hinges, **trace_opts)
        g = np.concatenate([np.asarray(d_rho).ravel(), np.asarray(d_h)])
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        p = p - lr * (m / (1 - b1 ** (it + 1))) / (np.sqrt(v / (1 - b2 ** (it + 1))) + eps)
        rho = _project_rho(p[:rho.size].reshape(rho.shape))
        ang = np.clip(p[rho.size:], hinge_lo, hinge_hi)
        p = np.concatenate([rho.ravel(), ang])
    return rho, ang, np.array(losses)
