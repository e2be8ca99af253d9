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
