"""Host logic of design optimisation through the tracer
(design.optimize_tracer) on CPU: srp_force / srp_force_grad replaced by an
affine force model F = A rho + B angles + c with its exact gradient, so the
Adam loop, the projection of the reflectances into their admissible set and
the clipping of the hinge angles are checked without a GPU."""
import types

import numpy as np
import pytest


def test_optimize_tracer_recovers_an_affine_model(monkeypatch):
    import paper_2602_10712_gb300 as srp
    from paper_2602_10712_gb300.design import optimize_tracer
    rng = np.random.default_rng(0)
    G, H, S = 4, 2, 6
    A = rng.normal(size=(S * 6, G * 2))
    Bm = rng.normal(size=(S * 6, H))
    c = rng.normal(size=S * 6)
    state = {}

    def forces(rho, ang):
        return (A @ np.asarray(rho, np.float64).ravel() + Bm @ ang + c).reshape(S, 6)

    monkeypatch.setattr(srp, "srp_design_instantiate", lambda v, vh, hg, ang: state.__setitem__("ang", np.array(ang)))
    monkeypatch.setattr(srp, "srp_build_bvh", lambda ctx, v, t, g, w: types.SimpleNamespace(close=lambda: None))
    refits = []
    monkeypatch.setattr(srp, "srp_bvh_refit", lambda ctx, b, v, t: refits.append(1))
    monkeypatch.setattr(srp, "srp_force", lambda ctx, bvhs, rho, sun, com, **kw: forces(rho[0], state["ang"])[None])

    def grad(ctx, b, rho, sun, com, up, tri_hinge=None, hinge_axes=None, **kw):
        u = np.asarray(up).ravel()
        return (A.T @ u).reshape(G, 2), Bm.T @ u

    monkeypatch.setattr(srp, "srp_force_grad", grad)
    rho_true = rng.uniform(0.05, 0.4, size=(G, 2))
    ang_true = np.array([0.3, -0.2])
    target = forces(rho_true, ang_true)
    mesh = types.SimpleNamespace(verts=None, vhinge=np.zeros(3, np.int32), hinges=None,
                                 tris=np.zeros((1, 3), np.int32), group=None)
    def run(lo, hi):
        return optimize_tracer(None, mesh, np.full((G, 2), 0.25), np.zeros(H), np.zeros((S, 3)), np.zeros(3),
                               target, steps=600, lr=0.01, hinge_lo=lo, hinge_hi=hi)

    # the generating design inside the admissible set: recovered
    rho, ang, losses = run(-1.0, 1.0)
    assert len(refits) == 600   # one host build, then a device refit per step
    assert losses[-1] < 1e-4 * losses[0]
    assert np.abs(rho - rho_true).max() < 0.02 and np.abs(ang - ang_true).max() < 0.02
    # a hinge range that excludes the first true angle (0.3): clipped to its bound
    rho, ang, losses = run(-0.25, 0.25)
    assert losses[-1] < losses[0]
    assert np.all(rho >= 0.0) and np.all(rho.sum(axis=1) <= 1.0 + 1e-12)
    assert np.all(np.abs(ang) <= 0.25 + 1e-12)
    assert ang[0] == pytest.approx(0.25)
