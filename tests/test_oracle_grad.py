"""Pins of the oracle's gradient (d upstream.(F,tau) / d(rho_s, rho_d,
hinge)) against finite differences of the oracle's forward estimate on the
same random numbers, against finite differences of the per-plate closed form
(box-wing model, Sec. 2.1) on an unoccluded panel, and sparsity."""

import numpy as np
import pytest

import oracle
import workloads as W


def _L(ft, up):
    return float(np.sum(ft * up))


@pytest.mark.parametrize("K", [1, 3])
def test_rho_gradient_matches_forward_fd(K):
    """Branch choice has fixed probability 1/2, so paths do not depend on rho
    and the estimate is a polynomial in rho (affine for K=1): central FD of
    the forward equals the reverse-mode gradient."""
    m = W.box_wing()
    rho = W.random_reflectances(64, seed=0).astype(np.float64)
    sun = np.stack([W.SUN_C1, np.array([-0.3, 0.5, 0.81]) / np.linalg.norm([-0.3, 0.5, 0.81])])
    up = np.random.default_rng(7).normal(size=(2, 6))
    nx = 48
    _, drho, _ = oracle.force_grad(m.verts, m.tris, m.group, rho, sun, np.zeros(3), up, nx=nx, K=K, seed=3)
    h = 1e-4
    for g in (0, 5, 12, 15):
        for j in (0, 1):
            rp = rho.copy(); rp[g, j] += h
            rm = rho.copy(); rm[g, j] -= h
            fp, _ = oracle.force(m.verts, m.tris, m.group, rp, sun, np.zeros(3), nx=nx, K=K, seed=3)
            fm, _ = oracle.force(m.verts, m.tris, m.group, rm, sun, np.zeros(3), nx=nx, K=K, seed=3)
            fd = (_L(fp, up) - _L(fm, up)) / (2 * h)
            assert abs(fd - drho[g, j]) <= 1e-7 * (abs(fd) + 1e-3), (g, j, fd, drho[g, j])
    # groups 16..63 hold no triangle: their gradient is exactly zero
    assert np.all(drho[16:] == 0.0)


def test_hinge_gradient_matches_fixed_hit_fd():
    """Analytic hinge derivative (hit points carried by their facet) equals
    the central difference of the same estimator re-evaluated at rotated
    geometry without re-tracing."""
    m = W.box_wing()
    rho = W.random_reflectances(64, seed=0)
    ang = np.array([0.3, -0.5])
    v = oracle.instantiate(m.verts, m.vhinge, m.hinges, ang)
    th = oracle.tri_hinge(m.tris, m.vhinge)
    sun = np.stack([W.SUN_C1, np.array([0.6, -0.2, 0.77]) / np.linalg.norm([0.6, -0.2, 0.77])])
    up = np.random.default_rng(8).normal(size=(2, 6))
    com = np.array([0.05, 0.0, -0.1])
    _, _, dh = oracle.force_grad(v, m.tris, m.group, rho, sun, com, up, nx=64, K=1, seed=4,
                                 tri_hinge=th, hinge_axes=m.hinges)
    fd = oracle.hinge_fd_fixed_hits(v, m.tris, m.group, rho, sun, com, up, th, m.hinges,
                                    nx=64, seed=4, h=1e-5)
    assert np.allclose(dh, fd, rtol=1e-7, atol=1e-9), (dh, fd)
    assert np.all(np.abs(dh) > 1e-3)


def test_hinge_gradient_matches_closed_form_fd():
    """On a lone hinged panel (no occluder), the estimator's hinge derivative
    converges to the derivative of the per-plate law P A cos G(n) with the
    panel rotated about its hinge (central FD of the closed form)."""
    bw = W.box_wing()
    verts = bw.verts[8:12].copy()
    tris = (bw.tris[12:14] - 8).astype(np.int32)
    vh = np.zeros(4, np.int32)
    hinges = bw.hinges[:1]
    group = np.zeros(2, np.int32)
    rho = np.array([[0.3, 0.25]])
    ang0 = 0.4
    e = np.array([0.35, 0.3, 0.89]); e /= np.linalg.norm(e)
    up = np.array([[0.3, -0.7, 1.1, 0.5, 0.2, -0.4]])
    com = np.array([0.0, 0.2, 0.1])
    v = oracle.instantiate(verts, vh, hinges, [ang0])
    _, _, dh = oracle.force_grad(v, tris, group, rho, e, com, up, nx=512, K=1, seed=2,
                                 tri_hinge=np.zeros(2, np.int32), hinge_axes=hinges)
    h = 1e-5
    fp = oracle.facet_law(oracle.instantiate(verts, vh, hinges, [ang0 + h], np.float64), tris, group, rho, e, com)
    fm = oracle.facet_law(oracle.instantiate(verts, vh, hinges, [ang0 - h], np.float64), tris, group, rho, e, com)
    fd = (np.sum(fp * up[0]) - np.sum(fm * up[0])) / (2 * h)
    assert abs(dh[0] - fd) <= 2e-3 * abs(fd), (dh, fd)


def test_force_grad_forward_equals_force():
    m = W.box_wing()
    rho = W.random_reflectances(64, seed=0)
    up = np.ones((1, 6))
    f1, _ = oracle.force(m.verts, m.tris, m.group, rho, W.SUN_C1, np.zeros(3), nx=32, K=2)
    f2, _, _ = oracle.force_grad(m.verts, m.tris, m.group, rho, W.SUN_C1, np.zeros(3), up, nx=32, K=2)
    assert np.array_equal(f1, f2)
