"""Pin of the oracle's hinge derivative for paths with bounces (K > 1).

The oracle differentiates each path in the fixed-visibility reading (its
facets, branch choices and random draws held; facets on the hinge turn;
later hits re-intersected with their facets' planes).  Where no facet of a
path's primary hit turns and no ray crosses a facet edge for small angles,
that reading is exactly the derivative of the estimator itself, re-traced.
Scene: a fixed 45-degree mirror (rho_s = 1, rho_d = 0) under a sun at +z
reflects the rays horizontally onto a vertical plate that turns about its
vertical edge; direct sun rays graze the plate (parallel to its plane) and
never hit it; unreferenced anchor vertices fix the ray grid's centre and
radius.  The oracle's K = 2 hinge gradient must equal the central
difference of up . (F, tau) over re-traced estimates at +-1e-3 rad."""
import numpy as np

from oracle import force, force_grad, instantiate


def _scene():
    r2 = np.sqrt(0.5)
    u1 = np.array([r2, 0.0, -r2])
    u2 = np.array([0.0, 1.0, 0.0])
    mirror = [s1 * u1 + s2 * u2 for s1, s2 in ((-1, -1), (1, -1), (1, 1), (-1, 1))]
    plate = [np.array([3.0, y, z]) for y, z in ((-1.5, -1.5), (1.5, -1.5), (1.5, 1.5), (-1.5, 1.5))]
    anchors = [np.array([sx, sy, sz]) * 5.0 for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)]
    verts = np.array(mirror + plate + anchors, np.float32)
    tris = np.array([[0, 1, 2], [0, 2, 3], [4, 5, 6], [4, 6, 7]], np.int32)
    group = np.array([0, 0, 1, 1], np.int32)
    vhinge = np.array([-1] * 4 + [0] * 4 + [-1] * 8, np.int32)
    hinges = np.array([[3.0, -1.5, 0.0, 0.0, 0.0, 1.0]])
    rho = np.array([[1.0, 0.0], [0.3, 0.4]])
    return verts, tris, group, vhinge, hinges, rho


def test_k2_hinge_gradient_equals_retraced_difference():
    verts, tris, group, vhinge, hinges, rho = _scene()
    sun = np.array([[0.0, 0.0, 1.0]])
    com = np.array([0.5, 0.2, -0.1])
    up = np.array([[0.3, -1.2, 0.7, 0.5, 0.9, -0.4]])
    kw = dict(nx=256, K=2, jitter=0, seed=3, P=1.0)
    th = np.array([vhinge[t[0]] for t in tris], np.int32)
    v0 = instantiate(verts, vhinge, hinges, np.array([0.05]))
    _, _, dh = force_grad(v0, tris, group, rho, sun, com, up, tri_hinge=th, hinge_axes=hinges, **kw)
    dlt = 1e-3
    vals = []
    for a in (0.05 + dlt, 0.05 - dlt):
        ft, _ = force(instantiate(verts, vhinge, hinges, np.array([a])), tris, group, rho, sun, com, **kw)
        vals.append(float(np.sum(up * ft)))
    fd = (vals[0] - vals[1]) / (2 * dlt)
    assert abs(fd) > 1e-3   # the plate's turn moves the deposits
    assert abs(dh[0] - fd) <= 1e-4 * abs(fd), (dh[0], fd)
