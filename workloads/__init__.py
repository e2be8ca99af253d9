"""Seeded synthetic inputs for the solar-radiation-pressure (SRP) tracer.

This module is shared by the CUDA path, the FP64 oracle and the benchmark.
It only *generates inputs*: triangle meshes in their rest pose, hinge
definitions, material-group assignments, reflectances and sun directions.
It holds none of the method's arithmetic (no ray generation, intersection,
shading, design instantiation or reduction); each side of the parity tests
implements those on its own.

The paper's spacecraft meshes are not available, so the workloads below are
procedural stand-ins shaped like the paper's: a box-wing body (the classic
"box-wing" decomposition of Sec. 2.1) and a ~50k-triangle satellite with a
tessellated paraboloid dish and random appendages, in the triangle-count
range of the paper's speed table (Sec. 4.1, Table "Speed": 40 to 24,746
triangles).

Conventions (all arrays are numpy):
  verts  float32 [V, 3]   rest-pose vertex positions in metres
  tris   int32   [T, 3]   vertex indices, counter-clockwise seen from the
                          outside for closed parts (outward normal)
  group  int32   [T]      material group of each triangle, 0 <= g < G
  vhinge int32   [V]      hinge id of each vertex, -1 for fixed vertices
  hinges float64 [H, 6]   per hinge: a point on the axis (3) and the unit
                          axis direction (3); positive angles rotate by the
                          right-hand rule about the axis
  rho    float32 [G, 2]   per group (specular rho_s, diffuse rho_d)
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Mesh", "box_wing", "box_wing_7group", "procedural_satellite",
    "random_reflectances", "fibonacci_directions", "random_unit_vectors",
    "config1", "config2", "config5_designs", "flat_plate", "icosphere",
    "axis_box", "SUN_C1", "orbit_states",
]

#: Sun direction of the single-direction box-wing workload, e = (1,2,3)/|.|.
SUN_C1 = np.array([1.0, 2.0, 3.0]) / math.sqrt(14.0)


@dataclasses.dataclass
class Mesh:
    verts: np.ndarray           # float32 [V,3]
    tris: np.ndarray            # int32 [T,3]
    group: np.ndarray           # int32 [T]
    vhinge: np.ndarray          # int32 [V]
    hinges: np.ndarray          # float64 [H,6]
    n_groups: int = 64

    @property
    def T(self) -> int:
        return int(self.tris.shape[0])

    @property
    def V(self) -> int:
        return int(self.verts.shape[0])

    @property
    def H(self) -> int:
        return int(self.hinges.shape[0])


def _quad(a, b, c, d):
    """Two triangles (a,b,c), (a,c,d) of a planar quad a-b-c-d (CCW)."""
    return [(a, b, c), (a, c, d)]


def axis_box(center, half, v0: int):
    """Closed axis-aligned box: 8 corners and 12 CCW (outward) triangles.

    Returns (verts [8,3], tris [12,3] offset by v0)."""
    cx, cy, cz = center
    hx, hy, hz = half
    v = np.array([[cx + sx * hx, cy + sy * hy, cz + sz * hz]
                  for sz in (-1, 1) for sy in (-1, 1) for sx in (-1, 1)])
    # corner index = (sz>0)*4 + (sy>0)*2 + (sx>0)
    t = []
    t += _quad(1, 3, 7, 5)   # +x
    t += _quad(0, 4, 6, 2)   # -x
    t += _quad(2, 6, 7, 3)   # +y
    t += _quad(0, 1, 5, 4)   # -y
    t += _quad(4, 5, 7, 6)   # +z
    t += _quad(0, 2, 3, 1)   # -z
    return v, np.asarray(t, dtype=np.int64) + v0


def box_wing():
    """Box-wing body: 1x1x2 m bus (12 triangles) + two 5x2 m panels (4).

    Bus x,y in [-0.5,0.5], z in [-1,1].  Panels lie in z = 0 with
    x in [-1,1] and y in [0.5,5.5] / [-5.5,-0.5]; each rotates about a hinge
    axis along +y through (0, +-0.5, 0) (angle 0 = panel normal along z).
    Triangle f is in material group f (16 of 64 groups used)."""
    bv, bt = axis_box((0.0, 0.0, 0.0), (0.5, 0.5, 1.0), 0)
    pv = np.array([[-1.0, 0.5, 0.0], [1.0, 0.5, 0.0], [1.0, 5.5, 0.0], [-1.0, 5.5, 0.0],
                   [-1.0, -0.5, 0.0], [-1.0, -5.5, 0.0], [1.0, -5.5, 0.0], [1.0, -0.5, 0.0]])
    pt = np.array(_quad(8, 9, 10, 11) + _quad(12, 13, 14, 15))
    verts = np.concatenate([bv, pv]).astype(np.float32)
    tris = np.concatenate([bt, pt]).astype(np.int32)
    vhinge = np.array([-1] * 8 + [0] * 4 + [1] * 4, dtype=np.int32)
    hinges = np.array([[0.0, 0.5, 0.0, 0.0, 1.0, 0.0],
                       [0.0, -0.5, 0.0, 0.0, 1.0, 0.0]])
    group = np.arange(16, dtype=np.int32)
    return Mesh(verts, tris, group, vhinge, hinges, 64)


def box_wing_7group():
    """Box-wing with 7 material groups: bus face j -> group j (j<6), both
    panels -> group 6.  Its design vector has 16 entries: 7 rho_s, 7 rho_d
    and 2 hinge angles."""
    m = box_wing()
    g = np.empty(16, dtype=np.int32)
    g[:12] = np.arange(12) // 2
    g[12:] = 6
    return Mesh(m.verts, m.tris, g, m.vhinge, m.hinges, 7)


def random_reflectances(n_groups: int, seed: int = 0, hi: float = 0.5):
    """rho_s, rho_d ~ U[0, hi] per group (group order, rho_s then rho_d)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, hi, size=(n_groups, 2)).astype(np.float32)


def _paraboloid_dish(z0, focal, radius, segments, rings, v0):
    """Open paraboloid z = z0 + r^2/(4 f), r <= radius; a fan of `segments`
    triangles at the apex and (rings-1) rings of quads."""
    j = np.arange(1, rings + 1, dtype=np.float64)
    r = radius * j / rings
    a = 2.0 * math.pi * np.arange(segments, dtype=np.float64) / segments
    ring_v = np.stack([np.outer(r, np.cos(a)), np.outer(r, np.sin(a)),
                       np.repeat((z0 + r * r / (4.0 * focal))[:, None], segments, axis=1)], axis=-1)
    verts = np.concatenate([np.array([[0.0, 0.0, z0]]), ring_v.reshape(-1, 3)])
    s_ = np.arange(segments)
    ring = lambda jj, ss: 1 + (jj - 1) * segments + (ss % segments)
    fan = np.stack([np.zeros(segments, np.int64), ring(1, s_), ring(1, s_ + 1)], axis=1)
    jj = np.arange(1, rings)[:, None]
    a_, b_ = ring(jj, s_), ring(jj, s_ + 1)
    c_, d_ = ring(jj + 1, s_ + 1), ring(jj + 1, s_)
    quads = np.stack([np.stack([a_, d_, c_], -1), np.stack([a_, c_, b_], -1)], axis=2).reshape(-1, 3)
    tris = np.concatenate([fan, quads]).astype(np.int64)
    return verts, tris + v0


def procedural_satellite(seed: int = 1, dish_segments: int = 256, dish_rings: int = 93,
                         n_boxes: int = 200, group_seed: int = 2, n_groups: int = 64):
    """~50k-triangle satellite: box-wing (16) + paraboloid dish on +z
    (f = 1 m, radius 1.5 m, 256 x 93 -> 47,360 triangles) + 200 random
    axis-aligned boxes (edge U[0.05,0.5] m, centres uniform in a 3 m ball,
    2,400 triangles) = 49,776 triangles; groups uniform over 64."""
    bw = box_wing()
    vs = [bw.verts.astype(np.float64)]
    ts = [bw.tris.astype(np.int64)]
    vh = [bw.vhinge]
    nv = bw.V
    dv, dt = _paraboloid_dish(1.0, 1.0, 1.5, dish_segments, dish_rings, nv)
    vs.append(dv); ts.append(dt); vh.append(np.full(len(dv), -1, np.int32)); nv += len(dv)
    rng = np.random.default_rng(seed)
    for _ in range(n_boxes):
        while True:
            c = rng.uniform(-3.0, 3.0, 3)
            if c @ c <= 9.0:
                break
        h = 0.5 * rng.uniform(0.05, 0.5, 3)
        bv, bt = axis_box(c, h, nv)
        vs.append(bv); ts.append(bt); vh.append(np.full(8, -1, np.int32)); nv += 8
    verts = np.concatenate(vs).astype(np.float32)
    tris = np.concatenate(ts).astype(np.int32)
    grng = np.random.default_rng(group_seed)
    group = grng.integers(0, n_groups, size=len(tris)).astype(np.int32)
    return Mesh(verts, tris, group, np.concatenate(vh).astype(np.int32), bw.hinges.copy(), n_groups)


def fibonacci_directions(n: int) -> np.ndarray:
    """Fibonacci sphere: z = 1-(2i+1)/n, phi = i*pi*(3-sqrt 5); float64 [n,3]."""
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    phi = i * math.pi * (3.0 - math.sqrt(5.0))
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    d = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def random_unit_vectors(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def flat_plate(size=(2.0, 1.0), normal_axis: int = 2):
    """Single rectangular plate (2 triangles) centred at the origin, normal
    along +axis `normal_axis`; both triangles in group 0."""
    a, b = size[0] / 2.0, size[1] / 2.0
    q = np.array([[-a, -b], [a, -b], [a, b], [-a, b]])
    v = np.zeros((4, 3))
    ax = [(1, 2), (2, 0), (0, 1)][normal_axis]
    v[:, ax[0]] = q[:, 0]
    v[:, ax[1]] = q[:, 1]
    tris = np.array(_quad(0, 1, 2, 3), dtype=np.int32)
    return Mesh(v.astype(np.float32), tris, np.zeros(2, np.int32),
                np.full(4, -1, np.int32), np.zeros((0, 6)), 1)


def icosphere(subdiv: int, radius: float = 1.0):
    """Geodesic sphere (icosahedron subdivided `subdiv` times, vertices
    projected to the sphere), outward CCW triangles, one group."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t),
         (0, -1, -t), (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    v = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in v]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
         (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
         (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(subdiv):
        cache = {}
        nf = []

        def mid(i, j):
            key = (min(i, j), max(i, j))
            if key not in cache:
                m = v[i] + v[j]
                v.append(m / np.linalg.norm(m))
                cache[key] = len(v) - 1
            return cache[key]
        for (a, b, c) in f:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        f = nf
    verts = (np.asarray(v) * radius).astype(np.float32)
    return Mesh(verts, np.asarray(f, dtype=np.int32), np.zeros(len(f), np.int32),
                np.full(len(verts), -1, np.int32), np.zeros((0, 6)), 1)


def config1():
    """Box-wing, 64 groups (facet f -> group f), rho ~ U[0,0.5] seed 0,
    one sun direction (1,2,3)/sqrt(14), COM at the origin."""
    m = box_wing()
    rho = random_reflectances(64, seed=0)
    return m, rho, SUN_C1[None, :].copy(), np.zeros(3)


def config2(n_sun: int = 4096):
    """~50k-triangle procedural satellite, 64 groups, Fibonacci suns."""
    m = procedural_satellite()
    rho = random_reflectances(64, seed=0)
    return m, rho, fibonacci_directions(n_sun), np.zeros(3)


def config5_designs(n_designs: int = 256, t_lo: int = 5000, t_hi: int = 200000, seed: int = 5):
    """Designs with log-uniform triangle counts in [t_lo, t_hi]: the
    procedural satellite with its dish ring count and box count scaled."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_designs):
        T = int(round(math.exp(rng.uniform(math.log(t_lo), math.log(t_hi)))))
        seg = 128 if T < 40000 else 256
        rings = max(2, int(round((0.95 * T - 16) / (2 * seg))))
        dish = seg * (2 * rings - 1)
        nb = max(1, int(round((T - 16 - dish) / 12)))
        out.append(procedural_satellite(seed=1000 + k, dish_segments=seg, dish_rings=rings,
                                        n_boxes=nb, group_seed=2000 + k))
    return out


def orbit_states(n: int, seed: int, radius: float = 26560e3, inc_deg: float = 55.0,
                 gm: float = 3.986004418e14) -> np.ndarray:
    """Initial states of the orbit workload, float64 [n, 13] = (r, v, q, w):
    circular orbits of the given radius and inclination (a GPS-like orbit by
    default) with the node and the argument of latitude uniform in
    [0, 2 pi), a uniformly random unit attitude quaternion (scalar first)
    and a body rate with components N(0, 1e-4) rad/s."""
    rng = np.random.default_rng(seed)
    raan = rng.uniform(0.0, 2.0 * math.pi, n)
    u = rng.uniform(0.0, 2.0 * math.pi, n)
    inc = math.radians(inc_deg)
    speed = math.sqrt(gm / radius)
    cO, sO, cu, su = np.cos(raan), np.sin(raan), np.cos(u), np.sin(u)
    ci, si = math.cos(inc), math.sin(inc)
    # in-plane unit vectors: radial p and along-track t
    p = np.stack([cO * cu - sO * su * ci, sO * cu + cO * su * ci, su * si], axis=1)
    t = np.stack([-cO * su - sO * cu * ci, -sO * su + cO * cu * ci, cu * si], axis=1)
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w = rng.normal(scale=1e-4, size=(n, 3))
    return np.concatenate([radius * p, speed * t, q, w], axis=1)
