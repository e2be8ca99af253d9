"""FP64 CPU oracle of the SRP ray-grid estimator -- TEST INFRASTRUCTURE.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  The product library never does, and
the two share no code: the oracle is plain C (srp_oracle.c, brute force over
all triangles, no BVH) plus the numpy helpers below, each written from the
paper's definitions:

* ``force``            -- the ray-grid Monte Carlo estimate of F and tau
                          (Sec. 3.2, Eq. Force and the torque integral), see
                          the step list at the top of srp_oracle.c.
* ``force_grad``       -- d(upstream . (F,tau)) / d(rho_s, rho_d, hinge)
                          of that same estimate (Sec. 4.1 "differentiable by
                          construction" w.r.t. reflectance; hinge angles in
                          the fixed-visibility reading).
* ``facet_law``        -- the per-plate closed form (box-wing model,
                          Sec. 2.1): sum over sunlit facets of
                          P A cos [(1-rs) d - (2 rs cos + 2/3 rd) n].
* ``force_area``       -- the paper's own estimator without bounces
                          (Sec. 3.2 "Estimation"): area-weighted surface
                          samples, a shadow ray toward the sun per sample
                          (next-event estimation), the per-plate expected
                          reflection deposited where the sample is lit.
* ``area_counts``      -- its sample allocation n_f = max(1, ceil(rho A_f)).
* ``force_thermal``    -- local Lambertian thermal emitters (Sec. 5.9):
                          expected 2/3 recoil at the emitting surface plus
                          the closed-form deposit where emitted packets hit
                          the spacecraft; ``thermal_counts`` its allocation.
* ``trace_samples``    -- per-sample designs (Sec. 3.2 "Estimation", Alg. 1
                          NNLoss): each sample instantiates its own design
                          and traces one jittered ray over a fixed square by
                          brute force.
* ``instantiate``      -- design instantiation: hinge rotations of the
                          panel vertices (Rodrigues' formula).
* ``philox``           -- Philox4x32-10 (Salmon et al., SC'11).

Pins (tests/test_oracle_*.py) tie these to closed forms, published test
vectors and brute-force invariants, not to the CUDA path.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess

import numpy as np


def host_threads() -> int:
    """Worker threads of the multi-threaded oracle calls: the CPUs this
    process may run on (its affinity mask), else the machine's count."""
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except (AttributeError, OSError):
        return os.cpu_count() or 1

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_SO = os.path.join(_LIBDIR, "libsrp_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile srp_oracle.c with gcc (portable flags: no -march)."""
    src = os.path.join(_HERE, "srp_oracle.c")
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread",
                               "-fno-fast-math", "-ffp-contract=off", src, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_SO)
        P = C.c_void_p
        i32, i64, u32, u64, f64 = C.c_int, C.c_int64, C.c_uint32, C.c_uint64, C.c_double
        lib.or_philox4x32_10.argtypes = [P, P, P]
        lib.or_onb.argtypes = [P, P, P]
        lib.or_grid.argtypes = [P, i32, P, P]
        lib.or_force.argtypes = [P, i32, P, P, i32, P, i32, P, i32, P,
                                 i32, i32, i32, i32, u64, f64,
                                 i64, i64, i64, u32, u32,
                                 i32, P, P,
                                 P, P, P, i32, P, P]
        lib.or_force.restype = i32
        lib.or_hinge_fd_fixed_hits.argtypes = [P, i32, P, P, i32, P, i32, P, i32, P,
                                               i32, i32, i32, u64, f64,
                                               P, P, P, i32, f64, P]
        lib.or_primary_hit.argtypes = [P, i32, P, i32, P, i32, i32, i32, u64, u32, u32, i64, P]
        lib.or_primary_hit.restype = i32
        lib.or_trace_rays.argtypes = [P, i32, P, P, i32, P, P, P, i32, i32, i32, i32, u64, f64,
                                      u32, u32, P, i64, P, P, i32]
        lib.or_trace_rays.restype = i32
        lib.or_area_counts.argtypes = [P, i32, P, i32, C.c_float, P]
        lib.or_area_counts.restype = i64
        lib.or_force_area.argtypes = [P, i32, P, P, i32, P, P, i32, P, C.c_float, u64, f64, u32, u32, i32, i32, P, P]
        lib.or_force_area.restype = i32
        lib.or_thermal_counts.argtypes = [P, i32, P, P, i32, P, C.c_float, P]
        lib.or_thermal_counts.restype = i64
        lib.or_force_thermal.argtypes = [P, i32, P, P, i32, P, P, P, C.c_float, u64, f64, u32, i32, P, P, P]
        lib.or_force_thermal.restype = i32
        lib.or_trace_samples.argtypes = [P, i32, P, P, i32, P, P, i32, P, P, i32, P, P, i64, P, f64, i32, u64, f64,
                                         u32, i32, P, P]
        lib.or_trace_samples.restype = i32
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def philox(counter, key):
    """Philox4x32-10 of one 4x32 counter and 2x32 key -> 4 uint32."""
    lib = _load()
    c = _c(counter, np.uint32); k = _c(key, np.uint32); o = np.zeros(4, np.uint32)
    lib.or_philox4x32_10(_p(c), _p(k), _p(o))
    return o


def onb(n):
    lib = _load()
    n = _c(n, np.float64); b1 = np.zeros(3); b2 = np.zeros(3)
    lib.or_onb(_p(n), _p(b1), _p(b2))
    return b1, b2


def grid(verts):
    """Grid centre (vertex AABB centre) and radius (max distance) in FP64."""
    lib = _load()
    v = _c(verts, np.float32); c = np.zeros(3); R = np.zeros(1)
    lib.or_grid(_p(v), int(v.shape[0]), _p(c), _p(R))
    return c, float(R[0])


def force(verts, tris, group, rho, sun, com, *, nx, ny=None, K=1, jitter=1, seed=0, P=1.0,
          ray_offset=0, ray_stride=1, ray_count=0, sun_base=0, design_index=0,
          threads=None):
    """Ray-grid F,tau of one design: returns (ft [S,6], sigma [S,6])."""
    lib = _load()
    ny = nx if ny is None else ny
    v = _c(verts, np.float32); t = _c(tris, np.int32); g = _c(group, np.int32)
    r = _c(rho, np.float64); s = _c(np.atleast_2d(sun), np.float64); cm = _c(com, np.float64)
    S = s.shape[0]
    ft = np.zeros((S, 6)); sg = np.zeros((S, 6))
    threads = threads or host_threads()
    rc = lib.or_force(_p(v), v.shape[0], _p(t), _p(g), t.shape[0], _p(r), r.shape[0], _p(s), S, _p(cm),
                      nx, ny, K, jitter, seed, P, ray_offset, ray_stride, ray_count,
                      sun_base, design_index, threads, _p(ft), _p(sg),
                      None, None, None, 0, None, None)
    if rc != 0:
        raise ValueError("oracle force: bad arguments")
    return ft, sg


def force_grad(verts, tris, group, rho, sun, com, upstream, *, nx, ny=None, K=1, jitter=1,
               seed=0, P=1.0, tri_hinge=None, hinge_axes=None, ray_offset=0, ray_stride=1,
               ray_count=0, sun_base=0, design_index=0, threads=None):
    """Gradient of L = sum_s upstream[s].(F_s,tau_s): (ft, d_rho [G,2], d_hinge [H])."""
    lib = _load()
    ny = nx if ny is None else ny
    v = _c(verts, np.float32); t = _c(tris, np.int32); g = _c(group, np.int32)
    r = _c(rho, np.float64); s = _c(np.atleast_2d(sun), np.float64); cm = _c(com, np.float64)
    up = _c(np.atleast_2d(upstream), np.float64)
    S = s.shape[0]; G = r.shape[0]
    if tri_hinge is None:
        th = np.full(t.shape[0], -1, np.int32); ha = np.zeros((0, 6)); H = 0
    else:
        th = _c(tri_hinge, np.int32); ha = _c(hinge_axes, np.float64).reshape(-1, 6); H = ha.shape[0]
    ft = np.zeros((S, 6)); drho = np.zeros((G, 2)); dh = np.zeros(max(H, 1))
    threads = threads or host_threads()
    rc = lib.or_force(_p(v), v.shape[0], _p(t), _p(g), t.shape[0], _p(r), G, _p(s), S, _p(cm),
                      nx, ny, K, jitter, seed, P, ray_offset, ray_stride, ray_count,
                      sun_base, design_index, threads, _p(ft), None,
                      _p(up), _p(th), _p(ha), H, _p(drho), _p(dh))
    if rc != 0:
        raise ValueError("oracle force_grad: bad arguments")
    return ft, drho, dh[:H]


def hinge_fd_fixed_hits(verts, tris, group, rho, sun, com, upstream, tri_hinge, hinge_axes,
                        *, nx, ny=None, jitter=1, seed=0, P=1.0, h=1e-6):
    """Central difference in the hinge angles of the K=1 estimator with
    every hit carried rigidly by its facet (no re-tracing)."""
    lib = _load()
    ny = nx if ny is None else ny
    v = _c(verts, np.float32); t = _c(tris, np.int32); g = _c(group, np.int32)
    r = _c(rho, np.float64); s = _c(np.atleast_2d(sun), np.float64); cm = _c(com, np.float64)
    up = _c(np.atleast_2d(upstream), np.float64)
    th = _c(tri_hinge, np.int32); ha = _c(hinge_axes, np.float64).reshape(-1, 6)
    out = np.zeros(ha.shape[0])
    lib.or_hinge_fd_fixed_hits(_p(v), v.shape[0], _p(t), _p(g), t.shape[0], _p(r), r.shape[0],
                               _p(s), s.shape[0], _p(cm), nx, ny, jitter, seed, P,
                               _p(up), _p(th), _p(ha), ha.shape[0], h, _p(out))
    return out


def trace_rays(verts, tris, group, rho, sun, com, ray_idx, *, nx, ny=None, K=1, jitter=1, seed=0,
               P=1.0, sun_index=0, design_index=0, threads=None):
    """Per-ray samples: (y [n,6] force/torque deposits, hits [n,K] original
    triangle index per bounce, -1 after the path ends)."""
    lib = _load()
    ny = nx if ny is None else ny
    v = _c(verts, np.float32); t = _c(tris, np.int32); g = _c(group, np.int32)
    r = _c(rho, np.float64); s = _c(sun, np.float64).reshape(3); cm = _c(com, np.float64)
    idx = _c(ray_idx, np.int64)
    y = np.zeros((idx.shape[0], 6)); h = np.zeros((idx.shape[0], K), np.int32)
    rc = lib.or_trace_rays(_p(v), v.shape[0], _p(t), _p(g), t.shape[0], _p(r), _p(s), _p(cm),
                           nx, ny, K, jitter, seed, P, sun_index, design_index, _p(idx), idx.shape[0],
                           _p(y), _p(h), threads or host_threads())
    if rc != 0:
        raise ValueError("oracle trace_rays: bad arguments")
    return y, h


def area_counts(verts, tris, density):
    """Samples per triangle of the area estimator: max(1, ceil(density*A)) in FP32."""
    lib = _load()
    v = _c(verts, np.float32); t = _c(tris, np.int32)
    c = np.zeros(t.shape[0], np.int32)
    lib.or_area_counts(_p(v), v.shape[0], _p(t), t.shape[0], float(density), _p(c))
    return c


def force_area(verts, tris, group, rho, sun, com, *, density, seed=0, P=1.0, sun_base=0, design_index=0,
               K=1, threads=None):
    """Area-sampling / next-event estimate of (F, tau) [S,6] and sigma [S,6];
    K = 2 adds one gathered Lambertian interreflection per sample and side."""
    if K not in (1, 2):
        raise ValueError("force_area: K must be 1 or 2")
    lib = _load()
    v = _c(verts, np.float32); t = _c(tris, np.int32); g = _c(group, np.int32)
    r = _c(rho, np.float64); s = _c(np.atleast_2d(sun), np.float64); cm = _c(com, np.float64)
    S = s.shape[0]
    ft = np.zeros((S, 6)); sg = np.zeros((S, 6))
    lib.or_force_area(_p(v), v.shape[0], _p(t), _p(g), t.shape[0], _p(r), _p(s), S, _p(cm), float(density), seed,
                      P, sun_base, design_index, K, threads or host_threads(), _p(ft), _p(sg))
    return ft, sg


def thermal_counts(verts, tris, group, emit, density):
    """Samples per triangle of the thermal estimator (0 where emit == 0)."""
    lib = _load()
    v = _c(verts, np.float32); t = _c(tris, np.int32); g = _c(group, np.int32); e = _c(emit, np.float32)
    c = np.zeros(t.shape[0], np.int32)
    lib.or_thermal_counts(_p(v), v.shape[0], _p(t), _p(g), t.shape[0], _p(e), float(density), _p(c))
    return c


def force_thermal(verts, tris, group, rho, emit, com, *, density, seed=0, P=1.0, design_index=0, threads=None):
    """Thermal-emitter estimate of (F, tau) [6], sigma [6] and the sample count."""
    lib = _load()
    v = _c(verts, np.float32); t = _c(tris, np.int32); g = _c(group, np.int32)
    r = _c(rho, np.float64); e = _c(emit, np.float32); cm = _c(com, np.float64)
    ft = np.zeros(6); sg = np.zeros(6); n = np.zeros(1, np.int64)
    lib.or_force_thermal(_p(v), v.shape[0], _p(t), _p(g), t.shape[0], _p(r), _p(e), _p(cm), float(density), seed,
                         P, design_index, threads or host_threads(), _p(ft), _p(sg), _p(n))
    return ft, sg, int(n[0])


def trace_samples(verts, vhinge, hinges, tris, group, angles, rho, sun, com, center, R, *, K=1, seed=0, P=1.0,
                  sample_base=0, threads=None):
    """Per-sample designs: (y [N,6], hits [N,K]) of one jittered ray per
    sample over its own instantiated mesh (brute force)."""
    lib = _load()
    v = _c(verts, np.float32); vh = _c(vhinge, np.int32); hg = _c(np.reshape(hinges, (-1, 6)), np.float64)
    t = _c(tris, np.int32); g = _c(group, np.int32)
    an = _c(np.reshape(angles, (np.shape(angles)[0], -1)), np.float64)
    r = _c(rho, np.float64); sn = _c(sun, np.float64); cm = _c(com, np.float64); ce = _c(center, np.float64)
    N = sn.shape[0]
    H = hg.shape[0]
    y = np.zeros((N, 6)); hits = np.zeros((N, K), np.int32)
    lib.or_trace_samples(_p(v), v.shape[0], _p(vh), _p(hg), H, _p(t), _p(g), t.shape[0], _p(an), _p(r), r.shape[-2],
                         _p(sn), _p(cm), N, _p(ce), float(R), K, seed, P, sample_base, threads or host_threads(),
                         _p(y), _p(hits))
    return y, hits


def primary_hit(verts, tris, sun, i, *, nx, ny=None, jitter=1, seed=0, sun_index=0, design_index=0):
    """Hit triangle (or -1) and t of primary grid ray i."""
    lib = _load()
    ny = nx if ny is None else ny
    v = _c(verts, np.float32); t = _c(tris, np.int32); s = _c(sun, np.float64)
    tt = np.zeros(1)
    f = lib.or_primary_hit(_p(v), v.shape[0], _p(t), t.shape[0], _p(s), nx, ny, jitter, seed,
                           sun_index, design_index, int(i), _p(tt))
    return int(f), float(tt[0])


# --------------------------------------------------------------------------
# numpy helpers (plain definitions)
# --------------------------------------------------------------------------
def rotation(axis, angle):
    """Rodrigues rotation matrix about a unit axis."""
    a = np.asarray(axis, np.float64)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(angle) * K + (1.0 - math.cos(angle)) * (K @ K)


def instantiate(verts, vhinge, hinges, angles, dtype=np.float32):
    """Design instantiation: rotate every hinged vertex about its hinge axis
    (point p, unit axis a) by its angle; returns [V,3] (float32 default)."""
    v = np.asarray(verts, np.float64).copy()
    for h in range(len(angles)):
        p = hinges[h, :3]; a = hinges[h, 3:]
        Rm = rotation(a, angles[h])
        sel = np.asarray(vhinge) == h
        v[sel] = (v[sel] - p) @ Rm.T + p
    return v.astype(dtype)


def tri_hinge(tris, vhinge):
    """Hinge id of each triangle (that of its first vertex, -1 if fixed)."""
    return np.asarray(vhinge)[np.asarray(tris)[:, 0]].astype(np.int32)


def facet_law(verts, tris, group, rho, sun, com, P=1.0):
    """Per-plate closed form for a body whose sunlit facets are all fully
    unoccluded (convex bodies, single plates): each facet whose OUTWARD
    normal faces the sun contributes P A cos [(1-rs) d - (2 rs cos + 2/3 rd) n]
    and the torque (centroid - COM) x that.  Returns [6]."""
    v = np.asarray(verts, np.float64)[np.asarray(tris)]
    e = np.asarray(sun, np.float64)
    d = -e / np.linalg.norm(e)
    out = np.zeros(6)
    for f in range(v.shape[0]):
        cr = np.cross(v[f, 1] - v[f, 0], v[f, 2] - v[f, 0])
        A = 0.5 * np.linalg.norm(cr)
        n = cr / np.linalg.norm(cr)
        cs = -(n @ d)
        if cs <= 0.0:
            continue
        rs, rd = np.asarray(rho, np.float64)[group[f]]
        F = P * A * cs * ((1.0 - rs) * d - (2.0 * rs * cs + 2.0 / 3.0 * rd) * n)
        cen = v[f].mean(axis=0)
        out[:3] += F
        out[3:] += np.cross(cen - np.asarray(com, np.float64), F)
    return out
