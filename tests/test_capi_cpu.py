"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads, and
exports every function include/srp.h declares; host-only entry points
(design instantiation, BVH construction) are checked against the oracle's
definitions and the BVH's structural invariants.  No GPU needed."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle
import paper_2602_10712_gb300 as srp
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(srp_\w+)\s*\(", txt, flags=re.M))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    lib = srp.load()
    names = declared_functions()
    assert "srp_force" in names and "srp_build_bvh" in names and len(names) >= 10
    for n in names:
        assert hasattr(lib, n), f"libsrp.so does not export {n}"


def test_design_instantiate_matches_oracle():
    m = W.box_wing()
    ang = np.array([0.7, -1.2])
    a = srp.srp_design_instantiate(m.verts, m.vhinge, m.hinges, ang)
    b = oracle.instantiate(m.verts, m.vhinge, m.hinges, ang)
    assert np.allclose(a, b, atol=2e-6)
    assert np.array_equal(a[:8], m.verts[:8])


def test_design_instantiate_rejects_bad_axis():
    m = W.box_wing()
    h = m.hinges.copy(); h[0, 3:] = [0, 2, 0]
    with pytest.raises(srp.SRPError) as ei:
        srp.srp_design_instantiate(m.verts, m.vhinge, h, [0.1, 0.2])
    assert ei.value.code == srp.SRP_EINVAL


def _walk(nodes, W_, T, verts, tris, order):
    nf = 32 if W_ == 4 else 64
    nodes = nodes.reshape(-1, nf)
    seen = np.zeros(T, int)

    def box(n, c):
        lo = np.array([nodes[n, 0 * W_ + c], nodes[n, 2 * W_ + c], nodes[n, 4 * W_ + c]])
        hi = np.array([nodes[n, 1 * W_ + c], nodes[n, 3 * W_ + c], nodes[n, 5 * W_ + c]])
        return lo, hi

    stack = [(0, None)]
    visited = 0
    while stack:
        n, parent_box = stack.pop()
        visited += 1
        ch = nodes[n, 6 * W_:7 * W_].view(np.int32)
        for c in range(W_):
            lo, hi = box(n, c)
            if lo[0] > hi[0]:
                continue  # empty slot
            if parent_box is not None:
                assert np.all(lo >= parent_box[0] - 1e-6) and np.all(hi <= parent_box[1] + 1e-6)
            if ch[c] >= 0:
                assert ch[c] > n
                stack.append((int(ch[c]), (lo, hi)))
            else:
                code = ~int(ch[c])
                first, cnt = code >> 3, (code & 7) + 1
                for k in range(first, first + cnt):
                    t = order[k]
                    seen[t] += 1
                    p = verts[tris[t]]
                    assert np.all(p >= lo) and np.all(p <= hi), "triangle outside its leaf box"
    return seen, visited


@pytest.mark.parametrize("width", [4, 8])
def test_bvh_host_invariants(width):
    """Every triangle in exactly one leaf; triangles inside their leaf box;
    child boxes inside parent boxes; every node reachable from the root."""
    m = W.procedural_satellite(dish_segments=32, dish_rings=12, n_boxes=20)
    nodes, order, nn = srp.srp_build_bvh_host(m.verts, m.tris, width)
    assert sorted(order.tolist()) == list(range(m.T))
    seen, visited = _walk(nodes, width, m.T, m.verts.astype(np.float64), m.tris, order)
    assert np.all(seen == 1)
    assert visited == nn


@pytest.mark.parametrize("T", [0, 1, 3, 5])
def test_bvh_host_tiny(T):
    m = W.icosphere(1)
    tris = m.tris[:T]
    nodes, order, nn = srp.srp_build_bvh_host(m.verts, tris, 4)
    assert nn >= 1
    if T:
        seen, _ = _walk(nodes, 4, T, m.verts.astype(np.float64), tris, order)
        assert np.all(seen == 1)


def test_bvh_host_rejects_bad_input():
    m = W.box_wing()
    with pytest.raises(srp.SRPError) as e:
        srp.srp_build_bvh_host(m.verts, m.tris, 6)
    assert e.value.code == srp.SRP_EINVAL
    bad = m.tris.copy(); bad[0, 0] = 999
    with pytest.raises(srp.SRPError):
        srp.srp_build_bvh_host(m.verts, bad, 4)
    v = m.verts.copy(); v[0, 0] = np.nan
    with pytest.raises(srp.SRPError):
        srp.srp_build_bvh_host(v, m.tris, 4)


def test_opts_struct_matches_header():
    """ctypes mirror of srp_trace_opts has the C layout (defaults round-trip)."""
    o = srp.make_opts()
    assert o.rays_x == 1024 and o.max_bounces == 1 and o.pressure == 1.0 and o.mem == srp.SRP_MEM_DEVICE
    assert C.sizeof(srp.TraceOpts) == 88 and srp.TraceOpts.pressure.offset == 24


def test_binding_rejects_undersized_or_mistyped_buffers():
    """Host-memory calls whose arrays are smaller than the sizes the call
    implies, or of the wrong element type, are rejected by the binding with
    SRP_EINVAL before the library is entered (the library would read or
    write past their ends).  The stand-in context and BVH are never used."""
    import types
    ctx = types.SimpleNamespace(device=0, handle=None)
    bvh = types.SimpleNamespace(handle=None, info=lambda: {"n_tris": 16})
    m, rho, sun, com = W.config1()

    def rejected(fn, *a, **kw):
        with pytest.raises(srp.SRPError) as e:
            fn(*a, **kw)
        assert e.value.code == srp.SRP_EINVAL, str(e.value)
        return str(e.value)

    # two designs, one design's reflectances and COM
    assert "rho" in rejected(srp.srp_force, ctx, [bvh, bvh], rho[None], sun, np.zeros((2, 3)))
    assert "com" in rejected(srp.srp_force, ctx, [bvh, bvh], np.stack([rho, rho]), sun, com[None])
    # outputs too small, of the wrong type or not contiguous
    assert "out_ft" in rejected(srp.srp_force, ctx, [bvh], rho[None], sun, com[None], out_ft=np.zeros((1, 0, 6)))
    assert "out_ft" in rejected(srp.srp_force, ctx, [bvh], rho[None], sun, com[None],
                                out_ft=np.zeros((1, 1, 6), np.float32))
    assert "out_sigma" in rejected(srp.srp_force, ctx, [bvh], rho[None], sun, com[None],
                                   out_sigma=np.zeros((1, 1, 6))[:, :, ::2])
    assert "out_samples" in rejected(srp.srp_force_area, ctx, [bvh], rho[None], sun, com[None], 10.0,
                                     out_samples=np.zeros(1, np.int32))
    assert "emit" in rejected(srp.srp_force_thermal, ctx, [bvh], rho[None], np.ones((0, 64), np.float32),
                              com[None], 10.0)
    assert "upstream" in rejected(srp.srp_force_grad, ctx, bvh, rho, W.fibonacci_directions(3), com,
                                  np.ones((2, 6)))
    assert "tri_hinge" in rejected(srp.srp_force_grad, ctx, bvh, rho, sun, com, np.ones((1, 6)),
                                   tri_hinge=np.zeros(4, np.int32), hinge_axes=m.hinges)
    assert "vhinge" in rejected(srp.srp_design_instantiate, m.verts, m.vhinge[:3], m.hinges, [0.1, 0.2])
    assert "angles" in rejected(srp.srp_design_instantiate, m.verts, m.vhinge, m.hinges, [0.1])
    o = srp.orbit_opts(n_theta=2)
    assert "n_theta" in rejected(srp.srp_integrate, ctx, o, np.zeros(13), np.zeros(3))


def test_plain_c_caller(tmp_path):
    """The ABI as a C program sees it: tests/c_abi_host.c includes
    include/srp.h, links libsrp.so and calls the host-only entry points."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    lib = srp._build.build()
    libdir = os.path.dirname(lib)
    exe = str(tmp_path / "c_abi_host")
    r = subprocess.run([gcc, "-std=c11", "-O1", "-Wall", "-I", os.path.join(ROOT, "include"),
                        os.path.join(ROOT, "tests", "c_abi_host.c"), "-L", libdir, "-lsrp", f"-Wl,-rpath,{libdir}",
                        "-lm", "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and "c-abi ok" in r.stdout, r.stdout + r.stderr
