"""Python binding of libsrp (include/srp.h): argument marshalling only.

Every step of the computation runs in the library's CUDA kernels; this module
converts numpy arrays / torch tensors to pointers, checks shapes and dtypes,
and raises on a non-zero status.  If the library cannot be loaded it raises:
there is no CPU fallback.

Names follow the C ABI: srp_ctx_create, srp_build_bvh, srp_force, ...
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import _build

__all__ = ["SRPError", "load", "srp_ctx_create", "srp_ctx_destroy", "srp_sync", "srp_build_bvh",
           "srp_bvh_destroy", "srp_bvh_get_info", "srp_force", "srp_design_instantiate", "TraceOpts",
           "srp_build_bvh_host", "srp_trace_rays", "srp_bvh_set_nodes", "srp_bvh_refit", "srp_force_noalloc", "srp_force_area", "srp_force_thermal", "srp_trace_samples", "srp_force_grad", "SRPForce", "MLP",
           "mlp_param_count", "srp_integrate", "orbit_opts", "OrbitOpts", "ForceGraph",
           "Context", "SRP_MEM_HOST", "SRP_MEM_DEVICE"]

SRP_OK, SRP_EINVAL, SRP_ENOMEM, SRP_ECUDA, SRP_EDEVICE_LIMIT, SRP_ETIMEOUT, SRP_EUNSUPPORTED = range(7)
SRP_MEM_HOST, SRP_MEM_DEVICE = 0, 1
_STATUS = {1: "SRP_EINVAL", 2: "SRP_ENOMEM", 3: "SRP_ECUDA", 4: "SRP_EDEVICE_LIMIT",
           5: "SRP_ETIMEOUT", 6: "SRP_EUNSUPPORTED"}


class SRPError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


class TraceOpts(C.Structure):
    _fields_ = [("rays_x", C.c_int32), ("rays_y", C.c_int32), ("max_bounces", C.c_int32),
                ("jitter", C.c_int32), ("seed", C.c_uint64), ("pressure", C.c_double),
                ("ray_offset", C.c_int64), ("ray_stride", C.c_int64), ("ray_count", C.c_int64),
                ("sun_base", C.c_int32), ("design_base", C.c_int32), ("mem", C.c_int32),
                ("sun_per_design", C.c_int32), ("block_threads", C.c_int32),
                ("chunks_per_item", C.c_int32), ("kernel_variant", C.c_int32), ("reserved", C.c_int32)]


class BVHInfo(C.Structure):
    _fields_ = [("width", C.c_int32), ("n_nodes", C.c_int32), ("n_leaves", C.c_int32),
                ("depth", C.c_int32), ("n_tris", C.c_int32), ("device_bytes", C.c_int64),
                ("build_ms", C.c_double), ("center", C.c_double * 3), ("radius", C.c_double)]


_lib = None
_P = C.c_void_p


_load_lock = threading.Lock()


def load(build_if_needed: bool = True):
    """Load libsrp.so (building it with nvcc first if it is missing/stale).
    Thread-safe: concurrent first calls build and load once."""
    global _lib
    if _lib is not None:
        return _lib
    with _load_lock:
        if _lib is not None:
            return _lib
        return _load_locked(build_if_needed)


def _load_locked(build_if_needed: bool):
    global _lib
    path = _build.build() if build_if_needed else _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libsrp.so not found at {path}: run __graft_entry__.build()")
    lib = C.CDLL(path)
    i32, i64 = C.c_int, C.c_int64
    lib.srp_last_error.restype = C.c_char_p
    lib.srp_trace_opts_default.argtypes = [C.POINTER(TraceOpts)]
    lib.srp_ctx_create.argtypes = [C.POINTER(_P), i32, _P]
    lib.srp_ctx_destroy.argtypes = [_P]
    lib.srp_sync.argtypes = [_P]
    lib.srp_design_instantiate.argtypes = [_P, i32, _P, _P, _P, i32, _P]
    lib.srp_build_bvh.argtypes = [_P, _P, i32, _P, _P, i32, i32, C.POINTER(_P)]
    lib.srp_bvh_destroy.argtypes = [_P]
    lib.srp_bvh_get_info.argtypes = [_P, C.POINTER(BVHInfo)]
    lib.srp_force.argtypes = [_P, _P, i32, _P, i32, _P, i32, _P, C.POINTER(TraceOpts), _P, _P]
    lib.srp_force_area.argtypes = [_P, _P, i32, _P, i32, _P, i32, _P, C.c_float, C.POINTER(TraceOpts), _P, _P, _P]
    lib.srp_trace_samples.argtypes = [_P, _P, i32, _P, _P, i32, _P, _P, i32, _P, _P, i32, _P, _P, i64, _P, C.c_double,
                                      C.POINTER(TraceOpts), _P, _P]
    lib.srp_force_thermal.argtypes = [_P, _P, i32, _P, i32, _P, _P, C.c_float, C.POINTER(TraceOpts), _P, _P, _P]
    lib.srp_collect_stats.argtypes = [_P, i32, _P]
    lib.srp_probe_read_bandwidth.argtypes = [_P, i64, i32, i32, C.POINTER(C.c_double)]
    lib.srp_bvh_set_nodes.argtypes = [_P, _P, _P, i64]
    lib.srp_bvh_refit.argtypes = [_P, _P, _P, i32, _P, i32]
    lib.srp_force_grad.argtypes = [_P, _P, _P, i32, _P, i32, _P, _P, _P, i32, C.POINTER(TraceOpts), _P, _P, _P]
    lib.srp_mlp_param_count.argtypes = [C.POINTER(C.c_int64)]
    lib.srp_mlp_create.argtypes = [_P, _P, C.c_uint64, C.POINTER(_P)]
    lib.srp_mlp_destroy.argtypes = [_P]
    lib.srp_mlp_set_params.argtypes = [_P, _P, _P]
    lib.srp_mlp_get_params.argtypes = [_P, _P, _P]
    lib.srp_mlp_infer.argtypes = [_P, _P, _P, i64, _P, i32]
    lib.srp_orbit_opts_default.argtypes = [_P]
    lib.srp_force_graph_create.argtypes = [_P, _P, i32, _P, i32, _P, i32, _P, C.POINTER(TraceOpts), _P, _P,
                                           C.POINTER(_P)]
    lib.srp_graph_launch.argtypes = [_P]
    lib.srp_graph_destroy.argtypes = [_P]
    lib.srp_integrate.argtypes = [_P, _P, _P, i32, _P, _P, _P, _P, _P, _P, _P, i32]
    lib.srp_mlp_train_step.argtypes = [_P, _P, _P, _P, i64, C.c_float, _P, _P, i32]
    lib.srp_mlp_grad_input.argtypes = [_P, _P, _P, _P, i64, _P, i32]
    lib.srp_mlp_train_epoch.argtypes = [_P, _P, _P, _P, i64, _P, i64, i64, _P]
    lib.srp_mlp_save.argtypes = [_P, _P, C.c_char_p]
    lib.srp_mlp_load.argtypes = [_P, _P, C.c_char_p]
    lib.srp_mlp_save_state.argtypes = [_P, _P, C.c_char_p]
    lib.srp_mlp_load_state.argtypes = [_P, _P, C.c_char_p]
    lib.srp_force_noalloc.argtypes = [_P, i32, _P, i32, _P, i32, _P, C.POINTER(TraceOpts), _P, _P, _P, _P]
    lib.srp_build_bvh_host.argtypes = [_P, i32, _P, i32, i32, _P, C.POINTER(C.c_int64), _P, C.POINTER(C.c_int32)]
    lib.srp_trace_rays.argtypes = [_P, _P, _P, i32, _P, _P, _P, i64, i32, i32, C.POINTER(TraceOpts), _P, _P]
    _lib = lib
    return lib


def _check(rc):
    if rc != SRP_OK:
        raise SRPError(rc, _lib.srp_last_error().decode(errors="replace"))


def _np(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _ptr(a):
    """Pointer of a numpy array or a torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(_P)
    return _P(a.data_ptr())


def _need(name, a, n, dtype, device, dev_index=None):
    """Check that `a` can back the n elements of `dtype` the library reads
    or writes through its pointer: a C-contiguous numpy array in host mode,
    a contiguous CUDA tensor (on device `dev_index` when given) in device
    mode, with at least n elements.  A smaller or mistyped buffer would be
    an out-of-bounds access inside the library, so it is rejected here with
    SRP_EINVAL."""
    if a is None:
        if n > 0:
            raise SRPError(SRP_EINVAL, f"{name} is missing ({n} elements needed)")
        return
    dt = np.dtype(dtype)
    if device:
        import torch
        tdt = getattr(torch, dt.name)
        if not (isinstance(a, torch.Tensor) and a.is_cuda and a.dtype == tdt and a.is_contiguous()):
            raise SRPError(SRP_EINVAL, f"{name} must be a contiguous CUDA {tdt} tensor")
        if dev_index is not None and a.device.index != dev_index:
            raise SRPError(SRP_EINVAL, f"{name} is on cuda:{a.device.index}, the context on cuda:{dev_index}")
        size = a.numel()
    else:
        if not (isinstance(a, np.ndarray) and a.dtype == dt and a.flags.c_contiguous):
            raise SRPError(SRP_EINVAL, f"{name} must be a C-contiguous numpy {dt.name} array")
        size = a.size
    if size < n:
        raise SRPError(SRP_EINVAL, f"{name} holds {size} elements; the call needs {n}")


def _need_items(ctx, device, D, S, G, rho, sun_dir, com, per_design_sun, outs):
    """Sizes of the (design, sun) calls: rho [D][G][2] float32, sun_dir
    [S][3] (or [D][S][3]) float64, com [D][3] float64, and each output
    (name, array, elements per item, dtype)."""
    di = ctx.device if ctx is not None else None
    _need("rho", rho, D * G * 2, np.float32, device, di)
    _need("sun_dir", sun_dir, (D if per_design_sun else 1) * S * 3, np.float64, device, di)
    _need("com", com, D * 3, np.float64, device, di)
    for name, a, per, dt in outs:
        if a is not None:
            _need(name, a, per, dt, device, di)


# ----------------------------------------------------------------- context
class Context:
    """An srp_ctx bound to one device and one CUDA stream (a torch stream or
    a raw cudaStream_t integer; default: torch's current stream)."""

    def __init__(self, device: int = 0, stream=None):
        lib = load()
        if stream is None:
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream
        elif hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        self.device = device
        self.stream = int(stream)
        h = _P()
        _check(lib.srp_ctx_create(C.byref(h), device, _P(self.stream)))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            _lib.srp_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def srp_ctx_create(device: int = 0, stream=None) -> Context:
    return Context(device, stream)


def srp_ctx_destroy(ctx: Context):
    ctx.close()


def srp_sync(ctx: Context):
    _check(load().srp_sync(ctx.handle))


class BVH:
    def __init__(self, handle):
        self.handle = handle

    def close(self):
        if getattr(self, "handle", None):
            _lib.srp_bvh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        return srp_bvh_get_info(self)


def srp_collect_stats(ctx: Context, enable: bool = True):
    """Counters since the last call: (node visits, triangle tests, segments)."""
    out = np.zeros(3, np.uint64)
    _check(load().srp_collect_stats(ctx.handle, 1 if enable else 0, _ptr(out)))
    return int(out[0]), int(out[1]), int(out[2])


def srp_probe_read_bandwidth(ctx: Context, nbytes: int, passes: int = 64, reps: int = 10) -> float:
    """Best read rate (GB/s) over a device buffer of nbytes, 16-byte loads
    cached in L2 only, from every SM (the roofline's L2 or HBM ceiling)."""
    out = C.c_double(0.0)
    _check(load().srp_probe_read_bandwidth(ctx.handle, int(nbytes), int(passes), int(reps), C.byref(out)))
    return out.value


def srp_design_instantiate(verts, vhinge, hinges, angles):
    lib = load()
    v = _np(verts, np.float32)
    out = np.empty_like(v)
    vh = _np(vhinge, np.int32)
    hg = _np(hinges, np.float64).reshape(-1, 6)
    an = _np(angles, np.float64).reshape(-1)
    if hg.shape[0] > 0 and (vh.size < v.shape[0] or an.size < hg.shape[0]):
        raise SRPError(SRP_EINVAL, "vhinge needs one entry per vertex and angles one per hinge")
    _check(lib.srp_design_instantiate(_ptr(v), v.shape[0], _ptr(vh), _ptr(hg), _ptr(an), hg.shape[0], _ptr(out)))
    return out


def srp_build_bvh(ctx: Context, verts, tris, group, width: int = 4) -> BVH:
    lib = load()
    v = _np(verts, np.float32).reshape(-1, 3)
    t = _np(tris, np.int32).reshape(-1, 3)
    g = _np(group, np.int32).reshape(-1)
    if g.shape[0] != t.shape[0]:
        raise ValueError("group must have one entry per triangle")
    h = _P()
    _check(lib.srp_build_bvh(ctx.handle, _ptr(v), v.shape[0], _ptr(t), _ptr(g), t.shape[0], width, C.byref(h)))
    return BVH(h)


def srp_bvh_destroy(b: BVH):
    b.close()


def srp_bvh_get_info(b: BVH) -> dict:
    info = BVHInfo()
    _check(load().srp_bvh_get_info(b.handle, C.byref(info)))
    return {"width": info.width, "n_nodes": info.n_nodes, "n_leaves": info.n_leaves, "depth": info.depth,
            "n_tris": info.n_tris, "device_bytes": info.device_bytes, "build_ms": info.build_ms,
            "center": tuple(info.center), "radius": info.radius}


def srp_bvh_set_nodes(ctx: Context, b: BVH, node_data):
    nd = _np(node_data, np.float32).reshape(-1)
    _check(load().srp_bvh_set_nodes(ctx.handle, b.handle, _ptr(nd), nd.shape[0]))


def srp_bvh_refit(ctx: Context, b: BVH, verts, tris):
    """Refit b to moved vertices of the mesh it was built from (same tris):
    the topology is kept, triangle records and node bounds are recomputed on
    the device, and the grid centre / radius as srp_build_bvh computes them."""
    v = _np(verts, np.float32).reshape(-1, 3)
    t = _np(tris, np.int32).reshape(-1, 3)
    _check(load().srp_bvh_refit(ctx.handle, b.handle, _ptr(v), v.shape[0], _ptr(t), t.shape[0]))


def srp_build_bvh_host(verts, tris, width: int = 4):
    """Host-only wide BVH: (node_data float32 [n_node_floats], tri_order int32 [T], n_nodes)."""
    lib = load()
    v = _np(verts, np.float32).reshape(-1, 3)
    t = _np(tris, np.int32).reshape(-1, 3)
    nf = C.c_int64(0); nn = C.c_int32(0)
    _check(lib.srp_build_bvh_host(_ptr(v), v.shape[0], _ptr(t), t.shape[0], width, None, C.byref(nf), None,
                                  C.byref(nn)))
    nodes = np.zeros(nf.value, np.float32)
    order = np.zeros(t.shape[0], np.int32)
    _check(lib.srp_build_bvh_host(_ptr(v), v.shape[0], _ptr(t), t.shape[0], width, _ptr(nodes), C.byref(nf),
                                  _ptr(order), C.byref(nn)))
    return nodes, order, nn.value


def make_opts(*, rays_x=1024, rays_y=None, max_bounces=1, jitter=1, seed=0, pressure=1.0,
              ray_offset=0, ray_stride=1, ray_count=0, sun_base=0, design_base=0, mem=SRP_MEM_DEVICE,
              sun_per_design=0, block_threads=0, chunks_per_item=0, kernel_variant=0) -> TraceOpts:
    o = TraceOpts()
    load().srp_trace_opts_default(C.byref(o))
    o.rays_x = rays_x
    o.rays_y = rays_x if rays_y is None else rays_y
    o.max_bounces = max_bounces; o.jitter = jitter; o.seed = seed; o.pressure = pressure
    o.ray_offset = ray_offset; o.ray_stride = ray_stride; o.ray_count = ray_count
    o.sun_base = sun_base; o.design_base = design_base; o.mem = mem
    o.sun_per_design = sun_per_design; o.block_threads = block_threads; o.chunks_per_item = chunks_per_item
    o.kernel_variant = kernel_variant
    return o


def srp_force(ctx: Context, bvhs, rho, sun_dir, com, out_ft=None, out_sigma=None, **opts):
    """Force and torque [D,S,6] (plus sigma) of D designs x S sun directions.

    Device mode: rho (float32 [D,G,2]), sun_dir (float64 [S,3] or [D,S,3]),
    com (float64 [D,3]) and the outputs are torch CUDA tensors; the call is
    asynchronous on the context's stream.  Host mode: numpy arrays; the call
    returns when the results are in the output arrays."""
    lib = load()
    bvhs = list(bvhs)
    D = len(bvhs)
    arr = (_P * max(D, 1))(*[b.handle for b in bvhs])
    device = not isinstance(rho, np.ndarray)
    if device:
        import torch
        for name, x, dt in (("rho", rho, torch.float32), ("sun_dir", sun_dir, torch.float64),
                            ("com", com, torch.float64)):
            if not (x.is_cuda and x.dtype == dt and x.is_contiguous()):
                raise TypeError(f"{name} must be a contiguous CUDA {dt} tensor")
        S = sun_dir.shape[-2]
        G = rho.shape[-2]
        if out_ft is None:
            out_ft = torch.empty((D, S, 6), dtype=torch.float64, device=rho.device)
        opts.setdefault("mem", SRP_MEM_DEVICE)
    else:
        rho = _np(rho, np.float32)
        sun_dir = _np(sun_dir, np.float64)
        com = _np(com, np.float64)
        S = sun_dir.shape[-2]
        G = rho.shape[-2]
        if out_ft is None:
            out_ft = np.zeros((D, S, 6))
        if out_sigma is True:
            out_sigma = np.zeros((D, S, 6))
        opts["mem"] = SRP_MEM_HOST
    if out_sigma is True:
        import torch
        out_sigma = torch.empty((D, S, 6), dtype=torch.float64, device=rho.device)
    if opts.get("sun_per_design"):
        if tuple(sun_dir.shape[:2]) != (D, S):
            raise ValueError("sun_dir must be [D,S,3] with sun_per_design")
    _need_items(ctx, device, D, S, G, rho, sun_dir, com, opts.get("sun_per_design"),
                [("out_ft", out_ft, D * S * 6, np.float64), ("out_sigma", out_sigma, D * S * 6, np.float64)])
    o = make_opts(**opts)
    _check(lib.srp_force(ctx.handle, arr, D, _ptr(rho), G, _ptr(sun_dir), S, _ptr(com), C.byref(o),
                         _ptr(out_ft), _ptr(out_sigma) if out_sigma is not None else None))
    return (out_ft, out_sigma) if out_sigma is not None else out_ft


def srp_force_area(ctx: Context, bvhs, rho, sun_dir, com, density, out_ft=None, out_sigma=None, out_samples=None,
                   **opts):
    """The paper's no-bounce estimator (surface samples + next-event shadow
    rays) of (F, tau) [D,S,6]; `density` is samples per unit area.  Same
    array conventions as srp_force; out_samples=True also returns the
    samples per design [D] (int64)."""
    lib = load()
    bvhs = list(bvhs)
    D = len(bvhs)
    arr = (_P * max(D, 1))(*[b.handle for b in bvhs])
    device = not isinstance(rho, np.ndarray)
    if device:
        import torch
        for name, x, dt in (("rho", rho, torch.float32), ("sun_dir", sun_dir, torch.float64),
                            ("com", com, torch.float64)):
            if not (x.is_cuda and x.dtype == dt and x.is_contiguous()):
                raise TypeError(f"{name} must be a contiguous CUDA {dt} tensor")
        S = sun_dir.shape[-2]
        G = rho.shape[-2]
        if out_ft is None:
            out_ft = torch.empty((D, S, 6), dtype=torch.float64, device=rho.device)
        if out_sigma is True:
            out_sigma = torch.empty((D, S, 6), dtype=torch.float64, device=rho.device)
        if out_samples is True:
            out_samples = torch.empty((D,), dtype=torch.int64, device=rho.device)
        opts.setdefault("mem", SRP_MEM_DEVICE)
    else:
        rho = _np(rho, np.float32)
        sun_dir = _np(sun_dir, np.float64)
        com = _np(com, np.float64)
        S = sun_dir.shape[-2]
        G = rho.shape[-2]
        if out_ft is None:
            out_ft = np.zeros((D, S, 6))
        if out_sigma is True:
            out_sigma = np.zeros((D, S, 6))
        if out_samples is True:
            out_samples = np.zeros(D, np.int64)
        opts["mem"] = SRP_MEM_HOST
    if opts.get("sun_per_design"):
        if tuple(sun_dir.shape[:2]) != (D, S):
            raise ValueError("sun_dir must be [D,S,3] with sun_per_design")
    _need_items(ctx, device, D, S, G, rho, sun_dir, com, opts.get("sun_per_design"),
                [("out_ft", out_ft, D * S * 6, np.float64), ("out_sigma", out_sigma, D * S * 6, np.float64),
                 ("out_samples", out_samples, D, np.int64)])
    o = make_opts(**opts)
    _check(lib.srp_force_area(ctx.handle, arr, D, _ptr(rho), G, _ptr(sun_dir), S, _ptr(com), float(density), C.byref(o),
                              _ptr(out_ft), _ptr(out_sigma) if out_sigma is not None else None,
                              _ptr(out_samples) if out_samples is not None else None))
    res = [out_ft]
    if out_sigma is not None:
        res.append(out_sigma)
    if out_samples is not None:
        res.append(out_samples)
    return res[0] if len(res) == 1 else tuple(res)


def srp_force_thermal(ctx: Context, bvhs, rho, emit, com, density, out_ft=None, out_sigma=None, out_samples=None,
                      **opts):
    """Force and torque [D,6] of local Lambertian thermal emitters: emit
    [D,G] flux per unit area per group (times opts pressure, e.g. 1/c for
    W/m^2).  Array conventions as srp_force_area."""
    lib = load()
    bvhs = list(bvhs)
    D = len(bvhs)
    arr = (_P * max(D, 1))(*[b.handle for b in bvhs])
    device = not isinstance(rho, np.ndarray)
    if device:
        import torch
        for name, x, dt in (("rho", rho, torch.float32), ("emit", emit, torch.float32), ("com", com, torch.float64)):
            if not (x.is_cuda and x.dtype == dt and x.is_contiguous()):
                raise TypeError(f"{name} must be a contiguous CUDA {dt} tensor")
        G = rho.shape[-2]
        if out_ft is None:
            out_ft = torch.empty((D, 6), dtype=torch.float64, device=rho.device)
        if out_sigma is True:
            out_sigma = torch.empty((D, 6), dtype=torch.float64, device=rho.device)
        if out_samples is True:
            out_samples = torch.empty((D,), dtype=torch.int64, device=rho.device)
        opts.setdefault("mem", SRP_MEM_DEVICE)
    else:
        rho = _np(rho, np.float32)
        emit = _np(emit, np.float32)
        com = _np(com, np.float64)
        G = rho.shape[-2]
        if emit.shape[-1] != G:
            raise ValueError("emit must be [D,G] with the G of rho")
        if out_ft is None:
            out_ft = np.zeros((D, 6))
        if out_sigma is True:
            out_sigma = np.zeros((D, 6))
        if out_samples is True:
            out_samples = np.zeros(D, np.int64)
        opts["mem"] = SRP_MEM_HOST
    di = ctx.device
    _need("rho", rho, D * G * 2, np.float32, device, di)
    _need("emit", emit, D * G, np.float32, device, di)
    _need("com", com, D * 3, np.float64, device, di)
    for name, a, n, dt in (("out_ft", out_ft, D * 6, np.float64), ("out_sigma", out_sigma, D * 6, np.float64),
                           ("out_samples", out_samples, D, np.int64)):
        if a is not None:
            _need(name, a, n, dt, device, di)
    o = make_opts(**opts)
    _check(lib.srp_force_thermal(ctx.handle, arr, D, _ptr(rho), G, _ptr(emit), _ptr(com), float(density), C.byref(o),
                                 _ptr(out_ft), _ptr(out_sigma) if out_sigma is not None else None,
                                 _ptr(out_samples) if out_samples is not None else None))
    res = [out_ft]
    if out_sigma is not None:
        res.append(out_sigma)
    if out_samples is not None:
        res.append(out_samples)
    return res[0] if len(res) == 1 else tuple(res)


def srp_trace_samples(ctx: Context, mesh_verts, vhinge, hinges, tris, group, angles, rho, sun, com, center, radius,
                      out_y=None, want_hits=False, **opts):
    """Per-sample designs: one jittered ray per sample over its own
    instantiated mesh (brute force).  The mesh is numpy (host); angles,
    rho [N,G,2], sun [N,3], com [N,3] numpy (host mode) or CUDA tensors
    (device mode).  Returns y [N,6] (and hits [N,K])."""
    lib = load()
    v = _np(mesh_verts, np.float32).reshape(-1, 3)
    vh = _np(vhinge, np.int32).reshape(-1)
    hg = _np(hinges, np.float64).reshape(-1, 6)
    t = _np(tris, np.int32).reshape(-1, 3)
    g = _np(group, np.int32).reshape(-1)
    H = hg.shape[0]
    K = opts.get("max_bounces", 1)
    ce = _np(center, np.float64).reshape(3)
    if isinstance(sun, np.ndarray):
        sun = _np(sun, np.float64).reshape(-1, 3)
        N = sun.shape[0]
        angles = _np(angles, np.float64).reshape(N, max(H, 1) if H else 0) if H else np.zeros((N, 0))
        rho = _np(rho, np.float32)
        com = _np(com, np.float64).reshape(N, 3)
        y = np.zeros((N, 6)) if out_y is None else out_y
        hits = np.zeros((N, K), np.int32) if want_hits else None
        opts["mem"] = SRP_MEM_HOST
    else:
        import torch
        N = sun.shape[0]
        y = torch.empty((N, 6), dtype=torch.float64, device=sun.device) if out_y is None else out_y
        hits = torch.empty((N, K), dtype=torch.int32, device=sun.device) if want_hits else None
        opts.setdefault("mem", SRP_MEM_DEVICE)
    G = rho.shape[-2]
    dm = opts["mem"] == SRP_MEM_DEVICE
    di = ctx.device
    if H:
        _need("angles", angles, N * H, np.float64, dm, di)
    _need("rho", rho, N * G * 2, np.float32, dm, di)
    _need("sun", sun, N * 3, np.float64, dm, di)
    _need("com", com, N * 3, np.float64, dm, di)
    _need("out_y", y, N * 6, np.float64, dm, di)
    if hits is not None:
        _need("hits", hits, N * K, np.int32, dm, di)
    if H and vh.shape[0] < v.shape[0]:
        raise SRPError(SRP_EINVAL, "vhinge needs one entry per vertex")
    if g.shape[0] < t.shape[0]:
        raise SRPError(SRP_EINVAL, "group needs one entry per triangle")
    o = make_opts(**opts)
    _check(lib.srp_trace_samples(ctx.handle, _ptr(v), v.shape[0], _ptr(vh), _ptr(hg), H, _ptr(t), _ptr(g), t.shape[0],
                                 _ptr(angles), _ptr(rho), G, _ptr(sun), _ptr(com), N, _ptr(ce), float(radius),
                                 C.byref(o), _ptr(y), _ptr(hits) if hits is not None else None))
    return (y, hits) if want_hits else y


def srp_trace_rays(ctx: Context, bvh: BVH, rho, sun_dir, com, ray_idx, sun_index=0, design_index=0, **opts):
    """Per-ray samples of one (design, sun): (y [n,6] float64, hits [n,K] int32).
    numpy inputs -> host mode (synchronous); torch CUDA tensors -> device mode."""
    lib = load()
    K = opts.get("max_bounces", 1)
    if isinstance(rho, np.ndarray) or isinstance(ray_idx, np.ndarray):
        rho = _np(rho, np.float32).reshape(-1, 2)
        sun_dir = _np(sun_dir, np.float64).reshape(3)
        com = _np(com, np.float64).reshape(3)
        ray_idx = _np(ray_idx, np.int64).reshape(-1)
        y = np.zeros((ray_idx.shape[0], 6)); h = np.zeros((ray_idx.shape[0], K), np.int32)
        opts["mem"] = SRP_MEM_HOST
    else:
        import torch
        y = torch.empty((ray_idx.shape[0], 6), dtype=torch.float64, device=rho.device)
        h = torch.empty((ray_idx.shape[0], K), dtype=torch.int32, device=rho.device)
        opts["mem"] = SRP_MEM_DEVICE
    dm = opts["mem"] == SRP_MEM_DEVICE
    _need("rho", rho, rho.shape[0] * 2, np.float32, dm, ctx.device)
    _need("sun_dir", sun_dir, 3, np.float64, dm, ctx.device)
    _need("com", com, 3, np.float64, dm, ctx.device)
    _need("ray_idx", ray_idx, ray_idx.shape[0], np.int64, dm, ctx.device)
    o = make_opts(**opts)
    _check(lib.srp_trace_rays(ctx.handle, bvh.handle, _ptr(rho), rho.shape[0], _ptr(sun_dir), _ptr(com),
                              _ptr(ray_idx), ray_idx.shape[0], sun_index, design_index, C.byref(o), _ptr(y), _ptr(h)))
    return y, h


def srp_force_noalloc(bvhs, rho, sun_dir, com, out_ft, out_sigma=None, status=None, stream=None, **opts):
    """srp_force for callers that cannot allocate device memory: every array
    (torch CUDA tensors: rho float32 [D,G,2], sun_dir float64 [S,3] or
    [D,S,3], com float64 [D,3], out_ft/out_sigma float64 [D,S,6], status
    int32 [1]) is supplied by the caller and the partial sums use a fixed
    8 MiB array inside the library; D*S <= 87,381.  Asynchronous on `stream`
    (default: torch's current stream) on the current device.  Overlapping
    calls race on the shared array; the first call per device should come
    before any stream capture."""
    lib = load()
    bvhs = list(bvhs)
    D = len(bvhs)
    arr = (_P * max(D, 1))(*[b.handle for b in bvhs])
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    elif hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    opts["mem"] = SRP_MEM_DEVICE
    S = sun_dir.shape[-2]
    _need_items(None, True, D, S, rho.shape[-2], rho, sun_dir, com, opts.get("sun_per_design"),
                [("out_ft", out_ft, D * S * 6, np.float64), ("out_sigma", out_sigma, D * S * 6, np.float64),
                 ("status", status, 1, np.int32)])
    o = make_opts(**opts)
    _check(lib.srp_force_noalloc(arr, D, _ptr(rho), rho.shape[-2], _ptr(sun_dir), sun_dir.shape[-2], _ptr(com),
                                 C.byref(o), _ptr(out_ft), _ptr(out_sigma), _ptr(status), _P(int(stream))))
    return out_ft


def srp_force_grad(ctx: Context, bvh: BVH, rho, sun_dir, com, upstream, tri_hinge=None, hinge_axes=None, **opts):
    """Gradient of L = sum_s upstream[s].(F_s, tau_s): (d_rho [G,2], d_hinge [H]).
    numpy inputs -> host mode (synchronous); torch CUDA tensors -> device
    mode (asynchronous; d_rho/d_hinge are new CUDA tensors)."""
    lib = load()
    H = 0 if hinge_axes is None else int(np.asarray(hinge_axes.shape[0] if hasattr(hinge_axes, "shape") else len(hinge_axes)))
    if isinstance(rho, np.ndarray):
        rho = _np(rho, np.float32).reshape(-1, 2)
        sun_dir = _np(sun_dir, np.float64).reshape(-1, 3)
        com = _np(com, np.float64).reshape(3)
        up = _np(upstream, np.float64).reshape(-1, 6)
        th = None if tri_hinge is None else _np(tri_hinge, np.int32)
        ha = None if hinge_axes is None else _np(hinge_axes, np.float64).reshape(-1, 6)
        d_rho = np.zeros((rho.shape[0], 2)); d_h = np.zeros(max(H, 1))
        opts["mem"] = SRP_MEM_HOST
    else:
        import torch
        up, th, ha = upstream, tri_hinge, hinge_axes
        d_rho = torch.empty((rho.shape[-2], 2), dtype=torch.float64, device=rho.device)
        d_h = torch.empty((max(H, 1),), dtype=torch.float64, device=rho.device)
        opts["mem"] = SRP_MEM_DEVICE
    dm = opts["mem"] == SRP_MEM_DEVICE
    G, S = rho.shape[-2], sun_dir.shape[-2]
    _need("rho", rho, G * 2, np.float32, dm, ctx.device)
    _need("sun_dir", sun_dir, S * 3, np.float64, dm, ctx.device)
    _need("com", com, 3, np.float64, dm, ctx.device)
    _need("upstream", up, S * 6, np.float64, dm, ctx.device)
    if H > 0:
        _need("tri_hinge", th, bvh.info()["n_tris"], np.int32, dm, ctx.device)
        _need("hinge_axes", ha, H * 6, np.float64, dm, ctx.device)
    o = make_opts(**opts)
    _check(lib.srp_force_grad(ctx.handle, bvh.handle, _ptr(rho), rho.shape[-2], _ptr(sun_dir), sun_dir.shape[-2],
                              _ptr(com), _ptr(th), _ptr(ha), H, C.byref(o), _ptr(up), _ptr(d_rho),
                              _ptr(d_h) if H > 0 else None))
    return d_rho, d_h[:H]


class SRPForce:
    """torch.autograd.Function over the tracer: (rho [G,2] float32, hinge
    angles [H] float64) -> (F, tau) [S,6] float64 for one hinged design.
    forward: srp_design_instantiate + srp_build_bvh + srp_force;
    backward: srp_force_grad with the incoming gradient as upstream weights.
    Use SRPForce.apply(ctx, design, rho, angles, sun_dir, com, opts_dict);
    `design` = dict(verts, tris, group, vhinge, hinges)."""

    @staticmethod
    def _fn():
        import torch

        class _F(torch.autograd.Function):
            @staticmethod
            def forward(fctx, ctx, design, rho, angles, sun_dir, com, opts):
                v = srp_design_instantiate(design["verts"], design["vhinge"], design["hinges"],
                                           angles.detach().cpu().numpy())
                bvh = srp_build_bvh(ctx, v, design["tris"], design["group"], opts.get("width", 4))
                o = {k: x for k, x in opts.items() if k != "width"}
                r = rho.detach().reshape(1, -1, 2).contiguous().to(torch.float32)
                sd = sun_dir.detach().contiguous().to(torch.float64)
                cm = com.detach().reshape(1, 3).contiguous().to(torch.float64)
                out = srp_force(ctx, [bvh], r, sd, cm, **o)[0]
                fctx.save_for_backward(rho, angles, sun_dir, com)
                fctx.bvh, fctx.srp_ctx, fctx.design, fctx.opts = bvh, ctx, design, o
                return out

            @staticmethod
            def backward(fctx, g):
                rho, angles, sun_dir, com = fctx.saved_tensors
                d = fctx.design
                H = len(d["hinges"])
                th = torch.from_numpy(np.asarray(d["vhinge"])[np.asarray(d["tris"])[:, 0]].astype(np.int32)).to(rho.device)
                ha = torch.from_numpy(np.asarray(d["hinges"], np.float64)).to(rho.device)
                o = dict(fctx.opts)
                use_h = H > 0
                dr, dh = srp_force_grad(fctx.srp_ctx, fctx.bvh, rho.detach().reshape(-1, 2).contiguous().float(),
                                        sun_dir.detach().contiguous().double(), com.detach().reshape(3).contiguous().double(),
                                        g.contiguous().double(), th if use_h else None, ha if use_h else None, **o)
                da = dh.to(angles.dtype) if use_h else None
                return None, None, dr.to(rho.dtype).reshape(rho.shape), da, None, None, None

        return _F

    @classmethod
    def apply(cls, *args):
        return cls._fn().apply(*args)


# ----------------------------------------------------------------- proxy MLP
def mlp_param_count() -> int:
    n = C.c_int64(0)
    _check(load().srp_mlp_param_count(C.byref(n)))
    return n.value


class MLP:
    """The neural proxy (srp_mlp): 19 -> 4x256 SiLU -> 6 on the tensor cores.
    Parameters are the flat FP32 vector (W_l row-major [out][in], then b_l,
    for l = 0..4)."""

    def __init__(self, ctx: Context, params=None, seed: int = 0):
        lib = load()
        self.ctx = ctx
        h = _P()
        p = None if params is None else _np(params, np.float32)
        if p is not None:
            _need("params", p, mlp_param_count(), np.float32, False)
        _check(lib.srp_mlp_create(ctx.handle, _ptr(p), seed, C.byref(h)))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            _lib.srp_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> np.ndarray:
        out = np.zeros(mlp_param_count(), np.float32)
        _check(load().srp_mlp_get_params(self.ctx.handle, self.handle, _ptr(out)))
        return out

    def set_params(self, p):
        p = _np(p, np.float32)
        _need("params", p, mlp_param_count(), np.float32, False)
        _check(load().srp_mlp_set_params(self.ctx.handle, self.handle, _ptr(p)))

    def infer(self, x, y=None):
        """y [B,6] = P(x [B,19]); numpy -> synchronous host call, torch CUDA
        float32 tensors -> asynchronous device call."""
        if isinstance(x, np.ndarray):
            x = _np(x, np.float32).reshape(-1, 19)
            y = np.zeros((x.shape[0], 6), np.float32) if y is None else y
            mem = SRP_MEM_HOST
        else:
            import torch
            y = torch.empty((x.shape[0], 6), dtype=torch.float32, device=x.device) if y is None else y
            mem = SRP_MEM_DEVICE
        dm, B = mem == SRP_MEM_DEVICE, x.shape[0]
        _need("x", x, B * 19, np.float32, dm, self.ctx.device)
        _need("y", y, B * 6, np.float32, dm, self.ctx.device)
        _check(load().srp_mlp_infer(self.ctx.handle, self.handle, _ptr(x), x.shape[0], _ptr(y), mem))
        return y

    def train_step(self, x, t, lr: float, want_loss: bool = True, want_grad: bool = False):
        """One Adam step on the L1 loss (lr = 0: gradient only).  Returns
        (loss or None, grad [P] or None); numpy -> host mode."""
        host = isinstance(x, np.ndarray)
        if host:
            x = _np(x, np.float32).reshape(-1, 19)
            t = _np(t, np.float32).reshape(-1, 6)
        B = x.shape[0]
        _need("x", x, B * 19, np.float32, not host, self.ctx.device)
        _need("t", t, B * 6, np.float32, not host, self.ctx.device)
        loss = np.zeros(1, np.float32) if want_loss else None
        grad = np.zeros(mlp_param_count(), np.float32) if want_grad else None
        _check(load().srp_mlp_train_step(self.ctx.handle, self.handle, _ptr(x), _ptr(t), x.shape[0], float(lr),
                                         _ptr(loss), _ptr(grad), SRP_MEM_HOST if host else SRP_MEM_DEVICE))
        return (float(loss[0]) if want_loss else None), grad

    def train_epoch(self, x, t, idx, batch: int, lr):
        """len(lr) Adam steps on batches gathered on the device: step s
        trains on rows idx[s*batch:(s+1)*batch] of x [n,19] and t [n,6]
        (CUDA float32 tensors) with learning rate lr[s]; idx is a CUDA int32
        tensor of len(lr)*batch row numbers.  Asynchronous (queued on the
        context's stream)."""
        lr = _np(lr, np.float32).reshape(-1)
        n_steps = lr.size
        n = x.shape[0]
        _need("x", x, n * 19, np.float32, True, self.ctx.device)
        _need("t", t, n * 6, np.float32, True, self.ctx.device)
        _need("idx", idx, n_steps * batch, np.int32, True, self.ctx.device)
        if t.shape[0] != n:
            raise ValueError("t must have the rows of x")
        _check(load().srp_mlp_train_epoch(self.ctx.handle, self.handle, _ptr(x), _ptr(t), n, _ptr(idx), int(batch),
                                          n_steps, lr.ctypes.data_as(_P)))

    def grad_input(self, x, wy, gx=None):
        """gx [B,19] = (dy/dx)^T wy for wy [B,6]; numpy -> host mode."""
        if isinstance(x, np.ndarray):
            x = _np(x, np.float32).reshape(-1, 19)
            wy = _np(wy, np.float32).reshape(-1, 6)
            gx = np.zeros((x.shape[0], 19), np.float32) if gx is None else gx
            mem = SRP_MEM_HOST
        else:
            import torch
            gx = torch.empty((x.shape[0], 19), dtype=torch.float32, device=x.device) if gx is None else gx
            mem = SRP_MEM_DEVICE
        if wy.shape[0] != x.shape[0]:
            raise ValueError("wy must have the batch of x")
        dm, B = mem == SRP_MEM_DEVICE, x.shape[0]
        _need("x", x, B * 19, np.float32, dm, self.ctx.device)
        _need("wy", wy, B * 6, np.float32, dm, self.ctx.device)
        _need("gx", gx, B * 19, np.float32, dm, self.ctx.device)
        _check(load().srp_mlp_grad_input(self.ctx.handle, self.handle, _ptr(x), _ptr(wy), x.shape[0], _ptr(gx), mem))
        return gx

    def save(self, path: str):
        _check(load().srp_mlp_save(self.ctx.handle, self.handle, os.fsencode(path)))

    def load_file(self, path: str):
        _check(load().srp_mlp_load(self.ctx.handle, self.handle, os.fsencode(path)))

    def save_state(self, path: str):
        """Checkpoint of training: parameters, Adam moments and step."""
        _check(load().srp_mlp_save_state(self.ctx.handle, self.handle, os.fsencode(path)))

    def load_state(self, path: str):
        """Resume training from a save_state file."""
        _check(load().srp_mlp_load_state(self.ctx.handle, self.handle, os.fsencode(path)))


# ----------------------------------------------------------------- orbits
SRP_FM_NONE, SRP_FM_CANNONBALL, SRP_FM_PROXY = 0, 1, 2


class OrbitOpts(C.Structure):
    _fields_ = [("mu", C.c_double), ("j2", C.c_double), ("re", C.c_double), ("mass", C.c_double),
                ("inertia", C.c_double * 3), ("pressure", C.c_double), ("sun", C.c_double * 3), ("dt", C.c_double),
                ("n_steps", C.c_int32), ("ckpt_every", C.c_int32), ("model", C.c_int32), ("n_theta", C.c_int32),
                ("in_scale", C.c_float * 19), ("in_offset", C.c_float * 19), ("out_mean", C.c_float * 6),
                ("out_std", C.c_float * 6), ("eclipse", C.c_int32), ("reserved0", C.c_int32), ("gm_sun", C.c_double),
                ("sun_dist", C.c_double), ("gm_moon", C.c_double), ("moon", C.c_double * 3)]


def orbit_opts(**kw) -> OrbitOpts:
    o = OrbitOpts()
    load().srp_orbit_opts_default(C.byref(o))
    for k, v in kw.items():
        if isinstance(v, (list, tuple, np.ndarray)):
            arr = getattr(o, k)
            for i, x in enumerate(v):
                arr[i] = x
        else:
            setattr(o, k, v)
    return o


def srp_integrate(ctx: Context, opts: OrbitOpts, z0, theta, proxy=None, want_traj=False, dL_dzN=None):
    """Integrate n trajectories (host numpy): returns dict(zN, traj, dL_dtheta, dL_dz0)."""
    lib = load()
    z0 = _np(z0, np.float64).reshape(-1, 13)
    n = z0.shape[0]
    th = _np(theta, np.float64).reshape(n, -1)
    if th.shape[1] != opts.n_theta:
        raise SRPError(SRP_EINVAL, f"theta has {th.shape[1]} values per trajectory, opts.n_theta = {opts.n_theta}")
    zN = np.zeros((n, 13))
    traj = np.zeros((n, opts.n_steps + 1, 13)) if want_traj else None
    lam = None if dL_dzN is None else _np(dL_dzN, np.float64).reshape(n, 13)
    dth = np.zeros((n, th.shape[1])) if lam is not None else None
    dz0 = np.zeros((n, 13)) if lam is not None else None
    _check(lib.srp_integrate(ctx.handle, C.byref(opts), proxy.handle if proxy is not None else None, n, _ptr(z0),
                             _ptr(th), _ptr(zN), _ptr(traj), _ptr(lam), _ptr(dth), _ptr(dz0), SRP_MEM_HOST))
    return {"zN": zN, "traj": traj, "dL_dtheta": dth, "dL_dz0": dz0}



class ForceGraph:
    """A CUDA graph of one srp_force evaluation on device tensors (captured
    once; launch() replays it on the context's stream)."""

    def __init__(self, ctx: Context, bvhs, rho, sun_dir, com, out_ft, out_sigma=None, **opts):
        lib = load()
        self.ctx = ctx
        self._keep = (list(bvhs), rho, sun_dir, com, out_ft, out_sigma)
        bv = list(bvhs)
        arr = (_P * max(len(bv), 1))(*[b.handle for b in bv])
        opts["mem"] = SRP_MEM_DEVICE
        D, S = len(bv), sun_dir.shape[-2]
        _need_items(ctx, True, D, S, rho.shape[-2], rho, sun_dir, com, opts.get("sun_per_design"),
                    [("out_ft", out_ft, D * S * 6, np.float64), ("out_sigma", out_sigma, D * S * 6, np.float64)])
        o = make_opts(**opts)
        h = _P()
        _check(lib.srp_force_graph_create(ctx.handle, arr, len(bv), _ptr(rho), rho.shape[-2], _ptr(sun_dir),
                                          sun_dir.shape[-2], _ptr(com), C.byref(o), _ptr(out_ft), _ptr(out_sigma),
                                          C.byref(h)))
        self.handle = h

    def launch(self):
        _check(load().srp_graph_launch(self.handle))

    def close(self):
        if getattr(self, "handle", None):
            _lib.srp_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
