"""Autotuner of the tracer's launch parameters.

For a design (or set of designs) and a workload, time srp_force on a sample
of the real work for every candidate (BVH width 4 or 8, kernel register
budget 4, 5 or 6 resident blocks per SM, rays per work unit -- the chunk a
warp takes from the queue; 0 keeps the library's plan) and return the
fastest.  By default
the sample is whole grids for a subset of the sun directions, so each
candidate runs the launch path of the workload itself (full grids take the
pre-pass that skips the 32-pixel batches missing the scene, which changes
how the candidates rank); `sample_rays` instead takes every k-th ray of each
grid (same rays_x/rays_y, so the traversal work per ray is the workload's),
for grids too large to time whole.
"""
from __future__ import annotations

import itertools
import time


from . import srp_build_bvh, srp_force


def autotune(ctx, meshes, rho, sun_dir, com, *, rays_x, rays_y=None, max_bounces=1, sample_rays=None,
             sample_suns=16, widths=(4, 8), variants=(5, 6, 7), rays_per_unit=(0, 1024, 4096, 16384), repeats=2,
             **opts):
    """Returns (best dict(width, kernel_variant, chunks_per_item), table of
    timings in rays/s); chunks_per_item = 0 is the library's own plan.  `meshes` are workloads.Mesh-like (verts, tris, group);
    rho [D,G,2], sun_dir [S,3] (or [D,S,3] with sun_per_design=1), com [D,3]
    are torch CUDA tensors."""
    import torch
    ry = rays_x if rays_y is None else rays_y
    n = rays_x * ry
    if sample_rays is None or sample_rays >= n:
        count, sub = n, {}
    else:
        stride = max(1, n // sample_rays)
        count = min(sample_rays, (n + stride - 1) // stride)
        sub = dict(ray_offset=0, ray_stride=stride, ray_count=count)
    S = sun_dir.shape[-2]
    sel = torch.arange(0, S, max(1, S // sample_suns), device=sun_dir.device)[:sample_suns]
    sun_s = sun_dir.index_select(-2, sel).contiguous()
    table = []
    bvhs = {w: [srp_build_bvh(ctx, m.verts, m.tris, m.group, w) for m in meshes] for w in widths}
    for w, v, rpu in itertools.product(widths, variants, rays_per_unit):
        cpi = 0 if rpu <= 0 else max(1, -(-count // rpu))
        kw = dict(rays_x=rays_x, rays_y=ry, max_bounces=max_bounces, kernel_variant=v, chunks_per_item=cpi, **sub,
                  **opts)
        srp_force(ctx, bvhs[w], rho, sun_s, com, **kw)
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(repeats):
            t0 = time.perf_counter()
            srp_force(ctx, bvhs[w], rho, sun_s, com, **kw)
            torch.cuda.synchronize()
            best = min(best, time.perf_counter() - t0)
        rate = len(meshes) * sun_s.shape[-2] * count / best
        table.append({"width": w, "kernel_variant": v, "chunks_per_item": cpi, "rays_per_s": rate})
    for bl in bvhs.values():
        for b in bl:
            b.close()
    best = max(table, key=lambda r: r["rays_per_s"])
    return {"width": best["width"], "kernel_variant": best["kernel_variant"],
            "chunks_per_item": best["chunks_per_item"]}, table
