// refit.cu -- srp_bvh_refit: the triangles of a design have moved (a new
// instantiation of the same mesh: hinge angles changed, Sec. 3.4's design
// loop), the BVH topology is kept and its contents are recomputed on the
// device: the leaf-order triangle records, then the child bounds of every
// node, deepest breadth-first level first.  A leaf slot's box is its
// triangles' AABB, an inner slot's the union of its child node's slots;
// each is padded outward as the host builder pads (relative 4e-7 plus an
// absolute 1e-6 of the scene scale), so the FP32 slab test stays
// conservative.  Closest hits do not depend on the boxes (ties go to the
// smaller original triangle index), so the forces equal those of a fresh
// build up to the grouping of sums; only the traversal cost changes as the
// topology ages.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <string>
#include <vector>

#include "srp_internal.h"

namespace srp {

constexpr int kRefitThreads = 256;

// triangle record k (leaf order): vertices of original triangle t = bits of
// .w of its first float4; the .w words (index, group) are kept
__global__ void refit_tri_kernel(float4* __restrict__ tri, int T, const float* __restrict__ verts,
                                 const int32_t* __restrict__ tris) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= T) return;
    float4* r = tri + 3 * (size_t)k;
    const int t = (int)__float_as_uint(r[0].w);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int v = __ldg(tris + 3 * (size_t)t + c);
        r[c] = make_float4(__ldg(verts + 3 * (size_t)v), __ldg(verts + 3 * (size_t)v + 1), __ldg(verts + 3 * (size_t)v + 2),
                           r[c].w);
    }
}

// One thread per (node, child slot) of nodes [n0, n1): the slot's box from
// its leaf triangles or from its child node's (already refitted) slots.
template <int W>
__global__ void refit_level_kernel(float* __restrict__ nodes, const float4* __restrict__ tri, int n0, int n1,
                                   float pad_abs) {
    constexpr int NF = W == 4 ? 32 : 64;   // floats per node
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n = n0 + e / W;
    const int c = (int)(e % W);
    if (n >= n1) return;
    float* nd = nodes + (size_t)n * NF;
    if (!(nd[c] <= nd[W + c])) return;   // empty slot (lo = +inf, hi = -inf)
    const int32_t code = reinterpret_cast<const int32_t*>(nd + 6 * W)[c];
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    if (code < 0) {
        const int first = (~code) >> 3, cnt = ((~code) & 7) + 1;
        for (int q = 0; q < cnt; ++q)
            for (int v = 0; v < 3; ++v) {
                const float4 p = tri[3 * (size_t)(first + q) + v];
                lo[0] = fminf(lo[0], p.x); hi[0] = fmaxf(hi[0], p.x);
                lo[1] = fminf(lo[1], p.y); hi[1] = fmaxf(hi[1], p.y);
                lo[2] = fminf(lo[2], p.z); hi[2] = fmaxf(hi[2], p.z);
            }
    } else {
        const float* ch = nodes + (size_t)code * NF;
        for (int k = 0; k < W; ++k) {
            if (!(ch[k] <= ch[W + k])) continue;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                lo[a] = fminf(lo[a], ch[(2 * a) * W + k]);
                hi[a] = fmaxf(hi[a], ch[(2 * a + 1) * W + k]);
            }
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        nd[(2 * a) * W + c] = lo[a] - (fabsf(lo[a]) * 4e-7f + pad_abs);
        nd[(2 * a + 1) * W + c] = hi[a] + (fabsf(hi[a]) * 4e-7f + pad_abs);
    }
}

// verts, tris: device arrays; levels: breadth-first level ranges.
cudaError_t launch_refit(srp_bvh* h, const float* verts, const int32_t* tris, float pad_abs, cudaStream_t st) {
    if (h->T > 0) {
        refit_tri_kernel<<<(h->T + kRefitThreads - 1) / kRefitThreads, kRefitThreads, 0, st>>>(
            (float4*)h->d_tri, h->T, verts, tris);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    for (int d = (int)h->level_start.size() - 2; d >= 0; --d) {
        const int n0 = h->level_start[d], n1 = h->level_start[d + 1];
        const int64_t work = (int64_t)(n1 - n0) * h->width;
        if (work <= 0) continue;
        const unsigned grid = (unsigned)((work + kRefitThreads - 1) / kRefitThreads);
        if (h->width == 8)
            refit_level_kernel<8><<<grid, kRefitThreads, 0, st>>>((float*)h->d_nodes, (const float4*)h->d_tri, n0, n1,
                                                                 pad_abs);
        else
            refit_level_kernel<4><<<grid, kRefitThreads, 0, st>>>((float*)h->d_nodes, (const float4*)h->d_tri, n0, n1,
                                                                 pad_abs);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace srp
