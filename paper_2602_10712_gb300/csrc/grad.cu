// grad.cu -- reverse-mode gradient of the SRP ray-grid estimate.
//
// For upstream weights g_s = dL/d(F_s, tau_s) (6 per sun direction) the
// kernel returns dL/d(rho_s, rho_d) per material group and dL/d(hinge
// angle) per hinge.  It replays exactly the forward's rays (same
// Philox counters, same traversal and shading helpers), so the gradient is
// that of the very estimate srp_force returns:
//  * reflectances: the branch choice has a fixed probability, so every path
//    is fixed and its deposits are polynomials in rho (exact derivative);
//    reverse sweep over the recorded hits, last hit first;
//  * hinges: each ray's primary surface element is carried rigidly by its
//    facet, so at K = 1 its contribution (w / cos0) cos(a) q.G(n(a)) is
//    differentiated in the rotation angle a (d n = axis x n, d x = axis x
//    (x - p)); at K > 1 the tangents run along the recorded path
//    (hinge_path_tangent).  The visibility of each ray is held fixed (the
//    estimate's boundary terms, where a shadow edge or silhouette moves,
//    are not included).
// Full grids of whole 32-pixel batches (8 x 4 blocks where the rows allow)
// trace only the batches that can meet
// the scene (the forward's span pre-pass; the rest contribute nothing).
// Accumulation: per-warp FP32 shared-memory sums over <= 512 rays, flushed
// into per-warp FP64 (an FP64 warp instruction is expensive on this GPU,
// so the flushes are kept rare), written as per-unit FP64 partials, summed
// by grad_reduce_kernel in a fixed order (one block per entry: strided
// thread sums, then a tree).
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "trace_common.cuh"

namespace srp {

struct GradParams {
    const double* up;       // [S][6] upstream weights
    const int32_t* thinge;  // [T] hinge id by ORIGINAL triangle index (-1: fixed), or NULL
    const double* hax;      // [H][6] hinge point (3), unit axis (3)
    int H;
    int ng;                 // 2G + H accumulated entries
    double* gpart;          // [units][ng]
};

constexpr int kMaxGradEntries = 2 * kMaxGroups + 8;

struct GradWarpSmem {
    float f[kMaxGradEntries];
    double d[kMaxGradEntries];
    float dirc[12];   // the unit's primary direction: 1/d and the shear rows
};

// d/da of one recorded path's L = sum_k q_k . dp_k for hinge `hh` (point
// ap, unit axis aa) in the fixed-visibility reading: the path keeps its
// facets, branch choices and random draws, facets on the hinge turn with
// it (d x = aa x (x - ap), d v = aa x v).  The primary hit point is carried
// by its facet (weight w c(a) / c0, as for K = 1); each later hit is the
// intersection of the outgoing ray with its facet's plane; the outgoing
// direction follows the turned normal (specular d + 2 c n; diffuse
// (n + u) / |n + u| with the sphere point u = l dout - n, l = 2 dout . n,
// held).  Forward-mode tangents along the path, base values as recorded.
__device__ float hinge_path_tangent(const DesignDev& dz, int hh, float3 ap, float3 aa, int m, int K, const int* hid,
                                    const int* fr, const int* br, const float3* xr, const float3* nr, const float3* dr,
                                    const float3* dout_r, const float* csr, const float* wr, const float* rsr,
                                    const float* rdr, float3 com, float3 gF, float3 gT) {
    const float3 zero = f3(0.0f, 0.0f, 0.0f);
    float3 dx = hid[0] == hh ? cross(aa, xr[0] - ap) : zero;
    float3 dn = hid[0] == hh ? cross(aa, nr[0]) : zero;
    float3 dd = zero;
    float dc = -dot(dn, dr[0]);
    float dw = wr[0] * dc / csr[0];
    float dL = 0.0f;
    for (int k = 0; k < m; ++k) {
        const float3 x = xr[k], n = nr[k], d = dr[k];
        const float c = csr[k], w = wr[k], rs = rsr[k], rd = rdr[k];
        const float3 q = gF + cross(gT, x - com), dq = cross(gT, dx);
        if (k + 1 == K) {
            const float cn = 2.0f * rs * c + (2.0f / 3.0f) * rd, dcn = 2.0f * rs * dc;
            const float3 G = (1.0f - rs) * d - cn * n;
            const float3 dG = (1.0f - rs) * dd - dcn * n - cn * dn;
            dL += w * dot(dq, G) + dot(q, dw * G + w * dG);
            break;
        }
        const float3 o = dout_r[k];
        float3 dO;
        float w2, dw2;
        if (br[k] == 0) {
            dO = dd + (2.0f * dc) * n + (2.0f * c) * dn;
            w2 = 2.0f * w * rs; dw2 = 2.0f * dw * rs;
        } else {
            const float l = 2.0f * dot(o, n);
            dO = (1.0f / l) * (dn - dot(o, dn) * o);
            w2 = 2.0f * w * rd; dw2 = 2.0f * dw * rd;
        }
        dL += dot(dq, w * d - w2 * o) + dot(q, dw * d + w * dd - dw2 * o - w2 * dO);
        if (k + 1 >= m) break;   // the outgoing ray left the craft
        const float4 v4 = __ldg(dz.tri + 3 * (size_t)fr[k + 1]);
        const float3 v0 = f3(v4.x, v4.y, v4.z), n1 = nr[k + 1];
        const float3 dv0 = hid[k + 1] == hh ? cross(aa, v0 - ap) : zero;
        const float3 dn1 = hid[k + 1] == hh ? cross(aa, n1) : zero;
        const float den = dot(n1, o);
        const float t = dot(n1, v0 - x) / den;
        const float dt = (dot(dn1, v0 - x) + dot(n1, dv0 - dx) - t * (dot(dn1, o) + dot(n1, dO))) / den;
        dx = dx + dt * o + t * dO;
        dn = dn1;
        dd = dO;
        dc = -(dot(dn, o) + dot(n1, dd));
        dw = dw2;
    }
    return dL;
}

template <int W>
// Six resident blocks per SM (<= 80 registers, a few spills): 24 warps hide
// the traversal's load latency better than 16 warps at 128 registers
// (+10 % at K = 1, +7 % at K = 3 on the box-wing, bit-identical).
__global__ void __launch_bounds__(128, 6) grad_kernel(const DesignDev dz, const TraceParams p, const GradParams g) {
    __shared__ GradWarpSmem sm[4];
    // hinge points and axes in FP32, converted once per block (a per-ray
    // FP64 load and conversion runs on the FP64 pipe, slow on this GPU)
    __shared__ float hxf[8][6];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    GradWarpSmem& ws = sm[warp];
    if (threadIdx.x < 6 * g.H) hxf[threadIdx.x / 6][threadIdx.x % 6] = (float)g.hax[threadIdx.x];
    __syncthreads();
    // each lane keeps the running sums of the last hit's group (rho_s and
    // rho_d entries) and of its hinge in registers while they repeat, and
    // adds them to the warp's shared sums when they change and before each
    // flush (neighbouring rays mostly end on the same facet)
    int cg = -1, chh = -1;
    float cs0 = 0.0f, cs1 = 0.0f, chs = 0.0f;
    const int64_t units = (int64_t)p.S * p.cpb;
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    uint32_t nvis = 0, ntest = 0;
    for (int e = lane; e < kMaxGradEntries; e += 32) { ws.f[e] = 0.0f; ws.d[e] = 0.0; }
    __syncwarp();
    for (int64_t u = gw; u < units; u += nw) {
        const int s = (int)(u / p.cpb);
        const int64_t cidx = u % p.cpb;
        const double* up = g.up + 6 * (size_t)s;
        const float3 gF = f3((float)up[0], (float)up[1], (float)up[2]);
        const float3 gT = f3((float)up[3], (float)up[4], (float)up[5]);
        // the item's grid constants and the direction-only part of the
        // primary rays' set-up (1/d and the shear rows), shared by the
        // unit's rays: from the span pre-pass's table on full grids, else
        // computed once per unit (the same values as a per-ray setup_ray)
        ItemConst ic;
        if (p.rowoff != nullptr) {
            item_load(ic, p.itab + 8 * (size_t)s, p.rho, p.design_base, p.sun_base + s);
            if (lane < 12) ws.dirc[lane] = __ldg(reinterpret_cast<const float*>(p.itab + 8 * (size_t)s + 5) + lane);
        } else {
            item_setup(ic, dz, p, p.sun + 3 * (size_t)s, p.com, p.rho, p.design_base, p.sun_base + s);
            if (lane == 0) item_dirc(ic, ws.dirc);
        }
        __syncwarp();
        // span mode (full grids of whole 32-pixel batches, as in the
        // forward): the unit's share of the item's batches that can meet
        // the scene -- a ray of any other batch misses every box, so its
        // path and its gradient contribution are empty; otherwise the
        // contiguous slots [k0, k1) of the ray subset
        const bool span = p.rowoff != nullptr;
        const int32_t* rowoff = nullptr;
        const int32_t* rowfirst = nullptr;
        int64_t k0, k1;
        int row = 0;
        if (span) {
            const int nband = p.ny / p.bh;
            rowoff = p.rowoff + (size_t)s * (nband + 1);
            rowfirst = p.rowfirst + (size_t)s * nband;
            const int64_t L = __ldg(rowoff + nband);
            k0 = cidx * L / p.cpb;
            k1 = (cidx + 1) * L / p.cpb;
            // the last row whose prefix is <= k0, 32 rows per round
            int lo = 0, hi = nband;
            while (hi - lo > 1) {
                const int step = (hi - lo + 31) / 32;
                const int r = lo + lane * step;
                const bool ok = r < hi && (int64_t)__ldg(rowoff + r) <= k0;
                const unsigned m = __ballot_sync(0xffffffffu, ok);
                lo += (31 - __clz(m)) * step;
                hi = min(hi, lo + step);
            }
            row = lo;
        } else {
            k0 = cidx * p.chunk;
            k1 = min(k0 + p.chunk, p.n);
        }
        int batch = 0;
        for (int64_t kb = k0; kb < k1; kb += span ? 1 : 32, ++batch) {
            int64_t k;
            uint64_t i;
            if (span) {
                while ((int64_t)__ldg(rowoff + row + 1) <= kb) ++row;
                i = span_ray((int64_t)row * p.bh * p.nx +
                                 (32 / p.bh) * ((int64_t)__ldg(rowfirst + row) + (kb - __ldg(rowoff + row))),
                             lane, p.bh, p.nx);
                k = kb;
            } else {
                k = kb + lane;
                i = (uint64_t)(p.off + k * p.stride);
            }
            if (k < k1 && p.K == 1) {
                // ---- one hit per path: the same arithmetic as the general
                // replay below at K = 1, with nothing recorded (registers
                // only, no per-ray arrays)
                const Seg s0 = primary_seg(ic, p, i);
                RaySetup rs;
                rs.o = s0.o; rs.d = s0.d;
                rs.inv = f3(ws.dirc[0], ws.dirc[1], ws.dirc[2]);
                rs.oinv = f3(s0.o.x * rs.inv.x, s0.o.y * rs.inv.y, s0.o.z * rs.inv.z);
                rs.mx = f3(ws.dirc[3], ws.dirc[4], ws.dirc[5]);
                rs.my = f3(ws.dirc[6], ws.dirc[7], ws.dirc[8]);
                rs.mz = f3(ws.dirc[9], ws.dirc[10], ws.dirc[11]);
                float t;
                const int f = closest_hit<W>(dz, rs, 0.0f, s0.src, t, p.err, nvis, ntest);
                if (f >= 0) {
                    const HitGeom h = hit_geom(dz, ic, f, t, s0);
                    const float3 qv = gF + cross(gT, h.x - ic.com);
                    const float qd = dot(qv, s0.d), qn = dot(qv, h.n);
                    if (h.g != cg) {
                        if (cg >= 0) { atomicAdd(&ws.f[2 * cg], cs0); atomicAdd(&ws.f[2 * cg + 1], cs1); }
                        cg = h.g; cs0 = 0.0f; cs1 = 0.0f;
                    }
                    cs0 += s0.w * (-qd - 2.0f * h.cs * qn);
                    cs1 += s0.w * (-(2.0f / 3.0f) * qn);
                    if (g.H > 0) {
                        const uint32_t orig = __float_as_uint(__ldg(dz.tri + 3 * (size_t)f).w);
                        const int hh = g.thinge ? __ldg(g.thinge + orig) : -1;
                        if (hh >= 0 && hh < g.H) {
                            const float* hp = hxf[hh];
                            const float3 ap = f3(hp[0], hp[1], hp[2]);
                            const float3 aa = f3(hp[3], hp[4], hp[5]);
                            const float3 x = h.x, n = h.n, d = s0.d;
                            const float c = h.cs, rs_ = h.rs, rd = h.rd;
                            const float cn = 2.0f * rs_ * c + (2.0f / 3.0f) * rd;
                            const float3 Gv = (1.0f - rs_) * d - cn * n;
                            const float3 dn = cross(aa, n);
                            const float3 dx = cross(aa, x - ap);
                            const float dc = -dot(dn, d);
                            const float3 dq = cross(gT, dx);
                            const float3 dG = (-2.0f * rs_ * dc) * n - cn * dn;
                            const float dphi = dc * dot(qv, Gv) + c * (dot(dq, Gv) + dot(qv, dG));
                            if (hh != chh) {
                                if (chh >= 0) atomicAdd(&ws.f[2 * p.G + chh], chs);
                                chh = hh; chs = 0.0f;
                            }
                            chs += (s0.w / c) * dphi;
                        }
                    }
                }
            } else if (k < k1) {
                Seg s0 = primary_seg(ic, p, i);
                // ---- forward replay with the path recorded
                int m = 0;
                int fr[kMaxBounces], br[kMaxBounces];
                float3 xr[kMaxBounces], nr[kMaxBounces], dr[kMaxBounces], dout_r[kMaxBounces];
                float csr[kMaxBounces], wr[kMaxBounces], rsr[kMaxBounces], rdr[kMaxBounces];
                int gr[kMaxBounces];
                Seg sg = s0;
#pragma unroll 1
                for (int kk = 1; kk <= p.K; ++kk) {
                    RaySetup rs;
                    if (kk == 1) {
                        rs.o = sg.o; rs.d = sg.d;
                        rs.inv = f3(ws.dirc[0], ws.dirc[1], ws.dirc[2]);
                        rs.oinv = f3(sg.o.x * rs.inv.x, sg.o.y * rs.inv.y, sg.o.z * rs.inv.z);
                        rs.mx = f3(ws.dirc[3], ws.dirc[4], ws.dirc[5]);
                        rs.my = f3(ws.dirc[6], ws.dirc[7], ws.dirc[8]);
                        rs.mz = f3(ws.dirc[9], ws.dirc[10], ws.dirc[11]);
                    } else {
                        setup_ray(rs, sg.o, sg.d);
                    }
                    float t;
                    const int f = closest_hit<W>(dz, rs, kk == 1 ? 0.0f : ic.tmin_b, sg.src, t, p.err, nvis, ntest);
                    if (f < 0) break;
                    const HitGeom h = hit_geom(dz, ic, f, t, sg);
                    const int q = kk - 1;
                    fr[q] = f; xr[q] = h.x; nr[q] = h.n; dr[q] = sg.d; csr[q] = h.cs; wr[q] = sg.w;
                    rsr[q] = h.rs; rdr[q] = h.rd; gr[q] = h.g;
                    m = kk;
                    if (kk == p.K) break;
                    float3 dout;
                    float wout;
                    br[q] = bounce_dir(ic, p, (uint32_t)i, kk, h, sg, dout, wout);
                    dout_r[q] = dout;
                    sg.o = h.x; sg.d = dout; sg.w = wout; sg.src = f;
                }
                // ---- reverse sweep: L = sum_k q_k . dp_k, q_k = gF + gT x (x_k - com)
                float wbar_next = 0.0f;
#pragma unroll 1
                for (int q = m - 1; q >= 0; --q) {
                    const float3 qv = gF + cross(gT, xr[q] - ic.com);
                    const float w = wr[q];
                    float wbar;
                    if (q + 1 == p.K) {
                        const float qd = dot(qv, dr[q]), qn = dot(qv, nr[q]);
                        if (gr[q] != cg) {
                            if (cg >= 0) { atomicAdd(&ws.f[2 * cg], cs0); atomicAdd(&ws.f[2 * cg + 1], cs1); }
                            cg = gr[q]; cs0 = 0.0f; cs1 = 0.0f;
                        }
                        cs0 += w * (-qd - 2.0f * csr[q] * qn);
                        cs1 += w * (-(2.0f / 3.0f) * qn);
                        wbar = (1.0f - rsr[q]) * qd - (2.0f * rsr[q] * csr[q] + (2.0f / 3.0f) * rdr[q]) * qn;
                    } else {
                        const float wbar_out = wbar_next - dot(qv, dout_r[q]);
                        wbar = dot(qv, dr[q]);
                        const float rb = br[q] == 0 ? rsr[q] : rdr[q];
                        atomicAdd(&ws.f[2 * gr[q] + br[q]], wbar_out * 2.0f * w);
                        wbar += wbar_out * 2.0f * rb;
                    }
                    wbar_next = wbar;
                }
                // ---- hinge angles, K > 1: tangents along the recorded path
                if (g.H > 0 && p.K > 1 && m > 0 && g.thinge) {
                    int hid[kMaxBounces];
                    for (int q = 0; q < m; ++q)
                        hid[q] = __ldg(g.thinge + __float_as_uint(__ldg(dz.tri + 3 * (size_t)fr[q]).w));
                    for (int q = 0; q < m; ++q) {
                        const int hh = hid[q];
                        bool dup = hh < 0 || hh >= g.H;
                        for (int q2 = 0; q2 < q; ++q2) dup = dup || hid[q2] == hh;
                        if (dup) continue;
                        const float* hp = hxf[hh];
                        const float3 ap = f3(hp[0], hp[1], hp[2]);
                        const float3 aa = f3(hp[3], hp[4], hp[5]);
                        const float dL = hinge_path_tangent(dz, hh, ap, aa, m, p.K, hid, fr, br, xr, nr, dr, dout_r, csr,
                                                            wr, rsr, rdr, ic.com, gF, gT);
                        atomicAdd(&ws.f[2 * p.G + hh], dL);
                    }
                }
                // ---- hinge angle (K = 1): surface element carried by its facet
                if (g.H > 0 && p.K == 1 && m == 1) {
                    const uint32_t orig = __float_as_uint(__ldg(dz.tri + 3 * (size_t)fr[0]).w);
                    const int hh = g.thinge ? __ldg(g.thinge + orig) : -1;
                    if (hh >= 0 && hh < g.H) {
                        const float* hp = hxf[hh];
                        const float3 ap = f3(hp[0], hp[1], hp[2]);
                        const float3 aa = f3(hp[3], hp[4], hp[5]);
                        const float3 x = xr[0], n = nr[0], d = dr[0];
                        const float c = csr[0], rs = rsr[0], rd = rdr[0];
                        const float3 qv = gF + cross(gT, x - ic.com);
                        const float cn = 2.0f * rs * c + (2.0f / 3.0f) * rd;
                        const float3 Gv = (1.0f - rs) * d - cn * n;
                        const float3 dn = cross(aa, n);
                        const float3 dx = cross(aa, x - ap);
                        const float dc = -dot(dn, d);
                        const float3 dq = cross(gT, dx);
                        const float3 dG = (-2.0f * rs * dc) * n - cn * dn;
                        const float dphi = dc * dot(qv, Gv) + c * (dot(dq, Gv) + dot(qv, dG));
                        if (hh != chh) {
                            if (chh >= 0) atomicAdd(&ws.f[2 * p.G + chh], chs);
                            chh = hh; chs = 0.0f;
                        }
                        chs += (wr[0] / c) * dphi;
                    }
                }
            }
            if ((batch & 15) == 15 || kb + (span ? 1 : 32) >= k1) {   // flush FP32 sums (<= 512 rays) to FP64
                if (cg >= 0) { atomicAdd(&ws.f[2 * cg], cs0); atomicAdd(&ws.f[2 * cg + 1], cs1); cg = -1; }
                if (chh >= 0) { atomicAdd(&ws.f[2 * p.G + chh], chs); chh = -1; }
            }
            __syncwarp();
            if ((batch & 15) == 15 || kb + (span ? 1 : 32) >= k1) {
                for (int e = lane; e < g.ng; e += 32) { ws.d[e] += (double)ws.f[e]; ws.f[e] = 0.0f; }
                __syncwarp();
            }
        }
        for (int e = lane; e < g.ng; e += 32) {
            g.gpart[(size_t)u * g.ng + e] = ws.d[e];
            ws.d[e] = 0.0;
        }
        __syncwarp();
    }
    if (p.stats) {
        unsigned long long a = nvis, b = ntest;
        for (int off = 16; off > 0; off >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, off);
            b += __shfl_xor_sync(0xffffffffu, b, off);
        }
        if (lane == 0) { atomicAdd(p.stats, a); atomicAdd(p.stats + 1, b); }
    }
}

constexpr int kGradReduceThreads = 256;

// Entry e = blockIdx.x: thread t sums units t, t + 256, ...; then a fixed
// tree over the threads (deterministic).
__global__ void __launch_bounds__(kGradReduceThreads) grad_reduce_kernel(const double* __restrict__ gpart, int64_t units,
                                                                         int ng, int G, double* d_rho, double* d_hinge) {
    __shared__ double red[kGradReduceThreads];
    const int e = blockIdx.x, t = threadIdx.x;
    double a = 0.0;
    for (int64_t u = t; u < units; u += kGradReduceThreads) a += gpart[(size_t)u * ng + e];
    red[t] = a;
    __syncthreads();
    for (int h = kGradReduceThreads / 2; h > 0; h >>= 1) {
        if (t < h) red[t] += red[t + h];
        __syncthreads();
    }
    if (t == 0) {
        if (e < 2 * G) d_rho[e] = red[0];
        else if (d_hinge) d_hinge[e - 2 * G] = red[0];
    }
}

cudaError_t launch_span(const TraceParams& p, int width, cudaStream_t st);

cudaError_t launch_grad(const DesignDev& dz, const TraceParams& p, const double* up, const int32_t* thinge,
                        const double* hax, int H, double* gpart, double* d_rho, double* d_hinge, int n_sm,
                        cudaStream_t st) {
    if (p.rowoff && (int64_t)p.S * p.cpb > 0 && p.n > 0) {
        const cudaError_t e = launch_span(p, dz.width, st);
        if (e != cudaSuccess) return e;
    }
    GradParams g;
    g.up = up; g.thinge = thinge; g.hax = hax; g.H = H; g.ng = 2 * p.G + H; g.gpart = gpart;
    const int64_t units = (int64_t)p.S * p.cpb;
    if (units > 0 && p.n > 0) {
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((units + 3) / 4, (int64_t)n_sm * 12));
        if (dz.width == 8) grad_kernel<8><<<grid, 128, 0, st>>>(dz, p, g);
        else grad_kernel<4><<<grid, 128, 0, st>>>(dz, p, g);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    grad_reduce_kernel<<<g.ng, kGradReduceThreads, 0, st>>>(gpart, units, g.ng, p.G, d_rho, d_hinge);
    return cudaGetLastError();
}

}  // namespace srp
