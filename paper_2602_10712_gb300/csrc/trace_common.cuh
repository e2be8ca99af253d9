// trace_common.cuh -- device-side pieces shared by the SRP tracer kernels
// (trace.cu) and the gradient kernels (grad.cu): Philox4x32-10, ray set-up,
// the watertight ray/triangle test, wide-BVH closest-hit traversal, ray
// generation and the per-hit shading of the estimator.  Keeping them in one
// place keeps the forward and the adjoint on identical arithmetic.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "srp_internal.h"

namespace srp {

struct DesignTable {
    DesignDev d[kMaxDesignsPerLaunch];
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), 10 rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}
// uniform in [0,1) from the top 24 bits (exact in FP32)
__device__ __forceinline__ float unit24(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }

// ---------------------------------------------------------------------------
// small vector helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return f3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
    return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 xyz(float4 v) { return f3(v.x, v.y, v.z); }

// ---------------------------------------------------------------------------
// Ray state for traversal: slab-test constants and watertight shear.
// ---------------------------------------------------------------------------
struct RaySetup {
    float3 o, d;
    float3 inv;      // 1/d (zeros replaced by +-1e-30)
    float3 oinv;     // o * inv
    float3 mx, my, mz;  // shear rows: A_x = mx.A, A_y = my.A, A_z = mz.A
};

__device__ __forceinline__ float safe_inv(float x) {
    return 1.0f / (fabsf(x) > 1e-30f ? x : copysignf(1e-30f, x));
}

__device__ __forceinline__ void setup_ray(RaySetup& r, float3 o, float3 d) {
    r.o = o; r.d = d;
    r.inv = f3(safe_inv(d.x), safe_inv(d.y), safe_inv(d.z));
    r.oinv = f3(o.x * r.inv.x, o.y * r.inv.y, o.z * r.inv.z);
    const float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
    int kz = 0;
    if (ay > ax && ay >= az) kz = 1;
    else if (az > ax && az > ay) kz = 2;
    int kx = kz == 2 ? 0 : kz + 1;
    int ky = kx == 2 ? 0 : kx + 1;
    const float dk[3] = {d.x, d.y, d.z};
    if (dk[kz] < 0.0f) { int t = kx; kx = ky; ky = t; }
    const float Sx = dk[kx] / dk[kz], Sy = dk[ky] / dk[kz], Sz = 1.0f / dk[kz];
    float m[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    m[0][kx] = 1.0f; m[0][kz] = -Sx;
    m[1][ky] = 1.0f; m[1][kz] = -Sy;
    m[2][kz] = Sz;
    r.mx = f3(m[0][0], m[0][1], m[0][2]);
    r.my = f3(m[1][0], m[1][1], m[1][2]);
    r.mz = f3(m[2][0], m[2][1], m[2][2]);
}

// Watertight test; returns t, or -1 when missed (callers need t > tmin >= 0).  Edge functions use
// products without FMA contraction so shared edges are exactly antisymmetric.
__device__ __forceinline__ float hit_triangle(const RaySetup& r, float3 p0, float3 p1, float3 p2) {
    const float3 A = p0 - r.o, B = p1 - r.o, C = p2 - r.o;
    const float Ax = dot(r.mx, A), Ay = dot(r.my, A);
    const float Bx = dot(r.mx, B), By = dot(r.my, B);
    const float Cx = dot(r.mx, C), Cy = dot(r.my, C);
    float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
    float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
    float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
    if (U == 0.0f || V == 0.0f || W == 0.0f) {   // recompute exactly-zero edges in FP64
        U = (float)((double)Cx * (double)By - (double)Cy * (double)Bx);
        V = (float)((double)Ax * (double)Cy - (double)Ay * (double)Cx);
        W = (float)((double)Bx * (double)Ay - (double)By * (double)Ax);
    }
    if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return -1.0f;
    const float det = U + V + W;
    if (det == 0.0f) return -1.0f;
    const float T = U * dot(r.mz, A) + V * dot(r.mz, B) + W * dot(r.mz, C);
    return T / det;
}

// Slab distances of four children on one axis, x[q] * s + c for q = 0..3,
// two children per packed FP32 FMA (fma.rn.f32x2, sm_100 and later: the
// same rounding as fmaf, half the instructions); s2 and c2 hold (s, s) and
// (c, c).  Measured on 512 of the benchmark's suns: +2.6 % rays/s at K <= 3,
// +2.1 % at K = 1, results bit-identical to the scalar FMAs.
__device__ __forceinline__ unsigned long long pack2(float v) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ void slab4(const float4 x, unsigned long long s2, unsigned long long c2, float (&o)[4]) {
    asm("{\n .reg .b64 xa, xb, ya, yb;\n"
        " mov.b64 xa, {%4, %5};\n mov.b64 xb, {%6, %7};\n"
        " fma.rn.f32x2 ya, xa, %8, %9;\n fma.rn.f32x2 yb, xb, %8, %9;\n"
        " mov.b64 {%0, %1}, ya;\n mov.b64 {%2, %3}, yb;\n}"
        : "=f"(o[0]), "=f"(o[1]), "=f"(o[2]), "=f"(o[3])
        : "f"(x.x), "f"(x.y), "f"(x.z), "f"(x.w), "l"(s2), "l"(c2));
}

// Compare-exchange of entries a < b of a sorting network on (key, child):
// the smaller key first; a child of -1 (key +inf) sorts last.
__device__ __forceinline__ void sort_cx(float (&k)[4], int (&c)[4], int a, int b) {
    const bool sw = k[b] < k[a];
    const float ka = k[a], kb = k[b];
    const int ca = c[a], cb = c[b];
    k[a] = sw ? kb : ka; k[b] = sw ? ka : kb;
    c[a] = sw ? cb : ca; c[b] = sw ? ca : cb;
}

// ---------------------------------------------------------------------------
// Closest hit through a W-wide BVH.  Returns the leaf-order triangle index
// (or -1) and sets tb.  Ties on t go to the smaller original index.
// ---------------------------------------------------------------------------
template <int W>
__device__ __forceinline__ int closest_hit(const DesignDev& dz, const RaySetup& r, float tmin, int skip,
                                           float& tb, int* err, uint32_t& nvis, uint32_t& ntest) {
    constexpr int NF4 = W == 4 ? 8 : 16;  // float4 per node
    const float4* __restrict__ nodes = dz.nodes;
    const float4* __restrict__ tri = dz.tri;
    int2 stack[kStackSize];
    int sp = 0;
    int best = -1;
    uint32_t best_id = 0xffffffffu;
    tb = INFINITY;
    int ni = 0;
    int visits = 0;
    // near/far slab planes chosen by load address (per-ray float4 offsets):
    // lo_a at float4 (2a)*(W/4) + h, hi_a at (2a+1)*(W/4) + h
    constexpr int Q = W / 4;
    const int nxo = r.inv.x < 0.0f ? Q : 0, nyo = r.inv.y < 0.0f ? Q : 0, nzo = r.inv.z < 0.0f ? Q : 0;
    const unsigned long long sx2 = pack2(r.inv.x), sy2 = pack2(r.inv.y), sz2 = pack2(r.inv.z);
    const unsigned long long cx2 = pack2(-r.oinv.x), cy2 = pack2(-r.oinv.y), cz2 = pack2(-r.oinv.z);
    while (true) {
        if (++visits > kVisitCap) { atomicOr(err, kErrVisitCap); return -1; }
        ++nvis;
        const float4* nd = nodes + (size_t)ni * NF4;
        float tn[W];
        bool hit[W];
        int child[W];
#pragma unroll
        for (int h = 0; h < Q; ++h) {
            const float4 ax = __ldg(nd + nxo + h), bx = __ldg(nd + (Q - nxo) + h);
            const float4 ay = __ldg(nd + 2 * Q + nyo + h), by = __ldg(nd + 2 * Q + (Q - nyo) + h);
            const float4 az = __ldg(nd + 4 * Q + nzo + h), bz = __ldg(nd + 4 * Q + (Q - nzo) + h);
            const int4 ch = __ldg(reinterpret_cast<const int4*>(nd + 6 * Q) + h);
            float nx_[4], fx_[4], ny_[4], fy_[4], nz_[4], fz_[4];
            slab4(ax, sx2, cx2, nx_); slab4(bx, sx2, cx2, fx_);
            slab4(ay, sy2, cy2, ny_); slab4(by, sy2, cy2, fy_);
            slab4(az, sz2, cz2, nz_); slab4(bz, sz2, cz2, fz_);
            const int ch_[4] = {ch.x, ch.y, ch.z, ch.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float n0 = nx_[q], f0 = fx_[q], n1 = ny_[q], f1 = fy_[q], n2 = nz_[q], f2 = fz_[q];
                const float tnear = fmaxf(fmaxf(n0, n1), fmaxf(n2, tmin));
                const float tfar = fminf(fminf(f0, f1), fminf(f2, tb));
                tn[4 * h + q] = tnear;
                hit[4 * h + q] = tnear <= tfar;
                child[4 * h + q] = ch_[q];
            }
        }
        // leaves first: they may shrink tb before inner children are queued.
        // The hit leaves of the node are taken one after another from a
        // slot mask (ascending slots), so lanes whose leaves sit in
        // different slots run their triangle tests in the same iterations
        // instead of one masked pass per slot.
        unsigned lm = 0u;
#pragma unroll
        for (int c = 0; c < W; ++c) lm |= (hit[c] && child[c] < 0) ? (1u << c) : 0u;
        while (lm != 0u) {
            const int c = __ffs(lm) - 1;
            lm &= lm - 1u;
            int ch = child[0];
#pragma unroll
            for (int j = 1; j < W; ++j) ch = c == j ? child[j] : ch;
            const int code = ~ch;
            const int first = code >> 3, cnt = (code & 7) + 1;
            ntest += cnt;
            for (int q = 0; q < cnt; ++q) {
                const int f = first + q;
                if (f == skip) continue;
                const float4 a = __ldg(tri + 3 * (size_t)f);
                const float4 b = __ldg(tri + 3 * (size_t)f + 1);
                const float4 cc = __ldg(tri + 3 * (size_t)f + 2);
                const float t = hit_triangle(r, xyz(a), xyz(b), xyz(cc));
                if (t > tmin && t <= tb) {
                    const uint32_t id = __float_as_uint(a.w);
                    if (t < tb || id < best_id) { tb = t; best = f; best_id = id; }
                }
            }
        }
        int next = -1;
        if (W == 4) {
            // the inner children still in reach sorted by entry distance
            // (five compare-exchanges), pushed farthest first so that the
            // nearest remaining one is popped first; the nearest is next
            float k[4];
            int cc[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const bool in = hit[c] && child[c] >= 0 && tn[c] <= tb;
                k[c] = in ? tn[c] : INFINITY;
                cc[c] = in ? child[c] : -1;
            }
            sort_cx(k, cc, 0, 1); sort_cx(k, cc, 2, 3); sort_cx(k, cc, 0, 2); sort_cx(k, cc, 1, 3); sort_cx(k, cc, 1, 2);
#pragma unroll
            for (int c = 3; c >= 1; --c) {
                if (cc[c] >= 0) {
                    if (sp >= kStackSize) { atomicOr(err, kErrStackOverflow); return -1; }
                    stack[sp++] = make_int2(cc[c], __float_as_int(k[c]));
                }
            }
            next = cc[0];
        } else {
            float tnext = INFINITY;
#pragma unroll
            for (int c = 0; c < W; ++c) {
                if (hit[c] && child[c] >= 0 && tn[c] <= tb) {
                    if (tn[c] < tnext) {
                        if (next >= 0) {
                            if (sp >= kStackSize) { atomicOr(err, kErrStackOverflow); return -1; }
                            stack[sp++] = make_int2(next, __float_as_int(tnext));
                        }
                        next = child[c]; tnext = tn[c];
                    } else {
                        if (sp >= kStackSize) { atomicOr(err, kErrStackOverflow); return -1; }
                        stack[sp++] = make_int2(child[c], __float_as_int(tn[c]));
                    }
                }
            }
        }
        if (next >= 0) { ni = next; continue; }
        bool found = false;
        while (sp > 0) {
            const int2 e = stack[--sp];
            if (__int_as_float(e.y) <= tb) { ni = e.x; found = true; break; }
        }
        if (!found) break;
    }
    return best;
}

// ---------------------------------------------------------------------------
// Any hit through a W-wide BVH (shadow rays): true as soon as one triangle
// other than `skip` is hit at t > tmin.  Same node layout and slab test as
// closest_hit, no far-plane shrinking and no child ordering beyond taking
// the nearest child next.
// ---------------------------------------------------------------------------
template <int W>
__device__ __forceinline__ bool any_hit(const DesignDev& dz, const RaySetup& r, float tmin, int skip, int* err,
                                        uint32_t& nvis, uint32_t& ntest) {
    constexpr int NF4 = W == 4 ? 8 : 16;
    constexpr int Q = W / 4;
    const float4* __restrict__ nodes = dz.nodes;
    const float4* __restrict__ tri = dz.tri;
    int stack[kStackSize];
    int sp = 0;
    int ni = 0;
    int visits = 0;
    const int nxo = r.inv.x < 0.0f ? Q : 0, nyo = r.inv.y < 0.0f ? Q : 0, nzo = r.inv.z < 0.0f ? Q : 0;
    const unsigned long long sx2 = pack2(r.inv.x), sy2 = pack2(r.inv.y), sz2 = pack2(r.inv.z);
    const unsigned long long cx2 = pack2(-r.oinv.x), cy2 = pack2(-r.oinv.y), cz2 = pack2(-r.oinv.z);
    while (true) {
        if (++visits > kVisitCap) { atomicOr(err, kErrVisitCap); return false; }
        ++nvis;
        const float4* nd = nodes + (size_t)ni * NF4;
        float tn[W];
        bool hit[W];
        int child[W];
#pragma unroll
        for (int h = 0; h < Q; ++h) {
            const float4 ax = __ldg(nd + nxo + h), bx = __ldg(nd + (Q - nxo) + h);
            const float4 ay = __ldg(nd + 2 * Q + nyo + h), by = __ldg(nd + 2 * Q + (Q - nyo) + h);
            const float4 az = __ldg(nd + 4 * Q + nzo + h), bz = __ldg(nd + 4 * Q + (Q - nzo) + h);
            const int4 ch = __ldg(reinterpret_cast<const int4*>(nd + 6 * Q) + h);
            float nx_[4], fx_[4], ny_[4], fy_[4], nz_[4], fz_[4];
            slab4(ax, sx2, cx2, nx_); slab4(bx, sx2, cx2, fx_);
            slab4(ay, sy2, cy2, ny_); slab4(by, sy2, cy2, fy_);
            slab4(az, sz2, cz2, nz_); slab4(bz, sz2, cz2, fz_);
            const int ch_[4] = {ch.x, ch.y, ch.z, ch.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float n0 = nx_[q], f0 = fx_[q], n1 = ny_[q], f1 = fy_[q], n2 = nz_[q], f2 = fz_[q];
                const float tnear = fmaxf(fmaxf(n0, n1), fmaxf(n2, tmin));
                const float tfar = fminf(fminf(f0, f1), f2);
                tn[4 * h + q] = tnear;
                hit[4 * h + q] = tnear <= tfar;
                child[4 * h + q] = ch_[q];
            }
        }
        // hit leaves from a slot mask, one loop (as in closest_hit)
        unsigned lm = 0u;
#pragma unroll
        for (int c = 0; c < W; ++c) lm |= (hit[c] && child[c] < 0) ? (1u << c) : 0u;
        while (lm != 0u) {
            const int c = __ffs(lm) - 1;
            lm &= lm - 1u;
            int ch = child[0];
#pragma unroll
            for (int j = 1; j < W; ++j) ch = c == j ? child[j] : ch;
            const int code = ~ch;
            const int first = code >> 3, cnt = (code & 7) + 1;
            ntest += cnt;
            for (int q = 0; q < cnt; ++q) {
                const int f = first + q;
                if (f == skip) continue;
                const float4 a = __ldg(tri + 3 * (size_t)f);
                const float4 b = __ldg(tri + 3 * (size_t)f + 1);
                const float4 cc = __ldg(tri + 3 * (size_t)f + 2);
                if (hit_triangle(r, xyz(a), xyz(b), xyz(cc)) > tmin) return true;
            }
        }
        int next = -1;
        float tnext = INFINITY;
#pragma unroll
        for (int c = 0; c < W; ++c) {
            if (hit[c] && child[c] >= 0) {
                if (tn[c] < tnext) {
                    if (next >= 0) {
                        if (sp >= kStackSize) { atomicOr(err, kErrStackOverflow); return false; }
                        stack[sp++] = next;
                    }
                    next = child[c]; tnext = tn[c];
                } else {
                    if (sp >= kStackSize) { atomicOr(err, kErrStackOverflow); return false; }
                    stack[sp++] = child[c];
                }
            }
        }
        if (next >= 0) { ni = next; continue; }
        if (sp == 0) break;
        ni = stack[--sp];
    }
    return false;
}

// ---------------------------------------------------------------------------
// A ray segment and the shading of its hit.
// ---------------------------------------------------------------------------
struct Seg {
    float3 o, d;
    float w;
    int src;  // leaf-order index of the triangle the segment leaves (-1: primary)
};

// Per-item constants shared by every ray of one (design, sun).
struct ItemConst {
    float3 ob, bu, bv, dd, com;
    float fdx, fdy, w0, tmin_b;
    const float* rho;
    int dglob, sglob;
};

__device__ __forceinline__ void item_setup(ItemConst& ic, const DesignDev& dz, const TraceParams& p,
                                           const double* sp, const double* cp, const float* rho,
                                           int dglob, int sglob) {
    // branchless ONB of d = -e (Duff et al. 2017) in FP64, rounded once
    const double dx_ = -sp[0], dy_ = -sp[1], dz_ = -sp[2];
    const double sgn = dz_ >= 0.0 ? 1.0 : -1.0;
    const double aa = -1.0 / (sgn + dz_);
    const double bb = dx_ * dy_ * aa;
    const double u0 = 1.0 + sgn * dx_ * dx_ * aa, u1 = sgn * bb, u2 = -sgn * dx_;
    const double v0 = bb, v1 = sgn + dy_ * dy_ * aa, v2 = -dy_;
    const double R = dz.R;
    const double pdx = 2.0 * R / p.nx, pdy = 2.0 * R / p.ny;
    ic.ob = f3((float)(dz.cx - R * u0 - R * v0 - 2.0 * R * dx_), (float)(dz.cy - R * u1 - R * v1 - 2.0 * R * dy_),
               (float)(dz.cz - R * u2 - R * v2 - 2.0 * R * dz_));
    ic.bu = f3((float)u0, (float)u1, (float)u2);
    ic.bv = f3((float)v0, (float)v1, (float)v2);
    ic.dd = f3((float)dx_, (float)dy_, (float)dz_);
    ic.fdx = (float)pdx; ic.fdy = (float)pdy;
    ic.w0 = (float)(p.P * pdx * pdy);
    ic.com = f3((float)cp[0], (float)cp[1], (float)cp[2]);
    ic.tmin_b = (float)(1e-6 * R);
    ic.rho = rho;
    ic.dglob = dglob; ic.sglob = sglob;
}

// The direction-only part of the primary rays' set-up (1/d and the shear
// rows of setup_ray), shared by every ray of an item.
__device__ __forceinline__ void item_dirc(const ItemConst& ic, float* dirc) {
    RaySetup rd;
    setup_ray(rd, f3(0.0f, 0.0f, 0.0f), ic.dd);
    dirc[0] = rd.inv.x; dirc[1] = rd.inv.y; dirc[2] = rd.inv.z;
    dirc[3] = rd.mx.x; dirc[4] = rd.mx.y; dirc[5] = rd.mx.z;
    dirc[6] = rd.my.x; dirc[7] = rd.my.y; dirc[8] = rd.my.z;
    dirc[9] = rd.mz.x; dirc[10] = rd.mz.y; dirc[11] = rd.mz.z;
}

// An item's FP32 grid constants and primary direction set-up as one
// 8 x float4 record (TraceParams::itab), and back.
__device__ __forceinline__ void item_store(const ItemConst& ic, float4* rec) {
    rec[0] = make_float4(ic.ob.x, ic.ob.y, ic.ob.z, ic.fdx);
    rec[1] = make_float4(ic.bu.x, ic.bu.y, ic.bu.z, ic.fdy);
    rec[2] = make_float4(ic.bv.x, ic.bv.y, ic.bv.z, ic.w0);
    rec[3] = make_float4(ic.dd.x, ic.dd.y, ic.dd.z, ic.tmin_b);
    rec[4] = make_float4(ic.com.x, ic.com.y, ic.com.z, 0.0f);
    float dc[12];
    item_dirc(ic, dc);
    rec[5] = make_float4(dc[0], dc[1], dc[2], dc[3]);
    rec[6] = make_float4(dc[4], dc[5], dc[6], dc[7]);
    rec[7] = make_float4(dc[8], dc[9], dc[10], dc[11]);
}
__device__ __forceinline__ void item_load(ItemConst& ic, const float4* rec, const float* rho, int dglob, int sglob) {
    const float4 a = __ldg(rec), b = __ldg(rec + 1), c = __ldg(rec + 2), d = __ldg(rec + 3), e = __ldg(rec + 4);
    ic.ob = f3(a.x, a.y, a.z); ic.fdx = a.w;
    ic.bu = f3(b.x, b.y, b.z); ic.fdy = b.w;
    ic.bv = f3(c.x, c.y, c.z); ic.w0 = c.w;
    ic.dd = f3(d.x, d.y, d.z); ic.tmin_b = d.w;
    ic.com = f3(e.x, e.y, e.z);
    ic.rho = rho;
    ic.dglob = dglob; ic.sglob = sglob;
}

// Span mode: the grid ray of lane l in the batch whose top-left pixel has
// grid index b; a batch is a block of 32 / bh columns x bh rows (bh = 1, 2
// or 4), lanes along its rows, so lanes 2c and 2c + 1 hold horizontally
// neighbouring pixels (the pairs of the collapsed-strata variance).
__device__ __forceinline__ uint64_t span_ray(int64_t b, int l, int bh, int nx) {
    const int sh = bh == 4 ? 3 : (bh == 2 ? 4 : 5);   // log2 of the block width
    return (uint64_t)(b + (int64_t)(l >> sh) * nx + (l & ((1 << sh) - 1)));
}

// Primary segment of grid ray i (jittered pixel origin, travel direction d).
__device__ __forceinline__ Seg primary_seg(const ItemConst& ic, const TraceParams& p, uint64_t i) {
    // i < nx * ny < 2^32 (checked on the host): 32-bit division
    const uint32_t i32 = (uint32_t)i, nx32 = (uint32_t)p.nx;
    const uint32_t py = i32 / nx32, px = i32 - py * nx32;
    float xi1 = 0.5f, xi2 = 0.5f;
    if (p.jitter) {
        const uint4 rnd = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)ic.sglob, (uint32_t)ic.dglob, 0u),
                                        (uint32_t)p.seed, (uint32_t)(p.seed >> 32));
        xi1 = unit24(rnd.x); xi2 = unit24(rnd.y);
    }
    const float a = ((float)px + xi1) * ic.fdx, b = ((float)py + xi2) * ic.fdy;
    Seg s;
    s.o = f3(fmaf(a, ic.bu.x, fmaf(b, ic.bv.x, ic.ob.x)), fmaf(a, ic.bu.y, fmaf(b, ic.bv.y, ic.ob.y)),
             fmaf(a, ic.bu.z, fmaf(b, ic.bv.z, ic.ob.z)));
    s.d = ic.dd;
    s.w = ic.w0;
    s.src = -1;
    return s;
}

// Geometry and material of hit on leaf-order triangle f at parameter t.
struct HitGeom {
    float3 x, n;   // hit point, unit normal facing the arriving ray
    float cs;      // cos = -n.d > 0
    float rs, rd;  // reflectances of the triangle's group
    int g;         // material group
};

// Geometry and material of a hit at parameter t on the triangle with vertices
// (a, b, c) (group id in b.w).
__device__ __forceinline__ HitGeom hit_geom_v(float4 a, float4 b, float4 c, const ItemConst& ic, float t,
                                              const Seg& s) {
    float3 n = cross(xyz(b) - xyz(a), xyz(c) - xyz(a));
    n = rsqrtf(dot(n, n)) * n;
    if (dot(n, s.d) > 0.0f) n = -1.0f * n;
    HitGeom h;
    h.n = n;
    h.cs = -dot(n, s.d);
    h.g = (int)__float_as_uint(b.w);
    h.rs = __ldg(ic.rho + 2 * h.g);
    h.rd = __ldg(ic.rho + 2 * h.g + 1);
    h.x = s.o + t * s.d;
    return h;
}

__device__ __forceinline__ HitGeom hit_geom(const DesignDev& dz, const ItemConst& ic, int f, float t, const Seg& s) {
    return hit_geom_v(__ldg(dz.tri + 3 * (size_t)f), __ldg(dz.tri + 3 * (size_t)f + 1),
                      __ldg(dz.tri + 3 * (size_t)f + 2), ic, t, s);
}

// Sampled reflection at hit k < K: branch 0 specular (weight 2 w rs),
// 1 Lambertian (weight 2 w rd, direction of n + uniform unit vector).
__device__ __forceinline__ int bounce_dir(const ItemConst& ic, const TraceParams& p, uint32_t i, int k,
                                          const HitGeom& h, const Seg& s, float3& dout, float& wout) {
    const uint4 rnd = philox4x32_10(make_uint4(i, (uint32_t)ic.sglob, (uint32_t)ic.dglob, (uint32_t)k),
                                    (uint32_t)p.seed, (uint32_t)(p.seed >> 32));
    if (unit24(rnd.x) < 0.5f) {
        dout = s.d + (2.0f * h.cs) * h.n;
        wout = 2.0f * s.w * h.rs;
        return 0;
    }
    const float z = 1.0f - 2.0f * unit24(rnd.y);
    const float rr = sqrtf(fmaxf(0.0f, 1.0f - z * z));
    float sp, cp;
    sincospif(2.0f * unit24(rnd.z), &sp, &cp);
    const float3 v = f3(h.n.x + rr * cp, h.n.y + rr * sp, h.n.z + z);
    const float l2 = dot(v, v);
    dout = l2 > 0.0f ? rsqrtf(l2) * v : h.n;
    wout = 2.0f * s.w * h.rd;
    return 1;
}

// Momentum deposit of hit k (1-based) on leaf-order triangle f at ray
// parameter t; returns true (and the outgoing segment) if the path goes on.
// Deposit of hit k of segment s with geometry h (triangle f); returns true
// and the next segment when the path continues (k < K).
__device__ __forceinline__ bool shade_core(const HitGeom& h, const ItemConst& ic, const TraceParams& p, uint32_t i,
                                           int k, int f, const Seg& s, float y[6], Seg& out) {
    const float3 arm = h.x - ic.com;
    if (k == p.K) {
        const float cn = 2.0f * h.rs * h.cs + (2.0f / 3.0f) * h.rd;
        const float3 dp = s.w * ((1.0f - h.rs) * s.d - cn * h.n);
        const float3 tq = cross(arm, dp);
        y[0] += dp.x; y[1] += dp.y; y[2] += dp.z; y[3] += tq.x; y[4] += tq.y; y[5] += tq.z;
        return false;
    }
    float3 dout;
    float wout;
    bounce_dir(ic, p, i, k, h, s, dout, wout);
    const float3 dp = s.w * s.d - wout * dout;
    const float3 tq = cross(arm, dp);
    y[0] += dp.x; y[1] += dp.y; y[2] += dp.z; y[3] += tq.x; y[4] += tq.y; y[5] += tq.z;
    out.o = h.x; out.d = dout; out.w = wout; out.src = f;
    return true;
}

__device__ __forceinline__ bool shade_hit(const DesignDev& dz, const ItemConst& ic, const TraceParams& p,
                                          uint32_t i, int k, int f, float t, const Seg& s, float y[6],
                                          Seg& out) {
    return shade_core(hit_geom(dz, ic, f, t, s), ic, p, i, k, f, s, y, out);
}


}  // namespace srp
