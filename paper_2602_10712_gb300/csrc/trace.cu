// trace.cu -- the SRP ray-grid tracer for sm_103a.
//
// One pass of the hot path (paper Sec. 3.2: force and torque integrals
// estimated by tracing radiation): for every (design, sun direction) item
// and every ray of its parallel-ray grid:
//   ray generation (Philox4x32-10 jitter, Duff et al. 2017 ONB)
//   -> closest hit through the W-wide BVH (slab tests, per-thread stack)
//   -> watertight ray/triangle test (Woop, Benthin, Wald 2013)
//   -> momentum deposit per the facet BRDF (absorbed / specular /
//      Lambertian), up to K hits with sampled specular/diffuse bounces
//   -> per-ray FP32 force and torque, accumulated per thread in FP64,
//      warp-shuffle + shared-memory block reduction to FP64 partials
// and a second kernel sums the partials of each item in a fixed order.
//
// Work decomposition: an item's n rays are split into `cpb` chunks of
// `chunk` rays (a multiple of 64); one block processes one chunk at a time,
// thread t handling rays k = start + t + j*blockDim, so a warp traces 32
// neighbouring pixels of one grid row (coherent parallel rays share BVH
// nodes through L1).  Blocks loop over chunks with a static stride.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

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

// Branchless orthonormal basis around unit n (Duff et al. 2017), FP32.
__device__ __forceinline__ void onb_f(float3 n, float3& b1, float3& b2) {
    const float sign = n.z >= 0.0f ? 1.0f : -1.0f;
    const float a = -1.0f / (sign + n.z);
    const float b = n.x * n.y * a;
    b1 = f3(1.0f + sign * n.x * n.x * a, sign * b, -sign * n.x);
    b2 = f3(b, sign + n.y * n.y * a, -n.y);
}

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
    const bool nx_ = r.inv.x < 0.0f, ny_ = r.inv.y < 0.0f, nz_ = r.inv.z < 0.0f;
    while (true) {
        if (++visits > kVisitCap) { atomicOr(err, kErrVisitCap); return -1; }
        ++nvis;
        const float4* nd = nodes + (size_t)ni * NF4;
        float tn[W];
        bool hit[W];
        int child[W];
#pragma unroll
        for (int h = 0; h < W / 4; ++h) {
            const float4 lox = __ldg(nd + 0 * (W / 4) + h), hix = __ldg(nd + 1 * (W / 4) + h);
            const float4 loy = __ldg(nd + 2 * (W / 4) + h), hiy = __ldg(nd + 3 * (W / 4) + h);
            const float4 loz = __ldg(nd + 4 * (W / 4) + h), hiz = __ldg(nd + 5 * (W / 4) + h);
            const int4 ch = __ldg(reinterpret_cast<const int4*>(nd + 6 * (W / 4)) + h);
            const float4 ax = nx_ ? hix : lox, bx = nx_ ? lox : hix;
            const float4 ay = ny_ ? hiy : loy, by = ny_ ? loy : hiy;
            const float4 az = nz_ ? hiz : loz, bz = nz_ ? loz : hiz;
            const float ax_[4] = {ax.x, ax.y, ax.z, ax.w}, bx_[4] = {bx.x, bx.y, bx.z, bx.w};
            const float ay_[4] = {ay.x, ay.y, ay.z, ay.w}, by_[4] = {by.x, by.y, by.z, by.w};
            const float az_[4] = {az.x, az.y, az.z, az.w}, bz_[4] = {bz.x, bz.y, bz.z, bz.w};
            const int ch_[4] = {ch.x, ch.y, ch.z, ch.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float n0 = fmaf(ax_[q], r.inv.x, -r.oinv.x), f0 = fmaf(bx_[q], r.inv.x, -r.oinv.x);
                const float n1 = fmaf(ay_[q], r.inv.y, -r.oinv.y), f1 = fmaf(by_[q], r.inv.y, -r.oinv.y);
                const float n2 = fmaf(az_[q], r.inv.z, -r.oinv.z), f2 = fmaf(bz_[q], r.inv.z, -r.oinv.z);
                const float tnear = fmaxf(fmaxf(n0, n1), fmaxf(n2, tmin));
                const float tfar = fminf(fminf(f0, f1), fminf(f2, tb));
                tn[4 * h + q] = tnear;
                hit[4 * h + q] = tnear <= tfar;
                child[4 * h + q] = ch_[q];
            }
        }
        // leaves first: they may shrink tb before inner children are queued
#pragma unroll
        for (int c = 0; c < W; ++c) {
            if (hit[c] && child[c] < 0) {
                const int code = ~child[c];
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
        }
        int next = -1;
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
// One primary ray with its bounces: force (y[0..2]) and torque (y[3..5]).
// ---------------------------------------------------------------------------
template <int W>
__device__ __forceinline__ void trace_ray(const DesignDev& dz, const TraceParams& p, int dglob, int sglob,
                                          uint32_t i, float3 o, float3 d, float w, float3 com,
                                          const float* __restrict__ rho, float tmin_b, float y[6],
                                          uint32_t& nvis, uint32_t& ntest, uint32_t& nseg,
                                          int32_t* hits = nullptr) {
    int src = -1;
    float tmin = 0.0f;
    for (int k = 1; k <= p.K; ++k) {
        RaySetup r;
        setup_ray(r, o, d);
        float t;
        ++nseg;
        const int f = closest_hit<W>(dz, r, tmin, src, t, p.err, nvis, ntest);
        if (f < 0) break;
        const float4 a = __ldg(dz.tri + 3 * (size_t)f);
        if (hits) hits[k - 1] = (int32_t)__float_as_uint(a.w);
        const float4 b = __ldg(dz.tri + 3 * (size_t)f + 1);
        const float4 c = __ldg(dz.tri + 3 * (size_t)f + 2);
        float3 n = cross(xyz(b) - xyz(a), xyz(c) - xyz(a));
        n = rsqrtf(dot(n, n)) * n;
        if (dot(n, d) > 0.0f) n = -1.0f * n;
        const float cs = -dot(n, d);
        const int g = (int)__float_as_uint(b.w);
        const float rs = __ldg(rho + 2 * g), rd = __ldg(rho + 2 * g + 1);
        const float3 x = o + t * d;
        const float3 arm = x - com;
        float3 dp;
        if (k == p.K) {
            const float cn = 2.0f * rs * cs + (2.0f / 3.0f) * rd;
            dp = w * ((1.0f - rs) * d - cn * n);
            const float3 tq = cross(arm, dp);
            y[0] += dp.x; y[1] += dp.y; y[2] += dp.z; y[3] += tq.x; y[4] += tq.y; y[5] += tq.z;
            break;
        }
        const uint4 rnd = philox4x32_10(make_uint4(i, (uint32_t)sglob, (uint32_t)dglob, (uint32_t)k),
                                        (uint32_t)p.seed, (uint32_t)(p.seed >> 32));
        float3 dout;
        float wout;
        if (unit24(rnd.x) < 0.5f) {
            dout = d + (2.0f * cs) * n;
            wout = 2.0f * w * rs;
        } else {
            float3 b1, b2;
            onb_f(n, b1, b2);
            const float u1 = unit24(rnd.y), u2 = unit24(rnd.z);
            const float rr = sqrtf(u1);
            float sp, cp;
            sincospif(2.0f * u2, &sp, &cp);
            const float lz = sqrtf(fmaxf(0.0f, 1.0f - u1));
            dout = (rr * cp) * b1 + (rr * sp) * b2 + lz * n;
            wout = 2.0f * w * rd;
        }
        dp = w * d - wout * dout;
        const float3 tq = cross(arm, dp);
        y[0] += dp.x; y[1] += dp.y; y[2] += dp.z; y[3] += tq.x; y[4] += tq.y; y[5] += tq.z;
        o = x; d = dout; w = wout; src = f; tmin = tmin_b;
    }
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// ---------------------------------------------------------------------------
// Trace kernel: blocks loop over units (item, chunk) of this launch.
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(256) trace_kernel(const __grid_constant__ DesignTable tab, const TraceParams p,
                                                    int d0, int Dl) {
    __shared__ double red[8][12];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int64_t units = (int64_t)Dl * p.S * p.cpb;
    for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
        const int64_t item_l = u / p.cpb;
        const int64_t cidx = u % p.cpb;
        const int dl = (int)(item_l / p.S), s = (int)(item_l % p.S);
        const int dg = d0 + dl;
        const DesignDev& dz = tab.d[dl];
        // per-item constants (FP64 set-up, rounded once)
        const double* sp = p.sun + 3 * ((size_t)(p.sun_per_design ? (int64_t)dg * p.S + s : s));
        const double dx_ = -sp[0], dy_ = -sp[1], dz_ = -sp[2];
        const double sgn = dz_ >= 0.0 ? 1.0 : -1.0;
        const double aa = -1.0 / (sgn + dz_);
        const double bb = dx_ * dy_ * aa;
        const double u0 = 1.0 + sgn * dx_ * dx_ * aa, u1 = sgn * bb, u2 = -sgn * dx_;
        const double v0 = bb, v1 = sgn + dy_ * dy_ * aa, v2 = -dy_;
        const double R = dz.R;
        const double pdx = 2.0 * R / p.nx, pdy = 2.0 * R / p.ny;
        const float3 ob = f3((float)(dz.cx - R * u0 - R * v0 - 2.0 * R * dx_),
                             (float)(dz.cy - R * u1 - R * v1 - 2.0 * R * dy_),
                             (float)(dz.cz - R * u2 - R * v2 - 2.0 * R * dz_));
        const float3 bu = f3((float)u0, (float)u1, (float)u2), bv = f3((float)v0, (float)v1, (float)v2);
        const float3 dd = f3((float)dx_, (float)dy_, (float)dz_);
        const float fdx = (float)pdx, fdy = (float)pdy;
        const float w0 = (float)(p.P * pdx * pdy);
        const float3 com = f3((float)p.com[3 * dg], (float)p.com[3 * dg + 1], (float)p.com[3 * dg + 2]);
        const float* rho = p.rho + (size_t)dg * p.G * 2;
        const float tmin_b = (float)(1e-6 * R);
        const int dglob = p.design_base + dg, sglob = p.sun_base + s;

        // per-thread sums: FP32 over up to 32 rays, then flushed into FP64
        double acc[6] = {0, 0, 0, 0, 0, 0}, sq[6] = {0, 0, 0, 0, 0, 0};
        float accf[6] = {0, 0, 0, 0, 0, 0}, sqf[6] = {0, 0, 0, 0, 0, 0};
        uint32_t nvis = 0, ntest = 0, nseg = 0;
        const int64_t k0 = cidx * p.chunk;
        const int64_t k1 = min(k0 + p.chunk, p.n);
        const int64_t span = k1 - k0;
        const int nj = (int)((span + blockDim.x - 1) / blockDim.x);
        for (int j = 0; j < nj; ++j) {
            const int64_t k = k0 + threadIdx.x + (int64_t)j * blockDim.x;
            float y[6] = {0, 0, 0, 0, 0, 0};
            const bool valid = k < k1;
            if (valid) {
                const uint64_t i = (uint64_t)(p.off + k * p.stride);
                const uint32_t px = (uint32_t)(i % (uint64_t)p.nx), py = (uint32_t)(i / (uint64_t)p.nx);
                float xi1 = 0.5f, xi2 = 0.5f;
                if (p.jitter) {
                    const uint4 rnd = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)sglob, (uint32_t)dglob, 0u),
                                                    (uint32_t)p.seed, (uint32_t)(p.seed >> 32));
                    xi1 = unit24(rnd.x); xi2 = unit24(rnd.y);
                }
                const float a = ((float)px + xi1) * fdx, b = ((float)py + xi2) * fdy;
                const float3 o = f3(fmaf(a, bu.x, fmaf(b, bv.x, ob.x)), fmaf(a, bu.y, fmaf(b, bv.y, ob.y)),
                                    fmaf(a, bu.z, fmaf(b, bv.z, ob.z)));
                trace_ray<W>(dz, p, dglob, sglob, (uint32_t)i, o, dd, w0, com, rho, tmin_b, y, nvis, ntest, nseg);
            }
            // collapsed strata: pair rays k (even) and k+1 held by lanes 2m, 2m+1
            const bool pvalid = __shfl_xor_sync(0xffffffffu, (int)valid, 1);
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                const float yo = __shfl_xor_sync(0xffffffffu, y[q], 1);
                accf[q] += y[q];
                if ((lane & 1) == 0 && valid) {
                    const float df = pvalid ? y[q] - yo : y[q];
                    sqf[q] = fmaf(df, df, sqf[q]);
                }
            }
            if ((j & 31) == 31 || j == nj - 1) {
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    acc[q] += (double)accf[q]; sq[q] += (double)sqf[q];
                    accf[q] = 0.0f; sqf[q] = 0.0f;
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 6; ++q) { acc[q] = warp_sum_d(acc[q]); sq[q] = warp_sum_d(sq[q]); }
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < 6; ++q) { red[warp][q] = acc[q]; red[warp][6 + q] = sq[q]; }
        }
        __syncthreads();
        if (threadIdx.x < 12) {
            double t = 0.0;
            for (int wi = 0; wi < nwarp; ++wi) t += red[wi][threadIdx.x];
            p.part[((size_t)(d0 * (int64_t)p.S * p.cpb) + u) * 12 + threadIdx.x] = t;
        }
        if (p.stats) {  // traversal work counters (node visits, triangle tests, segments)
            unsigned long long a = nvis, b = ntest, c = nseg;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                a += __shfl_xor_sync(0xffffffffu, a, off);
                b += __shfl_xor_sync(0xffffffffu, b, off);
                c += __shfl_xor_sync(0xffffffffu, c, off);
            }
            if (lane == 0) { atomicAdd(p.stats, a); atomicAdd(p.stats + 1, b); atomicAdd(p.stats + 2, c); }
        }
        __syncthreads();
    }
}

// Per-ray inspection: one thread per listed ray of one (design, sun).
template <int W>
__global__ void __launch_bounds__(128) trace_rays_kernel(const DesignDev dz, const TraceParams p,
                                                         const int64_t* __restrict__ ray_idx, int64_t nr,
                                                         int sidx, int didx, double* __restrict__ out_y,
                                                         int32_t* __restrict__ out_hits) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nr) return;
    const double dx_ = -p.sun[0], dy_ = -p.sun[1], dz_ = -p.sun[2];
    const double sgn = dz_ >= 0.0 ? 1.0 : -1.0;
    const double aa = -1.0 / (sgn + dz_);
    const double bb = dx_ * dy_ * aa;
    const double u0 = 1.0 + sgn * dx_ * dx_ * aa, u1 = sgn * bb, u2 = -sgn * dx_;
    const double v0 = bb, v1 = sgn + dy_ * dy_ * aa, v2 = -dy_;
    const double R = dz.R;
    const double pdx = 2.0 * R / p.nx, pdy = 2.0 * R / p.ny;
    const float3 ob = f3((float)(dz.cx - R * u0 - R * v0 - 2.0 * R * dx_),
                         (float)(dz.cy - R * u1 - R * v1 - 2.0 * R * dy_),
                         (float)(dz.cz - R * u2 - R * v2 - 2.0 * R * dz_));
    const float3 bu = f3((float)u0, (float)u1, (float)u2), bv = f3((float)v0, (float)v1, (float)v2);
    const float3 dd = f3((float)dx_, (float)dy_, (float)dz_);
    const float w0 = (float)(p.P * pdx * pdy);
    const float3 com = f3((float)p.com[0], (float)p.com[1], (float)p.com[2]);
    const int dglob = p.design_base + didx, sglob = p.sun_base + sidx;
    const uint64_t i = (uint64_t)ray_idx[q];
    const uint32_t px = (uint32_t)(i % (uint64_t)p.nx), py = (uint32_t)(i / (uint64_t)p.nx);
    float xi1 = 0.5f, xi2 = 0.5f;
    if (p.jitter) {
        const uint4 rnd = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)sglob, (uint32_t)dglob, 0u),
                                        (uint32_t)p.seed, (uint32_t)(p.seed >> 32));
        xi1 = unit24(rnd.x); xi2 = unit24(rnd.y);
    }
    const float a = ((float)px + xi1) * (float)pdx, b = ((float)py + xi2) * (float)pdy;
    const float3 o = f3(fmaf(a, bu.x, fmaf(b, bv.x, ob.x)), fmaf(a, bu.y, fmaf(b, bv.y, ob.y)),
                        fmaf(a, bu.z, fmaf(b, bv.z, ob.z)));
    float y[6] = {0, 0, 0, 0, 0, 0};
    int32_t hits[kMaxBounces] = {-1, -1, -1};
    uint32_t nvis = 0, ntest = 0, nseg = 0;
    trace_ray<W>(dz, p, dglob, sglob, (uint32_t)i, o, dd, w0, com, p.rho, (float)(1e-6 * R), y, nvis, ntest, nseg,
                 hits);
    for (int j = 0; j < 6; ++j) out_y[6 * q + j] = (double)y[j];
    for (int k = 0; k < p.K; ++k) out_hits[q * p.K + k] = hits[k];
}

// Sum each item's chunk partials in chunk order -> (F, tau), sigma.
__global__ void reduce_items_kernel(const double* __restrict__ part, int64_t items, int cpb,
                                    double* __restrict__ out_ft, double* __restrict__ out_sigma) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= items * 12) return;
    const int64_t item = gid / 12;
    const int q = (int)(gid % 12);
    double t = 0.0;
    for (int c = 0; c < cpb; ++c) t += part[((size_t)item * cpb + c) * 12 + q];
    if (q < 6) out_ft[item * 6 + q] = t;
    else if (out_sigma) out_sigma[item * 6 + (q - 6)] = sqrt(t);
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
template <int W>
static cudaError_t launch_w(const DesignTable& tab, const TraceParams& p, int d0, int Dl, int grid, int block,
                            cudaStream_t st) {
    trace_kernel<W><<<grid, block, 0, st>>>(tab, p, d0, Dl);
    return cudaGetLastError();
}

int trace_resident_blocks(int width, int block) {
    int nb = 0;
    if (width == 8)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, trace_kernel<8>, block, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, trace_kernel<4>, block, 0);
    return nb > 0 ? nb : 1;
}

cudaError_t launch_trace(const std::vector<DesignDev>& designs, const TraceParams& p, int width, int grid_cap,
                         int block, cudaStream_t st) {
    const int D = (int)designs.size();
    for (int d0 = 0; d0 < D; d0 += kMaxDesignsPerLaunch) {
        const int Dl = std::min(kMaxDesignsPerLaunch, D - d0);
        DesignTable tab;
        for (int k = 0; k < Dl; ++k) tab.d[k] = designs[d0 + k];
        const int64_t units = (int64_t)Dl * p.S * p.cpb;
        const int grid = (int)std::min<int64_t>(units, grid_cap);
        cudaError_t e = width == 8 ? launch_w<8>(tab, p, d0, Dl, grid, block, st)
                                   : launch_w<4>(tab, p, d0, Dl, grid, block, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_trace_rays(const DesignDev& dz, const TraceParams& p, const int64_t* ray_idx, int64_t nr,
                              int sidx, int didx, double* out_y, int32_t* out_hits, cudaStream_t st) {
    if (nr <= 0) return cudaSuccess;
    const int bs = 128;
    const unsigned grid = (unsigned)((nr + bs - 1) / bs);
    if (dz.width == 8)
        trace_rays_kernel<8><<<grid, bs, 0, st>>>(dz, p, ray_idx, nr, sidx, didx, out_y, out_hits);
    else
        trace_rays_kernel<4><<<grid, bs, 0, st>>>(dz, p, ray_idx, nr, sidx, didx, out_y, out_hits);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const double* part, int64_t items, int cpb, double* out_ft, double* out_sigma,
                          cudaStream_t st) {
    const int64_t n = items * 12;
    const int bs = 256;
    const int64_t grid = (n + bs - 1) / bs;
    reduce_items_kernel<<<(unsigned)grid, bs, 0, st>>>(part, items, cpb, out_ft, out_sigma);
    return cudaGetLastError();
}

}  // namespace srp
