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

// Primary segment of grid ray i (jittered pixel origin, travel direction d).
__device__ __forceinline__ Seg primary_seg(const ItemConst& ic, const TraceParams& p, uint64_t i) {
    const uint32_t px = (uint32_t)(i % (uint64_t)p.nx), py = (uint32_t)(i / (uint64_t)p.nx);
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

// Momentum deposit of hit k (1-based) on leaf-order triangle f at ray
// parameter t; returns true (and the outgoing segment) if the path goes on.
__device__ __forceinline__ bool shade_hit(const DesignDev& dz, const ItemConst& ic, const TraceParams& p,
                                          uint32_t i, int k, int f, float t, const Seg& s, float y[6],
                                          Seg& out) {
    const float4 a = __ldg(dz.tri + 3 * (size_t)f);
    const float4 b = __ldg(dz.tri + 3 * (size_t)f + 1);
    const float4 c = __ldg(dz.tri + 3 * (size_t)f + 2);
    float3 n = cross(xyz(b) - xyz(a), xyz(c) - xyz(a));
    n = rsqrtf(dot(n, n)) * n;
    if (dot(n, s.d) > 0.0f) n = -1.0f * n;
    const float cs = -dot(n, s.d);
    const int g = (int)__float_as_uint(b.w);
    const float rs = __ldg(ic.rho + 2 * g), rd = __ldg(ic.rho + 2 * g + 1);
    const float3 x = s.o + t * s.d;
    const float3 arm = x - ic.com;
    if (k == p.K) {
        const float cn = 2.0f * rs * cs + (2.0f / 3.0f) * rd;
        const float3 dp = s.w * ((1.0f - rs) * s.d - cn * n);
        const float3 tq = cross(arm, dp);
        y[0] += dp.x; y[1] += dp.y; y[2] += dp.z; y[3] += tq.x; y[4] += tq.y; y[5] += tq.z;
        return false;
    }
    const uint4 rnd = philox4x32_10(make_uint4(i, (uint32_t)ic.sglob, (uint32_t)ic.dglob, (uint32_t)k),
                                    (uint32_t)p.seed, (uint32_t)(p.seed >> 32));
    float3 dout;
    float wout;
    if (unit24(rnd.x) < 0.5f) {
        dout = s.d + (2.0f * cs) * n;
        wout = 2.0f * s.w * rs;
    } else {
        // Lambertian: direction of n + (uniform unit vector), pdf cos/pi
        const float z = 1.0f - 2.0f * unit24(rnd.y);
        const float rr = sqrtf(fmaxf(0.0f, 1.0f - z * z));
        float sp, cp;
        sincospif(2.0f * unit24(rnd.z), &sp, &cp);
        const float3 v = f3(n.x + rr * cp, n.y + rr * sp, n.z + z);
        const float l2 = dot(v, v);
        dout = l2 > 0.0f ? rsqrtf(l2) * v : n;
        wout = 2.0f * s.w * rd;
    }
    const float3 dp = s.w * s.d - wout * dout;
    const float3 tq = cross(arm, dp);
    y[0] += dp.x; y[1] += dp.y; y[2] += dp.z; y[3] += tq.x; y[4] += tq.y; y[5] += tq.z;
    out.o = x; out.d = dout; out.w = wout; out.src = f;
    return true;
}

// Whole path of one ray in one thread (used by the per-ray inspection).
template <int W>
__device__ __forceinline__ void trace_path(const DesignDev& dz, const ItemConst& ic, const TraceParams& p,
                                           uint32_t i, Seg s, float y[6], uint32_t& nvis, uint32_t& ntest,
                                           uint32_t& nseg, int32_t* hits) {
    for (int k = 1; k <= p.K; ++k) {
        RaySetup r;
        setup_ray(r, s.o, s.d);
        float t;
        ++nseg;
        const int f = closest_hit<W>(dz, r, k == 1 ? 0.0f : ic.tmin_b, s.src, t, p.err, nvis, ntest);
        if (f < 0) break;
        if (hits) hits[k - 1] = (int32_t)__float_as_uint(__ldg(dz.tri + 3 * (size_t)f).w);
        Seg nx;
        if (!shade_hit(dz, ic, p, i, k, f, t, s, y, nx)) break;
        s = nx;
    }
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// ---------------------------------------------------------------------------
// Trace kernel: a warp-level wavefront.  Every warp is an independent worker
// looping over units (item, chunk) with a static stride; a unit's rays are
// processed in tiles of 32*kBatches rays:
//   primary batches  the warp traces 32 neighbouring pixels at a time
//                    (coherent parallel rays share node fetches); each
//                    ray's deposit goes to its slot in shared memory and
//                    paths that continue are pushed on the warp's queue;
//   bounce batches   whenever 32 segments are queued, all 32 lanes trace
//                    them together; the tile's last segments are drained
//                    at its end;
//   tile reduce      per-ray sums -> per-lane FP32 partials (lane pairs
//                    give the collapsed-strata variance) -> FP64.
// Only __syncwarp is needed inside a unit.  Each ray's arithmetic and
// deposit order (bounce 1, 2, 3) are those of trace_path.
// ---------------------------------------------------------------------------
constexpr int kBatches = 8;               // primary batches of 32 rays per tile
constexpr int kTile = 32 * kBatches;      // rays per warp tile
constexpr int kQueue = 64;                // bounce segments per warp (<= 31 + 32 live)
constexpr int kWarpsPerBlock = 4;

struct WarpSmem {
    float ys[6][kTile];        // per-ray force/torque sums of the tile
    float4 qa[kQueue];         // (o.xyz, w)
    float4 qb[kQueue];         // (d.xyz, src)
    int qs[kQueue];            // slot | (bounce << 16)
    double dacc[12][32];       // per-lane FP64 sums (force, torque, squared pair differences)
};

__host__ __device__ constexpr size_t trace_smem_bytes(int block) {
    return (size_t)(block / 32) * sizeof(WarpSmem);
}

// Append the segments of lanes with `want` to the warp queue.
__device__ __forceinline__ void q_push(WarpSmem& ws, int& qcount, bool want, const Seg& s, int slot, int kb,
                                       int lane) {
    const unsigned m = __ballot_sync(0xffffffffu, want);
    if (want) {
        const int pos = qcount + __popc(m & ((1u << lane) - 1u));
        ws.qa[pos] = make_float4(s.o.x, s.o.y, s.o.z, s.w);
        ws.qb[pos] = make_float4(s.d.x, s.d.y, s.d.z, __int_as_float(s.src));
        ws.qs[pos] = slot | (kb << 16);
    }
    qcount += __popc(m);
    __syncwarp();
}

template <int W>
__global__ void __launch_bounds__(128, 4) trace_kernel(const __grid_constant__ DesignTable tab, const TraceParams p,
                                                       int d0, int Dl) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpSmem& ws = reinterpret_cast<WarpSmem*>(smem)[warp];
    const int64_t units = (int64_t)Dl * p.S * p.cpb;
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    uint32_t nvis = 0, ntest = 0, nseg = 0;
    for (int64_t u = gw; u < units; u += nw) {
        const int64_t item_l = u / p.cpb;
        const int64_t cidx = u % p.cpb;
        const int dl = (int)(item_l / p.S), s = (int)(item_l % p.S);
        const int dg = d0 + dl;
        const DesignDev& dz = tab.d[dl];
        ItemConst ic;
        item_setup(ic, dz, p, p.sun + 3 * ((size_t)(p.sun_per_design ? (int64_t)dg * p.S + s : s)), p.com + 3 * dg,
                   p.rho + (size_t)dg * p.G * 2, p.design_base + dg, p.sun_base + s);
#pragma unroll
        for (int q = 0; q < 12; ++q) ws.dacc[q][lane] = 0.0;
        const int64_t k0 = cidx * p.chunk;
        const int64_t k1 = min(k0 + p.chunk, p.n);
        int qcount = 0;
        for (int64_t ts = k0; ts < k1; ts += kTile) {
#pragma unroll
            for (int j = 0; j < kBatches; ++j)
#pragma unroll
                for (int q = 0; q < 6; ++q) ws.ys[q][j * 32 + lane] = 0.0f;
            __syncwarp();
            // ---- one work loop, one trace site: each iteration the warp takes
            // 32 queued bounce segments if there are that many, else the next
            // batch of 32 primary rays, else the remaining queued segments.
            int next_batch = 0;
#pragma unroll 1
            while (true) {
                int nb;
                const bool primary = qcount < 32 && next_batch < kBatches;
                if (primary) nb = 32;
                else if (qcount > 0) nb = min(qcount, 32);
                else break;
                bool has;
                Seg sg;
                int slot, kb;
                uint64_t i = 0;
                if (primary) {
                    slot = next_batch * 32 + lane;
                    const int64_t k = ts + slot;
                    has = k < k1;
                    kb = 1;
                    if (has) {
                        i = (uint64_t)(p.off + k * p.stride);
                        sg = primary_seg(ic, p, i);
                    }
                    ++next_batch;
                } else {
                    has = lane < nb;
                    slot = 0; kb = 0;
                    if (has) {
                        const int e = qcount - 1 - lane;
                        const float4 A = ws.qa[e], Bv = ws.qb[e];
                        const int q = ws.qs[e];
                        sg.o = f3(A.x, A.y, A.z); sg.w = A.w;
                        sg.d = f3(Bv.x, Bv.y, Bv.z); sg.src = __float_as_int(Bv.w);
                        slot = q & 0xffff; kb = q >> 16;
                        i = (uint64_t)(p.off + (ts + slot) * p.stride);
                    }
                    __syncwarp();
                    qcount -= nb;
                }
                bool cont = false;
                Seg nx;
                if (has) {
                    RaySetup rs;
                    setup_ray(rs, sg.o, sg.d);
                    float t;
                    ++nseg;
                    const int f = closest_hit<W>(dz, rs, kb == 1 ? 0.0f : ic.tmin_b, sg.src, t, p.err, nvis, ntest);
                    if (f >= 0) {
                        float y[6];
#pragma unroll
                        for (int q = 0; q < 6; ++q) y[q] = ws.ys[q][slot];
                        cont = shade_hit(dz, ic, p, (uint32_t)i, kb, f, t, sg, y, nx);
#pragma unroll
                        for (int q = 0; q < 6; ++q) ws.ys[q][slot] = y[q];
                    }
                }
                q_push(ws, qcount, cont, nx, slot, kb + 1, lane);
            }
            // ---- per-ray sums -> per-lane partials (slot parity = ray parity)
            float accf[6] = {0, 0, 0, 0, 0, 0}, sqf[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
            for (int j = 0; j < kBatches; ++j) {
                const int slot = j * 32 + lane;
                const bool valid = ts + slot < k1;
                const bool pvalid = __shfl_xor_sync(0xffffffffu, (int)valid, 1);
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    const float y = ws.ys[q][slot];
                    const float yo = __shfl_xor_sync(0xffffffffu, y, 1);
                    accf[q] += y;
                    if ((lane & 1) == 0 && valid) {
                        const float df = pvalid ? y - yo : y;
                        sqf[q] = fmaf(df, df, sqf[q]);
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                ws.dacc[q][lane] += (double)accf[q];
                ws.dacc[6 + q][lane] += (double)sqf[q];
            }
            __syncwarp();
        }
        // warp reduction in a fixed order -> the unit's partial
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            const double v = warp_sum_d(ws.dacc[q][lane]);
            if (lane == q) p.part[((size_t)(d0 * (int64_t)p.S * p.cpb) + u) * 12 + q] = v;
        }
        __syncwarp();
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
}

// Per-ray inspection: one thread per listed ray of one (design, sun).
template <int W>
__global__ void __launch_bounds__(128) trace_rays_kernel(const DesignDev dz, const TraceParams p,
                                                         const int64_t* __restrict__ ray_idx, int64_t nr,
                                                         int sidx, int didx, double* __restrict__ out_y,
                                                         int32_t* __restrict__ out_hits) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nr) return;
    ItemConst ic;
    item_setup(ic, dz, p, p.sun, p.com, p.rho, p.design_base + didx, p.sun_base + sidx);
    const uint64_t i = (uint64_t)ray_idx[q];
    float y[6] = {0, 0, 0, 0, 0, 0};
    int32_t hits[kMaxBounces] = {-1, -1, -1};
    uint32_t nvis = 0, ntest = 0, nseg = 0;
    trace_path<W>(dz, ic, p, (uint32_t)i, primary_seg(ic, p, i), y, nvis, ntest, nseg, hits);
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
    const size_t sm = trace_smem_bytes(block);
    cudaError_t e = cudaFuncSetAttribute(trace_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    trace_kernel<W><<<grid, block, sm, st>>>(tab, p, d0, Dl);
    return cudaGetLastError();
}

int trace_resident_blocks(int width, int block) {
    int nb = 0;
    const size_t sm = trace_smem_bytes(block);
    if (width == 8) {
        cudaFuncSetAttribute(trace_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, trace_kernel<8>, block, sm);
    } else {
        cudaFuncSetAttribute(trace_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, trace_kernel<4>, block, sm);
    }
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
        const int64_t wpb = block / 32;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((units + wpb - 1) / wpb, grid_cap));
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
