// area.cu -- the paper's own estimator without bounces (Sec. 3.2
// "Estimation", the "NB" variant of Table 3) for sm_103a.
//
// For every (design, sun) item: surface samples are spread over the
// triangles by area (triangle f gets n_f = max(1, ceil(density * A_f))
// samples, A_f and the product in FP32 with every operation rounded), a
// sample is a uniform point on its triangle (Osada et al. 2002 square-root
// mapping of two Philox4x32-10 uniforms), and next-event estimation toward
// the sun decides whether it is lit: an any-hit shadow ray from the point
// along e through the design's BVH.  A lit sample deposits the expected
// momentum of the facet BRDF,
//   (A_f / n_f) P cos [(1 - rs) d - (2 rs cos + 2/3 rd) n],   d = -e,
// and its torque about the centre of mass.  Samples are numbered
// k = prefix(f) + j in original triangle order; sigma is the collapsed-strata
// estimate over the pairs (2i, 2i + 1).
//
// Kernels:
//   area_prep_kernel   per (design, leaf slot): FP32 area, n_f, leaf map
//   area_scan_kernel   per design: exclusive prefix of n_f (one block)
//   area_kernel<W>     persistent warps over (item, chunk) units taken from
//                      an atomic queue; a lane owns one sample at a time,
//                      finds its triangle by binary search of the prefix,
//                      draws the point and traces the shadow ray; per-lane
//                      FP32 sums of 32 samples, FP32 warp tree, FP64 unit
//                      sums -> partials
// and the ray-grid tracer's reduce kernel sums the partials of each item.
//
// Interreflection mode (max_bounces = 2): each sample also gathers one
// Lambertian interreflection per side of its facet -- a cosine-sampled
// incoming direction, its closest hit y, next-event estimation at y -- and
// deposits the light y reflects toward it by its own facet BRDF (the
// indirect term of the paper's estimator, diffuse part).
//
// Thermal mode (Sec. 5.9, local Lambertian emitters): only triangles of
// groups with emit > 0 get samples; a sample's packet carries
// w = P emit A_f / n_f, recoils by its expectation -(2/3) w n_e at x (n_e the
// winding normal, the emitting side), leaves along unit(n_e + uniform unit
// vector) (cosine-distributed) and deposits the closed-form facet-BRDF
// momentum w[(1-rs) omega - (2 rs cos + 2/3 rd) n] at its closest hit.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "trace_common.cuh"

namespace srp {


constexpr int kAreaTile = 1024;   // samples per FP32 tile of a warp (32 per lane)

// FP32 area of a triangle, every operation rounded (no contraction).
__device__ __forceinline__ float tri_area_rn(float4 a, float4 b, float4 c) {
    const float e1x = __fsub_rn(b.x, a.x), e1y = __fsub_rn(b.y, a.y), e1z = __fsub_rn(b.z, a.z);
    const float e2x = __fsub_rn(c.x, a.x), e2y = __fsub_rn(c.y, a.y), e2z = __fsub_rn(c.z, a.z);
    const float cx = __fsub_rn(__fmul_rn(e1y, e2z), __fmul_rn(e1z, e2y));
    const float cy = __fsub_rn(__fmul_rn(e1z, e2x), __fmul_rn(e1x, e2z));
    const float cz = __fsub_rn(__fmul_rn(e1x, e2y), __fmul_rn(e1y, e2x));
    float s = __fmul_rn(cx, cx);
    s = __fadd_rn(s, __fmul_rn(cy, cy));
    s = __fadd_rn(s, __fmul_rn(cz, cz));
    return __fmul_rn(0.5f, __fsqrt_rn(s));
}

__global__ void __launch_bounds__(256) area_prep_kernel(const AreaParams p, int d0) {
    const int d = d0 + (int)blockIdx.y;
    const DesignDev dz = p.designs[d];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= dz.T) return;
    const float4 a = __ldg(dz.tri + 3 * (size_t)k), b = __ldg(dz.tri + 3 * (size_t)k + 1),
                 c = __ldg(dz.tri + 3 * (size_t)k + 2);
    const uint32_t f = __float_as_uint(a.w);
    if (f >= (uint32_t)dz.T) { atomicOr(p.err, kErrTriIndex); return; }
    const int64_t base = p.xbase[d];
    if (p.mode == 1) {
        const uint32_t g = __float_as_uint(b.w);
        if (!(g < (uint32_t)p.G && p.emit[(size_t)d * p.G + g] > 0.0f)) {
            p.cnt[base + f] = 0;
            p.map[base + f] = k;
            return;
        }
    }
    const float prod = __fmul_rn(p.density, tri_area_rn(a, b, c));
    int32_t n = 1;
    if (prod > 1.0f) {
        if (!(prod < 1.0e9f)) { atomicOr(p.err, kErrAreaCount); n = 1; }
        else n = (int32_t)ceilf(prod);
    }
    p.cnt[base + f] = n;
    p.map[base + f] = k;
}

// One block of 1024 threads per design: thread t scans a contiguous run of
// triangles; a block-wide scan of the run totals gives each run's offset.
__global__ void __launch_bounds__(1024) area_scan_kernel(const AreaParams p) {
    __shared__ long long wsum[32];
    const int d = blockIdx.x;
    const int T = p.designs[d].T;
    const int64_t base = p.xbase[d];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int run = (T + 1023) / 1024;
    const int t0 = min(T, tid * run), t1 = min(T, t0 + run);
    long long loc = 0;
    for (int f = t0; f < t1; ++f) loc += p.cnt[base + f];
    // inclusive warp scan, then scan of warp totals
    long long v = loc;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const long long o = __shfl_up_sync(0xffffffffu, v, off);
        if (lane >= off) v += o;
    }
    if (lane == 31) wsum[warp] = v;
    __syncthreads();
    if (warp == 0) {
        long long w = wsum[lane];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const long long o = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += o;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    long long run_off = v - loc + (warp > 0 ? wsum[warp - 1] : 0);
    const long long total = wsum[31];
    const bool over = total > p.cap || total > 0x7fffffffLL;
    for (int f = t0; f < t1; ++f) {
        p.ex[base + f] = over ? 0 : (int32_t)run_off;
        run_off += p.cnt[base + f];
    }
    if (tid == 0) {
        p.ex[base + T] = over ? 0 : (int32_t)total;
        p.ntot[d] = over ? 0 : total;
        if (over) atomicOr(p.err, kErrAreaCount);
    }
}

// Triangle of sample k: the largest f with ex[f] <= k (binary search).
__device__ __forceinline__ int find_tri(const int32_t* __restrict__ ex, int lo, int hi, int32_t k) {
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(ex + mid) <= k) lo = mid; else hi = mid;
    }
    return lo;
}

// One gathered Lambertian interreflection at x (leaf triangle L, side
// normal ns) along omega = unit(ns + uniform unit vector(ua, ub)): the
// closest hit y, y's side m facing x lit when m.e > 0 and its shadow ray
// along e is free; then irradiance E = rd_y P (m.e) arrives at x along
// -omega (cosine sampling cancels the 1/pi of the Lambertian radiance) and
// x deposits (A/n) E [(1 - rs)(-omega) - (2 rs cos + 2/3 rd) ns],
// cos = omega.ns, by its own facet BRDF.
template <int W>
__device__ __forceinline__ void gather_diffuse(const DesignDev& dz, int L, float3 x, float3 ns, float ua, float ub,
                                               float wA, float rs, float rd, float3 e, const RaySetup& rset,
                                               float3 com, const float* rho, float tmin, float P, int* err,
                                               float y[6], uint32_t& nvis, uint32_t& ntest, uint32_t& nseg) {
    const float z = 1.0f - 2.0f * ua;
    const float rr = sqrtf(fmaxf(0.0f, 1.0f - z * z));
    float sp, cp;
    sincospif(2.0f * ub, &sp, &cp);
    const float3 v = f3(ns.x + rr * cp, ns.y + rr * sp, ns.z + z);
    const float l2 = dot(v, v);
    if (!(l2 > 0.0f)) return;
    const float3 om = rsqrtf(l2) * v;
    RaySetup r;
    setup_ray(r, x, om);
    ++nseg;
    float t;
    const int h = closest_hit<W>(dz, r, tmin, L, t, err, nvis, ntest);
    if (h < 0) return;
    const float4 ha = __ldg(dz.tri + 3 * (size_t)h), hb = __ldg(dz.tri + 3 * (size_t)h + 1),
                 hc = __ldg(dz.tri + 3 * (size_t)h + 2);
    float3 m = cross(xyz(hb) - xyz(ha), xyz(hc) - xyz(ha));
    m = rsqrtf(dot(m, m)) * m;
    if (dot(m, om) > 0.0f) m = -1.0f * m;
    const float ce = dot(m, e);
    if (!(ce > 0.0f)) return;
    const float3 yp = x + t * om;
    RaySetup rs2 = rset;
    rs2.o = yp;
    rs2.oinv = f3(yp.x * rs2.inv.x, yp.y * rs2.inv.y, yp.z * rs2.inv.z);
    ++nseg;
    if (any_hit<W>(dz, rs2, tmin, h, err, nvis, ntest)) return;
    const int gh = (int)__float_as_uint(hb.w);
    const float E = __ldg(rho + 2 * gh + 1) * P * ce;
    const float cs = dot(om, ns);
    const float cn = 2.0f * rs * cs + (2.0f / 3.0f) * rd;
    const float a1 = wA * E * (1.0f - rs), a2 = wA * E * cn;
    const float3 dp = f3(-a1 * om.x - a2 * ns.x, -a1 * om.y - a2 * ns.y, -a1 * om.z - a2 * ns.z);
    const float3 tq = cross(x - com, dp);
    y[0] += dp.x; y[1] += dp.y; y[2] += dp.z; y[3] += tq.x; y[4] += tq.y; y[5] += tq.z;
}

// One sun-light sample: point on leaf triangle L (original index f, sample
// jj of nf), shadow ray along e, expected BRDF momentum if lit; with IND,
// one gathered Lambertian interreflection on each side of the facet (side
// +n_e from (u3, u4) of the sample's counter, side -n_e from the counter
// with bit 28 of the design word set).
// rset: setup_ray of the item's shadow direction e (origin 0): its 1/e and
// shear rows serve every sample of the item; only o/e is per sample.
template <int W, bool IND>
__device__ __forceinline__ void sample_sun(const DesignDev& dz, int L, int f, uint32_t jj, int32_t nf, float3 e,
                                           const RaySetup& rset, float3 com, const float* rho, float tmin, uint32_t sg,
                                           uint32_t dg, uint32_t key0, uint32_t key1, float P, int* err, float y[6],
                                           uint32_t& nvis, uint32_t& ntest, uint32_t& nseg) {
    const float4 a = __ldg(dz.tri + 3 * (size_t)L), b = __ldg(dz.tri + 3 * (size_t)L + 1),
                 c = __ldg(dz.tri + 3 * (size_t)L + 2);
    const float3 e1 = xyz(b) - xyz(a), e2 = xyz(c) - xyz(a);
    float3 ne = cross(e1, e2);
    const float len = sqrtf(dot(ne, ne));
    ne = (1.0f / len) * ne;
    float3 n = ne;
    float cs = dot(n, e);
    if (cs < 0.0f) { n = -1.0f * n; cs = -cs; }
    if (!IND && !(cs > 0.0f)) return;
    const uint4 rnd = philox4x32_10(make_uint4(jj, (uint32_t)f, sg, dg), key0, key1);
    const float u1 = unit24(rnd.x), u2 = unit24(rnd.y);
    const float sr = sqrtf(u1);
    const float b1 = sr * (1.0f - u2), b2 = sr * u2;
    const float3 x = f3(fmaf(b2, e2.x, fmaf(b1, e1.x, a.x)), fmaf(b2, e2.y, fmaf(b1, e1.y, a.y)),
                        fmaf(b2, e2.z, fmaf(b1, e1.z, a.z)));
    const int g = (int)__float_as_uint(b.w);
    const float rs = __ldg(rho + 2 * g), rd = __ldg(rho + 2 * g + 1);
    if (cs > 0.0f) {
        RaySetup r = rset;
        r.o = x;
        r.oinv = f3(x.x * r.inv.x, x.y * r.inv.y, x.z * r.inv.z);
        ++nseg;
        if (!any_hit<W>(dz, r, tmin, L, err, nvis, ntest)) {
            const float wgt = P * (0.5f * len) / (float)nf;
            const float cn = 2.0f * rs * cs + (2.0f / 3.0f) * rd;
            const float ws = wgt * cs, a1 = ws * (1.0f - rs), a2 = ws * cn;
            const float3 dp = f3(-a1 * e.x - a2 * n.x, -a1 * e.y - a2 * n.y, -a1 * e.z - a2 * n.z);
            const float3 tq = cross(x - com, dp);
            y[0] = dp.x; y[1] = dp.y; y[2] = dp.z; y[3] = tq.x; y[4] = tq.y; y[5] = tq.z;
        }
    }
    if (IND) {
        const float wA = (0.5f * len) / (float)nf;
        gather_diffuse<W>(dz, L, x, ne, unit24(rnd.z), unit24(rnd.w), wA, rs, rd, e, rset, com, rho, tmin, P, err, y,
                          nvis, ntest, nseg);
        const uint4 rnd2 = philox4x32_10(make_uint4(jj, (uint32_t)f, sg, dg | 0x10000000u), key0, key1);
        gather_diffuse<W>(dz, L, x, -1.0f * ne, unit24(rnd2.x), unit24(rnd2.y), wA, rs, rd, e, rset, com, rho, tmin,
                          P, err, y, nvis, ntest, nseg);
    }
}

// One thermal packet of leaf triangle L: expected recoil at the point, and
// the closed-form deposit at the closest hit of its cosine-distributed ray.
template <int W>
__device__ __forceinline__ void sample_thermal(const DesignDev& dz, int L, int f, uint32_t jj, int32_t nf,
                                               float3 com, const float* rho, const float* emit, float tmin,
                                               uint32_t dg, uint32_t key0, uint32_t key1, float P, int* err,
                                               float y[6], uint32_t& nvis, uint32_t& ntest, uint32_t& nseg) {
    const float4 a = __ldg(dz.tri + 3 * (size_t)L), b = __ldg(dz.tri + 3 * (size_t)L + 1),
                 c = __ldg(dz.tri + 3 * (size_t)L + 2);
    const float3 e1 = xyz(b) - xyz(a), e2 = xyz(c) - xyz(a);
    float3 ne = cross(e1, e2);
    const float len = sqrtf(dot(ne, ne));
    ne = (1.0f / len) * ne;
    const int g = (int)__float_as_uint(b.w);
    const float w = P * __ldg(emit + g) * (0.5f * len) / (float)nf;
    const uint4 rnd = philox4x32_10(make_uint4(jj, (uint32_t)f, 0u, dg), key0, key1);
    const float sr = sqrtf(unit24(rnd.x)), u2 = unit24(rnd.y);
    const float b1 = sr * (1.0f - u2), b2 = sr * u2;
    const float3 x = f3(fmaf(b2, e2.x, fmaf(b1, e1.x, a.x)), fmaf(b2, e2.y, fmaf(b1, e1.y, a.y)),
                        fmaf(b2, e2.z, fmaf(b1, e1.z, a.z)));
    const float wr = -(2.0f / 3.0f) * w;
    const float3 rc = wr * ne;
    const float3 tr = cross(x - com, rc);
    y[0] = rc.x; y[1] = rc.y; y[2] = rc.z; y[3] = tr.x; y[4] = tr.y; y[5] = tr.z;
    const float z = 1.0f - 2.0f * unit24(rnd.z);
    const float rr = sqrtf(fmaxf(0.0f, 1.0f - z * z));
    float sp, cp;
    sincospif(2.0f * unit24(rnd.w), &sp, &cp);
    const float3 v = f3(ne.x + rr * cp, ne.y + rr * sp, ne.z + z);
    const float l2 = dot(v, v);
    if (!(l2 > 0.0f)) return;
    const float3 om = rsqrtf(l2) * v;
    RaySetup r;
    setup_ray(r, x, om);
    ++nseg;
    float t;
    const int h = closest_hit<W>(dz, r, tmin, L, t, err, nvis, ntest);
    if (h < 0) return;
    const float4 ha = __ldg(dz.tri + 3 * (size_t)h), hb = __ldg(dz.tri + 3 * (size_t)h + 1),
                 hc = __ldg(dz.tri + 3 * (size_t)h + 2);
    float3 n = cross(xyz(hb) - xyz(ha), xyz(hc) - xyz(ha));
    n = rsqrtf(dot(n, n)) * n;
    if (dot(n, om) > 0.0f) n = -1.0f * n;
    const float cs = -dot(n, om);
    const int gh = (int)__float_as_uint(hb.w);
    const float rs = __ldg(rho + 2 * gh), rd = __ldg(rho + 2 * gh + 1);
    const float cn = 2.0f * rs * cs + (2.0f / 3.0f) * rd;
    const float a1 = w * (1.0f - rs), a2 = w * cn;
    const float3 dp = f3(a1 * om.x - a2 * n.x, a1 * om.y - a2 * n.y, a1 * om.z - a2 * n.z);
    const float3 yh = x + t * om;
    const float3 tq = cross(yh - com, dp);
    y[0] += dp.x; y[1] += dp.y; y[2] += dp.z; y[3] += tq.x; y[4] += tq.y; y[5] += tq.z;
}

template <int W, int MINB, int MODE>
__global__ void __launch_bounds__(128, MINB) area_kernel(const AreaParams p) {
    __shared__ double dacc[4][12];
    __shared__ float lacc[4][12][32];   // per-lane FP32 sums of a tile (kept out of registers)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t units = (int64_t)p.D * p.S * p.cpd;
    uint32_t nvis = 0, ntest = 0, nseg = 0;
    const uint32_t key0 = (uint32_t)p.seed, key1 = (uint32_t)(p.seed >> 32);
    while (true) {
        unsigned long long uq = 0;
        if (lane == 0) uq = atomicAdd(p.queue, 1ull);
        const int64_t u = (int64_t)__shfl_sync(0xffffffffu, uq, 0);
        if (u >= units) break;
        const int64_t item = u / p.cpd;
        const int64_t cidx = u % p.cpd;
        const int dl = (int)(item / p.S), s = (int)(item % p.S);
        const DesignDev dz = p.designs[dl];
        const int64_t base = p.xbase[dl];
        const int32_t N = (int32_t)p.ntot[dl];
        const int32_t k0 = (int32_t)min(cidx * p.chunk, (int64_t)N);
        const int32_t k1 = (int32_t)min(cidx * p.chunk + p.chunk, (int64_t)N);
        if (lane < 12) dacc[warp][lane] = 0.0;
        __syncwarp();
        if (k0 < k1) {
            float3 e = f3(0.0f, 0.0f, 1.0f);
            if (MODE != 1) {
                const double* sp = p.sun + 3 * (size_t)(p.sun_per_design ? (int64_t)dl * p.S + s : s);
                e = f3((float)sp[0], (float)sp[1], (float)sp[2]);
            }
            const float* emit = MODE == 1 ? p.emit + (size_t)dl * p.G : nullptr;
            RaySetup rset;
            setup_ray(rset, f3(0.0f, 0.0f, 0.0f), e);
            const double* cp = p.com + 3 * (size_t)dl;
            const float3 com = f3((float)cp[0], (float)cp[1], (float)cp[2]);
            const float* rho = p.rho + (size_t)dl * p.G * 2;
            const float tmin = (float)(1e-6 * dz.R);
            const uint32_t sg = (uint32_t)(p.sun_base + s);
            const uint32_t dg = (uint32_t)(p.design_base + dl) | (MODE != 1 ? 0x80000000u : 0x40000000u);
            const int32_t* __restrict__ ex = p.ex + base;
            const int32_t* __restrict__ map = p.map + base;
            const int T = dz.T;
            // triangle of the first sample of the current group of 32 (warp-uniform)
            int f_base = find_tri(ex, 0, T, k0);
            for (int32_t ts = k0; ts < k1; ts += kAreaTile) {
#pragma unroll
                for (int q = 0; q < 12; ++q) lacc[warp][q][lane] = 0.0f;
#pragma unroll 1
                for (int j = 0; j < 32 && ts + 32 * j < k1; ++j) {
                    const int32_t k = ts + 32 * j + lane;
                    const bool valid = k < k1;
                    // window of 33 prefix entries from f_base: lane i holds ex[f_base + i]
                    const int fi = f_base + lane;
                    const int32_t wl = fi <= T ? __ldg(ex + fi) : 0x7fffffff;
                    const int32_t w32 = f_base + 32 <= T ? __ldg(ex + f_base + 32) : 0x7fffffff;
                    const int32_t kk = valid ? k : k1 - 1;
                    int lo = 0;
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1) {
                        const int32_t wv = __shfl_sync(0xffffffffu, wl, lo + step);
                        if (wv <= kk) lo += step;
                    }
                    const int32_t ex_f = __shfl_sync(0xffffffffu, wl, lo);
                    const int32_t nxt = __shfl_sync(0xffffffffu, wl, min(lo + 1, 31));
                    int f = f_base + lo;
                    int32_t ex_lo = ex_f, ex_hi = lo == 31 ? w32 : nxt;
                    if (kk >= ex_hi) {  // the group spans more than 32 triangles
                        f = find_tri(ex, f_base + 32, T, kk);
                        ex_lo = __ldg(ex + f);
                        ex_hi = __ldg(ex + f + 1);
                    }
                    f_base = __shfl_sync(0xffffffffu, f, 31);
                    float y[6] = {0, 0, 0, 0, 0, 0};
                    if (valid) {
                        const uint32_t jj = (uint32_t)(k - ex_lo);
                        const int32_t nf = ex_hi - ex_lo;
                        const int L = __ldg(map + f);
                        if (MODE == 0)
                            sample_sun<W, false>(dz, L, f, jj, nf, e, rset, com, rho, tmin, sg, dg, key0, key1, p.P, p.err,
                                                 y, nvis, ntest, nseg);
                        else if (MODE == 2)
                            sample_sun<W, true>(dz, L, f, jj, nf, e, rset, com, rho, tmin, sg, dg, key0, key1, p.P, p.err,
                                                y, nvis, ntest, nseg);
                        else
                            sample_thermal<W>(dz, L, f, jj, nf, com, rho, emit, tmin, dg, key0, key1, p.P, p.err, y,
                                              nvis, ntest, nseg);
                    }
                    const bool pvalid = __shfl_xor_sync(0xffffffffu, (int)valid, 1);
#pragma unroll
                    for (int q = 0; q < 6; ++q) {
                        const float yo = __shfl_xor_sync(0xffffffffu, y[q], 1);
                        lacc[warp][q][lane] += y[q];
                        if ((lane & 1) == 0 && valid) {
                            const float df = pvalid ? y[q] - yo : y[q];
                            lacc[warp][6 + q][lane] = fmaf(df, df, lacc[warp][6 + q][lane]);
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    float a = lacc[warp][q][lane], b = lacc[warp][6 + q][lane];
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) {
                        a += __shfl_xor_sync(0xffffffffu, a, off);
                        b += __shfl_xor_sync(0xffffffffu, b, off);
                    }
                    if (lane == 0) { dacc[warp][q] += (double)a; dacc[warp][6 + q] += (double)b; }
                }
                __syncwarp();
            }
        }
        if (lane < 12) p.part[(size_t)u * 12 + lane] = dacc[warp][lane];
        __syncwarp();
    }
    if (p.stats) {
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

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
template <int W, int MINB>
static int area_blocks_v() {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, area_kernel<W, MINB, 0>, 128, 0);
    return nb > 0 ? nb : 1;
}

// Resident 128-thread blocks per SM of the variant (minimum blocks per SM
// the kernel is compiled for: 4, 6 or 8).
int area_resident_blocks(int width, int variant) {
    if (width == 8) return variant == 4 ? area_blocks_v<8, 4>() : variant == 8 ? area_blocks_v<8, 8>() : area_blocks_v<8, 6>();
    return variant == 4 ? area_blocks_v<4, 4>() : variant == 8 ? area_blocks_v<4, 8>() : area_blocks_v<4, 6>();
}

template <int W, int MODE>
static void area_launch_m(const AreaParams& p, int variant, int grid, cudaStream_t st) {
    if (variant == 4) area_kernel<W, 4, MODE><<<grid, 128, 0, st>>>(p);
    else if (variant == 8) area_kernel<W, 8, MODE><<<grid, 128, 0, st>>>(p);
    else area_kernel<W, 6, MODE><<<grid, 128, 0, st>>>(p);
}

template <int W>
static void area_launch_w(const AreaParams& p, int variant, int grid, cudaStream_t st) {
    if (p.mode == 1) area_launch_m<W, 1>(p, variant, grid, st);
    else if (p.mode == 2) area_launch_m<W, 2>(p, variant, grid, st);
    else area_launch_m<W, 0>(p, variant, grid, st);
}

// Prep + scan (the sample tables), then the persistent sampling kernel.
// p.queue must be zeroed on `st` before this call.
cudaError_t launch_area(const AreaParams& p, int width, int variant, int t_max, int grid_cap, cudaStream_t st) {
    if (p.D > 0 && t_max > 0) {
        // designs along grid y, at most 65,535 per launch (the y-dimension limit)
        for (int d0 = 0; d0 < p.D; d0 += 65535) {
            const unsigned nd = (unsigned)std::min(65535, p.D - d0);
            area_prep_kernel<<<dim3((unsigned)((t_max + 255) / 256), nd), 256, 0, st>>>(p, d0);
        }
        area_scan_kernel<<<(unsigned)p.D, 1024, 0, st>>>(p);
    }
    const int64_t units = (int64_t)p.D * p.S * p.cpd;
    if (units == 0) return cudaGetLastError();
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((units + 3) / 4, grid_cap));
    if (width == 8) area_launch_w<8>(p, variant, grid, st);
    else area_launch_w<4>(p, variant, grid, st);
    return cudaGetLastError();
}

}  // namespace srp
