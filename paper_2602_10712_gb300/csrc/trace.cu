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
// neighbouring pixels of one grid row, or on full grids (span mode) a
// block of 8 x 4 pixels (coherent parallel rays share BVH
// nodes through L1).  Blocks loop over chunks with a static stride.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "trace_common.cuh"

namespace srp {

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

// Out-of-line trace and shade, so the wavefront kernel holds one copy of
// each however many places it traces from (keeps the code in the I-cache).
struct HitOut {
    int f;
    float t;
    uint32_t nvis, ntest;
};

// dirc (or null): the direction-only parts of RaySetup (1/d and the shear
// rows), shared by every primary ray of an item and computed once per item
// by setup_ray; bounce segments pass null and set up in full.  One copy of
// the traversal serves both (two copies thrashed the instruction cache).
template <int W>
__device__ __noinline__ HitOut trace_segment(const float4* __restrict__ nodes, const float4* __restrict__ tri,
                                             float ox, float oy, float oz, float dx, float dy, float dz,
                                             float tmin, int skip, const float* dirc, int* err) {
    RaySetup r;
    if (dirc) {
        r.o = f3(ox, oy, oz);
        r.d = f3(dx, dy, dz);
        r.inv = f3(dirc[0], dirc[1], dirc[2]);
        r.oinv = f3(ox * r.inv.x, oy * r.inv.y, oz * r.inv.z);
        r.mx = f3(dirc[3], dirc[4], dirc[5]);
        r.my = f3(dirc[6], dirc[7], dirc[8]);
        r.mz = f3(dirc[9], dirc[10], dirc[11]);
    } else {
        setup_ray(r, f3(ox, oy, oz), f3(dx, dy, dz));
    }
    DesignDev z;
    z.nodes = nodes;
    z.tri = tri;
    HitOut h;
    h.nvis = 0;
    h.ntest = 0;
    h.f = closest_hit<W>(z, r, tmin, skip, h.t, err, h.nvis, h.ntest);
    return h;
}

struct ShadeOut {
    float ox, oy, oz, dx, dy, dz, w;
    int src;
    int cont;
};

// Shade hit k of segment (o, d, w) on triangle f; y points at the ray's
// six running sums (shared memory, stride ys) and is updated in place.
__device__ __noinline__ ShadeOut shade_segment(const float4* __restrict__ tri, const float* __restrict__ rho,
                                               float cx, float cy, float cz, int K, uint64_t seed, int sglob,
                                               int dglob, uint32_t i, int k, int f, float t, float ox, float oy,
                                               float oz, float dx, float dy, float dz, float w, float* y, int ys) {
    DesignDev z;
    z.tri = tri;
    ItemConst ic;
    ic.com = f3(cx, cy, cz);
    ic.rho = rho;
    ic.sglob = sglob;
    ic.dglob = dglob;
    TraceParams p;
    p.K = K;
    p.seed = seed;
    Seg s;
    s.o = f3(ox, oy, oz);
    s.d = f3(dx, dy, dz);
    s.w = w;
    s.src = -1;
    float yy[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) yy[q] = y[q * ys];
    Seg nx;
    const bool cont = shade_hit(z, ic, p, i, k, f, t, s, yy, nx);
#pragma unroll
    for (int q = 0; q < 6; ++q) y[q * ys] = yy[q];
    ShadeOut o;
    o.ox = nx.o.x; o.oy = nx.o.y; o.oz = nx.o.z; o.dx = nx.d.x; o.dy = nx.d.y; o.dz = nx.d.z;
    o.w = nx.w; o.src = nx.src; o.cont = cont ? 1 : 0;
    return o;
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
//                    (span mode: an 8 x 4 block, 16 x 2 or 32 x 1 when the
//                    grid's rows do not divide by 4)
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
#ifndef SRP_BATCHES
#define SRP_BATCHES 4
#endif
constexpr int kBatches = SRP_BATCHES;     // primary batches of 32 rays per tile
constexpr int kTile = 32 * kBatches;      // rays per warp tile
constexpr int kQueue = 64;                // bounce segments per warp (<= 31 + 32 live)

struct WarpSmem {
    float ys[6][kTile];        // per-ray force/torque sums of the tile
    float4 qa[kQueue];         // (o.xyz, w)
    float4 qb[kQueue];         // (d.xyz, src)
    int qs[kQueue];            // slot | (bounce << 16)
    double dacc[12];           // warp FP64 sums (force, torque, squared pair differences)
    float dirc[12];            // the item's 1/d and shear rows (primary segments)
    int64_t bbase[kBatches];   // ray index of the first ray of each batch of the tile
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

// Trace the top `nb` queued segments (one per lane) and shade their hits.
template <int W>
__device__ __forceinline__ void q_batch(WarpSmem& ws, int& qcount, int nb, const DesignDev& dz, const ItemConst& ic,
                                        const TraceParams& p, int64_t bstride, int lane, uint32_t& nvis,
                                        uint32_t& ntest, uint32_t& nseg) {
    const bool has = lane < nb;
    float4 A = make_float4(0, 0, 0, 0), Bv = make_float4(0, 0, 0, 0);
    int q = 0;
    if (has) {
        const int e = qcount - 1 - lane;
        A = ws.qa[e]; Bv = ws.qb[e]; q = ws.qs[e];
    }
    __syncwarp();
    qcount -= nb;
    const int slot = q & 0xffff, kb = q >> 16;
    bool cont = false;
    Seg nx;
    if (has) {
        ++nseg;
        const HitOut h = trace_segment<W>(dz.nodes, dz.tri, A.x, A.y, A.z, Bv.x, Bv.y, Bv.z, ic.tmin_b,
                                          __float_as_int(Bv.w), nullptr, p.err);
        nvis += h.nvis; ntest += h.ntest;
        if (h.f >= 0) {
            const uint64_t i = p.rowoff ? span_ray(ws.bbase[slot >> 5], slot & 31, p.bh, p.nx)
                                        : (uint64_t)(ws.bbase[slot >> 5] + (int64_t)(slot & 31) * bstride);
            const ShadeOut so = shade_segment(dz.tri, ic.rho, ic.com.x, ic.com.y, ic.com.z, p.K, p.seed, ic.sglob,
                                              ic.dglob, (uint32_t)i, kb, h.f, h.t, A.x, A.y, A.z, Bv.x, Bv.y, Bv.z,
                                              A.w, &ws.ys[0][slot], kTile);
            cont = so.cont != 0;
            nx.o = f3(so.ox, so.oy, so.oz); nx.d = f3(so.dx, so.dy, so.dz); nx.w = so.w; nx.src = so.src;
        }
    }
    q_push(ws, qcount, cont, nx, slot, kb + 1, lane);
}

template <int W, int MINB>
__global__ void __launch_bounds__(128, MINB) trace_kernel(const TraceParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpSmem& ws = reinterpret_cast<WarpSmem*>(smem)[warp];
    const int64_t units = (int64_t)p.D * p.S * p.cpb;
    uint32_t nvis = 0, ntest = 0, nseg = 0;
    // dynamic work queue: warps take units in order, so the warps resident
    // at a time work on the same (design, sun) item and uneven designs
    // balance themselves
    while (true) {
        unsigned long long uq = 0;
        if (lane == 0) uq = atomicAdd(p.queue, 1ull);
        const int64_t u = (int64_t)__shfl_sync(0xffffffffu, uq, 0);
        if (u >= units) break;
        const int64_t item_l = u / p.cpb;
        const int64_t cidx = u % p.cpb;
        const int dl = (int)(item_l / p.S), s = (int)(item_l % p.S);
        const int dg = dl;
        const DesignDev dz = p.designs[dl];
        const bool span = p.rowoff != nullptr;
        ItemConst ic;
        if (span) {   // the item's constants as span_kernel computed them
            item_load(ic, p.itab + 8 * (size_t)item_l, p.rho + (size_t)dg * p.G * 2, p.design_base + dg,
                      p.sun_base + s);
            if (lane < 12) ws.dirc[lane] = __ldg(reinterpret_cast<const float*>(p.itab + 8 * (size_t)item_l + 5) + lane);
        } else {
            item_setup(ic, dz, p, p.sun + 3 * ((size_t)(p.sun_per_design ? (int64_t)dg * p.S + s : s)),
                       p.com + 3 * dg, p.rho + (size_t)dg * p.G * 2, p.design_base + dg, p.sun_base + s);
            if (lane == 0) item_dirc(ic, ws.dirc);
        }
        if (lane < 12) ws.dacc[lane] = 0.0;
        __syncwarp();
        // The unit's rays come in batches of 32 (a tile holds kBatches of them):
        // span mode -- the unit's share of the item's live batches (batches of
        // 32 neighbouring pixels (a block of 32 / bh x bh) that can meet the
        // scene, in grid order; the
        // others cannot hit anything and deposit nothing); otherwise -- the
        // contiguous slots [k0, k1) of the ray subset.
        const int64_t bstride = span ? 1 : p.stride;
        int64_t t0, t1;           // this unit's batches (span) or slots
        int row = 0;
        const int32_t* rowoff = nullptr;
        const int32_t* rowfirst = nullptr;
        const int nband = span ? p.ny / p.bh : 0;
        if (span) {
            rowoff = p.rowoff + (size_t)item_l * (nband + 1);
            rowfirst = p.rowfirst + (size_t)item_l * nband;
            const int64_t L = __ldg(rowoff + nband);
            t0 = cidx * L / p.cpb;
            t1 = (cidx + 1) * L / p.cpb;
            // first band with batches at or after t0: the last band whose
            // prefix is <= t0, searched 32 bands at a time (one load per lane
            // and a ballot per round; the prefix is non-decreasing)
            int lo = 0, hi = nband;
            while (hi - lo > 1) {
                const int step = (hi - lo + 31) / 32;
                const int r = lo + lane * step;
                const bool ok = r < hi && (int64_t)__ldg(rowoff + r) <= t0;
                const unsigned m = __ballot_sync(0xffffffffu, ok);
                lo += (31 - __clz(m)) * step;
                hi = min(hi, lo + step);
            }
            row = lo;
        } else {
            t0 = cidx * p.chunk;
            t1 = min(t0 + p.chunk, p.n);
        }
        int qcount = 0;
        for (int64_t ts = t0; ts < t1; ts += span ? kBatches : kTile) {
            const int nslots = span ? 32 * (int)min((int64_t)kBatches, t1 - ts) : (int)min((int64_t)kTile, t1 - ts);
            if (lane == 0) {
                for (int j = 0; j < kBatches; ++j) {
                    int64_t b = 0;
                    if (span) {
                        if (32 * j < nslots) {
                            const int64_t lb = ts + j;
                            while ((int64_t)__ldg(rowoff + row + 1) <= lb) ++row;
                            b = (int64_t)row * p.bh * p.nx +
                                (32 / p.bh) * ((int64_t)__ldg(rowfirst + row) + (lb - __ldg(rowoff + row)));
                        }
                    } else {
                        b = p.off + (ts + 32 * j) * p.stride;
                    }
                    ws.bbase[j] = b;
                }
            }
#pragma unroll
            for (int j = 0; j < kBatches; ++j)
#pragma unroll
                for (int q = 0; q < 6; ++q) ws.ys[q][j * 32 + lane] = 0.0f;
            __syncwarp();
            // ---- primary batches (coherent), bounce batches whenever 32 are queued
#pragma unroll 1
            for (int j = 0; j < kBatches; ++j) {
                const int slot = j * 32 + lane;
                Seg nx;
                bool cont = false;
                if (slot < nslots) {
                    const uint64_t i = span ? span_ray(ws.bbase[j], lane, p.bh, p.nx)
                                            : (uint64_t)(ws.bbase[j] + (int64_t)lane * bstride);
                    const Seg sg = primary_seg(ic, p, i);
                    ++nseg;
                    const HitOut h = trace_segment<W>(dz.nodes, dz.tri, sg.o.x, sg.o.y, sg.o.z, sg.d.x, sg.d.y,
                                                      sg.d.z, 0.0f, -1, ws.dirc, p.err);
                    nvis += h.nvis; ntest += h.ntest;
                    if (h.f >= 0) {
                        const ShadeOut so = shade_segment(dz.tri, ic.rho, ic.com.x, ic.com.y, ic.com.z, p.K, p.seed,
                                                          ic.sglob, ic.dglob, (uint32_t)i, 1, h.f, h.t, sg.o.x,
                                                          sg.o.y, sg.o.z, sg.d.x, sg.d.y, sg.d.z, sg.w,
                                                          &ws.ys[0][slot], kTile);
                        cont = so.cont != 0;
                        nx.o = f3(so.ox, so.oy, so.oz); nx.d = f3(so.dx, so.dy, so.dz); nx.w = so.w; nx.src = so.src;
                    }
                }
                q_push(ws, qcount, cont, nx, slot, 2, lane);
                while (qcount >= 32) q_batch<W>(ws, qcount, 32, dz, ic, p, bstride, lane, nvis, ntest, nseg);
            }
            while (qcount > 0) q_batch<W>(ws, qcount, min(qcount, 32), dz, ic, p, bstride, lane, nvis, ntest, nseg);
            // ---- per-ray sums -> per-lane partials (slot parity = ray parity)
            float accf[6] = {0, 0, 0, 0, 0, 0}, sqf[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
            for (int j = 0; j < kBatches; ++j) {
                const int slot = j * 32 + lane;
                const bool valid = slot < nslots;
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
            // tile sums: fixed-order FP32 warp tree (<= 4 rays per lane), then FP64
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                float a = accf[q], b = sqf[q];
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    a += __shfl_xor_sync(0xffffffffu, a, off);
                    b += __shfl_xor_sync(0xffffffffu, b, off);
                }
                if (lane == 0) { ws.dacc[q] += (double)a; ws.dacc[6 + q] += (double)b; }
            }
            __syncwarp();
        }
        if (lane < 12) p.part[(size_t)u * 12 + lane] = ws.dacc[lane];
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

// ---------------------------------------------------------------------------
// Span pre-pass (full-grid launches): which batches of 32 neighbouring
// pixels (blocks of 32 / bh x bh, bh = TraceParams::bh) can meet the scene.
// One block per (design, sun) item projects the
// BVH boxes five levels below the root (W = 4: up to 1024; W = 8: two
// levels, up to 64) onto the grid plane as pixel rectangles widened by 2 pixels
// (FP32 rounding of the ray origins is ~1e-4 pixel); a ray outside every
// rectangle misses every box, so it cannot hit a triangle and deposits
// nothing.  Per band y of bh grid rows: rowfirst[y] = first batch of the
// band that meets a rectangle, count = batches up to the last one that
// does; rowoff = the exclusive prefix of the counts (rowoff[ny / bh] = the
// item's live batches).
// ---------------------------------------------------------------------------
// Box slots of the span pre-pass: W = 4 -- the nodes five levels below the
// root (1024 slots; on the benchmark's satellite, over 32 sun directions,
// five levels leave 21 % fewer live batches than three, six no more than
// five), W = 8 -- two levels (64).
template <int W>
__host__ __device__ constexpr int top_boxes() { return W == 4 ? 1024 : 64; }
constexpr int kMaxTopBoxes = 1024;

// Pixel rectangle of box slot bi: W = 4 -- the node five levels below the
// root along the base-4 child digits of bi (most significant first); W = 8
// -- two levels (bi>>3, bi&7).  A leaf on the way stands for its whole
// subtree (the slot whose remaining digits are 0 carries it, the others
// are empty).
template <int W>
__device__ __forceinline__ float4 top_rect(const DesignDev& dz, const ItemConst& ic, int bi) {
    const float* nd0 = reinterpret_cast<const float*>(dz.nodes);
    constexpr int NFL = W == 4 ? 32 : 64;   // floats per node
    constexpr int levels = W == 4 ? 5 : 2;
    int digit[5];
    if (W == 4) {
        for (int lv = 0; lv < 5; ++lv) digit[lv] = (bi >> (2 * (4 - lv))) & 3;
    } else {
        digit[0] = bi >> 3; digit[1] = bi & 7; digit[2] = 0; digit[3] = 0; digit[4] = 0;
    }
    const float* nd = nd0;
    float lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    bool ok = false;
    for (int lv = 0; lv < levels; ++lv) {
        const int c = digit[lv];
        for (int a = 0; a < 3; ++a) { lo[a] = __ldg(nd + 2 * W * a + c); hi[a] = __ldg(nd + 2 * W * a + W + c); }
        if (!(lo[0] <= hi[0])) { ok = false; break; }
        ok = true;
        const int code = __float_as_int(__ldg(nd + 6 * W + c));
        if (lv == levels - 1) break;
        if (code < 0) {   // a leaf: only the slot with the remaining digits 0 keeps it
            for (int l2 = lv + 1; l2 < levels; ++l2) ok = ok && digit[l2] == 0;
            break;
        }
        nd = nd0 + (size_t)code * NFL;
    }
    float4 rc = make_float4(INFINITY, -INFINITY, INFINITY, -INFINITY);
    if (ok) {
        const float3 cb = f3(0.5f * (lo[0] + hi[0]), 0.5f * (lo[1] + hi[1]), 0.5f * (lo[2] + hi[2]));
        const float3 h = f3(0.5f * (hi[0] - lo[0]), 0.5f * (hi[1] - lo[1]), 0.5f * (hi[2] - lo[2]));
        const float3 q = cb - ic.ob;
        const float ac = dot(q, ic.bu), bc = dot(q, ic.bv);
        const float ea = fabsf(ic.bu.x) * h.x + fabsf(ic.bu.y) * h.y + fabsf(ic.bu.z) * h.z;
        const float eb = fabsf(ic.bv.x) * h.x + fabsf(ic.bv.y) * h.y + fabsf(ic.bv.z) * h.z;
        rc = make_float4((ac - ea) / ic.fdx - 2.0f, (ac + ea) / ic.fdx + 2.0f, (bc - eb) / ic.fdy - 2.0f,
                         (bc + eb) / ic.fdy + 2.0f);
    }
    return rc;
}

template <int W>
__global__ void __launch_bounds__(128) span_kernel(const TraceParams p) {
    constexpr int kTopBoxes = top_boxes<W>();
    __shared__ float4 rect[kMaxTopBoxes];
    __shared__ int wtot[4];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int64_t items = (int64_t)p.D * p.S;
    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
        const int dl = (int)(item / p.S), s = (int)(item % p.S);
        const DesignDev dz = p.designs[dl];
        ItemConst ic;
        item_setup(ic, dz, p, p.sun + 3 * ((size_t)(p.sun_per_design ? (int64_t)dl * p.S + s : s)),
                   p.com + 3 * dl, p.rho + (size_t)dl * p.G * 2, p.design_base + dl, p.sun_base + s);
        if (t == 0) item_store(ic, p.itab + 8 * (size_t)item);
        // the non-empty rectangles, compacted (a small tree fills few of
        // the slots): per thread its slots t, t + 128, ..., then a block scan
        // of the counts gives each thread its output range
        constexpr int kPer = (kTopBoxes + 127) / 128;
        float4 mine[kPer];
        int nv = 0;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int bi = t + 128 * k;
            mine[k] = bi < kTopBoxes ? top_rect<W>(dz, ic, bi) : make_float4(INFINITY, -INFINITY, INFINITY, -INFINITY);
            nv += mine[k].x <= mine[k].y ? 1 : 0;
        }
        int incl = nv;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += o;
        }
        if (lane == 31) wtot[w] = incl;
        __syncthreads();
        int pos = incl - nv;
        for (int k = 0; k < w; ++k) pos += wtot[k];
        const int nrect = wtot[0] + wtot[1] + wtot[2] + wtot[3];
#pragma unroll
        for (int k = 0; k < kPer; ++k)
            if (mine[k].x <= mine[k].y) rect[pos++] = mine[k];
        __syncthreads();
        const int bh = p.bh, bw = 32 / bh;
        const int nbx = p.nx / bw, ny = p.ny / bh;   // batches per band, bands
        const float inv_bw = 1.0f / (float)bw;      // exact: bw is a power of two
        int32_t* ro = p.rowoff + (size_t)item * (ny + 1);
        int32_t* rf = p.rowfirst + (size_t)item * ny;
        int carry = 0;
        for (int y0 = 0; y0 < ny; y0 += 128) {
            const int y = y0 + t;   // band: grid rows bh y .. bh y + bh - 1
            int cnt = 0;
            if (y < ny) {
                float xmin = INFINITY, xmax = -INFINITY;
                for (int j = 0; j < nrect; ++j) {
                    const float4 r = rect[j];
                    if (r.z < (float)(bh * y + bh) && r.w > (float)(bh * y)) {
                        xmin = fminf(xmin, r.x);
                        xmax = fmaxf(xmax, r.y);
                    }
                }
                int bf = 0;
                if (xmin < xmax) {
                    const int b0 = (int)floorf(fminf(fmaxf(xmin * inv_bw, 0.0f), (float)nbx));
                    const int b1 = (int)ceilf(fminf(fmaxf(xmax * inv_bw, 0.0f), (float)nbx));
                    if (b1 > b0) { bf = b0; cnt = b1 - b0; }
                }
                rf[y] = bf;
            }
            // exclusive prefix of the counts over rows: warp scans, then the
            // warp totals in warp order
            int inc = cnt;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int o = __shfl_up_sync(0xffffffffu, inc, off);
                if (lane >= off) inc += o;
            }
            if (lane == 31) wtot[w] = inc;
            __syncthreads();
            int woff = 0;
            for (int k = 0; k < w; ++k) woff += wtot[k];
            if (y < ny) ro[y] = carry + woff + inc - cnt;
            carry += wtot[0] + wtot[1] + wtot[2] + wtot[3];
            __syncthreads();
        }
        if (t == 0) ro[ny] = carry;
    }
}

cudaError_t launch_span(const TraceParams& p, int width, cudaStream_t st) {
    const int64_t items = (int64_t)p.D * p.S;
    if (items == 0) return cudaSuccess;
    const unsigned grid = (unsigned)std::min<int64_t>(items, (int64_t)1 << 20);   // one block per item
    if (width == 8) span_kernel<8><<<grid, 128, 0, st>>>(p);
    else span_kernel<4><<<grid, 128, 0, st>>>(p);
    return cudaGetLastError();
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

// Sum each item's chunk partials -> (F, tau), sigma.  One block per item
// (grid-stride over items): thread t adds chunks t, t + 128, ... in chunk
// order (a chunk's 12 sums are 96 contiguous bytes, so a warp's loads are
// coalesced), then a fixed shuffle tree per warp and the four warp totals in
// warp order -- the same summation order on every call.
constexpr int kReduceThreads = 128;

__global__ void __launch_bounds__(kReduceThreads) reduce_items_kernel(const double* __restrict__ part, int64_t items,
                                                                     int cpb, double* __restrict__ out_ft,
                                                                     double* __restrict__ out_sigma) {
    __shared__ double wsum[12][kReduceThreads / 32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
        double acc[12];
#pragma unroll
        for (int q = 0; q < 12; ++q) acc[q] = 0.0;
        const double2* base = reinterpret_cast<const double2*>(part + (size_t)item * cpb * 12);
        for (int c = t; c < cpb; c += kReduceThreads) {
#pragma unroll
            for (int h = 0; h < 6; ++h) {
                const double2 v = __ldg(base + (size_t)c * 6 + h);
                acc[2 * h] += v.x;
                acc[2 * h + 1] += v.y;
            }
        }
#pragma unroll
        for (int q = 0; q < 12; ++q)
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], off);
        if (lane == 0)
#pragma unroll
            for (int q = 0; q < 12; ++q) wsum[q][w] = acc[q];
        __syncthreads();
        if (t < 12) {
            double s = wsum[t][0];
#pragma unroll
            for (int k = 1; k < kReduceThreads / 32; ++k) s += wsum[t][k];
            if (t < 6) out_ft[item * 6 + t] = s;
            else if (out_sigma) out_sigma[item * 6 + (t - 6)] = sqrt(s);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
template <int W, int MINB>
static int resident_blocks_v(int block) {
    int nb = 0;
    const size_t sm = trace_smem_bytes(block);
    cudaFuncSetAttribute(trace_kernel<W, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, trace_kernel<W, MINB>, block, sm);
    return nb > 0 ? nb : 1;
}

// Also performs the one-time kernel attribute set-up (call before launching).
int trace_resident_blocks(int width, int block, int variant) {
    if (width == 8) {
        if (variant == 4) return resident_blocks_v<8, 4>(block);
        if (variant == 6) return resident_blocks_v<8, 6>(block);
        if (variant == 7) return resident_blocks_v<8, 7>(block);
        if (variant == 8) return resident_blocks_v<8, 8>(block);
        return resident_blocks_v<8, 5>(block);
    }
    if (variant == 4) return resident_blocks_v<4, 4>(block);
    if (variant == 6) return resident_blocks_v<4, 6>(block);
    if (variant == 7) return resident_blocks_v<4, 7>(block);
    if (variant == 8) return resident_blocks_v<4, 8>(block);
    return resident_blocks_v<4, 5>(block);
}
int trace_resident_blocks(int width, int block) { return trace_resident_blocks(width, block, 5); }

// One persistent launch over every (design, sun, chunk) unit.  p.designs,
// p.queue (zeroed on the stream before the launch) and p.part are set.
cudaError_t launch_trace(const TraceParams& p, int width, int grid_cap, int block, cudaStream_t st) {
    const int64_t units = (int64_t)p.D * p.S * p.cpb;
    const int64_t wpb = block / 32;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((units + wpb - 1) / wpb, grid_cap));
    const size_t sm = trace_smem_bytes(block);
    if (width == 8) {
        if (p.variant == 4) trace_kernel<8, 4><<<grid, block, sm, st>>>(p);
        else if (p.variant == 6) trace_kernel<8, 6><<<grid, block, sm, st>>>(p);
        else if (p.variant == 7) trace_kernel<8, 7><<<grid, block, sm, st>>>(p);
        else if (p.variant == 8) trace_kernel<8, 8><<<grid, block, sm, st>>>(p);
        else trace_kernel<8, 5><<<grid, block, sm, st>>>(p);
    } else {
        if (p.variant == 4) trace_kernel<4, 4><<<grid, block, sm, st>>>(p);
        else if (p.variant == 6) trace_kernel<4, 6><<<grid, block, sm, st>>>(p);
        else if (p.variant == 7) trace_kernel<4, 7><<<grid, block, sm, st>>>(p);
        else if (p.variant == 8) trace_kernel<4, 8><<<grid, block, sm, st>>>(p);
        else trace_kernel<4, 5><<<grid, block, sm, st>>>(p);
    }
    return cudaGetLastError();
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
    if (items <= 0) return cudaSuccess;
    if (reinterpret_cast<uintptr_t>(part) % 16 != 0) return cudaErrorMisalignedAddress;   // double2 loads
    const unsigned grid = (unsigned)std::min<int64_t>(items, (int64_t)1 << 20);
    reduce_items_kernel<<<grid, kReduceThreads, 0, st>>>(part, items, cpb, out_ft, out_sigma);
    return cudaGetLastError();
}

}  // namespace srp
