// samples.cu -- tracing with a design per sample (Sec. 3.2 "Estimation":
// every sample intersects its own design, so one BVH per design does not
// pay; Alg. 1 NNLoss draws a random design per sample) for sm_103a.
//
// A setup kernel (one thread per sample) does the FP64 work once: the ONB
// of the sun direction and the grid origin (as the ray-grid tracer), and the
// hinge rotations (Rodrigues, FP32 rows + pivot).  A warp then owns one
// sample at a time:
//   it copies the sample's rotation rows to its shared-memory slot;
//   for meshes of up to 256 triangles it instantiates the base mesh into
//     its shared-memory slot (3 float4 per triangle: vertices, original
//     index and group in .w); larger meshes are instantiated triangle by
//     triangle as they are tested (from the L1-resident base mesh);
//   the sample's ray is the jittered single pixel of a 1 x 1 grid over the
//     square of side 2R about the given centre (Philox counter
//     (0, sample_base + s, 2^29, k), weight P (2R)^2);
//   closest hit by brute force: lane l tests triangles l, l+32, ...; a
//     warp argmin (ties -> smaller index) picks the hit; every lane then
//     runs the same shading (absorbed / specular / Lambertian, up to K
//     bounces) on the shared triangle, so the warp never diverges on it;
//   lane 0 writes the sample's (F, tau) estimate and its hit list.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "trace_common.cuh"

namespace srp {

struct SampleParams {
    int32_t V, H, T, G, K;
    int64_t N;
    uint64_t seed;
    double P;
    uint32_t sample_base;
    double c[3], R;
    const float* verts;     // [V][3]
    const int32_t* vhinge;  // [V], -1 = fixed
    const double* hinges;   // [H][6] pivot, unit axis
    const int32_t* tris;    // [T][3]
    const int32_t* group;   // [T]
    const double* angles;   // [N][H]
    const float* rho;       // [N][G][2]
    const double* sun;      // [N][3]
    const double* com;      // [N][3]
    double* out_y;          // [N][6]
    int32_t* out_hits;      // [N][K] or null
    unsigned long long* queue;
    float4* setup;          // [N][5]: ray frame of the sample (samples_setup_kernel)
    float4* rot;            // [N][H][3]: hinge rotation rows + pivot component
};

// One thread per sample: the FP64 parts (ONB of the sun direction, grid
// origin, hinge rotations) once per sample instead of once per lane.
__global__ void __launch_bounds__(128) samples_setup_kernel(const SampleParams p) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= p.N) return;
    TraceParams tp;
    tp.nx = 1; tp.ny = 1; tp.P = p.P;
    DesignDev dz;
    dz.cx = p.c[0]; dz.cy = p.c[1]; dz.cz = p.c[2]; dz.R = p.R;
    ItemConst ic;
    item_setup(ic, dz, tp, p.sun + 3 * (size_t)s, p.com + 3 * (size_t)s, nullptr, 0, 0);
    float4* o = p.setup + 5 * (size_t)s;
    o[0] = make_float4(ic.ob.x, ic.ob.y, ic.ob.z, ic.fdx);
    o[1] = make_float4(ic.bu.x, ic.bu.y, ic.bu.z, ic.fdy);
    o[2] = make_float4(ic.bv.x, ic.bv.y, ic.bv.z, ic.w0);
    o[3] = make_float4(ic.dd.x, ic.dd.y, ic.dd.z, ic.tmin_b);
    o[4] = make_float4(ic.com.x, ic.com.y, ic.com.z, 0.0f);
    for (int h = 0; h < p.H; ++h) {
        const double* hg = p.hinges + 6 * h;
        const double ax = hg[3], ay = hg[4], az = hg[5];
        const double nrm = sqrt(ax * ax + ay * ay + az * az);
        const double x = ax / nrm, y = ay / nrm, z = az / nrm;
        double sn, cs;
        sincos(p.angles[(size_t)s * p.H + h], &sn, &cs);
        const double t = 1.0 - cs;
        float4* r = p.rot + 3 * ((size_t)s * p.H + h);
        r[0] = make_float4((float)(cs + x * x * t), (float)(x * y * t - z * sn), (float)(x * z * t + y * sn), (float)hg[0]);
        r[1] = make_float4((float)(y * x * t + z * sn), (float)(cs + y * y * t), (float)(y * z * t - x * sn), (float)hg[1]);
        r[2] = make_float4((float)(z * x * t - y * sn), (float)(z * y * t + x * sn), (float)(cs + z * z * t), (float)hg[2]);
    }
}

// Shared memory of a warp: the instantiated mesh (RESIDENT) and the
// sample's rotation rows.
__host__ __device__ inline size_t samples_warp_f4(int T, int H, bool resident) {
    return (resident ? (size_t)3 * T : 0) + (size_t)3 * H;
}

// Vertex vi of the sample's design (rotated about its hinge pivot).
__device__ __forceinline__ float3 inst_vertex(const SampleParams& p, const float4* rot, int vi) {
    float3 v = f3(__ldg(p.verts + 3 * (size_t)vi), __ldg(p.verts + 3 * (size_t)vi + 1), __ldg(p.verts + 3 * (size_t)vi + 2));
    const int h = __ldg(p.vhinge + vi);
    if (h >= 0) {
        const float4 r0 = rot[3 * h], r1 = rot[3 * h + 1], r2 = rot[3 * h + 2];
        const float3 q = f3(v.x - r0.w, v.y - r1.w, v.z - r2.w);
        v = f3(r0.w + (r0.x * q.x + r0.y * q.y + r0.z * q.z), r1.w + (r1.x * q.x + r1.y * q.y + r1.z * q.z),
               r2.w + (r2.x * q.x + r2.y * q.y + r2.z * q.z));
    }
    return v;
}

// Triangle f of the sample's design as 3 float4 (.w: index, group, 0).
__device__ __forceinline__ void inst_tri(const SampleParams& p, const float4* rot, int f, float4 out[3]) {
#pragma unroll
    for (int cidx = 0; cidx < 3; ++cidx) {
        const float3 v = inst_vertex(p, rot, __ldg(p.tris + 3 * (size_t)f + cidx));
        float w = 0.0f;
        if (cidx == 0) w = __uint_as_float((uint32_t)f);
        if (cidx == 1) w = __uint_as_float((uint32_t)__ldg(p.group + f));
        out[cidx] = make_float4(v.x, v.y, v.z, w);
    }
}

// RESIDENT: the warp instantiates the whole mesh into shared memory once
// per sample (small meshes); otherwise each test instantiates its triangle
// from the base mesh (L1-resident), keeping shared memory -- and thus
// occupancy -- independent of T.
template <bool RESIDENT>
__global__ void __launch_bounds__(128) samples_kernel(const SampleParams p) {
    extern __shared__ float4 sm4[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float4* tri = sm4 + (size_t)warp * samples_warp_f4(p.T, p.H, RESIDENT);
    float4* rot = tri + (RESIDENT ? 3 * (size_t)p.T : 0);
    TraceParams tp;
    tp.nx = 1; tp.ny = 1; tp.K = p.K; tp.jitter = 1; tp.seed = p.seed; tp.P = p.P;
    while (true) {
        unsigned long long uq = 0;
        if (lane == 0) uq = atomicAdd(p.queue, 1ull);
        const int64_t s = (int64_t)__shfl_sync(0xffffffffu, uq, 0);
        if (s >= p.N) break;
        // hinge rotations of this sample (precomputed rows)
        for (int q = lane; q < 3 * p.H; q += 32) rot[q] = __ldg(p.rot + 3 * (size_t)s * p.H + q);
        __syncwarp();
        // instantiate the mesh into shared memory
        if (RESIDENT) {
            for (int f = lane; f < p.T; f += 32) {
                float4 tv[3];
                inst_tri(p, rot, f, tv);
                tri[3 * (size_t)f] = tv[0]; tri[3 * (size_t)f + 1] = tv[1]; tri[3 * (size_t)f + 2] = tv[2];
            }
            __syncwarp();
        }
        ItemConst ic;
        {
            const float4* su = p.setup + 5 * (size_t)s;
            const float4 a0 = __ldg(su), a1 = __ldg(su + 1), a2 = __ldg(su + 2), a3 = __ldg(su + 3), a4 = __ldg(su + 4);
            ic.ob = f3(a0.x, a0.y, a0.z); ic.fdx = a0.w;
            ic.bu = f3(a1.x, a1.y, a1.z); ic.fdy = a1.w;
            ic.bv = f3(a2.x, a2.y, a2.z); ic.w0 = a2.w;
            ic.dd = f3(a3.x, a3.y, a3.z); ic.tmin_b = a3.w;
            ic.com = f3(a4.x, a4.y, a4.z);
            ic.rho = p.rho + (size_t)s * p.G * 2;
            ic.dglob = (int)0x20000000;
            ic.sglob = (int)(p.sample_base + (uint32_t)s);
        }
        Seg sg = primary_seg(ic, tp, 0);
        float y[6] = {0, 0, 0, 0, 0, 0};
        int32_t hit_list[kMaxBounces] = {-1, -1, -1};
        for (int k = 1; k <= p.K; ++k) {
            RaySetup r;
            setup_ray(r, sg.o, sg.d);
            const float tmin = k == 1 ? 0.0f : ic.tmin_b;
            float bt = INFINITY;
            int bf = -1;
            for (int f = lane; f < p.T; f += 32) {
                if (f == sg.src) continue;
                float t;
                if (RESIDENT) {
                    t = hit_triangle(r, xyz(tri[3 * f]), xyz(tri[3 * f + 1]), xyz(tri[3 * f + 2]));
                } else {
                    float4 tv[3];
                    inst_tri(p, rot, f, tv);
                    t = hit_triangle(r, xyz(tv[0]), xyz(tv[1]), xyz(tv[2]));
                }
                if (t > tmin && t < bt) { bt = t; bf = f; }   // lane's triangles in increasing index
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const float ot = __shfl_xor_sync(0xffffffffu, bt, off);
                const int of = __shfl_xor_sync(0xffffffffu, bf, off);
                if (of >= 0 && (ot < bt || (ot == bt && (bf < 0 || of < bf)))) { bt = ot; bf = of; }
            }
            if (bf < 0) break;
            hit_list[k - 1] = bf;
            float4 hv[3];
            if (RESIDENT) { hv[0] = tri[3 * bf]; hv[1] = tri[3 * bf + 1]; hv[2] = tri[3 * bf + 2]; }
            else inst_tri(p, rot, bf, hv);
            const HitGeom hg = hit_geom_v(hv[0], hv[1], hv[2], ic, bt, sg);
            Seg nx;
            if (!shade_core(hg, ic, tp, 0u, k, bf, sg, y, nx)) break;
            sg = nx;
        }
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < 6; ++q) p.out_y[6 * (size_t)s + q] = (double)y[q];
            if (p.out_hits)
                for (int k = 0; k < p.K; ++k) p.out_hits[(size_t)s * p.K + k] = hit_list[k];
        }
        __syncwarp();
    }
}

// Meshes up to this many triangles are instantiated into shared memory
// (12 KB per warp, 4 warps per block); larger ones stream from the base mesh.
constexpr int kResidentMaxT = 256;

template <bool RESIDENT>
static cudaError_t launch_samples_t(const SampleParams& p, int n_sm, cudaStream_t st) {
    const size_t per_warp = samples_warp_f4(p.T, p.H, RESIDENT) * sizeof(float4);
    const int wpb = 4;
    const int block = 32 * wpb;
    const size_t sm = per_warp * wpb;
    cudaError_t e = cudaFuncSetAttribute(samples_kernel<RESIDENT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, samples_kernel<RESIDENT>, block, sm);
    if (e != cudaSuccess) return e;
    const int64_t want = (p.N + wpb - 1) / wpb;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)n_sm * std::max(nb, 1)));
    samples_kernel<RESIDENT><<<grid, block, sm, st>>>(p);
    return cudaGetLastError();
}

// Setup kernel, then the persistent per-sample kernel.
cudaError_t launch_samples(const SampleParams& p, int n_sm, cudaStream_t st) {
    if (p.N == 0) return cudaSuccess;
    samples_setup_kernel<<<(unsigned)((p.N + 127) / 128), 128, 0, st>>>(p);
    return p.T <= kResidentMaxT ? launch_samples_t<true>(p, n_sm, st) : launch_samples_t<false>(p, n_sm, st);
}

void set_last_error(const std::string& msg);
cudaStream_t ctx_stream(srp_ctx* c);
int ctx_device(srp_ctx* c);
int ctx_n_sm(srp_ctx* c);

}  // namespace srp

namespace {
int sfail(int code, const std::string& m) {
    srp::set_last_error(m);
    return code;
}
}  // namespace

extern "C" int srp_trace_samples(srp_ctx* c, const float* verts, int V, const int32_t* vhinge, const double* hinges,
                                 int H, const int32_t* tris, const int32_t* group, int T, const double* angles,
                                 const float* rho, int G, const double* sun, const double* com, int64_t N,
                                 const double* center, double radius, const srp_trace_opts* o, double* out_y,
                                 int32_t* out_hits) {
    using namespace srp;
    if (!c || !o) return sfail(SRP_EINVAL, "srp_trace_samples: NULL ctx/opts");
    if (V < 0 || T < 0 || H < 0 || N < 0) return sfail(SRP_EINVAL, "srp_trace_samples: negative size");
    if (H > 32) return sfail(SRP_EINVAL, "srp_trace_samples: at most 32 hinges");
    if (G < 1 || G > kMaxGroups) return sfail(SRP_EINVAL, "srp_trace_samples: G must be in 1..64");
    if (N > 0xffffffffLL) return sfail(SRP_EINVAL, "srp_trace_samples: N must be < 2^32");
    if (o->max_bounces < 1 || o->max_bounces > kMaxBounces)
        return sfail(SRP_EINVAL, "srp_trace_samples: max_bounces must be 1..3");
    if (!(o->pressure >= 0.0) || !std::isfinite(o->pressure)) return sfail(SRP_EINVAL, "srp_trace_samples: bad pressure");
    if (!center || !(radius > 0.0) || !std::isfinite(radius)) return sfail(SRP_EINVAL, "srp_trace_samples: bad centre/radius");
    if (o->mem != SRP_MEM_HOST && o->mem != SRP_MEM_DEVICE) return sfail(SRP_EINVAL, "srp_trace_samples: bad mem");
    if (T > (1 << 24)) return sfail(SRP_EINVAL, "srp_trace_samples: T must be < 2^24");
    if (T > 0 && (!verts || !tris || !group || (H > 0 && (!vhinge || !hinges))))
        return sfail(SRP_EINVAL, "srp_trace_samples: NULL mesh array");
    for (int t = 0; t < T; ++t) {
        for (int j = 0; j < 3; ++j)
            if (tris[3 * t + j] < 0 || tris[3 * t + j] >= V) return sfail(SRP_EINVAL, "srp_trace_samples: vertex index out of range");
        if (group[t] < 0 || group[t] >= G) return sfail(SRP_EINVAL, "srp_trace_samples: group out of [0, G)");
    }
    for (int v = 0; v < V && H > 0; ++v)
        if (vhinge[v] < -1 || vhinge[v] >= H) return sfail(SRP_EINVAL, "srp_trace_samples: hinge id out of range");
    for (int h = 0; h < H; ++h) {
        const double* a = hinges + 6 * h + 3;
        if (!(std::fabs(std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]) - 1.0) < 1e-6))
            return sfail(SRP_EINVAL, "srp_trace_samples: hinge axis not unit");
    }
    if (N == 0) return SRP_OK;
    if (!angles && H > 0) return sfail(SRP_EINVAL, "srp_trace_samples: NULL angles");
    if (!rho || !sun || !com || !out_y) return sfail(SRP_EINVAL, "srp_trace_samples: NULL per-sample array");
    const int K = o->max_bounces;
    if (o->mem == SRP_MEM_HOST) {
        for (int64_t q = 0; q < N * G; ++q) {
            const float rs = rho[2 * q], rd = rho[2 * q + 1];
            if (!(rs >= 0.0f && rd >= 0.0f && rs + rd <= 1.0f + 1e-6f))
                return sfail(SRP_EINVAL, "srp_trace_samples: reflectances must satisfy 0 <= rho_s, rho_d, sum <= 1");
        }
        for (int64_t q = 0; q < N; ++q) {
            const double* e = sun + 3 * q;
            if (!(std::fabs(std::sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]) - 1.0) < 1e-6))
                return sfail(SRP_EINVAL, "srp_trace_samples: sun directions must be unit vectors");
        }
    }
    cudaError_t e = cudaSetDevice(ctx_device(c));
    if (e != cudaSuccess) return sfail(SRP_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    cudaStream_t st = ctx_stream(c);
    // one stream-ordered scratch: queue | mesh | (host mode) per-sample inputs and outputs
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t b_q = al(sizeof(unsigned long long)), b_v = al(sizeof(float) * 3 * (size_t)V),
                 b_vh = al(sizeof(int32_t) * (size_t)std::max(V, 1)), b_h = al(sizeof(double) * 6 * (size_t)std::max(H, 1)),
                 b_t = al(sizeof(int32_t) * 3 * (size_t)T), b_g = al(sizeof(int32_t) * (size_t)T);
    const bool host = o->mem == SRP_MEM_HOST;
    const size_t b_an = host ? al(sizeof(double) * (size_t)N * std::max(H, 1)) : 0,
                 b_r = host ? al(sizeof(float) * 2 * (size_t)N * G) : 0, b_s = host ? al(sizeof(double) * 3 * (size_t)N) : 0,
                 b_c = host ? al(sizeof(double) * 3 * (size_t)N) : 0, b_y = host ? al(sizeof(double) * 6 * (size_t)N) : 0,
                 b_hi = host && out_hits ? al(sizeof(int32_t) * K * (size_t)N) : 0;
    const size_t b_su = al(sizeof(float4) * 5 * (size_t)N), b_ro = al(sizeof(float4) * 3 * (size_t)N * std::max(H, 1));
    const size_t total = b_q + b_v + b_vh + b_h + b_t + b_g + b_an + b_r + b_s + b_c + b_y + b_hi + b_su + b_ro;
    char* base = nullptr;
    e = cudaMallocAsync((void**)&base, total, st);
    if (e != cudaSuccess) return sfail(SRP_ENOMEM, "srp_trace_samples: scratch");
    char* q = base;
    auto take = [&](size_t b) { char* r = q; q += b; return r; };
    SampleParams p;
    p.V = V; p.H = H; p.T = T; p.G = G; p.K = K; p.N = N;
    p.seed = o->seed; p.P = o->pressure; p.sample_base = (uint32_t)o->sun_base;
    for (int j = 0; j < 3; ++j) p.c[j] = center[j];
    p.R = radius;
    p.queue = (unsigned long long*)take(b_q);
    p.verts = (const float*)take(b_v);
    p.vhinge = (const int32_t*)take(b_vh);
    p.hinges = (const double*)take(b_h);
    p.tris = (const int32_t*)take(b_t);
    p.group = (const int32_t*)take(b_g);
    p.setup = (float4*)take(b_su);
    p.rot = (float4*)take(b_ro);
    std::vector<int32_t> vh(std::max(V, 1), -1);
    if (H > 0) std::copy(vhinge, vhinge + V, vh.begin());
    bool ok = cudaMemsetAsync(p.queue, 0, sizeof(unsigned long long), st) == cudaSuccess;
    if (V) ok = ok && cudaMemcpyAsync((void*)p.verts, verts, sizeof(float) * 3 * V, cudaMemcpyHostToDevice, st) == cudaSuccess;
    ok = ok && cudaMemcpyAsync((void*)p.vhinge, vh.data(), sizeof(int32_t) * std::max(V, 1), cudaMemcpyHostToDevice, st) == cudaSuccess;
    if (H) ok = ok && cudaMemcpyAsync((void*)p.hinges, hinges, sizeof(double) * 6 * H, cudaMemcpyHostToDevice, st) == cudaSuccess;
    if (T) {
        ok = ok && cudaMemcpyAsync((void*)p.tris, tris, sizeof(int32_t) * 3 * T, cudaMemcpyHostToDevice, st) == cudaSuccess;
        ok = ok && cudaMemcpyAsync((void*)p.group, group, sizeof(int32_t) * T, cudaMemcpyHostToDevice, st) == cudaSuccess;
    }
    if (host) {
        p.angles = (const double*)take(b_an); p.rho = (const float*)take(b_r); p.sun = (const double*)take(b_s);
        p.com = (const double*)take(b_c); p.out_y = (double*)take(b_y);
        p.out_hits = out_hits ? (int32_t*)take(b_hi) : nullptr;
        if (H) ok = ok && cudaMemcpyAsync((void*)p.angles, angles, sizeof(double) * N * H, cudaMemcpyHostToDevice, st) == cudaSuccess;
        ok = ok && cudaMemcpyAsync((void*)p.rho, rho, sizeof(float) * 2 * N * G, cudaMemcpyHostToDevice, st) == cudaSuccess;
        ok = ok && cudaMemcpyAsync((void*)p.sun, sun, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, st) == cudaSuccess;
        ok = ok && cudaMemcpyAsync((void*)p.com, com, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, st) == cudaSuccess;
    } else {
        p.angles = angles; p.rho = rho; p.sun = sun; p.com = com; p.out_y = out_y; p.out_hits = out_hits;
    }
    if (ok) ok = launch_samples(p, ctx_n_sm(c), st) == cudaSuccess;
    if (ok && host) {
        ok = cudaMemcpyAsync(out_y, p.out_y, sizeof(double) * 6 * N, cudaMemcpyDeviceToHost, st) == cudaSuccess;
        if (out_hits)
            ok = ok && cudaMemcpyAsync(out_hits, p.out_hits, sizeof(int32_t) * K * N, cudaMemcpyDeviceToHost, st) == cudaSuccess;
    }
    cudaFreeAsync(base, st);
    if (!ok) return sfail(SRP_ECUDA, std::string("srp_trace_samples: ") + cudaGetErrorString(cudaGetLastError()));
    if (host) return srp_sync(c);
    return SRP_OK;
}
