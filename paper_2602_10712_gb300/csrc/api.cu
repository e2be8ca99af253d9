// api.cu -- C ABI of the SRP library: contexts, validation, BVH upload and
// the host side of srp_force (see include/srp.h for the contract).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "srp_internal.h"

namespace srp {
int trace_resident_blocks(int width, int block, int variant);
cudaError_t launch_span(const TraceParams& p, int width, cudaStream_t st);
cudaError_t launch_trace(const TraceParams& p, int width, int grid_cap, int block, cudaStream_t st);
cudaError_t launch_reduce(const double* part, int64_t items, int cpb, double* out_ft, double* out_sigma,
                          cudaStream_t st);
cudaError_t launch_trace_rays(const DesignDev& dz, const TraceParams& p, const int64_t* ray_idx, int64_t nr,
                              int sidx, int didx, double* out_y, int32_t* out_hits, cudaStream_t st);
void set_last_error(const std::string& msg);
cudaError_t run_read_probe(int64_t bytes, int passes, int reps, cudaStream_t st, double* out_gbs);
int area_resident_blocks(int width, int variant);
cudaError_t launch_area(const AreaParams& p, int width, int variant, int t_max, int grid_cap, cudaStream_t st);
cudaError_t launch_grad(const DesignDev& dz, const TraceParams& p, const double* up, const int32_t* thinge,
                        const double* hax, int H, double* gpart, double* d_rho, double* d_hinge, int n_sm,
                        cudaStream_t st);
cudaError_t launch_refit(srp_bvh* h, const float* verts, const int32_t* tris, float pad_abs, cudaStream_t st);

}  // namespace srp

using namespace srp;

namespace {
thread_local std::string g_err;
}  // namespace

// Message for srp_last_error() from other translation units of the library.
void srp::set_last_error(const std::string& msg) { g_err = msg; }


namespace {

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}
int cuda_fail(cudaError_t e, const char* where) {
    return fail(SRP_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
#define CU(call, where)                                   \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, where); \
    } while (0)

// A device buffer that only grows.
struct DevBuf {
    void* p = nullptr;
    size_t n = 0;
    cudaError_t ensure(size_t bytes) {
        if (bytes <= n) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr; n = 0;
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e == cudaSuccess) n = bytes;
        return e;
    }
    void release() { if (p) cudaFree(p); p = nullptr; n = 0; }
};
}  // namespace

struct srp_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int n_sm = 0;
    int* d_err = nullptr;
    unsigned long long* d_stats = nullptr;     // traversal counters
    bool stats_on = false;
    DevBuf part;                               // trace partials
    DevBuf gpart;                              // gradient partials
    DevBuf dtab;                               // device design table
    DesignDev* htab = nullptr;                 // pinned staging of the table
    size_t htab_n = 0;
    std::vector<DesignDev> last_tab;           // table currently on the device
    cudaEvent_t tab_ev = nullptr;              // last table upload
    unsigned long long* d_queue = nullptr;     // work-queue counter
    DevBuf stage_in, stage_out;                // host-mem staging
    DevBuf span;                               // full-grid launches: rowfirst | rowoff (int32)
    DevBuf atab;                               // area estimator: cnt | map | ex (int32)
    DevBuf axb;                                // area estimator: xbase | ntot (int64)
};

extern "C" {

const char* srp_last_error(void) { return g_err.c_str(); }

void srp_trace_opts_default(srp_trace_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->rays_x = 1024; o->rays_y = 1024;
    o->max_bounces = 1;
    o->jitter = 1;
    o->seed = 0;
    o->pressure = 1.0;
    o->ray_offset = 0; o->ray_stride = 1; o->ray_count = 0;
    o->mem = SRP_MEM_DEVICE;
    o->sun_per_design = 0;
    o->block_threads = 0;
    o->chunks_per_item = 0;
}

int srp_ctx_create(srp_ctx** out, int device, void* cuda_stream) {
    if (!out) return fail(SRP_EINVAL, "srp_ctx_create: out is NULL");
    *out = nullptr;
    int n = 0;
    CU(cudaGetDeviceCount(&n), "cudaGetDeviceCount");
    if (device < 0 || device >= n) return fail(SRP_EINVAL, "srp_ctx_create: no such device");
    CU(cudaSetDevice(device), "cudaSetDevice");
    srp_ctx* c = new (std::nothrow) srp_ctx();
    if (!c) return fail(SRP_ENOMEM, "srp_ctx_create: out of host memory");
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) { delete c; return cuda_fail(e, "cudaGetDeviceProperties"); }
    c->n_sm = prop.multiProcessorCount;
    e = cudaMalloc((void**)&c->d_err, sizeof(int));
    if (e != cudaSuccess) { delete c; return cuda_fail(e, "cudaMalloc(err)"); }
    e = cudaMemset(c->d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_stats, 4 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_queue, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->tab_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemset(c->d_stats, 0, 4 * sizeof(unsigned long long));
    if (e != cudaSuccess) {
        if (c->tab_ev) cudaEventDestroy(c->tab_ev);
        if (c->d_queue) cudaFree(c->d_queue);
        if (c->d_stats) cudaFree(c->d_stats);
        cudaFree(c->d_err);
        delete c;
        return cuda_fail(e, "ctx set-up");
    }
    *out = c;
    return SRP_OK;
}

int srp_ctx_destroy(srp_ctx* c) {
    if (!c) return SRP_OK;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    c->part.release(); c->gpart.release(); c->stage_in.release(); c->stage_out.release(); c->dtab.release();
    c->atab.release(); c->axb.release(); c->span.release();
    if (c->htab) cudaFreeHost(c->htab);
    if (c->tab_ev) cudaEventDestroy(c->tab_ev);
    if (c->d_queue) cudaFree(c->d_queue);
    if (c->d_err) cudaFree(c->d_err);
    if (c->d_stats) cudaFree(c->d_stats);
    delete c;
    return SRP_OK;
}

int srp_sync(srp_ctx* c) {
    if (!c) return fail(SRP_EINVAL, "srp_sync: ctx is NULL");
    CU(cudaSetDevice(c->device), "cudaSetDevice");
    CU(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    int flag = 0;
    CU(cudaMemcpy(&flag, c->d_err, sizeof(int), cudaMemcpyDeviceToHost), "cudaMemcpy(err)");
    if (flag) {
        CU(cudaMemset(c->d_err, 0, sizeof(int)), "cudaMemset(err)");
        std::string what;
        if (flag & kErrStackOverflow) what += " traversal stack overflow;";
        if (flag & kErrVisitCap) what += " node-visit cap reached (corrupt BVH?);";
        if (flag & kErrAreaCount) what += " area-estimator sample count above its planned bound;";
        if (flag & kErrTriIndex) what += " triangle index outside the mesh (corrupt triangle table?);";
        if (flag & kErrRowIndex) what += " training batch index outside the data set (its rows read as zero);";
        if (flag & kErrWaitTimeout) what += " a bounded wait of a tensor-core kernel gave up;";
        // a wait that gave up alone is a timeout; any traversal or table limit takes precedence
        const int code = flag == kErrWaitTimeout ? SRP_ETIMEOUT : SRP_EDEVICE_LIMIT;
        return fail(code, "device limit:" + what);
    }
    return SRP_OK;
}

int srp_collect_stats(srp_ctx* c, int enable, uint64_t out[3]) {
    if (!c) return fail(SRP_EINVAL, "srp_collect_stats: ctx is NULL");
    CU(cudaSetDevice(c->device), "cudaSetDevice");
    if (out) {
        CU(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
        unsigned long long h[3];
        CU(cudaMemcpy(h, c->d_stats, sizeof h, cudaMemcpyDeviceToHost), "cudaMemcpy(stats)");
        for (int j = 0; j < 3; ++j) out[j] = (uint64_t)h[j];
    }
    CU(cudaMemset(c->d_stats, 0, 3 * sizeof(unsigned long long)), "cudaMemset(stats)");
    c->stats_on = enable != 0;
    return SRP_OK;
}

int srp_probe_read_bandwidth(srp_ctx* c, int64_t bytes, int passes, int reps, double* out_gbs) {
    if (!c || !out_gbs) return fail(SRP_EINVAL, "srp_probe_read_bandwidth: NULL ctx/out");
    *out_gbs = 0.0;
    if (bytes < 16 || passes < 1 || reps < 1)
        return fail(SRP_EINVAL, "srp_probe_read_bandwidth: bytes >= 16, passes >= 1 and reps >= 1 required");
    CU(cudaSetDevice(c->device), "cudaSetDevice");
    cudaError_t e = run_read_probe(bytes, passes, reps, c->stream, out_gbs);
    if (e == cudaErrorMemoryAllocation) return fail(SRP_ENOMEM, "srp_probe_read_bandwidth: device out of memory");
    if (e != cudaSuccess) return cuda_fail(e, "srp_probe_read_bandwidth");
    return SRP_OK;
}

int srp_design_instantiate(const float* vin, int V, const int32_t* vhinge, const double* hinges,
                           const double* angles, int H, float* vout) {
    if (V < 0 || H < 0) return fail(SRP_EINVAL, "srp_design_instantiate: negative size");
    if (V > 0 && (!vin || !vout)) return fail(SRP_EINVAL, "srp_design_instantiate: NULL vertices");
    if (H > 0 && (!vhinge || !hinges || !angles)) return fail(SRP_EINVAL, "srp_design_instantiate: NULL hinge data");
    std::vector<double> Rm(9 * (size_t)H);
    for (int h = 0; h < H; ++h) {
        const double* a = hinges + 6 * h + 3;
        const double nrm = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
        if (!(std::fabs(nrm - 1.0) < 1e-6)) return fail(SRP_EINVAL, "srp_design_instantiate: hinge axis not unit");
        const double c = std::cos(angles[h]), s = std::sin(angles[h]), t = 1.0 - c;
        const double x = a[0] / nrm, y = a[1] / nrm, z = a[2] / nrm;
        double* R = &Rm[9 * h];
        R[0] = c + x * x * t;     R[1] = x * y * t - z * s; R[2] = x * z * t + y * s;
        R[3] = y * x * t + z * s; R[4] = c + y * y * t;     R[5] = y * z * t - x * s;
        R[6] = z * x * t - y * s; R[7] = z * y * t + x * s; R[8] = c + z * z * t;
    }
    for (int v = 0; v < V; ++v) {
        const int h = H > 0 ? vhinge[v] : -1;
        if (h >= H) return fail(SRP_EINVAL, "srp_design_instantiate: hinge id out of range");
        if (h < 0) {
            if (vout != vin) for (int j = 0; j < 3; ++j) vout[3 * v + j] = vin[3 * v + j];
            continue;
        }
        const double* p = hinges + 6 * h;
        const double* R = &Rm[9 * h];
        const double q[3] = {vin[3 * v] - p[0], vin[3 * v + 1] - p[1], vin[3 * v + 2] - p[2]};
        for (int j = 0; j < 3; ++j)
            vout[3 * v + j] = (float)(p[j] + R[3 * j] * q[0] + R[3 * j + 1] * q[1] + R[3 * j + 2] * q[2]);
    }
    return SRP_OK;
}

int srp_build_bvh(srp_ctx* c, const float* verts, int V, const int32_t* tris, const int32_t* group, int T,
                  int width, srp_bvh** out) {
    if (!c || !out) return fail(SRP_EINVAL, "srp_build_bvh: NULL ctx/out");
    *out = nullptr;
    if (V < 0 || T < 0) return fail(SRP_EINVAL, "srp_build_bvh: negative size");
    if (T > 0 && (!verts || !tris || !group)) return fail(SRP_EINVAL, "srp_build_bvh: NULL arrays");
    if (T >= (1 << 28)) return fail(SRP_EINVAL, "srp_build_bvh: too many triangles (>= 2^28)");
    for (int t = 0; t < T; ++t)
        if (group[t] < 0 || group[t] >= kMaxGroups) return fail(SRP_EINVAL, "srp_build_bvh: group out of [0,64)");
    auto t0 = std::chrono::steady_clock::now();
    BuiltBVH b;
    std::string err;
    int rc = build_wide_bvh(verts, V, tris, T, width, &b, &err);
    if (rc != SRP_OK) return fail(rc, "srp_build_bvh: " + err);
    // grid: centre = vertex AABB centre, radius = max distance (FP64)
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int v = 0; v < V; ++v)
        for (int j = 0; j < 3; ++j) {
            lo[j] = std::min(lo[j], (double)verts[3 * v + j]);
            hi[j] = std::max(hi[j], (double)verts[3 * v + j]);
        }
    double cen[3] = {0, 0, 0}, R2 = 0.0;
    if (V > 0) {
        for (int j = 0; j < 3; ++j) cen[j] = 0.5 * (lo[j] + hi[j]);
        for (int v = 0; v < V; ++v) {
            double r2 = 0;
            for (int j = 0; j < 3; ++j) { double q = verts[3 * v + j] - cen[j]; r2 += q * q; }
            R2 = std::max(R2, r2);
        }
    }
    std::vector<float> tri(12 * (size_t)std::max(T, 1), 0.0f);
    for (int k = 0; k < T; ++k) {
        const int t = b.tri_order[k];
        for (int cidx = 0; cidx < 3; ++cidx)
            for (int j = 0; j < 3; ++j) tri[12 * k + 4 * cidx + j] = verts[3 * (size_t)tris[3 * t + cidx] + j];
        uint32_t id = (uint32_t)t, g = (uint32_t)group[t];
        std::memcpy(&tri[12 * k + 3], &id, 4);
        std::memcpy(&tri[12 * k + 7], &g, 4);
    }
    auto t1 = std::chrono::steady_clock::now();
    CU(cudaSetDevice(c->device), "cudaSetDevice");
    srp_bvh* h = new (std::nothrow) srp_bvh();
    if (!h) return fail(SRP_ENOMEM, "srp_build_bvh: out of host memory");
    h->device = c->device; h->width = width; h->T = T;
    h->max_group = -1;
    for (int t = 0; t < T; ++t) h->max_group = std::max(h->max_group, (int)group[t]);
    h->n_nodes = b.n_nodes; h->n_leaves = b.n_leaves; h->depth = b.depth;
    h->level_start = b.level_start;
    h->build_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    for (int j = 0; j < 3; ++j) h->c[j] = cen[j];
    h->R = std::sqrt(R2);
    h->area = 0.0;
    for (int t = 0; t < T; ++t) {
        const float* a = verts + 3 * (size_t)tris[3 * t];
        const float* b = verts + 3 * (size_t)tris[3 * t + 1];
        const float* q = verts + 3 * (size_t)tris[3 * t + 2];
        const double e1[3] = {(double)b[0] - a[0], (double)b[1] - a[1], (double)b[2] - a[2]};
        const double e2[3] = {(double)q[0] - a[0], (double)q[1] - a[1], (double)q[2] - a[2]};
        const double cx = e1[1] * e2[2] - e1[2] * e2[1], cy = e1[2] * e2[0] - e1[0] * e2[2],
                     cz = e1[0] * e2[1] - e1[1] * e2[0];
        h->area += 0.5 * std::sqrt(cx * cx + cy * cy + cz * cz);
    }
    const size_t tb = tri.size() * sizeof(float), nb = b.node_data.size() * sizeof(float);
    h->bytes = (int64_t)(tb + nb);
    cudaError_t e = cudaMalloc(&h->d_tri, tb);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_nodes, nb);
    if (e == cudaSuccess) e = cudaMemcpy(h->d_tri, tri.data(), tb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->d_nodes, b.node_data.data(), nb, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        if (h->d_tri) cudaFree(h->d_tri);
        if (h->d_nodes) cudaFree(h->d_nodes);
        delete h;
        return e == cudaErrorMemoryAllocation ? fail(SRP_ENOMEM, "srp_build_bvh: device out of memory")
                                              : cuda_fail(e, "srp_build_bvh upload");
    }
    *out = h;
    return SRP_OK;
}

int srp_build_bvh_host(const float* verts, int V, const int32_t* tris, int T, int width, float* node_data,
                       int64_t* n_node_floats, int32_t* tri_order, int32_t* n_nodes) {
    if (V < 0 || T < 0 || !n_node_floats || !n_nodes) return fail(SRP_EINVAL, "srp_build_bvh_host: bad arguments");
    if (T > 0 && (!verts || !tris)) return fail(SRP_EINVAL, "srp_build_bvh_host: NULL arrays");
    if (T >= (1 << 28)) return fail(SRP_EINVAL, "srp_build_bvh_host: too many triangles");
    BuiltBVH b;
    std::string err;
    int rc = build_wide_bvh(verts, V, tris, T, width, &b, &err);
    if (rc != SRP_OK) return fail(rc, "srp_build_bvh_host: " + err);
    if (!node_data) {
        *n_node_floats = (int64_t)b.node_data.size();
        *n_nodes = b.n_nodes;
        return SRP_OK;
    }
    if (*n_node_floats < (int64_t)b.node_data.size()) return fail(SRP_EINVAL, "srp_build_bvh_host: node buffer too small");
    std::memcpy(node_data, b.node_data.data(), sizeof(float) * b.node_data.size());
    if (tri_order && T > 0) std::memcpy(tri_order, b.tri_order.data(), sizeof(int32_t) * T);
    *n_node_floats = (int64_t)b.node_data.size();
    *n_nodes = b.n_nodes;
    return SRP_OK;
}

int srp_bvh_set_nodes(srp_ctx* c, srp_bvh* h, const float* node_data, int64_t n_floats) {
    if (!c || !h || !node_data) return fail(SRP_EINVAL, "srp_bvh_set_nodes: NULL argument");
    const int nf = h->width == 4 ? 32 : 64;
    if (n_floats != (int64_t)h->n_nodes * nf) return fail(SRP_EINVAL, "srp_bvh_set_nodes: size differs from the BVH's");
    const int W = h->width;
    for (int64_t n = 0; n < h->n_nodes; ++n) {
        const int32_t* ch = reinterpret_cast<const int32_t*>(node_data + n * nf + 6 * W);
        for (int k = 0; k < W; ++k) {
            const float lo = node_data[n * nf + k];  // lo_x of child k
            const float hi = node_data[n * nf + W + k];
            if (!(lo <= hi)) continue;  // empty slot (never traversed)
            const int32_t code = ch[k];
            if (code >= 0) {
                if (code >= h->n_nodes) return fail(SRP_EINVAL, "srp_bvh_set_nodes: inner child index out of range");
            } else {
                const int32_t d = ~code;
                const int64_t first = d >> 3, cnt = (d & 7) + 1;
                if (first + cnt > h->T) return fail(SRP_EINVAL, "srp_bvh_set_nodes: leaf range out of range");
            }
        }
    }
    CU(cudaSetDevice(h->device), "cudaSetDevice");
    CU(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    CU(cudaMemcpy(h->d_nodes, node_data, sizeof(float) * n_floats, cudaMemcpyHostToDevice), "H2D nodes");
    c->last_tab.clear();  // force a fresh design-table upload
    // breadth-first levels of the new tree, if its numbering is breadth
    // first (srp_bvh_refit needs that); otherwise none
    h->level_start.clear();
    {
        std::vector<int32_t> depth(h->n_nodes, -1);
        std::vector<int32_t> queue = {0};
        depth[0] = 0;
        bool ok = true;
        for (size_t qi = 0; qi < queue.size() && ok; ++qi) {
            const int32_t n = queue[qi];
            const int32_t* ch = reinterpret_cast<const int32_t*>(node_data + (int64_t)n * nf + 6 * W);
            for (int k = 0; k < W; ++k) {
                if (!(node_data[(int64_t)n * nf + k] <= node_data[(int64_t)n * nf + W + k]) || ch[k] < 0) continue;
                if (depth[ch[k]] >= 0) { ok = false; break; }   // shared child or cycle
                depth[ch[k]] = depth[n] + 1;
                queue.push_back(ch[k]);
            }
        }
        for (int32_t n = 1; n < h->n_nodes && ok; ++n)
            if (depth[n] < depth[n - 1]) ok = false;   // unreachable (-1) or not breadth first
        if (ok) {
            for (int32_t n = 0; n < h->n_nodes; ++n)
                if (n == 0 || depth[n] != depth[n - 1]) h->level_start.push_back(n);
            h->level_start.push_back(h->n_nodes);
        }
    }
    return SRP_OK;
}

int srp_bvh_refit(srp_ctx* c, srp_bvh* h, const float* verts, int V, const int32_t* tris, int T) {
    if (!c || !h) return fail(SRP_EINVAL, "srp_bvh_refit: NULL ctx/bvh");
    if (V < 0 || T != h->T) return fail(SRP_EINVAL, "srp_bvh_refit: T differs from the BVH's (or V < 0)");
    if (T > 0 && (!verts || !tris)) return fail(SRP_EINVAL, "srp_bvh_refit: NULL arrays");
    if (h->level_start.size() < 2)
        return fail(SRP_EUNSUPPORTED, "srp_bvh_refit: the node array was replaced by one not numbered breadth first");
    // the builder's checks and its padding scale (over the triangles' vertices)
    float scale = 0.0f;
    for (int t = 0; t < T; ++t)
        for (int k = 0; k < 3; ++k) {
            const int v = tris[3 * (size_t)t + k];
            if (v < 0 || v >= V) return fail(SRP_EINVAL, "srp_bvh_refit: triangle vertex index out of range");
            for (int j = 0; j < 3; ++j) {
                const float x = verts[3 * (size_t)v + j];
                if (!std::isfinite(x)) return fail(SRP_EINVAL, "srp_bvh_refit: non-finite vertex coordinate");
                scale = std::max(scale, std::fabs(x));
            }
        }
    const float pad_abs = 1e-6f * (scale + 1e-3f);
    // grid centre and radius over all vertices, surface area (FP64), as srp_build_bvh
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int v = 0; v < V; ++v)
        for (int j = 0; j < 3; ++j) {
            lo[j] = std::min(lo[j], (double)verts[3 * (size_t)v + j]);
            hi[j] = std::max(hi[j], (double)verts[3 * (size_t)v + j]);
        }
    double cen[3] = {0, 0, 0}, R2 = 0.0;
    if (V > 0) {
        for (int j = 0; j < 3; ++j) cen[j] = 0.5 * (lo[j] + hi[j]);
        for (int v = 0; v < V; ++v) {
            double r2 = 0;
            for (int j = 0; j < 3; ++j) { const double q = verts[3 * (size_t)v + j] - cen[j]; r2 += q * q; }
            R2 = std::max(R2, r2);
        }
    }
    double area = 0.0;
    for (int t = 0; t < T; ++t) {
        const float* a = verts + 3 * (size_t)tris[3 * t];
        const float* b = verts + 3 * (size_t)tris[3 * t + 1];
        const float* q = verts + 3 * (size_t)tris[3 * t + 2];
        const double e1[3] = {(double)b[0] - a[0], (double)b[1] - a[1], (double)b[2] - a[2]};
        const double e2[3] = {(double)q[0] - a[0], (double)q[1] - a[1], (double)q[2] - a[2]};
        const double cx = e1[1] * e2[2] - e1[2] * e2[1], cy = e1[2] * e2[0] - e1[0] * e2[2],
                     cz = e1[0] * e2[1] - e1[1] * e2[0];
        area += 0.5 * std::sqrt(cx * cx + cy * cy + cz * cz);
    }
    CU(cudaSetDevice(h->device), "cudaSetDevice");
    float* d_v = nullptr;
    int32_t* d_t = nullptr;
    const size_t vb = sizeof(float) * 3 * (size_t)std::max(V, 1), tb = sizeof(int32_t) * 3 * (size_t)std::max(T, 1);
    cudaError_t e = cudaMallocAsync((void**)&d_v, vb, c->stream);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&d_t, tb, c->stream);
    if (e == cudaSuccess && V > 0) e = cudaMemcpyAsync(d_v, verts, sizeof(float) * 3 * (size_t)V, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && T > 0) e = cudaMemcpyAsync(d_t, tris, sizeof(int32_t) * 3 * (size_t)T, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = launch_refit(h, d_v, d_t, pad_abs, c->stream);
    if (d_v) cudaFreeAsync(d_v, c->stream);
    if (d_t) cudaFreeAsync(d_t, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "srp_bvh_refit");
    for (int j = 0; j < 3; ++j) h->c[j] = cen[j];
    h->R = std::sqrt(R2);
    h->area = area;
    c->last_tab.clear();  // the design table carries c and R
    return SRP_OK;
}

int srp_bvh_destroy(srp_bvh* h) {
    if (!h) return SRP_OK;
    cudaSetDevice(h->device);
    if (h->d_tri) cudaFree(h->d_tri);
    if (h->d_nodes) cudaFree(h->d_nodes);
    delete h;
    return SRP_OK;
}

int srp_bvh_get_info(const srp_bvh* h, srp_bvh_info* info) {
    if (!h || !info) return fail(SRP_EINVAL, "srp_bvh_get_info: NULL argument");
    info->width = h->width; info->n_nodes = h->n_nodes; info->n_leaves = h->n_leaves;
    info->depth = h->depth; info->n_tris = h->T;
    info->device_bytes = h->bytes; info->build_ms = h->build_ms;
    for (int j = 0; j < 3; ++j) info->center[j] = h->c[j];
    info->radius = h->R;
    return SRP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// srp_force
// ---------------------------------------------------------------------------
namespace {

int validate_values(const float* rho, int D, int G, const double* sun, int64_t nsun) {
    for (int64_t q = 0; q < (int64_t)D * G; ++q) {
        const float rs = rho[2 * q], rd = rho[2 * q + 1];
        if (!(rs >= 0.0f && rs <= 1.0f && rd >= 0.0f && rd <= 1.0f && rs + rd <= 1.0f + 1e-6f))
            return fail(SRP_EINVAL, "srp_force: reflectances must satisfy 0 <= rho_s, rho_d and rho_s + rho_d <= 1");
    }
    for (int64_t s = 0; s < nsun; ++s) {
        const double* e = sun + 3 * s;
        const double nn = std::sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
        if (!(std::fabs(nn - 1.0) < 1e-6)) return fail(SRP_EINVAL, "srp_force: sun_dir must be unit vectors");
    }
    return SRP_OK;
}

}  // namespace

// Shared by srp_force and its variants: everything but memory placement.
namespace srp {
int force_plan(srp_ctx* c, const srp_bvh* const* bvhs, int D, int G, int S, const srp_trace_opts* o,
               std::vector<DesignDev>* designs, TraceParams* p, int* width, int* block, int* grid_cap) {
    if (o && o->kernel_variant != 0 && (o->kernel_variant < 4 || o->kernel_variant > 8))
        return fail(SRP_EINVAL, "srp_force: kernel_variant must be 0, 4, 5, 6, 7 or 8");
    const int variant = (o && o->kernel_variant) ? o->kernel_variant : 7;
    if (!c || !o) return fail(SRP_EINVAL, "srp_force: NULL ctx/opts");
    if (D < 0 || S < 0) return fail(SRP_EINVAL, "srp_force: negative D or S");
    if (G < 1 || G > kMaxGroups) return fail(SRP_EINVAL, "srp_force: G must be in 1..64");
    if (o->rays_x < 1 || o->rays_y < 1) return fail(SRP_EINVAL, "srp_force: rays_x/rays_y must be >= 1");
    const int64_t grid_n = (int64_t)o->rays_x * o->rays_y;
    if (grid_n > 0xffffffffLL) return fail(SRP_EINVAL, "srp_force: rays_x*rays_y must be < 2^32");
    if (o->max_bounces < 1 || o->max_bounces > kMaxBounces) return fail(SRP_EINVAL, "srp_force: max_bounces must be 1..3");
    if (!(o->pressure >= 0.0) || !std::isfinite(o->pressure)) return fail(SRP_EINVAL, "srp_force: bad pressure");
    int64_t n = o->ray_count, off = o->ray_offset, stride = o->ray_stride;
    if (n == 0) { n = grid_n; off = 0; stride = 1; }
    if (n < 0 || off < 0 || stride < 1 || off + (n - 1) * stride >= grid_n)
        return fail(SRP_EINVAL, "srp_force: ray subset outside the grid");
    int w = 0;
    designs->resize(D);
    for (int d = 0; d < D; ++d) {
        const srp_bvh* h = bvhs ? bvhs[d] : nullptr;
        if (!h) return fail(SRP_EINVAL, "srp_force: NULL bvh");
        if (h->device != c->device) return fail(SRP_EINVAL, "srp_force: bvh built on another device");
        if (w == 0) w = h->width;
        if (h->width != w) return fail(SRP_EUNSUPPORTED, "srp_force: all designs of one call need the same BVH width");
        if (h->max_group >= G)
            return fail(SRP_EINVAL, "srp_force: design " + std::to_string(d) + " uses material group " +
                                        std::to_string(h->max_group) + " but rho has G = " + std::to_string(G) + " groups");
        DesignDev& dz = (*designs)[d];
        dz.tri = (const float4*)h->d_tri; dz.nodes = (const float4*)h->d_nodes;
        dz.cx = h->c[0]; dz.cy = h->c[1]; dz.cz = h->c[2]; dz.R = h->R;
        dz.T = h->T; dz.width = h->width;
    }
    *width = w ? w : 4;
    int bt = o->block_threads ? o->block_threads : 128;
    if (bt != 128) return fail(SRP_EINVAL, "srp_force: block_threads must be 0 or 128");
    *block = bt;
    const int64_t items = (int64_t)D * S;
    int64_t cpb = o->chunks_per_item;
    if (cpb < 0) return fail(SRP_EINVAL, "srp_force: negative chunks_per_item");
    if (cpb == 0) {
        // Enough chunks per item that the resident warps (which take units in
        // order) work on a few (design, sun) items at a time: rays of one
        // direction share BVH nodes in L1 (a mix of many directions per SM
        // thrashed it, 2x slower), while longer units spend less on their
        // set-up (item constants, the span row search, partials).  One unit
        // per four resident warps measured fastest on the satellite (1,024
        // units per item: +1.9 % rays/s at K <= 3 and +4.3 % at K = 1 over
        // one per warp; 512 the same; 8,192 -2 % / -7 %).  At least ~40k
        // units for balance; at most 16M units of partials (1.5 GB); chunks
        // of at least 256 rays.
        const int64_t warps = (int64_t)c->n_sm * trace_resident_blocks(w ? w : 4, bt, variant) * (bt / 32);
        cpb = items > 0 ? std::max<int64_t>((40960 + items - 1) / items, warps / 4) : 1;
        if (items > 0) cpb = std::min<int64_t>(cpb, std::max<int64_t>(1, (int64_t)16777216 / items));
        cpb = std::max<int64_t>(1, std::min<int64_t>(cpb, (n + 255) / 256));
    }
    int64_t chunk = (n + cpb - 1) / cpb;
    chunk = std::max<int64_t>(64, (chunk + 63) / 64 * 64);
    cpb = std::max<int64_t>(1, (n + chunk - 1) / chunk);
    p->D = D; p->S = S; p->G = G;
    p->nx = o->rays_x; p->ny = o->rays_y; p->K = o->max_bounces; p->jitter = o->jitter ? 1 : 0;
    p->sun_per_design = o->sun_per_design ? 1 : 0;
    p->seed = o->seed; p->P = o->pressure;
    p->off = off; p->stride = stride; p->n = n;
    p->sun_base = o->sun_base; p->design_base = o->design_base;
    p->chunk = chunk; p->cpb = (int32_t)cpb;
    p->err = c->d_err;
    p->stats = c->stats_on ? c->d_stats : nullptr;
    p->variant = variant;
    p->queue = c->d_queue;
    *grid_cap = c->n_sm * trace_resident_blocks(*width, bt, variant);
    // full grids of whole 32-pixel batches: trace only the batches that can
    // meet the scene (span_kernel); the tables need items * (2 ny + 1) int32
    // (up to 4 GiB: 256 designs x 1024 suns x 1024 rows take 2.1 GB)
    p->rowfirst = nullptr;
    p->rowoff = nullptr;
    const size_t row_bytes = (sizeof(int32_t) * (size_t)items * (2 * (size_t)o->rays_y + 1) + 255) / 256 * 256;
    const size_t span_bytes = row_bytes + 8 * sizeof(float4) * (size_t)items;
    if (items > 0 && off == 0 && stride == 1 && n == grid_n && o->rays_x % 32 == 0 && span_bytes <= ((size_t)4 << 30)) {
        if (c->span.ensure(span_bytes) != cudaSuccess) return fail(SRP_ENOMEM, "srp_force: cannot allocate the span tables");
        p->rowfirst = (int32_t*)c->span.p;
        p->rowoff = p->rowfirst + (size_t)items * o->rays_y;
        p->itab = (float4*)((char*)c->span.p + row_bytes);
        p->bh = span_batch_rows(o->rays_y);
    }
    return SRP_OK;
}

// Put the design table on the device (skipped when unchanged since the
// previous call); the pinned staging buffer is reused only after its
// previous upload has completed.
int upload_designs(srp_ctx* c, const std::vector<DesignDev>& designs) {
    const size_t n = designs.size();
    if (n == 0) return SRP_OK;
    if (c->last_tab.size() == n && std::memcmp(c->last_tab.data(), designs.data(), n * sizeof(DesignDev)) == 0)
        return SRP_OK;
    CU(cudaEventSynchronize(c->tab_ev), "cudaEventSynchronize");
    if (c->htab_n < n) {
        if (c->htab) cudaFreeHost(c->htab);
        c->htab = nullptr; c->htab_n = 0;
        CU(cudaMallocHost((void**)&c->htab, n * sizeof(DesignDev)), "cudaMallocHost(design table)");
        c->htab_n = n;
    }
    if (c->dtab.ensure(n * sizeof(DesignDev)) != cudaSuccess) return fail(SRP_ENOMEM, "srp_force: design table");
    std::memcpy(c->htab, designs.data(), n * sizeof(DesignDev));
    CU(cudaMemcpyAsync(c->dtab.p, c->htab, n * sizeof(DesignDev), cudaMemcpyHostToDevice, c->stream), "H2D designs");
    CU(cudaEventRecord(c->tab_ev, c->stream), "cudaEventRecord");
    c->last_tab = designs;
    return SRP_OK;
}

// Stream work of one evaluation: queue reset, trace, reduce (on `st`).
int force_enqueue(TraceParams& p, int width, int block, int grid_cap, double* d_part, double* d_ft,
                  double* d_sigma, cudaStream_t st) {
    p.part = d_part;
    const int64_t items = (int64_t)p.D * p.S;
    if (items == 0 || p.n == 0) {
        if (items > 0) {
            CU(cudaMemsetAsync(d_ft, 0, sizeof(double) * 6 * items, st), "cudaMemsetAsync");
            if (d_sigma) CU(cudaMemsetAsync(d_sigma, 0, sizeof(double) * 6 * items, st), "cudaMemsetAsync");
        }
        return SRP_OK;
    }
    CU(cudaMemsetAsync(p.queue, 0, sizeof(unsigned long long), st), "cudaMemsetAsync(queue)");
    if (p.rowoff) CU(launch_span(p, width, st), "span_kernel launch");
    CU(launch_trace(p, width, grid_cap, block, st), "trace_kernel launch");
    CU(launch_reduce(d_part, items, p.cpb, d_ft, d_sigma, st), "reduce kernel launch");
    return SRP_OK;
}

int force_launch(srp_ctx* c, const std::vector<DesignDev>& designs, TraceParams& p, int width, int block,
                 int grid_cap, double* d_part, double* d_ft, double* d_sigma) {
    int rc = upload_designs(c, designs);
    if (rc != SRP_OK) return rc;
    p.designs = (const DesignDev*)c->dtab.p;
    return force_enqueue(p, width, block, grid_cap, d_part, d_ft, d_sigma, c->stream);
}
}  // namespace srp

extern "C" int srp_force(srp_ctx* c, const srp_bvh* const* bvhs, int D, const float* rho, int G,
                         const double* sun_dir, int S, const double* com, const srp_trace_opts* o,
                         double* out_ft, double* out_sigma) {
    std::vector<DesignDev> designs;
    TraceParams p;
    std::memset(&p, 0, sizeof p);
    int width, block, grid_cap;
    int rc = force_plan(c, bvhs, D, G, S, o, &designs, &p, &width, &block, &grid_cap);
    if (rc != SRP_OK) return rc;
    const int64_t items = (int64_t)D * S;
    if (items > 0 && (!rho || !sun_dir || !com || !out_ft))
        return fail(SRP_EINVAL, "srp_force: NULL array argument");
    CU(cudaSetDevice(c->device), "cudaSetDevice");
    const size_t part_bytes = sizeof(double) * 12 * (size_t)std::max<int64_t>(items * p.cpb, 1);
    cudaError_t e = c->part.ensure(part_bytes);
    if (e != cudaSuccess) return fail(SRP_ENOMEM, "srp_force: cannot allocate partials");
    const int64_t nsun = o->sun_per_design ? (int64_t)D * S : S;
    if (o->mem == SRP_MEM_DEVICE) {
        p.rho = rho; p.sun = sun_dir; p.com = com;
        return force_launch(c, designs, p, width, block, grid_cap, (double*)c->part.p, out_ft, out_sigma);
    }
    if (o->mem != SRP_MEM_HOST) return fail(SRP_EINVAL, "srp_force: mem must be SRP_MEM_HOST or SRP_MEM_DEVICE");
    if (items > 0) {
        rc = validate_values(rho, D, G, sun_dir, nsun);
        if (rc != SRP_OK) return rc;
    }
    // stage: rho | sun | com  and  ft | sigma
    const size_t rb = sizeof(float) * 2 * (size_t)D * G, sb = sizeof(double) * 3 * (size_t)nsun,
                 cb = sizeof(double) * 3 * (size_t)D;
    const size_t rb_al = (rb + 255) / 256 * 256, sb_al = (sb + 255) / 256 * 256;
    if (c->stage_in.ensure(rb_al + sb_al + cb + 256) != cudaSuccess) return fail(SRP_ENOMEM, "srp_force: staging");
    const size_t ob = sizeof(double) * 6 * (size_t)items;
    const size_t ob_al = (ob + 255) / 256 * 256;
    if (c->stage_out.ensure(2 * ob_al + 256) != cudaSuccess) return fail(SRP_ENOMEM, "srp_force: staging");
    char* in = (char*)c->stage_in.p;
    char* outb = (char*)c->stage_out.p;
    if (items > 0) {
        CU(cudaMemcpyAsync(in, rho, rb, cudaMemcpyHostToDevice, c->stream), "H2D rho");
        CU(cudaMemcpyAsync(in + rb_al, sun_dir, sb, cudaMemcpyHostToDevice, c->stream), "H2D sun");
        CU(cudaMemcpyAsync(in + rb_al + sb_al, com, cb, cudaMemcpyHostToDevice, c->stream), "H2D com");
    }
    p.rho = (const float*)in; p.sun = (const double*)(in + rb_al); p.com = (const double*)(in + rb_al + sb_al);
    double* d_ft = (double*)outb;
    double* d_sg = out_sigma ? (double*)(outb + ob_al) : nullptr;
    rc = force_launch(c, designs, p, width, block, grid_cap, (double*)c->part.p, d_ft, d_sg);
    if (rc != SRP_OK) return rc;
    if (items > 0) {
        CU(cudaMemcpyAsync(out_ft, d_ft, ob, cudaMemcpyDeviceToHost, c->stream), "D2H ft");
        if (out_sigma) CU(cudaMemcpyAsync(out_sigma, d_sg, ob, cudaMemcpyDeviceToHost, c->stream), "D2H sigma");
    }
    return srp_sync(c);
}

extern "C" int srp_trace_rays(srp_ctx* c, const srp_bvh* bvh, const float* rho, int G, const double* sun_dir,
                              const double* com, const int64_t* ray_idx, int64_t n, int sun_index,
                              int design_index, const srp_trace_opts* o, double* out_y, int32_t* out_hits) {
    if (!o) return fail(SRP_EINVAL, "srp_trace_rays: NULL opts");
    srp_trace_opts oo = *o;
    oo.ray_offset = 0; oo.ray_stride = 1; oo.ray_count = 0; oo.sun_per_design = 0;
    std::vector<DesignDev> designs;
    TraceParams p;
    std::memset(&p, 0, sizeof p);
    int width, block, grid_cap;
    const srp_bvh* one[1] = {bvh};
    int rc = force_plan(c, one, 1, G, 1, &oo, &designs, &p, &width, &block, &grid_cap);
    if (rc != SRP_OK) return rc;
    if (n < 0) return fail(SRP_EINVAL, "srp_trace_rays: negative n");
    if (n == 0) return SRP_OK;
    if (!rho || !sun_dir || !com || !ray_idx || !out_y || !out_hits) return fail(SRP_EINVAL, "srp_trace_rays: NULL array");
    CU(cudaSetDevice(c->device), "cudaSetDevice");
    const int64_t grid_n = (int64_t)o->rays_x * o->rays_y;
    const int K = o->max_bounces;
    if (o->mem == SRP_MEM_DEVICE) {
        p.rho = rho; p.sun = sun_dir; p.com = com;
        CU(launch_trace_rays(designs[0], p, ray_idx, n, sun_index, design_index, out_y, out_hits, c->stream),
           "trace_rays launch");
        return SRP_OK;
    }
    for (int64_t q = 0; q < n; ++q)
        if (ray_idx[q] < 0 || ray_idx[q] >= grid_n) return fail(SRP_EINVAL, "srp_trace_rays: ray index outside the grid");
    rc = validate_values(rho, 1, G, sun_dir, 1);
    if (rc != SRP_OK) return rc;
    const size_t rb = 256 * ((sizeof(float) * 2 * G + 255) / 256), sb = 256, cb = 256;
    const size_t ib = 256 * ((sizeof(int64_t) * n + 255) / 256);
    const size_t yb = 256 * ((sizeof(double) * 6 * n + 255) / 256), hb = sizeof(int32_t) * K * n;
    if (c->stage_in.ensure(rb + sb + cb + ib) != cudaSuccess) return fail(SRP_ENOMEM, "srp_trace_rays: staging");
    if (c->stage_out.ensure(yb + hb + 256) != cudaSuccess) return fail(SRP_ENOMEM, "srp_trace_rays: staging");
    char* in = (char*)c->stage_in.p;
    char* ob = (char*)c->stage_out.p;
    CU(cudaMemcpyAsync(in, rho, sizeof(float) * 2 * G, cudaMemcpyHostToDevice, c->stream), "H2D");
    CU(cudaMemcpyAsync(in + rb, sun_dir, 3 * sizeof(double), cudaMemcpyHostToDevice, c->stream), "H2D");
    CU(cudaMemcpyAsync(in + rb + sb, com, 3 * sizeof(double), cudaMemcpyHostToDevice, c->stream), "H2D");
    CU(cudaMemcpyAsync(in + rb + sb + cb, ray_idx, sizeof(int64_t) * n, cudaMemcpyHostToDevice, c->stream), "H2D");
    p.rho = (const float*)in; p.sun = (const double*)(in + rb); p.com = (const double*)(in + rb + sb);
    CU(launch_trace_rays(designs[0], p, (const int64_t*)(in + rb + sb + cb), n, sun_index, design_index,
                         (double*)ob, (int32_t*)(ob + yb), c->stream), "trace_rays launch");
    CU(cudaMemcpyAsync(out_y, ob, sizeof(double) * 6 * n, cudaMemcpyDeviceToHost, c->stream), "D2H");
    CU(cudaMemcpyAsync(out_hits, ob + yb, hb, cudaMemcpyDeviceToHost, c->stream), "D2H");
    return srp_sync(c);
}

extern "C" int srp_force_grad(srp_ctx* c, const srp_bvh* bvh, const float* rho, int G, const double* sun_dir, int S,
                              const double* com, const int32_t* tri_hinge, const double* hinge_axes, int H,
                              const srp_trace_opts* o, const double* upstream, double* d_rho, double* d_hinge) {
    if (!o) return fail(SRP_EINVAL, "srp_force_grad: NULL opts");
    if (H < 0 || H > 8) return fail(SRP_EINVAL, "srp_force_grad: H must be in 0..8");
    if (H > 0 && (!tri_hinge || !hinge_axes || !d_hinge)) return fail(SRP_EINVAL, "srp_force_grad: NULL hinge arrays");
    srp_trace_opts oo = *o;
    oo.sun_per_design = 0;
    std::vector<DesignDev> designs;
    TraceParams p;
    std::memset(&p, 0, sizeof p);
    int width, block, grid_cap;
    const srp_bvh* one[1] = {bvh};
    if (oo.chunks_per_item == 0) {
        const int64_t grid_n = (int64_t)o->rays_x * o->rays_y;
        const int64_t n = o->ray_count > 0 ? o->ray_count : grid_n;
        int64_t cpb = S > 0 ? (8192 + S - 1) / S : 1;
        cpb = std::max<int64_t>(1, std::min<int64_t>(cpb, (n + 255) / 256));
        oo.chunks_per_item = (int32_t)cpb;
    }
    int rc = force_plan(c, one, 1, G, S, &oo, &designs, &p, &width, &block, &grid_cap);
    if (rc != SRP_OK) return rc;
    if (S > 0 && (!rho || !sun_dir || !com || !upstream || !d_rho))
        return fail(SRP_EINVAL, "srp_force_grad: NULL array argument");
    CU(cudaSetDevice(c->device), "cudaSetDevice");
    if (p.rowoff) {   // the span pre-pass reads the design from the device table
        rc = upload_designs(c, designs);
        if (rc != SRP_OK) return rc;
        p.designs = (const DesignDev*)c->dtab.p;
    }
    const int ng = 2 * G + H;
    const int64_t units = (int64_t)S * p.cpb;
    if (c->gpart.ensure(sizeof(double) * ng * (size_t)std::max<int64_t>(units, 1)) != cudaSuccess)
        return fail(SRP_ENOMEM, "srp_force_grad: cannot allocate gradient partials");
    if (o->mem == SRP_MEM_DEVICE) {
        p.rho = rho; p.sun = sun_dir; p.com = com;
        CU(launch_grad(designs[0], p, upstream, tri_hinge, hinge_axes, H, (double*)c->gpart.p, d_rho, d_hinge,
                       c->n_sm, c->stream), "grad kernel launch");
        return SRP_OK;
    }
    if (o->mem != SRP_MEM_HOST) return fail(SRP_EINVAL, "srp_force_grad: mem must be SRP_MEM_HOST or SRP_MEM_DEVICE");
    if (S > 0) {
        rc = validate_values(rho, 1, G, sun_dir, S);
        if (rc != SRP_OK) return rc;
    }
    for (int h = 0; h < H; ++h) {
        const double* a = hinge_axes + 6 * h + 3;
        if (!(std::fabs(std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]) - 1.0) < 1e-6))
            return fail(SRP_EINVAL, "srp_force_grad: hinge axes must be unit vectors");
    }
    const int T = bvh->T;
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t rb = al(sizeof(float) * 2 * G), sb = al(sizeof(double) * 3 * S), cb = al(sizeof(double) * 3),
                 ub = al(sizeof(double) * 6 * S), tb = al(sizeof(int32_t) * std::max(T, 1)),
                 hb = al(sizeof(double) * 6 * std::max(H, 1));
    if (c->stage_in.ensure(rb + sb + cb + ub + tb + hb) != cudaSuccess) return fail(SRP_ENOMEM, "srp_force_grad: staging");
    if (c->stage_out.ensure(al(sizeof(double) * ng) + 256) != cudaSuccess) return fail(SRP_ENOMEM, "srp_force_grad: staging");
    char* in = (char*)c->stage_in.p;
    char* ob = (char*)c->stage_out.p;
    size_t off = 0;
    auto put = [&](const void* src, size_t bytes, size_t slot) -> char* {
        char* dst = in + off;
        if (bytes) cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream);
        off += slot;
        return dst;
    };
    p.rho = (const float*)put(rho, sizeof(float) * 2 * G, rb);
    p.sun = (const double*)put(sun_dir, sizeof(double) * 3 * S, sb);
    p.com = (const double*)put(com, sizeof(double) * 3, cb);
    const double* d_up = (const double*)put(upstream, sizeof(double) * 6 * S, ub);
    const int32_t* d_th = H > 0 ? (const int32_t*)put(tri_hinge, sizeof(int32_t) * T, tb) : nullptr;
    if (H == 0) off += tb;
    const double* d_hx = H > 0 ? (const double*)put(hinge_axes, sizeof(double) * 6 * H, hb) : nullptr;
    CU(cudaGetLastError(), "H2D staging");
    double* dr = (double*)ob;
    double* dh = H > 0 ? dr + 2 * G : nullptr;
    CU(launch_grad(designs[0], p, d_up, d_th, d_hx, H, (double*)c->gpart.p, dr, dh, c->n_sm, c->stream),
       "grad kernel launch");
    CU(cudaMemcpyAsync(d_rho, dr, sizeof(double) * 2 * G, cudaMemcpyDeviceToHost, c->stream), "D2H d_rho");
    if (H > 0) CU(cudaMemcpyAsync(d_hinge, dh, sizeof(double) * H, cudaMemcpyDeviceToHost, c->stream), "D2H d_hinge");
    return srp_sync(c);
}

// Context internals for other translation units of the library.
namespace srp {
cudaStream_t ctx_stream(srp_ctx* c) { return c->stream; }
int ctx_device(srp_ctx* c) { return c->device; }
int* ctx_err(srp_ctx* c) { return c->d_err; }
int ctx_n_sm(srp_ctx* c) { return c->n_sm; }
}  // namespace srp

// ---------------------------------------------------------------------------
// CUDA graph of one srp_force evaluation (device memory)
// ---------------------------------------------------------------------------
struct srp_graph {
    srp_ctx* ctx = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    void* dtab = nullptr;  // the graph's own design table
};

extern "C" int srp_force_graph_create(srp_ctx* c, const srp_bvh* const* bvhs, int D, const float* rho, int G,
                                      const double* sun_dir, int S, const double* com, const srp_trace_opts* o,
                                      double* out_ft, double* out_sigma, srp_graph** out) {
    if (!out) return fail(SRP_EINVAL, "srp_force_graph_create: NULL out");
    *out = nullptr;
    if (!o || o->mem != SRP_MEM_DEVICE) return fail(SRP_EINVAL, "srp_force_graph_create: needs device memory (mem = SRP_MEM_DEVICE)");
    std::vector<DesignDev> designs;
    TraceParams p;
    std::memset(&p, 0, sizeof p);
    int width, block, grid_cap;
    int rc = force_plan(c, bvhs, D, G, S, o, &designs, &p, &width, &block, &grid_cap);
    if (rc != SRP_OK) return rc;
    const int64_t items = (int64_t)D * S;
    if (items > 0 && (!rho || !sun_dir || !com || !out_ft)) return fail(SRP_EINVAL, "srp_force_graph_create: NULL array");
    CU(cudaSetDevice(c->device), "cudaSetDevice");
    if (c->part.ensure(sizeof(double) * 12 * (size_t)std::max<int64_t>(items * p.cpb, 1)) != cudaSuccess)
        return fail(SRP_ENOMEM, "srp_force_graph_create: partials");
    srp_graph* g = new (std::nothrow) srp_graph();
    if (!g) return fail(SRP_ENOMEM, "srp_force_graph_create: host memory");
    g->ctx = c;
    const size_t tb = std::max<size_t>(designs.size(), 1) * sizeof(DesignDev);
    cudaError_t e = cudaMalloc(&g->dtab, tb);
    if (e == cudaSuccess && !designs.empty())
        e = cudaMemcpy(g->dtab, designs.data(), designs.size() * sizeof(DesignDev), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaFree(g->dtab); delete g; return cuda_fail(e, "srp_force_graph_create: design table"); }
    p.rho = rho; p.sun = sun_dir; p.com = com;
    p.designs = (const DesignDev*)g->dtab;
    // capture on a private stream (the context's may be the legacy default
    // stream, which cannot be captured); the graph is launched on the
    // context's stream
    cudaStream_t cap = nullptr;
    e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        if (cap) cudaStreamDestroy(cap);
        cudaFree(g->dtab); delete g;
        return cuda_fail(e, "cudaStreamBeginCapture");
    }
    rc = force_enqueue(p, width, block, grid_cap, (double*)c->part.p, out_ft, out_sigma, cap);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(cap, &graph);
    cudaStreamDestroy(cap);
    if (rc != SRP_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaFree(g->dtab); delete g;
        return rc != SRP_OK ? rc : cuda_fail(e, "cudaStreamEndCapture");
    }
    g->graph = graph;
    e = cudaGraphInstantiate(&g->exec, graph, 0);
    if (e != cudaSuccess) { cudaGraphDestroy(graph); cudaFree(g->dtab); delete g; return cuda_fail(e, "cudaGraphInstantiate"); }
    *out = g;
    return SRP_OK;
}

extern "C" int srp_graph_launch(srp_graph* g) {
    if (!g) return fail(SRP_EINVAL, "srp_graph_launch: NULL graph");
    CU(cudaSetDevice(g->ctx->device), "cudaSetDevice");
    CU(cudaGraphLaunch(g->exec, g->ctx->stream), "cudaGraphLaunch");
    return SRP_OK;
}

extern "C" int srp_graph_destroy(srp_graph* g) {
    if (!g) return SRP_OK;
    cudaSetDevice(g->ctx->device);
    cudaStreamSynchronize(g->ctx->stream);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->dtab) cudaFree(g->dtab);
    delete g;
    return SRP_OK;
}

// ---------------------------------------------------------------------------
// srp_force_area: surface sampling with next-event estimation (area.cu)
// ---------------------------------------------------------------------------
namespace {
// Shared host side of srp_force_area (mode 0) and srp_force_thermal (mode 1;
// S = 1, no sun directions, emit [D][G]).
int area_common(srp_ctx* c, int mode, const srp_bvh* const* bvhs, int D, const float* rho, int G,
                const double* sun_dir, int S, const double* com, const float* emit, float density,
                const srp_trace_opts* o, double* out_ft, double* out_sigma, int64_t* out_samples) {
    const std::string fn = mode == 1 ? "srp_force_thermal" : "srp_force_area";
    if (!c || !o) return fail(SRP_EINVAL, fn + ": NULL ctx/opts");
    if (D < 0 || S < 0) return fail(SRP_EINVAL, fn + ": negative D or S");
    if (D > kMaxDesignsPerLaunch) return fail(SRP_EINVAL, fn + ": too many designs in one call");
    if (G < 1 || G > kMaxGroups) return fail(SRP_EINVAL, fn + ": G must be in 1..64");
    if (mode == 1 && o->max_bounces != 1)
        return fail(SRP_EUNSUPPORTED, fn + ": thermal packets deposit at their first hit (max_bounces = 1)");
    if (mode == 0 && o->max_bounces != 1 && o->max_bounces != 2)
        return fail(SRP_EUNSUPPORTED, fn + ": max_bounces must be 1 (direct light) or 2 (plus one Lambertian "
                                          "interreflection)");
    if (!(density >= 0.0f) || !std::isfinite(density)) return fail(SRP_EINVAL, fn + ": bad density");
    if (!(o->pressure >= 0.0) || !std::isfinite(o->pressure)) return fail(SRP_EINVAL, fn + ": bad pressure");
    if (o->block_threads != 0 && o->block_threads != 128)
        return fail(SRP_EINVAL, fn + ": block_threads must be 0 or 128");
    if (o->mem != SRP_MEM_HOST && o->mem != SRP_MEM_DEVICE)
        return fail(SRP_EINVAL, fn + ": mem must be SRP_MEM_HOST or SRP_MEM_DEVICE");
    if (o->kernel_variant != 0 && o->kernel_variant != 4 && o->kernel_variant != 6 && o->kernel_variant != 8)
        return fail(SRP_EINVAL, fn + ": kernel_variant must be 0, 4, 6 or 8");
    const int variant = o->kernel_variant ? o->kernel_variant : 8;
    std::vector<DesignDev> designs(D);
    std::vector<int64_t> xbase(D);
    int w = 0, t_max = 0;
    int64_t sum_x = 0, b_max = 0;
    for (int d = 0; d < D; ++d) {
        const srp_bvh* h = bvhs ? bvhs[d] : nullptr;
        if (!h) return fail(SRP_EINVAL, fn + ": NULL bvh");
        if (h->device != c->device) return fail(SRP_EINVAL, fn + ": bvh built on another device");
        if (w == 0) w = h->width;
        if (h->width != w) return fail(SRP_EUNSUPPORTED, fn + ": all designs of one call need the same BVH width");
        if (h->max_group >= G)
            return fail(SRP_EINVAL, fn + ": design " + std::to_string(d) + " uses material group " +
                                        std::to_string(h->max_group) + " but rho has G = " + std::to_string(G) + " groups");
        DesignDev& dz = designs[d];
        dz.tri = (const float4*)h->d_tri; dz.nodes = (const float4*)h->d_nodes;
        dz.cx = h->c[0]; dz.cy = h->c[1]; dz.cz = h->c[2]; dz.R = h->R;
        dz.T = h->T; dz.width = h->width;
        // bound on sum_f max(1, ceil(density * A_f)): FP32 areas and products
        // differ from the FP64 total by a few ulps each
        const double bnd = (double)h->T + std::ceil((double)density * h->area * (1.0 + 1e-5)) + 64.0;
        if (!(bnd < 2147483647.0)) return fail(SRP_EINVAL, fn + ": more than 2^31 samples for one design");
        b_max = std::max<int64_t>(b_max, (int64_t)bnd);
        xbase[d] = sum_x;
        sum_x += (int64_t)h->T + 1;
        t_max = std::max(t_max, h->T);
    }
    const int width = w ? w : 4;
    const int64_t items = (int64_t)D * S;
    if (items > 0 && (!rho || (mode == 0 && !sun_dir) || (mode == 1 && !emit) || !com || !out_ft))
        return fail(SRP_EINVAL, fn + ": NULL array argument");
    CU(cudaSetDevice(c->device), "cudaSetDevice");
    // units: chunks of a multiple of 1024 samples, at most 16M units of partials
    const int64_t tile = 1024;
    int64_t chunk = tile;
    int64_t cpd = std::max<int64_t>(1, (b_max + chunk - 1) / chunk);
    const int64_t max_units = 16777216;
    if (items > 0 && items * cpd > max_units) {
        const int64_t per_item = std::max<int64_t>(1, max_units / items);
        chunk = (b_max + per_item - 1) / per_item;
        chunk = std::max<int64_t>(tile, (chunk + tile - 1) / tile * tile);
        cpd = std::max<int64_t>(1, (b_max + chunk - 1) / chunk);
    }
    const size_t tab_n = (size_t)std::max<int64_t>(sum_x, 1);
    if (c->atab.ensure(3 * tab_n * sizeof(int32_t)) != cudaSuccess) return fail(SRP_ENOMEM, fn + ": sample tables");
    if (c->axb.ensure(2 * (size_t)std::max(D, 1) * sizeof(int64_t)) != cudaSuccess)
        return fail(SRP_ENOMEM, fn + ": sample tables");
    const size_t part_bytes = sizeof(double) * 12 * (size_t)std::max<int64_t>(items * cpd, 1);
    if (c->part.ensure(part_bytes) != cudaSuccess) return fail(SRP_ENOMEM, fn + ": cannot allocate partials");
    int rc = upload_designs(c, designs);
    if (rc != SRP_OK) return rc;
    int64_t* d_xb = (int64_t*)c->axb.p;
    if (D > 0) CU(cudaMemcpyAsync(d_xb, xbase.data(), sizeof(int64_t) * D, cudaMemcpyHostToDevice, c->stream), "H2D xbase");
    AreaParams p;
    std::memset(&p, 0, sizeof p);
    p.mode = mode == 0 && o->max_bounces == 2 ? 2 : mode;
    p.D = D; p.S = S; p.G = G; p.sun_per_design = (mode == 0 && o->sun_per_design) ? 1 : 0;
    p.seed = o->seed; p.P = (float)o->pressure; p.density = density;
    p.sun_base = o->sun_base; p.design_base = o->design_base;
    p.chunk = chunk; p.cpd = (int32_t)cpd; p.cap = cpd * chunk;
    p.designs = (const DesignDev*)c->dtab.p;
    p.xbase = d_xb; p.ntot = d_xb + std::max(D, 1);
    p.cnt = (int32_t*)c->atab.p; p.map = p.cnt + tab_n; p.ex = p.map + tab_n;
    p.part = (double*)c->part.p;
    p.err = c->d_err;
    p.stats = c->stats_on ? c->d_stats : nullptr;
    p.queue = c->d_queue;
    const int grid_cap = c->n_sm * area_resident_blocks(width, variant);
    const int64_t nsun = mode == 1 ? 0 : (p.sun_per_design ? (int64_t)D * S : S);
    double* d_ft = out_ft;
    double* d_sg = out_sigma;
    const size_t ob = sizeof(double) * 6 * (size_t)items;
    if (o->mem == SRP_MEM_DEVICE) {
        p.rho = rho; p.sun = sun_dir; p.com = com; p.emit = emit;
    } else {
        if (items > 0) {
            rc = validate_values(rho, D, G, sun_dir, nsun);
            if (rc != SRP_OK) return rc;
            if (mode == 1)
                for (int64_t q = 0; q < (int64_t)D * G; ++q)
                    if (!(emit[q] >= 0.0f) || !std::isfinite(emit[q]))
                        return fail(SRP_EINVAL, fn + ": emit must be finite and >= 0");
        }
        const size_t rb = sizeof(float) * 2 * (size_t)D * G, sb = sizeof(double) * 3 * (size_t)nsun,
                     cb = sizeof(double) * 3 * (size_t)D, eb = mode == 1 ? sizeof(float) * (size_t)D * G : 0;
        const size_t rb_al = (rb + 255) / 256 * 256, sb_al = (sb + 255) / 256 * 256, cb_al = (cb + 255) / 256 * 256;
        if (c->stage_in.ensure(rb_al + sb_al + cb_al + eb + 256) != cudaSuccess) return fail(SRP_ENOMEM, fn + ": staging");
        const size_t ob_al = (ob + 255) / 256 * 256;
        if (c->stage_out.ensure(2 * ob_al + 256) != cudaSuccess) return fail(SRP_ENOMEM, fn + ": staging");
        char* in = (char*)c->stage_in.p;
        if (items > 0) {
            CU(cudaMemcpyAsync(in, rho, rb, cudaMemcpyHostToDevice, c->stream), "H2D rho");
            CU(cudaMemcpyAsync(in + rb_al, sun_dir, sb, cudaMemcpyHostToDevice, c->stream), "H2D sun");
            CU(cudaMemcpyAsync(in + rb_al + sb_al, com, cb, cudaMemcpyHostToDevice, c->stream), "H2D com");
            if (eb) CU(cudaMemcpyAsync(in + rb_al + sb_al + cb_al, emit, eb, cudaMemcpyHostToDevice, c->stream), "H2D emit");
        }
        p.rho = (const float*)in; p.sun = (const double*)(in + rb_al); p.com = (const double*)(in + rb_al + sb_al);
        p.emit = (const float*)(in + rb_al + sb_al + cb_al);
        d_ft = (double*)c->stage_out.p;
        d_sg = out_sigma ? (double*)((char*)c->stage_out.p + ob_al) : nullptr;
    }
    CU(cudaMemsetAsync(p.queue, 0, sizeof(unsigned long long), c->stream), "cudaMemsetAsync(queue)");
    CU(launch_area(p, width, variant, t_max, grid_cap, c->stream), "area kernels launch");
    if (items > 0) CU(launch_reduce(p.part, items, p.cpd, d_ft, d_sg, c->stream), "reduce kernel launch");
    if (o->mem == SRP_MEM_DEVICE) {
        if (out_samples && D > 0)
            CU(cudaMemcpyAsync(out_samples, p.ntot, sizeof(int64_t) * D, cudaMemcpyDeviceToDevice, c->stream), "D2D samples");
        return SRP_OK;
    }
    if (items > 0) {
        CU(cudaMemcpyAsync(out_ft, d_ft, ob, cudaMemcpyDeviceToHost, c->stream), "D2H ft");
        if (out_sigma) CU(cudaMemcpyAsync(out_sigma, d_sg, ob, cudaMemcpyDeviceToHost, c->stream), "D2H sigma");
    }
    if (out_samples && D > 0)
        CU(cudaMemcpyAsync(out_samples, p.ntot, sizeof(int64_t) * D, cudaMemcpyDeviceToHost, c->stream), "D2H samples");
    return srp_sync(c);
}
}  // namespace

extern "C" int srp_force_area(srp_ctx* c, const srp_bvh* const* bvhs, int D, const float* rho, int G,
                              const double* sun_dir, int S, const double* com, float density,
                              const srp_trace_opts* o, double* out_ft, double* out_sigma, int64_t* out_samples) {
    return area_common(c, 0, bvhs, D, rho, G, sun_dir, S, com, nullptr, density, o, out_ft, out_sigma, out_samples);
}

extern "C" int srp_force_thermal(srp_ctx* c, const srp_bvh* const* bvhs, int D, const float* rho, int G,
                                 const float* emit, const double* com, float density, const srp_trace_opts* o,
                                 double* out_ft, double* out_sigma, int64_t* out_samples) {
    return area_common(c, 1, bvhs, D, rho, G, nullptr, 1, com, emit, density, o, out_ft, out_sigma, out_samples);
}
