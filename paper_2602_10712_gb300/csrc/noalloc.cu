// noalloc.cu -- srp_force_noalloc: the force/torque evaluation of srp_force
// for callers that must not allocate GPU memory.
//
// Some callers cannot call cudaMalloc (or anything that allocates) at the
// point where they need forces: code running under an allocator policy that
// forbids new device allocations after start-up (for example a long-running
// flight-dynamics service that sizes its memory once), code that is only
// handed a stream and device pointers by a host framework, or real-time
// loops where an allocation could stall.  srp_force keeps its per-chunk FP64
// partial sums in scratch memory that the context allocates and grows on
// demand; this entry point keeps them instead in one fixed, file-scope
// device array that the library reserves when it is loaded.
//
// Properties (also stated in include/srp.h):
//  - the scratch array holds at most kScratchBytes (8 MiB) of partials,
//    i.e. D*S*chunks <= 87,381 work units; larger requests are rejected
//    with SRP_EINVAL and a message naming the limit;
//  - every fixed array here (the partials, the design table, the error
//    word and the work-queue counter) is shared by every call on a device
//    and keeps the last call's contents; two calls whose work overlaps on
//    the GPU (different streams, no ordering between them) race on all of
//    them: besides wrong sums, one call may rewrite the design table while
//    the other's kernel reads it, pairing one design's triangles with
//    another's nodes, which can read out of bounds;
//  - on full grids whose width is a multiple of 32 it runs srp_force's
//    batch pre-pass (only the 32-pixel batches that can meet the scene are
//    traced) with its per-row tables and per-item constants in a second
//    fixed array of kSpanBytes (16 MiB): items * (8 ny + 4) + 128 items
//    bytes must fit (about 2,000 items at ny = 1024); larger calls, ray
//    subsets and other widths trace every ray;
//  - the first call on each device looks up the array's device address
//    (cudaGetSymbolAddress) with that device current; make that first call
//    before any stream capture begins;
//  - nothing here calls cudaMalloc, cudaFree or an allocating library, and
//    a successful call takes no host heap memory (only error messages do).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "srp_internal.h"

namespace srp {
void set_last_error(const std::string& msg);
int trace_resident_blocks(int width, int block, int variant);
cudaError_t launch_trace(const TraceParams& p, int width, int grid_cap, int block, cudaStream_t st);
cudaError_t launch_span(const TraceParams& p, int width, cudaStream_t st);
cudaError_t launch_reduce(const double* part, int64_t items, int cpb, double* out_ft, double* out_sigma,
                          cudaStream_t st);
}  // namespace srp

using namespace srp;

namespace {

constexpr size_t kScratchBytes = 8u << 20;                       // 8 MiB
constexpr size_t kSpanBytes = 16u << 20;                         // 16 MiB
constexpr int64_t kScratchUnits = (int64_t)(kScratchBytes / (12 * sizeof(double)));
constexpr int kMaxDevices = 64;
constexpr int kNoAllocDesigns = 4096;

// The fixed scratch: per-unit FP64 partials, the kernels' error word, the
// work-queue counter and the design table.
static __device__ __align__(256) double g_scratch[kScratchBytes / sizeof(double)];
static __device__ __align__(256) int g_err_word;
static __device__ __align__(256) unsigned long long g_queue_word;
static __device__ __align__(256) DesignDev g_design_table[kNoAllocDesigns];
// the batch pre-pass's tables (row starts, row prefix, item constants)
static __device__ __align__(256) int32_t g_span[kSpanBytes / sizeof(int32_t)];

struct DevState {
    bool ready = false;
    double* part = nullptr;  // device address of g_scratch on this device
    int* err = nullptr;      // device address of g_err_word on this device
    unsigned long long* queue = nullptr;  // device address of g_queue_word
    DesignDev* table = nullptr;           // device address of g_design_table
    int32_t* span = nullptr;              // device address of g_span
    int n_sm = 0;
    int resident[2] = {0, 0};  // resident blocks per SM for widths 4 and 8
};
DevState g_dev[kMaxDevices];
std::mutex g_mu;

int fail(int code, const std::string& m) {
    srp::set_last_error(m);  // reported by srp_last_error()
    return code;
}

// Writes designs [d0, d0 + n) of the fixed table from a chunk passed by value
// as the kernel parameter (3.5 KB, within the 4 KB parameter space): the
// bytes travel with the launch, so no host buffer has to outlive the call.
constexpr int kStage = 64;
struct DesignChunk {
    DesignDev d[kStage];
};
__global__ void store_designs_kernel(const DesignChunk c, int d0, int n) {
    const int k = threadIdx.x;
    if (k < n) g_design_table[d0 + k] = c.d[k];
}

// One-time set-up for the current device (its first call lands here).
int setup_device(int dev, DevState** out) {
    std::lock_guard<std::mutex> lk(g_mu);
    DevState& s = g_dev[dev];
    if (!s.ready) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
        if (e != cudaSuccess) return fail(SRP_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        s.part = static_cast<double*>(ptr);
        e = cudaGetSymbolAddress(&ptr, g_err_word);
        if (e != cudaSuccess) return fail(SRP_ECUDA, std::string("cudaGetSymbolAddress(error word): ") + cudaGetErrorString(e));
        s.err = static_cast<int*>(ptr);
        e = cudaGetSymbolAddress(&ptr, g_queue_word);
        if (e != cudaSuccess) return fail(SRP_ECUDA, std::string("cudaGetSymbolAddress(queue): ") + cudaGetErrorString(e));
        s.queue = static_cast<unsigned long long*>(ptr);
        e = cudaGetSymbolAddress(&ptr, g_design_table);
        if (e != cudaSuccess) return fail(SRP_ECUDA, std::string("cudaGetSymbolAddress(designs): ") + cudaGetErrorString(e));
        s.table = static_cast<DesignDev*>(ptr);
        e = cudaGetSymbolAddress(&ptr, g_span);
        if (e != cudaSuccess) return fail(SRP_ECUDA, std::string("cudaGetSymbolAddress(span tables): ") + cudaGetErrorString(e));
        s.span = static_cast<int32_t*>(ptr);
        int v = 0;
        e = cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return fail(SRP_ECUDA, std::string("cudaDeviceGetAttribute: ") + cudaGetErrorString(e));
        s.n_sm = v;
        s.resident[0] = trace_resident_blocks(4, 128, 7);
        s.resident[1] = trace_resident_blocks(8, 128, 7);
        s.ready = true;
    }
    *out = &s;
    return SRP_OK;
}

}  // namespace

extern "C" int srp_force_noalloc(const srp_bvh* const* bvhs, int D, const float* rho, int G, const double* sun_dir,
                                 int S, const double* com, const srp_trace_opts* o, double* out_ft,
                                 double* out_sigma, int32_t* d_status, void* cuda_stream) {
    if (!o) return fail(SRP_EINVAL, "srp_force_noalloc: NULL opts");
    if (o->mem != SRP_MEM_DEVICE) return fail(SRP_EINVAL, "srp_force_noalloc: all arrays must be device memory (mem = SRP_MEM_DEVICE)");
    if (D < 0 || S < 0) return fail(SRP_EINVAL, "srp_force_noalloc: negative D or S");
    if (G < 1 || G > kMaxGroups) return fail(SRP_EINVAL, "srp_force_noalloc: G must be in 1..64");
    if (o->rays_x < 1 || o->rays_y < 1) return fail(SRP_EINVAL, "srp_force_noalloc: rays_x/rays_y must be >= 1");
    const int64_t grid_n = (int64_t)o->rays_x * o->rays_y;
    if (grid_n > 0xffffffffLL) return fail(SRP_EINVAL, "srp_force_noalloc: rays_x*rays_y must be < 2^32");
    if (o->max_bounces < 1 || o->max_bounces > kMaxBounces) return fail(SRP_EINVAL, "srp_force_noalloc: max_bounces must be 1..3");
    if (!(o->pressure >= 0.0) || !std::isfinite(o->pressure)) return fail(SRP_EINVAL, "srp_force_noalloc: bad pressure");
    if (o->block_threads != 0 && o->block_threads != 128) return fail(SRP_EINVAL, "srp_force_noalloc: block_threads must be 0 or 128");
    int64_t n = o->ray_count, off = o->ray_offset, stride = o->ray_stride;
    if (n == 0) { n = grid_n; off = 0; stride = 1; }
    if (n < 0 || off < 0 || stride < 1 || off + (n - 1) * stride >= grid_n)
        return fail(SRP_EINVAL, "srp_force_noalloc: ray subset outside the grid");
    const int64_t items = (int64_t)D * S;
    if (items > 0 && (!bvhs || !rho || !sun_dir || !com || !out_ft))
        return fail(SRP_EINVAL, "srp_force_noalloc: NULL array argument");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(SRP_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(SRP_EUNSUPPORTED, "srp_force_noalloc: device index too large");
    if (D > kNoAllocDesigns)
        return fail(SRP_EINVAL, "srp_force_noalloc: D = " + std::to_string(D) + " exceeds the fixed design-table capacity of " +
                                    std::to_string(kNoAllocDesigns) + " designs; use srp_force");
    if (o->kernel_variant != 0) return fail(SRP_EINVAL, "srp_force_noalloc: kernel_variant must be 0");
    // every design is checked before anything is enqueued; the table itself is
    // written further down, through a small stack buffer (no heap allocation)
    int width = 0;
    for (int d = 0; d < D; ++d) {
        const srp_bvh* h = bvhs[d];
        if (!h) return fail(SRP_EINVAL, "srp_force_noalloc: NULL bvh");
        if (h->device != dev) return fail(SRP_EINVAL, "srp_force_noalloc: bvh built on another device than the current one");
        if (width == 0) width = h->width;
        if (h->width != width) return fail(SRP_EUNSUPPORTED, "srp_force_noalloc: all designs of one call need the same BVH width");
        if (h->max_group >= G)
            return fail(SRP_EINVAL, "srp_force_noalloc: design " + std::to_string(d) + " uses material group " +
                                        std::to_string(h->max_group) + " but rho has G = " + std::to_string(G) + " groups");
    }
    if (width == 0) width = 4;
    if (items > kScratchUnits)
        return fail(SRP_EINVAL, "srp_force_noalloc: D*S = " + std::to_string(items) +
                                    " exceeds the fixed scratch capacity of " + std::to_string(kScratchUnits) +
                                    " (design, sun) items (8 MiB of partial sums); use srp_force");
    DevState* ds = nullptr;
    int rc = setup_device(dev, &ds);
    if (rc != SRP_OK) return rc;
    // chunks per item: the automatic rule of srp_force (at least ~40k units
    // in all, and at least one unit per four resident warps per item so that
    // the warps resident at a time share a few (design, sun) items' BVH
    // nodes in L1; chunks of at least 256 rays), then capped by the fixed
    // scratch
    int64_t cpb = o->chunks_per_item;
    if (cpb < 0) return fail(SRP_EINVAL, "srp_force_noalloc: negative chunks_per_item");
    if (cpb == 0) {
        const int64_t warps = (int64_t)ds->n_sm * ds->resident[width == 8 ? 1 : 0] * 4;
        cpb = items > 0 ? std::max<int64_t>((40960 + items - 1) / items, warps / 4) : 1;
        cpb = std::max<int64_t>(1, std::min<int64_t>(cpb, (n + 255) / 256));
    }
    int64_t chunk = (n + cpb - 1) / cpb;
    chunk = std::max<int64_t>(64, (chunk + 63) / 64 * 64);
    cpb = std::max<int64_t>(1, (n + chunk - 1) / chunk);
    if (items * cpb > kScratchUnits) {
        if (o->chunks_per_item != 0)
            return fail(SRP_EINVAL, "srp_force_noalloc: D*S*chunks_per_item exceeds the fixed scratch capacity of " +
                                        std::to_string(kScratchUnits) + " work units");
        cpb = std::max<int64_t>(1, kScratchUnits / std::max<int64_t>(items, 1));
        chunk = (n + cpb - 1) / cpb;
        chunk = std::max<int64_t>(64, (chunk + 63) / 64 * 64);
        cpb = std::max<int64_t>(1, (n + chunk - 1) / chunk);
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (items == 0 || n == 0) {
        if (items > 0) {
            e = cudaMemsetAsync(out_ft, 0, sizeof(double) * 6 * items, st);
            if (e == cudaSuccess && out_sigma) e = cudaMemsetAsync(out_sigma, 0, sizeof(double) * 6 * items, st);
            if (e != cudaSuccess) return fail(SRP_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
        }
        if (d_status) {
            e = cudaMemsetAsync(d_status, 0, sizeof(int32_t), st);
            if (e != cudaSuccess) return fail(SRP_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
        }
        return SRP_OK;
    }
    TraceParams p;
    std::memset(&p, 0, sizeof p);
    p.D = D; p.S = S; p.G = G;
    p.nx = o->rays_x; p.ny = o->rays_y; p.K = o->max_bounces; p.jitter = o->jitter ? 1 : 0;
    p.sun_per_design = o->sun_per_design ? 1 : 0;
    p.seed = o->seed; p.P = o->pressure;
    p.off = off; p.stride = stride; p.n = n;
    p.sun_base = o->sun_base; p.design_base = o->design_base;
    p.chunk = chunk; p.cpb = (int32_t)cpb;
    p.rho = rho; p.sun = sun_dir; p.com = com;
    p.part = ds->part;          // every unit overwrites its 12 partials: no clearing needed
    p.err = ds->err;
    p.stats = nullptr;
    p.variant = 7;
    p.queue = ds->queue;
    p.designs = ds->table;
    // full grids of whole 32-pixel batches: the batch pre-pass of srp_force,
    // its tables in the fixed array when they fit (span_kernel rewrites every
    // entry on each call)
    const size_t row_bytes = (sizeof(int32_t) * (size_t)items * (2 * (size_t)o->rays_y + 1) + 255) / 256 * 256;
    if (off == 0 && stride == 1 && n == grid_n && o->rays_x % 32 == 0 &&
        row_bytes + 8 * sizeof(float4) * (size_t)items <= kSpanBytes) {
        p.rowfirst = ds->span;
        p.rowoff = ds->span + (size_t)items * o->rays_y;
        p.itab = (float4*)((char*)ds->span + row_bytes);
        p.bh = span_batch_rows(o->rays_y);
    }
    // the design table: written into the fixed array by small kernels that
    // carry 64 entries each in their parameters (stream-ordered, no host
    // buffer outlives the call)
    for (int d0 = 0; d0 < D; d0 += kStage) {
        const int nd = std::min(kStage, D - d0);
        DesignChunk chunk_tab;
        std::memset(&chunk_tab, 0, sizeof chunk_tab);
        for (int k = 0; k < nd; ++k) {
            const srp_bvh* h = bvhs[d0 + k];
            DesignDev& z = chunk_tab.d[k];
            z.tri = (const float4*)h->d_tri; z.nodes = (const float4*)h->d_nodes;
            z.cx = h->c[0]; z.cy = h->c[1]; z.cz = h->c[2]; z.R = h->R;
            z.T = h->T; z.width = h->width;
        }
        store_designs_kernel<<<1, kStage, 0, st>>>(chunk_tab, d0, nd);
        e = cudaGetLastError();
        if (e != cudaSuccess) return fail(SRP_ECUDA, std::string("design table kernel launch: ") + cudaGetErrorString(e));
    }
    // the error word only collects flags (OR) and the queue counts up: both start at zero
    e = cudaMemsetAsync(ds->err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ds->queue, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return fail(SRP_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    const int grid_cap = ds->n_sm * ds->resident[width == 8 ? 1 : 0];
    if (p.rowoff) {
        e = launch_span(p, width, st);
        if (e != cudaSuccess) return fail(SRP_ECUDA, std::string("span_kernel launch: ") + cudaGetErrorString(e));
    }
    e = launch_trace(p, width, grid_cap, 128, st);
    if (e != cudaSuccess) return fail(SRP_ECUDA, std::string("trace_kernel launch: ") + cudaGetErrorString(e));
    e = launch_reduce(ds->part, items, p.cpb, out_ft, out_sigma, st);
    if (e != cudaSuccess) return fail(SRP_ECUDA, std::string("reduce kernel launch: ") + cudaGetErrorString(e));
    if (d_status) {
        e = cudaMemcpyAsync(d_status, ds->err, sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return fail(SRP_ECUDA, std::string("cudaMemcpyAsync(status): ") + cudaGetErrorString(e));
    }
    return SRP_OK;
}

