// srp_internal.h -- internal layouts of the SRP library (host + device).
//
// Device memory layout of one design (an srp_bvh):
//   tri   float4 [T][3]   triangles in BVH leaf order:
//                         [0] = (v0.xyz, bits(original index))
//                         [1] = (v1.xyz, bits(material group))
//                         [2] = (v2.xyz, 0)
//   nodes W-wide nodes, structure-of-arrays inside each node:
//     W = 4: 128 B  = lo_x, hi_x, lo_y, hi_y, lo_z, hi_z (float4 each,
//                     lane c = child c), child (int4), pad (int4)
//     W = 8: 256 B  = the same six bounds as 2 float4 each (12 float4),
//                     child as 2 int4, 2 int4 pad
//   child >= 0: inner node index; child < 0: leaf, ~child = first << 3 |
//   (count - 1), count in 1..8 triangles starting at tri[first].  Empty
//   slots have lo = +inf, hi = -inf and never hit.
#pragma once
#include <stdint.h>
#include <vector_types.h>
#include <string>
#include <vector>

#include "../../include/srp.h"

namespace srp {

constexpr int kMaxGroups = 64;
constexpr int kMaxBounces = 3;
constexpr int kStackSize = 64;          // traversal stack entries per ray
constexpr int kMaxDesignsPerLaunch = 1 << 20;  // designs of one srp_force call (device table)
constexpr int kVisitCap = 1 << 20;      // node visits per ray segment (corruption guard)

// Error flags written by kernels (bitwise OR into one device word).
constexpr int kErrStackOverflow = 1;
constexpr int kErrVisitCap = 2;
constexpr int kErrWaitTimeout = 4;      // a bounded mbarrier wait of a tensor-core kernel gave up
constexpr int kErrAreaCount = 8;        // area estimator: sample counts above the planned bound
constexpr int kErrTriIndex = 16;        // triangle table holds an index outside 0..T-1
constexpr int kErrRowIndex = 32;        // training batch index outside the data set's rows

struct BuiltBVH {                  // host result of the builder
    int width = 4;
    std::vector<float> node_data;  // W-wide nodes, packed as described above
    std::vector<int32_t> tri_order;  // leaf order -> original triangle index
    int n_nodes = 0, n_leaves = 0, depth = 0;
    // nodes are numbered breadth first: level d (root = 0) is the index range
    // [level_start[d], level_start[d + 1]); depth + 1 entries
    std::vector<int32_t> level_start;
};

// Binned-SAH binary build, collapsed to `width` (4 or 8) children.
// Bounds are padded outward so the FP32 slab test is conservative.
int build_wide_bvh(const float* verts, int V, const int32_t* tris, int T, int width,
                   BuiltBVH* out, std::string* err);

// Per-design parameters passed to the trace kernel by value.
struct DesignDev {
    const float4* tri;
    const float4* nodes;
    double cx, cy, cz, R;      // ray-grid centre and radius
    int32_t T, width;
};

struct TraceParams {
    int32_t D, S, G;
    int32_t nx, ny, K, jitter, sun_per_design;
    uint64_t seed;
    double P;
    int64_t off, stride, n;    // ray subset (n rays per item)
    int32_t sun_base, design_base;
    int64_t chunk;             // rays per unit (multiple of 64)
    int32_t cpb;               // chunks (units) per item
    const float* rho;          // [D][G][2]
    const double* sun;         // [S][3] or [D][S][3]
    const double* com;         // [D][3]
    double* part;              // [D*S*cpb][12]
    int* err;                  // device error word
    unsigned long long* stats; // [3] node visits, triangle tests, segments (or NULL)
    const DesignDev* designs;  // [D] device-side design table
    unsigned long long* queue; // work-queue counter (zeroed before each launch)
    int32_t variant;           // register budget: minimum resident blocks 4 or 5
    // full-grid launches: a batch is a block of 32 / bh x bh pixels (bh = 1,
    // 2 or 4 rows, the tallest that divides ny); per item and band of bh
    // grid rows, the first batch that can meet the scene and the prefix of
    // such batches (span_kernel); null: every ray of the subset is traced
    int32_t* rowfirst;         // [D*S][ny / bh]
    int32_t* rowoff;           // [D*S][ny / bh + 1]
    int32_t bh;
    // full-grid launches: per item the FP32 constants of its ray grid (the
    // FP64 item set-up done once by span_kernel for the tracer's units):
    // (ob, fdx), (bu, fdy), (bv, w0), (dd, tmin_b), (com, 0), then the 12
    // direction-only values of the primary rays' set-up (1/d, shear rows)
    float4* itab;              // [D*S][8]
};

// Rows of a span-mode batch for a grid of ny rows: the tallest of 4, 2, 1
// that divides ny (the block is 32 / rows pixels wide).  Compact blocks keep
// a warp's parallel rays closer together than a 32-pixel strip.
#ifndef SRP_SPAN_ROWS_MAX
#define SRP_SPAN_ROWS_MAX 4
#endif
inline int span_batch_rows(int ny) {
    if (SRP_SPAN_ROWS_MAX >= 4 && ny % 4 == 0) return 4;
    if (SRP_SPAN_ROWS_MAX >= 2 && ny % 2 == 0) return 2;
    return 1;
}

// Parameters of the area-sampling estimator (area.cu).
struct AreaParams {
    int32_t mode;             // 0: sun light with next-event shadow rays; 1: thermal emitters;
                              // 2: sun light plus one gathered Lambertian interreflection
    int32_t D, S, G, sun_per_design;
    uint64_t seed;
    float P, density;
    int32_t sun_base, design_base;
    int64_t chunk;            // samples per unit (multiple of 1024)
    int32_t cpd;              // units per item
    int64_t cap;              // planned bound on the samples of one design (cpd * chunk)
    const DesignDev* designs;
    const int64_t* xbase;     // [D] first entry of design d in cnt/map/ex (T_d + 1 entries each)
    int32_t* cnt;             // samples of original triangle f
    int32_t* map;             // leaf slot of original triangle f
    int32_t* ex;              // exclusive prefix of cnt (T_d + 1 entries)
    int64_t* ntot;            // [D] samples of design d
    const float* rho;
    const double* sun;
    const double* com;
    const float* emit;        // thermal: [D][G] emitted momentum flux per unit area (times P)
    double* part;             // [units][12]
    int* err;
    unsigned long long* stats;
    unsigned long long* queue;
};

}  // namespace srp

struct srp_bvh {
    int device;
    int width;
    int T, n_nodes, n_leaves, depth;
    double build_ms;
    double c[3], R;
    void* d_tri;    // float4[T][3]
    void* d_nodes;  // node data
    int64_t bytes;
    double area;    // total surface area (FP64, from the build's vertices)
    int max_group;  // largest material group id of the mesh (-1 when empty)
    std::vector<int32_t> level_start;   // breadth-first level ranges of the nodes (srp_bvh_refit)
};
