/*
 * srp.h -- C ABI of the GB300 (sm_103a) solar-radiation-pressure library.
 *
 * The library computes, for triangulated spacecraft designs lit by the sun
 * from direction w (a unit vector TOWARD the sun), the net radiation force
 *   F(w, theta)   = integral over the surface M(theta) of f(x, w, theta) dx
 * and torque about the centre of mass
 *   tau(w, theta) = integral over M of (x - x_COM(theta)) x f(x, w, theta) dx
 * (paper, Sec. 3.2, the force-field integral Eq. "Force" and the two surface
 * integrals after it), where the force field f converts the radiance arriving
 * at x into force through the light-to-force map l2f (Sec. 3.2): photons
 * transfer their momentum when they arrive and reflected photons carry
 * momentum away.  Units: with pressure P in N/m^2 and lengths in metres,
 * F is in N and tau in N m.  P = 1 gives "unit radiation" (Sec. 3.3).
 *
 * Estimator.  A grid of parallel rays covers the square of side 2R centred on
 * the design's vertex-AABB centre c, R = max |vertex - c|, in the plane normal
 * to the travel direction d = -w.  Ray i = py*rays_x + px starts at pixel
 * (px, py) jittered by (xi1, xi2) from Philox4x32-10 with counter
 * (i, sun index, design index, 0) and key (seed lo, seed hi), and carries
 * momentum weight w0 = P dx dy.  Closest hits are found through a wide BVH.
 * At hit k of at most K = max_bounces (normal n flipped to face the ray,
 * cos = -n.d, reflectances (rho_s, rho_d) of the triangle's material group):
 *   k == K : deposit w [(1 - rho_s) d - (2 rho_s cos + 2/3 rho_d) n]
 *            (the expected reflection: the per-plate law of Sec. 2.1)
 *   k <  K : with probability 1/2 reflect specularly (weight 2 w rho_s),
 *            else diffusely with a cosine-weighted direction (weight
 *            2 w rho_d), deposit w d - w' d', and trace on (Philox counter
 *            (i, sun, design, k)).
 * The torque deposit is (x - COM) x deposit.  The branch probability does
 * not depend on rho, so results are polynomials in rho along fixed paths.
 * Sums are FP64; sigma is the collapsed-strata standard error (neighbouring
 * rays k = 2j, 2j+1 paired: var = sum (y_2j - y_2j+1)^2).
 *
 * Conventions.
 *  - Every function returns an int status (SRP_OK on success).  The message
 *    of the last failure on the calling thread is srp_last_error().
 *  - All calls are asynchronous on the context's CUDA stream unless their
 *    buffers are host memory (mem = SRP_MEM_HOST), in which case they copy
 *    in, compute, copy out and synchronise before returning.
 *  - The caller owns every array argument; the library owns the opaque
 *    handles (srp_ctx, srp_bvh) and frees them in srp_*_destroy.
 *  - Device-side failures (a traversal stack overflow or a visit cap hit on
 *    a corrupted BVH) set a flag that the next srp_sync() (or any HOST-mem
 *    call) reports as SRP_EDEVICE_LIMIT; a bounded wait of a tensor-core
 *    kernel that gave up, alone, is reported as SRP_ETIMEOUT.  No kernel
 *    traps or spins forever.
 */
#ifndef SRP_H
#define SRP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define SRP_OK 0
#define SRP_EINVAL 1          /* invalid argument (message says which)      */
#define SRP_ENOMEM 2          /* host or device allocation failed           */
#define SRP_ECUDA 3           /* a CUDA runtime call failed                 */
#define SRP_EDEVICE_LIMIT 4   /* a bounded device loop hit its limit        */
#define SRP_ETIMEOUT 5        /* a bounded device wait gave up              */
#define SRP_EUNSUPPORTED 6    /* valid request the library does not support */

typedef enum { SRP_MEM_HOST = 0, SRP_MEM_DEVICE = 1 } srp_mem;

typedef struct srp_ctx srp_ctx;
typedef struct srp_bvh srp_bvh;

/* Options of one force evaluation.  srp_trace_opts_default() fills the
 * defaults shown in brackets. */
typedef struct srp_trace_opts {
    int32_t rays_x, rays_y;   /* ray grid resolution [1024 x 1024]          */
    int32_t max_bounces;      /* K in 1..3 [1]                              */
    int32_t jitter;           /* 1 stratified jitter, 0 pixel centres [1]  */
    uint64_t seed;            /* Philox key [0]                             */
    double pressure;          /* P in N/m^2 [1.0 = unit radiation]          */
    int64_t ray_offset;       /* ray subset: trace i = off + k*stride for   */
    int64_t ray_stride;       /*   k < ray_count; ray_count 0 = whole grid  */
    int64_t ray_count;        /*   [0, 1, 0]                                */
    int32_t sun_base;         /* added to the sun index in the RNG counter  */
    int32_t design_base;      /* added to the design index in the counter   */
    int32_t mem;              /* srp_mem of rho/sun_dir/com/outputs [DEVICE]*/
    int32_t sun_per_design;   /* 1: sun_dir is [D][S][3], 0: [S][3] [0]     */
    int32_t block_threads;    /* 0 or 128 (threads per block)               */
    int32_t chunks_per_item;  /* 0 = automatic; else ray chunks per item    */
    int32_t kernel_variant;   /* min resident blocks/SM: 0 = default (7), 4, 5, 6, 7, 8 */
    int32_t reserved;         /* must be 0                                  */
} srp_trace_opts;

/* ---- context ----------------------------------------------------------- */
const char* srp_last_error(void);
void srp_trace_opts_default(srp_trace_opts* o);

/* Create a context on CUDA device `device`, issuing work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream). */
int srp_ctx_create(srp_ctx** out, int device, void* cuda_stream);
int srp_ctx_destroy(srp_ctx* ctx);
/* Wait for the context's stream; report deferred device errors. */
int srp_sync(srp_ctx* ctx);

/* Traversal work counters of the tracer kernels on this context (for the
 * roofline's algorithmic work): out[0] BVH node visits, out[1] ray/triangle
 * tests, out[2] ray segments traced.  Synchronises the stream, copies the
 * counters accumulated since the previous call into `out` (if not NULL),
 * zeroes them, and turns collection on (enable != 0) or off for later
 * launches.  The kernels count in registers either way; only the final
 * per-warp atomic adds depend on `enable`. */
int srp_collect_stats(srp_ctx* ctx, int enable, uint64_t out[3]);

/* Read-bandwidth probe (for the roofline of the traversal; the paper has no
 * counterpart).  Allocates a device buffer of `bytes` (rounded down to a
 * multiple of 16, >= 16) on the context's device and reads it with 16-byte
 * loads cached in L2 only (ld.global.cg) from every SM at full occupancy,
 * 16 independent loads in flight per thread: one launch sweeps the buffer
 * `passes` times (a buffer smaller than what the grid reads in one round,
 * about 80 MB, is read several times per round, by different SMs, as every
 * SM reads the same BVH).  After one warm-up launch it times `reps`
 * launches with CUDA events on the context's stream and writes the best
 * rate in GB/s (1e9 bytes read per second) to *out_gbs.  A buffer that fits
 * in L2 measures the L2 read rate, one of several GB the HBM read rate.
 * Synchronous; frees the buffer before it returns.  SRP_EINVAL for bad
 * arguments, SRP_ENOMEM if the buffer cannot be allocated. */
int srp_probe_read_bandwidth(srp_ctx* ctx, int64_t bytes, int passes, int reps, double* out_gbs);

/* ---- design instantiation (Sec. 3.2: "a mapping from design parameters to
 * triangle meshes") ------------------------------------------------------- */
/* Rotate every vertex v with vhinge[v] = h >= 0 about hinge h's axis
 * (hinges[h] = point p (3) then unit axis a (3), right-hand rule) by
 * angles[h]:  v' = p + Rot(a, angle)(v - p).  Host arrays:
 * verts_in/out [V][3] float32 (may alias), vhinge [V], hinges [H][6],
 * angles [H].  Pure host code; no device work. */
int srp_design_instantiate(const float* verts_in, int V, const int32_t* vhinge,
                           const double* hinges, const double* angles, int H,
                           float* verts_out);

/* ---- acceleration structure ------------------------------------------- */
/* Build a BVH of `width` (4 or 8) children per node over one design's
 * triangles (binned SAH on the host, collapsed to a wide SoA layout) and
 * upload triangles and nodes to the context's device.  Host arrays:
 * verts [V][3] float32 (world frame), tris [T][3] int32 vertex indices,
 * group [T] int32 material group (0 <= group < 64).  T may be 0.
 * The handle keeps the grid centre c and radius R of the design. */
int srp_build_bvh(srp_ctx* ctx, const float* verts, int V, const int32_t* tris,
                  const int32_t* group, int T, int width, srp_bvh** out);
int srp_bvh_destroy(srp_bvh* bvh);

typedef struct srp_bvh_info {
    int32_t width, n_nodes, n_leaves, depth, n_tris;
    int64_t device_bytes;     /* nodes + triangles on the device            */
    double build_ms;          /* host build time                             */
    double center[3], radius; /* ray-grid centre c and radius R              */
} srp_bvh_info;
int srp_bvh_get_info(const srp_bvh* bvh, srp_bvh_info* info);

/* Replace the device node array of `bvh` with node_data [n_floats] (host,
 * the layout srp_build_bvh_host produces; same node count and width), e.g.
 * a structure built or stored elsewhere.  Every child index is checked
 * against the node and triangle counts (SRP_EINVAL otherwise); a
 * structurally wrong but in-range tree (a cycle) is caught on the device
 * by the traversal's stack-depth and node-visit limits, reported as
 * SRP_EDEVICE_LIMIT. */
int srp_bvh_set_nodes(srp_ctx* ctx, srp_bvh* bvh, const float* node_data, int64_t n_floats);

/* Refit `bvh` to moved vertices of the same mesh (Sec. 3.4: each step of a
 * design optimisation re-instantiates the design at new hinge angles):
 * the topology is kept and, on the device, the leaf-order triangle records
 * take the new vertex positions and every node's child bounds are
 * recomputed bottom up (a leaf slot: its triangles' AABB; an inner slot:
 * the union of its child's slots), padded outward as srp_build_bvh pads;
 * the grid centre c, radius R and surface area are recomputed (FP64, host)
 * exactly as srp_build_bvh computes them.  Host arrays as srp_build_bvh:
 * verts [V][3] float32, tris [T][3] int32 with T equal to the BVH's (the
 * triangle list must be the one the BVH was built from; group ids are
 * kept).  Forces traced through a refitted BVH equal those through a fresh
 * build up to the grouping of sums (closest hits do not depend on the
 * boxes); traversal cost grows as the boxes drift from the topology.
 * Stream-ordered on the context's stream and synchronous (returns after
 * the refit has completed).  SRP_EINVAL: NULL, T mismatch, vertex index
 * out of range or non-finite coordinate (nothing is changed);
 * SRP_EUNSUPPORTED: the node array was replaced (srp_bvh_set_nodes) by one
 * not numbered breadth first.  Calls using `bvh` on other streams must not
 * overlap the refit. */
int srp_bvh_refit(srp_ctx* ctx, srp_bvh* bvh, const float* verts, int V, const int32_t* tris, int T);

/* Host-only build of the same wide BVH, for inspection and serialisation
 * (no device, no context).  Two-call pattern: with node_data == NULL it
 * stores the sizes in *n_node_floats and *n_nodes and returns.  Otherwise
 * node_data [*n_node_floats] receives the node array (layout: per node,
 * 6*W floats of child bounds lo_x[W] hi_x[W] lo_y[W] hi_y[W] lo_z[W] hi_z[W],
 * then W int32 child codes: >= 0 inner node index, < 0 leaf with
 * ~code = first << 3 | (count-1) into the leaf-order triangle list, then
 * padding to 128 B (W=4) or 256 B (W=8)), and tri_order [T] the original
 * triangle index of each leaf-order slot. */
int srp_build_bvh_host(const float* verts, int V, const int32_t* tris, int T, int width,
                       float* node_data, int64_t* n_node_floats, int32_t* tri_order, int32_t* n_nodes);

/* ---- force and torque (Sec. 3.2) ---------------------------------------- */
/* For D designs (bvhs[d], built on this context) and S sun directions:
 *   rho      [D][G][2] float32  (rho_s, rho_d) per material group, each in
 *                               [0,1] with rho_s + rho_d <= 1; G <= 64 and
 *                               G above every group id of every design's
 *                               mesh (else SRP_EINVAL; the same holds for
 *                               every call below that takes rho and bvhs)
 *   sun_dir  [S][3] (or [D][S][3] with opts->sun_per_design) float64 unit
 *                               vectors toward the sun
 *   com      [D][3] float64     torque reference point (centre of mass)
 *   out_ft   [D][S][6] float64  (F, tau)
 *   out_sigma[D][S][6] float64  standard errors, or NULL
 * Array memory is opts->mem (all host or all device).  Device-mem calls are
 * asynchronous; the scratch they use belongs to the context, so calls on
 * one context must not overlap on different streams.  Validation of rho
 * and sun_dir values happens only for host-mem calls.  Whole grids
 * (ray_count 0) with rays_x a multiple of 32 first find, per band of grid
 * rows, the batches of 32 pixels (blocks of 8 x 4 when rays_y is a multiple
 * of 4, 16 x 2 when it is even, else 32 x 1) whose rays can meet the design
 * (the BVH's top boxes
 * projected onto the grid) and trace only those: the others deposit
 * exactly nothing, so the estimate is the whole grid's, its sums grouped
 * over the traced batches. */
int srp_force(srp_ctx* ctx, const srp_bvh* const* bvhs, int D, const float* rho, int G,
              const double* sun_dir, int S, const double* com, const srp_trace_opts* opts,
              double* out_ft, double* out_sigma);

/* ---- the paper's own estimator (Sec. 3.2 "Estimation": surface samples,
 * next-event estimation toward the sun, BRDF-sampled incoming light; the
 * no-bounce variant "NB" of Table 3 with max_bounces = 1) ------------------
 * Same items, arrays, memory rules and outputs as srp_force, estimated by
 * surface sampling with next-event estimation instead of a ray grid:
 *   - triangle f (original order) receives n_f = max(1, ceil(density*A_f))
 *     samples (A_f and the product in FP32, every operation rounded);
 *   - sample j of triangle f is the uniform point of Philox4x32-10 counter
 *     (j, f, sun_base + s, (design_base + d) | 2^31), key (seed lo, hi):
 *     x = v0 + sqrt(u1)(1-u2) e1 + sqrt(u1) u2 e2 (u = top 24 bits / 2^24);
 *   - with n the facet normal turned toward the sun and cos = n.e > 0, an
 *     any-hit shadow ray from x along e (the source triangle skipped, hits
 *     at t > 1e-6 R counted) decides whether x is lit; a lit sample adds
 *     (A_f/n_f) P cos [(1-rs) d - (2 rs cos + 2/3 rd) n], d = -e, and its
 *     torque (x - com) x F;
 *   - max_bounces = 2 adds, on each side n_s = +-n_e of the facet (n_e the
 *     winding normal), one gathered Lambertian interreflection: direction
 *     omega = unit(n_s + s), s the uniform unit vector z = 1 - 2 ua,
 *     phi = 2 pi ub ((ua, ub) = (u3, u4) of the sample's counter for +n_e,
 *     (u1, u2) of the counter with design word | 2^28 for -n_e); its
 *     closest hit y (source skipped, t > 1e-6 R) on the side m facing x is
 *     lit when m.e > 0 and the shadow ray from y along e is free; then
 *     E = rd_y P (m.e) and x adds (A_f/n_f) E [(1-rs)(-omega) -
 *     (2 rs cos + 2/3 rd) n_s], cos = omega.n_s, and its torque.  Only the
 *     diffuse part of y's reflection is gathered (its specular lobe is a
 *     delta that a sampled direction does not reach);
 *   - out_sigma: collapsed-strata standard errors over the sample pairs
 *     (2i, 2i+1) of k = prefix(f) + j.
 * opts: seed, pressure, mem, sun_per_design, sun_base, design_base,
 * block_threads (0 or 128), kernel_variant (0 = 8, or 4, 6, 8: the
 * minimum resident 128-thread blocks per SM the sampling kernel is
 * compiled for) and max_bounces (1 or 2; SRP_EUNSUPPORTED otherwise) are
 * used; the ray-grid fields are ignored.
 * density: samples per unit area, finite and >= 0; a design's samples must
 * stay below 2^31 (SRP_EINVAL when the planned bound exceeds it).
 * out_samples [D] int64 (opts->mem, or NULL): samples per design.
 * Uses the context's scratch like srp_force (no overlap across streams). */
int srp_force_area(srp_ctx* ctx, const srp_bvh* const* bvhs, int D, const float* rho, int G,
                   const double* sun_dir, int S, const double* com, float density,
                   const srp_trace_opts* opts, double* out_ft, double* out_sigma, int64_t* out_samples);

/* ---- local Lambertian thermal emitters (Sec. 5.9 "Design": heat of
 * on-board compute radiated from the spacecraft's faces) ------------------
 * For D designs (one item each, no sun):
 *   emit [D][G] float32   emitted flux per unit area of the triangles of each
 *                         group (>= 0; e.g. W/m^2 with opts->pressure = 1/c
 *                         gives newtons); a triangle emits on the side of
 *                         its winding normal n_e = unit((v1-v0) x (v2-v0))
 *   rho, com, bvhs, opts->mem, out_sigma, out_samples as srp_force_area;
 *   out_ft [D][6] float64 (F, tau) of the emission and of its absorption and
 *                         reflection by the spacecraft itself.
 * Emitting triangles (emit > 0) receive n_f = max(1, ceil(density*A_f))
 * samples (FP32 as in srp_force_area), others none.  Sample j of triangle
 * f: Philox4x32-10 counter (j, f, 0, (design_base + d) | 2^30); point x
 * from (u0, u1) as in srp_force_area; packet w = pressure * emit * A_f / n_f;
 * recoil -(2/3) w n_e at x (the expected recoil of a Lambertian emitter);
 * direction omega = unit(n_e + s), s the uniform unit vector
 * z = 1 - 2 u2, phi = 2 pi u3 (cosine-distributed about n_e); the closest
 * hit of x + t omega (source triangle skipped, t > 1e-6 R) receives
 * w [(1-rs) omega - (2 rs cos + 2/3 rd) n] (n the hit normal facing the
 * ray, cos = -n.omega) and its torque.  Same validation and errors as
 * srp_force_area; max_bounces must be 1; emit values are validated for
 * host-mem calls. */
int srp_force_thermal(srp_ctx* ctx, const srp_bvh* const* bvhs, int D, const float* rho, int G,
                      const float* emit, const double* com, float density, const srp_trace_opts* opts,
                      double* out_ft, double* out_sigma, int64_t* out_samples);

/* ---- a design per sample (Sec. 3.2 "Estimation": each sample meets its
 * own design, so the intersection is brute force over that design's
 * triangles; Alg. 1 NNLoss draws a random design per sample) -------------
 * Base mesh (host memory always): verts [V][3] float32, vhinge [V] int32
 * (-1 fixed, else the hinge that moves the vertex), hinges [H][6] float64
 * (pivot, unit axis; H <= 32), tris [T][3], group [T] in [0, G).
 * Per sample s (opts->mem): angles [N][H] float64 hinge angles, rho
 * [N][G][2] float32, sun [N][3] float64 unit vectors toward the sun, com
 * [N][3] float64; out_y [N][6] float64 the sample's (F, tau) estimate,
 * out_hits [N][K] int32 hit triangles (-1 after the path ends) or NULL.
 * Sample s instantiates the mesh (vertex rotated about its hinge pivot by
 * its angle, Rodrigues) and traces the jittered single pixel of a 1 x 1 grid
 * over the square of side 2*radius about center (which must bound every
 * design): Philox4x32-10 counter (0, opts->sun_base + s, 2^29, k), key
 * (seed lo, hi), weight pressure * (2 radius)^2, then srp_force's path
 * (max_bounces K <= 3, same shading, ties and t_min = 1e-6 radius).  Each
 * sample is one unbiased estimate of srp_force for its design and sun.
 * Meshes of up to 256 triangles are instantiated once per sample into
 * shared memory; larger ones are instantiated triangle by triangle as they
 * are tested.  T < 2^24, N < 2^32. */
int srp_trace_samples(srp_ctx* ctx, const float* verts, int V, const int32_t* vhinge, const double* hinges, int H,
                      const int32_t* tris, const int32_t* group, int T, const double* angles, const float* rho,
                      int G, const double* sun, const double* com, int64_t N, const double* center, double radius,
                      const srp_trace_opts* opts, double* out_y, int32_t* out_hits);

/* ---- gradient (Sec. 4.1: the simulation is differentiable by construction
 * in continuous parameters such as reflectance; Sec. 3.4 design parameters)
 * For ONE design (bvh) and S sun directions, with upstream weights
 * upstream [S][6] = dL/d(F_s, tau_s), returns the gradient of
 * L = sum_s upstream_s . (F_s, tau_s) of the same estimate srp_force
 * computes (same rays, same options):
 *   d_rho   [G][2] float64   dL/d(rho_s, rho_d) per material group (exact
 *                            along the fixed paths: the bounce branch
 *                            probability does not depend on rho)
 *   d_hinge [H]    float64   dL/d(hinge angle) (H = 0 skips it), visibility
 *                            fixed: each path keeps its facets, branch
 *                            choices and random draws; its primary hit point
 *                            is carried rigidly by its facet as the hinge
 *                            turns, later hits are re-intersected with their
 *                            (turning or fixed) facets' planes, outgoing
 *                            directions follow the turned normals
 * tri_hinge [T] int32 (by original triangle index; -1 = not on a hinge) and
 * hinge_axes [H][6] (point, unit axis; the axes the design was instantiated
 * with, srp_design_instantiate) describe the hinges; H <= 8.  The COM is
 * held fixed.  Memory per opts->mem.  Full grids whose rays_x is a
 * multiple of 32 replay only the 32-pixel batches that can meet the scene
 * (srp_force's batch pre-pass; a ray of another batch has an empty path).
 * Results are reproducible to FP32 rounding (per-warp FP32 atomics). */
int srp_force_grad(srp_ctx* ctx, const srp_bvh* bvh, const float* rho, int G,
                   const double* sun_dir, int S, const double* com,
                   const int32_t* tri_hinge, const double* hinge_axes, int H,
                   const srp_trace_opts* opts, const double* upstream,
                   double* d_rho, double* d_hinge);

/* ---- the neural proxy P(omega, theta | psi) (Sec. 3.3) --------------------
 * 19 inputs (body-frame sun direction, 16 design parameters) -> 4 hidden
 * layers of 256 with SiLU -> 6 outputs (force, torque); BF16 tensor-core
 * GEMMs with FP32 accumulation, FP32 master weights, Adam (Sec. 3.3).
 * Parameter vector (float32, srp_mlp_param_count() entries): for
 * l = 0..4, W_l [out][in] row-major then b_l [out]; sizes 19-256-256-256-
 * 256-6.  Training minimises the L1 risk mean_b sum_j |y_j - t_j| (Alg. 1,
 * NNLoss).  Inputs/targets are whatever scaling the caller chose. */
typedef struct srp_mlp srp_mlp;
int srp_mlp_param_count(int64_t* out);
/* params: host [P] initial weights, or NULL for He-uniform from `seed`. */
int srp_mlp_create(srp_ctx* ctx, const float* params, uint64_t seed, srp_mlp** out);
int srp_mlp_destroy(srp_mlp* mlp);
int srp_mlp_set_params(srp_ctx* ctx, srp_mlp* mlp, const float* params /* host [P]; resets Adam */);
int srp_mlp_get_params(srp_ctx* ctx, const srp_mlp* mlp, float* out /* host [P] */);
/* y [B][6] = P(x [B][19]); mem = srp_mem of x and y. */
int srp_mlp_infer(srp_ctx* ctx, const srp_mlp* mlp, const float* x, int64_t B, float* y, int mem);
/* One step on (x [B][19], t [B][6]): gradient of the L1 risk, then Adam
 * (beta 0.9 / 0.999, eps 1e-8) with learning rate lr when lr > 0.
 * loss_out (host float, may be NULL) receives the risk before the step;
 * grad_out (host [P], may be NULL) the gradient.  1 <= B <= 2^24. */
int srp_mlp_train_step(srp_ctx* ctx, srp_mlp* mlp, const float* x, const float* t, int64_t B, float lr,
                       float* loss_out, float* grad_out, int mem);
/* n_steps Adam steps (the optimisation loop of Sec. 3.3) on batches
 * gathered from a data set resident on the device: x [n][19] and t [n][6]
 * (device float32), idx [n_steps][batch] (device int32, row numbers of the
 * data set: step s trains on rows idx[s*batch .. s*batch + batch - 1]),
 * lr [n_steps] (host float32, each finite and > 0).  Each step computes
 * the arithmetic of srp_mlp_train_step on the gathered (x, t) with lr[s];
 * the gather is part of the first kernel's loads, and the steps are queued
 * from this call without host round trips.  Asynchronous on the context's
 * stream (idx and the data must stay valid until it has run); the caller
 * reads the loss with srp_mlp_train_step (lr = 0) or the parameters with
 * srp_mlp_get_params.  1 <= n <= 2^31, 1 <= batch <= 2^24, n_steps >= 0.
 * An index outside 0..n-1 reads a zero row and is reported by the next
 * srp_sync as SRP_EDEVICE_LIMIT. */
int srp_mlp_train_epoch(srp_ctx* ctx, srp_mlp* mlp, const float* x, const float* t, int64_t n,
                        const int32_t* idx, int64_t batch, int64_t n_steps, const float* lr);
/* Input gradient of the proxy (what Alg. 1 back-propagates from the orbit
 * loss into the design): gx [B][19] = (dy/dx)^T wy for wy [B][6], per row;
 * BF16 GEMMs with FP32 accumulation as in training.  mem = srp_mem of x, wy
 * and gx; device-mem calls are asynchronous.  0 <= B <= 2^24.  Shares the
 * network's training scratch (do not overlap with train_step on another
 * stream). */
int srp_mlp_grad_input(srp_ctx* ctx, srp_mlp* mlp, const float* x, const float* wy, int64_t B, float* gx, int mem);
/* Parameter files: 8-byte tag "SRPMLP1\0", int64 count, FP32 parameters in
 * the order above (host byte order).  Load resets Adam; a file of another
 * size or tag is SRP_EINVAL. */
int srp_mlp_save(srp_ctx* ctx, const srp_mlp* mlp, const char* path);
int srp_mlp_load(srp_ctx* ctx, srp_mlp* mlp, const char* path);
/* Trainer state for checkpoint and resume of training (Sec. 3.3 trains the
 * proxy by Adam): parameters, both Adam moment vectors and the step count.
 * File: 8-byte tag "SRPMLS1\0", int64 P, int64 step, then parameters, first
 * moments and second moments as float32 [P] each (host byte order).  Save
 * waits for the context's stream; load replaces all of it, so the next
 * srp_mlp_train_step continues the interrupted run (the weight-gradient
 * reduction sums in a run-dependent FP32 order, so a resumed run matches an
 * uninterrupted one to that rounding, not bit for bit).  A file of another
 * tag or size, or with non-finite or negative second moments, is SRP_EINVAL
 * and leaves the network unchanged. */
int srp_mlp_save_state(srp_ctx* ctx, const srp_mlp* mlp, const char* path);
int srp_mlp_load_state(srp_ctx* ctx, srp_mlp* mlp, const char* path);

/* ---- orbit integration and its adjoint (Sec. 3.4, Eq. "ODE", RK4 of
 * Sec. 3.4.1, adjoint of Sec. 3.4.3) --------------------------------------
 * State z (13) = (r [m], v [m/s] inertial; unit quaternion q = (q0..q3)
 * taking body vectors to inertial; body rate w [rad/s]).
 *   r' = v,  v' = R(q) F / m + gravity(r) (two-body + J2),
 *   q' = q (x) (0, w) / 2,  w' = I^-1 (tau - w x I w)  (I diagonal),
 * (F, tau) = pressure * (out_std * y + out_mean), y = force model at the
 * body-frame sun direction wbar = R(q)^T sun and the design theta:
 *   SRP_FM_NONE        y = 0
 *   SRP_FM_CANNONBALL  y = (-theta[0] wbar, 0) (theta[0] = area x (1+4 rho_d/9))
 *   SRP_FM_PROXY       y = MLP(in_scale * (wbar, theta) + in_offset), n_theta = 16
 * Optional terms (Sec. 3.4 "additional accelerations"): the cylinder
 * eclipse (SRP off while r.sun < 0 and |r - (r.sun) sun| < re) and point
 * masses at fixed inertial positions, GM [(s - r)/|s - r|^3 - s/|s|^3]
 * (the paper's Sun/Moon from ephemerides; positions are inputs here).
 * The eclipse switch is piecewise constant: its derivative is zero (the
 * adjoint does not see the shadow boundary).
 * RK4 in FP64 with step dt (the MLP runs in FP32).  With dL_dzN given, the
 * discrete adjoint of the RK4 map (checkpoints every ckpt_every steps,
 * 0 = ceil(sqrt(n_steps)), at most 64) returns dL/dtheta and dL/dz0. */
#define SRP_FM_NONE 0
#define SRP_FM_CANNONBALL 1
#define SRP_FM_PROXY 2
typedef struct srp_orbit_opts {
    double mu, j2, re;        /* [3.986004418e14, 1.08263e-3, 6378137]       */
    double mass;              /* kg [1000]                                    */
    double inertia[3];        /* diagonal, kg m^2 [500, 400, 300]             */
    double pressure;          /* N/m^2 [1361 / c]                             */
    double sun[3];            /* inertial unit vector toward the sun [1,0,0] */
    double dt;                /* s [60]                                       */
    int32_t n_steps;          /* [1440]                                       */
    int32_t ckpt_every;       /* [0]                                          */
    int32_t model;            /* SRP_FM_* [NONE]                              */
    int32_t n_theta;          /* 1..16 [1]                                    */
    float in_scale[19], in_offset[19];   /* proxy input map [1, 0]            */
    float out_mean[6], out_std[6];       /* model output map [0, 1]           */
    int32_t eclipse;          /* 1: cylinder shadow of radius re along -sun  */
                              /*    switches F and tau off [0]               */
    int32_t reserved0;
    double gm_sun;            /* m^3/s^2 point mass at sun_dist * sun [0=off] */
    double sun_dist;          /* m [1.495978707e11]                           */
    double gm_moon;           /* m^3/s^2 point mass at moon [0 = off]         */
    double moon[3];           /* inertial position, m [0]                     */
} srp_orbit_opts;
void srp_orbit_opts_default(srp_orbit_opts* o);
/* n_traj trajectories, one CTA each:  z0 [n][13], theta [n][n_theta] ->
 * zN [n][13], traj [n][n_steps+1][13] (or NULL); adjoint when dL_dzN
 * [n][13] is given: dL_dtheta [n][n_theta], dL_dz0 [n][13] (either may be
 * NULL).  proxy may be NULL unless model = SRP_FM_PROXY.  mem = srp_mem of
 * every array. */
int srp_integrate(srp_ctx* ctx, const srp_orbit_opts* opts, const srp_mlp* proxy, int n_traj,
                  const double* z0, const double* theta, double* zN, double* traj,
                  const double* dL_dzN, double* dL_dtheta, double* dL_dz0, int mem);

/* Force and torque without any GPU allocation.  The paper has no
 * counterpart; this exists for callers that cannot allocate device memory
 * when they need forces (an allocator policy that forbids allocations after
 * start-up, a host framework that only hands over a stream and device
 * pointers, a real-time loop that must not stall on an allocation).
 * Same arguments and results as srp_force with mem = SRP_MEM_DEVICE (all
 * arrays device memory, required), but no context: work is issued on
 * `cuda_stream` (a cudaStream_t, NULL = legacy default stream) on the
 * CURRENT device, where the bvhs must have been built.  The per-chunk FP64
 * partial sums live in one fixed 8 MiB array inside the library (a
 * file-scope device variable, held by every GPU that loads the library
 * until the process exits), so D*S may be at most 87,381 (and
 * D*S*chunks_per_item the same when given), and the design table in a
 * fixed array of 4,096 entries (D <= 4,096); larger requests fail with
 * SRP_EINVAL.  Every fixed array (the partials, the design table, the
 * pre-pass tables, the error word and the work-queue counter) is shared by every call on a
 * device and keeps the last call's contents: calls whose work overlaps on
 * the GPU (unordered streams) race on all of them and must not be issued --
 * besides corrupting the sums, one call can rewrite the design table while
 * the other's kernel reads it and then read out of bounds.  The first call
 * on each device looks up the arrays' addresses with that device current;
 * make it before any stream capture begins.  On full grids whose rays_x
 * is a multiple of 32 it runs srp_force's batch pre-pass (the 32-pixel
 * batches that cannot meet the scene are not traced), with its per-row
 * tables and per-item constants in a second fixed array of 16 MiB (shared
 * like the others): D*S*(8*rays_y + 4) + 128*D*S bytes must fit, about
 * 2,000 (design, sun) items at rays_y = 1024; larger calls, ray subsets and
 * other widths trace every ray (slower on such grids, sums grouped
 * differently: equal up to the rounding of that grouping).  With
 * chunks_per_item = 0 it picks chunks as srp_force does, capped so that
 * D*S*chunks fits the array.
 * d_status (device int32, may be NULL) receives the device-limit flags of
 * the call (0 = none; see SRP_EDEVICE_LIMIT).  Asynchronous; calls no
 * cudaMalloc/cudaFree or other allocating routine, and takes no host heap
 * memory either when it succeeds (the design table travels to the device in
 * the parameters of small kernel launches, 64 entries each). */
int srp_force_noalloc(const srp_bvh* const* bvhs, int D, const float* rho, int G,
                      const double* sun_dir, int S, const double* com, const srp_trace_opts* opts,
                      double* out_ft, double* out_sigma, int32_t* d_status, void* cuda_stream);

/* CUDA graph of one srp_force evaluation: the same arguments (device
 * memory only, opts->mem = SRP_MEM_DEVICE) are captured once, with the
 * design table copied into the graph; srp_graph_launch replays the
 * evaluation (queue reset, the batch pre-pass of whole grids, one
 * persistent trace launch over every (design, sun, chunk) unit, reduction)
 * on the context's stream, reading
 * rho/sun_dir/com and writing out_ft/out_sigma at the captured addresses.
 * The graph uses the context's scratch (partial sums, pre-pass tables) at
 * the addresses it had when the graph was captured: no other srp_force or
 * graph of the same context may run concurrently, and a later call on the
 * same context that needs more scratch than the graph's evaluation (more
 * (design, sun) items or chunks, more grid rows) grows the scratch by
 * reallocating it, after which the graph must not be launched again --
 * create graphs after the context's largest call, or give each graph a
 * context of its own. */
typedef struct srp_graph srp_graph;
int srp_force_graph_create(srp_ctx* ctx, const srp_bvh* const* bvhs, int D, const float* rho, int G,
                           const double* sun_dir, int S, const double* com, const srp_trace_opts* opts,
                           double* out_ft, double* out_sigma, srp_graph** out);
int srp_graph_launch(srp_graph* graph);
int srp_graph_destroy(srp_graph* graph);

/* Per-ray inspection (the estimator's individual samples): trace the n
 * grid rays ray_idx[n] (int64, each < rays_x*rays_y) of ONE design and ONE
 * sun direction with the same arithmetic as srp_force.
 *   rho [G][2] float32, sun_dir [3] float64, com [3] float64
 *   sun_index, design_index: the indices used in the Philox counter
 *   out_y    [n][6] float64: the ray's force and torque deposits
 *   out_hits [n][K] int32: original index of the triangle hit at each
 *            bounce (-1 when the path has ended), K = opts->max_bounces
 * Memory per opts->mem.  ray_offset/stride/count and sun_per_design in
 * opts are ignored. */
int srp_trace_rays(srp_ctx* ctx, const srp_bvh* bvh, const float* rho, int G, const double* sun_dir,
                   const double* com, const int64_t* ray_idx, int64_t n, int sun_index, int design_index,
                   const srp_trace_opts* opts, double* out_y, int32_t* out_hits);

#ifdef __cplusplus
}
#endif
#endif /* SRP_H */
