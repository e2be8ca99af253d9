// train.cu -- training step and input gradient of the neural proxy
// (Sec. 3.3: the proxy is fitted to traced forces by minimising the L1 risk
// with Adam; Sec. 3.4 differentiates it inside the design loop) on the
// tcgen05 tensor cores, BF16 operands and FP32 accumulators in TMEM.
//
// One step is four kernels (three without the Adam update):
//   train_fwd_kernel  one CTA per 128-row tile: the five layers in turn
//                     (weights by bulk copy, one thread issues the MMAs, 16
//                     epilogue warps, four per TMEM lane quarter, each on
//                     64 of the 256 columns);
//                     the epilogue adds the bias, applies SiLU, writes the
//                     next layer's BF16 A operand into shared memory and
//                     keeps silu'(z) (FP32) for the backward pass; each
//                     layer's A operand is bulk-copied out as it stands (a
//                     tile image) for the weight gradients; the last
//                     layer gives the L1 loss, dL/dy = sign(y - t)/B and the
//                     output bias gradient;
//   train_bwd_kernel  one CTA per tile: dL/dh = dL/dz W through the layers
//                     from the top (transposed packed weights), the
//                     epilogue multiplies by silu'(z), writes the BF16
//                     operand of the next product (copied out as a tile
//                     image of dL/dz) and sums the bias gradient over the
//                     tile's rows;
//   train_dw_kernel   the weight gradients dW_l = (dL/dz_l)^T h_l, batch
//                     along K split over CTAs, the tile images read as
//                     MN-major operands (bulk-copied, double-buffered), FP32
//                     vector atomics into the gradient;
//   adam_pack_kernel  Adam, and the updated weights into both BF16 packed
//                     layouts, when lr > 0.
// Rounding points (what the oracle's round_act / round_grad reproduce):
// every product consumes BF16 operands -- weights, inputs, activations,
// back-propagated dL/dz -- and accumulates in FP32; silu'(z), the bias
// gradients and the loss are FP32 from unrounded values.
// Every mbarrier wait is bounded; a CTA that gives up records
// kErrWaitTimeout, waits (bounded) for its copies and MMAs in flight, frees
// its TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "mlp_common.cuh"
#include "srp_internal.h"

namespace srp {

// ---------------------------------------------------------------------------
// Workspace.  Bp = B rounded up to 128.  The operands of the weight
// gradients are kept as "tile images": per 128-row batch tile, the BF16
// A operand of a layer exactly as it sat in shared memory (K-major core
// matrices, the F features along K: element (r, f) of tile t at byte
// t * 128 * F * 2 + kmajor_off(r, f, F)), bulk-copied out by the forward and
// backward kernels.  Rows 64 h .. 64 h + 63 of a tile are one contiguous run
// of 64 * F * 2 bytes, and the weight-gradient kernel reads such a run MN-major
// (features along M or N, batch rows along K) -- no transposition anywhere.
// ---------------------------------------------------------------------------
struct TrainWS {
    float* S[4];                 // silu'(z_l), Bp x 256 FP32 in row groups (s_quad), l = 0..3
    __nv_bfloat16* Him[5];       // tile images of the layer inputs: Him[0] = x (F = 32), Him[l] = h_l (F = 256)
    __nv_bfloat16* DZim[5];      // tile images of dL/dz_l (F = 256), DZim[4] = dL/dy (F = 16)
    float* dY;                   // dL/dy [Bp][8] FP32 (columns 6, 7 zero)
    float* lossp;                // [Bp / 32]: the L1 loss of each 32-row warp of the forward's output layer
    float* loss;                 // [1]: their sum, by the weight-gradient kernel
};

__host__ __device__ inline int64_t train_bp(int64_t B) { return (B + 127) / 128 * 128; }

static size_t al1k(size_t x) { return (x + 1023) / 1024 * 1024; }

size_t train_bytes(int64_t B) {
    const size_t Bp = (size_t)train_bp(B);
    return 4 * al1k(Bp * 256 * 4) + al1k(32 * Bp * 2) + 4 * al1k(256 * Bp * 2) + 4 * al1k(256 * Bp * 2) +
           al1k(16 * Bp * 2) + al1k(Bp * 8 * 4) + al1k(Bp / 32 * 4) + 1024;
}

static TrainWS train_carve(void* base, int64_t B) {
    const size_t Bp = (size_t)train_bp(B);
    unsigned char* q = (unsigned char*)base;
    TrainWS w;
    for (int l = 0; l < 4; ++l) { w.S[l] = (float*)q; q += al1k(Bp * 256 * 4); }
    w.Him[0] = (__nv_bfloat16*)q; q += al1k(32 * Bp * 2);
    for (int l = 1; l < 5; ++l) { w.Him[l] = (__nv_bfloat16*)q; q += al1k(256 * Bp * 2); }
    for (int l = 0; l < 4; ++l) { w.DZim[l] = (__nv_bfloat16*)q; q += al1k(256 * Bp * 2); }
    w.DZim[4] = (__nv_bfloat16*)q; q += al1k(16 * Bp * 2);
    w.dY = (float*)q; q += al1k(Bp * 8 * 4);
    w.lossp = (float*)q; q += al1k(Bp / 32 * 4);
    w.loss = (float*)q;
    return w;
}

float* train_loss_ptr(void* work, int64_t B) { return train_carve(work, B).loss; }

// silu'(z) of one layer, Bp x 256 FP32, stored by groups of 32 rows and
// quads of 4 features: element (row, f) at float
// ((row / 32) * 64 + f / 4) * 128 + (row % 32) * 4 + f % 4.  The epilogue
// thread of row r holds 32 consecutive features of its row, so the warp's
// float4 store (or load) of one quad is 512 contiguous bytes rather than 32
// lines 1 KB apart.  Returns the quad of (row, f), f a multiple of 4.
__device__ __forceinline__ float4* s_quad(float* S, int64_t row, int f) {
    return reinterpret_cast<float4*>(S + (((row >> 5) * 64 + (f >> 2)) * 128 + (row & 31) * 4));
}

// Offsets (elements) of every layer's FP32 weights and biases in the flat
// parameter vector and of its two BF16 packed layouts, in constant memory:
// the kernels index them by a runtime layer number without a local-memory
// copy of the table.
struct TrainOffsets {
    int64_t w[kMlpLayers], b[kMlpLayers], p[kMlpLayers], pT[kMlpLayers];
};
__host__ __device__ constexpr TrainOffsets train_offsets() {
    TrainOffsets t{};
    int64_t o = 0, q = 0;
    for (int l = 0; l < kMlpLayers; ++l) {
        t.w[l] = o;
        o += (int64_t)mlp_in(l) * mlp_out(l);
        t.b[l] = o;
        o += mlp_out(l);
        t.p[l] = q;
        q += (int64_t)mlp_N(l) * mlp_K(l);
    }
    for (int l = 0; l < kMlpLayers; ++l) {
        t.pT[l] = q;
        q += (int64_t)mlp_NT(l) * mlp_KT(l);
    }
    return t;
}
static __constant__ TrainOffsets c_off = train_offsets();

__device__ __forceinline__ uint32_t bf16x2(float lo, float hi) {
    uint32_t p;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(p) : "f"(hi), "f"(lo));
    return p;
}

// Warp transpose-reduction: lane c ends with the sum over the warp's 32
// lanes of their t[c] (recursive halving: 31 shuffles for 32 columns).
__device__ __forceinline__ float warp_colsum32(float (&t)[32], int lane) {
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < off; ++i) {
            const float send = up ? t[i] : t[i + off];
            const float keep = up ? t[i + off] : t[i];
            t[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
    return t[0];
}

// A tile's 128 rows are processed by one CTA (PAIR = 1) or, when the batch
// has too few tiles to fill the GPU, by a cluster of two CTAs (PAIR = 2, one
// SM each): in every 256-wide layer CTA rank c then computes the output
// features [128 c, 128 c + 128) -- half the MMA N and half the epilogue --
// and writes its half of the next layer's BF16 A operand into its own
// shared memory; one thread then bulk-copies that half into the partner's
// (distributed shared memory, 16 runs of 2 KB, completing on an mbarrier of
// the receiving CTA, which expects the 32 KB before it waits).  The pair's A
// operand is double buffered (layer l reads act[l & 1], its epilogue writes
// act[(l + 1) & 1]), so a CTA never writes into a buffer its partner's
// tensor core may still read.  The narrow layers (the 6 outputs, the 19
// input gradients) run on rank 0 alone.  16 warps per CTA: warp w reads
// TMEM lane quarter w % 4 (32 rows) and a quarter of the CTA's columns.
// Once a layer's MMAs are issued, the thread that issued them also copies
// the A operand out to its tile image (rank c of a pair: rows 64 c ..
// 64 c + 63), and waits for that copy to have read shared memory before the
// epilogue may write into it again.
constexpr int kTrThreads = 512;
constexpr int kDwThreads = 128;

template <int PAIR>
struct TrainSmem {
    static constexpr int NH = 256 / PAIR;                // output features of a 256-wide layer per CTA
    alignas(1024) unsigned char act[PAIR][128 * 256 * 2];   // A operand(s) (64 KB each)
    alignas(1024) unsigned char w[256 * NH * 2];         // B operand: this CTA's share of a layer
    alignas(16) float colsum[NH];   // backward: bias-gradient sums of the tile; forward: this CTA's biases of the layer
    alignas(8) uint64_t bar_w;
    alignas(8) uint64_t bar_mma;
    alignas(8) uint64_t bar_peer[2];                     // the partner's k-th half of an A operand landed (k & 1)
    uint32_t tmem_base;
    int fail;
};

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// shared::cluster address of the same shared variable in CTA `rank`
__device__ __forceinline__ uint32_t peer_addr(const void* p, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(tc::smem_u32(p)), "r"(rank));
    return r;
}
// bulk copy of `bytes` from this CTA's shared memory to shared::cluster
// address `dst`, completing (complete_tx) on the mbarrier at `bar`
__device__ __forceinline__ void bulk_s2peer(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     dst),
                 "r"(tc::smem_u32(src)), "r"(bytes), "r"(bar)
                 : "memory");
}
constexpr uint32_t kPeerHalfBytes = 128u * 128u * 2u;   // a partner's half of a K = 256 A operand
__device__ __forceinline__ bool mbar_wait_cluster_bounded(uint64_t* bar, uint32_t parity, uint32_t limit) {
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(tc::smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
        if (it > 64) __nanosleep(64);
    }
    return false;
}
// both CTAs of the pair (kernel start and end only: every thread reaches them)
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Programmatic dependent launch.  The backward, weight-gradient and Adam
// kernels are launched with programmatic stream serialisation: they may
// start while their predecessor in the stream still runs, do their set-up
// (barriers, TMEM, weights that no kernel of the step writes), and wait
// here before reading anything the predecessor wrote.  Each kernel lets its
// dependent be scheduled once all of its own CTAs are resident.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Thread 0: rows [r0, r0 + nr) of each of the K / KC chunks of a packed
// layer (N x KC K-major tiles) into sm.w, one bulk copy per chunk.
template <int PAIR>
__device__ __forceinline__ void load_w_rows(TrainSmem<PAIR>& sm, const unsigned char* layer, int N, int K, int KC, int r0,
                                            int nr) {
    const uint32_t cb = (uint32_t)(nr * KC * 2);
    tc::mbar_expect_tx(&sm.bar_w, cb * (uint32_t)(K / KC));
    for (int c = 0; c < K / KC; ++c)
        tc::bulk_g2s(sm.w + c * cb, layer + (size_t)c * N * KC * 2 + (size_t)r0 * KC * 2, cb, &sm.bar_w);
}

// Thread 0: D = A (act[buf], K columns) x B^T (sm.w: N rows, chunks of KC), commit.
template <int PAIR>
__device__ __forceinline__ void issue_layer(TrainSmem<PAIR>& sm, uint32_t tbase, int buf, int N, int K, int KC) {
    const uint32_t idesc = tc::idesc_bf16(128, (uint32_t)N);
    const uint32_t a0 = tc::smem_u32(sm.act[buf % PAIR]), b0 = tc::smem_u32(sm.w);
    const uint32_t sboA = (uint32_t)(K / 8) * 128u, sboB = (uint32_t)(KC / 8) * 128u;
    for (int kk = 0; kk < K / 16; ++kk) {
        const int c = kk / (KC / 16), j = kk - c * (KC / 16);
        const uint64_t ad = tc::sdesc(a0 + 256u * (uint32_t)kk, 128u, sboA);
        const uint64_t bd = tc::sdesc(b0 + (uint32_t)c * (uint32_t)(N * KC * 2) + 256u * (uint32_t)j, 128u, sboB);
        tc::mma_bf16(tbase, ad, bd, idesc, kk > 0 ? 1u : 0u);
    }
    tc::mma_commit(&sm.bar_mma);
}

// The partner's k-th signal (k = 0, 1, ...) arrives on bar_peer[k & 1] and
// completes its phase k >> 1: the two barriers alternate, so a partner one
// signal ahead (the most it can be) never advances the barrier being
// waited on past the phase awaited.
// Thread 0 arms the phase with the 32 KB it expects (the partner's copy may
// land before or after) and waits for it.
template <int PAIR>
__device__ __forceinline__ bool wait_peer(TrainSmem<PAIR>& sm, int k) {
    tc::mbar_expect_tx(&sm.bar_peer[k & 1], kPeerHalfBytes);
    return mbar_wait_cluster_bounded(&sm.bar_peer[k & 1], (uint32_t)(k >> 1) & 1u, kWaitLimit);
}

// Copy-out of an A operand into its tile image: `bytes` from byte `off` of
// the buffer to img + off (img null: none).
struct ImgCopy {
    unsigned char* img;
    uint32_t off, bytes;
};

// The copy-out of a tile's A operand (F features) into image `img`: the
// whole tile, or (pairs) rank c's rows 64 c .. 64 c + 63.
template <int PAIR>
__device__ __forceinline__ ImgCopy img_copy(__nv_bfloat16* img, int64_t tile, int F, uint32_t rank, bool whole) {
    unsigned char* base = reinterpret_cast<unsigned char*>(img) + (size_t)tile * 128 * F * 2;
    const uint32_t half = 64u * (uint32_t)F * 2u;
    if (PAIR == 1 || whole) return ImgCopy{base, 0u, 2u * half};
    return ImgCopy{base, rank * half, half};
}

// The per-layer handshake: thread 0 waits for the weights and, when
// `peer_k` >= 0, for the partner's signal peer_k (its half of the A
// operand), issues the MMAs and the copy-out `cp`; everyone waits for the
// MMAs (thread 0 also for the copy to have read its source).  Returns 0, or
// 1 (weights or the partner never arrived) / 2 (MMAs never completed) when a
// bounded wait gave up (block-uniform).
template <int PAIR>
__device__ __forceinline__ int run_layer(TrainSmem<PAIR>& sm, uint32_t tbase, int buf, int N, int K, int KC, int peer_k,
                                         uint32_t& ph_w, uint32_t& ph_m, ImgCopy cp = ImgCopy{nullptr, 0u, 0u}) {
    if (threadIdx.x == 0) {
        bool ok = tc::mbar_wait_bounded(&sm.bar_w, ph_w, kWaitLimit);
        if (ok && peer_k >= 0) ok = wait_peer(sm, peer_k);
        sm.fail = ok ? 0 : 1;
        if (ok) {
            tc::tc_fence_after();
            issue_layer(sm, tbase, buf, N, K, KC);
            if (cp.img) {
                tc::bulk_s2g(cp.img + cp.off, sm.act[buf % PAIR] + cp.off, cp.bytes);
                tc::bulk_commit();
            }
        }
    }
    __syncthreads();
    if (sm.fail) return 1;
    ph_w ^= 1u;
    const bool ok = tc::mbar_wait_bounded(&sm.bar_mma, ph_m, kWaitLimit);
    if (threadIdx.x == 0 && cp.img) tc::bulk_wait_read0();
    ph_m ^= 1u;
    if (__syncthreads_or(!ok)) return 2;
    tc::tc_fence_after();
    return 0;
}

template <int PAIR>
__device__ __forceinline__ void train_setup(TrainSmem<PAIR>& sm) {
    if (threadIdx.x == 0) {
        tc::mbar_init(&sm.bar_w, 1);
        tc::mbar_init(&sm.bar_mma, 1);
        tc::mbar_init(&sm.bar_peer[0], 1);
        tc::mbar_init(&sm.bar_peer[1], 1);
        tc::fence_mbar_init();
    }
    if (threadIdx.x < 32) {
        tc::tmem_alloc(&sm.tmem_base, TrainSmem<PAIR>::NH);
        tc::tmem_relinquish();
    }
    for (int i = threadIdx.x; i < TrainSmem<PAIR>::NH; i += kTrThreads) sm.colsum[i] = 0.0f;
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (PAIR == 2) cluster_sync();   // the partner's barriers exist before anyone arrives on them
}

// After the epilogue: this CTA's writes into A buffer `buf` visible to the
// async proxy (its tensor core and bulk copies), then thread 0 copies this
// CTA's half (features 128 c .. 128 c + 127: 2 KB in each of the 16 8-row
// groups) into the partner's `buf`, as signal k.
template <int PAIR>
__device__ __forceinline__ void signal_peer(TrainSmem<PAIR>& sm, uint32_t peer, int k, const unsigned char* buf) {
    tc::fence_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    if (PAIR == 2 && threadIdx.x == 0) {
        const uint32_t bar = peer_addr(&sm.bar_peer[k & 1], peer);
        const uint32_t half = (peer ^ 1u) * 2048u;
        for (int g = 0; g < 16; ++g) {
            const unsigned char* src = buf + g * 4096 + half;
            bulk_s2peer(peer_addr(src, peer), src, 2048u, bar);
        }
    }
}

// End of the kernel: record a failed wait, let the copy or the MMAs in
// flight land (bounded), wait (bounded) for the partner's last signal so
// that no write into this CTA's shared memory is still under way, free
// TMEM, and leave together with the partner.
template <int PAIR>
__device__ __forceinline__ void train_teardown(TrainSmem<PAIR>& sm, uint32_t tbase, int failed, uint32_t ph_w,
                                               uint32_t ph_m, int last_peer_k, int* err) {
    if (threadIdx.x == 0) {
        if (failed) {
            atomicOr(err, kErrWaitTimeout);
            if (failed == 1) tc::mbar_wait_bounded(&sm.bar_w, ph_w, kWaitLimit);
            else tc::mbar_wait_bounded(&sm.bar_mma, ph_m ^ 1u, kWaitLimit);
        }
        if (last_peer_k >= 0 && !wait_peer(sm, last_peer_k)) atomicOr(err, kErrWaitTimeout);
        tc::bulk_wait0();   // the tile-image copies have landed
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (threadIdx.x < 32) tc::tmem_dealloc(tbase, TrainSmem<PAIR>::NH);
    if (PAIR == 2) cluster_sync();
}

// Writes the thread's 32 BF16 values (pk, features f0 .. f0 + 31 of row r)
// into A buffer `dst` (K = 256 layout) of this CTA.
__device__ __forceinline__ void put_act(unsigned char* dst, const uint32_t (&pk)[16], int r, int f0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        unsigned char* p = dst + tc::kmajor_off((uint32_t)r, (uint32_t)(f0 + 8 * q), 256u);
        *reinterpret_cast<uint4*>(p) = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
    }
}

// ---------------------------------------------------------------------------
// Forward.  mode 0: training (targets t: loss, dL/dy, output bias gradient,
// tile images of the inputs and activations for the weight gradients);
// mode 1: the input gradient's forward (silu'(z) of the hidden layers only).
// idx (may be NULL): batch row r reads row idx[r] of x and tgt, which hold
// n_src rows (the batch gather of a training epoch, fused into the loads);
// an index outside 0..n_src-1 sets kErrRowIndex and reads zeros.
// ---------------------------------------------------------------------------
template <int PAIR>
__global__ void __launch_bounds__(kTrThreads, 1)
    train_fwd_kernel(const float* __restrict__ x, const float* __restrict__ tgt, const int32_t* __restrict__ idx,
                     int64_t n_src, int64_t B, int64_t Bp, const __nv_bfloat16* __restrict__ packed,
                     const float* __restrict__ params, TrainWS ws, float* __restrict__ grad, int mode, int* err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    using Smem = TrainSmem<PAIR>;
    constexpr int NH = Smem::NH;
    Smem& sm = *reinterpret_cast<Smem*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, part = warp >> 2, r = 32 * quarter + lane;
    const uint32_t rank = PAIR == 2 ? cluster_rank() : 0u, peer = rank ^ 1u;
    const unsigned char* pb = reinterpret_cast<const unsigned char*>(packed);
    train_setup(sm);
    const uint32_t tbase = sm.tmem_base;
    grid_dep_launch();
    const int64_t tile = blockIdx.x / PAIR, row = tile * 128 + r;
    // the data-set row of this batch row (warps 0-3 read x and tgt)
    bool in_rows = row < B;
    int64_t src = row;
    if (idx != nullptr && part == 0 && in_rows) {
        src = (int64_t)__ldg(idx + row);
        if (src < 0 || src >= n_src) {
            if (rank == 0) atomicOr(err, kErrRowIndex);
            in_rows = false;
        }
    }
    if (tid == 0) load_w_rows(sm, pb + 2 * c_off.p[0], mlp_N(0), mlp_K(0), mlp_KC(0), NH * (int)rank, NH);
    // training: the gradient starts from zero (the backward and weight-
    // gradient kernels accumulate into it once this grid has completed)
    if (mode == 0)
        for (int64_t e = (int64_t)blockIdx.x * kTrThreads + tid; e < kMlpParams; e += (int64_t)gridDim.x * kTrThreads)
            grad[e] = 0.0f;
    // the tile's inputs (warps 0-3, one row each): BF16 A operand (K = 32,
    // zero padded) in both CTAs
    if (part == 0) {
        float v[19];
#pragma unroll
        for (int j = 0; j < 19; ++j) v[j] = in_rows ? __ldg(x + src * 19 + j) : 0.0f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t u[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int k = 8 * q + 2 * j;
                u[j] = bf16x2(k < 19 ? v[k] : 0.0f, k + 1 < 19 ? v[k + 1] : 0.0f);
            }
            *reinterpret_cast<uint4*>(sm.act[0] + tc::kmajor_off(r, 8 * q, 32)) = make_uint4(u[0], u[1], u[2], u[3]);
        }
    }
    tc::fence_async_smem();
    __syncthreads();
    uint32_t ph_w = 0, ph_m = 0;
    int failed = 0;
    const uint32_t taddr = tbase + ((uint32_t)(32 * quarter) << 16);
    // hidden layers 0-3: this CTA's NH features (all of them, or one half)
    for (int l = 0; l < kMlpLayers - 1; ++l) {
        // the layer's biases of this CTA's features into shared memory (the
        // last NH threads; the previous epilogue's reads ended at its
        // barrier, run_layer's barrier orders these writes before the reads)
        if (tid >= kTrThreads - NH) {
            const int c = tid - (kTrThreads - NH);
            sm.colsum[c] = __ldg(params + c_off.b[l] + NH * (int)rank + c);
        }
        const ImgCopy cp = mode == 0 ? img_copy<PAIR>(ws.Him[l], tile, mlp_K(l), rank, false) : ImgCopy{nullptr, 0u, 0u};
        failed = run_layer(sm, tbase, l & 1, NH, mlp_K(l), mlp_KC(l), PAIR == 2 ? l - 1 : -1, ph_w, ph_m, cp);
        if (failed) break;
        // the weights of layer l are consumed: bring the next layer's
        if (tid == 0) {
            if (l + 1 < kMlpLayers - 1)
                load_w_rows(sm, pb + 2 * c_off.p[l + 1], mlp_N(l + 1), mlp_K(l + 1), mlp_KC(l + 1), NH * (int)rank, NH);
            else if (mode == 0 && rank == 0)
                load_w_rows(sm, pb + 2 * c_off.p[kMlpLayers - 1], mlp_N(kMlpLayers - 1), mlp_K(kMlpLayers - 1),
                            mlp_KC(kMlpLayers - 1), 0, mlp_N(kMlpLayers - 1));
        }
        // silu' of the last 32-feature chunk is stored after the hand-off to
        // the partner, so that the proxy fence before it does not wait for
        // these global stores
        float v[32];
        int f_last = 0;
#pragma unroll 1
        for (int cc = 0; cc < NH / 128; ++cc) {
            const int f_loc = (NH / 4) * part + 32 * cc, f_glob = NH * (int)rank + f_loc;   // 32 features
            const float* bias = sm.colsum + f_loc;
            tc::tmem_ld32(taddr + (uint32_t)f_loc, v);
            uint32_t pk[16];
#pragma unroll
            for (int j = 0; j < 32; j += 2) {
                float h[2];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const float z = v[j + e] + bias[j + e];
                    // sigmoid by the hardware exp2 and reciprocal (about 2^-21
                    // relative each, for every z: no cancellation)
                    const float s = __fdividef(1.0f, 1.0f + __expf(-z));
                    h[e] = z * s;
                    v[j + e] = s * (1.0f + z * (1.0f - s));   // silu'(z)
                }
                pk[j / 2] = bf16x2(h[0], h[1]);
            }
            put_act(sm.act[((l + 1) & 1) % PAIR], pk, r, f_glob);
            if (cc + 1 < NH / 128) {
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    *s_quad(ws.S[l], row, f_glob + 4 * q) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            }
            f_last = f_glob;
        }
        signal_peer(sm, peer, l, sm.act[((l + 1) & 1) % PAIR]);
#pragma unroll
        for (int q = 0; q < 8; ++q)
            *s_quad(ws.S[l], row, f_last + 4 * q) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    }
    int last_peer_k = (failed || PAIR == 1) ? -1 : kMlpLayers - 2;   // the partner's signal of layer 3
    if (!failed && mode == 0 && rank == 0) {
        // output layer on rank 0 (the image of its whole input tile too):
        // the loss of each warp's 32 rows and dL/dy
        const int l = kMlpLayers - 1;
        failed = run_layer(sm, tbase, l & 1, mlp_N(l), mlp_K(l), mlp_KC(l), PAIR == 2 ? l - 1 : -1, ph_w, ph_m,
                           img_copy<PAIR>(ws.Him[l], tile, mlp_K(l), rank, true));
        last_peer_k = -1;   // already waited for before the MMAs (or failed)
        if (!failed && part == 0) {
            float v[16];
            tc::tmem_ld16(taddr, v);
            const float invB = 1.0f / (float)B;
            float lsum = 0.0f;
            float dy[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                dy[j] = 0.0f;
                if (j < 6 && row < B) {
                    const float d = v[j] + __ldg(params + c_off.b[l] + j) - (in_rows ? __ldg(tgt + src * 6 + j) : 0.0f);
                    dy[j] = d > 0.0f ? invB : (d < 0.0f ? -invB : 0.0f);
                    lsum += fabsf(d);
                }
            }
            reinterpret_cast<float4*>(ws.dY + row * 8)[0] = make_float4(dy[0], dy[1], dy[2], dy[3]);
            reinterpret_cast<float4*>(ws.dY + row * 8)[1] = make_float4(dy[4], dy[5], dy[6], dy[7]);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
            if (lane == 0) ws.lossp[tile * 4 + quarter] = lsum * invB;
        }
    }
    train_teardown(sm, tbase, failed, ph_w, ph_m, last_peer_k, err);
}

// ---------------------------------------------------------------------------
// Backward.  dy: dL/dy rows (ld floats per row; training: the forward's dY,
// input gradient: the caller's weights wy).  mode 0: training (down to
// dL/dz_0, tile images of dL/dz and bias gradients); mode 1: the input gradient
// gx = dL/dz_0 W_0 (FP32 [B][19], on rank 0).
// ---------------------------------------------------------------------------
template <int PAIR>
__global__ void __launch_bounds__(kTrThreads, 1)
    train_bwd_kernel(const float* __restrict__ dy, int ld, int64_t B, int64_t Bp,
                     const __nv_bfloat16* __restrict__ packed, TrainWS ws, float* __restrict__ grad,
                     float* __restrict__ gx, int mode, int* err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    using Smem = TrainSmem<PAIR>;
    constexpr int NH = Smem::NH;
    Smem& sm = *reinterpret_cast<Smem*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, part = warp >> 2, r = 32 * quarter + lane;
    const uint32_t rank = PAIR == 2 ? cluster_rank() : 0u, peer = rank ^ 1u;
    const unsigned char* pb = reinterpret_cast<const unsigned char*>(packed);
    train_setup(sm);
    const uint32_t tbase = sm.tmem_base;
    grid_dep_launch();
    const int64_t tile = blockIdx.x / PAIR, row = tile * 128 + r;
    const int top = kMlpLayers - 1;
    if (tid == 0)
        load_w_rows(sm, pb + 2 * c_off.pT[top], mlp_NT(top), mlp_KT(top), mlp_KCT(top), NH * (int)rank, NH);
    grid_dep_wait();   // dy (training: the forward's dL/dy) and silu'(z) are the forward's
    if (part == 0) {
        float a[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) a[j] = (j < 6 && row < B) ? __ldg(dy + row * ld + j) : 0.0f;
#pragma unroll
        for (int q = 0; q < 2; ++q)
            *reinterpret_cast<uint4*>(sm.act[0] + tc::kmajor_off(r, 8 * q, 16)) =
                make_uint4(bf16x2(a[8 * q], a[8 * q + 1]), bf16x2(a[8 * q + 2], a[8 * q + 3]),
                           bf16x2(a[8 * q + 4], a[8 * q + 5]), bf16x2(a[8 * q + 6], a[8 * q + 7]));
        if (mode == 0 && rank == 0) {
            // output bias gradient: the column sums of dL/dy over the warp's rows
#pragma unroll
            for (int j = 0; j < 6; ++j) {
                float sdy = a[j];
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) sdy += __shfl_xor_sync(0xffffffffu, sdy, off);
                if (lane == 0 && sdy != 0.0f) atomicAdd(grad + c_off.b[top] + j, sdy);
            }
        }
    }
    tc::fence_async_smem();
    __syncthreads();
    uint32_t ph_w = 0, ph_m = 0;
    int failed = 0;
    const uint32_t taddr = tbase + ((uint32_t)(32 * quarter) << 16);
    int n_sig = 0;   // partner signals expected so far
    // layers 4..1: this CTA's NH input features (all of them, or one half)
    for (int l = top; l >= 1; --l) {
        const int buf = (top - l) & 1;
        // this thread's silu'(z_{l-1}) of its first 32 features into
        // registers while the tensor core works (the next 32, if any, load
        // during the first chunk's stores)
        float4 s4[8];
        {
            const int f0 = NH * (int)rank + (NH / 4) * part;
#pragma unroll
            for (int q = 0; q < 8; ++q) s4[q] = __ldg(s_quad(ws.S[l - 1], row, f0 + 4 * q));
        }
        const ImgCopy cp = mode == 0 ? img_copy<PAIR>(ws.DZim[l], tile, mlp_KT(l), rank, false) : ImgCopy{nullptr, 0u, 0u};
        failed = run_layer(sm, tbase, buf, NH, mlp_KT(l), mlp_KCT(l), PAIR == 2 ? n_sig - 1 : -1, ph_w, ph_m, cp);
        if (failed) break;
        if (tid == 0) {
            if (l - 1 >= 1)
                load_w_rows(sm, pb + 2 * c_off.pT[l - 1], mlp_NT(l - 1), mlp_KT(l - 1), mlp_KCT(l - 1),
                            NH * (int)rank, NH);
            else if (mode == 1 && rank == 0)
                load_w_rows(sm, pb + 2 * c_off.pT[0], mlp_NT(0), mlp_KT(0), mlp_KCT(0), 0, mlp_NT(0));
        }
#pragma unroll 1
        for (int cc = 0; cc < NH / 128; ++cc) {
            const int f_loc = (NH / 4) * part + 32 * cc, f_glob = NH * (int)rank + f_loc;   // 32 features
            // dL/dz_{l-1} = (dL/dz_l W_l) * silu'(z_{l-1})
            float v[32];
            tc::tmem_ld32(taddr + (uint32_t)f_loc, v);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                v[4 * q] *= s4[q].x; v[4 * q + 1] *= s4[q].y; v[4 * q + 2] *= s4[q].z; v[4 * q + 3] *= s4[q].w;
            }
            if (cc + 1 < NH / 128) {
#pragma unroll
                for (int q = 0; q < 8; ++q) s4[q] = __ldg(s_quad(ws.S[l - 1], row, f_glob + 32 + 4 * q));
            }
            uint32_t pk[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) pk[j] = bf16x2(v[2 * j], v[2 * j + 1]);
            put_act(sm.act[(buf ^ 1) % PAIR], pk, r, f_glob);
            if (mode == 0) {
                // bias gradient of layer l-1: this warp's 32 rows, column f_loc + lane
                const float cs = warp_colsum32(v, lane);
                atomicAdd(&sm.colsum[f_loc + lane], cs);
            }
        }
        signal_peer(sm, peer, n_sig, sm.act[(buf ^ 1) % PAIR]);   // (its __syncthreads also orders the colsum adds)
        ++n_sig;
        if (mode == 0) {
            for (int c = tid; c < NH; c += kTrThreads) {
                atomicAdd(grad + c_off.b[l - 1] + NH * (int)rank + c, sm.colsum[c]);
                sm.colsum[c] = 0.0f;
            }
        }
    }
    int last_peer_k = (failed || PAIR == 1) ? -1 : n_sig - 1;
    if (!failed && mode == 0) {
        // the image of dL/dz_0 (no MMA consumes it here): once the
        // partner's half has landed, thread 0 copies it out
        if (tid == 0) {
            const bool ok = PAIR == 1 || wait_peer(sm, n_sig - 1);
            if (!ok) atomicOr(err, kErrWaitTimeout);
            if (ok) {
                const ImgCopy cp = img_copy<PAIR>(ws.DZim[0], tile, 256, rank, false);
                tc::bulk_s2g(cp.img + cp.off, sm.act[(top & 1) % PAIR] + cp.off, cp.bytes);
                tc::bulk_commit();
            }
        }
        last_peer_k = -1;
    }
    if (!failed && mode == 1 && rank == 0) {
        // input gradient on rank 0: gx = dL/dz_0 W_0 (19 of the 32 columns)
        failed = run_layer(sm, tbase, (top - 0) & 1, mlp_NT(0), mlp_KT(0), mlp_KCT(0), PAIR == 2 ? n_sig - 1 : -1, ph_w,
                           ph_m);
        last_peer_k = -1;
        if (!failed && part == 0) {
            float v[32];
            tc::tmem_ld32(taddr, v);
            if (row < B) {
#pragma unroll
                for (int j = 0; j < 19; ++j) gx[row * 19 + j] = v[j];
            }
        }
    }
    train_teardown(sm, tbase, failed, ph_w, ph_m, last_peer_k, err);
}

// ---------------------------------------------------------------------------
// Weight gradients.  The batch rows are the K of the products, both operands
// read MN-major from the tile images (features along M or N):
//   l = 0..3: dW_l[o][i] += sum_r dZ_l[r][o] H_l[r][i]    (M = o, N = i)
//   l = 4:    dW_4[o][i] += sum_r H_4[r][i] dY[r][o]      (M = i, N = o:
//             the 6 outputs fit an N = 16 tile; stored transposed)
// Work items: "heavy" (l = 1..3, M tile mt, K slice ks) and "light" (mt,
// ks) covering layers 0 and 4 together (two accumulators), 8 x nks items,
// nks chosen on the host so that they about fill the SMs in one wave; a
// slice is `slice` chunks of 64 rows.  One chunk of an image (64 rows x F
// features) is 8 row groups of F * 16 bytes; an A operand takes the 2 KB of
// features [128 mt, 128 mt + 128) from each (8 bulk copies, SBO 128 and
// LBO 2 KB in shared memory), a B operand the whole chunk (one copy, SBO
// 128, LBO F * 16).  Four stages of up to 48 KB keep 192 KB of operands in
// flight per SM; the issuing thread refills the stage of chunk i - 1 with
// chunk i + 3 right after queueing chunk i's MMAs, so the tensor core never
// waits for the refill.  The epilogue transposes each warp's 32 x 32 FP32
// block through shared memory so that each red.global.add.v4 covers 4 rows
// x 128 bytes, not 32 scattered rows.
// ---------------------------------------------------------------------------
constexpr int kDwStages = 4;
constexpr uint32_t kDwA = 16384u, kDwB = 32768u;   // stage bytes of the A and B regions

struct DwSmem {
    alignas(1024) unsigned char a[kDwStages][kDwA];
    alignas(1024) unsigned char b[kDwStages][kDwB];
    alignas(8) uint64_t full[kDwStages];
    alignas(8) uint64_t mma[kDwStages];
    float red[kDwThreads];
    uint32_t tmem_base;
    int fail;
};

// One product of a work item: operand images, where a chunk of each lands
// in a stage, N and the accumulator's first TMEM column.
struct DwJob {
    const unsigned char* A;   // image, F = 256 (features [128 mt, 128 mt + 128) taken)
    const unsigned char* Bm;  // image, F = N
    uint32_t a_off, b_off;    // stage offsets: a_off in the A region (< kDwA) or, | 0x80000000, in the B region
    int N, col;
};

__device__ __forceinline__ int dw_jobs(const TrainWS& ws, int idx, int nks, DwJob (&jb)[2], int& mt, int& ks, int& l) {
    if (idx < 6 * nks) {
        l = 1 + idx / (2 * nks);
        mt = (idx / nks) & 1;
        ks = idx % nks;
        jb[0] = DwJob{reinterpret_cast<const unsigned char*>(ws.DZim[l]), reinterpret_cast<const unsigned char*>(ws.Him[l]),
                      0u, 0u, 256, 0};
        return 1;
    }
    const int j = idx - 6 * nks;
    l = 0;
    mt = j / nks;
    ks = j % nks;
    // layer 0: A in the A region, B (x, 4 KB) at 16 KB of the B region;
    // layer 4: A at 0 of the B region, B (dL/dy, 2 KB) at 20 KB
    jb[0] = DwJob{reinterpret_cast<const unsigned char*>(ws.DZim[0]), reinterpret_cast<const unsigned char*>(ws.Him[0]),
                  0u, 16384u, 32, 0};
    jb[1] = DwJob{reinterpret_cast<const unsigned char*>(ws.Him[4]), reinterpret_cast<const unsigned char*>(ws.DZim[4]),
                  0x80000000u, 20480u, 16, 32};
    return 2;
}

__device__ __forceinline__ unsigned char* dw_a_dst(DwSmem& sm, int s, uint32_t a_off) {
    return (a_off & 0x80000000u) ? sm.b[s] + (a_off & 0x7fffffffu) : sm.a[s] + a_off;
}

__global__ void __launch_bounds__(kDwThreads, 1) train_dw_kernel(int64_t Bp, int nks, int slice, TrainWS ws,
                                                                float* __restrict__ grad, int* err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    DwSmem& sm = *reinterpret_cast<DwSmem*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    DwJob jb[2];
    int mt = 0, ks = 0, l = 0;
    const int nj = dw_jobs(ws, blockIdx.x, nks, jb, mt, ks, l);
    const int64_t nkt_all = Bp >> 6;
    const int64_t kt0 = (int64_t)ks * slice;
    const int nk = (int)max((int64_t)0, min((int64_t)slice, nkt_all - kt0));
    if (tid == 0) {
        for (int s = 0; s < kDwStages; ++s) { tc::mbar_init(&sm.full[s], 1); tc::mbar_init(&sm.mma[s], 1); }
        tc::fence_mbar_init();
        sm.fail = 0;
    }
    if (tid < 32) {
        tc::tmem_alloc(&sm.tmem_base, 256);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tbase = sm.tmem_base;
    grid_dep_launch();
    grid_dep_wait();   // the tile images and loss partials are the forward's and backward's
    if (blockIdx.x == 0) {
        // the step's loss: the forward's per-warp partial sums, strided over
        // the threads, then the threads' sums in order
        float acc = 0.0f;
        for (int64_t i = tid; i < (Bp >> 5); i += kDwThreads) acc += ws.lossp[i];
        sm.red[tid] = acc;
        __syncthreads();
        if (tid == 0) {
            float tot = 0.0f;
            for (int i = 0; i < kDwThreads; ++i) tot += sm.red[i];
            ws.loss[0] = tot;
        }
    }
    auto issue = [&](int i) {
        const int s = i % kDwStages;
        const int64_t kt = kt0 + i;
        uint32_t bytes = 0;
        for (int q = 0; q < nj; ++q) bytes += 8u * 2048u + 64u * (uint32_t)jb[q].N * 2u;
        tc::mbar_expect_tx(&sm.full[s], bytes);
        for (int q = 0; q < nj; ++q) {
            const unsigned char* as = jb[q].A + (size_t)kt * (64u * 256u * 2u) + (size_t)mt * 2048u;
            unsigned char* ad = dw_a_dst(sm, s, jb[q].a_off);
            for (int g = 0; g < 8; ++g) tc::bulk_g2s(ad + g * 2048, as + (size_t)g * 4096u, 2048u, &sm.full[s]);
            const uint32_t bc = 64u * (uint32_t)jb[q].N * 2u;
            tc::bulk_g2s(sm.b[s] + jb[q].b_off, jb[q].Bm + (size_t)kt * bc, bc, &sm.full[s]);
        }
    };
    int failed = 0;
    if (tid == 0 && nk > 0) {
        for (int i = 0; i < kDwStages && i < nk; ++i) issue(i);
        for (int i = 0; i < nk; ++i) {
            const int s = i % kDwStages;
            if (!tc::mbar_wait_bounded(&sm.full[s], (uint32_t)(i / kDwStages) & 1u, kWaitLimit)) { failed = 1; break; }
            tc::tc_fence_after();
            for (int q = 0; q < nj; ++q) {
                const uint32_t idesc = tc::idesc_bf16(128, (uint32_t)jb[q].N) | tc::kMnMajorA | tc::kMnMajorB;
                const uint32_t a0 = tc::smem_u32(dw_a_dst(sm, s, jb[q].a_off)), b0 = tc::smem_u32(sm.b[s] + jb[q].b_off);
                const uint32_t b_lbo = (uint32_t)jb[q].N * 16u;
#pragma unroll
                for (int j = 0; j < 4; ++j)   // 16 rows (two K groups) per MMA
                    tc::mma_bf16(tbase + (uint32_t)jb[q].col, tc::sdesc(a0 + 4096u * j, 2048u, 128u),
                                 tc::sdesc(b0 + 2u * b_lbo * j, b_lbo, 128u), idesc, (i > 0 || j > 0) ? 1u : 0u);
            }
            tc::mma_commit(&sm.mma[s]);
            // refill the previous chunk's stage once its MMAs are done (this
            // chunk's are queued behind them)
            const int ip = i - 1;
            if (ip >= 0 && ip + kDwStages < nk) {
                const int sp = ip % kDwStages;
                if (!tc::mbar_wait_bounded(&sm.mma[sp], (uint32_t)(ip / kDwStages) & 1u, kWaitLimit)) { failed = 2; break; }
                issue(ip + kDwStages);
            }
        }
        sm.fail = failed;
    }
    __syncthreads();
    failed = sm.fail;
    if (!failed && nk > 0) {
        const int last = nk - 1;
        const bool ok = tc::mbar_wait_bounded(&sm.mma[last % kDwStages], (uint32_t)(last / kDwStages) & 1u, kWaitLimit);
        if (__syncthreads_or(!ok)) failed = 2;
    }
    if (failed) {
        if (tid == 0) {
            atomicOr(err, kErrWaitTimeout);
            // copies and MMAs in flight land before the CTA leaves
            for (int s = 0; s < kDwStages; ++s) {
                tc::mbar_wait_bounded(&sm.full[s], 0u, 1u << 16);
                tc::mbar_wait_bounded(&sm.mma[s], 0u, 1u << 16);
            }
        }
    } else if (nk > 0) {
        tc::tc_fence_after();
        const int m0 = 128 * mt + 32 * warp;   // first M row of the warp (TMEM lane quarter)
        const uint32_t taddr = tbase + ((uint32_t)(32 * warp) << 16);
        // per-warp 32 x 32 FP32 transpose block (rows 36 floats apart) in the
        // stage buffers, free once the last MMA has completed
        float* sc = reinterpret_cast<float*>(sm.a[0]) + warp * (32 * 36);
        if (l > 0) {
            float4* dst = reinterpret_cast<float4*>(grad + c_off.w[l]);
#pragma unroll 1
            for (int cc = 0; cc < 8; ++cc) {
                float v[32];
                tc::tmem_ld32(taddr + 32u * (uint32_t)cc, v);
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    *reinterpret_cast<float4*>(sc + lane * 36 + 4 * q) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                __syncwarp();
#pragma unroll
                for (int rr = 0; rr < 8; ++rr) {
                    const int r = 4 * rr + (lane >> 3), c4 = lane & 7;   // row r, columns 4 c4 .. 4 c4 + 3
                    const float4 x = *reinterpret_cast<const float4*>(sc + r * 36 + 4 * c4);
                    atomicAdd(dst + (int64_t)(m0 + r) * 64 + 8 * cc + c4, x);
                }
                __syncwarp();
            }
        } else {
            // layer 0: dW_0[o][i], o = M row, i < 19 (rows of 19 floats)
            float v[32];
            tc::tmem_ld32(taddr, v);
#pragma unroll
            for (int q = 0; q < 8; ++q)
                *reinterpret_cast<float4*>(sc + lane * 36 + 4 * q) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            __syncwarp();
            if (lane < 19)
                for (int r = 0; r < 32; ++r) atomicAdd(grad + c_off.w[0] + (int64_t)(m0 + r) * 19 + lane, sc[r * 36 + lane]);
            // layer 4: dW_4[o][i], i = M row (consecutive over the warp), o < 6
            float u[16];
            tc::tmem_ld16(taddr + 32u, u);
#pragma unroll
            for (int o = 0; o < 6; ++o) atomicAdd(grad + c_off.w[4] + o * 256 + m0 + lane, u[o]);
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (tid < 32) tc::tmem_dealloc(tbase, 256);
}

// Adam (Kingma & Ba): bias-corrected moments, in place (ic1, ic2: the
// reciprocals of the bias corrections 1 - b1^t, 1 - b2^t); every updated
// weight is also written, rounded to BF16, into both packed layouts (the
// padding of the packed buffers is zero from their creation).  The layer of
// element e and its packed offsets come from shifts and compares: the K
// chunk of the forward layout is 32 (layer 0) or 64 columns, of the
// transposed one 16 (layer 4) or 64.
__global__ void adam_pack_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                                 float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float ic1,
                                 float ic2, __nv_bfloat16* __restrict__ packed) {
    grid_dep_wait();   // the gradient is the weight-gradient kernel's
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const float gg = g[e];
        const float mm = b1 * m[e] + (1.0f - b1) * gg;
        const float vv = b2 * v[e] + (1.0f - b2) * gg * gg;
        m[e] = mm;
        v[e] = vv;
        const float pv = p[e] - lr * (mm * ic1) / (sqrtf(vv * ic2) + eps);
        p[e] = pv;
        const int l = (int)(e >= c_off.w[1]) + (int)(e >= c_off.w[2]) + (int)(e >= c_off.w[3]) + (int)(e >= c_off.w[4]);
        const int64_t q = e - c_off.w[l];
        if (q < c_off.b[l] - c_off.w[l]) {   // a weight W_l[o][i], not a bias
            const int o = l == 0 ? (int)(q / 19) : (int)(q >> 8);
            const int i = (int)(q - (int64_t)o * (l == 0 ? 19 : 256));
            const __nv_bfloat16 bv = __float2bfloat16_rn(pv);
            // forward layout: N (= out, padded) rows x K (= in, padded) in chunks of KC columns
            const int kcs = l == 0 ? 5 : 6, N = l == 4 ? 16 : 256;
            const int c = i >> kcs, k = i & ((1 << kcs) - 1);
            const uint32_t fo = (uint32_t)c * (uint32_t)(N << kcs) * 2u + tc::kmajor_off((uint32_t)o, (uint32_t)k, 1u << kcs);
            packed[c_off.p[l] + fo / 2] = bv;
            // transposed layout: NT (= in, padded) rows x KT (= out, padded) in chunks of KCT columns
            const int kts = l == 4 ? 4 : 6, NT = l == 0 ? 32 : 256;
            const int ct = o >> kts, kt = o & ((1 << kts) - 1);
            const uint32_t to = (uint32_t)ct * (uint32_t)(NT << kts) * 2u + tc::kmajor_off((uint32_t)i, (uint32_t)kt, 1u << kts);
            packed[c_off.pT[l] + to / 2] = bv;
        }
    }
}

static cudaError_t train_attrs() {
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    const void* f[4] = {(const void*)train_fwd_kernel<1>, (const void*)train_bwd_kernel<1>,
                        (const void*)train_fwd_kernel<2>, (const void*)train_bwd_kernel<2>};
    const int sz[4] = {(int)sizeof(TrainSmem<1>), (int)sizeof(TrainSmem<1>), (int)sizeof(TrainSmem<2>),
                       (int)sizeof(TrainSmem<2>)};
    for (int i = 0; i < 4 && e == cudaSuccess; ++i)
        e = cudaFuncSetAttribute(f[i], cudaFuncAttributeMaxDynamicSharedMemorySize, sz[i]);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(train_dw_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(DwSmem));
    if (e == cudaSuccess) done = true;
    return e;
}

// Pairs (two-CTA clusters) when the batch's tiles leave at least half the
// SMs idle, one CTA per tile otherwise.
static int train_pair(int64_t Bp) {
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 1;
    return 2 * (Bp / 128) <= n_sm ? 2 : 1;
}

// Launch with cudaLaunchKernelEx: clusters of `cluster` CTAs (1: none);
// `pdl`: programmatic stream serialisation (the kernel may start while its
// predecessor still runs and waits for it in grid_dep_wait).
template <typename... Args>
static cudaError_t launch_ex(void (*kern)(Args...), unsigned grid, unsigned block, size_t smem, int cluster, bool pdl,
                             cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[2];
    unsigned na = 0;
    if (cluster > 1) {
        at[na].id = cudaLaunchAttributeClusterDimension;
        at[na].val.clusterDim.x = (unsigned)cluster;
        at[na].val.clusterDim.y = 1;
        at[na].val.clusterDim.z = 1;
        ++na;
    }
    if (pdl) {
        at[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[na].val.programmaticStreamSerializationAllowed = 1;
        ++na;
    }
    cfg.attrs = at;
    cfg.numAttrs = na;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

static cudaError_t launch_fwd(int pair, unsigned tiles, cudaStream_t st, const float* x, const float* tgt,
                              const int32_t* idx, int64_t n_src, int64_t B, int64_t Bp, const __nv_bfloat16* pk,
                              const float* params, const TrainWS& ws, float* grad, int mode, int* err) {
    if (pair == 2)
        return launch_ex(train_fwd_kernel<2>, 2 * tiles, kTrThreads, sizeof(TrainSmem<2>), 2, false, st, x, tgt, idx,
                         n_src, B, Bp, pk, params, ws, grad, mode, err);
    return launch_ex(train_fwd_kernel<1>, tiles, kTrThreads, sizeof(TrainSmem<1>), 1, false, st, x, tgt, idx, n_src, B,
                     Bp, pk, params, ws, grad, mode, err);
}

static cudaError_t launch_bwd(int pair, unsigned tiles, cudaStream_t st, const float* dy, int ld, int64_t B, int64_t Bp,
                              const __nv_bfloat16* pk, const TrainWS& ws, float* grad, float* gx, int mode, int* err) {
    if (pair == 2)
        return launch_ex(train_bwd_kernel<2>, 2 * tiles, kTrThreads, sizeof(TrainSmem<2>), 2, true, st, dy, ld, B, Bp,
                         pk, ws, grad, gx, mode, err);
    return launch_ex(train_bwd_kernel<1>, tiles, kTrThreads, sizeof(TrainSmem<1>), 1, true, st, dy, ld, B, Bp, pk, ws,
                     grad, gx, mode, err);
}

// One optimisation step; grad receives dL/dparams; Adam applied when lr > 0.
// idx (may be NULL): the batch's rows of x and tgt (n_src rows each).
cudaError_t mlp_train(const float* x, const float* tgt, const int32_t* idx, int64_t n_src, int64_t B, float* params,
                      float* grad, float* adam_m, float* adam_v, int64_t step, float lr, void* work, void* packed,
                      int* err, cudaStream_t st) {
    cudaError_t e = train_attrs();
    if (e != cudaSuccess) return e;
    const int64_t Bp = train_bp(B);
    const TrainWS ws = train_carve(work, B);
    const unsigned tiles = (unsigned)(Bp / 128);
    const int pair = train_pair(Bp);
    const __nv_bfloat16* pk = (const __nv_bfloat16*)packed;
    if ((e = launch_fwd(pair, tiles, st, x, tgt, idx, n_src, B, Bp, pk, params, ws, grad, 0, err)) != cudaSuccess)
        return e;
    if ((e = launch_bwd(pair, tiles, st, ws.dY, 8, B, Bp, pk, ws, grad, nullptr, 0, err)) != cudaSuccess) return e;
    // K slices: 8 work items per slice (6 heavy, 2 light), about one per SM
    int n_sm = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        n_sm = 8;
    const int64_t chunks = Bp >> 6;
    const int want = std::max(1, n_sm / 8);
    const int slice = (int)((chunks + want - 1) / want);
    const int nks = (int)((chunks + slice - 1) / slice);
    if ((e = launch_ex(train_dw_kernel, (unsigned)(8 * nks), kDwThreads, sizeof(DwSmem), 1, true, st, Bp, nks, slice,
                       ws, grad, err)) != cudaSuccess)
        return e;
    if (lr > 0.0f) {
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
        e = launch_ex(adam_pack_kernel, (unsigned)((kMlpParams + 255) / 256), 256u, 0, 1, true, st, params,
                      (const float*)grad, adam_m, adam_v, (int64_t)kMlpParams, lr, b1, b2, 1e-8f, 1.0f / c1, 1.0f / c2,
                      (__nv_bfloat16*)packed);
    }
    return e;
}

// Input gradient gx[B][19] = (dy/dx)^T wy (wy [B][6]): the forward's
// silu'(z), then the backward chain down to the inputs.
cudaError_t mlp_input_grad(const float* x, const float* wy, int64_t B, const float* params, const void* packed,
                           float* gx, void* work, int* err, cudaStream_t st) {
    cudaError_t e = train_attrs();
    if (e != cudaSuccess) return e;
    const int64_t Bp = train_bp(B);
    const TrainWS ws = train_carve(work, B);
    const unsigned tiles = (unsigned)(Bp / 128);
    const int pair = train_pair(Bp);
    const __nv_bfloat16* pk = (const __nv_bfloat16*)packed;
    if ((e = launch_fwd(pair, tiles, st, x, nullptr, nullptr, B, B, Bp, pk, params, ws, nullptr, 1, err)) != cudaSuccess)
        return e;
    if ((e = launch_bwd(pair, tiles, st, wy, 6, B, Bp, pk, ws, nullptr, gx, 1, err)) != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace srp
