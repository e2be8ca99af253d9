// mlp.cu -- the neural proxy P(omega, theta | psi) of Sec. 3.3 on the
// Blackwell tensor cores: 19 inputs (sun direction + 16 design parameters)
// -> 4 hidden layers of 256 (SiLU) -> 6 outputs (force, torque), BF16
// operands, FP32 accumulation in TMEM, FP32 master weights.
//
// Parameter vector (FP32, the layout the API exchanges):
//   for l = 0..4: W_l [out_l][in_l] row-major, then b_l [out_l]
//   sizes (19,256,256,256,256,6): 204,038 floats.
// Device copies per layer: BF16 weights padded to (N_l, K_l) =
//   (256,32), (256,256) x3, (16,256) and stored in the K-major no-swizzle
//   core-matrix layout (tc_common.cuh), so a layer is one contiguous block
//   that a 1-D bulk copy moves into shared memory.
//
// Forward kernel (one CTA of 512 threads per 128 batch rows):
//   X (FP32) -> BF16 tile in smem; per layer: bulk-copy W_l into smem,
//   one thread issues K_l/16 tcgen05.mma (M=128, N=N_l, K=16) into a
//   256-column TMEM accumulator, commit -> mbarrier; the four warps read
//   their 32 TMEM lanes (= rows) with tcgen05.ld, add the bias, apply SiLU,
//   round to BF16 and write the next layer's A tile.  Every wait is
//   bounded; on a timeout the kernel records an error, waits (bounded) for
//   its in-flight operations, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "mlp_common.cuh"
#include "srp_internal.h"
#include "tc_common.cuh"

namespace srp {

// FP32 master weights -> BF16 packed per layer (zero padding), forward and
// transposed layouts.
__global__ void mlp_pack_kernel(const float* __restrict__ params, __nv_bfloat16* __restrict__ packed) {
    const MlpLayout L = mlp_layout();
    const int64_t tot = L.packed_elems;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        int l = 0;
        while (l + 1 < kMlpLayers && e >= L.p_off[l + 1]) ++l;
        const int64_t loc = e - L.p_off[l];
        const int K = mlp_K(l);
        const int n = (int)(loc / K), k = (int)(loc % K);
        const float w = (n < mlp_out(l) && k < mlp_in(l)) ? params[L.w_off[l] + (int64_t)n * mlp_in(l) + k] : 0.0f;
        packed[L.p_off[l] + mlp_packed_off(l, n, k) / 2] = __float2bfloat16_rn(w);
    }
    const int64_t totT = mlp_packed_all_elems() - tot;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < totT; e += (int64_t)gridDim.x * blockDim.x) {
        int l = 0;
        while (l + 1 < kMlpLayers && tot + e >= mlp_pT_off(l + 1)) ++l;
        const int64_t loc = tot + e - mlp_pT_off(l);
        const int K = mlp_KT(l);
        const int n = (int)(loc / K), k = (int)(loc % K);   // n: input feature, k: output feature
        const float w = (k < mlp_out(l) && n < mlp_in(l)) ? params[L.w_off[l] + (int64_t)k * mlp_in(l) + n] : 0.0f;
        packed[mlp_pT_off(l) + mlp_packedT_off(l, n, k) / 2] = __float2bfloat16_rn(w);
    }
}

// Forward kernel: persistent, one CTA per SM, 128-row tiles.
//   warps 0-15  epilogue: warp w reads TMEM lane quarter w % 4 (rows) and,
//               in each 64-feature chunk c, the 16 features
//               64 c + 16 (w / 4) ...; all 16 warps finish chunk 0, then 1,
//               2, 3; warps 0-3 also load each tile's inputs and write its
//               outputs;
//   warp 16     producer: bulk copies of the weights and tcgen05.mma issue.
// Layer l + 1's MMAs over K chunk c need only chunk c of layer l's
// activations, so each chunk is signalled on its own mbarrier as soon as it
// is written and the tensor core runs layer l + 1 while the later chunks of
// layer l's epilogue are still in flight; consecutive layers alternate
// between two 256-column TMEM accumulators.  Layers 0 and 4 (24 KB) stay
// resident; the 128 KB hidden layers 1-3 stream through one buffer in four
// 32 KB chunks, each copy issued as soon as the previous layer's MMAs have
// released it.
constexpr int kEpiWarps = 16;
constexpr int kFwdThreads = 32 * (kEpiWarps + 1);

struct MlpFwdSmem {
    alignas(1024) unsigned char act[128 * 256 * 2];   // A: the layer's input activations (64 KB)
    alignas(1024) unsigned char w[256 * 256 * 2];     // B: streamed hidden layer, 4 chunks of 32 KB
    alignas(1024) unsigned char w0[256 * 32 * 2];     // B: layer 0 (resident)
    alignas(1024) unsigned char w4[16 * 256 * 2];     // B: layer 4 (resident)
    float bias[4 * 256 + 16];                         // biases: halved for layers 0-3, as is for 4
    alignas(8) uint64_t bar_w[4];     // streamed weight chunk c landed
    alignas(8) uint64_t bar_res;      // resident weights landed
    alignas(8) uint64_t bar_mma;      // a layer's MMAs completed
    alignas(8) uint64_t bar_act[4];   // activation chunk c written (16 warps arrive)
    alignas(8) uint64_t bar_in;       // a tile's inputs written and every epilogue warp past the
                                      // previous tile's last layer (16 warps arrive)
    uint32_t tmem_base;
};

// silu(z) = z sigmoid(z) = h + h tanh(h), h = z/2: one hardware tanh
// (tanh.approx.f32, ~2^-11 relative) per activation instead of an exp and a
// reciprocal; the result is rounded to BF16 (2^-9) right after.  The error
// is about 2^-11 |h| in absolute terms: below the BF16 rounding where
// silu(z) is O(z), but for z below about -4 (silu(z) -> 0 while h tanh(h)
// cancels h) it is large relative to the value itself.  The inference
// kernel takes it for speed; the training kernels (train.cu) evaluate
// z / (1 + exp(-z)) with the accurate expf.
__device__ __forceinline__ float tanh_approx(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// (r0, r1) = (a0, a1) * (b0, b1) + (c0, c1) by one packed FP32 FMA
// (fma.rn.f32x2: the rounding of two fmaf, one instruction).
__device__ __forceinline__ void fma_x2(float a0, float a1, float b0, float b1, float c0, float c1, float& r0,
                                       float& r1) {
    asm("{\n .reg .b64 a, b, c, r;\n"
        " mov.b64 a, {%2, %3};\n mov.b64 b, {%4, %5};\n mov.b64 c, {%6, %7};\n"
        " fma.rn.f32x2 r, a, b, c;\n mov.b64 {%0, %1}, r;\n}"
        : "=f"(r0), "=f"(r1)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1), "f"(c0), "f"(c1));
}

// Two floats -> BF16 (round to nearest even), a in the low half.
__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    const __nv_bfloat162_raw h = __floats2bfloat162_rn(a, b);
    return (uint32_t)h.x | ((uint32_t)h.y << 16);
}

// Producer: request the four chunks of streamed layer l (1..3).
__device__ __forceinline__ void load_stream(MlpFwdSmem& sm, const unsigned char* packed_b, const MlpLayout& L, int l) {
    const unsigned char* src = packed_b + 2 * L.p_off[l];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        tc::mbar_expect_tx(&sm.bar_w[c], 32768u);
        tc::bulk_g2s(sm.w + 32768u * c, src + 32768u * c, 32768u, &sm.bar_w[c]);
    }
}

// Warps 0-3: row tid of a tile's inputs (19 features; zeros past B) ...
__device__ __forceinline__ void load_inputs(const float* __restrict__ x, int64_t B, int64_t row0, int tid,
                                            float (&v)[19]) {
    const int64_t row = row0 + tid;
#pragma unroll
    for (int j = 0; j < 19; ++j) v[j] = row < B ? __ldg(x + row * 19 + j) : 0.0f;
}
// ... into the A buffer in layer 0's layout (K = 32, zero padded), then
// arrive on bar_in.
__device__ __forceinline__ void store_inputs(MlpFwdSmem& sm, const float (&v)[19], int tid, int lane) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint32_t u[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int k = 8 * q + 2 * j;
            u[j] = pack_bf16x2(k < 19 ? v[k] : 0.0f, k + 1 < 19 ? v[k + 1] : 0.0f);
        }
        *reinterpret_cast<uint4*>(sm.act + tc::kmajor_off(tid, 8 * q, 32)) = make_uint4(u[0], u[1], u[2], u[3]);
    }
    tc::fence_async_smem();
    __syncwarp();
    if (lane == 0) tc::mbar_arrive(&sm.bar_in);
}

// Epilogue of one 16-feature piece of chunk c for row r: accumulator words
// u (TMEM), hb = half the bias (smem).  h = z/2 = fma(0.5, acc, b/2) equals
// 0.5 (acc + b) exactly (scaling by 2 commutes with rounding); silu =
// h + h tanh(h), two activations per packed FMA; BF16 pairs by one cvt
// each; into the A buffer; then signal
// chunk c.  Only the last chunk's signal carries the tcgen05 fence: the
// next layer writes the other accumulator, and this one is rewritten only
// after chunk 3 has been signalled.
__device__ __forceinline__ void epi_chunk(MlpFwdSmem& sm, const uint32_t (&u)[16], const float* hb, int c, int part,
                                          int r, int lane) {
    const int c0 = 64 * c + 16 * part;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        uint32_t p[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int k = 8 * q + 2 * j;
            const float2 b2 = *reinterpret_cast<const float2*>(hb + c0 + k);
            float h0, h1, s0, s1;
            fma_x2(0.5f, 0.5f, __uint_as_float(u[k]), __uint_as_float(u[k + 1]), b2.x, b2.y, h0, h1);
            fma_x2(h0, h1, tanh_approx(h0), tanh_approx(h1), h0, h1, s0, s1);
            asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(p[j]) : "f"(s1), "f"(s0));   // s0 in the low half
        }
        *reinterpret_cast<uint4*>(sm.act + tc::kmajor_off(r, c0 + 8 * q, 256)) = make_uint4(p[0], p[1], p[2], p[3]);
    }
    if (c == 3) tc::tc_fence_before();
    tc::fence_async_smem();
    __syncwarp();
    if (lane == 0) tc::mbar_arrive(&sm.bar_act[c]);
}

__global__ void __launch_bounds__(kFwdThreads, 1) mlp_fwd_kernel(const float* __restrict__ x, int64_t B,
                                                        const __nv_bfloat16* __restrict__ packed,
                                                        const float* __restrict__ params, float* __restrict__ y,
                                                        int* err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    MlpFwdSmem& sm = *reinterpret_cast<MlpFwdSmem*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const MlpLayout L = mlp_layout();
    const int64_t tiles = (B + 127) / 128;
    for (int i = tid; i < 4 * 256 + 16; i += kFwdThreads) {
        const int l = i >> 8, n = i & 255;
        sm.bias[i] = l < 4 ? 0.5f * params[L.b_off[l] + n] : (n < 6 ? params[L.b_off[4] + n] : 0.0f);
    }
    if (tid == 0) {
        for (int c = 0; c < 4; ++c) { tc::mbar_init(&sm.bar_w[c], 1); tc::mbar_init(&sm.bar_act[c], kEpiWarps); }
        tc::mbar_init(&sm.bar_res, 1);
        tc::mbar_init(&sm.bar_mma, 1);
        tc::mbar_init(&sm.bar_in, kEpiWarps);
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(&sm.tmem_base, 512);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tbase = sm.tmem_base;
    int failed = 0;
    if (warp == kEpiWarps) {
        // ---------------- producer ----------------
        if (lane == 0) {
            const unsigned char* pb = reinterpret_cast<const unsigned char*>(packed);
            tc::mbar_expect_tx(&sm.bar_res, 16384u + 8192u);
            tc::bulk_g2s(sm.w0, pb + 2 * L.p_off[0], 16384u, &sm.bar_res);
            tc::bulk_g2s(sm.w4, pb + 2 * L.p_off[4], 8192u, &sm.bar_res);
            bool pending_w = blockIdx.x < tiles;   // a streamed layer requested and not yet waited
            if (pending_w) load_stream(sm, pb, L, 1);
            bool pending_mma = false;   // committed, completion not yet waited
            bool issued = false;        // MMAs issued since the last commit
            uint32_t ph_w = 0, ph_m = 0, ph_in = 0, ph_a[4] = {0, 0, 0, 0}, g = 0;
            if (!tc::mbar_wait_bounded(&sm.bar_res, 0, kWaitLimit)) failed = 1;
            for (int64_t t = blockIdx.x; t < tiles && !failed; t += gridDim.x) {
                for (int l = 0; l < kMlpLayers && !failed; ++l) {
                    const uint32_t acc = tbase + ((g & 1u) ? 256u : 0u);
                    const int N = mlp_N(l);
                    const uint32_t idesc = tc::idesc_bf16(128, N);
                    const bool streamed = l >= 1 && l <= 3;
                    const int nch = l == 0 ? 1 : 4;
                    for (int c = 0; c < nch && !failed; ++c) {
                        if (l == 0) {
                            if (!tc::mbar_wait_bounded(&sm.bar_in, ph_in, kWaitLimit)) { failed = 1; break; }
                            ph_in ^= 1u;
                        } else {
                            if (!tc::mbar_wait_bounded(&sm.bar_act[c], ph_a[c], kWaitLimit)) { failed = 1; break; }
                            ph_a[c] ^= 1u;
                        }
                        if (streamed && !tc::mbar_wait_bounded(&sm.bar_w[c], ph_w, kWaitLimit)) { failed = 1; break; }
                        tc::tc_fence_after();
                        const int KC = mlp_KC(l);
                        const uint32_t sboA = l == 0 ? 512u : 4096u, sboB = (uint32_t)(KC / 8) * 128u;
                        const uint32_t bch = tc::smem_u32(l == 0 ? sm.w0 : (streamed ? sm.w : sm.w4)) +
                                             (uint32_t)c * (uint32_t)(N * KC * 2);
                        for (int j = 0; j < KC / 16; ++j) {
                            const int kk = c * (KC / 16) + j;
                            const uint64_t ad = tc::sdesc(tc::smem_u32(sm.act) + 256u * kk, 128u, sboA);
                            const uint64_t bd = tc::sdesc(bch + 256u * j, 128u, sboB);
                            tc::mma_bf16(acc, ad, bd, idesc, kk > 0 ? 1u : 0u);
                        }
                        issued = true;
                    }
                    if (failed) break;
                    if (streamed) { ph_w ^= 1u; pending_w = false; }
                    tc::mma_commit(&sm.bar_mma);
                    pending_mma = true;
                    issued = false;
                    ++g;
                    // the layer's accumulator is done once the epilogue sees
                    // it; the streamed buffer is free for the next layer
                    if (!tc::mbar_wait_bounded(&sm.bar_mma, ph_m, kWaitLimit)) { failed = 1; break; }
                    ph_m ^= 1u;
                    pending_mma = false;
                    if (l == 1 || l == 2) { load_stream(sm, pb, L, l + 1); pending_w = true; }
                    if (l == 3 && t + gridDim.x < tiles) { load_stream(sm, pb, L, 1); pending_w = true; }
                }
            }
            if (failed) {
                atomicOr(err, kErrWaitTimeout);
                // let copies and MMAs in flight land before the CTA leaves
                if (pending_w)
                    for (int c = 0; c < 4; ++c) tc::mbar_wait_bounded(&sm.bar_w[c], ph_w, kWaitLimit);
                if (issued && !pending_mma) { tc::mma_commit(&sm.bar_mma); pending_mma = true; }
                if (pending_mma) tc::mbar_wait_bounded(&sm.bar_mma, ph_m, kWaitLimit);
            }
        }
    } else {
        // ---------------- epilogue warps ----------------
        const int quarter = warp & 3, part = warp >> 2;
        const int r = 32 * quarter + lane;
        uint32_t ph_m = 0, g = 0;
        float xin[19];   // warps 0-3: the next tile's inputs, loaded a tile ahead
        if (part == 0) {
            load_inputs(x, B, (int64_t)blockIdx.x * 128, tid, xin);
            store_inputs(sm, xin, tid, lane);
            load_inputs(x, B, ((int64_t)blockIdx.x + gridDim.x) * 128, tid, xin);
        } else if (lane == 0) {
            tc::mbar_arrive(&sm.bar_in);
        }
        for (int64_t t = blockIdx.x; t < tiles && !failed; t += gridDim.x) {
            const int64_t row0 = t * 128;
            for (int l = 0; l < kMlpLayers; ++l) {
                if (!tc::mbar_wait_bounded(&sm.bar_mma, ph_m, kWaitLimit)) { failed = 1; break; }
                ph_m ^= 1u;
                tc::tc_fence_after();
                const uint32_t taddr = tbase + ((g & 1u) ? 256u : 0u) + ((uint32_t)(32 * quarter) << 16);
                ++g;
                if (l < kMlpLayers - 1) {
                    const float* hb = sm.bias + 256 * l;
                    // chunk c + 1's TMEM load is in flight while chunk c is computed
                    uint32_t ra[16], rb[16];
                    tc::tmem_ld16_nowait(taddr + (uint32_t)(16 * part), ra);
                    tc::tmem_wait_ld16(ra);
                    tc::tmem_ld16_nowait(taddr + (uint32_t)(64 + 16 * part), rb);
                    epi_chunk(sm, ra, hb, 0, part, r, lane);
                    tc::tmem_wait_ld16(rb);
                    tc::tmem_ld16_nowait(taddr + (uint32_t)(128 + 16 * part), ra);
                    epi_chunk(sm, rb, hb, 1, part, r, lane);
                    tc::tmem_wait_ld16(ra);
                    tc::tmem_ld16_nowait(taddr + (uint32_t)(192 + 16 * part), rb);
                    epi_chunk(sm, ra, hb, 2, part, r, lane);
                    tc::tmem_wait_ld16(rb);
                    epi_chunk(sm, rb, hb, 3, part, r, lane);
                } else if (part == 0) {
                    const float* bias = sm.bias + 4 * 256;
                    float v[16];
                    tc::tmem_ld16(taddr, v);
                    const int64_t row = row0 + r;
                    if (row < B) {
#pragma unroll
                        for (int j = 0; j < 6; ++j) y[row * 6 + j] = v[j] + bias[j];
                    }
                    tc::tc_fence_before();
                    if (t + gridDim.x < tiles) {
                        store_inputs(sm, xin, tid, lane);
                        load_inputs(x, B, (t + 2 * (int64_t)gridDim.x) * 128, tid, xin);
                    }
                } else if (lane == 0 && t + gridDim.x < tiles) {
                    tc::mbar_arrive(&sm.bar_in);
                }
            }
        }
        if (failed && lane == 0) atomicOr(err, kErrWaitTimeout);
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (warp == 0) tc::tmem_dealloc(tbase, 512);
}

cudaError_t mlp_pack(const float* params, void* packed, cudaStream_t st) {
    mlp_pack_kernel<<<256, 256, 0, st>>>(params, (__nv_bfloat16*)packed);
    return cudaGetLastError();
}

cudaError_t mlp_forward(const float* x, int64_t B, const void* packed, const float* params, float* y, int* err,
                        cudaStream_t st) {
    if (B <= 0) return cudaSuccess;
    const size_t sm = sizeof(MlpFwdSmem);
    cudaError_t e = cudaFuncSetAttribute(mlp_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int64_t tiles = (B + 127) / 128;
    const unsigned grid = (unsigned)std::min<int64_t>(tiles, (int64_t)nsm);
    mlp_fwd_kernel<<<grid, kFwdThreads, sm, st>>>(x, B, (const __nv_bfloat16*)packed, params, y, err);
    return cudaGetLastError();
}


// Training and the input gradient run on the fused kernels of train.cu.
size_t train_bytes(int64_t B);
float* train_loss_ptr(void* work, int64_t B);
cudaError_t mlp_train(const float* x, const float* tgt, const int32_t* idx, int64_t n_src, int64_t B, float* params,
                      float* grad, float* adam_m, float* adam_v, int64_t step, float lr, void* work, void* packed,
                      int* err, cudaStream_t st);
cudaError_t mlp_input_grad(const float* x, const float* wy, int64_t B, const float* params, const void* packed,
                           float* gx, void* work, int* err, cudaStream_t st);

int64_t mlp_param_count() { return kMlpParams; }
int64_t mlp_packed_bytes() { return mlp_packed_all_elems() * 2; }

void set_last_error(const std::string& msg);
cudaStream_t ctx_stream(srp_ctx* c);
int ctx_device(srp_ctx* c);
int* ctx_err(srp_ctx* c);
int ctx_n_sm(srp_ctx* c);
const float* mlp_params_ptr(const srp_mlp* m);

}  // namespace srp

// ---------------------------------------------------------------------------
// C ABI of the proxy network
// ---------------------------------------------------------------------------
struct srp_mlp {
    int device = 0;
    float* params = nullptr;   // FP32 master weights [P]
    void* packed = nullptr;    // BF16 per-layer packed weights
    float* adam_m = nullptr;   // Adam first moments [P]
    float* adam_v = nullptr;   // Adam second moments [P]
    float* grad = nullptr;     // gradient [P]
    int64_t step = 0;          // Adam step count
    void* work = nullptr;      // training scratch
    size_t work_bytes = 0;
};

namespace {
using namespace srp;
int mfail(int code, const std::string& m) {
    set_last_error(m);
    return code;
}
#define MCU(call, where)                                                                  \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) return mfail(SRP_ECUDA, std::string(where) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// He-uniform initial weights from a splitmix64 stream (deterministic in seed).
void init_params_host(uint64_t seed, std::vector<float>& p) {
    const MlpLayout L = mlp_layout();
    uint64_t st = seed * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
    auto next = [&]() {
        uint64_t z = (st += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    p.assign(kMlpParams, 0.0f);
    for (int l = 0; l < kMlpLayers; ++l) {
        const double lim = std::sqrt(6.0 / mlp_in(l));
        for (int64_t q = 0; q < (int64_t)mlp_in(l) * mlp_out(l); ++q) {
            const double u = (double)(next() >> 11) * (1.0 / 9007199254740992.0);
            p[L.w_off[l] + q] = (float)((2.0 * u - 1.0) * lim);
        }
    }
}
}  // namespace

const float* srp::mlp_params_ptr(const srp_mlp* m) { return m->params; }

extern "C" int srp_mlp_param_count(int64_t* out) {
    if (!out) return mfail(SRP_EINVAL, "srp_mlp_param_count: NULL out");
    *out = kMlpParams;
    return SRP_OK;
}

extern "C" int srp_mlp_set_params(srp_ctx* c, srp_mlp* m, const float* params) {
    if (!c || !m || !params) return mfail(SRP_EINVAL, "srp_mlp_set_params: NULL argument");
    for (int64_t q = 0; q < kMlpParams; ++q)
        if (!std::isfinite(params[q])) return mfail(SRP_EINVAL, "srp_mlp_set_params: non-finite parameter");
    MCU(cudaSetDevice(m->device), "cudaSetDevice");
    cudaStream_t st = ctx_stream(c);
    MCU(cudaMemcpyAsync(m->params, params, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, st), "H2D params");
    MCU(mlp_pack(m->params, m->packed, st), "pack kernel");
    MCU(cudaMemsetAsync(m->adam_m, 0, sizeof(float) * kMlpParams, st), "memset");
    MCU(cudaMemsetAsync(m->adam_v, 0, sizeof(float) * kMlpParams, st), "memset");
    m->step = 0;
    MCU(cudaStreamSynchronize(st), "sync");
    return SRP_OK;
}

extern "C" int srp_mlp_create(srp_ctx* c, const float* params, uint64_t seed, srp_mlp** out) {
    if (!c || !out) return mfail(SRP_EINVAL, "srp_mlp_create: NULL ctx/out");
    *out = nullptr;
    MCU(cudaSetDevice(ctx_device(c)), "cudaSetDevice");
    srp_mlp* m = new (std::nothrow) srp_mlp();
    if (!m) return mfail(SRP_ENOMEM, "srp_mlp_create: out of host memory");
    m->device = ctx_device(c);
    cudaError_t e = cudaMalloc((void**)&m->params, sizeof(float) * kMlpParams);
    if (e == cudaSuccess) e = cudaMalloc(&m->packed, (size_t)mlp_packed_bytes());
    if (e == cudaSuccess) e = cudaMalloc((void**)&m->adam_m, sizeof(float) * kMlpParams);
    if (e == cudaSuccess) e = cudaMalloc((void**)&m->adam_v, sizeof(float) * kMlpParams);
    if (e == cudaSuccess) e = cudaMalloc((void**)&m->grad, sizeof(float) * kMlpParams);
    if (e == cudaSuccess) e = cudaMemset(m->packed, 0, (size_t)mlp_packed_bytes());
    if (e != cudaSuccess) {
        cudaFree(m->params); cudaFree(m->packed); cudaFree(m->adam_m); cudaFree(m->adam_v); cudaFree(m->grad);
        delete m;
        return mfail(SRP_ENOMEM, "srp_mlp_create: device allocation failed");
    }
    std::vector<float> init;
    if (!params) {
        init_params_host(seed, init);
        params = init.data();
    }
    int rc = srp_mlp_set_params(c, m, params);
    if (rc != SRP_OK) {
        cudaFree(m->params); cudaFree(m->packed); cudaFree(m->adam_m); cudaFree(m->adam_v); cudaFree(m->grad);
        delete m;
        return rc;
    }
    *out = m;
    return SRP_OK;
}

extern "C" int srp_mlp_destroy(srp_mlp* m) {
    if (!m) return SRP_OK;
    cudaSetDevice(m->device);
    cudaDeviceSynchronize();
    cudaFree(m->params); cudaFree(m->packed); cudaFree(m->adam_m); cudaFree(m->adam_v); cudaFree(m->grad);
    if (m->work) cudaFree(m->work);
    delete m;
    return SRP_OK;
}

extern "C" int srp_mlp_get_params(srp_ctx* c, const srp_mlp* m, float* out) {
    if (!c || !m || !out) return mfail(SRP_EINVAL, "srp_mlp_get_params: NULL argument");
    MCU(cudaSetDevice(m->device), "cudaSetDevice");
    MCU(cudaMemcpyAsync(out, m->params, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost, ctx_stream(c)), "D2H");
    MCU(cudaStreamSynchronize(ctx_stream(c)), "sync");
    return SRP_OK;
}

extern "C" int srp_mlp_infer(srp_ctx* c, const srp_mlp* m, const float* x, int64_t B, float* y, int mem) {
    if (!c || !m) return mfail(SRP_EINVAL, "srp_mlp_infer: NULL ctx/mlp");
    if (B < 0) return mfail(SRP_EINVAL, "srp_mlp_infer: negative batch");
    if (B == 0) return SRP_OK;
    if (!x || !y) return mfail(SRP_EINVAL, "srp_mlp_infer: NULL x/y");
    MCU(cudaSetDevice(m->device), "cudaSetDevice");
    cudaStream_t st = ctx_stream(c);
    if (mem == SRP_MEM_DEVICE) {
        MCU(mlp_forward(x, B, m->packed, m->params, y, ctx_err(c), st), "mlp forward launch");
        return SRP_OK;
    }
    if (mem != SRP_MEM_HOST) return mfail(SRP_EINVAL, "srp_mlp_infer: bad mem");
    // host memory: stream-ordered staging, freed on every path out
    float *dx = nullptr, *dy = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&dx, sizeof(float) * 19 * B, st);
    const char* where = "cudaMallocAsync";
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&dy, sizeof(float) * 6 * B, st);
    if (e == cudaSuccess) {
        where = "H2D x";
        e = cudaMemcpyAsync(dx, x, sizeof(float) * 19 * B, cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess) {
        where = "mlp forward launch";
        e = mlp_forward(dx, B, m->packed, m->params, dy, ctx_err(c), st);
    }
    if (e == cudaSuccess) {
        where = "D2H y";
        e = cudaMemcpyAsync(y, dy, sizeof(float) * 6 * B, cudaMemcpyDeviceToHost, st);
    }
    if (dx) cudaFreeAsync(dx, st);
    if (dy) cudaFreeAsync(dy, st);
    if (e != cudaSuccess) return mfail(SRP_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
    return srp_sync(c);
}


extern "C" int srp_mlp_train_step(srp_ctx* c, srp_mlp* m, const float* x, const float* t, int64_t B, float lr,
                                  float* loss_out, float* grad_out, int mem) {
    if (!c || !m) return mfail(SRP_EINVAL, "srp_mlp_train_step: NULL ctx/mlp");
    if (B < 1 || B > (1 << 24)) return mfail(SRP_EINVAL, "srp_mlp_train_step: batch must be in 1..2^24");
    if (!x || !t) return mfail(SRP_EINVAL, "srp_mlp_train_step: NULL x/t");
    if (!(lr >= 0.0f) || !std::isfinite(lr)) return mfail(SRP_EINVAL, "srp_mlp_train_step: bad learning rate");
    MCU(cudaSetDevice(m->device), "cudaSetDevice");
    cudaStream_t st = ctx_stream(c);
    const size_t need = train_bytes(B) + (mem == SRP_MEM_HOST ? sizeof(float) * 25 * (size_t)B + 512 : 0);
    if (m->work_bytes < need) {
        if (m->work) cudaFree(m->work);
        m->work = nullptr; m->work_bytes = 0;
        if (cudaMalloc(&m->work, need) != cudaSuccess) return mfail(SRP_ENOMEM, "srp_mlp_train_step: workspace");
        m->work_bytes = need;
    }
    const float* dx = x;
    const float* dt = t;
    if (mem == SRP_MEM_HOST) {
        float* sx = (float*)((char*)m->work + (train_bytes(B) + 255) / 256 * 256);
        float* stg = sx + 19 * B;
        MCU(cudaMemcpyAsync(sx, x, sizeof(float) * 19 * B, cudaMemcpyHostToDevice, st), "H2D x");
        MCU(cudaMemcpyAsync(stg, t, sizeof(float) * 6 * B, cudaMemcpyHostToDevice, st), "H2D t");
        dx = sx; dt = stg;
    } else if (mem != SRP_MEM_DEVICE) {
        return mfail(SRP_EINVAL, "srp_mlp_train_step: bad mem");
    }
    if (lr > 0.0f) m->step += 1;
    MCU(mlp_train(dx, dt, nullptr, B, B, m->params, m->grad, m->adam_m, m->adam_v, m->step, lr, m->work, m->packed,
                  ctx_err(c), st),
        "training launch");
    if (grad_out) MCU(cudaMemcpyAsync(grad_out, m->grad, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost, st), "D2H grad");
    if (loss_out) MCU(cudaMemcpyAsync(loss_out, train_loss_ptr(m->work, B), sizeof(float), cudaMemcpyDeviceToHost, st), "D2H loss");
    if (grad_out || loss_out || mem == SRP_MEM_HOST) return srp_sync(c);
    return SRP_OK;
}

extern "C" int srp_mlp_train_epoch(srp_ctx* c, srp_mlp* m, const float* x, const float* t, int64_t n,
                                   const int32_t* idx, int64_t batch, int64_t n_steps, const float* lr) {
    if (!c || !m) return mfail(SRP_EINVAL, "srp_mlp_train_epoch: NULL ctx/mlp");
    if (n < 1) return mfail(SRP_EINVAL, "srp_mlp_train_epoch: the data set needs at least one row");
    if (batch < 1 || batch > (1 << 24)) return mfail(SRP_EINVAL, "srp_mlp_train_epoch: batch must be in 1..2^24");
    if (n_steps < 0) return mfail(SRP_EINVAL, "srp_mlp_train_epoch: negative step count");
    if (n_steps == 0) return SRP_OK;
    if (!x || !t || !idx || !lr) return mfail(SRP_EINVAL, "srp_mlp_train_epoch: NULL x/t/idx/lr");
    if (n > ((int64_t)1 << 31)) return mfail(SRP_EINVAL, "srp_mlp_train_epoch: more rows than int32 indices address");
    for (int64_t s = 0; s < n_steps; ++s)
        if (!(lr[s] > 0.0f) || !std::isfinite(lr[s]))
            return mfail(SRP_EINVAL, "srp_mlp_train_epoch: every learning rate must be finite and > 0");
    MCU(cudaSetDevice(m->device), "cudaSetDevice");
    cudaStream_t st = ctx_stream(c);
    const size_t need = train_bytes(batch);
    if (m->work_bytes < need) {
        if (m->work) cudaFree(m->work);
        m->work = nullptr; m->work_bytes = 0;
        if (cudaMalloc(&m->work, need) != cudaSuccess) return mfail(SRP_ENOMEM, "srp_mlp_train_epoch: workspace");
        m->work_bytes = need;
    }
    for (int64_t s = 0; s < n_steps; ++s) {
        m->step += 1;
        MCU(mlp_train(x, t, idx + s * batch, n, batch, m->params, m->grad, m->adam_m, m->adam_v, m->step, lr[s],
                      m->work, m->packed, ctx_err(c), st),
            "training launch");
    }
    return SRP_OK;
}

extern "C" int srp_mlp_grad_input(srp_ctx* c, srp_mlp* m, const float* x, const float* wy, int64_t B, float* gx,
                                  int mem) {
    if (!c || !m) return mfail(SRP_EINVAL, "srp_mlp_grad_input: NULL ctx/mlp");
    if (B < 0 || B > (1 << 24)) return mfail(SRP_EINVAL, "srp_mlp_grad_input: batch must be in 0..2^24");
    if (B == 0) return SRP_OK;
    if (!x || !wy || !gx) return mfail(SRP_EINVAL, "srp_mlp_grad_input: NULL x/wy/gx");
    if (mem != SRP_MEM_HOST && mem != SRP_MEM_DEVICE) return mfail(SRP_EINVAL, "srp_mlp_grad_input: bad mem");
    MCU(cudaSetDevice(m->device), "cudaSetDevice");
    cudaStream_t st = ctx_stream(c);
    const size_t stage = mem == SRP_MEM_HOST ? sizeof(float) * 44 * (size_t)B + 1024 : 0;
    const size_t need = train_bytes(B) + stage;
    if (m->work_bytes < need) {
        if (m->work) cudaFree(m->work);
        m->work = nullptr; m->work_bytes = 0;
        if (cudaMalloc(&m->work, need) != cudaSuccess) return mfail(SRP_ENOMEM, "srp_mlp_grad_input: workspace");
        m->work_bytes = need;
    }
    if (mem == SRP_MEM_DEVICE) {
        MCU(mlp_input_grad(x, wy, B, m->params, m->packed, gx, m->work, ctx_err(c), st), "input-gradient launch");
        return SRP_OK;
    }
    float* sx = (float*)((char*)m->work + (train_bytes(B) + 255) / 256 * 256);
    float* sw = sx + 19 * B;
    float* sg = sw + 6 * B;
    MCU(cudaMemcpyAsync(sx, x, sizeof(float) * 19 * B, cudaMemcpyHostToDevice, st), "H2D x");
    MCU(cudaMemcpyAsync(sw, wy, sizeof(float) * 6 * B, cudaMemcpyHostToDevice, st), "H2D wy");
    MCU(mlp_input_grad(sx, sw, B, m->params, m->packed, sg, m->work, ctx_err(c), st), "input-gradient launch");
    MCU(cudaMemcpyAsync(gx, sg, sizeof(float) * 19 * B, cudaMemcpyDeviceToHost, st), "D2H gx");
    return srp_sync(c);
}

// File format: 8-byte tag "SRPMLP1", int64 parameter count, then the FP32
// parameters in the order of srp_mlp_param_count (host byte order).
extern "C" int srp_mlp_save(srp_ctx* c, const srp_mlp* m, const char* path) {
    if (!c || !m || !path) return mfail(SRP_EINVAL, "srp_mlp_save: NULL argument");
    std::vector<float> p(kMlpParams);
    int rc = srp_mlp_get_params(c, m, p.data());
    if (rc != SRP_OK) return rc;
    FILE* f = std::fopen(path, "wb");
    if (!f) return mfail(SRP_EINVAL, std::string("srp_mlp_save: cannot open ") + path);
    const char tag[8] = {'S', 'R', 'P', 'M', 'L', 'P', '1', 0};
    const int64_t n = kMlpParams;
    bool ok = std::fwrite(tag, 1, 8, f) == 8 && std::fwrite(&n, sizeof n, 1, f) == 1 &&
              std::fwrite(p.data(), sizeof(float), p.size(), f) == p.size();
    ok = (std::fclose(f) == 0) && ok;
    return ok ? SRP_OK : mfail(SRP_EINVAL, std::string("srp_mlp_save: write failed: ") + path);
}

extern "C" int srp_mlp_load(srp_ctx* c, srp_mlp* m, const char* path) {
    if (!c || !m || !path) return mfail(SRP_EINVAL, "srp_mlp_load: NULL argument");
    FILE* f = std::fopen(path, "rb");
    if (!f) return mfail(SRP_EINVAL, std::string("srp_mlp_load: cannot open ") + path);
    char tag[8];
    int64_t n = 0;
    std::vector<float> p(kMlpParams);
    bool ok = std::fread(tag, 1, 8, f) == 8 && std::memcmp(tag, "SRPMLP1", 8) == 0 &&
              std::fread(&n, sizeof n, 1, f) == 1 && n == kMlpParams &&
              std::fread(p.data(), sizeof(float), p.size(), f) == p.size();
    std::fclose(f);
    if (!ok) return mfail(SRP_EINVAL, std::string("srp_mlp_load: not a parameter file of this network: ") + path);
    return srp_mlp_set_params(c, m, p.data());
}


// Trainer state: tag "SRPMLS1\0", int64 P, int64 Adam step, then params, the
// first and the second moments as float32 [P] each (host byte order).
extern "C" int srp_mlp_save_state(srp_ctx* c, const srp_mlp* m, const char* path) {
    if (!c || !m || !path) return mfail(SRP_EINVAL, "srp_mlp_save_state: NULL argument");
    MCU(cudaSetDevice(m->device), "cudaSetDevice");
    MCU(cudaStreamSynchronize(ctx_stream(c)), "sync");   // training steps in flight finish first
    std::vector<float> buf(3 * (size_t)kMlpParams);
    const float* src[3] = {m->params, m->adam_m, m->adam_v};
    for (int a = 0; a < 3; ++a)
        MCU(cudaMemcpy(buf.data() + (size_t)a * kMlpParams, src[a], sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost),
            "D2H state");
    FILE* f = std::fopen(path, "wb");
    if (!f) return mfail(SRP_EINVAL, std::string("srp_mlp_save_state: cannot open ") + path);
    const char tag[8] = {'S', 'R', 'P', 'M', 'L', 'S', '1', 0};
    const int64_t head[2] = {kMlpParams, m->step};
    bool ok = std::fwrite(tag, 1, 8, f) == 8 && std::fwrite(head, sizeof(int64_t), 2, f) == 2 &&
              std::fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    ok = (std::fclose(f) == 0) && ok;
    return ok ? SRP_OK : mfail(SRP_EINVAL, std::string("srp_mlp_save_state: write failed: ") + path);
}

extern "C" int srp_mlp_load_state(srp_ctx* c, srp_mlp* m, const char* path) {
    if (!c || !m || !path) return mfail(SRP_EINVAL, "srp_mlp_load_state: NULL argument");
    FILE* f = std::fopen(path, "rb");
    if (!f) return mfail(SRP_EINVAL, std::string("srp_mlp_load_state: cannot open ") + path);
    char tag[8];
    int64_t head[2] = {0, 0};
    std::vector<float> buf(3 * (size_t)kMlpParams);
    bool ok = std::fread(tag, 1, 8, f) == 8 && std::memcmp(tag, "SRPMLS1", 8) == 0 &&
              std::fread(head, sizeof(int64_t), 2, f) == 2 && head[0] == kMlpParams && head[1] >= 0 &&
              std::fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    std::fclose(f);
    if (!ok) return mfail(SRP_EINVAL, std::string("srp_mlp_load_state: not a trainer-state file of this network: ") + path);
    const float* mv = buf.data() + kMlpParams;
    for (int64_t q = 0; q < 2 * kMlpParams; ++q)
        if (!std::isfinite(mv[q]) || (q >= kMlpParams && mv[q] < 0.0f))
            return mfail(SRP_EINVAL, "srp_mlp_load_state: invalid Adam moments");
    int rc = srp_mlp_set_params(c, m, buf.data());   // parameters and their BF16 copies; resets Adam
    if (rc != SRP_OK) return rc;
    MCU(cudaMemcpy(m->adam_m, mv, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice), "H2D moments");
    MCU(cudaMemcpy(m->adam_v, mv + kMlpParams, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice), "H2D moments");
    m->step = head[1];
    return SRP_OK;
}
