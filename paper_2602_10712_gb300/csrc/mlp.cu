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
// Forward kernel (one CTA of 128 threads per 128 batch rows):
//   X (FP32) -> BF16 tile in smem; per layer: bulk-copy W_l into smem,
//   one thread issues K_l/16 tcgen05.mma (M=128, N=N_l, K=16) into a
//   256-column TMEM accumulator, commit -> mbarrier; the four warps read
//   their 32 TMEM lanes (= rows) with tcgen05.ld, add the bias, apply SiLU,
//   round to BF16 and write the next layer's A tile.  Every wait is
//   bounded; on a timeout the kernel records an error, waits (bounded) for
//   its in-flight operations, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "srp_internal.h"
#include "tc_common.cuh"

namespace srp {

constexpr int kMlpLayers = 5;
__host__ __device__ constexpr int mlp_in(int l) { return l == 0 ? 19 : 256; }
__host__ __device__ constexpr int mlp_out(int l) { return l == kMlpLayers - 1 ? 6 : 256; }
__host__ __device__ constexpr int mlp_K(int l) { return l == 0 ? 32 : 256; }                 // padded K
__host__ __device__ constexpr int mlp_N(int l) { return l == kMlpLayers - 1 ? 16 : 256; }    // padded N
constexpr int kMlpParams = 19 * 256 + 256 + 3 * (256 * 256 + 256) + 256 * 6 + 6;
constexpr uint32_t kWaitLimit = 1u << 24;
constexpr int kErrMlpTimeout = 4;

struct MlpLayout {
    int64_t w_off[kMlpLayers];   // FP32 weight offset in the flat vector
    int64_t b_off[kMlpLayers];
    int64_t p_off[kMlpLayers];   // BF16 packed offset (elements)
    int64_t packed_elems;
};

__host__ __device__ inline MlpLayout mlp_layout() {
    MlpLayout L;
    int64_t o = 0, q = 0;
    for (int l = 0; l < kMlpLayers; ++l) {
        L.w_off[l] = o;
        o += (int64_t)mlp_in(l) * mlp_out(l);
        L.b_off[l] = o;
        o += mlp_out(l);
        L.p_off[l] = q;
        q += (int64_t)mlp_N(l) * mlp_K(l);
    }
    L.packed_elems = q;
    return L;
}

// FP32 master weights -> BF16 packed per layer (zero padding).
__global__ void mlp_pack_kernel(const float* __restrict__ params, __nv_bfloat16* __restrict__ packed) {
    const MlpLayout L = mlp_layout();
    const int64_t tot = L.packed_elems;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        int l = 0;
        while (l + 1 < kMlpLayers && e >= L.p_off[l + 1]) ++l;
        const int64_t loc = e - L.p_off[l];
        const int K = mlp_K(l), N = mlp_N(l);
        const int n = (int)(loc / K), k = (int)(loc % K);
        (void)N;
        const float w = (n < mlp_out(l) && k < mlp_in(l)) ? params[L.w_off[l] + (int64_t)n * mlp_in(l) + k] : 0.0f;
        packed[L.p_off[l] + tc::kmajor_off(n, k, K) / 2] = __float2bfloat16_rn(w);
    }
}

struct MlpFwdSmem {
    alignas(1024) unsigned char act[128 * 256 * 2];   // A tile (64 KB)
    alignas(1024) unsigned char w[256 * 256 * 2];     // B tile (128 KB)
    alignas(8) uint64_t bar_w;
    alignas(8) uint64_t bar_mma;
    uint32_t tmem_base;
    int failed;
};

__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + __expf(-z)); }

__global__ void __launch_bounds__(128, 1) mlp_fwd_kernel(const float* __restrict__ x, int64_t B,
                                                        const __nv_bfloat16* __restrict__ packed,
                                                        const float* __restrict__ params, float* __restrict__ y,
                                                        int* err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    MlpFwdSmem& sm = *reinterpret_cast<MlpFwdSmem*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const MlpLayout L = mlp_layout();
    const int64_t row0 = (int64_t)blockIdx.x * 128;
    if (tid == 0) {
        tc::mbar_init(&sm.bar_w, 1);
        tc::mbar_init(&sm.bar_mma, 1);
        sm.failed = 0;
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(&sm.tmem_base, 256);
        tc::tmem_relinquish();
    }
    // input tile: row r = tid, K = 32 (19 used)
    {
        const int64_t row = row0 + tid;
        float v[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = 0.0f;
        if (row < B) {
#pragma unroll
            for (int j = 0; j < 19; ++j) v[j] = x[row * 19 + j];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            __align__(16) __nv_bfloat16 h[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) h[j] = __float2bfloat16_rn(v[8 * q + j]);
            *reinterpret_cast<uint4*>(sm.act + tc::kmajor_off(tid, 8 * q, 32)) = *reinterpret_cast<uint4*>(h);
        }
    }
    tc::fence_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tbase = sm.tmem_base;
    uint32_t ph_w = 0, ph_m = 0;
    for (int l = 0; l < kMlpLayers; ++l) {
        const int K = mlp_K(l), N = mlp_N(l);
        const uint32_t wbytes = (uint32_t)(N * K * 2);
        if (tid == 0) {
            tc::mbar_expect_tx(&sm.bar_w, wbytes);
            const unsigned char* src = reinterpret_cast<const unsigned char*>(packed + L.p_off[l]);
            for (uint32_t o = 0; o < wbytes; o += 32768u) {
                const uint32_t nb = wbytes - o < 32768u ? wbytes - o : 32768u;
                tc::bulk_g2s(sm.w + o, src + o, nb, &sm.bar_w);
            }
        }
        if (!tc::mbar_wait_bounded(&sm.bar_w, ph_w, kWaitLimit)) sm.failed = 1;
        ph_w ^= 1;
        __syncthreads();
        if (sm.failed) break;
        if (tid == 0) {
            tc::tc_fence_after();
            const uint32_t a0 = tc::smem_u32(sm.act), b0 = tc::smem_u32(sm.w);
            const uint32_t sbo = (uint32_t)(K / 8) * 128u;
            const uint32_t idesc = tc::idesc_bf16(128, N);
            for (int kk = 0; kk < K / 16; ++kk) {
                const uint64_t ad = tc::sdesc(a0 + kk * 256u, 128u, sbo);
                const uint64_t bd = tc::sdesc(b0 + kk * 256u, 128u, sbo);
                tc::mma_bf16(tbase, ad, bd, idesc, kk > 0 ? 1u : 0u);
            }
            tc::mma_commit(&sm.bar_mma);
        }
        if (!tc::mbar_wait_bounded(&sm.bar_mma, ph_m, kWaitLimit)) sm.failed = 1;
        ph_m ^= 1;
        __syncthreads();
        if (sm.failed) break;
        tc::tc_fence_after();
        // epilogue: warp w owns TMEM lanes (rows) 32w..32w+31
        const int r = 32 * warp + lane;
        const uint32_t taddr = tbase + ((uint32_t)(32 * warp) << 16);
        if (l < kMlpLayers - 1) {
            const float* bias = params + L.b_off[l];
            for (int c = 0; c < N / 32; ++c) {
                float v[32];
                tc::tmem_ld32(taddr + 32u * c, v);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    __align__(16) __nv_bfloat16 h[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) h[j] = __float2bfloat16_rn(silu_f(v[8 * q + j] + bias[32 * c + 8 * q + j]));
                    *reinterpret_cast<uint4*>(sm.act + tc::kmajor_off(r, 32 * c + 8 * q, 256)) =
                        *reinterpret_cast<uint4*>(h);
                }
            }
        } else {
            const float* bias = params + L.b_off[l];
            float v[32];
            tc::tmem_ld32(taddr, v);
            const int64_t row = row0 + r;
            if (row < B) {
#pragma unroll
                for (int j = 0; j < 6; ++j) y[row * 6 + j] = v[j] + bias[j];
            }
        }
        tc::fence_async_smem();
        tc::tc_fence_before();
        __syncthreads();
        tc::tc_fence_after();
    }
    if (sm.failed) {
        if (tid == 0) atomicOr(err, kErrMlpTimeout);
        // wait (bounded) for anything still in flight before freeing TMEM
        tc::mbar_wait_bounded(&sm.bar_mma, ph_m, kWaitLimit);
        tc::mbar_wait_bounded(&sm.bar_w, ph_w, kWaitLimit);
        __syncthreads();
    }
    if (warp == 0) tc::tmem_dealloc(tbase, 256);
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
    const unsigned grid = (unsigned)((B + 127) / 128);
    mlp_fwd_kernel<<<grid, 128, sm, st>>>(x, B, (const __nv_bfloat16*)packed, params, y, err);
    return cudaGetLastError();
}

int64_t mlp_param_count() { return kMlpParams; }
int64_t mlp_packed_bytes() { return mlp_layout().packed_elems * 2; }

void set_last_error(const std::string& msg);
cudaStream_t ctx_stream(srp_ctx* c);
int ctx_device(srp_ctx* c);
int* ctx_err(srp_ctx* c);
int ctx_n_sm(srp_ctx* c);

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
    float *dx = nullptr, *dy = nullptr;
    MCU(cudaMallocAsync((void**)&dx, sizeof(float) * 19 * B, st), "cudaMallocAsync");
    MCU(cudaMallocAsync((void**)&dy, sizeof(float) * 6 * B, st), "cudaMallocAsync");
    MCU(cudaMemcpyAsync(dx, x, sizeof(float) * 19 * B, cudaMemcpyHostToDevice, st), "H2D x");
    MCU(mlp_forward(dx, B, m->packed, m->params, dy, ctx_err(c), st), "mlp forward launch");
    MCU(cudaMemcpyAsync(y, dy, sizeof(float) * 6 * B, cudaMemcpyDeviceToHost, st), "D2H y");
    MCU(cudaFreeAsync(dx, st), "cudaFreeAsync");
    MCU(cudaFreeAsync(dy, st), "cudaFreeAsync");
    return srp_sync(c);
}
