// gemm.cu -- a general BF16 tensor-core GEMM on tcgen05 for the proxy
// network's training passes:  C[M x N] (+)= alpha * sum_k A(m,k) * B(n,k).
//
// Operands are FP32 in global memory, read either row-major in K
// (element (r,k) at p[r*ld + k]) or transposed (p[k*ld + r]), so the same
// kernel computes Z = H W^T (forward), dH = dZ W (backward, W read
// transposed) and dW = dZ^T H (backward, both read transposed, K = batch).
// CTA tile 128 x BN (BN <= 128, multiple of 32) x 64 in K: 128 threads
// convert a K chunk of A and B to BF16 into shared memory (K-major
// no-swizzle core-matrix layout) while the tensor core works on the previous
// chunk (double buffer, one mbarrier per buffer signalled by tcgen05.commit);
// one thread issues four tcgen05.mma (M=128, N=BN, K=16) per chunk into a
// 256-column TMEM accumulator; the epilogue reads TMEM with tcgen05.ld and
// stores (or, for split-K over gridDim.z, atomically adds) FP32 C.
// All waits are bounded; on a timeout the CTA flags an error, waits
// (bounded) for its MMAs, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "srp_internal.h"
#include "tc_common.cuh"

namespace srp {

struct GemmOp {
    const float* p;
    int64_t ld;
    int trans;  // 0: (r,k) at p[r*ld+k]; 1: at p[k*ld+r]
};

struct GemmArgs {
    GemmOp A, B;
    int M, N, K;
    int BN;           // N tile (multiple of 32, <= 256)
    int k_split;      // K elements per gridDim.z slice (multiple of 64)
    float alpha;
    float* C;
    int64_t ldc;
    int atomic;       // 1: atomicAdd into C, 0: store
    int* err;
};

constexpr int kGemmBK = 64;
constexpr uint32_t kGemmWait = 1u << 24;

struct GemmSmem {
    alignas(1024) unsigned char a[2][128 * kGemmBK * 2];   // 2 x 16 KB
    alignas(1024) unsigned char b[2][256 * kGemmBK * 2];   // 2 x 32 KB
    alignas(8) uint64_t bar[2];
    uint32_t tmem_base;
};

// Stage rows [r0, r0+R) x k [k0, k0+64) of an operand into smem (BF16).
// Items are (row r, 8-wide K chunk k8); a warp's 32 items are 8 rows x 4
// chunks of one 8-row group, whose 16-byte slots in the core-matrix layout
// are 512 contiguous bytes (no bank conflicts; one thread per row put a
// warp's stores 1 KB apart).  An operand stored row-major in K is read with
// two 16-byte loads per item when its base and leading dimension allow it.
__device__ __forceinline__ void gemm_stage(unsigned char* dst, const GemmOp& op, bool vec, int r0, int R,
                                           int rows_valid, int k0, int k_end, int tid) {
    for (int it = tid; it < R * (kGemmBK / 8); it += 128) {
        const int r = (it & 7) + 8 * (it >> 6), k8 = (it >> 3) & 7;
        const int gr = r0 + r, kb = k0 + 8 * k8;
        float v[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        if (r < rows_valid) {
            if (!op.trans && vec && kb + 7 < k_end) {
                const float4* q = reinterpret_cast<const float4*>(op.p + (int64_t)gr * op.ld + kb);
                const float4 q0 = __ldg(q), q1 = __ldg(q + 1);
                v[0] = q0.x; v[1] = q0.y; v[2] = q0.z; v[3] = q0.w;
                v[4] = q1.x; v[5] = q1.y; v[6] = q1.z; v[7] = q1.w;
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int k = kb + j;
                    if (k < k_end) v[j] = op.trans ? op.p[(int64_t)k * op.ld + gr] : op.p[(int64_t)gr * op.ld + k];
                }
            }
        }
        __align__(16) __nv_bfloat16 h[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) h[j] = __float2bfloat16_rn(v[j]);
        *reinterpret_cast<uint4*>(dst + tc::kmajor_off(r, 8 * k8, kGemmBK)) = *reinterpret_cast<uint4*>(h);
    }
}

__global__ void __launch_bounds__(128, 1) gemm_kernel(const GemmArgs g) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    GemmSmem& sm = *reinterpret_cast<GemmSmem*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * 128, n0 = blockIdx.y * g.BN;
    const int kz0 = blockIdx.z * g.k_split;
    const int kz1 = min(g.K, kz0 + g.k_split);
    const int nk = kz1 > kz0 ? (kz1 - kz0 + kGemmBK - 1) / kGemmBK : 0;
    if (tid == 0) {
        tc::mbar_init(&sm.bar[0], 1);
        tc::mbar_init(&sm.bar[1], 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(&sm.tmem_base, 256);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tbase = sm.tmem_base;
    const uint32_t idesc = tc::idesc_bf16(128, g.BN);
    const int mv = min(128, g.M - m0), nv = min(g.BN, g.N - n0);
    const bool vec_a = (reinterpret_cast<uintptr_t>(g.A.p) & 15) == 0 && (g.A.ld & 3) == 0;
    const bool vec_b = (reinterpret_cast<uintptr_t>(g.B.p) & 15) == 0 && (g.B.ld & 3) == 0;
    int failed = 0;  // block-uniform (decided with __syncthreads_or)
    for (int i = 0; i < nk; ++i) {
        const int buf = i & 1;
        bool ok = true;
        if (i >= 2) ok = tc::mbar_wait_bounded(&sm.bar[buf], ((i >> 1) - 1) & 1, kGemmWait);
        if (__syncthreads_or(!ok)) { failed = 1; break; }
        const int k0 = kz0 + i * kGemmBK;
        gemm_stage(sm.a[buf], g.A, vec_a, m0, 128, mv, k0, kz1, tid);
        gemm_stage(sm.b[buf], g.B, vec_b, n0, g.BN, nv, k0, kz1, tid);
        tc::fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc::tc_fence_after();
            const uint32_t a0 = tc::smem_u32(sm.a[buf]), b0 = tc::smem_u32(sm.b[buf]);
            const uint32_t sbo = (kGemmBK / 8) * 128u;
#pragma unroll
            for (int kk = 0; kk < kGemmBK / 16; ++kk)
                tc::mma_bf16(tbase, tc::sdesc(a0 + kk * 256u, 128u, sbo), tc::sdesc(b0 + kk * 256u, 128u, sbo), idesc,
                             (i > 0 || kk > 0) ? 1u : 0u);
            tc::mma_commit(&sm.bar[buf]);
        }
    }
    const bool have = nk > 0;
    if (!failed && have) {
        const int last = nk - 1;
        const bool ok = tc::mbar_wait_bounded(&sm.bar[last & 1], (last >> 1) & 1, kGemmWait);
        failed = __syncthreads_or(!ok);
    }
    if (failed) {
        if (tid == 0) atomicOr(g.err, kErrWaitTimeout);
        // bounded wait for MMAs possibly still running, then free TMEM
        const int last = nk - 1;
        tc::mbar_wait_bounded(&sm.bar[last & 1], (last >> 1) & 1, kGemmWait);
        __syncthreads();
        if (warp == 0) tc::tmem_dealloc(tbase, 256);
        return;
    }
    tc::tc_fence_after();
    if (have) {
        const int r = 32 * warp + lane;
        const uint32_t taddr = tbase + ((uint32_t)(32 * warp) << 16);
        for (int c = 0; c < g.BN / 32; ++c) {
            float v[32];
            tc::tmem_ld32(taddr + 32u * c, v);
            if (r < mv) {
                float* crow = g.C + (int64_t)(m0 + r) * g.ldc + n0 + 32 * c;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    if (32 * c + j < nv) {
                        if (g.atomic) atomicAdd(crow + j, g.alpha * v[j]);
                        else crow[j] = g.alpha * v[j];
                    }
                }
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, 256);
}

// C = alpha * A B^T (or += with atomic=1 and split-K).  k_split = 0: no split.
cudaError_t tc_gemm(GemmOp A, GemmOp B, int M, int N, int K, float alpha, float* C, int64_t ldc, int atomic,
                    int k_split, int* err, cudaStream_t st) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    GemmArgs g;
    g.A = A; g.B = B; g.M = M; g.N = N; g.K = K;
    g.BN = std::min(128, (N + 31) / 32 * 32);   // N tiles of 128: twice the CTAs of 256 at N = 256
    g.k_split = k_split > 0 ? (k_split + kGemmBK - 1) / kGemmBK * kGemmBK : std::max(K, 1);
    g.alpha = alpha; g.C = C; g.ldc = ldc; g.atomic = atomic; g.err = err;
    const size_t sm = sizeof(GemmSmem);
    cudaError_t e = cudaFuncSetAttribute(gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 grid((M + 127) / 128, (N + g.BN - 1) / g.BN, std::max(1, (K + g.k_split - 1) / g.k_split));
    gemm_kernel<<<grid, 128, sm, st>>>(g);
    return cudaGetLastError();
}

}  // namespace srp
