// mlp_common.cuh -- shapes and packed BF16 weight layouts of the neural
// proxy 19 -> 256 x4 (SiLU) -> 6, shared by the inference kernel (mlp.cu)
// and the training kernels (train.cu).
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

#include "tc_common.cuh"

namespace srp {

constexpr int kMlpLayers = 5;
__host__ __device__ constexpr int mlp_in(int l) { return l == 0 ? 19 : 256; }
__host__ __device__ constexpr int mlp_out(int l) { return l == kMlpLayers - 1 ? 6 : 256; }
__host__ __device__ constexpr int mlp_K(int l) { return l == 0 ? 32 : 256; }                 // padded K
__host__ __device__ constexpr int mlp_N(int l) { return l == kMlpLayers - 1 ? 16 : 256; }    // padded N
constexpr int kMlpParams = 19 * 256 + 256 + 3 * (256 * 256 + 256) + 256 * 6 + 6;
constexpr uint32_t kWaitLimit = 1u << 24;

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

// Packed BF16 weights: per layer, K cut into chunks of KC = min(64, K)
// columns; each chunk is a contiguous K-major no-swizzle N x KC tile, so
// one bulk copy brings one chunk and the MMAs of that K range can start as
// soon as it lands.
__host__ __device__ constexpr int mlp_KC(int l) { return mlp_K(l) < 64 ? mlp_K(l) : 64; }
__host__ __device__ inline uint32_t mlp_packed_off(int l, int n, int k) {   // bytes within layer l
    const int KC = mlp_KC(l), c = k / KC;
    return (uint32_t)c * (uint32_t)(mlp_N(l) * KC * 2) + tc::kmajor_off((uint32_t)n, (uint32_t)(k - c * KC), (uint32_t)KC);
}

// Transposed packed weights for the backward pass dH = dZ W: layer l as an
// NT x KT K-major tile (NT = in padded, KT = out padded: rows are input
// features, K runs over output features), in chunks of KCT = min(64, KT)
// columns like the forward layout.  They follow the forward weights in the
// same buffer.
__host__ __device__ constexpr int mlp_NT(int l) { return l == 0 ? 32 : 256; }
__host__ __device__ constexpr int mlp_KT(int l) { return l == kMlpLayers - 1 ? 16 : 256; }
__host__ __device__ constexpr int mlp_KCT(int l) { return mlp_KT(l) < 64 ? mlp_KT(l) : 64; }
__host__ __device__ inline int64_t mlp_pT_off(int l) {   // elements, from the start of the packed buffer
    int64_t q = mlp_layout().packed_elems;
    for (int j = 0; j < l; ++j) q += (int64_t)mlp_NT(j) * mlp_KT(j);
    return q;
}
__host__ __device__ inline int64_t mlp_packed_all_elems() { return mlp_pT_off(kMlpLayers); }
__host__ __device__ inline uint32_t mlp_packedT_off(int l, int n, int k) {   // bytes within layer l
    const int KC = mlp_KCT(l), c = k / KC;
    return (uint32_t)c * (uint32_t)(mlp_NT(l) * KC * 2) + tc::kmajor_off((uint32_t)n, (uint32_t)(k - c * KC), (uint32_t)KC);
}

}  // namespace srp
