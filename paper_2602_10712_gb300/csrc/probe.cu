// probe.cu -- read-bandwidth probe: the memory ceiling that the traversal's
// algorithmic bytes are held against.
//
// A BVH walk reads node and triangle records that (for one design of up to
// a few hundred thousand triangles) stay resident in the 129 MB L2, so its
// bandwidth roof is the L2's, not HBM's.  The probe reads a buffer of a given
// size from every SM with 16-byte loads that bypass L1 (ld.global.cg: cached
// in L2 only), 16 independent loads in flight per thread, a full-occupancy
// grid (resident blocks x SMs), many passes per launch.  A buffer that fits
// in L2 gives the L2 read rate; one of several GB gives the HBM read rate.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

namespace srp {

constexpr int kProbeThreads = 512;
constexpr int kProbeUnroll = 16;

__device__ __forceinline__ uint4 ld_cg_v4(const uint4* p) {
    uint4 v;
    asm volatile("ld.global.cg.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

// Every round, every thread issues kProbeUnroll independent 16-byte loads at
// consecutive grid strides (mod the buffer): words tid + k nth, k counting
// on across rounds.  `rounds` is chosen on the host so that one launch
// sweeps the buffer `passes` times (at least one round per pass); a buffer
// smaller than one round's reach (nth x kProbeUnroll words) is read by
// several SMs per round, as every SM reads the same BVH.  Bytes counted:
// rounds x nth x kProbeUnroll x 16.
__global__ void __launch_bounds__(kProbeThreads) read_probe_kernel(const uint4* __restrict__ buf, int64_t n16,
                                                                   int64_t rounds, uint32_t* __restrict__ sink) {
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0;
    int64_t base = tid % n16;
    const int64_t step = nth % n16;
    for (int64_t p = 0; p < rounds; ++p) {
        uint4 v[kProbeUnroll];
        int64_t j = base;
#pragma unroll
        for (int u = 0; u < kProbeUnroll; ++u) {
            v[u] = ld_cg_v4(buf + j);
            j += step;
            if (j >= n16) j -= n16;
        }
#pragma unroll
        for (int u = 0; u < kProbeUnroll; ++u) acc ^= v[u].x ^ v[u].y ^ v[u].z ^ v[u].w;
        base = j;
    }
    // the loads stay live: the result is stored unless it matches a value
    // the buffer's fill pattern cannot produce
    if (acc == 0x5bd1e995u) sink[0] = acc;
}

// Allocates `bytes` (rounded down to 16), fills it, runs one warm-up launch
// and `reps` timed launches of `passes` passes on `st`; returns the best
// rate in GB/s (1e9 bytes/s) of bytes read.
cudaError_t run_read_probe(int64_t bytes, int passes, int reps, cudaStream_t st, double* out_gbs) {
    *out_gbs = 0.0;
    const int64_t n16 = bytes / 16;
    if (n16 <= 0 || passes < 1 || reps < 1) return cudaErrorInvalidValue;
    int dev = 0, n_sm = 0, nb = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, read_probe_kernel, kProbeThreads, 0);
    if (e != cudaSuccess) return e;
    const int grid = n_sm * std::max(nb, 1);
    const int64_t reach = (int64_t)grid * kProbeThreads * kProbeUnroll;   // words per round
    const int64_t rounds = (int64_t)passes * std::max<int64_t>(1, (n16 + reach - 1) / reach);
    uint4* buf = nullptr;
    uint32_t* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaMalloc(&buf, (size_t)n16 * 16);
    if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0x11, (size_t)n16 * 16, st);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        read_probe_kernel<<<grid, kProbeThreads, 0, st>>>(buf, n16, rounds, sink);
        e = cudaGetLastError();
    }
    float best = 0.0f;
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) {
            read_probe_kernel<<<grid, kProbeThreads, 0, st>>>(buf, n16, rounds, sink);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms > 0.0f && (best == 0.0f || ms < best)) best = ms;
    }
    if (e == cudaSuccess && best > 0.0f) *out_gbs = (double)reach * 16.0 * (double)rounds / (best * 1e-3) / 1e9;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (buf) cudaFree(buf);
    return e;
}

}  // namespace srp
