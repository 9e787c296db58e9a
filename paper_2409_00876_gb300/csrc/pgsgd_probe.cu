// Measurement helpers; the layout never calls them.
// L2 read bandwidth of this GPU, the ceiling for graphs whose records fit in
// L2 (the 200 k-node workload: 3.5 MB of node records, 112 MB of step
// records). Two patterns over one L2-resident buffer: streaming 16-byte
// vector loads (each warp reads 512 contiguous bytes) and random 16-byte loads
// (one 32-byte sector each, as the update kernel's record reads).
// HBM random-read rate: random 16-byte loads from a multi-GB buffer (the
// step-record reads of the chromosome graph, whose 7.5 GB of step records
// are far beyond L2), the ceiling for a kernel bound by random sectors.
#include <algorithm>
#include <cstdint>

#include "../../include/pgsgd.h"
#include "pgsgd_internal.h"

namespace pgsgd {
namespace {

// Four independent 16-byte loads in flight per thread; a warp reads 512
// contiguous bytes per load instruction.
__global__ void l2_stream_kernel(const uint4* __restrict__ buf, uint64_t n, uint32_t reps, uint32_t* out) {
    uint32_t acc = 0;
    const uint64_t nthr = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    for (uint32_t r = 0; r < reps; ++r) {
        for (uint64_t k = tid; k < n; k += 4 * nthr) {
            uint4 v[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const uint64_t idx = k + m * nthr;
                v[m] = make_uint4(0u, 0u, 0u, 0u);
                if (idx < n)
                    asm volatile("ld.global.cg.v4.u32 {%0,%1,%2,%3}, [%4];"
                                 : "=r"(v[m].x), "=r"(v[m].y), "=r"(v[m].z), "=r"(v[m].w) : "l"(buf + idx));
            }
#pragma unroll
            for (int m = 0; m < 4; ++m) acc ^= v[m].x ^ v[m].w;
        }
    }
    out[tid] = acc;
}

__device__ __forceinline__ uint64_t splitmix(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// loads_per_thread independent random 16-byte loads per thread, 4 in flight.
__global__ void l2_random_kernel(const uint4* __restrict__ buf, uint64_t n, uint32_t loads_per_thread, uint32_t* out) {
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    uint32_t acc = 0;
    for (uint32_t r = 0; r < loads_per_thread; r += 4) {
        uint4 v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint64_t idx = mulhi64(splitmix(tid * 0x100000001B3ull + r + k), n);  // < n
            asm volatile("ld.global.cg.v4.u32 {%0,%1,%2,%3}, [%4];"
                         : "=r"(v[k].x), "=r"(v[k].y), "=r"(v[k].z), "=r"(v[k].w) : "l"(buf + idx));
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) acc ^= v[k].x ^ v[k].w;
    }
    out[tid] = acc;
}

// Random reads from a buffer far larger than L2, in the forms the update
// kernel's step-record reads take. mode 0: one 16-byte load per thread with
// the evict-first policy and the 64-byte L2 prefetch-size hint (the update
// kernel's load_step); mode 1: the same load without the hint; mode 2: a
// random 64-byte block per group of four lanes (four coalesced 16-byte
// pieces, so the whole DRAM access is used). loads_per_thread independent
// loads per thread, four in flight. Every index is below n (mulhi64 of a
// 64-bit hash by n).
template <int MODE>
__global__ void hbm_gather_kernel(const uint4* __restrict__ buf, uint64_t n, uint32_t loads_per_thread,
                                  uint64_t salt, uint32_t* out) {
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t pol = policy_evict_first();
    uint32_t acc = 0;
    for (uint32_t r = 0; r < loads_per_thread; r += 4) {
        uint4 v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint64_t key = (MODE == 2 ? (tid >> 2) : tid) * 0x100000001B3ull + salt + r + k;
            uint64_t idx;
            if (MODE == 2) idx = mulhi64(splitmix(key), n >> 2) * 4 + (tid & 3);  // < n (n is a multiple of 4)
            else idx = mulhi64(splitmix(key), n);                                 // < n
            const uint4* q = buf + idx;
            if (MODE == 0)
                asm volatile("ld.global.cg.L2::cache_hint.L2::64B.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
                             : "=r"(v[k].x), "=r"(v[k].y), "=r"(v[k].z), "=r"(v[k].w) : "l"(q), "l"(pol));
            else
                asm volatile("ld.global.cg.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
                             : "=r"(v[k].x), "=r"(v[k].y), "=r"(v[k].z), "=r"(v[k].w) : "l"(q), "l"(pol));
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) acc ^= v[k].x ^ v[k].w;
    }
    out[tid] = acc;
}

}  // namespace
}  // namespace pgsgd

using namespace pgsgd;

extern "C" int pgsgd_hbm_gather_bandwidth(uint64_t bytes, uint32_t reps, int mode, int blocks_per_sm,
                                          double* loads_per_s, void* cuda_stream) {
    if (!loads_per_s) return report_error(PGSGD_EINVAL, "loads_per_s is NULL");
    if (bytes < (1ull << 30) || bytes > (64ull << 30))
        return report_error(PGSGD_EINVAL, "bytes must be in [1 GiB, 64 GiB]");
    if (reps == 0 || reps > 100) return report_error(PGSGD_EINVAL, "reps must be in [1, 100]");
    if (mode < 0 || mode > 2) return report_error(PGSGD_EINVAL, "mode must be 0, 1 or 2");
    if (blocks_per_sm < 1 || blocks_per_sm > 8) return report_error(PGSGD_EINVAL, "blocks_per_sm must be in [1, 8]");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t n = (bytes / 64) * 4;  // 16-byte records, a whole number of 64-byte blocks
    const int block = 256, grid = sms * blocks_per_sm;
    const uint32_t loads_per_thread = 512;
    uint4* buf = nullptr;
    uint32_t* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
        cudaFree(buf);
        cudaFree(out);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    cudaError_t e = cudaMalloc(&buf, n * 16);
    if (e == cudaSuccess) e = cudaMalloc(&out, (size_t)grid * block * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemsetAsync(buf, 1, n * 16, st);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cleanup();
        return report_error(PGSGD_ENOMEM, "HBM gather probe setup: %s", cudaGetErrorString(e));
    }
    float ms = 0.f;
    for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {  // pass 0 warms up
        e = cudaEventRecord(e0, st);
        for (uint32_t r = 0; r < reps && e == cudaSuccess; ++r) {
            const uint64_t salt = 0x5851F42D4C957F2Dull * (pass * 1000ull + r + 1);
            if (mode == 0) hbm_gather_kernel<0><<<grid, block, 0, st>>>(buf, n, loads_per_thread, salt, out);
            else if (mode == 1) hbm_gather_kernel<1><<<grid, block, 0, st>>>(buf, n, loads_per_thread, salt, out);
            else hbm_gather_kernel<2><<<grid, block, 0, st>>>(buf, n, loads_per_thread, salt, out);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    cleanup();
    if (e != cudaSuccess) return report_error(PGSGD_ECUDA, "HBM gather probe: %s", cudaGetErrorString(e));
    const double loads = (double)grid * block * loads_per_thread * reps / (mode == 2 ? 4.0 : 1.0);
    *loads_per_s = loads / (ms * 1e-3);
    return PGSGD_OK;
}

extern "C" int pgsgd_l2_bandwidth(uint64_t bytes, uint32_t reps, int mode, double* gbs, void* cuda_stream) {
    if (!gbs) return report_error(PGSGD_EINVAL, "gbs is NULL");
    if (bytes < (1u << 20) || bytes > (1ull << 30)) return report_error(PGSGD_EINVAL, "bytes must be in [1 MiB, 1 GiB]");
    if (reps == 0 || reps > 1000) return report_error(PGSGD_EINVAL, "reps must be in [1, 1000]");
    if (mode != 0 && mode != 1) return report_error(PGSGD_EINVAL, "mode must be 0 (streaming) or 1 (random)");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t n = bytes / 16;
    const int block = 256, grid = sms * 8;
    const uint32_t loads_per_thread = 256;
    uint4* buf = nullptr;
    uint32_t* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
        cudaFree(buf);
        cudaFree(out);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    cudaError_t e = cudaMalloc(&buf, n * 16);
    if (e == cudaSuccess) e = cudaMalloc(&out, (size_t)grid * block * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemsetAsync(buf, 1, n * 16, st);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cleanup();
        return report_error(PGSGD_ENOMEM, "L2 probe setup: %s", cudaGetErrorString(e));
    }
    float ms = 0.f;
    double moved = 0.0;
    for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {  // pass 0 warms L2
        e = cudaEventRecord(e0, st);
        if (mode == 0) {
            l2_stream_kernel<<<grid, block, 0, st>>>(buf, n, reps, out);
            moved = (double)n * 16.0 * reps;
        } else {
            for (uint32_t r = 0; r < reps; ++r) l2_random_kernel<<<grid, block, 0, st>>>(buf, n, loads_per_thread, out);
            moved = (double)grid * block * loads_per_thread * 32.0 * reps;  // one 32-byte sector per load
        }
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    cleanup();
    if (e != cudaSuccess) return report_error(PGSGD_ECUDA, "L2 probe: %s", cudaGetErrorString(e));
    *gbs = moved / (ms * 1e-3) / 1e9;
    return PGSGD_OK;
}
