// Measurement helpers; the layout never calls them.
// L2 read bandwidth of this GPU, the ceiling for graphs whose records fit in
// L2 (the 200 k-node workload: 3.5 MB of node records, 112 MB of step
// records). Two patterns over one L2-resident buffer: streaming 16-byte
// vector loads (each warp reads 512 contiguous bytes) and random 16-byte loads
// (one 32-byte sector each, as the update kernel's record reads).
// HBM random-read rate: random 16-byte loads from a multi-GB buffer in the
// pattern of the step-record reads of a chromosome-scale graph (7.5 GB of
// step records, far beyond L2), the ceiling for a kernel bound by them.
#include <algorithm>
#include <cstdint>

#include "../../include/pgsgd.h"
#include "pgsgd_internal.h"

namespace pgsgd {
namespace {

constexpr uint32_t kGatherPaths = 90;          // "paths" of the gather probe's buffer
constexpr uint32_t kGatherSmall = 5500000;     // node-sized array: 88 MB of 16-byte records

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

// Random reads from a buffer far larger than L2, in the pattern of the
// update and stress kernels on a large graph: the buffer is cut into 90
// equal "paths" of 16-byte records; unit Q picks path p = Q mod 90 and, from
// one Philox4x32-10 block of counter (Q / 90, 0, p, 0), two records i and j
// uniform on that path (mulhi64 of a 64-bit word), read with the step-record
// load (evict-first, 64-byte prefetch hint). mode 1 adds two random 8-byte
// reads per unit from a node-sized array (88 MB, evict-last, L2-resident), as
// an update's two point reads. Grid-stride over the units, one unit in
// flight per thread. Every index is below its array's length.
template <int MODE>
__global__ void __launch_bounds__(256, 4) hbm_gather_kernel(const StepRec* __restrict__ buf, uint64_t per_path,
                                                            const NodeRec* __restrict__ small, uint32_t n_small,
                                                            uint64_t units, uint32_t* out) {
    const uint64_t pol_stream = policy_evict_first(), pol_keep = policy_evict_last();
    const uint64_t nthr = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    uint32_t acc = 0;
    for (uint64_t Q = tid; Q < units; Q += nthr) {
        const uint32_t p = (uint32_t)(Q % kGatherPaths);
        const uint64_t q = Q / kGatherPaths;
        const uint4 w = philox4x32_10(make_uint4((uint32_t)q, (uint32_t)(q >> 32), p, 0u), 0x5EEDu, 0u);
        const uint64_t i = mulhi64((uint64_t)w.x | ((uint64_t)w.y << 32), per_path);
        const uint64_t j = mulhi64(((uint64_t)w.w << 32) | w.z, per_path);
        const StepRec a = load_step(buf + p * per_path + i, pol_stream, true);
        const StepRec b = load_step(buf + p * per_path + j, pol_stream, true);
        acc ^= a.nr ^ b.pos;
        if (MODE == 1) {
            const float2 va = load_point(small + (a.nr ^ w.z) % n_small, 0, pol_keep, true);
            const float2 vb = load_point(small + (b.nr ^ w.w) % n_small, 1, pol_keep, true);
            acc ^= __float_as_uint(va.x) ^ __float_as_uint(vb.y);
        }
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
    if (mode != 0 && mode != 1) return report_error(PGSGD_EINVAL, "mode must be 0 or 1");
    if (blocks_per_sm < 1 || blocks_per_sm > 64) return report_error(PGSGD_EINVAL, "blocks_per_sm must be in [1, 64]");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t per_path = bytes / 16 / kGatherPaths;  // records per path
    const uint64_t n = per_path * kGatherPaths;
    const uint32_t n_small = kGatherSmall;
    const int block = 256, grid = sms * blocks_per_sm;
    const uint64_t units = 4 * n;  // each record read about 8 times per launch
    StepRec* buf = nullptr;
    NodeRec* small = nullptr;
    uint32_t* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
        cudaFree(buf);
        cudaFree(small);
        cudaFree(out);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    cudaError_t e = cudaMalloc(&buf, n * sizeof(StepRec));
    if (e == cudaSuccess) e = cudaMalloc(&small, (size_t)n_small * sizeof(NodeRec));
    if (e == cudaSuccess) e = cudaMalloc(&out, (size_t)grid * block * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemsetAsync(buf, 1, n * sizeof(StepRec), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(small, 0, (size_t)n_small * sizeof(NodeRec), st);
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
            if (mode == 0) hbm_gather_kernel<0><<<grid, block, 0, st>>>(buf, per_path, small, n_small, units, out);
            else hbm_gather_kernel<1><<<grid, block, 0, st>>>(buf, per_path, small, n_small, units, out);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    cleanup();
    if (e != cudaSuccess) return report_error(PGSGD_ECUDA, "HBM gather probe: %s", cudaGetErrorString(e));
    *loads_per_s = 2.0 * (double)units * reps / (ms * 1e-3);  // the large buffer's random reads
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
