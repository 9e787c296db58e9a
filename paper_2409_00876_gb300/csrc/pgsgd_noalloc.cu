// pgsgd_stress_noalloc: the sampled path stress computed without any device
// allocation, for callers that cannot call cudaMalloc (see include/pgsgd.h).
//
// The per-block partial sums that pgsgd_stress keeps in a per-handle device
// buffer live here in one file-scope __device__ array instead. Every GPU that
// loads the library holds that array (96 KiB) until the process exits,
// and every call on a device shares it: calls whose work overlaps on the GPU
// race on it. Each call's blocks write every slot its final reduction reads,
// so nothing has to be cleared between calls.
#include "../../include/pgsgd.h"
#include "pgsgd_internal.h"

namespace pgsgd {
namespace {

constexpr int kNoAllocBlocks = 4096;               // partial-sum slots
constexpr uint32_t kNoAllocMaxPaths = 8192;        // path and sample tables in shared memory
constexpr int kNoAllocSlots = 3 * kNoAllocBlocks + 2;  // + sample count of the call

// Scratch: [block][3] = (sum of terms, sum of squared terms, valid samples),
// then the call's total number of samples at [3 * kNoAllocBlocks].
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocSlots];

// In host code g_noalloc_scratch names a host-side shadow, not device memory:
// every call looks up its device address on the current device. Nothing is
// cached, so a call stays valid after cudaDeviceReset or on a new primary
// context, where the module (and the array) may load at another address.

__global__ void stress_noalloc_kernel(const uint32_t* __restrict__ node_len,
                                      const uint64_t* __restrict__ path_off, uint32_t P,
                                      const uint32_t* __restrict__ step_node,
                                      const uint8_t* __restrict__ step_rev,
                                      const int64_t* __restrict__ step_pos,
                                      const double* __restrict__ xy, uint32_t per_step,
                                      uint32_t key0, uint32_t key1, double* scratch) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* s_poff = reinterpret_cast<uint64_t*>(smem);  // [P + 1]
    uint64_t* s_soff = s_poff + P + 1;                     // [P + 1]
    __shared__ uint64_t chunk[256];
    for (uint32_t k = threadIdx.x; k <= P; k += blockDim.x) s_poff[k] = path_off[k];
    __syncthreads();
    // sample offsets: per_step * n_p samples for every path with n_p >= 2
    const uint32_t per_thr = (P + blockDim.x - 1) / blockDim.x;
    const uint32_t a0 = threadIdx.x * per_thr, a1 = min(P, a0 + per_thr);
    uint64_t local = 0;
    for (uint32_t p = a0; p < a1; ++p) {
        const uint64_t n = s_poff[p + 1] - s_poff[p];
        local += n >= 2 ? (uint64_t)per_step * n : 0;
    }
    chunk[threadIdx.x] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t run = 0;
        for (uint32_t t = 0; t < blockDim.x; ++t) {
            const uint64_t c = chunk[t];
            chunk[t] = run;
            run += c;
        }
        s_soff[P] = run;
    }
    __syncthreads();
    uint64_t run = chunk[threadIdx.x];
    for (uint32_t p = a0; p < a1; ++p) {
        s_soff[p] = run;
        const uint64_t n = s_poff[p + 1] - s_poff[p];
        run += n >= 2 ? (uint64_t)per_step * n : 0;
    }
    __syncthreads();
    const uint64_t n_samples = s_soff[P];
    if (blockIdx.x == 0 && threadIdx.x == 0) scratch[3 * kNoAllocBlocks] = (double)n_samples;

    double sum = 0.0, sq = 0.0, cnt = 0.0;
    for (uint64_t Q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; Q < n_samples;
         Q += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t p = find_path(s_soff, P, Q);
        const uint64_t q = Q - s_soff[p];
        const uint64_t off = s_poff[p];
        const uint64_t n = s_poff[p + 1] - off;
        const uint32_t c2 = 0x80000000u | p;
        const uint4 w = philox4x32_10(make_uint4((uint32_t)q, (uint32_t)(q >> 32), c2, 0u), key0, key1);
        const uint64_t i = off + mulhi64((uint64_t)w.x | ((uint64_t)w.y << 32), n);
        const uint64_t x = mulhi64(((uint64_t)w.w << 32) | (w.z & ~15u), n - 1);
        const uint64_t j = off + x + (x >= i - off);
        const uint32_t ei = w.z & 1u, ej = (w.z >> 1) & 1u;
        const uint32_t ni = step_node[i], nj = step_node[j];
        const int64_t pa = step_pos[i] + (((ei ^ step_rev[i]) & 1u) ? (int64_t)node_len[ni] : 0);
        const int64_t pb = step_pos[j] + (((ej ^ step_rev[j]) & 1u) ? (int64_t)node_len[nj] : 0);
        const int64_t d = pa > pb ? pa - pb : pb - pa;
        if (d == 0) continue;
        const float dx = (float)(xy[4 * (uint64_t)ni + 2 * ei] - xy[4 * (uint64_t)nj + 2 * ej]);
        const float dy = (float)(xy[4 * (uint64_t)ni + 2 * ei + 1] - xy[4 * (uint64_t)nj + 2 * ej + 1]);
        const float df = __ll2float_rn(d);
        const float t = (sqrtf(dx * dx + dy * dy) - df) / df;
        const float term = t * t;
        sum += (double)term;
        sq += (double)term * (double)term;
        cnt += 1.0;
    }
    __shared__ double red[3][32];
    for (int o = 16; o > 0; o >>= 1) {
        sum += __shfl_down_sync(0xffffffffu, sum, o);
        sq += __shfl_down_sync(0xffffffffu, sq, o);
        cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { red[0][warp] = sum; red[1][warp] = sq; red[2][warp] = cnt; }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        sum = lane < nw ? red[0][lane] : 0.0;
        sq = lane < nw ? red[1][lane] : 0.0;
        cnt = lane < nw ? red[2][lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            sum += __shfl_down_sync(0xffffffffu, sum, o);
            sq += __shfl_down_sync(0xffffffffu, sq, o);
            cnt += __shfl_down_sync(0xffffffffu, cnt, o);
        }
        if (lane == 0) {
            scratch[3 * blockIdx.x] = sum;
            scratch[3 * blockIdx.x + 1] = sq;
            scratch[3 * blockIdx.x + 2] = cnt;
        }
    }
}

// One block: sum the grid's partials in a fixed order and write the result.
__global__ void stress_noalloc_finalize(const double* __restrict__ scratch, int n_blocks,
                                        pgsgd_stress_result* out) {
    __shared__ double red[3][256];
    double s = 0.0, q = 0.0, c = 0.0;
    for (int b = threadIdx.x; b < n_blocks; b += blockDim.x) {
        s += scratch[3 * b];
        q += scratch[3 * b + 1];
        c += scratch[3 * b + 2];
    }
    red[0][threadIdx.x] = s; red[1][threadIdx.x] = q; red[2][threadIdx.x] = c;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            red[0][threadIdx.x] += red[0][threadIdx.x + w];
            red[1][threadIdx.x] += red[1][threadIdx.x + w];
            red[2][threadIdx.x] += red[2][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double n = red[2][0];
        const double mean = n > 0 ? red[0][0] / n : 0.0;
        const double var = n > 1 ? fmax(0.0, (red[1][0] - n * mean * mean) / (n - 1.0)) : 0.0;
        const double sd = sqrt(var);
        const double half = n > 0 ? 1.96 * sd / sqrt(n) : 0.0;
        pgsgd_stress_result r;
        r.mean = mean;
        r.stddev = sd;
        r.ci_lo = mean - half;
        r.ci_hi = mean + half;
        r.n_valid = (uint64_t)n;
        r.n_skipped = (uint64_t)scratch[3 * kNoAllocBlocks] - (uint64_t)n;
        *out = r;
    }
}

}  // namespace
}  // namespace pgsgd

using namespace pgsgd;

extern "C" int pgsgd_stress_noalloc(const uint32_t* node_len, uint32_t n_nodes, const uint64_t* path_off,
                                    uint32_t n_paths, const uint32_t* step_node, const uint8_t* step_rev,
                                    const int64_t* step_pos, const double* xy, uint32_t samples_per_step,
                                    uint64_t seed, pgsgd_stress_result* out, void* cuda_stream) {
    if (!node_len || !path_off || !step_node || !step_rev || !step_pos || !xy || !out)
        return report_error(PGSGD_EINVAL, "pgsgd_stress_noalloc: a required pointer is NULL");
    if (n_nodes == 0 || n_paths == 0 || samples_per_step == 0)
        return report_error(PGSGD_EINVAL, "pgsgd_stress_noalloc: n_nodes, n_paths and samples_per_step must be > 0");
    if (n_paths > kNoAllocMaxPaths)
        return report_error(PGSGD_ERANGE,
                            "pgsgd_stress_noalloc: n_paths %u exceeds its maximum of %u (the path tables live in "
                            "shared memory)", n_paths, kNoAllocMaxPaths);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
        return report_error(PGSGD_ECUDA, "pgsgd_stress_noalloc: device query: %s", cudaGetErrorString(e));
    // with the caller's device current: the array's device address on it, and
    // the kernel's shared-memory limit (host calls that allocate nothing)
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
        return report_error(PGSGD_ECUDA, "pgsgd_stress_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    double* scratch = static_cast<double*>(p);
    const size_t max_smem = 2 * (size_t)(kNoAllocMaxPaths + 1) * sizeof(uint64_t);
    e = cudaFuncSetAttribute(stress_noalloc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_smem);
    if (e != cudaSuccess)
        return report_error(PGSGD_ECUDA, "pgsgd_stress_noalloc: shared memory attribute: %s", cudaGetErrorString(e));
    int grid = sms * 8;
    if (grid > kNoAllocBlocks) grid = kNoAllocBlocks;  // never more partials than the array holds
    if (grid < 1) grid = 1;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const size_t smem = 2 * (size_t)(n_paths + 1) * sizeof(uint64_t);
    stress_noalloc_kernel<<<grid, 256, smem, st>>>(node_len, path_off, n_paths, step_node, step_rev, step_pos,
                                                   xy, samples_per_step, (uint32_t)seed,
                                                   (uint32_t)(seed >> 32), scratch);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        stress_noalloc_finalize<<<1, 256, 0, st>>>(scratch, grid, out);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return report_error(PGSGD_ECUDA, "pgsgd_stress_noalloc: launch: %s", cudaGetErrorString(e));
    return PGSGD_OK;
}
