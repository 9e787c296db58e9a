// Path stress (Eq. 1, Section VI-A) over every pair of distinct steps of every
// path: the mean over the pair's four endpoint combinations with d_ref > 0,
// averaged over the pairs that have at least one. O(sum n_p^2) work: a warp
// takes one row (path p, step i) and its lanes stride over the steps j > i.
#include "../../include/pgsgd.h"
#include "pgsgd_internal.h"

namespace pgsgd {
namespace {

__global__ void full_stress_kernel(const StepRec* __restrict__ steps, const NodeRec* __restrict__ nodes,
                                   const uint64_t* __restrict__ path_off, uint32_t P, uint64_t S,
                                   double* __restrict__ partials) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* s_off = reinterpret_cast<uint64_t*>(smem);
    for (uint32_t k = threadIdx.x; k <= P; k += blockDim.x) s_off[k] = path_off[k];
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    double sum = 0.0, pairs = 0.0;
    for (uint64_t row = warp; row < S; row += n_warps) {
        const uint32_t p = find_path(s_off, P, row);
        const uint64_t end = s_off[p + 1];
        const StepRec si = steps[row];
        const NodeRec a = nodes[step_node(si)];
        for (uint64_t col = row + 1 + lane; col < end; col += 32) {
            const StepRec sj = steps[col];
            const NodeRec b = nodes[step_node(sj)];
            float acc = 0.0f;
            int valid = 0;
#pragma unroll
            for (uint32_t e = 0; e < 4; ++e) {
                const uint32_t ea = e >> 1, eb = e & 1u;
                const int64_t pa = endpoint_pos(si, ea), pb = endpoint_pos(sj, eb);
                const int64_t d = pa > pb ? pa - pb : pb - pa;
                if (d == 0) continue;
                const float xa = ea ? a.ex : a.sx, ya = ea ? a.ey : a.sy;
                const float xb = eb ? b.ex : b.sx, yb = eb ? b.ey : b.sy;
                const float dx = __ll2float_rn((int64_t)si.ax - (int64_t)sj.ax) + (xa - xb);
                const float dy = ya - yb;
                const float df = __ll2float_rn(d);
                const float t = (sqrtf(dx * dx + dy * dy) - df) / df;
                acc += t * t;
                ++valid;
            }
            if (valid) {
                sum += (double)(acc / (float)valid);
                pairs += 1.0;
            }
        }
    }
    __shared__ double red[2][32];
    for (int o = 16; o > 0; o >>= 1) {
        sum += __shfl_down_sync(0xffffffffu, sum, o);
        pairs += __shfl_down_sync(0xffffffffu, pairs, o);
    }
    const int wid = threadIdx.x >> 5;
    if (lane == 0) { red[0][wid] = sum; red[1][wid] = pairs; }
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        sum = lane < nw ? red[0][lane] : 0.0;
        pairs = lane < nw ? red[1][lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            sum += __shfl_down_sync(0xffffffffu, sum, o);
            pairs += __shfl_down_sync(0xffffffffu, pairs, o);
        }
        if (lane == 0) {
            partials[3 * (uint64_t)blockIdx.x] = sum;
            partials[3 * (uint64_t)blockIdx.x + 1] = 0.0;
            partials[3 * (uint64_t)blockIdx.x + 2] = pairs;
        }
    }
}

}  // namespace

cudaError_t launch_full_stress(const StepRec* steps, const NodeRec* nodes, const uint64_t* path_off, uint32_t P,
                               uint64_t S, double* partials, int grid, cudaStream_t st) {
    const size_t smem = (size_t)(P + 1) * sizeof(uint64_t);
    cudaError_t e = cudaFuncSetAttribute(full_stress_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    full_stress_kernel<<<grid, 256, smem, st>>>(steps, nodes, path_off, P, S, partials);
    return cudaGetLastError();
}

}  // namespace pgsgd
