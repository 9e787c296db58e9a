// Differentiable sampled path stress: the forward value and a hand-written
// backward kernel for d(stress)/d(layout), plus a debug kernel that exposes
// the gradient of single update pairs.
//
// The objective is Eq. 2's estimator (Section VI-B) over a fixed set of
// n_pairs samples: sample q draws counter (q_lo, q_hi, 0xC0000000, 0); the
// global step g picks the path in proportion to |p| and step i uniformly; the
// partner j is uniform among the other steps (w3 and the upper 28 bits of w2);
// bits 0 and 1 of w2 pick the endpoints. Samples on paths with fewer than two
// steps or with d_ref = 0 are left out.
//   F = (1 / n_valid) sum_q t_q^2,  t_q = (|v_i - v_j| - d) / d
//   dF/dv_i = (2 / n_valid) t_q (v_i - v_j) / (d |v_i - v_j|),  dF/dv_j = -dF/dv_i
#include "../../include/pgsgd.h"
#include "pgsgd_internal.h"

namespace pgsgd {
namespace {

struct DPair {
    uint64_t gi, gj;
    uint32_t ei, ej;
    bool valid;
};

__device__ __forceinline__ DPair dstress_pair(const SamplerArgs& a, const PathTable& pt, uint64_t q) {
    DPair r;
    const uint4 w = philox4x32_10(make_uint4((uint32_t)q, (uint32_t)(q >> 32), 0xC0000000u, 0u), a.key0, a.key1);
    const uint64_t g = mulhi64((uint64_t)w.x | ((uint64_t)w.y << 32), a.n_steps);
    const uint32_t p = find_path_guided(pt, g);
    const uint64_t off = pt.off[p], n = pt.off[p + 1] - off;
    r.valid = n >= 2;
    const uint64_t i = g - off;
    const uint64_t x = r.valid ? mulhi64(((uint64_t)w.w << 32) | (w.z & ~15u), n - 1) : 0;
    r.gi = off + i;
    r.gj = off + x + (x >= i);
    r.ei = w.z & 1u;
    r.ej = (w.z >> 1) & 1u;
    return r;
}

// FP32 difference v_i - v_j of two endpoints, x anchors differenced in integers.
__device__ __forceinline__ void endpoint_delta(const NodeRec& a, int32_t axa, uint32_t ea, const NodeRec& b,
                                               int32_t axb, uint32_t eb, float& dx, float& dy) {
    const float xa = ea ? a.ex : a.sx, ya = ea ? a.ey : a.sy;
    const float xb = eb ? b.ex : b.sx, yb = eb ? b.ey : b.sy;
    dx = __ll2float_rn((int64_t)axa - (int64_t)axb) + (xa - xb);
    dy = ya - yb;
}

__global__ void dstress_forward_kernel(SamplerArgs a0, const NodeRec* __restrict__ nodes, uint64_t n_pairs,
                                       double* __restrict__ partials) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ZipfConsts zc;
    const PathTable pt = stage_paths(a0, smem, zc);
    const uint64_t pol_stream = policy_evict_first(), pol_keep = policy_evict_last();
    double sum = 0.0, cnt = 0.0;
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < n_pairs;
         q += (uint64_t)gridDim.x * blockDim.x) {
        const DPair r = dstress_pair(a0, pt, q);
        if (!r.valid) continue;
        const StepRec si = load_step(a0.steps + r.gi, pol_stream), sj = load_step(a0.steps + r.gj, pol_stream);
        const int64_t pa = endpoint_pos(si, r.ei), pb = endpoint_pos(sj, r.ej);
        const int64_t d = pa > pb ? pa - pb : pb - pa;
        if (d == 0) continue;
        const NodeRec na = load_node(nodes + step_node(si), pol_keep), nb = load_node(nodes + step_node(sj), pol_keep);
        float dx, dy;
        endpoint_delta(na, si.ax, r.ei, nb, sj.ax, r.ej, dx, dy);
        const float df = __ll2float_rn(d);
        const float t = (sqrtf(dx * dx + dy * dy) - df) / df;
        sum += (double)(t * t);
        cnt += 1.0;
    }
    __shared__ double red[2][32];
    for (int o = 16; o > 0; o >>= 1) {
        sum += __shfl_down_sync(0xffffffffu, sum, o);
        cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { red[0][warp] = sum; red[1][warp] = cnt; }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        sum = lane < nw ? red[0][lane] : 0.0;
        cnt = lane < nw ? red[1][lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            sum += __shfl_down_sync(0xffffffffu, sum, o);
            cnt += __shfl_down_sync(0xffffffffu, cnt, o);
        }
        if (lane == 0) {
            // the third slot stays 0 so the stress finalize kernel can sum these
            partials[3 * (uint64_t)blockIdx.x] = sum;
            partials[3 * (uint64_t)blockIdx.x + 1] = 0.0;
            partials[3 * (uint64_t)blockIdx.x + 2] = cnt;
        }
    }
}

// grad[v] (FP32 [4]) += scale * d(t_q^2)/d(endpoints) for every valid sample;
// grad must be zero on entry. Vector atomic adds of the two 2-D contributions.
__global__ void dstress_backward_kernel(SamplerArgs a0, const NodeRec* __restrict__ nodes, uint64_t n_pairs,
                                        float scale, float* __restrict__ grad) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ZipfConsts zc;
    const PathTable pt = stage_paths(a0, smem, zc);
    const uint64_t pol_stream = policy_evict_first(), pol_keep = policy_evict_last();
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < n_pairs;
         q += (uint64_t)gridDim.x * blockDim.x) {
        const DPair r = dstress_pair(a0, pt, q);
        if (!r.valid) continue;
        const StepRec si = load_step(a0.steps + r.gi, pol_stream), sj = load_step(a0.steps + r.gj, pol_stream);
        const int64_t pa = endpoint_pos(si, r.ei), pb = endpoint_pos(sj, r.ej);
        const int64_t d = pa > pb ? pa - pb : pb - pa;
        if (d == 0) continue;
        const NodeRec na = load_node(nodes + step_node(si), pol_keep), nb = load_node(nodes + step_node(sj), pol_keep);
        float dx, dy;
        endpoint_delta(na, si.ax, r.ei, nb, sj.ax, r.ej, dx, dy);
        const float mag = sqrtf(dx * dx + dy * dy);
        if (!(mag > 0.0f)) continue;
        const float df = __ll2float_rn(d);
        const float t = (mag - df) / df;
        const float c = scale * 2.0f * t / (df * mag);
        float* gi = grad + 4 * (uint64_t)step_node(si) + 2 * r.ei;
        float* gj = grad + 4 * (uint64_t)step_node(sj) + 2 * r.ej;
        atomicAdd(reinterpret_cast<float2*>(gi), make_float2(c * dx, c * dy));
        atomicAdd(reinterpret_cast<float2*>(gj), make_float2(-c * dx, -c * dy));
    }
}

// Gradient of the single-pair stress ((|v_i - v_j| - d) / d)^2 of every update
// u in [u_begin, u_begin + count) of iteration t: out[q] = (d/dv_i, d/dv_j).
__global__ void pair_grad_kernel(SamplerArgs a0, uint64_t u_begin, uint64_t count,
                                 const NodeRec* __restrict__ nodes, float4* out) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ZipfConsts zc;
    const PathTable pt = stage_paths(a0, smem, zc);
    SamplerArgs a = a0;
    a.zc = zc;
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < count;
         q += (uint64_t)gridDim.x * blockDim.x) {
        const Pair pr = draw_pair(a, pt, u_begin + q);
        float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
        if (!pr.short_path) {
            const StepRec si = a.steps[pr.base + pr.i], sj = a.steps[pr.base + pr.j];
            const NodeRec na = nodes[step_node(si)], nb = nodes[step_node(sj)];
            const uint32_t ea = (pr.w2 >> 2) & 1u, eb = (pr.w2 >> 3) & 1u;
            const int64_t pa = endpoint_pos(si, ea), pb = endpoint_pos(sj, eb);
            const int64_t d = pa > pb ? pa - pb : pb - pa;
            if (d != 0) {
                float dx, dy;
                endpoint_delta(na, si.ax, ea, nb, sj.ax, eb, dx, dy);
                const float mag = sqrtf(dx * dx + dy * dy);
                if (mag > 0.0f) {
                    const float df = __ll2float_rn(d);
                    const float c = 2.0f * ((mag - df) / df) / (df * mag);
                    o = make_float4(c * dx, c * dy, -c * dx, -c * dy);
                }
            }
        }
        out[q] = o;
    }
}

int grid_for_pairs(uint64_t work, int sm_count, int per_sm) {
    uint64_t g = (work + 255) / 256;
    const uint64_t cap = (uint64_t)sm_count * per_sm;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

template <class K>
cudaError_t set_smem(K kernel, size_t smem) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

}  // namespace

cudaError_t launch_dstress_forward(const SamplerArgs& s, const NodeRec* nodes, uint64_t n_pairs, double* partials,
                                   int grid, cudaStream_t st) {
    const size_t smem = update_smem_bytes(s.n_paths, s.n_guide);
    cudaError_t e = set_smem(dstress_forward_kernel, smem);
    if (e != cudaSuccess) return e;
    dstress_forward_kernel<<<grid, 256, smem, st>>>(s, nodes, n_pairs, partials);
    return cudaGetLastError();
}

cudaError_t launch_dstress_backward(const SamplerArgs& s, const NodeRec* nodes, uint64_t n_pairs, float scale,
                                    float* grad, int sm_count, cudaStream_t st) {
    if (n_pairs == 0) return cudaSuccess;
    const size_t smem = update_smem_bytes(s.n_paths, s.n_guide);
    cudaError_t e = set_smem(dstress_backward_kernel, smem);
    if (e != cudaSuccess) return e;
    dstress_backward_kernel<<<grid_for_pairs(n_pairs, sm_count, 16), 256, smem, st>>>(s, nodes, n_pairs, scale,
                                                                                     grad);
    return cudaGetLastError();
}

cudaError_t launch_pair_grad(const SamplerArgs& s, uint64_t u_begin, uint64_t count, const NodeRec* nodes,
                             float4* out, int sm_count, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    const size_t smem = update_smem_bytes(s.n_paths, s.n_guide);
    cudaError_t e = set_smem(pair_grad_kernel, smem);
    if (e != cudaSuccess) return e;
    pair_grad_kernel<<<grid_for_pairs(count, sm_count, 8), 256, smem, st>>>(s, u_begin, count, nodes, out);
    return cudaGetLastError();
}

}  // namespace pgsgd
