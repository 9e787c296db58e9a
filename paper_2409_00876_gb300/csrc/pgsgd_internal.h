// Internal interface between the C ABI (pgsgd_api.cu) and the kernels
// (pgsgd_kernels.cu). Not installed; no torch types anywhere.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "pgsgd_device.cuh"

namespace pgsgd {

// Error bits a device kernel may raise in the graph's flag word.
enum : uint32_t {
    FLAG_BAD_NODE = 1u << 0,   // step node id >= n_nodes
    FLAG_BAD_REV = 1u << 1,    // orientation not 0/1
    FLAG_BAD_POS = 1u << 2,    // positions not consistent with node lengths
    FLAG_POS_RANGE = 1u << 3,  // position outside [0, 2^32)
    FLAG_ZERO_LEN = 1u << 4,   // node length 0
    FLAG_COORD_RANGE = 1u << 5,  // coordinate too large for the anchored form
    FLAG_COORD_NAN = 1u << 6,    // coordinate not finite
};

constexpr uint32_t kMaxPaths = 16384;

struct UpdateLaunch {
    SamplerArgs s;
    NodeRec* nodes;
    uint64_t u_begin;    // first update index
    uint64_t n_updates;  // updates in this launch
    float eta;
    int block, grid, upt, minb;
    int store_mode;      // 0 = plain store, 1 = 64-bit atomic exchange
    bool l2_hints;       // evict-first step records, evict-last node records
    int pf64;            // 64-byte L2 prefetch hint: bit 0 step loads, bit 1 node loads
    bool atomic;
};

struct StressLaunch {
    const StepRec* steps;
    const uint64_t* path_off;   // [P + 1]
    const uint64_t* sample_off; // [P + 1] first sample index of every path
    const NodeRec* nodes;
    uint64_t n_samples;
    uint32_t n_paths;
    uint32_t key0, key1;
    double* partials;           // [grid][3]
    double* per_path;           // [P][3] or nullptr
    int block, grid;
};

// Shared memory of the staged path tables (offsets, Zipf thresholds, Zipf B, guide).
__host__ __device__ inline size_t update_smem_bytes(uint32_t n_paths, uint32_t n_guide) {
    return (size_t)(n_paths + 1) * sizeof(uint64_t) + (size_t)(kZipfTable + n_paths) * sizeof(float) +
           (size_t)(n_guide + 1) * sizeof(uint16_t);
}
size_t stress_smem_bytes(uint32_t n_paths);

cudaError_t launch_check_lengths(const uint32_t* node_len, uint32_t n, uint32_t* flags, int sm_count,
                                 cudaStream_t st);
cudaError_t launch_pack_steps(const uint32_t* step_node, const uint8_t* step_rev, const int64_t* step_pos,
                              const uint32_t* node_len, uint32_t n_nodes, const uint64_t* path_off,
                              uint32_t n_paths, uint64_t n_steps, StepRec* steps, uint32_t* flags,
                              int sm_count, cudaStream_t st);
cudaError_t launch_path_extent(const StepRec* steps, const uint64_t* path_off, uint32_t n_paths,
                               int64_t* out_nt, cudaStream_t st);
cudaError_t launch_set_coords(const double* xy, NodeRec* nodes, int32_t* anchor, uint32_t n, int anchored,
                              uint32_t* flags, int sm_count, cudaStream_t st);
cudaError_t launch_get_coords(const NodeRec* nodes, const int32_t* anchor, double* xy, uint32_t n,
                              int sm_count, cudaStream_t st);
cudaError_t launch_rebase(NodeRec* nodes, int32_t* anchor, uint32_t n, uint32_t* changed, int sm_count,
                          cudaStream_t st);
cudaError_t launch_refresh_anchors(StepRec* steps, const int32_t* anchor, uint64_t n_steps,
                                   const uint32_t* changed, int sm_count, cudaStream_t st);
cudaError_t launch_zipf_setup(const uint64_t* path_off, uint32_t n_paths, float theta, float* zipf_B,
                              float* zipf_T, cudaStream_t st);
cudaError_t launch_update(const UpdateLaunch& L, cudaStream_t st);
cudaError_t launch_debug_sample(const SamplerArgs& s, uint64_t u_begin, uint64_t count, void* out,
                                int sm_count, cudaStream_t st);
cudaError_t launch_debug_sweep(const SamplerArgs& s, uint64_t u_begin, uint64_t count, const NodeRec* nodes,
                               float eta, float4* out, int sm_count, cudaStream_t st);
cudaError_t launch_stress(const StressLaunch& L, cudaStream_t st);
cudaError_t launch_stress_finalize(const double* partials, int n, double* out3, cudaStream_t st);

cudaError_t launch_dstress_forward(const SamplerArgs& s, const NodeRec* nodes, uint64_t n_pairs, double* partials,
                                   int grid, cudaStream_t st);
cudaError_t launch_dstress_backward(const SamplerArgs& s, const NodeRec* nodes, uint64_t n_pairs, float scale,
                                    float* grad, int sm_count, cudaStream_t st);
cudaError_t launch_pair_grad(const SamplerArgs& s, uint64_t u_begin, uint64_t count, const NodeRec* nodes,
                             float4* out, int sm_count, cudaStream_t st);

cudaError_t launch_full_stress(const StepRec* steps, const NodeRec* nodes, const uint64_t* path_off, uint32_t P,
                               uint64_t S, double* partials, int grid, cudaStream_t st);

// Record the calling thread's error message (read by pgsgd_last_error) and
// return status.
int report_error(int status, const char* fmt, ...);

}  // namespace pgsgd
