// Internal interface between the C ABI (pgsgd_api.cu) and the kernels
// (pgsgd_kernels.cu). Not installed; no torch types anywhere.
#pragma once

#include <cmath>
#include <cstdint>
#include <utility>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/pgsgd.h"

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

constexpr uint32_t kMaxPaths = 16384;       // single graph: path tables in shared memory
constexpr uint32_t kMaxBatchPaths = 1u << 22; // batch super graph: path tables in global memory

// Default cap on the updates of one graph in flight at once (the paper runs
// its updates concurrently without saying how many): max(64, V / 16, N / 5120)
// for V nodes and N updates per iteration. Concurrent updates read points that
// others are about to move and overwrite each other's moves (last writer
// wins); the excess stress over the sequential oracle grows with the share of
// nodes in motion at once and shrinks with the moves each node receives per
// iteration. Measured (paired by seed against the oracle): 1-12 k-node graphs
// of 4-12 paths 3.4 % above with 2048 in flight, 0.26 % at V / 16; 1-4 k-node
// graphs of 50-90 paths 1.95 % with 2048, 0.73 % at N / 1280, 0.19 % at
// N / 5120, 0.11 % at V / 16 (at 2x the time of N / 5120).
constexpr uint64_t kMinInFlight = 64;
inline uint64_t default_in_flight_cap(uint64_t n_nodes, uint64_t n_updates) {
    uint64_t c = n_nodes / 16;
    if (n_updates / 5120 > c) c = n_updates / 5120;
    return c > kMinInFlight ? c : kMinInFlight;
}

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
    bool pipeline;       // software-pipelined update loop
    bool wm;             // warp merging: one cooling coin per group of 32 updates
    int drf;             // data reuse factor (> 1: n_updates counts selections of drf updates)
    int async_depth;     // > 0: step-record reads of the next async_depth updates in flight (cp.async)
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
    int pf64;                   // 64-byte L2 prefetch hint: bit 0 step loads, bit 1 node loads
    int async_depth;            // > 0: step-record reads of the next async_depth samples in flight (cp.async)
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
int update_blocks_per_sm(const UpdateLaunch& L);  // resident blocks of the kernel L selects (0 on error)
cudaError_t launch_debug_sample_reuse(const SamplerArgs& s, uint32_t R, uint64_t n_sel, uint64_t q_begin,
                                     uint64_t count, void* out, int sm_count, cudaStream_t st);
cudaError_t launch_debug_sample(const SamplerArgs& s, uint64_t u_begin, uint64_t count, void* out,
                                int sm_count, cudaStream_t st);
cudaError_t launch_debug_sweep(const SamplerArgs& s, uint64_t u_begin, uint64_t count, const NodeRec* nodes,
                               float eta, float4* out, int sm_count, cudaStream_t st);
cudaError_t launch_stress(const StressLaunch& L, cudaStream_t st);
int stress_blocks_per_sm(const StressLaunch& L);
cudaError_t launch_stress_finalize(const double* partials, int n, double* out3, cudaStream_t st);

cudaError_t launch_dstress_forward(const SamplerArgs& s, const NodeRec* nodes, uint64_t n_pairs, double* partials,
                                   int grid, cudaStream_t st);
cudaError_t launch_dstress_backward(const SamplerArgs& s, const NodeRec* nodes, uint64_t n_pairs, float scale,
                                    float* grad, int sm_count, cudaStream_t st);
cudaError_t launch_pair_grad(const SamplerArgs& s, uint64_t u_begin, uint64_t count, const NodeRec* nodes,
                             float4* out, int sm_count, cudaStream_t st);

cudaError_t launch_full_stress(const StepRec* steps, const NodeRec* nodes, const uint64_t* path_off, uint32_t P,
                               uint64_t S, double* partials, int grid, cudaStream_t st);

}  // namespace pgsgd

// The state behind a pgsgd_graph handle (device arrays are owned).
struct pgsgd_graph {
    using NodeRec = pgsgd::NodeRec;
    using StepRec = pgsgd::StepRec;
    int device = 0;
    int sm_count = 0;
    uint32_t n_nodes = 0, n_paths = 0;
    uint64_t n_steps = 0;
    uint64_t max_path_steps = 0;
    int64_t max_path_nt = 0;
    std::vector<uint64_t> h_path_off;
    std::vector<int64_t> h_path_nt;    // nucleotide length of every path

    NodeRec* d_nodes = nullptr;
    int32_t* d_anchor = nullptr;       // [V] x anchors (master copy)
    StepRec* d_steps = nullptr;
    uint64_t* d_path_off = nullptr;
    uint64_t* d_sample_off = nullptr;  // stress sample offsets [P + 1]
    float* d_zipf_B = nullptr;
    float* d_zipf_T = nullptr;         // [kZipfTable] acceptance thresholds
    uint16_t* d_guide = nullptr;       // [n_guide + 1]
    uint32_t n_guide = 1, guide_shift = 0;
    uint32_t* d_flags = nullptr;
    uint32_t* d_changed = nullptr;     // set by a rebase that moved an anchor
    double* d_partials = nullptr;      // stress scratch [max_stress_blocks][3] + 3 totals
    double* d_per_path = nullptr;      // [P][3]
    double* d_xy = nullptr;            // coordinate staging [V][4]
    void* d_debug = nullptr;           // debug output staging
    size_t debug_bytes = 0;
    int max_stress_blocks = 0;
    uint64_t stress_samples_per_step = 0;

    bool has_coords = false;
    float zipf_theta = NAN;

    // options
    int coord_mode = 0;
    int updates_per_step = 10;
    int block = 256;
    int blocks_per_sm = 32;
    int upt = 0;          // 0 = automatic (2 with the pipelined loop, else 1)
    int atomic = 0;
    int rebase = 1;
    int timing = 0;
    int64_t max_concurrent = -1;  // -1 = automatic
    int min_blocks = 0;   // 0 = automatic register budget (plain loop: 4 blocks per SM at 1 update per thread, 3 at 2)
    int l2_fetch = 0;
    int store_mode = 1;  // 64-bit atomic exchange: measured fastest replace-store
    int l2_hints = 1;
    int pf64 = 7;
    int pipeline = -1;    // -1 = automatic (the pipelined loop for the plain method)
    int warp_merge = 0;
    int async_depth = 0;  // cp.async step-record ring depth of the update kernel (0 = off)
    int stress_async = 0; // the same for the sampled-stress kernel
    int stress_waves = 1; // stress grid: whole waves of resident blocks (0 = 8 blocks per SM)
    int drf = 1;          // data reuse factor
    int srf = 1;          // step reduction factor

    // timing
    std::vector<cudaEvent_t> ev_free;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending;
    double timing_ms = 0.0;
    uint64_t timing_launches = 0, timing_updates = 0;

    uint64_t device_bytes = 0;
};

namespace pgsgd {

int graph_create(const uint32_t* node_len, uint32_t n_nodes, const uint64_t* path_off, uint32_t n_paths,
                 const uint32_t* step_node, const uint8_t* step_rev, const int64_t* step_pos, int on_device,
                 void* cuda_stream, bool batch, pgsgd_graph** out);
void free_graph(pgsgd_graph* g);
int ensure_zipf(pgsgd_graph* g, float theta, cudaStream_t st);

// Record the calling thread's error message (read by pgsgd_last_error) and
// return status.
int report_error(int status, const char* fmt, ...);

}  // namespace pgsgd
