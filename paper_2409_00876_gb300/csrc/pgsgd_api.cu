// C ABI of libpgsgd.so (declared in include/pgsgd.h): graph handle,
// validation, device memory ownership, the iteration loop of Algorithm 1
// and the sampled-stress reduction. Host code only; kernels live in
// pgsgd_kernels.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/pgsgd.h"
#include "pgsgd_internal.h"

using namespace pgsgd;


namespace {

thread_local std::string g_last_error;

int fail(int status, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return status;
}

}  // namespace

int pgsgd::report_error(int status, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return status;
}

namespace {

int cuda_fail(cudaError_t e, const char* what) {
    return fail(e == cudaErrorMemoryAllocation ? PGSGD_ENOMEM : PGSGD_ECUDA, "%s: %s (%s)", what,
                cudaGetErrorString(e), cudaGetErrorName(e));
}

#define CK(call, what)                                       \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);   \
    } while (0)

cudaStream_t S(void* s) { return static_cast<cudaStream_t>(s); }

template <class T>
cudaError_t dalloc(pgsgd_graph* g, T** p, size_t count) {
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
    if (e == cudaSuccess) g->device_bytes += count * sizeof(T);
    return e;
}

}  // namespace

void pgsgd::free_graph(pgsgd_graph* g) {
    if (!g) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(g->device);
    cudaFree(g->d_nodes);
    cudaFree(g->d_anchor);
    cudaFree(g->d_changed);
    cudaFree(g->d_steps);
    cudaFree(g->d_path_off);
    cudaFree(g->d_sample_off);
    cudaFree(g->d_zipf_B);
    cudaFree(g->d_zipf_T);
    cudaFree(g->d_guide);
    cudaFree(g->d_flags);
    cudaFree(g->d_partials);
    cudaFree(g->d_per_path);
    cudaFree(g->d_xy);
    cudaFree(g->d_debug);
    for (auto& pr : g->ev_pending) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    for (auto e : g->ev_free) cudaEventDestroy(e);
    if (prev >= 0) cudaSetDevice(prev);
    delete g;
}

namespace {

const char* flag_text(uint32_t f) {
    if (f & FLAG_BAD_NODE) return "a step's node id is >= n_nodes";
    if (f & FLAG_BAD_REV) return "a step's orientation is not 0 or 1";
    if (f & FLAG_ZERO_LEN) return "a node has length 0";
    if (f & FLAG_BAD_POS) return "step positions do not start at 0 or do not advance by node length";
    if (f & FLAG_COORD_NAN) return "a coordinate is not finite";
    return "unknown";
}

// Read and clear the device flag word.
int check_flags(pgsgd_graph* g, cudaStream_t st, const char* what) {
    uint32_t f = 0;
    CK(cudaMemcpyAsync(&f, g->d_flags, sizeof f, cudaMemcpyDeviceToHost, st), "flag readback");
    CK(cudaStreamSynchronize(st), "flag sync");
    if (f) {
        CK(cudaMemsetAsync(g->d_flags, 0, sizeof(uint32_t), st), "flag clear");
        CK(cudaStreamSynchronize(st), "flag clear sync");
        if (f & (FLAG_POS_RANGE | FLAG_COORD_RANGE))
            return fail(PGSGD_ERANGE, "%s: %s", what,
                        (f & FLAG_POS_RANGE) ? "a step position is outside [0, 2^32)"
                                             : "a coordinate magnitude is >= 2^30 (anchored mode)");
        return fail(PGSGD_EINVAL, "%s: %s", what, flag_text(f));
    }
    return PGSGD_OK;
}

}  // namespace

int pgsgd::ensure_zipf(pgsgd_graph* g, float theta, cudaStream_t st) {
    if (g->zipf_theta == theta) return PGSGD_OK;
    CK(launch_zipf_setup(g->d_path_off, g->n_paths, theta, g->d_zipf_B, g->d_zipf_T, st), "zipf setup");
    g->zipf_theta = theta;
    return PGSGD_OK;
}

namespace {

SamplerArgs sampler_args(const pgsgd_graph* g, uint32_t T, uint32_t t, float theta, uint64_t seed) {
    SamplerArgs a;
    a.steps = g->d_steps;
    a.path_off = g->d_path_off;
    a.zipf_B = g->d_zipf_B;
    a.zipf_T = g->d_zipf_T;
    a.guide = g->d_guide;
    a.n_guide = g->n_guide;
    a.guide_shift = g->guide_shift;
    a.n_steps = g->n_steps;
    a.n_paths = g->n_paths;
    a.T = T;
    a.t = t;
    a.key0 = (uint32_t)seed;
    a.key1 = (uint32_t)(seed >> 32);
    a.wm = g->warp_merge ? 1u : 0u;
    a.zc.theta = theta;
    a.zc.omt = a.zc.A = a.zc.s = 0.0f;
    return a;
}

int ensure_debug(pgsgd_graph* g, size_t bytes) {
    if (g->debug_bytes >= bytes) return PGSGD_OK;
    if (g->d_debug) {
        cudaFree(g->d_debug);
        g->device_bytes -= g->debug_bytes;
        g->d_debug = nullptr;
        g->debug_bytes = 0;
    }
    CK(cudaMalloc(&g->d_debug, bytes), "debug buffer");
    g->debug_bytes = bytes;
    g->device_bytes += bytes;
    return PGSGD_OK;
}

int check_theta(double theta) {
    if (!(theta >= 0.0 && theta <= 4.0)) return fail(PGSGD_EINVAL, "theta %g outside [0, 4]", theta);
    return PGSGD_OK;
}

cudaEvent_t take_event(pgsgd_graph* g) {
    if (!g->ev_free.empty()) {
        cudaEvent_t e = g->ev_free.back();
        g->ev_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

}  // namespace

extern "C" {

const char* pgsgd_last_error(void) { return g_last_error.c_str(); }

const char* pgsgd_status_string(int status) {
    switch (status) {
        case PGSGD_OK: return "PGSGD_OK";
        case PGSGD_EINVAL: return "PGSGD_EINVAL";
        case PGSGD_ERANGE: return "PGSGD_ERANGE";
        case PGSGD_ENOMEM: return "PGSGD_ENOMEM";
        case PGSGD_ECUDA: return "PGSGD_ECUDA";
        case PGSGD_ETIMEOUT: return "PGSGD_ETIMEOUT";
        case PGSGD_EDEVICE: return "PGSGD_EDEVICE";
        default: return "PGSGD_UNKNOWN";
    }
}

int pgsgd_create(const uint32_t* node_len, uint32_t n_nodes, const uint64_t* path_off,
                 uint32_t n_paths, const uint32_t* step_node, const uint8_t* step_rev,
                 const int64_t* step_pos, int on_device, void* cuda_stream, pgsgd_graph** out) {
    return pgsgd::graph_create(node_len, n_nodes, path_off, n_paths, step_node, step_rev, step_pos, on_device,
                               cuda_stream, false, out);
}

}  // extern "C"

int pgsgd::graph_create(const uint32_t* node_len, uint32_t n_nodes, const uint64_t* path_off, uint32_t n_paths,
                        const uint32_t* step_node, const uint8_t* step_rev, const int64_t* step_pos, int on_device,
                        void* cuda_stream, bool batch, pgsgd_graph** out) {
    g_last_error.clear();
    if (!out) return fail(PGSGD_EINVAL, "out is NULL");
    *out = nullptr;
    if (!node_len || !path_off) return fail(PGSGD_EINVAL, "node_len and path_off are required");
    if (n_nodes == 0) return fail(PGSGD_EINVAL, "n_nodes is 0");
    if (n_nodes >= (1u << 31)) return fail(PGSGD_ERANGE, "n_nodes %u >= 2^31", n_nodes);
    if (n_paths == 0) return fail(PGSGD_EINVAL, "n_paths is 0");
    const uint32_t max_paths = batch ? kMaxBatchPaths : kMaxPaths;
    if (n_paths > max_paths) return fail(PGSGD_ERANGE, "n_paths %u > %u", n_paths, max_paths);
    if (on_device != 0 && on_device != 1) return fail(PGSGD_EINVAL, "on_device must be 0 or 1");
    cudaStream_t st = S(cuda_stream);

    // The path table is small: validate it on the host.
    std::vector<uint64_t> off(n_paths + 1);
    if (on_device) {
        CK(cudaMemcpy(off.data(), path_off, off.size() * sizeof(uint64_t), cudaMemcpyDeviceToHost),
           "path_off readback");
    } else {
        std::memcpy(off.data(), path_off, off.size() * sizeof(uint64_t));
    }
    if (off[0] != 0) return fail(PGSGD_EINVAL, "path_off[0] = %llu, must be 0", (unsigned long long)off[0]);
    uint64_t max_steps = 0;
    for (uint32_t p = 0; p < n_paths; ++p) {
        if (off[p + 1] < off[p]) return fail(PGSGD_EINVAL, "path_off decreases at path %u", p);
        max_steps = std::max<uint64_t>(max_steps, off[p + 1] - off[p]);
    }
    const uint64_t S_ = off[n_paths];
    if (S_ > 0 && (!step_node || !step_rev || !step_pos))
        return fail(PGSGD_EINVAL, "step arrays are required when the paths have steps");

    pgsgd_graph* g = new (std::nothrow) pgsgd_graph();
    if (!g) return fail(PGSGD_ENOMEM, "host allocation");
    cudaError_t e = cudaGetDevice(&g->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, g->device);
    if (e != cudaSuccess) {
        delete g;
        return cuda_fail(e, "device query");
    }
    g->n_nodes = n_nodes;
    g->n_paths = n_paths;
    g->n_steps = S_;
    g->max_path_steps = max_steps;
    g->h_path_off = off;

    int rc = PGSGD_OK;
    uint32_t* t_len = nullptr;
    uint32_t* t_node = nullptr;
    uint8_t* t_rev = nullptr;
    int64_t* t_pos = nullptr;
    std::vector<int64_t> nt(n_paths);
    int64_t* d_nt = nullptr;
    do {
#define TRY(call, what)                        \
    {                                          \
        cudaError_t e_ = (call);               \
        if (e_ != cudaSuccess) {               \
            rc = cuda_fail(e_, what);          \
            break;                             \
        }                                      \
    }
        TRY(dalloc(g, &g->d_nodes, n_nodes), "node records");
        TRY(dalloc(g, &g->d_anchor, n_nodes), "node anchors");
        TRY(dalloc(g, &g->d_changed, 1), "anchor flag");
        TRY(dalloc(g, &g->d_steps, S_), "step records");
        TRY(dalloc(g, &g->d_path_off, n_paths + 1), "path table");
        TRY(dalloc(g, &g->d_sample_off, n_paths + 1), "stress sample table");
        TRY(dalloc(g, &g->d_zipf_B, n_paths), "zipf table");
        TRY(dalloc(g, &g->d_zipf_T, kZipfTable), "zipf thresholds");
        if (!batch) {
            // guide: buckets of 2^shift steps, at most kGuideBuckets of them;
            // guide[b] = path holding step b << shift, guide[n] = P - 1
            uint32_t shift = 0;
            while (S_ > 0 && ((S_ - 1) >> shift) >= (uint64_t)kGuideBuckets) ++shift;
            const uint32_t nb = S_ > 0 ? (uint32_t)((S_ - 1) >> shift) + 1 : 1;
            std::vector<uint16_t> guide(nb + 1);
            for (uint32_t b = 0; b < nb; ++b) {
                const uint64_t gs = (uint64_t)b << shift;
                uint32_t lo = 0, hi = n_paths;
                while (hi - lo > 1) {
                    const uint32_t mid = lo + (hi - lo) / 2;
                    if (off[mid] <= gs) lo = mid; else hi = mid;
                }
                guide[b] = (uint16_t)lo;
            }
            guide[nb] = (uint16_t)(n_paths - 1);
            g->n_guide = nb;
            g->guide_shift = shift;
            TRY(dalloc(g, &g->d_guide, nb + 1), "path guide");
            TRY(cudaMemcpy(g->d_guide, guide.data(), guide.size() * sizeof(uint16_t), cudaMemcpyHostToDevice),
                "path guide upload");
        }
        TRY(dalloc(g, &g->d_flags, 1), "flags");
        g->max_stress_blocks = g->sm_count * 8;
        TRY(dalloc(g, &g->d_partials, 3 * (size_t)g->max_stress_blocks + 3), "stress scratch");
        TRY(dalloc(g, &g->d_per_path, 3 * (size_t)n_paths), "per-path stress");
        TRY(cudaMemsetAsync(g->d_flags, 0, sizeof(uint32_t), st), "flags clear");
        TRY(cudaMemcpyAsync(g->d_path_off, off.data(), off.size() * sizeof(uint64_t),
                            cudaMemcpyHostToDevice, st), "path table upload");
        const uint32_t* src_len = node_len;
        const uint32_t* src_node = step_node;
        const uint8_t* src_rev = step_rev;
        const int64_t* src_pos = step_pos;
        if (!on_device) {
            TRY(cudaMalloc(&t_len, (size_t)n_nodes * 4), "staging");
            TRY(cudaMemcpyAsync(t_len, node_len, (size_t)n_nodes * 4, cudaMemcpyHostToDevice, st), "upload");
            src_len = t_len;
            if (S_) {
                TRY(cudaMalloc(&t_node, S_ * 4), "staging");
                TRY(cudaMalloc(&t_rev, S_), "staging");
                TRY(cudaMalloc(&t_pos, S_ * 8), "staging");
                TRY(cudaMemcpyAsync(t_node, step_node, S_ * 4, cudaMemcpyHostToDevice, st), "upload");
                TRY(cudaMemcpyAsync(t_rev, step_rev, S_, cudaMemcpyHostToDevice, st), "upload");
                TRY(cudaMemcpyAsync(t_pos, step_pos, S_ * 8, cudaMemcpyHostToDevice, st), "upload");
                src_node = t_node;
                src_rev = t_rev;
                src_pos = t_pos;
            }
        }
        TRY(cudaMemsetAsync(g->d_nodes, 0, (size_t)n_nodes * sizeof(NodeRec), st), "node clear");
        TRY(cudaMemsetAsync(g->d_anchor, 0, (size_t)n_nodes * sizeof(int32_t), st), "anchor clear");
        TRY(cudaMemsetAsync(g->d_changed, 0, sizeof(uint32_t), st), "anchor flag clear");
        TRY(launch_check_lengths(src_len, n_nodes, g->d_flags, g->sm_count, st), "check lengths");
        TRY(launch_pack_steps(src_node, src_rev, src_pos, src_len, n_nodes, g->d_path_off, n_paths, S_,
                              g->d_steps, g->d_flags, g->sm_count, st), "pack steps");
        rc = check_flags(g, st, "pgsgd_create");
        if (rc) break;
        TRY(cudaMalloc(&d_nt, (size_t)n_paths * 8), "extent buffer");
        TRY(launch_path_extent(g->d_steps, g->d_path_off, n_paths, d_nt, st), "path extent");
        TRY(cudaMemcpyAsync(nt.data(), d_nt, (size_t)n_paths * 8, cudaMemcpyDeviceToHost, st), "extent readback");
        TRY(cudaStreamSynchronize(st), "create sync");
        for (int64_t v : nt) g->max_path_nt = std::max(g->max_path_nt, v);
        g->h_path_nt = nt;
#undef TRY
    } while (0);
    cudaFree(t_len);
    cudaFree(t_node);
    cudaFree(t_rev);
    cudaFree(t_pos);
    cudaFree(d_nt);
    if (rc != PGSGD_OK) {
        cudaStreamSynchronize(st);
        free_graph(g);
        return rc;
    }
    *out = g;
    return PGSGD_OK;
}

extern "C" {

int pgsgd_destroy(pgsgd_graph* g) {
    free_graph(g);
    return PGSGD_OK;
}

int pgsgd_set_option(pgsgd_graph* g, int option, int64_t v) {
    if (!g) return fail(PGSGD_EINVAL, "graph is NULL");
    switch (option) {
        case PGSGD_OPT_COORD_MODE:
            if (v != 0 && v != 1) return fail(PGSGD_EINVAL, "coord mode must be 0 or 1");
            g->coord_mode = (int)v;
            g->has_coords = false;
            return PGSGD_OK;
        case PGSGD_OPT_UPDATES_PER_STEP:
            if (v < 1 || v > 1000) return fail(PGSGD_EINVAL, "updates per step must be in [1, 1000]");
            g->updates_per_step = (int)v;
            return PGSGD_OK;
        case PGSGD_OPT_BLOCK:
            if (v < 64 || v > 256 || v % 32) return fail(PGSGD_EINVAL, "block must be 64..256, multiple of 32");
            g->block = (int)v;
            return PGSGD_OK;
        case PGSGD_OPT_BLOCKS_PER_SM:
            if (v < 1 || v > 64) return fail(PGSGD_EINVAL, "blocks per SM must be in [1, 64]");
            g->blocks_per_sm = (int)v;
            return PGSGD_OK;
        case PGSGD_OPT_UPDATES_PER_THREAD:
            if (v != 0 && v != 1 && v != 2 && v != 4)
                return fail(PGSGD_EINVAL, "updates per thread must be 0 (automatic), 1, 2 or 4");
            g->upt = (int)v;
            return PGSGD_OK;
        case PGSGD_OPT_ATOMIC_UPDATES:
            g->atomic = v ? 1 : 0;
            return PGSGD_OK;
        case PGSGD_OPT_REBASE:
            g->rebase = v ? 1 : 0;
            return PGSGD_OK;
        case PGSGD_OPT_TIMING:
            g->timing = v ? 1 : 0;
            return PGSGD_OK;
        case PGSGD_OPT_MAX_CONCURRENT:
            if (v < -1) return fail(PGSGD_EINVAL, "max concurrent must be >= -1");
            g->max_concurrent = v;
            return PGSGD_OK;
        case PGSGD_OPT_MIN_BLOCKS:
            if (v < 0 || v > 6) return fail(PGSGD_EINVAL, "min blocks must be in [0, 6]");
            g->min_blocks = (int)v;
            return PGSGD_OK;
        case PGSGD_OPT_STORE_MODE:
            if (v != 0 && v != 1) return fail(PGSGD_EINVAL, "store mode must be 0 or 1");
            g->store_mode = (int)v;
            return PGSGD_OK;
        case PGSGD_OPT_L2_HINTS:
            g->l2_hints = v ? 1 : 0;
            return PGSGD_OK;
        case PGSGD_OPT_PREFETCH64:
            if (v < 0 || v > 15) return fail(PGSGD_EINVAL, "prefetch option must be in [0, 15]");
            g->pf64 = (int)v;
            return PGSGD_OK;
        case PGSGD_OPT_PIPELINE:
            if (v < -1 || v > 1) return fail(PGSGD_EINVAL, "pipeline must be -1 (automatic), 0 or 1");
            g->pipeline = (int)v;
            return PGSGD_OK;
        case PGSGD_OPT_WARP_MERGE:
            g->warp_merge = v ? 1 : 0;
            return PGSGD_OK;
        case PGSGD_OPT_ASYNC_DEPTH:
            if (v != 0 && v != 2 && v != 3 && v != 4 && v != 6 && v != 8)
                return fail(PGSGD_EINVAL, "async depth must be 0, 2, 3, 4, 6 or 8");
            g->async_depth = (int)v;
            return PGSGD_OK;
        case PGSGD_OPT_STRESS_ASYNC:
            if (v != 0 && v != 2 && v != 4 && v != 8)
                return fail(PGSGD_EINVAL, "stress async depth must be 0, 2, 4 or 8");
            g->stress_async = (int)v;
            return PGSGD_OK;
        case PGSGD_OPT_STRESS_WAVES:
            if (v < 0 || v > 8) return fail(PGSGD_EINVAL, "stress waves must be in [0, 8]");
            g->stress_waves = (int)v;
            return PGSGD_OK;
        case PGSGD_OPT_DRF:
            if (v != 1 && v != 2 && v != 4 && v != 8) return fail(PGSGD_EINVAL, "data reuse factor must be 1, 2, 4 or 8");
            g->drf = (int)v;
            return PGSGD_OK;
        case PGSGD_OPT_SRF:
            if (v < 1 || v > (1 << 20)) return fail(PGSGD_EINVAL, "step reduction factor must be in [1, 2^20]");
            g->srf = (int)v;
            return PGSGD_OK;
        case PGSGD_OPT_L2_FETCH:
            if (v != 0 && v != 32 && v != 64 && v != 128)
                return fail(PGSGD_EINVAL, "L2 fetch granularity must be 0, 32, 64 or 128");
            g->l2_fetch = (int)v;
            return PGSGD_OK;
        default:
            return fail(PGSGD_EINVAL, "unknown option %d", option);
    }
}

int pgsgd_get_option(const pgsgd_graph* g, int option, int64_t* v) {
    if (!g || !v) return fail(PGSGD_EINVAL, "NULL argument");
    switch (option) {
        case PGSGD_OPT_COORD_MODE: *v = g->coord_mode; return PGSGD_OK;
        case PGSGD_OPT_UPDATES_PER_STEP: *v = g->updates_per_step; return PGSGD_OK;
        case PGSGD_OPT_BLOCK: *v = g->block; return PGSGD_OK;
        case PGSGD_OPT_BLOCKS_PER_SM: *v = g->blocks_per_sm; return PGSGD_OK;
        case PGSGD_OPT_UPDATES_PER_THREAD: *v = g->upt; return PGSGD_OK;
        case PGSGD_OPT_ATOMIC_UPDATES: *v = g->atomic; return PGSGD_OK;
        case PGSGD_OPT_REBASE: *v = g->rebase; return PGSGD_OK;
        case PGSGD_OPT_TIMING: *v = g->timing; return PGSGD_OK;
        case PGSGD_OPT_MAX_CONCURRENT: *v = g->max_concurrent; return PGSGD_OK;
        case PGSGD_OPT_MIN_BLOCKS: *v = g->min_blocks; return PGSGD_OK;
        case PGSGD_OPT_L2_FETCH: *v = g->l2_fetch; return PGSGD_OK;
        case PGSGD_OPT_STORE_MODE: *v = g->store_mode; return PGSGD_OK;
        case PGSGD_OPT_L2_HINTS: *v = g->l2_hints; return PGSGD_OK;
        case PGSGD_OPT_PREFETCH64: *v = g->pf64; return PGSGD_OK;
        case PGSGD_OPT_PIPELINE: *v = g->pipeline; return PGSGD_OK;
        case PGSGD_OPT_WARP_MERGE: *v = g->warp_merge; return PGSGD_OK;
        case PGSGD_OPT_ASYNC_DEPTH: *v = g->async_depth; return PGSGD_OK;
        case PGSGD_OPT_STRESS_ASYNC: *v = g->stress_async; return PGSGD_OK;
        case PGSGD_OPT_STRESS_WAVES: *v = g->stress_waves; return PGSGD_OK;
        case PGSGD_OPT_DRF: *v = g->drf; return PGSGD_OK;
        case PGSGD_OPT_SRF: *v = g->srf; return PGSGD_OK;
        default: return fail(PGSGD_EINVAL, "unknown option %d", option);
    }
}

int pgsgd_info_get(const pgsgd_graph* g, pgsgd_info* out) {
    if (!g || !out) return fail(PGSGD_EINVAL, "NULL argument");
    out->n_steps = g->n_steps;
    out->device_bytes = g->device_bytes;
    out->max_path_steps = g->max_path_steps;
    out->max_path_nt = g->max_path_nt;
    out->n_nodes = g->n_nodes;
    out->n_paths = g->n_paths;
    out->device = g->device;
    out->sm_count = g->sm_count;
    return PGSGD_OK;
}

int pgsgd_set_coords(pgsgd_graph* g, const double* xy, int on_device, void* cuda_stream) {
    if (!g || !xy) return fail(PGSGD_EINVAL, "NULL argument");
    cudaStream_t st = S(cuda_stream);
    const size_t bytes = (size_t)g->n_nodes * 4 * sizeof(double);
    const double* src = xy;
    if (!on_device) {
        if (!g->d_xy) CK(dalloc(g, &g->d_xy, (size_t)g->n_nodes * 4), "coordinate staging");
        CK(cudaMemcpyAsync(g->d_xy, xy, bytes, cudaMemcpyHostToDevice, st), "coordinate upload");
        src = g->d_xy;
    }
    CK(launch_set_coords(src, g->d_nodes, g->d_anchor, g->n_nodes, g->coord_mode == 0, g->d_flags, g->sm_count,
                         st),
       "set coords");
    // every step record gets its node's new anchor
    const uint32_t one = 1;
    CK(cudaMemcpyAsync(g->d_changed, &one, sizeof one, cudaMemcpyHostToDevice, st), "anchor flag");
    CK(launch_refresh_anchors(g->d_steps, g->d_anchor, g->n_steps, g->d_changed, g->sm_count, st),
       "refresh anchors");
    CK(cudaMemsetAsync(g->d_changed, 0, sizeof(uint32_t), st), "anchor flag clear");
    int rc = check_flags(g, st, "pgsgd_set_coords");
    if (rc) return rc;
    g->has_coords = true;
    return PGSGD_OK;
}

int pgsgd_get_coords(pgsgd_graph* g, double* xy, int on_device, void* cuda_stream) {
    if (!g || !xy) return fail(PGSGD_EINVAL, "NULL argument");
    if (!g->has_coords) return fail(PGSGD_EINVAL, "no layout: call pgsgd_set_coords first");
    cudaStream_t st = S(cuda_stream);
    const size_t bytes = (size_t)g->n_nodes * 4 * sizeof(double);
    if (on_device) {
        CK(launch_get_coords(g->d_nodes, g->d_anchor, xy, g->n_nodes, g->sm_count, st), "get coords");
        return PGSGD_OK;
    }
    if (!g->d_xy) CK(dalloc(g, &g->d_xy, (size_t)g->n_nodes * 4), "coordinate staging");
    CK(launch_get_coords(g->d_nodes, g->d_anchor, g->d_xy, g->n_nodes, g->sm_count, st), "get coords");
    CK(cudaMemcpyAsync(xy, g->d_xy, bytes, cudaMemcpyDeviceToHost, st), "coordinate download");
    CK(cudaStreamSynchronize(st), "coordinate sync");
    return PGSGD_OK;
}

int pgsgd_layout(pgsgd_graph* g, uint32_t iter_max, const double* eta, double eta_max, double eta_min,
                 double theta, uint64_t seed, uint32_t iter_begin, uint32_t iter_end, void* cuda_stream) {
    if (!g) return fail(PGSGD_EINVAL, "graph is NULL");
    if (!g->has_coords) return fail(PGSGD_EINVAL, "no layout: call pgsgd_set_coords first");
    if (iter_max == 0) return fail(PGSGD_EINVAL, "iter_max is 0");
    if (iter_begin > iter_end || iter_end > iter_max)
        return fail(PGSGD_EINVAL, "need iter_begin <= iter_end <= iter_max");
    int rc = check_theta(theta);
    if (rc) return rc;
    cudaStream_t st = S(cuda_stream);
    // learning rate eta_t of Algorithm 1: Zheng et al.'s exponential annealing
    std::vector<double> sched(iter_max);
    if (eta) {
        for (uint32_t t = 0; t < iter_max; ++t) sched[t] = eta[t];
    } else {
        const double emax = eta_max > 0 ? eta_max : (double)g->max_path_nt * (double)g->max_path_nt;
        const double emin = eta_min > 0 ? eta_min : 0.01;
        if (!(emax > 0)) return fail(PGSGD_EINVAL, "eta_max must be positive");
        if (iter_max == 1) {
            sched[0] = emax;
        } else {
            const double lambda = std::log(emax / emin) / (double)(iter_max - 1);
            for (uint32_t t = 0; t < iter_max; ++t) sched[t] = emax * std::exp(-lambda * (double)t);
        }
    }
    // a negative rate moves a pair apart and a NaN poisons both nodes
    for (uint32_t t = 0; t < iter_max; ++t)
        if (!(std::isfinite(sched[t]) && sched[t] >= 0.0))
            return fail(PGSGD_EINVAL, "learning rate %g at iteration %u is not finite and >= 0", sched[t], t);
    const float th = (float)theta;
    rc = ensure_zipf(g, th, st);
    if (rc) return rc;
    // launch shape: the automatic choice (pipeline -1, updates per thread 0) is
    // the pipelined loop at 2 updates per thread for the plain method, one
    // update per thread otherwise
    const bool plain = !g->warp_merge && g->drf == 1;
    if (g->pipeline == 1 && !plain)
        return fail(PGSGD_EINVAL, "warp merging and data reuse run the plain update loop: set pipeline 0");
    const bool async_loop = g->async_depth > 0 && plain;
    const int pipe = g->pipeline >= 0 ? g->pipeline : (plain && !async_loop ? 1 : 0);
    // concurrency cap: at most `cap` updates in flight (0 = none)
    int64_t cap = g->max_concurrent;
    if (cap == -1) cap = (int64_t)default_in_flight_cap(g->n_nodes, (uint64_t)g->updates_per_step * g->n_steps);
    // the automatic shape keeps 1 update per thread where 2 would put a
    // 64-thread block above the cap
    const int upt = g->upt > 0 ? g->upt : (pipe && !(cap > 0 && cap < 128) ? 2 : 1);
    if (async_loop && (pipe || upt != 1))
        return fail(PGSGD_EINVAL, "the asynchronous step-record loop runs one update per thread: set pipeline 0 "
                                  "and updates_per_thread 1");
    // updates per iteration (Algorithm 1: 10 x steps) cut by the step reduction
    // factor; with data reuse the kernel counts selections of drf updates
    const uint64_t N_full = (uint64_t)g->updates_per_step * g->n_steps;
    const uint64_t N = (N_full + (uint64_t)g->srf - 1) / (uint64_t)g->srf;
    const uint64_t updates_per_launch = N * (uint64_t)g->drf;
    UpdateLaunch L;
    L.nodes = g->d_nodes;
    L.u_begin = 0;
    L.n_updates = N;
    // a cap below one block's worth shrinks the block (whole warps, at least
    // 64 threads) before the grid is cut to the cap
    const int64_t per_thread = g->drf > 1 ? g->drf : upt;
    L.block = g->block;
    if (cap > 0 && cap < (int64_t)g->block * per_thread)
        L.block = (int)std::max<int64_t>(64, cap / per_thread / 32 * 32);
    L.upt = upt;
    // automatic register budget for the plain loop: 4 resident blocks per SM
    // at 1 update per thread, 3 at 2 (no spills either way), else the
    // compiler's choice
    L.minb = g->min_blocks ? g->min_blocks : pipe ? (upt == 2 ? 2 : 1) : upt == 1 ? 4 : upt == 2 ? 3 : 1;
    L.async_depth = async_loop ? g->async_depth : 0;
    L.store_mode = g->store_mode;
    L.l2_hints = g->l2_hints != 0;
    L.pf64 = g->pf64;
    L.pipeline = pipe != 0;
    L.wm = g->warp_merge != 0;
    L.drf = g->drf;
    L.atomic = g->atomic != 0;
    L.s = sampler_args(g, iter_max, iter_begin, th, seed);
    // grid: a multiple of the SM count; the concurrency cap bounds the updates
    // in flight at once, so it shrinks the grid only where it is below what
    // the resident blocks hold (a large graph keeps the full grid, whose
    // resident blocks hold fewer updates than the cap)
    int grid = g->sm_count * g->blocks_per_sm;
    if (cap > 0) {
        // the cap counts updates: a thread keeps upt updates, or one selection of drf updates, in flight
        const int64_t per_block = (int64_t)L.block * per_thread;
        const int64_t gmax = std::max<int64_t>(1, cap / per_block);
        const int nb = update_blocks_per_sm(L);
        const int64_t resident = (int64_t)nb * g->sm_count;
        if (gmax < grid && (nb <= 0 || gmax < resident)) grid = (int)gmax;
    }
    L.grid = grid;
    if (g->l2_fetch) CK(cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, g->l2_fetch), "L2 fetch limit");
    for (uint32_t t = iter_begin; t < iter_end; ++t) {
        L.s = sampler_args(g, iter_max, t, th, seed);
        L.eta = (float)sched[t];
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (g->timing) {
            e0 = take_event(g);
            e1 = take_event(g);
            CK(cudaEventRecord(e0, st), "timing event");
        }
        CK(launch_update(L, st), "update kernel");
        if (g->timing) {
            CK(cudaEventRecord(e1, st), "timing event");
            g->ev_pending.emplace_back(e0, e1);
            g->timing_launches += 1;
            g->timing_updates += updates_per_launch;
        }
        if (g->rebase && g->coord_mode == 0) {
            CK(launch_rebase(g->d_nodes, g->d_anchor, g->n_nodes, g->d_changed, g->sm_count, st), "rebase");
            CK(launch_refresh_anchors(g->d_steps, g->d_anchor, g->n_steps, g->d_changed, g->sm_count, st),
               "refresh anchors");
            CK(cudaMemsetAsync(g->d_changed, 0, sizeof(uint32_t), st), "anchor flag clear");
        }
    }
    return PGSGD_OK;
}

int pgsgd_timing_read(pgsgd_graph* g, double* total_ms, uint64_t* launches, uint64_t* updates, int reset) {
    if (!g) return fail(PGSGD_EINVAL, "graph is NULL");
    for (auto& pr : g->ev_pending) {
        CK(cudaEventSynchronize(pr.second), "timing sync");
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, pr.first, pr.second), "timing read");
        g->timing_ms += ms;
        g->ev_free.push_back(pr.first);
        g->ev_free.push_back(pr.second);
    }
    g->ev_pending.clear();
    if (total_ms) *total_ms = g->timing_ms;
    if (launches) *launches = g->timing_launches;
    if (updates) *updates = g->timing_updates;
    if (reset) {
        g->timing_ms = 0.0;
        g->timing_launches = 0;
        g->timing_updates = 0;
    }
    return PGSGD_OK;
}

int pgsgd_stress(pgsgd_graph* g, uint32_t samples_per_step, uint64_t seed, pgsgd_stress_result* out,
                 double* per_path, void* cuda_stream) {
    if (!g || !out) return fail(PGSGD_EINVAL, "NULL argument");
    if (!g->has_coords) return fail(PGSGD_EINVAL, "no layout: call pgsgd_set_coords first");
    if (samples_per_step == 0) return fail(PGSGD_EINVAL, "samples_per_step is 0");
    cudaStream_t st = S(cuda_stream);
    uint64_t n_samples = 0;
    if (g->stress_samples_per_step != samples_per_step) {
        std::vector<uint64_t> so(g->n_paths + 1, 0);
        for (uint32_t p = 0; p < g->n_paths; ++p) {
            const uint64_t n = g->h_path_off[p + 1] - g->h_path_off[p];
            so[p + 1] = so[p] + (n >= 2 ? (uint64_t)samples_per_step * n : 0);
        }
        CK(cudaMemcpyAsync(g->d_sample_off, so.data(), so.size() * 8, cudaMemcpyHostToDevice, st),
           "sample table upload");
        CK(cudaStreamSynchronize(st), "sample table sync");
        g->stress_samples_per_step = samples_per_step;
    }
    for (uint32_t p = 0; p < g->n_paths; ++p) {
        const uint64_t n = g->h_path_off[p + 1] - g->h_path_off[p];
        if (n >= 2) n_samples += (uint64_t)samples_per_step * n;
    }
    StressLaunch L;
    L.steps = g->d_steps;
    L.path_off = g->d_path_off;
    L.sample_off = g->d_sample_off;
    L.nodes = g->d_nodes;
    L.n_samples = n_samples;
    L.n_paths = g->n_paths;
    L.key0 = (uint32_t)seed;
    L.key1 = (uint32_t)(seed >> 32);
    L.partials = g->d_partials;
    L.per_path = per_path ? g->d_per_path : nullptr;
    L.pf64 = (g->pf64 >> 2) & 3;
    L.block = 256;
    L.async_depth = g->stress_async;
    const uint64_t want = (n_samples + 2 * 256 - 1) / (2 * 256);
    L.grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)g->max_stress_blocks));
    if (g->stress_waves > 0) {
        // whole waves: every resident block slot busy until the end (a grid-stride loop spreads the samples evenly)
        const int nb = stress_blocks_per_sm(L);
        if (nb > 0) {
            const int64_t wave = (int64_t)nb * g->sm_count;
            const int64_t waves = std::max<int64_t>(1, std::min<int64_t>(g->stress_waves, g->max_stress_blocks / wave));
            L.grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)(waves * wave)));
        }
    }
    if (per_path) CK(cudaMemsetAsync(g->d_per_path, 0, (size_t)g->n_paths * 3 * 8, st), "per-path clear");
    CK(launch_stress(L, st), "stress kernel");
    double* tot = g->d_partials + 3 * (size_t)g->max_stress_blocks;
    CK(launch_stress_finalize(g->d_partials, L.grid, tot, st), "stress finalize");
    double h[3];
    CK(cudaMemcpyAsync(h, tot, sizeof h, cudaMemcpyDeviceToHost, st), "stress readback");
    if (per_path)
        CK(cudaMemcpyAsync(per_path, g->d_per_path, (size_t)g->n_paths * 3 * 8, cudaMemcpyDeviceToHost, st),
           "per-path readback");
    CK(cudaStreamSynchronize(st), "stress sync");
    const double n = h[2];
    const double mean = n > 0 ? h[0] / n : 0.0;
    const double var = n > 1 ? std::max(0.0, (h[1] - n * mean * mean) / (n - 1.0)) : 0.0;
    const double sd = std::sqrt(var);
    const double half = n > 0 ? 1.96 * sd / std::sqrt(n) : 0.0;
    out->mean = mean;
    out->stddev = sd;
    out->ci_lo = mean - half;
    out->ci_hi = mean + half;
    out->n_valid = (uint64_t)n;
    out->n_skipped = n_samples - (uint64_t)n;
    return PGSGD_OK;
}

int pgsgd_debug_sample(pgsgd_graph* g, uint32_t t, uint32_t iter_max, double theta, uint64_t seed,
                       uint64_t u_begin, uint64_t count, pgsgd_sample* out, void* cuda_stream) {
    if (!g || (!out && count)) return fail(PGSGD_EINVAL, "NULL argument");
    if (iter_max == 0 || t >= iter_max) return fail(PGSGD_EINVAL, "need t < iter_max");
    int rc = check_theta(theta);
    if (rc) return rc;
    if (count == 0) return PGSGD_OK;
    cudaStream_t st = S(cuda_stream);
    rc = ensure_zipf(g, (float)theta, st);
    if (rc) return rc;
    rc = ensure_debug(g, count * sizeof(pgsgd_sample));
    if (rc) return rc;
    CK(launch_debug_sample(sampler_args(g, iter_max, t, (float)theta, seed), u_begin, count, g->d_debug,
                           g->sm_count, st), "debug sample");
    CK(cudaMemcpyAsync(out, g->d_debug, count * sizeof(pgsgd_sample), cudaMemcpyDeviceToHost, st),
       "debug readback");
    CK(cudaStreamSynchronize(st), "debug sync");
    return PGSGD_OK;
}

int pgsgd_debug_sample_reuse(pgsgd_graph* g, uint32_t t, uint32_t iter_max, double theta, uint64_t seed,
                             uint64_t q_begin, uint64_t count, pgsgd_sample* out, void* cuda_stream) {
    if (!g || (!out && count)) return fail(PGSGD_EINVAL, "NULL argument");
    if (iter_max == 0 || t >= iter_max) return fail(PGSGD_EINVAL, "need t < iter_max");
    if (g->drf < 2) return fail(PGSGD_EINVAL, "data reuse is off (PGSGD_OPT_DRF = 1)");
    int rc = check_theta(theta);
    if (rc) return rc;
    if (count == 0) return PGSGD_OK;
    cudaStream_t st = S(cuda_stream);
    rc = ensure_zipf(g, (float)theta, st);
    if (rc) return rc;
    const uint64_t n = count * (uint64_t)g->drf;
    rc = ensure_debug(g, n * sizeof(pgsgd_sample));
    if (rc) return rc;
    const uint64_t n_sel = ((uint64_t)g->updates_per_step * g->n_steps + g->srf - 1) / (uint64_t)g->srf;
    const SamplerArgs a = sampler_args(g, iter_max, t, (float)theta, seed);
    CK(launch_debug_sample_reuse(a, (uint32_t)g->drf, n_sel, q_begin, count, g->d_debug, g->sm_count, st),
       "debug sample kernel");
    CK(cudaMemcpyAsync(out, g->d_debug, n * sizeof(pgsgd_sample), cudaMemcpyDeviceToHost, st), "debug readback");
    CK(cudaStreamSynchronize(st), "debug sync");
    return PGSGD_OK;
}

int pgsgd_debug_sweep(pgsgd_graph* g, uint32_t t, uint32_t iter_max, double eta, double theta,
                      uint64_t seed, uint64_t u_begin, uint64_t count, float* out, void* cuda_stream) {
    if (!g || (!out && count)) return fail(PGSGD_EINVAL, "NULL argument");
    if (!g->has_coords) return fail(PGSGD_EINVAL, "no layout: call pgsgd_set_coords first");
    if (iter_max == 0 || t >= iter_max) return fail(PGSGD_EINVAL, "need t < iter_max");
    int rc = check_theta(theta);
    if (rc) return rc;
    if (count == 0) return PGSGD_OK;
    cudaStream_t st = S(cuda_stream);
    rc = ensure_zipf(g, (float)theta, st);
    if (rc) return rc;
    rc = ensure_debug(g, count * sizeof(float4));
    if (rc) return rc;
    CK(launch_debug_sweep(sampler_args(g, iter_max, t, (float)theta, seed), u_begin, count, g->d_nodes,
                          (float)eta, static_cast<float4*>(g->d_debug), g->sm_count, st), "debug sweep");
    CK(cudaMemcpyAsync(out, g->d_debug, count * sizeof(float4), cudaMemcpyDeviceToHost, st), "sweep readback");
    CK(cudaStreamSynchronize(st), "sweep sync");
    return PGSGD_OK;
}

int pgsgd_dstress(pgsgd_graph* g, uint64_t n_pairs, uint64_t seed, double* value, uint64_t* n_valid,
                  void* cuda_stream) {
    if (!g || !value) return fail(PGSGD_EINVAL, "NULL argument");
    if (!g->has_coords) return fail(PGSGD_EINVAL, "no layout: call pgsgd_set_coords first");
    cudaStream_t st = S(cuda_stream);
    int rc = ensure_zipf(g, 0.99f, st);
    if (rc) return rc;
    const SamplerArgs a = sampler_args(g, 1, 0, 0.99f, seed);
    const uint64_t want = (n_pairs + 255) / 256;
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)g->max_stress_blocks));
    CK(launch_dstress_forward(a, g->d_nodes, n_pairs, g->d_partials, grid, st), "dstress forward");
    double* tot = g->d_partials + 3 * (size_t)g->max_stress_blocks;
    CK(launch_stress_finalize(g->d_partials, grid, tot, st), "dstress finalize");
    double h[3];
    CK(cudaMemcpyAsync(h, tot, sizeof h, cudaMemcpyDeviceToHost, st), "dstress readback");
    CK(cudaStreamSynchronize(st), "dstress sync");
    *value = h[2] > 0 ? h[0] / h[2] : 0.0;
    if (n_valid) *n_valid = (uint64_t)h[2];
    return PGSGD_OK;
}

int pgsgd_dstress_backward(pgsgd_graph* g, uint64_t n_pairs, uint64_t seed, double scale, float* grad,
                           void* cuda_stream) {
    if (!g || !grad) return fail(PGSGD_EINVAL, "NULL argument");
    if (!g->has_coords) return fail(PGSGD_EINVAL, "no layout: call pgsgd_set_coords first");
    cudaStream_t st = S(cuda_stream);
    int rc = ensure_zipf(g, 0.99f, st);
    if (rc) return rc;
    CK(cudaMemsetAsync(grad, 0, (size_t)g->n_nodes * 4 * sizeof(float), st), "gradient clear");
    CK(launch_dstress_backward(sampler_args(g, 1, 0, 0.99f, seed), g->d_nodes, n_pairs, (float)scale, grad,
                               g->sm_count, st),
       "dstress backward");
    return PGSGD_OK;
}

int pgsgd_debug_pair_grad(pgsgd_graph* g, uint32_t t, uint32_t iter_max, double theta, uint64_t seed,
                          uint64_t u_begin, uint64_t count, float* out, void* cuda_stream) {
    if (!g || (!out && count)) return fail(PGSGD_EINVAL, "NULL argument");
    if (!g->has_coords) return fail(PGSGD_EINVAL, "no layout: call pgsgd_set_coords first");
    if (iter_max == 0 || t >= iter_max) return fail(PGSGD_EINVAL, "need t < iter_max");
    int rc = check_theta(theta);
    if (rc) return rc;
    if (count == 0) return PGSGD_OK;
    cudaStream_t st = S(cuda_stream);
    rc = ensure_zipf(g, (float)theta, st);
    if (rc) return rc;
    rc = ensure_debug(g, count * sizeof(float4));
    if (rc) return rc;
    CK(launch_pair_grad(sampler_args(g, iter_max, t, (float)theta, seed), u_begin, count, g->d_nodes,
                        static_cast<float4*>(g->d_debug), g->sm_count, st),
       "pair gradient");
    CK(cudaMemcpyAsync(out, g->d_debug, count * sizeof(float4), cudaMemcpyDeviceToHost, st), "pair grad readback");
    CK(cudaStreamSynchronize(st), "pair grad sync");
    return PGSGD_OK;
}

int pgsgd_full_stress(pgsgd_graph* g, double* value, uint64_t* n_pairs, void* cuda_stream) {
    if (!g || !value) return fail(PGSGD_EINVAL, "NULL argument");
    if (!g->has_coords) return fail(PGSGD_EINVAL, "no layout: call pgsgd_set_coords first");
    cudaStream_t st = S(cuda_stream);
    const int grid = g->max_stress_blocks;
    CK(launch_full_stress(g->d_steps, g->d_nodes, g->d_path_off, g->n_paths, g->n_steps, g->d_partials, grid, st),
       "full stress");
    double* tot = g->d_partials + 3 * (size_t)g->max_stress_blocks;
    CK(launch_stress_finalize(g->d_partials, grid, tot, st), "full stress finalize");
    double h[3];
    CK(cudaMemcpyAsync(h, tot, sizeof h, cudaMemcpyDeviceToHost, st), "full stress readback");
    CK(cudaStreamSynchronize(st), "full stress sync");
    *value = h[2] > 0 ? h[0] / h[2] : 0.0;
    if (n_pairs) *n_pairs = (uint64_t)h[2];
    return PGSGD_OK;
}

}  // extern "C"
