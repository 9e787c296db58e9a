// Batched PG-SGD layout: many independent graphs laid out by the same kernels
// at once. The paper lays out one graph per run and notes that small graphs
// leave most of the GPU idle while kernel launches dominate (Section IV-B);
// here every graph keeps its own sampler key, learning-rate schedule and
// iteration count, so graph g's draws are exactly those of a one-graph layout
// of g (Algorithm 1 with counter (u, t, block) under g's seed), while the work
// of all graphs shares the GPU.
//
// Work unit: a chunk = a run of consecutive update indices of one graph in
// one iteration. Three schedules run the same chunk code:
//   mode 0  one launch per iteration over all graphs: every graph gets
//           `lanes` blocks, lane k runs chunks k, k + lanes, ...; the launches
//           of a layout are captured once into a CUDA graph and replayed;
//   mode 1  one persistent launch for all iterations: blocks claim chunks
//           from per-graph queues (a 64-bit word = iteration << 32 | next
//           chunk); the block that completes a graph's last chunk of an
//           iteration opens the next one, so graphs advance independently.
//           Waits for claimable work are bounded by a wall-clock budget and
//           end in PGSGD_ETIMEOUT;
//   mode 2  the comparison point: per iteration, one launch per graph.
// Per graph at most `max_active` chunks are in flight, each run by `threads`
// threads of its block, i.e. at most max_active * threads * upt updates at
// once (default cap max(64, V_g / 16, N_g / 5120) updates, the single-graph
// kernel's rule): a graph whose cap is below one block's worth runs one
// chunk at a time on part of the block, so small graphs see no more
// simultaneous updates than when laid out alone.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/pgsgd.h"
#include "../../include/pgsgd_batch.h"
#include "pgsgd_internal.h"

namespace pgsgd {
namespace {

// One graph of the batch, in schedule (rank) order.
struct BatchGraph {
    uint64_t step0;       // first step of the graph in the packed step array
    uint64_t n_steps;     // S_g
    uint64_t n_updates;   // N_g per iteration
    uint32_t path0;       // first path
    uint32_t n_paths;     // P_g
    uint32_t n_chunks;    // ceil(N_g / chunk)
    uint32_t max_active;  // chunks in flight at most (persistent) = lanes (launch modes)
    uint32_t key0, key1;  // Philox key = the graph's seed
    uint32_t threads;     // threads of a block that run the graph's chunks (a multiple of 32)
    uint32_t pad[3];
};
static_assert(sizeof(BatchGraph) == 64, "BatchGraph layout");

struct BatchLaunch {
    const BatchGraph* graphs;  // [G] rank order
    const float* eta;          // [G][T] rank order
    const StepRec* steps;
    const uint64_t* path_off;  // [P + 1] global
    const float* zipf_B;       // [P]
    const float* zipf_T;       // [kZipfTable]
    NodeRec* nodes;
    uint64_t chunk;            // updates per chunk
    uint32_t n_graphs;
    uint32_t T;                // iterations of the schedule
    uint32_t iter_begin, iter_end;
    float theta;
    int store_mode;
    int pf64;
    uint64_t timeout_ns;       // persistent mode: longest wait for claimable work
};

struct BatchQueues {
    unsigned long long* q;  // [G] iteration << 32 | next chunk
    uint32_t* done;         // [G] chunks completed in the open iteration
    uint32_t* finished;     // graphs done with iteration iter_end - 1
    uint32_t* err;          // error bits (BERR_*)
};

enum : uint32_t { BERR_TIMEOUT = 1u, BERR_NODE_RANGE = 2u };

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t* p) { return *(const volatile uint32_t*)p; }
__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long* p) {
    return *(const volatile unsigned long long*)p;
}

// Shared-memory layout of a block's current graph: path offsets relative to
// the graph's first step [P_g + 1], Zipf thresholds [kZipfTable], Zipf B
// [P_g], and a one-bucket guide (every step maps to bucket 0, whose search
// range is all P_g paths).
struct BatchSmem {
    uint64_t* off;
    float* T;
    float* B;
    uint16_t* guide;
};

__host__ __device__ inline size_t batch_smem_bytes(uint32_t max_paths) {
    return (size_t)(max_paths + 1) * sizeof(uint64_t) + (size_t)(kZipfTable + max_paths) * sizeof(float) +
           2 * sizeof(uint16_t);
}

__device__ __forceinline__ BatchSmem batch_smem(unsigned char* smem, uint32_t max_paths) {
    BatchSmem s;
    s.off = reinterpret_cast<uint64_t*>(smem);
    s.T = reinterpret_cast<float*>(s.off + max_paths + 1);
    s.B = s.T + kZipfTable;
    s.guide = reinterpret_cast<uint16_t*>(s.B + max_paths);
    return s;
}

// Once per block: the Zipf thresholds and constants of theta.
__device__ __forceinline__ void stage_theta(const BatchLaunch& L, const BatchSmem& s, ZipfConsts& zc) {
    for (uint32_t k = threadIdx.x; k < (uint32_t)kZipfTable; k += blockDim.x) s.T[k] = L.zipf_T[k];
    if (threadIdx.x == 0) {
        ZipfConsts z;
        z.theta = L.theta;
        zipf_theta_consts(z.theta, z.omt, z.A, z.s);
        zc = z;
    }
}

// The path table of graph G (all threads; the caller synchronises after).
__device__ __forceinline__ void stage_graph(const BatchLaunch& L, const BatchGraph& G, const BatchSmem& s) {
    for (uint32_t k = threadIdx.x; k <= G.n_paths; k += blockDim.x) s.off[k] = L.path_off[G.path0 + k] - G.step0;
    for (uint32_t k = threadIdx.x; k < G.n_paths; k += blockDim.x) s.B[k] = L.zipf_B[G.path0 + k];
    if (threadIdx.x == 0) {
        s.guide[0] = 0;
        s.guide[1] = (uint16_t)(G.n_paths ? G.n_paths - 1 : 0);
    }
}

__device__ __forceinline__ BatchGraph load_graph(const BatchGraph* p) {
    BatchGraph G;
    const uint4* q = reinterpret_cast<const uint4*>(p);
    const uint4 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2), d = __ldg(q + 3);
    G.step0 = (uint64_t)a.x | ((uint64_t)a.y << 32);
    G.n_steps = (uint64_t)a.z | ((uint64_t)a.w << 32);
    G.n_updates = (uint64_t)b.x | ((uint64_t)b.y << 32);
    G.path0 = b.z;
    G.n_paths = b.w;
    G.n_chunks = c.x;
    G.max_active = c.y;
    G.key0 = c.z;
    G.key1 = c.w;
    G.threads = d.x;
    return G;
}

__device__ __forceinline__ SamplerArgs graph_sampler(const BatchLaunch& L, const BatchGraph& G, uint32_t t,
                                                     const ZipfConsts& zc) {
    SamplerArgs a;
    a.steps = L.steps + G.step0;
    a.path_off = nullptr;
    a.zipf_B = nullptr;
    a.zipf_T = nullptr;
    a.guide = nullptr;
    a.n_steps = G.n_steps;
    a.n_paths = G.n_paths;
    a.n_guide = 1;
    a.guide_shift = 63;
    a.T = L.T;
    a.t = t;
    a.key0 = G.key0;
    a.key1 = G.key1;
    a.zc = zc;
    return a;
}

// The updates [c * chunk, min((c + 1) * chunk, N_g)) of iteration t of the
// graph of rank r, by the block's first G.threads threads (the caller skips
// the others; whole warps, so every warp runs or idles as one).
template <int UPT, bool PIPE>
__device__ __forceinline__ void run_chunk(const BatchLaunch& L, const BatchGraph& G, uint32_t r, const BatchSmem& s,
                                          const ZipfConsts& zc, uint32_t t, uint32_t c, uint64_t pol_stream,
                                          uint64_t pol_keep) {
    const SamplerArgs a = graph_sampler(L, G, t, zc);
    const PathTable pt{s.off, s.B, s.T, s.guide, G.n_paths, 63};
    const UpdateOpts o{L.eta[(uint64_t)r * L.T + t], L.store_mode, L.pf64, false};
    const uint64_t cb = (uint64_t)c * L.chunk;
    const uint64_t ce = min(cb + L.chunk, G.n_updates);
    if (PIPE) {
        update_range_pipelined<UPT>(a, pt, L.nodes, cb + threadIdx.x, G.threads, ce, o, pol_stream, pol_keep);
    } else {
        for (uint64_t base = cb + threadIdx.x; base < ce; base += (uint64_t)G.threads * UPT)
            update_trip<UPT>(a, pt, L.nodes, base, G.threads, ce, o, pol_stream, pol_keep);
    }
}

// ---------------------------------------------------------------- modes 0 and 2

// Block b runs lane lanes[b] = (graph rank, lane k) of iteration t.
template <int UPT, bool PIPE>
__global__ void __launch_bounds__(256) batch_lane_kernel(BatchLaunch L, uint32_t max_paths, uint32_t t,
                                                         const uint2* __restrict__ lanes) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ZipfConsts zc;
    const BatchSmem s = batch_smem(smem, max_paths);
    const uint2 ln = lanes[blockIdx.x];
    const BatchGraph G = load_graph(L.graphs + ln.x);
    stage_theta(L, s, zc);
    stage_graph(L, G, s);
    __syncthreads();
    const uint64_t pol_stream = policy_evict_first(), pol_keep = policy_evict_last();
    const uint32_t stride = G.max_active;
    if (threadIdx.x >= G.threads) return;  // no barrier follows
    for (uint32_t c = ln.y; c < G.n_chunks; c += stride)
        run_chunk<UPT, PIPE>(L, G, ln.x, s, zc, t, c, pol_stream, pol_keep);
}

// ---------------------------------------------------------------- mode 1

__device__ __forceinline__ bool can_claim(unsigned long long qv, uint32_t n_chunks, uint32_t cap, uint32_t done,
                                          uint32_t iter_end) {
    const uint32_t it = (uint32_t)(qv >> 32), nx = (uint32_t)qv;
    return it < iter_end && nx < n_chunks && nx - done < cap;
}

// Warp 0: claim one chunk, scanning graphs in rank order (longest lanes first).
// Returns 0 = claimed (r, t, c), 1 = nothing claimable now, 2 = all graphs
// finished, 3 = error raised.
__device__ int claim_chunk(const BatchLaunch& L, const BatchQueues& Q, uint32_t& r, uint32_t& t, uint32_t& c) {
    const int lane = threadIdx.x & 31;
    // lane 0 reads the shared words so every decision is warp-uniform
    if (__shfl_sync(0xffffffffu, lane == 0 ? ld_volatile(Q.err) : 0u, 0)) return 3;
    for (uint32_t base = 0; base < L.n_graphs; base += 32) {
        const uint32_t k = base + lane;
        unsigned long long qv = 0;
        uint32_t nch = 0, cap = 0;
        bool ok = false;
        if (k < L.n_graphs) {
            nch = __ldg(&L.graphs[k].n_chunks);
            cap = __ldg(&L.graphs[k].max_active);
            qv = ld_volatile(Q.q + k);
            ok = can_claim(qv, nch, cap, ld_volatile(Q.done + k), L.iter_end);
        }
        uint32_t mask = __ballot_sync(0xffffffffu, ok);
        while (mask) {
            const int leader = __ffs(mask) - 1;
            int got = 0;
            if (lane == leader) {
                for (int tries = 0; tries < 4 && ok; ++tries) {
                    const unsigned long long old = atomicCAS(Q.q + k, qv, qv + 1);
                    if (old == qv) { got = 1; break; }
                    qv = old;
                    ok = can_claim(qv, nch, cap, ld_volatile(Q.done + k), L.iter_end);
                }
            }
            got = __shfl_sync(0xffffffffu, got, leader);
            if (got) {
                qv = __shfl_sync(0xffffffffu, qv, leader);
                r = base + leader;
                t = (uint32_t)(qv >> 32);
                c = (uint32_t)qv;
                __threadfence();
                return 0;
            }
            mask &= mask - 1;
        }
    }
    const uint32_t fin = __shfl_sync(0xffffffffu, lane == 0 ? ld_volatile(Q.finished) : 0u, 0);
    return fin >= L.n_graphs ? 2 : 1;
}

// Thread 0, after the whole block's writes of chunk (r, t) are fenced.
__device__ __forceinline__ void complete_chunk(const BatchLaunch& L, const BatchQueues& Q, uint32_t r, uint32_t t) {
    const uint32_t nch = __ldg(&L.graphs[r].n_chunks);
    const uint32_t old = atomicAdd(Q.done + r, 1u);
    if (old + 1 != nch) return;
    // last chunk of iteration t: reset the count, then open iteration t + 1
    atomicExch(Q.done + r, 0u);
    __threadfence();
    atomicExch(Q.q + r, (unsigned long long)(t + 1) << 32);
    if (t + 1 >= L.iter_end) {
        __threadfence();
        atomicAdd(Q.finished, 1u);
    }
}

// A register budget of 3 resident blocks per SM (2 at 4 updates per thread)
// as the lane kernels have; without it the queue logic took the kernel to
// 102-124 registers and 2 blocks per SM.
// Warp 0 claims the block's next chunk while the other warps finish their
// share of the current one, so a claim's scan of the queues costs no time
// between chunks; the current chunk is completed (and its graph's next
// iteration possibly opened) after the block's barrier, then the claimed
// command is published for the next trip.
template <int UPT, bool PIPE>
__global__ void __launch_bounds__(256, UPT == 4 ? 2 : 3) batch_persistent_kernel(BatchLaunch L, uint32_t max_paths, BatchQueues Q) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ZipfConsts zc;
    __shared__ uint32_t s_cmd[4];  // status, rank, iteration, chunk
    const BatchSmem s = batch_smem(smem, max_paths);
    stage_theta(L, s, zc);
    const uint64_t pol_stream = policy_evict_first(), pol_keep = policy_evict_last();
    uint32_t cur = 0xffffffffu;
    BatchGraph G{};
    bool waiting = false;
    uint64_t wait_start = 0;
    // warp 0: one claim; lane 0 (thread 0) keeps the bounded-wait bookkeeping
    auto claim = [&](uint32_t (&cmd)[4]) {
        uint32_t r = 0, t = 0, c = 0;
        int st = claim_chunk(L, Q, r, t, c);
        if (threadIdx.x == 0) {
            if (st == 1) {
                // nothing claimable: every open chunk is held by a running
                // block, so this ends unless a queue is stuck; bounded
                const uint64_t now = global_ns();
                if (!waiting) {
                    waiting = true;
                    wait_start = now;
                } else if (now - wait_start > L.timeout_ns) {
                    atomicOr(Q.err, BERR_TIMEOUT);
                    st = 3;
                }
            } else {
                waiting = false;
            }
        }
        cmd[0] = (uint32_t)st;
        cmd[1] = r;
        cmd[2] = t;
        cmd[3] = c;
    };
    if (threadIdx.x < 32) {
        uint32_t cmd[4];
        claim(cmd);
        if (threadIdx.x == 0)
            for (int k = 0; k < 4; ++k) s_cmd[k] = cmd[k];
    }
    __syncthreads();
    for (;;) {
        const uint32_t st = s_cmd[0], r = s_cmd[1], t = s_cmd[2], c = s_cmd[3];
        if (st >= 2) break;
        if (st == 0) {
            if (r != cur) {
                G = load_graph(L.graphs + r);
                stage_graph(L, G, s);
                __syncthreads();
                cur = r;
            }
            if (threadIdx.x < G.threads) run_chunk<UPT, PIPE>(L, G, r, s, zc, t, c, pol_stream, pol_keep);
            __threadfence();
        }
        uint32_t next[4] = {0u, 0u, 0u, 0u};
        if (threadIdx.x < 32) {
            claim(next);
            if (next[0] == 1) __nanosleep(2000);
        }
        __syncthreads();  // every thread's share of the current chunk is done and fenced; all read s_cmd
        if (threadIdx.x == 0) {
            if (st == 0) complete_chunk(L, Q, r, t);
            for (int k = 0; k < 4; ++k) s_cmd[k] = next[k];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- ingest, stress, debug

// Local node ids -> global ids (node_off of the step's graph added); a local
// id outside its graph's node range raises BERR_NODE_RANGE.
__global__ void globalize_kernel(uint32_t* __restrict__ step_node, const uint64_t* __restrict__ path_off,
                                 uint32_t P, const uint32_t* __restrict__ path_graph,
                                 const uint64_t* __restrict__ graph_node_off, uint64_t S, uint32_t* err) {
    uint32_t bad = 0;
    for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < S;
         s += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t p = find_path(path_off, P, s);
        const uint32_t g = path_graph[p];
        const uint64_t lo = graph_node_off[g], n = graph_node_off[g + 1] - lo;
        const uint32_t v = step_node[s];
        if ((uint64_t)v >= n) {
            bad = BERR_NODE_RANGE;
            continue;
        }
        step_node[s] = (uint32_t)(lo + v);
    }
    if (bad) atomicOr(err, bad);
}

struct BatchStress {
    const StepRec* steps;
    const uint64_t* path_off;    // [P + 1]
    const uint64_t* sample_off;  // [P + 1]
    const uint2* path_info;      // [P] (graph index, local path id)
    const NodeRec* nodes;
    uint64_t n_samples;
    uint32_t P;
    uint32_t key0, key1;
    int pf64;                    // 64-byte L2 prefetch hint: bit 0 step loads, bit 1 node loads
    double* per_graph;           // [G][3]: sum, sum of squares, count
};

// Eq. 2 per graph: sample q of the graph's local path p draws Philox counter
// (q, 0x80000000 | p, 0) under the stress seed, the same pairs as the
// one-graph stress kernel on that graph alone.
__global__ void batch_stress_kernel(BatchStress L) {
    const uint64_t pol_stream = policy_evict_first(), pol_keep = policy_evict_last();
    const uint64_t nthr = (uint64_t)gridDim.x * blockDim.x;
    uint32_t p = 0;
    uint64_t s_lo = 0, s_hi = 0;  // sample range of path p (empty until the first search)
    uint32_t cur_g = 0xffffffffu;
    double ps = 0.0, pq = 0.0, pc = 0.0;
    for (uint64_t Q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; Q < L.n_samples; Q += nthr) {
        if (Q >= s_hi || Q < s_lo) {
            p = find_path(L.sample_off, L.P, Q);
            s_lo = L.sample_off[p];
            s_hi = L.sample_off[p + 1];
        }
        const uint2 info = L.path_info[p];
        const uint64_t q = Q - s_lo;
        const uint64_t off = L.path_off[p];
        const uint64_t n = L.path_off[p + 1] - off;
        const uint4 w = philox4x32_10(make_uint4((uint32_t)q, (uint32_t)(q >> 32), 0x80000000u | info.y, 0u),
                                      L.key0, L.key1);
        const uint64_t i = mulhi64((uint64_t)w.x | ((uint64_t)w.y << 32), n);
        const uint64_t x = mulhi64(((uint64_t)w.w << 32) | (w.z & ~15u), n - 1);
        const uint64_t j = x + (x >= i);
        const uint32_t ei = w.z & 1u, ej = (w.z >> 1) & 1u;
        const StepRec si = load_step(L.steps + off + i, pol_stream, L.pf64 & 1);
        const StepRec sj = load_step(L.steps + off + j, pol_stream, L.pf64 & 1);
        const int64_t pa = endpoint_pos(si, ei), pb = endpoint_pos(sj, ej);
        const int64_t d = pa > pb ? pa - pb : pb - pa;
        if (d == 0) continue;
        const NodeRec na = load_node(L.nodes + step_node(si), pol_keep, L.pf64 & 2);
        const NodeRec nb = load_node(L.nodes + step_node(sj), pol_keep, L.pf64 & 2);
        const float xa = ei ? na.ex : na.sx, ya = ei ? na.ey : na.sy;
        const float xb = ej ? nb.ex : nb.sx, yb = ej ? nb.ey : nb.sy;
        const float dx = __ll2float_rn((int64_t)si.ax - (int64_t)sj.ax) + (xa - xb);
        const float dy = ya - yb;
        const float df = __ll2float_rn(d);
        const float tq = (sqrtf(dx * dx + dy * dy) - df) / df;
        const float term = tq * tq;
        if (info.x != cur_g) {
            if (cur_g != 0xffffffffu) {
                atomicAdd(L.per_graph + 3 * (uint64_t)cur_g, ps);
                atomicAdd(L.per_graph + 3 * (uint64_t)cur_g + 1, pq);
                atomicAdd(L.per_graph + 3 * (uint64_t)cur_g + 2, pc);
            }
            cur_g = info.x;
            ps = pq = pc = 0.0;
        }
        ps += (double)term;
        pq += (double)term * (double)term;
        pc += 1.0;
    }
    if (cur_g != 0xffffffffu) {
        atomicAdd(L.per_graph + 3 * (uint64_t)cur_g, ps);
        atomicAdd(L.per_graph + 3 * (uint64_t)cur_g + 1, pq);
        atomicAdd(L.per_graph + 3 * (uint64_t)cur_g + 2, pc);
    }
}

// The pairs that updates [u_begin, u_begin + count) of iteration t of the
// graph of rank r draw, in the graph's own step and path numbering.
__global__ void batch_debug_sample_kernel(BatchLaunch L, uint32_t max_paths, uint32_t r, uint32_t t,
                                          uint64_t u_begin, uint64_t count, pgsgd_sample* out) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ZipfConsts zc;
    const BatchSmem s = batch_smem(smem, max_paths);
    const BatchGraph G = load_graph(L.graphs + r);
    stage_theta(L, s, zc);
    stage_graph(L, G, s);
    __syncthreads();
    const SamplerArgs a = graph_sampler(L, G, t, zc);
    const PathTable pt{s.off, s.B, s.T, s.guide, G.n_paths, 63};
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < count;
         q += (uint64_t)gridDim.x * blockDim.x) {
        const Pair pr = draw_pair(a, pt, u_begin + q);
        pgsgd_sample o;
        o.g = pr.g;
        o.i = pr.i;
        o.j = pr.j;
        o.path = pr.path;
        o.cooling = (uint8_t)pr.cooling;
        o.e_i = (pr.w2 >> 2) & 1u;
        o.e_j = (pr.w2 >> 3) & 1u;
        o.d_ref = 0;
        if (pr.short_path) {
            o.skip = 1;
        } else {
            const StepRec si = a.steps[pr.base + pr.i], sj = a.steps[pr.base + pr.j];
            const int64_t pa = endpoint_pos(si, o.e_i), pb = endpoint_pos(sj, o.e_j);
            o.d_ref = pa > pb ? pa - pb : pb - pa;
            o.skip = o.d_ref == 0 ? 2 : 0;
        }
        out[q] = o;
    }
}

template <class K>
cudaError_t allow_smem(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace
}  // namespace pgsgd

using namespace pgsgd;

// The state behind a pgsgd_batch handle.
struct pgsgd_batch {
    pgsgd_graph* g = nullptr;       // the concatenated graphs (global node ids)
    uint32_t n_graphs = 0;
    std::vector<uint64_t> node_off;  // [G + 1]
    std::vector<uint32_t> path_off;  // [G + 1] graph -> first path
    std::vector<uint64_t> n_steps;   // [G]
    std::vector<int64_t> max_nt;     // [G] longest path in nucleotides
    uint32_t max_paths = 0;          // most paths of one graph

    // options
    int mode = 0;
    int cuda_graph = 1;
    int block = 256;
    int upt = 2;
    int64_t chunk = 16384;
    int64_t max_concurrent = -1;
    int updates_per_step = 10;
    int64_t timeout_ms = 10000;
    int timing = 0;
    int stall_test = 0;
    int blocks_per_sm = 0;
    int pipeline = 0;
    int pf64 = 7;

    // device state
    BatchGraph* d_graphs = nullptr;
    float* d_eta = nullptr;
    size_t eta_cap = 0;
    uint2* d_lanes = nullptr;
    size_t lanes_cap = 0;
    unsigned long long* d_q = nullptr;
    uint32_t* d_done = nullptr;
    uint32_t* d_misc = nullptr;       // [0] finished, [1] error bits
    uint64_t* d_sample_off = nullptr;
    uint2* d_path_info = nullptr;
    double* d_per_graph = nullptr;
    void* d_debug = nullptr;
    size_t debug_bytes = 0;
    uint32_t stress_sps = 0;
    std::vector<uint64_t> stress_samples;  // [G] samples per graph at stress_sps

    // the current plan (rank order)
    std::vector<uint32_t> rank_to_graph;
    std::vector<BatchGraph> plan;
    std::vector<uint32_t> lane_start;  // [G + 1] first lane of every rank

    // captured iteration loop
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::string exec_key;

    // timing
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    bool ev_pending = false;
    double timing_ms = 0.0;
    uint64_t timing_launches = 0, timing_updates = 0;
    uint64_t last_launches = 0;
    int last_grid = 0;
};

namespace {

int fail(int status, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return report_error(status, "%s", buf);
}

#define BCK(call, what)                                                                         \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return fail(PGSGD_ECUDA, "%s: %s", what, cudaGetErrorString(e_)); \
    } while (0)

cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

template <class T>
int dev_alloc(T** p, size_t n) {
    if (cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(PGSGD_ENOMEM, "device allocation of %zu bytes failed", n * sizeof(T));
    }
    return PGSGD_OK;
}

void free_batch(pgsgd_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    cudaFree(b->d_graphs);
    cudaFree(b->d_eta);
    cudaFree(b->d_lanes);
    cudaFree(b->d_q);
    cudaFree(b->d_done);
    cudaFree(b->d_misc);
    cudaFree(b->d_sample_off);
    cudaFree(b->d_path_info);
    cudaFree(b->d_per_graph);
    cudaFree(b->d_debug);
    free_graph(b->g);
    delete b;
}

// Plan shared by pgsgd_batch_plan and the layout: chunks, in-flight chunk cap
// and threads per lane of every graph, and the rank order: the longest lanes
// first (a lane's sequential rounds of updates: its updates, at most
// ceil(chunks / lanes) chunks, over threads x upt), ties by most updates, then
// graph index, so that the lanes a concurrency cap makes long start in the
// first wave instead of extending the iteration at its end.
int make_plan(uint32_t G, const uint64_t* n_updates, const uint64_t* n_nodes, int block, int upt, uint64_t chunk,
              int64_t max_concurrent, uint32_t* rank_to_graph, uint32_t* n_chunks, uint32_t* lanes,
              uint32_t* threads) {
    if (block < 64 || block > 256 || block % 32) return fail(PGSGD_EINVAL, "block %d not in 64..256 step 32", block);
    if (upt != 1 && upt != 2 && upt != 4) return fail(PGSGD_EINVAL, "updates per thread %d not 1, 2 or 4", upt);
    if (chunk == 0 || chunk > (1ull << 31)) return fail(PGSGD_EINVAL, "chunk %llu not in 1..2^31",
                                                        (unsigned long long)chunk);
    if (max_concurrent < -1) return fail(PGSGD_EINVAL, "max_concurrent %lld < -1", (long long)max_concurrent);
    const uint64_t per_block = (uint64_t)block * upt;
    for (uint32_t gi = 0; gi < G; ++gi) {
        const uint64_t nc = (n_updates[gi] + chunk - 1) / chunk;
        if (nc >= (1ull << 32) - 1) return fail(PGSGD_ERANGE, "graph %u: %llu chunks per iteration", gi,
                                               (unsigned long long)nc);
        n_chunks[gi] = (uint32_t)nc;
        uint64_t active;
        uint32_t thr = (uint32_t)block;
        if (max_concurrent == 0) {
            active = nc;
        } else {
            const uint64_t cap = max_concurrent > 0 ? (uint64_t)max_concurrent
                                                    : default_in_flight_cap(n_nodes[gi], n_updates[gi]);
            active = std::max<uint64_t>(1, cap / per_block);
            // below one block's worth: one chunk at a time on whole warps of the block
            if (cap < per_block) thr = (uint32_t)std::max<uint64_t>(32, cap / (uint64_t)upt / 32 * 32);
        }
        lanes[gi] = (uint32_t)std::min<uint64_t>(std::max<uint64_t>(active, 1), std::max<uint64_t>(nc, 1));
        if (nc == 0) lanes[gi] = 0;
        threads[gi] = thr;
    }
    std::vector<uint64_t> rounds(G, 0);
    for (uint32_t gi = 0; gi < G; ++gi) {
        if (!lanes[gi]) continue;
        const uint64_t per_trip = (uint64_t)threads[gi] * upt;
        const uint64_t per_lane = std::min<uint64_t>(n_updates[gi], (n_chunks[gi] + lanes[gi] - 1) / lanes[gi] * chunk);
        rounds[gi] = (per_lane + per_trip - 1) / per_trip;
    }
    std::vector<uint32_t> order(G);
    std::iota(order.begin(), order.end(), 0u);
    std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) {
        return rounds[a] != rounds[b] ? rounds[a] > rounds[b] : n_updates[a] > n_updates[b];
    });
    for (uint32_t r = 0; r < G; ++r) rank_to_graph[r] = order[r];
    return PGSGD_OK;
}

template <int UPT, bool PIPE>
cudaError_t launch_lanes(const BatchLaunch& L, uint32_t max_paths, uint32_t t, const uint2* lanes, uint32_t n,
                         int block, size_t smem, cudaStream_t st) {
    batch_lane_kernel<UPT, PIPE><<<n, block, smem, st>>>(L, max_paths, t, lanes);
    return cudaGetLastError();
}

cudaError_t launch_lanes_upt(int upt, bool pipe, const BatchLaunch& L, uint32_t max_paths, uint32_t t,
                             const uint2* lanes, uint32_t n, int block, size_t smem, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    if (pipe) {
        if (upt == 1) return launch_lanes<1, true>(L, max_paths, t, lanes, n, block, smem, st);
        if (upt == 4) return launch_lanes<4, true>(L, max_paths, t, lanes, n, block, smem, st);
        return launch_lanes<2, true>(L, max_paths, t, lanes, n, block, smem, st);
    }
    if (upt == 1) return launch_lanes<1, false>(L, max_paths, t, lanes, n, block, smem, st);
    if (upt == 4) return launch_lanes<4, false>(L, max_paths, t, lanes, n, block, smem, st);
    return launch_lanes<2, false>(L, max_paths, t, lanes, n, block, smem, st);
}

template <int UPT, bool PIPE>
cudaError_t persistent_launch(const BatchLaunch& L, uint32_t max_paths, const BatchQueues& Q, int block, size_t smem,
                              int sm_count, int per_sm_opt, int* grid, cudaStream_t st) {
    int nb = 0;
    cudaError_t e =
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_persistent_kernel<UPT, PIPE>, block, smem);
    if (e != cudaSuccess) return e;
    if (nb < 1) nb = 1;
    if (per_sm_opt > 0 && per_sm_opt < nb) nb = per_sm_opt;
    *grid = nb * sm_count;
    batch_persistent_kernel<UPT, PIPE><<<*grid, block, smem, st>>>(L, max_paths, Q);
    return cudaGetLastError();
}

cudaError_t launch_persistent_upt(int upt, bool pipe, const BatchLaunch& L, uint32_t max_paths,
                                  const BatchQueues& Q, int block, size_t smem, int sm_count, int per_sm_opt,
                                  int* grid, cudaStream_t st) {
    if (pipe) {
        if (upt == 1) return persistent_launch<1, true>(L, max_paths, Q, block, smem, sm_count, per_sm_opt, grid, st);
        if (upt == 4) return persistent_launch<4, true>(L, max_paths, Q, block, smem, sm_count, per_sm_opt, grid, st);
        return persistent_launch<2, true>(L, max_paths, Q, block, smem, sm_count, per_sm_opt, grid, st);
    }
    if (upt == 1) return persistent_launch<1, false>(L, max_paths, Q, block, smem, sm_count, per_sm_opt, grid, st);
    if (upt == 4) return persistent_launch<4, false>(L, max_paths, Q, block, smem, sm_count, per_sm_opt, grid, st);
    return persistent_launch<2, false>(L, max_paths, Q, block, smem, sm_count, per_sm_opt, grid, st);
}

cudaError_t set_batch_smem(size_t smem) {
    cudaError_t e;
#define PGSGD_ALLOW(k)                       \
    e = allow_smem(k, smem);                 \
    if (e != cudaSuccess) return e;
    PGSGD_ALLOW((batch_lane_kernel<1, false>))
    PGSGD_ALLOW((batch_lane_kernel<2, false>))
    PGSGD_ALLOW((batch_lane_kernel<4, false>))
    PGSGD_ALLOW((batch_lane_kernel<1, true>))
    PGSGD_ALLOW((batch_lane_kernel<2, true>))
    PGSGD_ALLOW((batch_lane_kernel<4, true>))
    PGSGD_ALLOW((batch_persistent_kernel<1, false>))
    PGSGD_ALLOW((batch_persistent_kernel<2, false>))
    PGSGD_ALLOW((batch_persistent_kernel<4, false>))
    PGSGD_ALLOW((batch_persistent_kernel<1, true>))
    PGSGD_ALLOW((batch_persistent_kernel<2, true>))
    PGSGD_ALLOW((batch_persistent_kernel<4, true>))
    PGSGD_ALLOW(batch_debug_sample_kernel)
#undef PGSGD_ALLOW
    return cudaSuccess;
}

// Zheng et al.'s annealing with graph-specific eta_max (eta_t of Algorithm 1).
void default_schedule(double eta_max, uint32_t T, float* out) {
    const double emin = 0.01;
    if (T == 1) {
        out[0] = (float)eta_max;
        return;
    }
    const double lambda = std::log(eta_max / emin) / (double)(T - 1);
    for (uint32_t t = 0; t < T; ++t) out[t] = (float)(eta_max * std::exp(-lambda * (double)t));
}

int check_graph_open(const pgsgd_batch* b) {
    if (!b) return fail(PGSGD_EINVAL, "batch is NULL");
    return PGSGD_OK;
}

}  // namespace

extern "C" {

int pgsgd_batch_plan(uint32_t n_graphs, const uint64_t* n_updates, const uint64_t* n_nodes, int block, int upt,
                     uint64_t chunk, int64_t max_concurrent, uint32_t* rank_to_graph, uint32_t* n_chunks,
                     uint32_t* lanes, uint32_t* threads) {
    if (n_graphs && (!n_updates || !n_nodes || !rank_to_graph || !n_chunks || !lanes || !threads))
        return fail(PGSGD_EINVAL, "NULL argument");
    return make_plan(n_graphs, n_updates, n_nodes, block, upt, chunk, max_concurrent, rank_to_graph, n_chunks,
                     lanes, threads);
}

int pgsgd_batch_create(uint32_t n_graphs, const uint64_t* graph_node_off, const uint64_t* graph_path_off,
                       const uint32_t* node_len, const uint64_t* path_off, const uint32_t* step_node,
                       const uint8_t* step_rev, const int64_t* step_pos, int on_device, void* cuda_stream,
                       pgsgd_batch** out) {
    if (!out) return fail(PGSGD_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_graphs == 0) return fail(PGSGD_EINVAL, "n_graphs is 0");
    if (!graph_node_off || !graph_path_off || !node_len || !path_off)
        return fail(PGSGD_EINVAL, "graph_node_off, graph_path_off, node_len and path_off are required");
    if (graph_node_off[0] != 0 || graph_path_off[0] != 0)
        return fail(PGSGD_EINVAL, "graph_node_off[0] and graph_path_off[0] must be 0");
    for (uint32_t k = 0; k < n_graphs; ++k) {
        if (graph_node_off[k + 1] < graph_node_off[k]) return fail(PGSGD_EINVAL, "graph_node_off decreases at %u", k);
        if (graph_path_off[k + 1] < graph_path_off[k]) return fail(PGSGD_EINVAL, "graph_path_off decreases at %u", k);
        if (graph_path_off[k + 1] - graph_path_off[k] > kMaxPaths)
            return fail(PGSGD_ERANGE, "graph %u has %llu paths > %u", k,
                        (unsigned long long)(graph_path_off[k + 1] - graph_path_off[k]), kMaxPaths);
    }
    const uint64_t V = graph_node_off[n_graphs], P = graph_path_off[n_graphs];
    if (V == 0 || V >= (1ull << 31)) return fail(PGSGD_ERANGE, "total nodes %llu not in 1..2^31-1",
                                                (unsigned long long)V);
    if (P == 0 || P > kMaxBatchPaths) return fail(PGSGD_ERANGE, "total paths %llu not in 1..%u",
                                                 (unsigned long long)P, kMaxBatchPaths);
    cudaStream_t st = S(cuda_stream);
    // path -> graph, and the path offsets on the host
    std::vector<uint32_t> path_graph(P);
    for (uint32_t k = 0; k < n_graphs; ++k)
        for (uint64_t p = graph_path_off[k]; p < graph_path_off[k + 1]; ++p) path_graph[p] = k;
    std::vector<uint64_t> h_off(P + 1);
    if (on_device)
        BCK(cudaMemcpy(h_off.data(), path_off, (P + 1) * 8, cudaMemcpyDeviceToHost), "path_off readback");
    else
        std::memcpy(h_off.data(), path_off, (P + 1) * 8);
    if (h_off[0] != 0) return fail(PGSGD_EINVAL, "path_off[0] must be 0");
    for (uint64_t p = 0; p < P; ++p)
        if (h_off[p + 1] < h_off[p]) return fail(PGSGD_EINVAL, "path_off decreases at %llu", (unsigned long long)p);
    const uint64_t S_total = h_off[P];
    if (S_total && (!step_node || !step_rev || !step_pos)) return fail(PGSGD_EINVAL, "step arrays are required");

    // local -> global node ids
    pgsgd_graph* g = nullptr;
    int rc;
    if (!on_device) {
        std::vector<uint32_t> gn(S_total);
        for (uint64_t p = 0; p < P; ++p) {
            const uint32_t k = path_graph[p];
            const uint64_t lo = graph_node_off[k], n = graph_node_off[k + 1] - lo;
            for (uint64_t s = h_off[p]; s < h_off[p + 1]; ++s) {
                if ((uint64_t)step_node[s] >= n)
                    return fail(PGSGD_EINVAL, "step %llu of graph %u: node %u outside the graph's %llu nodes",
                                (unsigned long long)s, k, step_node[s], (unsigned long long)n);
                gn[s] = (uint32_t)(lo + step_node[s]);
            }
        }
        rc = graph_create(node_len, (uint32_t)V, path_off, (uint32_t)P, gn.data(), step_rev, step_pos, 0,
                          cuda_stream, true, &g);
        if (rc) return rc;
    } else {
        uint32_t *d_node = nullptr, *d_pg = nullptr, *d_err = nullptr;
        uint64_t* d_gno = nullptr;
        auto cleanup = [&]() {
            cudaFree(d_node);
            cudaFree(d_pg);
            cudaFree(d_err);
            cudaFree(d_gno);
        };
        if ((rc = dev_alloc(&d_node, S_total)) || (rc = dev_alloc(&d_pg, P)) || (rc = dev_alloc(&d_err, 1)) ||
            (rc = dev_alloc(&d_gno, (size_t)n_graphs + 1))) {
            cleanup();
            return rc;
        }
        cudaError_t e = cudaMemcpyAsync(d_node, step_node, S_total * 4, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_pg, path_graph.data(), P * 4, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_gno, graph_node_off, ((size_t)n_graphs + 1) * 8, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, 4, st);
        int dev = 0, sms = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess && S_total) {
            const uint64_t want = (S_total + 255) / 256;
            const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)sms * 16));
            globalize_kernel<<<grid, 256, 0, st>>>(d_node, path_off, (uint32_t)P, d_pg, d_gno, S_total, d_err);
            e = cudaGetLastError();
        }
        uint32_t h_err = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, d_err, 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            cleanup();
            return fail(PGSGD_ECUDA, "batch ingest: %s", cudaGetErrorString(e));
        }
        if (h_err) {
            cleanup();
            return fail(PGSGD_EINVAL, "a step's node id lies outside its graph's node range");
        }
        rc = graph_create(node_len, (uint32_t)V, path_off, (uint32_t)P, d_node, step_rev, step_pos, 1, cuda_stream,
                          true, &g);
        cleanup();
        if (rc) return rc;
    }

    pgsgd_batch* b = new pgsgd_batch;
    b->g = g;
    b->n_graphs = n_graphs;
    b->node_off.assign(graph_node_off, graph_node_off + n_graphs + 1);
    b->path_off.resize(n_graphs + 1);
    b->n_steps.resize(n_graphs);
    b->max_nt.resize(n_graphs);
    for (uint32_t k = 0; k <= n_graphs; ++k) b->path_off[k] = (uint32_t)graph_path_off[k];
    std::vector<uint2> info(P);
    for (uint32_t k = 0; k < n_graphs; ++k) {
        const uint32_t p0 = b->path_off[k], p1 = b->path_off[k + 1];
        b->n_steps[k] = h_off[p1] - h_off[p0];
        int64_t m = 0;
        for (uint32_t p = p0; p < p1; ++p) {
            m = std::max(m, g->h_path_nt[p]);
            info[p] = make_uint2(k, p - p0);
        }
        b->max_nt[k] = m;
        b->max_paths = std::max(b->max_paths, p1 - p0);
    }
    if ((rc = dev_alloc(&b->d_graphs, n_graphs)) || (rc = dev_alloc(&b->d_q, n_graphs)) ||
        (rc = dev_alloc(&b->d_done, n_graphs)) || (rc = dev_alloc(&b->d_misc, 2)) ||
        (rc = dev_alloc(&b->d_sample_off, P + 1)) || (rc = dev_alloc(&b->d_path_info, P)) ||
        (rc = dev_alloc(&b->d_per_graph, (size_t)n_graphs * 3))) {
        free_batch(b);
        return rc;
    }
    cudaError_t e = cudaMemcpy(b->d_path_info, info.data(), P * sizeof(uint2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev1);
    if (e == cudaSuccess) e = set_batch_smem(batch_smem_bytes(b->max_paths));
    if (e != cudaSuccess) {
        free_batch(b);
        return fail(PGSGD_ECUDA, "batch setup: %s", cudaGetErrorString(e));
    }
    *out = b;
    return PGSGD_OK;
}

int pgsgd_batch_destroy(pgsgd_batch* b) {
    free_batch(b);
    return PGSGD_OK;
}

int pgsgd_batch_set_option(pgsgd_batch* b, int option, int64_t v) {
    int rc = check_graph_open(b);
    if (rc) return rc;
    switch (option) {
    case PGSGD_BOPT_MODE:
        if (v < 0 || v > 2) return fail(PGSGD_EINVAL, "mode %lld not 0, 1 or 2", (long long)v);
        b->mode = (int)v;
        break;
    case PGSGD_BOPT_CUDA_GRAPH: b->cuda_graph = v != 0; break;
    case PGSGD_BOPT_BLOCK:
        if (v < 64 || v > 256 || v % 32) return fail(PGSGD_EINVAL, "block %lld not in 64..256 step 32", (long long)v);
        b->block = (int)v;
        break;
    case PGSGD_BOPT_UPDATES_PER_THREAD:
        if (v != 1 && v != 2 && v != 4) return fail(PGSGD_EINVAL, "updates per thread %lld not 1, 2 or 4", (long long)v);
        b->upt = (int)v;
        break;
    case PGSGD_BOPT_CHUNK:
        if (v < 1 || v > (1ll << 31)) return fail(PGSGD_EINVAL, "chunk %lld not in 1..2^31", (long long)v);
        b->chunk = v;
        break;
    case PGSGD_BOPT_MAX_CONCURRENT:
        if (v < -1) return fail(PGSGD_EINVAL, "max_concurrent %lld < -1", (long long)v);
        b->max_concurrent = v;
        break;
    case PGSGD_BOPT_UPDATES_PER_STEP:
        if (v < 1 || v > 1000) return fail(PGSGD_EINVAL, "updates_per_step %lld not in 1..1000", (long long)v);
        b->updates_per_step = (int)v;
        break;
    case PGSGD_BOPT_TIMEOUT_MS:
        if (v < 1 || v > 3600000) return fail(PGSGD_EINVAL, "timeout %lld ms not in 1..3600000", (long long)v);
        b->timeout_ms = v;
        break;
    case PGSGD_BOPT_TIMING: b->timing = v != 0; break;
    case PGSGD_BOPT_STALL_TEST: b->stall_test = v != 0; break;
    case PGSGD_BOPT_BLOCKS_PER_SM:
        if (v < 0 || v > 32) return fail(PGSGD_EINVAL, "blocks per SM %lld not in 0..32", (long long)v);
        b->blocks_per_sm = (int)v;
        break;
    case PGSGD_BOPT_PIPELINE: b->pipeline = v != 0; break;
    case PGSGD_BOPT_PREFETCH64:
        if (v < 0 || v > 15) return fail(PGSGD_EINVAL, "prefetch option %lld not in 0..15", (long long)v);
        b->pf64 = (int)v;
        break;
    default: return fail(PGSGD_EINVAL, "unknown batch option %d", option);
    }
    return PGSGD_OK;
}

int pgsgd_batch_get_option(const pgsgd_batch* b, int option, int64_t* v) {
    if (!b || !v) return fail(PGSGD_EINVAL, "NULL argument");
    switch (option) {
    case PGSGD_BOPT_MODE: *v = b->mode; break;
    case PGSGD_BOPT_CUDA_GRAPH: *v = b->cuda_graph; break;
    case PGSGD_BOPT_BLOCK: *v = b->block; break;
    case PGSGD_BOPT_UPDATES_PER_THREAD: *v = b->upt; break;
    case PGSGD_BOPT_CHUNK: *v = b->chunk; break;
    case PGSGD_BOPT_MAX_CONCURRENT: *v = b->max_concurrent; break;
    case PGSGD_BOPT_UPDATES_PER_STEP: *v = b->updates_per_step; break;
    case PGSGD_BOPT_TIMEOUT_MS: *v = b->timeout_ms; break;
    case PGSGD_BOPT_TIMING: *v = b->timing; break;
    case PGSGD_BOPT_STALL_TEST: *v = b->stall_test; break;
    case PGSGD_BOPT_BLOCKS_PER_SM: *v = b->blocks_per_sm; break;
    case PGSGD_BOPT_PIPELINE: *v = b->pipeline; break;
    case PGSGD_BOPT_PREFETCH64: *v = b->pf64; break;
    default: return fail(PGSGD_EINVAL, "unknown batch option %d", option);
    }
    return PGSGD_OK;
}

int pgsgd_batch_info_get(const pgsgd_batch* b, pgsgd_batch_info* out) {
    if (!b || !out) return fail(PGSGD_EINVAL, "NULL argument");
    out->n_graphs = b->n_graphs;
    out->n_nodes = b->g->n_nodes;
    out->n_paths = b->g->n_paths;
    out->max_graph_paths = b->max_paths;
    out->n_steps = b->g->n_steps;
    out->device_bytes = b->g->device_bytes;
    out->last_launches = b->last_launches;
    out->last_grid = b->last_grid;
    return PGSGD_OK;
}

int pgsgd_batch_set_coords(pgsgd_batch* b, const double* xy, int on_device, void* cuda_stream) {
    int rc = check_graph_open(b);
    if (rc) return rc;
    // fixed anchors: the batch kernels never rebase
    return pgsgd_set_coords(b->g, xy, on_device, cuda_stream);
}

int pgsgd_batch_get_coords(pgsgd_batch* b, double* xy, int on_device, void* cuda_stream) {
    int rc = check_graph_open(b);
    if (rc) return rc;
    return pgsgd_get_coords(b->g, xy, on_device, cuda_stream);
}

}  // extern "C"

namespace {

// Rank order, chunks and lanes for the current options; uploads the graph
// table (keys and all) and the lane table.
int prepare(pgsgd_batch* b, const uint64_t* seeds, cudaStream_t st) {
    const uint32_t G = b->n_graphs;
    std::vector<uint64_t> nu(G), nn(G);
    for (uint32_t k = 0; k < G; ++k) {
        nu[k] = (uint64_t)b->updates_per_step * b->n_steps[k];
        nn[k] = b->node_off[k + 1] - b->node_off[k];
    }
    std::vector<uint32_t> r2g(G), nch(G), lanes(G), thr(G);
    int rc = make_plan(G, nu.data(), nn.data(), b->block, b->upt, (uint64_t)b->chunk, b->max_concurrent, r2g.data(),
                       nch.data(), lanes.data(), thr.data());
    if (rc) return rc;
    b->rank_to_graph = r2g;
    b->plan.assign(G, BatchGraph{});
    b->lane_start.assign(G + 1, 0);
    for (uint32_t r = 0; r < G; ++r) {
        const uint32_t k = r2g[r];
        BatchGraph& x = b->plan[r];
        x.path0 = b->path_off[k];
        x.n_paths = b->path_off[k + 1] - b->path_off[k];
        x.step0 = x.n_paths ? b->g->h_path_off[x.path0] : 0;
        x.n_steps = b->n_steps[k];
        x.n_updates = nu[k];
        x.n_chunks = nch[k];
        x.max_active = lanes[k];
        x.threads = thr[k];
        x.key0 = (uint32_t)seeds[k];
        x.key1 = (uint32_t)(seeds[k] >> 32);
        b->lane_start[r + 1] = b->lane_start[r] + lanes[k];
    }
    const uint32_t n_lanes = b->lane_start[G];
    if (n_lanes > b->lanes_cap) {
        cudaFree(b->d_lanes);
        b->d_lanes = nullptr;
        b->lanes_cap = 0;
        if ((rc = dev_alloc(&b->d_lanes, n_lanes))) return rc;
        b->lanes_cap = n_lanes;
        b->exec_key.clear();  // the captured graph holds the old pointer
    }
    std::vector<uint2> lt(n_lanes);
    for (uint32_t r = 0; r < G; ++r)
        for (uint32_t k = b->lane_start[r]; k < b->lane_start[r + 1]; ++k) lt[k] = make_uint2(r, k - b->lane_start[r]);
    BCK(cudaMemcpyAsync(b->d_graphs, b->plan.data(), G * sizeof(BatchGraph), cudaMemcpyHostToDevice, st),
        "graph table upload");
    if (n_lanes)
        BCK(cudaMemcpyAsync(b->d_lanes, lt.data(), n_lanes * sizeof(uint2), cudaMemcpyHostToDevice, st),
            "lane table upload");
    BCK(cudaStreamSynchronize(st), "plan upload");
    return PGSGD_OK;
}

}  // namespace

extern "C" {

int pgsgd_batch_layout(pgsgd_batch* b, uint32_t iter_max, const double* eta, double theta, const uint64_t* seeds,
                       uint32_t iter_begin, uint32_t iter_end, void* cuda_stream) {
    int rc = check_graph_open(b);
    if (rc) return rc;
    if (!seeds) return fail(PGSGD_EINVAL, "seeds is NULL");
    if (!b->g->has_coords) return fail(PGSGD_EINVAL, "no layout: call pgsgd_batch_set_coords first");
    if (iter_max == 0) return fail(PGSGD_EINVAL, "iter_max is 0");
    if (iter_begin > iter_end || iter_end > iter_max) return fail(PGSGD_EINVAL, "need iter_begin <= iter_end <= iter_max");
    if (!(theta >= 0.0 && theta <= 4.0)) return fail(PGSGD_EINVAL, "theta %g not in [0, 4]", theta);
    const uint32_t G = b->n_graphs;
    if (eta)
        for (size_t e = 0; e < (size_t)G * iter_max; ++e)
            if (!(std::isfinite(eta[e]) && eta[e] >= 0.0))
                return fail(PGSGD_EINVAL, "learning rate %g of graph %zu at iteration %zu is not finite and >= 0",
                            eta[e], e / iter_max, e % iter_max);
    if (iter_begin == iter_end) return PGSGD_OK;
    cudaStream_t st = S(cuda_stream);
    const float th = (float)theta;
    if ((rc = ensure_zipf(b->g, th, st))) return rc;
    if ((rc = prepare(b, seeds, st))) return rc;

    // learning rates [rank][iter_max]
    const size_t ne = (size_t)G * iter_max;
    if (ne > b->eta_cap) {
        cudaFree(b->d_eta);
        b->d_eta = nullptr;
        b->eta_cap = 0;
        if ((rc = dev_alloc(&b->d_eta, ne))) return rc;
        b->eta_cap = ne;
        b->exec_key.clear();
    }
    std::vector<float> h_eta(ne);
    for (uint32_t r = 0; r < G; ++r) {
        const uint32_t k = b->rank_to_graph[r];
        float* row = h_eta.data() + (size_t)r * iter_max;
        if (eta) {
            for (uint32_t t = 0; t < iter_max; ++t) row[t] = (float)eta[(size_t)k * iter_max + t];
        } else {
            const double emax = (double)b->max_nt[k] * (double)b->max_nt[k];
            default_schedule(emax > 0 ? emax : 1.0, iter_max, row);
        }
    }
    BCK(cudaMemcpyAsync(b->d_eta, h_eta.data(), ne * sizeof(float), cudaMemcpyHostToDevice, st), "eta upload");

    BatchLaunch L;
    L.graphs = b->d_graphs;
    L.eta = b->d_eta;
    L.steps = b->g->d_steps;
    L.path_off = b->g->d_path_off;
    L.zipf_B = b->g->d_zipf_B;
    L.zipf_T = b->g->d_zipf_T;
    L.nodes = b->g->d_nodes;
    L.chunk = (uint64_t)b->chunk;
    L.n_graphs = G;
    L.T = iter_max;
    L.iter_begin = iter_begin;
    L.iter_end = iter_end;
    L.theta = th;
    L.store_mode = 1;
    L.pf64 = b->pf64 & 3;
    L.timeout_ns = (uint64_t)b->timeout_ms * 1000000ull;
    const size_t smem = batch_smem_bytes(b->max_paths);
    const uint32_t n_lanes = b->lane_start[G];
    uint64_t updates = 0;
    for (uint32_t r = 0; r < G; ++r) updates += b->plan[r].n_updates;
    updates *= (iter_end - iter_begin);

    if (b->timing) {
        if (b->ev_pending) {
            double ms = 0;
            uint64_t l = 0, u = 0;
            if ((rc = pgsgd_batch_timing_read(b, &ms, &l, &u, 0))) return rc;
        }
        BCK(cudaEventRecord(b->ev0, st), "timing event");
    }
    uint64_t launches = 0;
    if (b->mode == 1) {
        // queues: iteration iter_begin open on every graph with work
        std::vector<unsigned long long> q(G);
        uint32_t idle = 0;
        for (uint32_t r = 0; r < G; ++r) {
            if (b->plan[r].n_chunks == 0) {
                q[r] = (unsigned long long)iter_end << 32;
                ++idle;
            } else {
                q[r] = (unsigned long long)iter_begin << 32;
            }
        }
        std::vector<uint32_t> done(G, 0);
        if (b->stall_test && G) done[0] = 0xffffffffu;  // rank 0 can never complete an iteration
        const uint32_t misc[2] = {idle, 0};
        BCK(cudaMemcpyAsync(b->d_q, q.data(), G * 8, cudaMemcpyHostToDevice, st), "queue upload");
        BCK(cudaMemcpyAsync(b->d_done, done.data(), G * 4, cudaMemcpyHostToDevice, st), "queue upload");
        BCK(cudaMemcpyAsync(b->d_misc, misc, 8, cudaMemcpyHostToDevice, st), "queue upload");
        BatchQueues Q{b->d_q, b->d_done, b->d_misc, b->d_misc + 1};
        int grid = 0;
        const cudaError_t e = launch_persistent_upt(b->upt, b->pipeline != 0, L, b->max_paths, Q, b->block, smem,
                                                    b->g->sm_count, b->blocks_per_sm, &grid, st);
        BCK(e, "persistent batch kernel");
        b->last_grid = grid;
        launches = 1;
    } else {
        const bool capture = b->cuda_graph != 0;
        char key[256];
        snprintf(key, sizeof key, "%d/%u/%u/%u/%d/%d/%lld/%.9g/%p/%p/%u/%d/%d", b->mode, iter_max, iter_begin,
                 iter_end, b->block, b->upt, (long long)b->chunk, (double)th, (void*)b->d_eta, (void*)b->d_lanes,
                 n_lanes, b->pipeline, b->pf64);
        // the lane table and per-rank lane ranges are part of the replayed work
        std::string k2 = key;
        for (uint32_t r = 0; r <= G; ++r) k2 += "," + std::to_string(b->lane_start[r]);
        auto enqueue = [&](cudaStream_t s) -> cudaError_t {
            for (uint32_t t = iter_begin; t < iter_end; ++t) {
                if (b->mode == 0) {
                    cudaError_t e = launch_lanes_upt(b->upt, b->pipeline != 0, L, b->max_paths, t, b->d_lanes, n_lanes,
                                                     b->block, smem, s);
                    if (e != cudaSuccess) return e;
                } else {
                    for (uint32_t r = 0; r < G; ++r) {
                        const uint32_t n = b->lane_start[r + 1] - b->lane_start[r];
                        cudaError_t e = launch_lanes_upt(b->upt, b->pipeline != 0, L, b->max_paths, t,
                                                         b->d_lanes + b->lane_start[r], n, b->block, smem, s);
                        if (e != cudaSuccess) return e;
                    }
                }
            }
            return cudaSuccess;
        };
        for (uint32_t t = iter_begin; t < iter_end; ++t) {
            if (b->mode == 0) launches += n_lanes ? 1 : 0;
            else
                for (uint32_t r = 0; r < G; ++r) launches += b->lane_start[r + 1] > b->lane_start[r] ? 1 : 0;
        }
        if (capture) {
            if (b->exec_key != k2) {
                if (b->exec) {
                    cudaGraphExecDestroy(b->exec);
                    b->exec = nullptr;
                }
                b->exec_key.clear();
                cudaGraph_t graph = nullptr;
                BCK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
                cudaError_t e = enqueue(b->cap_stream);
                cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &graph);
                if (e != cudaSuccess || e2 != cudaSuccess) {
                    if (graph) cudaGraphDestroy(graph);
                    return fail(PGSGD_ECUDA, "iteration-loop capture: %s",
                                cudaGetErrorString(e != cudaSuccess ? e : e2));
                }
                e = cudaGraphInstantiate(&b->exec, graph, 0);
                cudaGraphDestroy(graph);
                BCK(e, "graph instantiate");
                b->exec_key = k2;
            }
            BCK(cudaGraphLaunch(b->exec, st), "graph launch");
        } else {
            BCK(enqueue(st), "batch kernel");
        }
        b->last_grid = b->mode == 0 ? (int)n_lanes : 0;
    }
    if (b->timing) {
        BCK(cudaEventRecord(b->ev1, st), "timing event");
        b->ev_pending = true;
        b->timing_launches += launches;
        b->timing_updates += updates;
    }
    b->last_launches = launches;
    if (b->mode == 1) {
        uint32_t err = 0;
        BCK(cudaMemcpyAsync(&err, b->d_misc + 1, 4, cudaMemcpyDeviceToHost, st), "queue status readback");
        BCK(cudaStreamSynchronize(st), "persistent batch kernel");
        if (err & BERR_TIMEOUT)
            return fail(PGSGD_ETIMEOUT, "persistent batch kernel: no claimable work for %lld ms; queues stuck",
                        (long long)b->timeout_ms);
    }
    return PGSGD_OK;
}

int pgsgd_batch_timing_read(pgsgd_batch* b, double* total_ms, uint64_t* launches, uint64_t* updates, int reset) {
    if (!b) return fail(PGSGD_EINVAL, "batch is NULL");
    if (b->ev_pending) {
        BCK(cudaEventSynchronize(b->ev1), "timing sync");
        float ms = 0.f;
        BCK(cudaEventElapsedTime(&ms, b->ev0, b->ev1), "timing read");
        b->timing_ms += ms;
        b->ev_pending = false;
    }
    if (total_ms) *total_ms = b->timing_ms;
    if (launches) *launches = b->timing_launches;
    if (updates) *updates = b->timing_updates;
    if (reset) {
        b->timing_ms = 0.0;
        b->timing_launches = 0;
        b->timing_updates = 0;
    }
    return PGSGD_OK;
}

int pgsgd_batch_stress(pgsgd_batch* b, uint32_t samples_per_step, uint64_t seed, pgsgd_stress_result* out,
                       void* cuda_stream) {
    int rc = check_graph_open(b);
    if (rc) return rc;
    if (!out) return fail(PGSGD_EINVAL, "out is NULL");
    if (!b->g->has_coords) return fail(PGSGD_EINVAL, "no layout: call pgsgd_batch_set_coords first");
    if (samples_per_step == 0) return fail(PGSGD_EINVAL, "samples_per_step is 0");
    cudaStream_t st = S(cuda_stream);
    const uint32_t G = b->n_graphs, P = b->g->n_paths;
    const std::vector<uint64_t>& off = b->g->h_path_off;
    if (b->stress_sps != samples_per_step) {
        std::vector<uint64_t> so(P + 1, 0);
        b->stress_samples.assign(G, 0);
        for (uint32_t k = 0; k < G; ++k)
            for (uint32_t p = b->path_off[k]; p < b->path_off[k + 1]; ++p) {
                const uint64_t n = off[p + 1] - off[p];
                const uint64_t m = n >= 2 ? (uint64_t)samples_per_step * n : 0;
                so[p + 1] = so[p] + m;
                b->stress_samples[k] += m;
            }
        BCK(cudaMemcpyAsync(b->d_sample_off, so.data(), (P + 1) * 8, cudaMemcpyHostToDevice, st), "sample table");
        BCK(cudaStreamSynchronize(st), "sample table");
        b->stress_sps = samples_per_step;
    }
    uint64_t n_samples = 0;
    for (uint64_t m : b->stress_samples) n_samples += m;
    BCK(cudaMemsetAsync(b->d_per_graph, 0, (size_t)G * 3 * 8, st), "stress clear");
    if (n_samples) {
        BatchStress L;
        L.steps = b->g->d_steps;
        L.path_off = b->g->d_path_off;
        L.sample_off = b->d_sample_off;
        L.path_info = b->d_path_info;
        L.nodes = b->g->d_nodes;
        L.n_samples = n_samples;
        L.P = P;
        L.key0 = (uint32_t)seed;
        L.key1 = (uint32_t)(seed >> 32);
        L.pf64 = (b->pf64 >> 2) & 3;
        L.per_graph = b->d_per_graph;
        const uint64_t want = (n_samples + 255) / 256;
        const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)b->g->sm_count * 16));
        batch_stress_kernel<<<grid, 256, 0, st>>>(L);
        BCK(cudaGetLastError(), "batch stress kernel");
    }
    std::vector<double> h((size_t)G * 3);
    BCK(cudaMemcpyAsync(h.data(), b->d_per_graph, h.size() * 8, cudaMemcpyDeviceToHost, st), "stress readback");
    BCK(cudaStreamSynchronize(st), "stress sync");
    for (uint32_t k = 0; k < G; ++k) {
        const double n = h[3 * k + 2];
        const double mean = n > 0 ? h[3 * k] / n : 0.0;
        const double var = n > 1 ? std::max(0.0, (h[3 * k + 1] - n * mean * mean) / (n - 1.0)) : 0.0;
        const double sd = std::sqrt(var);
        const double half = n > 0 ? 1.96 * sd / std::sqrt(n) : 0.0;
        out[k].mean = mean;
        out[k].stddev = sd;
        out[k].ci_lo = mean - half;
        out[k].ci_hi = mean + half;
        out[k].n_valid = (uint64_t)n;
        out[k].n_skipped = b->stress_samples[k] - (uint64_t)n;
    }
    return PGSGD_OK;
}

int pgsgd_batch_debug_sample(pgsgd_batch* b, uint32_t graph, uint32_t t, uint32_t iter_max, double theta,
                             uint64_t seed, uint64_t u_begin, uint64_t count, pgsgd_sample* out, void* cuda_stream) {
    int rc = check_graph_open(b);
    if (rc) return rc;
    if (!out && count) return fail(PGSGD_EINVAL, "out is NULL");
    if (graph >= b->n_graphs) return fail(PGSGD_EINVAL, "graph %u >= %u", graph, b->n_graphs);
    if (iter_max == 0 || t >= iter_max) return fail(PGSGD_EINVAL, "need t < iter_max");
    if (!(theta >= 0.0 && theta <= 4.0)) return fail(PGSGD_EINVAL, "theta %g not in [0, 4]", theta);
    if (count == 0) return PGSGD_OK;
    cudaStream_t st = S(cuda_stream);
    const float th = (float)theta;
    if ((rc = ensure_zipf(b->g, th, st))) return rc;
    // a one-graph table holding only this graph's key
    BatchGraph x{};
    x.path0 = b->path_off[graph];
    x.n_paths = b->path_off[graph + 1] - x.path0;
    x.step0 = x.n_paths ? b->g->h_path_off[x.path0] : 0;
    x.n_steps = b->n_steps[graph];
    x.key0 = (uint32_t)seed;
    x.key1 = (uint32_t)(seed >> 32);
    if (x.n_steps == 0) return fail(PGSGD_EINVAL, "graph %u has no steps", graph);
    const size_t bytes = count * sizeof(pgsgd_sample) + 64;
    if (bytes > b->debug_bytes) {
        cudaFree(b->d_debug);
        b->d_debug = nullptr;
        b->debug_bytes = 0;
        unsigned char* p = nullptr;
        if ((rc = dev_alloc(&p, bytes))) return rc;
        b->d_debug = p;
        b->debug_bytes = bytes;
    }
    BatchGraph* d_x = reinterpret_cast<BatchGraph*>(b->d_debug);
    pgsgd_sample* d_out = reinterpret_cast<pgsgd_sample*>(reinterpret_cast<unsigned char*>(b->d_debug) + 64);
    BCK(cudaMemcpyAsync(d_x, &x, sizeof x, cudaMemcpyHostToDevice, st), "debug upload");
    BatchLaunch L{};
    L.graphs = d_x;
    L.steps = b->g->d_steps;
    L.path_off = b->g->d_path_off;
    L.zipf_B = b->g->d_zipf_B;
    L.zipf_T = b->g->d_zipf_T;
    L.n_graphs = 1;
    L.T = iter_max;
    L.theta = th;
    const uint64_t want = (count + 255) / 256;
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)b->g->sm_count * 8));
    batch_debug_sample_kernel<<<grid, 256, batch_smem_bytes(b->max_paths), st>>>(L, b->max_paths, 0, t, u_begin,
                                                                                 count, d_out);
    BCK(cudaGetLastError(), "batch debug sample kernel");
    BCK(cudaMemcpyAsync(out, d_out, count * sizeof(pgsgd_sample), cudaMemcpyDeviceToHost, st), "debug readback");
    BCK(cudaStreamSynchronize(st), "debug sync");
    return PGSGD_OK;
}

}  // extern "C"
