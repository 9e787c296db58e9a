// CUDA kernels of the PG-SGD path for GB300 (sm_103a): graph ingest and
// validation, the lock-free update kernel of Algorithm 1, the sampled
// path-stress kernel of Eq. 2, coordinate conversion and anchor upkeep, and
// the debug kernels that expose the sampler and a Jacobi sweep for parity
// checks.
//
// The path is random gathers and scatters over HBM (Section III-B: memory
// bound, no dense contraction), so there are no tensor cores here. An update
// reads two 16-byte step records (streamed, evict-first in L2) and two
// 16-byte node records (the L2-resident working set, evict-last), and writes
// back 8 bytes of each node with an atomic exchange at L2.
#include "../../include/pgsgd.h"
#include "pgsgd_internal.h"

namespace pgsgd {

namespace {

constexpr uint32_t kPackStagedPaths = 16384;  // 128 KiB of path offsets in shared memory

// ---------------------------------------------------------------- ingest

__global__ void check_lengths_kernel(const uint32_t* __restrict__ node_len, uint32_t n, uint32_t* flags) {
    uint32_t bad = 0;
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x)
        if (node_len[v] == 0) bad |= FLAG_ZERO_LEN;
    if (bad) atomicOr(flags, bad);
}

__global__ void pack_steps_kernel(const uint32_t* __restrict__ step_node,
                                  const uint8_t* __restrict__ step_rev,
                                  const int64_t* __restrict__ step_pos,
                                  const uint32_t* __restrict__ node_len, uint32_t n_nodes,
                                  const uint64_t* __restrict__ path_off, uint32_t P, uint64_t S,
                                  StepRec* __restrict__ steps, uint32_t* flags) {
    // path offsets staged in shared memory unless there are too many paths
    extern __shared__ uint64_t s_off[];
    const bool staged = P <= kPackStagedPaths;
    if (staged)
        for (uint32_t k = threadIdx.x; k <= P; k += blockDim.x) s_off[k] = path_off[k];
    __syncthreads();
    const uint64_t* off = staged ? s_off : path_off;
    uint32_t bad = 0;
    for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < S;
         s += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t p = find_path(off, P, s);
        const bool first = s == off[p];
        const bool last = s + 1 == off[p + 1];
        const uint32_t nd = step_node[s];
        const uint32_t rv = step_rev[s];
        const int64_t ps = step_pos[s];
        const bool nd_ok = nd < n_nodes;
        if (!nd_ok) bad |= FLAG_BAD_NODE;
        if (rv > 1) bad |= FLAG_BAD_REV;
        if (ps < 0 || ps >= (int64_t)(1ll << 32)) bad |= FLAG_POS_RANGE;
        if (first && ps != 0) bad |= FLAG_BAD_POS;
        const uint32_t len = nd_ok ? node_len[nd] : 0u;
        if (!last && nd_ok && step_pos[s + 1] != ps + (int64_t)len) bad |= FLAG_BAD_POS;
        StepRec r;
        r.nr = (nd & 0x7fffffffu) | ((rv & 1u) << 31);
        r.pos = (uint32_t)ps;
        r.len = len;
        r.ax = 0;
        steps[s] = r;
    }
    if (bad) atomicOr(flags, bad);
}

__global__ void path_extent_kernel(const StepRec* __restrict__ steps, const uint64_t* __restrict__ path_off,
                                   uint32_t P, int64_t* __restrict__ out_nt) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const uint64_t a = path_off[p], b = path_off[p + 1];
    if (a == b) { out_nt[p] = 0; return; }
    const StepRec s = steps[b - 1];
    out_nt[p] = (int64_t)s.pos + (int64_t)s.len;
}

// ---------------------------------------------------------------- coordinates and anchors

__global__ void set_coords_kernel(const double* __restrict__ xy, NodeRec* __restrict__ nodes,
                                  int32_t* __restrict__ anchor, uint32_t n, int anchored,
                                  uint32_t* flags) {
    uint32_t bad = 0;
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x) {
        const double sx = xy[4 * v], sy = xy[4 * v + 1], ex = xy[4 * v + 2], ey = xy[4 * v + 3];
        if (!isfinite(sx) || !isfinite(sy) || !isfinite(ex) || !isfinite(ey)) bad |= FLAG_COORD_NAN;
        int32_t ax = 0;
        if (anchored) {
            // anchor x only where FP32 would lose sub-nucleotide resolution;
            // below 4096 the FP32 value itself is kept exactly
            const double lim = 1073741824.0;  // 2^30
            if (fabs(sx) >= lim || fabs(ex) >= lim) bad |= FLAG_COORD_RANGE;
            else ax = fabs(sx) >= 4096.0 ? (int32_t)rint(sx) : 0;
        }
        anchor[v] = ax;
        NodeRec r;
        r.sx = (float)(sx - ax);
        r.sy = (float)sy;
        r.ex = (float)(ex - ax);
        r.ey = (float)ey;
        nodes[v] = r;
    }
    if (bad) atomicOr(flags, bad);
}

__global__ void get_coords_kernel(const NodeRec* __restrict__ nodes, const int32_t* __restrict__ anchor,
                                  double* __restrict__ xy, uint32_t n) {
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x) {
        const NodeRec r = nodes[v];
        const double ax = (double)anchor[v];
        xy[4 * v] = ax + (double)r.sx;
        xy[4 * v + 1] = (double)r.sy;
        xy[4 * v + 2] = ax + (double)r.ex;
        xy[4 * v + 3] = (double)r.ey;
    }
}

// Move a node's x anchor to its rounded start point once the start offset
// has drifted past 8, so offsets stay small: an FP32 offset below 8 resolves
// 1e-6 nt. Subtracting an integer within half a unit of sx leaves sx exact.
// Sets *changed when any anchor moved.
__global__ void rebase_kernel(NodeRec* __restrict__ nodes, int32_t* __restrict__ anchor, uint32_t n,
                              uint32_t* changed) {
    int any = 0;
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x) {
        NodeRec r = nodes[v];
        if (fabsf(r.sx) > 8.0f) {
            const float sh = rintf(r.sx);
            const int64_t na = (int64_t)anchor[v] + (int64_t)sh;
            if (na > -(1ll << 30) && na < (1ll << 30)) {
                anchor[v] = (int32_t)na;
                r.sx -= sh;
                r.ex -= sh;
                nodes[v] = r;
                any = 1;
            }
        }
    }
    if (__syncthreads_or(any) && threadIdx.x == 0) atomicOr(changed, 1u);
}

// Copy every node's current anchor into the step records that visit it; does
// nothing unless *changed is set.
__global__ void refresh_anchors_kernel(StepRec* __restrict__ steps, const int32_t* __restrict__ anchor,
                                       uint64_t S, const uint32_t* __restrict__ changed) {
    if (*changed == 0) return;
    for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < S;
         s += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t nd = steps[s].nr & 0x7fffffffu;
        steps[s].ax = anchor[nd];
    }
}

// ---------------------------------------------------------------- Zipf per theta

// Per-theta tables: B[p] = H(n_p - 1/2) for every path, and the acceptance
// thresholds T[k] = H(k + 1/2) - h(k) for k < 256 (T[0] unused).
__global__ void zipf_setup_kernel(const uint64_t* __restrict__ path_off, uint32_t P, float theta,
                                  float* __restrict__ out_B, float* __restrict__ out_T) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    const float omt = __fsub_rn(1.0f, theta);
    if (p < P) {
        const uint64_t n = path_off[p + 1] - path_off[p];
        out_B[p] = n >= 2 ? zipf_B(n - 1, omt) : 0.0f;
    }
    if (p < (uint32_t)kZipfTable) out_T[p] = p == 0 ? 0.0f : zipf_threshold(p, omt, theta);
}

// ---------------------------------------------------------------- update math

// (stage_paths and pair_move live in pgsgd_device.cuh)

// ---------------------------------------------------------------- the update kernel

// One launch = one iteration's N updates (or a slice), grid-stride over the
// update index u; every loop trip is one update_trip of UPT updates (PIPE:
// the software-pipelined loop, drawing the next trip while this trip's step
// records load).
template <int UPT, int MINB, bool PIPE>
__global__ void __launch_bounds__(256, MINB) update_kernel(UpdateLaunch L) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ZipfConsts zc;
    const PathTable pt = stage_paths(L.s, smem, zc);
    SamplerArgs a = L.s;
    a.zc = zc;
    const uint64_t pol_stream = L.l2_hints ? policy_evict_first() : 0;
    const uint64_t pol_keep = L.l2_hints ? policy_evict_last() : 0;
    const uint64_t nthr = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t gtid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const UpdateOpts o{L.eta, L.store_mode, L.pf64, L.atomic};
    const uint64_t u_end = L.u_begin + L.n_updates;
    if (PIPE) {
        update_range_pipelined<UPT>(a, pt, L.nodes, L.u_begin + gtid, nthr, u_end, o, pol_stream, pol_keep);
    } else {
        for (uint64_t base = L.u_begin + gtid; base < u_end; base += nthr * UPT)
            update_trip<UPT>(a, pt, L.nodes, base, nthr, u_end, o, pol_stream, pol_keep);
    }
}

// The update kernel with the step-record reads made asynchronous: every
// thread keeps the step records of its next D updates in flight, copied
// global -> shared memory by cp.async (16 bytes each, evict-first, 64-byte
// prefetch hint) into slots of its own, so an outstanding read costs shared
// memory instead of registers. A trip waits for its oldest group, reads the
// two records from its slots, loads the two points and moves them as
// finish_trip does, then draws the update D trips ahead and issues its reads
// into the freed slots. Same updates per thread (u_begin + gtid + m * nthr),
// same draws and moves as update_kernel<1, MINB, false>. Slots: after the
// staged path tables, [D][2][blockDim] 16-byte records (16-byte aligned).
__device__ __forceinline__ void cp_async_step(StepRec* dst, const StepRec* src, uint64_t pol) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global.L2::cache_hint.L2::64B [%0], [%1], 16, %2;"
                 :: "r"(d), "l"(src), "l"(pol) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory"); }

__host__ __device__ inline size_t async_slots_offset(uint32_t n_paths, uint32_t n_guide) {
    return (update_smem_bytes(n_paths, n_guide) + 15) & ~(size_t)15;
}

template <int D, int MINB>
__global__ void __launch_bounds__(256, MINB) update_kernel_async(UpdateLaunch L) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ZipfConsts zc;
    const PathTable pt = stage_paths(L.s, smem, zc);
    SamplerArgs a = L.s;
    a.zc = zc;
    StepRec* slots = reinterpret_cast<StepRec*>(smem + async_slots_offset(L.s.n_paths, L.s.n_guide));
    const uint32_t B = blockDim.x, tid = threadIdx.x;
    const uint64_t pol_stream = L.l2_hints ? policy_evict_first() : 0;
    const uint64_t pol_keep = L.l2_hints ? policy_evict_last() : 0;
    const uint64_t nthr = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t u_first = L.u_begin + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t u_end = L.u_begin + L.n_updates;
    const UpdateOpts o{L.eta, L.store_mode, L.pf64, L.atomic};
    // per slot: the coin word of its update, or 0xffffffff when the slot holds no update
    uint32_t w2s[D];
    auto issue = [&](int k, uint64_t u) {
        w2s[k] = 0xffffffffu;
        if (u < u_end) {
            const Pair pr = draw_pair(a, pt, u);
            if (!pr.short_path) {
                w2s[k] = pr.w2 & 0xfu;  // the coins are bits 0-3
                cp_async_step(slots + (2 * k) * B + tid, a.steps + pr.base + pr.i, pol_stream);
                cp_async_step(slots + (2 * k + 1) * B + tid, a.steps + pr.base + pr.j, pol_stream);
            }
        }
        cp_async_commit();  // one group per slot, empty or not, so the group count stays exact
    };
#pragma unroll
    for (int k = 0; k < D; ++k) issue(k, u_first + (uint64_t)k * nthr);
    for (uint64_t base = u_first; base < u_end; base += (uint64_t)D * nthr) {
#pragma unroll
        for (int k = 0; k < D; ++k) {
            cp_async_wait<D - 1>();  // slot k's group (the oldest) has landed
            if (w2s[k] != 0xffffffffu) {
                TripDraws<1> d;
                d.act[0] = true;
                d.w2[0] = w2s[k];
                d.gi[0] = d.gj[0] = 0;
                StepRec si[1], sj[1];
                si[0] = slots[(2 * k) * B + tid];
                sj[0] = slots[(2 * k + 1) * B + tid];
                finish_trip<1>(L.nodes, d, si, sj, o, pol_keep);
            }
            issue(k, base + (uint64_t)(k + D) * nthr);
        }
    }
    cp_async_wait<0>();
}

// Warp merging (Section V-B3): the update kernel with one cooling coin per
// group of 32 updates, shared by shuffle. The loop bound is the warp's first
// update so all 32 lanes run every trip (u_begin is a multiple of 32).
template <int UPT>
__global__ void __launch_bounds__(256, 1) update_kernel_wm(UpdateLaunch L) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ZipfConsts zc;
    const PathTable pt = stage_paths(L.s, smem, zc);
    SamplerArgs a = L.s;
    a.zc = zc;
    const uint64_t pol_stream = L.l2_hints ? policy_evict_first() : 0;
    const uint64_t pol_keep = L.l2_hints ? policy_evict_last() : 0;
    const uint64_t nthr = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t gtid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t lane = threadIdx.x & 31u;
    const UpdateOpts o{L.eta, L.store_mode, L.pf64, L.atomic};
    const uint64_t u_end = L.u_begin + L.n_updates;
    for (uint64_t base = L.u_begin + gtid; base - lane < u_end; base += nthr * UPT)
        update_trip_wm<UPT>(a, pt, L.nodes, base, nthr, u_end, o, pol_stream, pol_keep);
}

// Warp-level data reuse (Section VII-D): n_updates = selections, each doing
// R updates (reuse_range).
template <int R>
__global__ void __launch_bounds__(256, 1) update_reuse_kernel(UpdateLaunch L) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ZipfConsts zc;
    const PathTable pt = stage_paths(L.s, smem, zc);
    SamplerArgs a = L.s;
    a.zc = zc;
    const uint64_t pol_stream = L.l2_hints ? policy_evict_first() : 0;
    const uint64_t pol_keep = L.l2_hints ? policy_evict_last() : 0;
    const uint64_t nthr = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t gtid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    reuse_range<R>(a, pt, L.nodes, L.u_begin + gtid, nthr, L.u_begin + L.n_updates, L.eta, L.wm, L.pf64, pol_stream,
                   pol_keep);
}

// ---------------------------------------------------------------- debug kernels

__global__ void debug_sample_kernel(SamplerArgs a0, uint64_t u_begin, uint64_t count, pgsgd_sample* out) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ZipfConsts zc;
    const PathTable pt = stage_paths(a0, smem, zc);
    SamplerArgs a = a0;
    a.zc = zc;
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < count;
         q += (uint64_t)gridDim.x * blockDim.x) {
        const Pair pr = draw_pair_any(a, pt, u_begin + q);
        pgsgd_sample r;
        r.g = pr.g; r.i = pr.i; r.j = pr.j; r.path = pr.path;
        r.cooling = (uint8_t)pr.cooling;
        r.e_i = (pr.w2 >> 2) & 1u;
        r.e_j = (pr.w2 >> 3) & 1u;
        r.d_ref = 0;
        if (pr.short_path) {
            r.skip = 1;
        } else {
            const StepRec si = a.steps[pr.base + pr.i], sj = a.steps[pr.base + pr.j];
            const int64_t pa = endpoint_pos(si, r.e_i), pb = endpoint_pos(sj, r.e_j);
            r.d_ref = pa > pb ? pa - pb : pb - pa;
            r.skip = r.d_ref == 0 ? 2 : 0;
        }
        out[q] = r;
    }
}

__global__ void debug_sweep_kernel(SamplerArgs a0, uint64_t u_begin, uint64_t count,
                                   const NodeRec* __restrict__ nodes, float eta, float4* out) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ZipfConsts zc;
    const PathTable pt = stage_paths(a0, smem, zc);
    SamplerArgs a = a0;
    a.zc = zc;
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < count;
         q += (uint64_t)gridDim.x * blockDim.x) {
        const Pair pr = draw_pair_any(a, pt, u_begin + q);
        float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
        if (!pr.short_path) {
            const StepRec si = a.steps[pr.base + pr.i], sj = a.steps[pr.base + pr.j];
            const NodeRec na = nodes[step_node(si)], nb = nodes[step_node(sj)];
            const uint32_t ea = (pr.w2 >> 2) & 1u, eb = (pr.w2 >> 3) & 1u;
            const int64_t pa = endpoint_pos(si, ea), pb = endpoint_pos(sj, eb);
            const int64_t d = pa > pb ? pa - pb : pb - pa;
            if (d != 0) {
                const Move m = pair_move(na, si.ax, ea, nb, sj.ax, eb, d, eta);
                if (m.moved) o = make_float4(m.dxi, m.dyi, m.dxj, m.dyj);
            }
        }
        out[q] = o;
    }
}

// The R pairs of every selection q in [q_begin, q_begin + count) under data
// reuse, computed from scratch (no shuffles): out[(q - q_begin) R + k].
__global__ void debug_sample_reuse_kernel(SamplerArgs a0, uint32_t R, uint64_t n_sel, uint64_t q_begin,
                                          uint64_t count, pgsgd_sample* out) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ZipfConsts zc;
    const PathTable pt = stage_paths(a0, smem, zc);
    SamplerArgs a = a0;
    a.zc = zc;
    for (uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; c < count * R;
         c += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t q = q_begin + c / R;
        const uint32_t k = (uint32_t)(c % R);
        const uint64_t grp = q >> 5;
        const uint32_t p = group_path(a, pt, grp);
        const uint64_t qm = (grp << 5) | (((uint32_t)q + reuse_offset(a, grp, k)) & 31u);
        const uint4 wq = pair_block(a, q), wm = pair_block(a, qm);
        const Selection mine = draw_selection(a, pt, q, p, wq, a.wm ? group_coin(a, q) : (wq.z & 1u));
        const Selection other = draw_selection(a, pt, qm, p, wm, a.wm ? group_coin(a, qm) : (wm.z & 1u));
        const uint64_t base = pt.off[p];
        pgsgd_sample r;
        r.g = base + mine.i;
        r.i = mine.i;
        r.j = other.j;
        r.path = p;
        r.cooling = (uint8_t)other.cooling;
        r.e_i = (mine.w2 >> 2) & 1u;
        r.e_j = (other.w2 >> 3) & 1u;
        r.d_ref = 0;
        r.skip = 0;
        if (!(mine.valid && other.valid && q < n_sel && qm < n_sel)) {
            r.skip = 1;
        } else {
            const StepRec si = a.steps[base + mine.i], sj = a.steps[base + other.j];
            const int64_t pa = endpoint_pos(si, r.e_i), pb = endpoint_pos(sj, r.e_j);
            r.d_ref = pa > pb ? pa - pb : pb - pa;
            r.skip = r.d_ref == 0 ? 2 : 0;
        }
        out[c] = r;
    }
}

// ---------------------------------------------------------------- sampled stress

// Block reduction of (sum, squares, count) in a fixed order: warp shuffles,
// then warp 0; the block's totals go to partials[3 * blockIdx.x ..].
__device__ __forceinline__ void block_sums_to_partials(double sum, double sq, double cnt, double* partials) {
    __shared__ double red[3][32];
    for (int off = 16; off > 0; off >>= 1) {
        sum += __shfl_down_sync(0xffffffffu, sum, off);
        sq += __shfl_down_sync(0xffffffffu, sq, off);
        cnt += __shfl_down_sync(0xffffffffu, cnt, off);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { red[0][warp] = sum; red[1][warp] = sq; red[2][warp] = cnt; }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        sum = lane < nw ? red[0][lane] : 0.0;
        sq = lane < nw ? red[1][lane] : 0.0;
        cnt = lane < nw ? red[2][lane] : 0.0;
        for (int off = 16; off > 0; off >>= 1) {
            sum += __shfl_down_sync(0xffffffffu, sum, off);
            sq += __shfl_down_sync(0xffffffffu, sq, off);
            cnt += __shfl_down_sync(0xffffffffu, cnt, off);
        }
        if (lane == 0) {
            partials[3 * (uint64_t)blockIdx.x] = sum;
            partials[3 * (uint64_t)blockIdx.x + 1] = sq;
            partials[3 * (uint64_t)blockIdx.x + 2] = cnt;
        }
    }
}

template <int SPT>
__global__ void stress_kernel(StressLaunch L) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* s_soff = reinterpret_cast<uint64_t*>(smem);   // [P + 1] sample offsets
    uint64_t* s_poff = s_soff + L.n_paths + 1;              // [P + 1] step offsets
    for (uint32_t k = threadIdx.x; k <= L.n_paths; k += blockDim.x) {
        s_soff[k] = L.sample_off[k];
        s_poff[k] = L.path_off[k];
    }
    __syncthreads();
    const uint64_t pol_stream = policy_evict_first();
    const uint64_t pol_keep = policy_evict_last();
    const uint64_t nthr = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t gtid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    double sum = 0.0, sq = 0.0, cnt = 0.0;
    // running per-path sums, flushed to global when the path changes
    uint32_t cur_p = 0xffffffffu;
    double ps = 0.0, pq = 0.0, pc = 0.0;
    for (uint64_t base = gtid; base < L.n_samples; base += nthr * SPT) {
        uint32_t p[SPT];
        StepRec si[SPT], sj[SPT];
        uint32_t ei[SPT], ej[SPT];
        bool act[SPT];
#pragma unroll
        for (int k = 0; k < SPT; ++k) {
            const uint64_t Q = base + (uint64_t)k * nthr;
            act[k] = Q < L.n_samples;
            if (!act[k]) continue;
            p[k] = find_path(s_soff, L.n_paths, Q);
            const uint64_t q = Q - s_soff[p[k]];
            const uint64_t off = s_poff[p[k]];
            const uint64_t n = s_poff[p[k] + 1] - off;
            const uint32_t c2 = 0x80000000u | p[k];
            const uint4 w = philox4x32_10(make_uint4((uint32_t)q, (uint32_t)(q >> 32), c2, 0u),
                                          L.key0, L.key1);
            const uint64_t i = mulhi64((uint64_t)w.x | ((uint64_t)w.y << 32), n);
            const uint64_t x = mulhi64(((uint64_t)w.w << 32) | (w.z & ~15u), n - 1);
            const uint64_t j = x + (x >= i);
            ei[k] = w.z & 1u;
            ej[k] = (w.z >> 1) & 1u;
            si[k] = load_step(L.steps + off + i, pol_stream, L.pf64 & 1);
            sj[k] = load_step(L.steps + off + j, pol_stream, L.pf64 & 1);
        }
        NodeRec na[SPT], nb[SPT];
#pragma unroll
        for (int k = 0; k < SPT; ++k) {
            if (!act[k]) continue;
            na[k] = load_node(L.nodes + step_node(si[k]), pol_keep, L.pf64 & 2);
            nb[k] = load_node(L.nodes + step_node(sj[k]), pol_keep, L.pf64 & 2);
        }
#pragma unroll
        for (int k = 0; k < SPT; ++k) {
            if (!act[k]) continue;
            const int64_t pa = endpoint_pos(si[k], ei[k]), pb = endpoint_pos(sj[k], ej[k]);
            const int64_t d = pa > pb ? pa - pb : pb - pa;
            if (d == 0) continue;
            const float xa = ei[k] ? na[k].ex : na[k].sx, ya = ei[k] ? na[k].ey : na[k].sy;
            const float xb = ej[k] ? nb[k].ex : nb[k].sx, yb = ej[k] ? nb[k].ey : nb[k].sy;
            const float dx = __ll2float_rn((int64_t)si[k].ax - (int64_t)sj[k].ax) + (xa - xb);
            const float dy = ya - yb;
            const float df = __ll2float_rn(d);
            const float t = (sqrtf(dx * dx + dy * dy) - df) / df;
            const float term = t * t;
            sum += (double)term;
            sq += (double)term * (double)term;
            cnt += 1.0;
            if (L.per_path) {
                if (p[k] != cur_p) {
                    if (cur_p != 0xffffffffu) {
                        atomicAdd(L.per_path + 3 * (uint64_t)cur_p, ps);
                        atomicAdd(L.per_path + 3 * (uint64_t)cur_p + 1, pq);
                        atomicAdd(L.per_path + 3 * (uint64_t)cur_p + 2, pc);
                    }
                    cur_p = p[k]; ps = pq = pc = 0.0;
                }
                ps += (double)term; pq += (double)term * (double)term; pc += 1.0;
            }
        }
    }
    if (L.per_path && cur_p != 0xffffffffu) {
        atomicAdd(L.per_path + 3 * (uint64_t)cur_p, ps);
        atomicAdd(L.per_path + 3 * (uint64_t)cur_p + 1, pq);
        atomicAdd(L.per_path + 3 * (uint64_t)cur_p + 2, pc);
    }
    block_sums_to_partials(sum, sq, cnt, L.partials);
}

// The sampled-stress kernel with the step-record reads made asynchronous, as
// in update_kernel_async: every thread keeps the step records of its next D
// samples in flight (cp.async into slots of its own in shared memory), then
// reads the two node records (read-only here) and adds the term. Same
// samples in the same per-thread order as stress_kernel, so the same sums.
// Slots: after the two staged offset tables, [D][2][blockDim] records.
template <int D>
__global__ void __launch_bounds__(256) stress_kernel_async(StressLaunch L) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* s_soff = reinterpret_cast<uint64_t*>(smem);   // [P + 1] sample offsets
    uint64_t* s_poff = s_soff + L.n_paths + 1;              // [P + 1] step offsets
    StepRec* slots = reinterpret_cast<StepRec*>(s_poff + L.n_paths + 1);  // 2 (P + 1) x 8 bytes: 16-byte aligned
    for (uint32_t k = threadIdx.x; k <= L.n_paths; k += blockDim.x) {
        s_soff[k] = L.sample_off[k];
        s_poff[k] = L.path_off[k];
    }
    __syncthreads();
    const uint32_t B = blockDim.x, tid = threadIdx.x;
    const uint64_t pol_stream = policy_evict_first();
    const uint64_t pol_keep = policy_evict_last();
    const uint64_t nthr = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t first = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    double sum = 0.0, sq = 0.0, cnt = 0.0;
    uint32_t cur_p = 0xffffffffu;
    double ps = 0.0, pq = 0.0, pc = 0.0;
    // per slot: path | endpoint coins << 30 of its sample, or 0xffffffff when empty
    uint32_t tag[D];
    auto issue = [&](int k, uint64_t Q) {
        tag[k] = 0xffffffffu;
        if (Q < L.n_samples) {
            const uint32_t p = find_path(s_soff, L.n_paths, Q);
            const uint64_t q = Q - s_soff[p];
            const uint64_t off = s_poff[p];
            const uint64_t n = s_poff[p + 1] - off;
            const uint4 w = philox4x32_10(make_uint4((uint32_t)q, (uint32_t)(q >> 32), 0x80000000u | p, 0u),
                                          L.key0, L.key1);
            const uint64_t i = mulhi64((uint64_t)w.x | ((uint64_t)w.y << 32), n);
            const uint64_t x = mulhi64(((uint64_t)w.w << 32) | (w.z & ~15u), n - 1);
            const uint64_t j = x + (x >= i);
            tag[k] = p | ((w.z & 3u) << 30);  // p < 2^14 (the path table lives in shared memory)
            cp_async_step(slots + (2 * k) * B + tid, L.steps + off + i, pol_stream);
            cp_async_step(slots + (2 * k + 1) * B + tid, L.steps + off + j, pol_stream);
        }
        cp_async_commit();
    };
#pragma unroll
    for (int k = 0; k < D; ++k) issue(k, first + (uint64_t)k * nthr);
    for (uint64_t base = first; base < L.n_samples; base += (uint64_t)D * nthr) {
#pragma unroll
        for (int k = 0; k < D; ++k) {
            cp_async_wait<D - 1>();
            const uint32_t tg = tag[k];
            if (tg != 0xffffffffu) {
                const StepRec si = slots[(2 * k) * B + tid], sj = slots[(2 * k + 1) * B + tid];
                const uint32_t p = tg & 0x3fffffffu, ei = (tg >> 30) & 1u, ej = tg >> 31;
                const int64_t pa = endpoint_pos(si, ei), pb = endpoint_pos(sj, ej);
                const int64_t d = pa > pb ? pa - pb : pb - pa;
                if (d != 0) {
                    const float2 va = load_point(L.nodes + step_node(si), ei, pol_keep, L.pf64 & 2);
                    const float2 vb = load_point(L.nodes + step_node(sj), ej, pol_keep, L.pf64 & 2);
                    const float dx = __ll2float_rn((int64_t)si.ax - (int64_t)sj.ax) + (va.x - vb.x);
                    const float dy = va.y - vb.y;
                    const float df = __ll2float_rn(d);
                    const float t = (sqrtf(dx * dx + dy * dy) - df) / df;
                    const float term = t * t;
                    sum += (double)term;
                    sq += (double)term * (double)term;
                    cnt += 1.0;
                    if (L.per_path) {
                        if (p != cur_p) {
                            if (cur_p != 0xffffffffu) {
                                atomicAdd(L.per_path + 3 * (uint64_t)cur_p, ps);
                                atomicAdd(L.per_path + 3 * (uint64_t)cur_p + 1, pq);
                                atomicAdd(L.per_path + 3 * (uint64_t)cur_p + 2, pc);
                            }
                            cur_p = p; ps = pq = pc = 0.0;
                        }
                        ps += (double)term; pq += (double)term * (double)term; pc += 1.0;
                    }
                }
            }
            issue(k, base + (uint64_t)(k + D) * nthr);
        }
    }
    cp_async_wait<0>();
    if (L.per_path && cur_p != 0xffffffffu) {
        atomicAdd(L.per_path + 3 * (uint64_t)cur_p, ps);
        atomicAdd(L.per_path + 3 * (uint64_t)cur_p + 1, pq);
        atomicAdd(L.per_path + 3 * (uint64_t)cur_p + 2, pc);
    }
    block_sums_to_partials(sum, sq, cnt, L.partials);
}

// Sum the per-block partials in a fixed order (one block of 256 threads).
__global__ void stress_finalize_kernel(const double* __restrict__ partials, int n, double* __restrict__ out3) {
    __shared__ double red[3][256];
    double s = 0.0, q = 0.0, c = 0.0;
    for (int b = threadIdx.x; b < n; b += blockDim.x) {
        s += partials[3 * b];
        q += partials[3 * b + 1];
        c += partials[3 * b + 2];
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
    if (threadIdx.x == 0) { out3[0] = red[0][0]; out3[1] = red[1][0]; out3[2] = red[2][0]; }
}

int grid_for(uint64_t work, int block, int sm_count, int per_sm) {
    uint64_t g = (work + block - 1) / block;
    const uint64_t cap = (uint64_t)sm_count * per_sm;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

size_t stress_smem_bytes(uint32_t n_paths) { return 2 * (size_t)(n_paths + 1) * sizeof(uint64_t); }

cudaError_t launch_check_lengths(const uint32_t* node_len, uint32_t n, uint32_t* flags, int sm_count,
                                 cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    check_lengths_kernel<<<grid_for(n, 256, sm_count, 16), 256, 0, st>>>(node_len, n, flags);
    return cudaGetLastError();
}

cudaError_t launch_pack_steps(const uint32_t* step_node, const uint8_t* step_rev, const int64_t* step_pos,
                              const uint32_t* node_len, uint32_t n_nodes, const uint64_t* path_off,
                              uint32_t n_paths, uint64_t n_steps, StepRec* steps, uint32_t* flags,
                              int sm_count, cudaStream_t st) {
    if (n_steps == 0) return cudaSuccess;
    const size_t smem = n_paths <= kPackStagedPaths ? (size_t)(n_paths + 1) * sizeof(uint64_t) : 0;
    cudaError_t e = cudaFuncSetAttribute(pack_steps_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    pack_steps_kernel<<<grid_for(n_steps, 256, sm_count, 8), 256, smem, st>>>(
        step_node, step_rev, step_pos, node_len, n_nodes, path_off, n_paths, n_steps, steps, flags);
    return cudaGetLastError();
}

cudaError_t launch_path_extent(const StepRec* steps, const uint64_t* path_off, uint32_t n_paths,
                               int64_t* out_nt, cudaStream_t st) {
    path_extent_kernel<<<(n_paths + 127) / 128, 128, 0, st>>>(steps, path_off, n_paths, out_nt);
    return cudaGetLastError();
}

cudaError_t launch_set_coords(const double* xy, NodeRec* nodes, int32_t* anchor, uint32_t n, int anchored,
                              uint32_t* flags, int sm_count, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    set_coords_kernel<<<grid_for(n, 256, sm_count, 16), 256, 0, st>>>(xy, nodes, anchor, n, anchored, flags);
    return cudaGetLastError();
}

cudaError_t launch_get_coords(const NodeRec* nodes, const int32_t* anchor, double* xy, uint32_t n,
                              int sm_count, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    get_coords_kernel<<<grid_for(n, 256, sm_count, 16), 256, 0, st>>>(nodes, anchor, xy, n);
    return cudaGetLastError();
}

cudaError_t launch_rebase(NodeRec* nodes, int32_t* anchor, uint32_t n, uint32_t* changed, int sm_count,
                          cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    rebase_kernel<<<grid_for(n, 256, sm_count, 16), 256, 0, st>>>(nodes, anchor, n, changed);
    return cudaGetLastError();
}

cudaError_t launch_refresh_anchors(StepRec* steps, const int32_t* anchor, uint64_t n_steps,
                                   const uint32_t* changed, int sm_count, cudaStream_t st) {
    if (n_steps == 0) return cudaSuccess;
    refresh_anchors_kernel<<<grid_for(n_steps, 256, sm_count, 8), 256, 0, st>>>(steps, anchor, n_steps,
                                                                                 changed);
    return cudaGetLastError();
}

cudaError_t launch_zipf_setup(const uint64_t* path_off, uint32_t n_paths, float theta, float* zipf_B,
                              float* zipf_T, cudaStream_t st) {
    const uint32_t n = n_paths > (uint32_t)kZipfTable ? n_paths : (uint32_t)kZipfTable;
    zipf_setup_kernel<<<(n + 127) / 128, 128, 0, st>>>(path_off, n_paths, theta, zipf_B, zipf_T);
    return cudaGetLastError();
}

// The update kernel an UpdateLaunch selects, with its dynamic shared memory.
struct UpdateKernelChoice {
    const void* fn;
    size_t smem;
};

template <class K>
static UpdateKernelChoice pick(K kernel, size_t smem) {
    return UpdateKernelChoice{reinterpret_cast<const void*>(kernel), smem};
}

static cudaError_t choose_update_kernel(const UpdateLaunch& L, UpdateKernelChoice* c) {
    const size_t smem = update_smem_bytes(L.s.n_paths, L.s.n_guide);
    if (L.async_depth > 0) {
        const size_t sa = async_slots_offset(L.s.n_paths, L.s.n_guide) +
                          (size_t)L.async_depth * 2 * L.block * sizeof(StepRec);
        switch (L.async_depth * 10 + L.minb) {
            case 24: *c = pick(update_kernel_async<2, 4>, sa); return cudaSuccess;
            case 34: *c = pick(update_kernel_async<3, 4>, sa); return cudaSuccess;
            case 44: *c = pick(update_kernel_async<4, 4>, sa); return cudaSuccess;
            case 45: *c = pick(update_kernel_async<4, 5>, sa); return cudaSuccess;
            case 64: *c = pick(update_kernel_async<6, 4>, sa); return cudaSuccess;
            case 84: *c = pick(update_kernel_async<8, 4>, sa); return cudaSuccess;
            case 43: *c = pick(update_kernel_async<4, 3>, sa); return cudaSuccess;
            default: return cudaErrorInvalidValue;
        }
    }
    if (L.drf > 1) {
        switch (L.drf) {
            case 2: *c = pick(update_reuse_kernel<2>, smem); return cudaSuccess;
            case 4: *c = pick(update_reuse_kernel<4>, smem); return cudaSuccess;
            case 8: *c = pick(update_reuse_kernel<8>, smem); return cudaSuccess;
            default: return cudaErrorInvalidValue;
        }
    }
    if (L.wm) {
        switch (L.upt) {
            case 1: *c = pick(update_kernel_wm<1>, smem); return cudaSuccess;
            case 2: *c = pick(update_kernel_wm<2>, smem); return cudaSuccess;
            case 4: *c = pick(update_kernel_wm<4>, smem); return cudaSuccess;
            default: return cudaErrorInvalidValue;
        }
    }
    if (L.pipeline) {
        switch (L.upt * 10 + L.minb) {
            case 11: *c = pick(update_kernel<1, 1, true>, smem); return cudaSuccess;
            case 13: *c = pick(update_kernel<1, 3, true>, smem); return cudaSuccess;
            case 21: *c = pick(update_kernel<2, 1, true>, smem); return cudaSuccess;
            case 22: *c = pick(update_kernel<2, 2, true>, smem); return cudaSuccess;
            case 23: *c = pick(update_kernel<2, 3, true>, smem); return cudaSuccess;
            case 41: *c = pick(update_kernel<4, 1, true>, smem); return cudaSuccess;
            case 42: *c = pick(update_kernel<4, 2, true>, smem); return cudaSuccess;
            default: return cudaErrorInvalidValue;
        }
    }
    switch (L.upt * 10 + L.minb) {
        case 11: *c = pick(update_kernel<1, 1, false>, smem); return cudaSuccess;
        case 14: *c = pick(update_kernel<1, 4, false>, smem); return cudaSuccess;
        case 16: *c = pick(update_kernel<1, 6, false>, smem); return cudaSuccess;
        case 21: *c = pick(update_kernel<2, 1, false>, smem); return cudaSuccess;
        case 23: *c = pick(update_kernel<2, 3, false>, smem); return cudaSuccess;
        case 24: *c = pick(update_kernel<2, 4, false>, smem); return cudaSuccess;
        case 41: *c = pick(update_kernel<4, 1, false>, smem); return cudaSuccess;
        case 42: *c = pick(update_kernel<4, 2, false>, smem); return cudaSuccess;
        case 43: *c = pick(update_kernel<4, 3, false>, smem); return cudaSuccess;
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_update(const UpdateLaunch& L, cudaStream_t st) {
    if (L.n_updates == 0) return cudaSuccess;
    UpdateKernelChoice c;
    cudaError_t e = choose_update_kernel(L, &c);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(c.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem);
    if (e != cudaSuccess) return e;
    void* args[] = {const_cast<UpdateLaunch*>(&L)};
    return cudaLaunchKernel(c.fn, dim3((unsigned)L.grid), dim3((unsigned)L.block), args, c.smem, st);
}

int update_blocks_per_sm(const UpdateLaunch& L) {
    UpdateKernelChoice c;
    int nb = 0;
    if (choose_update_kernel(L, &c) != cudaSuccess) return 0;
    if (cudaFuncSetAttribute(c.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, c.fn, L.block, c.smem) != cudaSuccess) return 0;
    return nb;
}

cudaError_t launch_debug_sample_reuse(const SamplerArgs& s, uint32_t R, uint64_t n_sel, uint64_t q_begin,
                                     uint64_t count, void* out, int sm_count, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    const size_t smem = update_smem_bytes(s.n_paths, s.n_guide);
    cudaError_t e = cudaFuncSetAttribute(debug_sample_reuse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    debug_sample_reuse_kernel<<<grid_for(count * R, 256, sm_count, 8), 256, smem, st>>>(
        s, R, n_sel, q_begin, count, static_cast<pgsgd_sample*>(out));
    return cudaGetLastError();
}

cudaError_t launch_debug_sample(const SamplerArgs& s, uint64_t u_begin, uint64_t count, void* out,
                                int sm_count, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    const size_t smem = update_smem_bytes(s.n_paths, s.n_guide);
    cudaError_t e = cudaFuncSetAttribute(debug_sample_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    debug_sample_kernel<<<grid_for(count, 256, sm_count, 8), 256, smem, st>>>(s, u_begin, count,
                                                                              static_cast<pgsgd_sample*>(out));
    return cudaGetLastError();
}

cudaError_t launch_debug_sweep(const SamplerArgs& s, uint64_t u_begin, uint64_t count, const NodeRec* nodes,
                               float eta, float4* out, int sm_count, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    const size_t smem = update_smem_bytes(s.n_paths, s.n_guide);
    cudaError_t e = cudaFuncSetAttribute(debug_sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    debug_sweep_kernel<<<grid_for(count, 256, sm_count, 8), 256, smem, st>>>(s, u_begin, count, nodes, eta,
                                                                             out);
    return cudaGetLastError();
}

template <int D>
static cudaError_t launch_stress_async_t(const StressLaunch& L, cudaStream_t st) {
    const size_t smem = stress_smem_bytes(L.n_paths) + (size_t)D * 2 * L.block * sizeof(StepRec);
    cudaError_t e = cudaFuncSetAttribute(stress_kernel_async<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    stress_kernel_async<D><<<L.grid, L.block, smem, st>>>(L);
    return cudaGetLastError();
}

// Resident 256-thread blocks per SM of the stress kernel that L.async_depth selects.
int stress_blocks_per_sm(const StressLaunch& L) {
    int nb = 0;
    const size_t base = stress_smem_bytes(L.n_paths);
    cudaError_t e = cudaSuccess;
    switch (L.async_depth) {
        case 0: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, stress_kernel<2>, L.block, base); break;
        case 2: e = cudaFuncSetAttribute(stress_kernel_async<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200000);
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, stress_kernel_async<2>, L.block, base + 2 * 2 * L.block * 16);
            break;
        case 4: e = cudaFuncSetAttribute(stress_kernel_async<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200000);
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, stress_kernel_async<4>, L.block, base + 4 * 2 * L.block * 16);
            break;
        case 8: e = cudaFuncSetAttribute(stress_kernel_async<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200000);
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, stress_kernel_async<8>, L.block, base + 8 * 2 * L.block * 16);
            break;
        default: return 0;
    }
    return e == cudaSuccess ? nb : 0;
}

cudaError_t launch_stress(const StressLaunch& L, cudaStream_t st) {
    switch (L.async_depth) {
        case 2: return launch_stress_async_t<2>(L, st);
        case 4: return launch_stress_async_t<4>(L, st);
        case 8: return launch_stress_async_t<8>(L, st);
        case 0: break;
        default: return cudaErrorInvalidValue;
    }
    const size_t smem = stress_smem_bytes(L.n_paths);
    cudaError_t e = cudaFuncSetAttribute(stress_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    stress_kernel<2><<<L.grid, L.block, smem, st>>>(L);
    return cudaGetLastError();
}

cudaError_t launch_stress_finalize(const double* partials, int n, double* out3, cudaStream_t st) {
    stress_finalize_kernel<<<1, 256, 0, st>>>(partials, n, out3);
    return cudaGetLastError();
}

}  // namespace pgsgd
