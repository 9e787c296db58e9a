// Device-side building blocks of the PG-SGD path: the packed records, the
// Philox4x32-10 generator, binary32 elementary functions with a fixed
// operation order, the Zipf rejection-inversion sampler and the per-update
// pair draw of Algorithm 1 (Section II-C: path, steps, cooling and coins).
//
// Every floating-point operation that decides an integer (the Zipf draw) is
// written with explicit round-to-nearest intrinsics (__fadd_rn, __fmul_rn,
// __fdiv_rn, ...), which the compiler never contracts into fused
// multiply-adds, so the draw is the same on every run and matches the
// sampler definition operation for operation.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pgsgd {

constexpr int kZipfTable = 256;     // Zipf acceptance thresholds kept for k < 256
constexpr int kGuideBuckets = 1024; // path-lookup guide buckets (at most)

// ---------------------------------------------------------------- records

// The layout of one node: the two endpoints of its segment (Section II-C: a
// node is drawn as a line segment). x is an FP32 offset from the node's
// integer x anchor (0 in plain-FP32 mode); y is plain FP32. 16 bytes: the
// whole node array of a 5.5 M-node chromosome graph (88 MB) stays resident in
// the GB300's L2, so the lock-free read-modify-writes of Algorithm 1 hit L2.
struct __align__(16) NodeRec {
    float sx, sy, ex, ey;
};
static_assert(sizeof(NodeRec) == 16, "node record is 16 bytes");

// One path step (Section V-B1's path data, extended): node id (bits 0-30) and
// orientation (bit 31), the nucleotide position where the path enters the
// step, and read-only copies of the node's length and x anchor, so that one
// 16-byte read gives everything an update needs besides the coordinates.
struct __align__(16) StepRec {
    uint32_t nr;   // node | rev << 31
    uint32_t pos;  // < 2^32
    uint32_t len;  // node length
    int32_t ax;    // node's x anchor (refreshed after every rebase)
};
static_assert(sizeof(StepRec) == 16, "step record is 16 bytes");

__device__ __forceinline__ uint32_t step_node(const StepRec& s) { return s.nr & 0x7fffffffu; }
__device__ __forceinline__ uint32_t step_rev(const StepRec& s) { return s.nr >> 31; }

// Path position of endpoint e (0 = start point, 1 = end point) of a step: a
// step taken in reverse meets its node's end point first.
__device__ __forceinline__ int64_t endpoint_pos(const StepRec& s, uint32_t e) {
    return (int64_t)s.pos + (((e ^ step_rev(s)) & 1u) ? (int64_t)s.len : 0);
}

// ---------------------------------------------------------------- memory access

// L2 residency policies: step records are streamed (evict first), node
// records are the hot working set (evict last).
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// One random step record: a single 16-byte read at L2 (.cg), one sector.
// pf64 adds the 64-byte L2 prefetch-size hint.
__device__ __forceinline__ StepRec load_step(const StepRec* p, uint64_t pol, bool pf64 = false) {
    StepRec r;
    uint32_t ax;
    if (pf64)
        asm volatile("ld.global.cg.L2::cache_hint.L2::64B.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
                     : "=r"(r.nr), "=r"(r.pos), "=r"(r.len), "=r"(ax)
                     : "l"(p), "l"(pol));
    else
        asm volatile("ld.global.cg.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
                     : "=r"(r.nr), "=r"(r.pos), "=r"(r.len), "=r"(ax)
                     : "l"(p), "l"(pol));
    r.ax = (int32_t)ax;
    return r;
}

// Node records change during a launch (Hogwild!): read them at L2 (.cg),
// never from a possibly stale L1 line.
__device__ __forceinline__ NodeRec load_node(const NodeRec* p, uint64_t pol, bool pf64 = false) {
    NodeRec r;
    if (pf64)
        asm volatile("ld.global.cg.L2::cache_hint.L2::64B.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
                     : "=f"(r.sx), "=f"(r.sy), "=f"(r.ex), "=f"(r.ey)
                     : "l"(p), "l"(pol));
    else
        asm volatile("ld.global.cg.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
                     : "=f"(r.sx), "=f"(r.sy), "=f"(r.ex), "=f"(r.ey)
                     : "l"(p), "l"(pol));
    return r;
}

// One endpoint (e = 0 start, 1 end) of a node record: an 8-byte read of the
// point a move needs (the same 32-byte sector as the whole record).
__device__ __forceinline__ float2 load_point(const NodeRec* p, uint32_t e, uint64_t pol, bool pf64 = false) {
    float2 r;
    const float* q = &p->sx + 2 * e;
    if (pf64)
        asm volatile("ld.global.cg.L2::cache_hint.L2::64B.v2.f32 {%0,%1}, [%2], %3;"
                     : "=f"(r.x), "=f"(r.y) : "l"(q), "l"(pol));
    else
        asm volatile("ld.global.cg.L2::cache_hint.v2.f32 {%0,%1}, [%2], %3;"
                     : "=f"(r.x), "=f"(r.y) : "l"(q), "l"(pol));
    return r;
}

// Write one moved point (8 bytes) by replacing it: a 64-bit atomic exchange
// executed at L2 (last writer wins, like the paper's racy stores, but on
// GB300 several times faster than any st.global form for this pattern).
__device__ __forceinline__ void exchange_point(float* p, float x, float y, uint64_t pol) {
    const unsigned long long v = ((unsigned long long)__float_as_uint(y) << 32) | __float_as_uint(x);
    unsigned long long old;
    asm volatile("atom.global.exch.L2::cache_hint.b64 %0, [%1], %2, %3;"
                 : "=l"(old) : "l"(p), "l"(v), "l"(pol) : "memory");
    (void)old;
}

// ---------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3"
// (SC'11): ten rounds of two 32x32->64 multiplies with a Weyl key schedule.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi_a = __umulhi(0xD2511F53u, c.x), lo_a = 0xD2511F53u * c.x;
        const uint32_t hi_b = __umulhi(0xCD9E8D57u, c.z), lo_b = 0xCD9E8D57u * c.z;
        c = make_uint4(hi_b ^ c.y ^ k0, lo_b, hi_a ^ c.w ^ k1, lo_a);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// High 64 bits of a 64x64 product: a uniform 64-bit word mapped onto [0, n).
__device__ __forceinline__ uint64_t mulhi64(uint64_t a, uint64_t b) { return __umul64hi(a, b); }

// ---------------------------------------------------------------- binary32 math
// ln: x = 2^e m with m in [sqrt(1/2), sqrt(2)), ln m = 2 atanh(s),
// s = (m - 1) / (m + 1), odd series to s^11; exp: y = n ln2 + r with a
// two-part ln2 (Cody and Waite), Taylor polynomial of degree 7 for e^r.

#define PG_LN2_HI 0x1.62e4p-1f
#define PG_LN2_LO 0x1.7f7d1cp-20f
#define PG_INV_LN2 0x1.715476p+0f
#define PG_SQRT2 0x1.6a09e6p+0f

__device__ __forceinline__ float f_ln(float x) {
    const uint32_t b = __float_as_uint(x);
    int e = (int)((b >> 23) & 0xffu) - 127;
    float m = __uint_as_float((b & 0x7fffffu) | 0x3f800000u);
    if (m > PG_SQRT2) { m = __fmul_rn(m, 0.5f); e = e + 1; }
    const float f = __fsub_rn(m, 1.0f);
    const float s = __fdiv_rn(f, __fadd_rn(2.0f, f));
    const float z = __fmul_rn(s, s);
    float p = 0x1.745d18p-4f;
    p = __fadd_rn(__fmul_rn(p, z), 0x1.c71c72p-4f);
    p = __fadd_rn(__fmul_rn(p, z), 0x1.24924ap-3f);
    p = __fadd_rn(__fmul_rn(p, z), 0x1.99999ap-3f);
    p = __fadd_rn(__fmul_rn(p, z), 0x1.555556p-2f);
    p = __fadd_rn(__fmul_rn(p, z), 1.0f);
    const float lnm = __fmul_rn(__fadd_rn(s, s), p);
    const float fe = __int2float_rn(e);
    const float lo = __fadd_rn(__fmul_rn(fe, PG_LN2_LO), lnm);
    return __fadd_rn(__fmul_rn(fe, PG_LN2_HI), lo);
}

__device__ __forceinline__ float f_exp(float y) {
    const float t = __fadd_rn(__fmul_rn(y, PG_INV_LN2), 0.5f);
    const int n = __float2int_rd(t);
    const float fn = __int2float_rn(n);
    float r = __fsub_rn(y, __fmul_rn(fn, PG_LN2_HI));
    r = __fsub_rn(r, __fmul_rn(fn, PG_LN2_LO));
    float p = 0x1.a01a02p-13f;
    p = __fadd_rn(__fmul_rn(p, r), 0x1.6c16c2p-10f);
    p = __fadd_rn(__fmul_rn(p, r), 0x1.111112p-7f);
    p = __fadd_rn(__fmul_rn(p, r), 0x1.555556p-5f);
    p = __fadd_rn(__fmul_rn(p, r), 0x1.555556p-3f);
    p = __fadd_rn(__fmul_rn(p, r), 0.5f);
    p = __fadd_rn(__fmul_rn(p, r), 1.0f);
    p = __fadd_rn(__fmul_rn(p, r), 1.0f);
    return __fmul_rn(p, __uint_as_float((uint32_t)(n + 127) << 23));
}

// (e^t - 1) / t
__device__ __forceinline__ float f_phi(float t) {
    if (fabsf(t) < 0.5f) {
        float p = 0x1.71de3ap-19f;
        p = __fadd_rn(__fmul_rn(p, t), 0x1.a01a02p-16f);
        p = __fadd_rn(__fmul_rn(p, t), 0x1.a01a02p-13f);
        p = __fadd_rn(__fmul_rn(p, t), 0x1.6c16c2p-10f);
        p = __fadd_rn(__fmul_rn(p, t), 0x1.111112p-7f);
        p = __fadd_rn(__fmul_rn(p, t), 0x1.555556p-5f);
        p = __fadd_rn(__fmul_rn(p, t), 0x1.555556p-3f);
        p = __fadd_rn(__fmul_rn(p, t), 0.5f);
        p = __fadd_rn(__fmul_rn(p, t), 1.0f);
        return p;
    }
    return __fdiv_rn(__fsub_rn(f_exp(t), 1.0f), t);
}

// ln(1 + t) / t
__device__ __forceinline__ float f_psi(float t) {
    if (fabsf(t) < 0.25f) {
        float p = -0x1.555556p-4f;
        p = __fadd_rn(__fmul_rn(p, t), 0x1.745d18p-4f);
        p = __fadd_rn(__fmul_rn(p, t), -0x1.99999ap-4f);
        p = __fadd_rn(__fmul_rn(p, t), 0x1.c71c72p-4f);
        p = __fadd_rn(__fmul_rn(p, t), -0.125f);
        p = __fadd_rn(__fmul_rn(p, t), 0x1.24924ap-3f);
        p = __fadd_rn(__fmul_rn(p, t), -0x1.555556p-3f);
        p = __fadd_rn(__fmul_rn(p, t), 0x1.99999ap-3f);
        p = __fadd_rn(__fmul_rn(p, t), -0.25f);
        p = __fadd_rn(__fmul_rn(p, t), 0x1.555556p-2f);
        p = __fadd_rn(__fmul_rn(p, t), -0.5f);
        p = __fadd_rn(__fmul_rn(p, t), 1.0f);
        return p;
    }
    return __fdiv_rn(f_ln(__fadd_rn(1.0f, t)), t);
}

// ---------------------------------------------------------------- Zipf
// Rejection-inversion (Hoermann and Derflinger, ACM TOMACS 1996) for
// P(k) ~ k^-theta on [1, N]. h(x) = x^-theta, H(x) = int_1^x h,
// H(x) = ln x * phi((1 - theta) ln x), H^-1(y) = exp(y * psi((1 - theta) y)).

__device__ __forceinline__ float zipf_H(float x, float omt) {
    const float L = f_ln(x);
    return __fmul_rn(L, f_phi(__fmul_rn(omt, L)));
}
__device__ __forceinline__ float zipf_Hinv(float y, float omt) {
    const float q = f_psi(__fmul_rn(omt, y));
    return f_exp(__fmul_rn(y, q));
}
__device__ __forceinline__ float zipf_h(float x, float theta) {
    return f_exp(-__fmul_rn(theta, f_ln(x)));
}

// Per-theta constants: A = H(3/2) - h(1), s = 2 - H^-1(H(5/2) - h(2)).
__device__ __forceinline__ void zipf_theta_consts(float theta, float& omt, float& A, float& s) {
    omt = __fsub_rn(1.0f, theta);
    A = __fsub_rn(zipf_H(1.5f, omt), 1.0f);
    const float h2 = __fsub_rn(zipf_H(2.5f, omt), zipf_h(2.0f, theta));
    s = __fsub_rn(2.0f, zipf_Hinv(h2, omt));
}
// Per-support constant B = H(N + 1/2).
__device__ __forceinline__ float zipf_B(uint64_t N, float omt) {
    return zipf_H(__fadd_rn(__ull2float_rn(N), 0.5f), omt);
}

struct ZipfConsts {
    float theta, omt, A, s;
};

// Acceptance threshold H(k + 1/2) - h(k) of a trial that lands on k.
__device__ __forceinline__ float zipf_threshold(uint32_t k, float omt, float theta) {
    const float fk = __uint2float_rn(k);
    return __fsub_rn(zipf_H(__fadd_rn(fk, 0.5f), omt), zipf_h(fk, theta));
}

// One trial with the 32-bit word w. Draws with k >= 256 are accepted without
// the rejection test: there the exact rejection chance is below
// theta (theta + 1) / (24 * 256^2) of h(k), smaller than binary32 rounding of H.
// Below 256 the threshold comes from T[k], which holds zipf_threshold(k)
// computed with the same operations (so the decision is the same).
__device__ __forceinline__ bool zipf_trial(const ZipfConsts& z, const float* T, float B, uint64_t N,
                                           uint32_t w, uint64_t& k_out) {
    const float U = __fmul_rn(__uint2float_rn(w >> 8), 0x1p-24f);
    const float u = __fadd_rn(B, __fmul_rn(U, __fsub_rn(z.A, B)));
    const float x = zipf_Hinv(u, z.omt);
    const float kf = floorf(__fadd_rn(x, 0.5f));
    uint64_t k = kf < 1.0f ? 1ull : (uint64_t)__float2ull_rz(kf);
    if (k > N) k = N;
    k_out = k;
    if (k >= (uint64_t)kZipfTable) return true;
    const float fk = __ull2float_rn(k);
    if (__fsub_rn(fk, x) <= z.s) return true;
    return u >= T[k];
}

// ---------------------------------------------------------------- the pair draw

struct SamplerArgs {
    const StepRec* steps;      // step records [S]
    const uint64_t* path_off;  // [P + 1]
    const float* zipf_B;       // [P] H(n_p - 1/2); unused for n_p < 2
    const float* zipf_T;       // [kZipfTable] H(k + 1/2) - h(k) for the current theta
    const uint16_t* guide;     // [n_guide + 1] first path of every bucket of 2^shift steps
    uint64_t n_steps;          // S
    uint32_t n_paths;          // P
    uint32_t n_guide;          // buckets
    uint32_t guide_shift;
    uint32_t T;                // iterations in the schedule
    uint32_t t;                // this iteration
    uint32_t key0, key1;       // Philox key = seed
    uint32_t wm;               // warp merging: cooling coin per group of 32 updates (debug kernels)
    ZipfConsts zc;
};

// Path table staged in shared memory by every block.
struct PathTable {
    const uint64_t* off;    // [P + 1]
    const float* B;         // [P]
    const float* T;         // [kZipfTable]
    const uint16_t* guide;  // [n_guide + 1]
    uint32_t P;
    uint32_t shift;
};

// Largest p in [lo, hi) with off[p] <= g, given off[lo] <= g < off[hi].
__device__ __forceinline__ uint32_t search_path(const uint64_t* off, uint32_t lo, uint32_t hi, uint64_t g) {
    while (hi - lo > 1) {
        const uint32_t mid = lo + ((hi - lo) >> 1);
        if (off[mid] <= g) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ uint32_t find_path(const uint64_t* off, uint32_t P, uint64_t g) {
    return search_path(off, 0, P, g);
}

// Same result as find_path: the guide bounds the search to the paths that
// meet g's bucket, usually a single one.
__device__ __forceinline__ uint32_t find_path_guided(const PathTable& pt, uint64_t g) {
    const uint32_t b = (uint32_t)(g >> pt.shift);
    return search_path(pt.off, pt.guide[b], (uint32_t)pt.guide[b + 1] + 1, g);
}

struct Pair {
    uint64_t base;     // global index of the path's first step
    uint64_t i, j;     // step indices within the path
    uint64_t g;        // global step drawn
    uint32_t path;
    uint32_t w2;       // coin word: bit 0 cooling coin, bits 2-3 endpoints
    uint32_t cooling;  // 1 = power-law pair
    uint32_t short_path;  // 1 = path has < 2 steps: no update
};

// One power-law trial with word w: k ~ Zipf(theta) on [1, n - 1] from bits
// 8-31 of w, direction from bit 4 (1 = forward); accepted when the Zipf test
// accepts and step i +- k lies on the path.
__device__ __forceinline__ bool partner_trial(const ZipfConsts& zc, const float* T, float B, uint64_t n, uint64_t i,
                                              uint32_t w, uint64_t& j) {
    uint64_t k = 1;
    if (!zipf_trial(zc, T, B, n - 1, w, k)) return false;
    if (w & 16u) {
        if (i + k < n) { j = i + k; return true; }
    } else if (i >= k) {
        j = i - k;
        return true;
    }
    return false;
}

// Partner step j of step i in a path of n >= 2 steps (Algorithm 1's
// partner draw) from the words w2, w3 of block 0 of the update's counter (c0, c1, t).
// Uniform: j = x + (x >= i), x = mulhi64(w3 << 32 | (w2 & ~15), n - 1).
// Power law: P(j) proportional to |j - i|^-theta over the path's other
// steps: trials with the words w3, w2 & ~15, then blocks 1, 2, ... of the
// counter (drawn only when needed), 64 at most, then j = i + 1 (i - 1 at the
// last step).
__device__ __forceinline__ uint64_t draw_partner(const ZipfConsts& zc, const float* T, float B, uint64_t n,
                                                 uint64_t i, bool cooling, uint32_t w2, uint32_t w3, uint32_t c0,
                                                 uint32_t c1, uint32_t t, uint32_t key0, uint32_t key1) {
    if (!cooling) {
        const uint64_t x = mulhi64(((uint64_t)w3 << 32) | (w2 & ~15u), n - 1);
        return x + (x >= i);
    }
    uint64_t j = 0;
    if (partner_trial(zc, T, B, n, i, w3, j) || partner_trial(zc, T, B, n, i, w2 & ~15u, j)) return j;
    for (uint32_t blk = 1; blk <= 16; ++blk) {  // trials 2..63
        const uint4 x = philox4x32_10(make_uint4(c0, c1, t, blk), key0, key1);
        if (partner_trial(zc, T, B, n, i, x.x, j) || partner_trial(zc, T, B, n, i, x.y, j) ||
            (blk < 16 && (partner_trial(zc, T, B, n, i, x.z, j) || partner_trial(zc, T, B, n, i, x.w, j))))
            return j;
    }
    return i + 1 < n ? i + 1 : i - 1;
}

__device__ __forceinline__ uint4 pair_block(const SamplerArgs& a, uint64_t u) {
    return philox4x32_10(make_uint4((uint32_t)u, (uint32_t)(u >> 32), a.t, 0u), a.key0, a.key1);
}

// The pair of update u from its block-0 words w, with cooling coin `coin`.
__device__ __forceinline__ Pair pair_from_block(const SamplerArgs& a, const PathTable& pt, uint64_t u, uint4 w,
                                                uint32_t coin) {
    Pair r;
    const uint32_t c0 = (uint32_t)u, c1 = (uint32_t)(u >> 32);
    r.g = mulhi64((uint64_t)w.x | ((uint64_t)w.y << 32), a.n_steps);
    r.path = find_path_guided(pt, r.g);
    r.base = pt.off[r.path];
    const uint64_t n = pt.off[r.path + 1] - r.base;
    r.i = r.g - r.base;
    r.w2 = w.z;
    r.cooling = (2ull * a.t >= a.T) || coin;
    r.short_path = n < 2;
    r.j = r.short_path ? r.i
                       : draw_partner(a.zc, pt.T, pt.B[r.path], n, r.i, r.cooling, w.z, w.w, c0, c1, a.t, a.key0,
                                      a.key1);
    return r;
}

// Draw the pair of update u in iteration t (Algorithm 1: path, steps, cooling). One
// Philox block serves the whole draw: w0, w1 pick the step, bits 0, 2 and 3
// of w2 are the cooling and endpoint coins, w3 and the upper 28 bits of w2
// feed the uniform partner or the first two power-law trials. Later blocks
// are drawn only after both of those trials fail (about 1 power-law draw in
// 200).
__device__ __forceinline__ Pair draw_pair(const SamplerArgs& a, const PathTable& pt, uint64_t u) {
    const uint4 w = pair_block(a, u);
    return pair_from_block(a, pt, u, w, w.z & 1u);
}

// Warp merging (Section V-B3): the cooling coin of update u is bit 0 of w2
// of update 32 floor(u / 32), computed here from scratch (no warp needed).
__device__ __forceinline__ uint32_t group_coin(const SamplerArgs& a, uint64_t u) {
    return pair_block(a, u & ~31ull).z & 1u;
}

// draw_pair, or with a.wm its warp-merged form (debug and checking kernels).
__device__ __forceinline__ Pair draw_pair_any(const SamplerArgs& a, const PathTable& pt, uint64_t u) {
    const uint4 w = pair_block(a, u);
    return pair_from_block(a, pt, u, w, a.wm ? group_coin(a, u) : (w.z & 1u));
}

// ---------------------------------------------------------------- shared kernel helpers

// Stage the path table, the guide and the per-theta Zipf tables in shared memory.
__device__ __forceinline__ PathTable stage_paths(const SamplerArgs& a, unsigned char* smem,
                                                 ZipfConsts& zc_shared) {
    uint64_t* s_off = reinterpret_cast<uint64_t*>(smem);
    float* s_T = reinterpret_cast<float*>(s_off + a.n_paths + 1);
    float* s_B = s_T + kZipfTable;
    uint16_t* s_guide = reinterpret_cast<uint16_t*>(s_B + a.n_paths);
    for (uint32_t k = threadIdx.x; k <= a.n_paths; k += blockDim.x) s_off[k] = a.path_off[k];
    for (uint32_t k = threadIdx.x; k < a.n_paths; k += blockDim.x) s_B[k] = a.zipf_B[k];
    for (uint32_t k = threadIdx.x; k < (uint32_t)kZipfTable; k += blockDim.x) s_T[k] = a.zipf_T[k];
    for (uint32_t k = threadIdx.x; k <= a.n_guide; k += blockDim.x) s_guide[k] = a.guide[k];
    if (threadIdx.x == 0) {
        ZipfConsts z;
        z.theta = a.zc.theta;
        zipf_theta_consts(z.theta, z.omt, z.A, z.s);
        zc_shared = z;
    }
    __syncthreads();
    return PathTable{s_off, s_B, s_T, s_guide, a.n_paths, a.guide_shift};
}


struct Move {
    float dxi, dyi, dxj, dyj;  // change of v_i and v_j
    bool moved;
};

// The update of Zheng et al. that Algorithm 1 applies (Fig. 3):
// w = d^-2, mu = min(eta w, 1), r = mu (|v_i - v_j| - d) / (2 |v_i - v_j|),
// v_i -= r (v_i - v_j), v_j += r (v_i - v_j), for the points (xa, ya) and
// (xb, yb). FP32; x anchors differenced in integers so chromosome-scale
// coordinates keep their resolution.
__device__ __forceinline__ Move point_move(float xa, float ya, int32_t axa, float xb, float yb, int32_t axb,
                                           int64_t d, float eta) {
    Move m;
    const float dx = __ll2float_rn((int64_t)axa - (int64_t)axb) + (xa - xb);
    const float dy = ya - yb;
    const float mag = sqrtf(dx * dx + dy * dy);
    m.moved = mag > 0.0f;
    const float df = __ll2float_rn(d);
    const float w = 1.0f / (df * df);
    const float mu = fminf(eta * w, 1.0f);
    const float r = m.moved ? mu * (mag - df) / (2.0f * mag) : 0.0f;
    const float rx = r * dx, ry = r * dy;
    m.dxi = -rx; m.dyi = -ry; m.dxj = rx; m.dyj = ry;
    return m;
}

// The same for endpoint ea of node a and endpoint eb of node b.
__device__ __forceinline__ Move pair_move(const NodeRec& a, int32_t axa, uint32_t ea, const NodeRec& b,
                                          int32_t axb, uint32_t eb, int64_t d, float eta) {
    return point_move(ea ? a.ex : a.sx, ea ? a.ey : a.sy, axa, eb ? b.ex : b.sx, eb ? b.ey : b.sy, axb, d, eta);
}


struct UpdateOpts {
    float eta;
    int store_mode;  // 0 = plain store, 1 = 64-bit atomic exchange
    int pf64;        // 64-byte L2 prefetch hint: bit 0 step loads, bit 1 node loads
    bool atomic;     // add the moves atomically instead of replacing the points
};

// The pairs of UPT independent updates u0 + k * stride (k < UPT; only those
// below u_end are active) of Algorithm 1's pair draw.
template <int UPT>
struct TripDraws {
    uint64_t gi[UPT], gj[UPT];  // global step indices of n_i and n_j
    uint32_t w2[UPT];           // coin word (endpoint bits 2 and 3)
    bool act[UPT];
};

template <int UPT>
__device__ __forceinline__ void draw_trip(const SamplerArgs& a, const PathTable& pt, uint64_t u0, uint64_t stride,
                                          uint64_t u_end, TripDraws<UPT>& d) {
#pragma unroll
    for (int k = 0; k < UPT; ++k) {
        const uint64_t u = u0 + (uint64_t)k * stride;
        d.act[k] = u < u_end;
        if (d.act[k]) {
            const Pair pr = draw_pair(a, pt, u);
            d.act[k] = !pr.short_path;
            d.gi[k] = pr.base + pr.i;
            d.gj[k] = pr.base + pr.j;
            d.w2[k] = pr.w2;
        }
    }
}

template <int UPT>
__device__ __forceinline__ void load_trip_steps(const StepRec* __restrict__ steps, const TripDraws<UPT>& d,
                                                StepRec (&si)[UPT], StepRec (&sj)[UPT], uint64_t pol_stream,
                                                int pf64) {
#pragma unroll
    for (int k = 0; k < UPT; ++k) {
        if (d.act[k]) {
            si[k] = load_step(steps + d.gi[k], pol_stream, pf64 & 1);
            sj[k] = load_step(steps + d.gj[k], pol_stream, pf64 & 1);
        }
    }
}

// Endpoint loads, the moves of Algorithm 1, and the stores.
// Only the chosen endpoint of each node is read (8 bytes, 2 registers).
template <int UPT>
__device__ __forceinline__ void finish_trip(NodeRec* __restrict__ nodes, const TripDraws<UPT>& d,
                                            const StepRec (&si)[UPT], const StepRec (&sj)[UPT], const UpdateOpts& o,
                                            uint64_t pol_keep) {
    float2 va[UPT], vb[UPT];
#pragma unroll
    for (int k = 0; k < UPT; ++k) {
        if (d.act[k]) {
            va[k] = load_point(nodes + step_node(si[k]), (d.w2[k] >> 2) & 1u, pol_keep, o.pf64 & 2);
            vb[k] = load_point(nodes + step_node(sj[k]), (d.w2[k] >> 3) & 1u, pol_keep, o.pf64 & 2);
        }
    }
#pragma unroll
    for (int k = 0; k < UPT; ++k) {
        if (!d.act[k]) continue;
        const uint32_t ea = (d.w2[k] >> 2) & 1u, eb = (d.w2[k] >> 3) & 1u;
        const int64_t pa = endpoint_pos(si[k], ea), pb = endpoint_pos(sj[k], eb);
        const int64_t dd = pa > pb ? pa - pb : pb - pa;
        if (dd == 0) continue;
        const Move m = point_move(va[k].x, va[k].y, si[k].ax, vb[k].x, vb[k].y, sj[k].ax, dd, o.eta);
        if (!m.moved) continue;
        float* pa_ptr = &nodes[step_node(si[k])].sx + 2 * ea;
        float* pb_ptr = &nodes[step_node(sj[k])].sx + 2 * eb;
        if (o.atomic) {
            atomicAdd(reinterpret_cast<float2*>(pa_ptr), make_float2(m.dxi, m.dyi));
            atomicAdd(reinterpret_cast<float2*>(pb_ptr), make_float2(m.dxj, m.dyj));
        } else if (o.store_mode == 0) {
            *reinterpret_cast<float2*>(pa_ptr) = make_float2(va[k].x + m.dxi, va[k].y + m.dyi);
            *reinterpret_cast<float2*>(pb_ptr) = make_float2(vb[k].x + m.dxj, vb[k].y + m.dyj);
        } else {
            exchange_point(pa_ptr, va[k].x + m.dxi, va[k].y + m.dyi, pol_keep);
            exchange_point(pb_ptr, vb[k].x + m.dxj, vb[k].y + m.dyj, pol_keep);
        }
    }
}

// UPT independent updates kept in flight together: all draws first (ALU),
// then all step-record loads, then all node-record loads, then the moves.
template <int UPT>
__device__ __forceinline__ void update_trip(const SamplerArgs& a, const PathTable& pt, NodeRec* __restrict__ nodes,
                                            uint64_t u0, uint64_t stride, uint64_t u_end, const UpdateOpts& o,
                                            uint64_t pol_stream, uint64_t pol_keep) {
    TripDraws<UPT> d;
    draw_trip<UPT>(a, pt, u0, stride, u_end, d);
    StepRec si[UPT], sj[UPT];
    load_trip_steps<UPT>(a.steps, d, si, sj, pol_stream, o.pf64);
    finish_trip<UPT>(nodes, d, si, sj, o, pol_keep);
}

// The updates u_first + m * stride < u_end, UPT per trip, software
// pipelined: a trip's step-record loads are issued before the next trip's
// pairs are drawn, so the sampler's arithmetic overlaps the loads' latency.
// The same updates, draws and moves as update_trip over the same range.
template <int UPT>
__device__ __forceinline__ void update_range_pipelined(const SamplerArgs& a, const PathTable& pt,
                                                       NodeRec* __restrict__ nodes, uint64_t u_first, uint64_t stride,
                                                       uint64_t u_end, const UpdateOpts& o, uint64_t pol_stream,
                                                       uint64_t pol_keep) {
    const uint64_t trip = stride * UPT;
    TripDraws<UPT> cur;
    draw_trip<UPT>(a, pt, u_first, stride, u_end, cur);
    for (uint64_t base = u_first; base < u_end; base += trip) {
        StepRec si[UPT], sj[UPT];
        load_trip_steps<UPT>(a.steps, cur, si, sj, pol_stream, o.pf64);
        TripDraws<UPT> nxt;
        draw_trip<UPT>(a, pt, base + trip, stride, u_end, nxt);
        finish_trip<UPT>(nodes, cur, si, sj, o, pol_keep);
        cur = nxt;
    }
}

// ---------------------------------------------------------------- warp merging and data reuse

// Warp merging: a warp's lanes hold 32 consecutive update indices starting
// at a multiple of 32 (lane l holds 32 G + l), so lane 0's coin is the
// group's and the warp shares it by shuffle. All 32 lanes must call this.
template <int UPT>
__device__ __forceinline__ void draw_trip_wm(const SamplerArgs& a, const PathTable& pt, uint64_t u0, uint64_t stride,
                                             uint64_t u_end, TripDraws<UPT>& d) {
#pragma unroll
    for (int k = 0; k < UPT; ++k) {
        const uint64_t u = u0 + (uint64_t)k * stride;
        const uint4 w = pair_block(a, u);
        const uint32_t coin = __shfl_sync(0xffffffffu, w.z & 1u, 0);
        d.act[k] = u < u_end;
        if (d.act[k]) {
            const Pair pr = pair_from_block(a, pt, u, w, coin);
            d.act[k] = !pr.short_path;
            d.gi[k] = pr.base + pr.i;
            d.gj[k] = pr.base + pr.j;
            d.w2[k] = pr.w2;
        }
    }
}

template <int UPT>
__device__ __forceinline__ void update_trip_wm(const SamplerArgs& a, const PathTable& pt, NodeRec* __restrict__ nodes,
                                               uint64_t u0, uint64_t stride, uint64_t u_end, const UpdateOpts& o,
                                               uint64_t pol_stream, uint64_t pol_keep) {
    TripDraws<UPT> d;
    draw_trip_wm<UPT>(a, pt, u0, stride, u_end, d);
    StepRec si[UPT], sj[UPT];
    load_trip_steps<UPT>(a.steps, d, si, sj, pol_stream, o.pf64);
    finish_trip<UPT>(nodes, d, si, sj, o, pol_keep);
}

// Data reuse (Section VII-D). Group grp = q / 32 of selections shares one
// path, drawn in proportion to |p| from block 0 of counter (grp, t,
// 0x20000000); blocks 1 and 2 give the round offsets o_k = 1 + mulhi32(word,
// 31), word k - 1 in order.
__device__ __forceinline__ uint4 group_block(const SamplerArgs& a, uint64_t grp, uint32_t b) {
    return philox4x32_10(make_uint4((uint32_t)grp, (uint32_t)(grp >> 32), a.t, 0x20000000u | b), a.key0, a.key1);
}

__device__ __forceinline__ uint32_t group_path(const SamplerArgs& a, const PathTable& pt, uint64_t grp) {
    const uint4 w = group_block(a, grp, 0);
    return find_path_guided(pt, mulhi64((uint64_t)w.x | ((uint64_t)w.y << 32), a.n_steps));
}

__device__ __forceinline__ uint32_t word_of(uint4 w, int k) {
    return k == 0 ? w.x : k == 1 ? w.y : k == 2 ? w.z : w.w;
}

// Offset of round k >= 1 (one block per call: for checking kernels).
__device__ __forceinline__ uint32_t reuse_offset(const SamplerArgs& a, uint64_t grp, uint32_t k) {
    if (k == 0) return 0;
    const uint32_t idx = k - 1;
    return 1u + __umulhi(word_of(group_block(a, grp, 1 + idx / 4), idx % 4), 31u);
}

// All R offsets of a group (o[0] = 0), one block per four rounds.
template <int R>
__device__ __forceinline__ void reuse_offsets(const SamplerArgs& a, uint64_t grp, uint32_t (&o)[R]) {
    o[0] = 0;
    uint4 w = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
    for (int k = 1; k < R; ++k) {
        const int idx = k - 1;
        if (idx % 4 == 0) w = group_block(a, grp, 1 + idx / 4);
        o[k] = 1u + __umulhi(word_of(w, idx % 4), 31u);
    }
}

struct Selection {
    uint64_t i, j;     // steps within the group's path
    uint32_t w2;       // coin word: endpoint bits 2 and 3
    uint32_t cooling;
    bool valid;        // the path has at least two steps
};

// Selection q on path p from its block-0 words w: step i uniform on the path,
// partner j as an update draws it.
__device__ __forceinline__ Selection draw_selection(const SamplerArgs& a, const PathTable& pt, uint64_t q, uint32_t p,
                                                    uint4 w, uint32_t coin) {
    Selection s;
    const uint64_t off = pt.off[p], n = pt.off[p + 1] - off;
    s.w2 = w.z;
    s.cooling = (2ull * a.t >= a.T) || coin;
    s.valid = n >= 2;
    s.i = s.valid ? mulhi64((uint64_t)w.x | ((uint64_t)w.y << 32), n) : 0;
    s.j = s.valid ? draw_partner(a.zc, pt.T, pt.B[p], n, s.i, s.cooling, w.z, w.w, (uint32_t)q, (uint32_t)(q >> 32),
                                 a.t, a.key0, a.key1)
                  : 0;
    return s;
}

// Selections q_first + m * stride below n_sel, one per thread per trip, each
// performing R updates: round k pairs this lane's (i, e_i) with lane
// (lane + o_k)'s (j, e_j). Points live in registers across the rounds; the
// lane holding a j-point receives its move by shuffle. Each selection writes
// its two points once, after the last round. Every lane of a warp runs the
// same trips (the loop bound is the warp's first selection), so the shuffles
// always see 32 lanes; stride and q_first - lane are multiples of 32.
template <int R>
__device__ __forceinline__ void reuse_range(const SamplerArgs& a, const PathTable& pt, NodeRec* __restrict__ nodes,
                                            uint64_t q_first, uint64_t stride, uint64_t n_sel, float eta, bool wm,
                                            int pf64, uint64_t pol_stream, uint64_t pol_keep) {
    const uint32_t lane = threadIdx.x & 31u;
    for (uint64_t q = q_first; q - lane < n_sel; q += stride) {
        const uint64_t grp = q >> 5;
        const uint32_t p = group_path(a, pt, grp);
        uint32_t o[R];
        reuse_offsets<R>(a, grp, o);
        const uint4 w = pair_block(a, q);
        const uint32_t coin = wm ? __shfl_sync(0xffffffffu, w.z & 1u, 0) : (w.z & 1u);
        const Selection s = draw_selection(a, pt, q, p, w, coin);
        const bool sel = s.valid && q < n_sel;
        const uint64_t base = pt.off[p];
        const uint32_t ei = (s.w2 >> 2) & 1u, ej = (s.w2 >> 3) & 1u;
        uint32_t ni = 0, nj = 0;
        float xi = 0.f, yi = 0.f, xj = 0.f, yj = 0.f;
        int32_t axi = 0, axj = 0;
        long long pi = 0, pj = 0;
        if (sel) {
            const StepRec si = load_step(a.steps + base + s.i, pol_stream, pf64 & 1);
            const StepRec sj = load_step(a.steps + base + s.j, pol_stream, pf64 & 1);
            ni = step_node(si);
            nj = step_node(sj);
            const NodeRec na = load_node(nodes + ni, pol_keep, pf64 & 2);
            const NodeRec nb = load_node(nodes + nj, pol_keep, pf64 & 2);
            xi = ei ? na.ex : na.sx;
            yi = ei ? na.ey : na.sy;
            xj = ej ? nb.ex : nb.sx;
            yj = ej ? nb.ey : nb.sy;
            axi = si.ax;
            axj = sj.ax;
            pi = endpoint_pos(si, ei);
            pj = endpoint_pos(sj, ej);
        }
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const uint32_t m = (lane + o[k]) & 31u;
            const float xm = __shfl_sync(0xffffffffu, xj, m), ym = __shfl_sync(0xffffffffu, yj, m);
            const int32_t axm = __shfl_sync(0xffffffffu, axj, m);
            const long long pm = __shfl_sync(0xffffffffu, pj, m);
            const int selm = __shfl_sync(0xffffffffu, (int)sel, m);
            float nxm = xm, nym = ym;
            if (sel && selm) {
                const long long d = pi > pm ? pi - pm : pm - pi;
                if (d != 0) {
                    const Move mv = point_move(xi, yi, axi, xm, ym, axm, (int64_t)d, eta);
                    if (mv.moved) {
                        xi += mv.dxi;
                        yi += mv.dyi;
                        nxm = xm + mv.dxj;
                        nym = ym + mv.dyj;
                    }
                }
            }
            // the move of lane m's j-point goes back to lane m
            const uint32_t src = (lane - o[k]) & 31u;
            const float rx = __shfl_sync(0xffffffffu, nxm, src), ry = __shfl_sync(0xffffffffu, nym, src);
            if (sel) {
                xj = rx;
                yj = ry;
            }
        }
        if (sel) {
            exchange_point(&nodes[ni].sx + 2 * ei, xi, yi, pol_keep);
            exchange_point(&nodes[nj].sx + 2 * ej, xj, yj, pol_keep);
        }
    }
}
}  // namespace pgsgd
