/*
 * CPU oracle for path-guided SGD pangenome layout (PG-SGD) and its path-stress
 * metrics, after "Rapid GPU-Based Pangenome Graph Layout" (SC24).
 *
 * TEST INFRASTRUCTURE ONLY. This file is a plain, slow, sequential restatement
 * of the method used to check the CUDA library. Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load it. It shares no code,
 * header or table with the CUDA library: both follow the same written sampler
 * definition and each implements it on its own.
 *
 * What is here, by the passage it follows:
 *   - Algorithm 1 (Section II-C): the outer loop over iterations with learning
 *     rate eta = S[iter], the inner loop of N_steps = 10 * sum |p| updates,
 *     path choice proportional to |p|, the cooling switch (iter >= N_iters / 2
 *     or a coin), the power-law / uniform choice of the second node, the coin
 *     for each visualization point, the pair stress and the update of both
 *     points. The update is the one of Zheng et al. that the paper adopts
 *     (Section II-C, Fig. 3): w = d^-2, mu = min(eta w, 1),
 *     r = mu (|v_i - v_j| - d) / (2 |v_i - v_j|), v_i -= r (v_i - v_j),
 *     v_j += r (v_i - v_j).
 *   - Hogwild! execution of the inner loop (Section III-A): the optional
 *     threaded mode runs the inner loop on several threads with unsynchronised
 *     (relaxed atomic) loads and stores of the coordinates. One thread gives
 *     the sequential definition.
 *   - Eq. 1 (Section VI-A): path stress, every same-path node pair averaged over
 *     its four endpoint combinations.
 *   - Eq. 2 (Section VI-B): sampled path stress over 100 |p| pairs per path and
 *     its 95 % confidence interval mu +- 1.96 sigma / sqrt(n), sigma from a
 *     second pass over the same samples.
 *
 * Readings where the paper is silent (readings R2-R9 and R11 of the list of
 * readings kept with the library's design):
 *   - Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key
 *     (seed_lo, seed_hi). Update u of iteration t uses counter
 *     (u_lo, u_hi, t, b) for block b = 0, 1, ...; words w0..w3 come from block
 *     0, and further blocks only when the power-law draw rejects. Stress
 *     sample q of path p uses counter (q_lo, q_hi, 0x80000000 | p, 0) under
 *     the stress seed.
 *   - Step i: g = mulhi64(w0 | w1 << 32, S); p is the path whose step range
 *     holds g; i = g - off[p]. This is "p with probability |p| / S, then i
 *     uniform in p". Paths with fewer than two steps give no update.
 *   - cooling = (2 t >= T) or (w2 & 1).
 *   - Power law: j is drawn with probability proportional to |j - i|^-theta
 *     over the other steps of the path. A trial draws k from Zipf(theta) on
 *     [1, n_p - 1] by rejection-inversion (Hoermann and Derflinger, ACM
 *     TOMACS 6(3), 1996) evaluated in IEEE binary32 with the operation order
 *     fixed below (no fused multiply-add anywhere; a draw with k >= 256 is
 *     accepted without the rejection test) from bits 8-31 of its 32-bit
 *     word, and a direction from bit 4 of the word (1 = forward); it is
 *     accepted when the Zipf test accepts and i +- k lies on the path. The
 *     trial words are w3, then w2 & ~15, then the four words of block 1,
 *     block 2 and so on, at most 64 trials (then j = i + 1, or i - 1 at the
 *     path's last step).
 *   - Uniform: r = w3 << 32 | (w2 & ~15) (60 random bits: bits 0-3 of w2 are
 *     the coins); x = mulhi64(r, n_p - 1); j = x + (x >= i). Uniform over the
 *     other steps to within (n_p - 1) / 2^60 relative.
 *   - Endpoint bits e_i = (w2 >> 2) & 1, e_j = (w2 >> 3) & 1, 0 = start point,
 *     1 = end point. A step entered in reverse orientation meets the node's end
 *     first, so the endpoint's path position is pos + ((e ^ rev) ? len : 0).
 *     d_ref = |ep_i - ep_j| in exact integers; d_ref = 0 gives no update.
 *   - |v_i - v_j| = 0 gives no update (no direction to move along).
 *   - Learning rate: eta_t = eta_max exp(-lambda t), lambda =
 *     ln(eta_max / eta_min) / (T - 1) (the annealing of Zheng et al.).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Philox4x32-10, from the definition in Salmon et al. (SC'11), Sec. 4. */
/* ------------------------------------------------------------------ */

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod_a = (uint64_t)0xD2511F53u * x0; /* multiplier M0 on word 0 */
        uint64_t prod_b = (uint64_t)0xCD9E8D57u * x2; /* multiplier M1 on word 2 */
        uint32_t hi_a = (uint32_t)(prod_a >> 32), lo_a = (uint32_t)prod_a;
        uint32_t hi_b = (uint32_t)(prod_b >> 32), lo_b = (uint32_t)prod_b;
        uint32_t y0 = hi_b ^ x1 ^ k0;
        uint32_t y1 = lo_b;
        uint32_t y2 = hi_a ^ x3 ^ k1;
        uint32_t y3 = lo_a;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B9u; /* Weyl key schedule */
        k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static void philox_block(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                         uint32_t c3, uint32_t out[4])
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/* Upper 64 bits of the 128-bit product: maps a uniform 64-bit word onto [0, n). */
static uint64_t mulhi64(uint64_t a, uint64_t b)
{
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
}

/* ------------------------------------------------------------------ */
/* binary32 elementary functions with a fixed operation order.         */
/* ln: x = 2^e m, m in [sqrt(1/2), sqrt(2)); ln m = 2 atanh(s) with     */
/* s = (m - 1) / (m + 1), as the odd series 2 s (1 + z/3 + ... + z^5/11)*/
/* in z = s^2. exp: y = n ln2 + r with ln2 split in two parts (Cody and */
/* Waite), e^r by its Taylor polynomial of degree 7, then times 2^n.    */
/* ------------------------------------------------------------------ */

static const float LN2_HI = 0x1.62e4p-1f;      /* ln 2 rounded to 15 bits */
static const float LN2_LO = 0x1.7f7d1cp-20f;   /* ln 2 - LN2_HI */
static const float INV_LN2 = 0x1.715476p+0f;
static const float SQRT2 = 0x1.6a09e6p+0f;

static float fbits(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }
static uint32_t ubits(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }

float orc_ln_f32(float x)
{
    uint32_t b = ubits(x);
    int e = (int)((b >> 23) & 0xffu) - 127;
    float m = fbits((b & 0x7fffffu) | 0x3f800000u);
    if (m > SQRT2) { m = m * 0.5f; e = e + 1; }
    float f = m - 1.0f;
    float s = f / (2.0f + f);
    float z = s * s;
    float p = 0x1.745d18p-4f;          /* 1/11 */
    p = p * z; p = p + 0x1.c71c72p-4f; /* 1/9 */
    p = p * z; p = p + 0x1.24924ap-3f; /* 1/7 */
    p = p * z; p = p + 0x1.99999ap-3f; /* 1/5 */
    p = p * z; p = p + 0x1.555556p-2f; /* 1/3 */
    p = p * z; p = p + 1.0f;
    float two_s = s + s;
    float lnm = two_s * p;
    float fe = (float)e;
    float lo = fe * LN2_LO;
    lo = lo + lnm;
    float hi = fe * LN2_HI;
    return hi + lo;
}

float orc_exp_f32(float y)
{
    float t = y * INV_LN2;
    t = t + 0.5f;
    int n = (int)floorf(t);
    float fn = (float)n;
    float a = fn * LN2_HI;
    float r = y - a;
    float c = fn * LN2_LO;
    r = r - c;
    float p = 0x1.a01a02p-13f;         /* 1/7! */
    p = p * r; p = p + 0x1.6c16c2p-10f; /* 1/6! */
    p = p * r; p = p + 0x1.111112p-7f;  /* 1/5! */
    p = p * r; p = p + 0x1.555556p-5f;  /* 1/4! */
    p = p * r; p = p + 0x1.555556p-3f;  /* 1/3! */
    p = p * r; p = p + 0.5f;
    p = p * r; p = p + 1.0f;
    p = p * r; p = p + 1.0f;
    float scale = fbits((uint32_t)(n + 127) << 23);
    return p * scale;
}

/* phi(t) = (e^t - 1) / t, Taylor polynomial to t^8 for |t| < 1/2. */
static float phi_f32(float t)
{
    if (fabsf(t) < 0.5f) {
        float p = 0x1.71de3ap-19f;          /* 1/9! */
        p = p * t; p = p + 0x1.a01a02p-16f; /* 1/8! */
        p = p * t; p = p + 0x1.a01a02p-13f; /* 1/7! */
        p = p * t; p = p + 0x1.6c16c2p-10f; /* 1/6! */
        p = p * t; p = p + 0x1.111112p-7f;  /* 1/5! */
        p = p * t; p = p + 0x1.555556p-5f;  /* 1/4! */
        p = p * t; p = p + 0x1.555556p-3f;  /* 1/3! */
        p = p * t; p = p + 0.5f;
        p = p * t; p = p + 1.0f;
        return p;
    }
    float e = orc_exp_f32(t);
    e = e - 1.0f;
    return e / t;
}

/* psi(t) = ln(1 + t) / t, alternating series to t^11 for |t| < 1/4. */
static float psi_f32(float t)
{
    if (fabsf(t) < 0.25f) {
        float p = -0x1.555556p-4f;           /* -1/12 */
        p = p * t; p = p + 0x1.745d18p-4f;   /*  1/11 */
        p = p * t; p = p + -0x1.99999ap-4f;  /* -1/10 */
        p = p * t; p = p + 0x1.c71c72p-4f;   /*  1/9 */
        p = p * t; p = p + -0.125f;          /* -1/8 */
        p = p * t; p = p + 0x1.24924ap-3f;   /*  1/7 */
        p = p * t; p = p + -0x1.555556p-3f;  /* -1/6 */
        p = p * t; p = p + 0x1.99999ap-3f;   /*  1/5 */
        p = p * t; p = p + -0.25f;           /* -1/4 */
        p = p * t; p = p + 0x1.555556p-2f;   /*  1/3 */
        p = p * t; p = p + -0.5f;            /* -1/2 */
        p = p * t; p = p + 1.0f;
        return p;
    }
    float one_t = 1.0f + t;
    return orc_ln_f32(one_t) / t;
}

/* Zipf(theta) on [1, N] by rejection-inversion. h(x) = x^-theta is the      */
/* unnormalised mass extended to reals, H its antiderivative with H(1) = 0. */
/* H(x) = ln x * phi((1-theta) ln x); H^-1(y) = exp(y * psi((1-theta) y)).  */
typedef struct { float theta, omt, A, B, s; uint64_t N; } zipf_t;

static float zipf_H(float x, float omt)
{
    float L = orc_ln_f32(x);
    float t = omt * L;
    return L * phi_f32(t);
}

static float zipf_Hinv(float y, float omt)
{
    float t = omt * y;
    float q = psi_f32(t);
    float a = y * q;
    return orc_exp_f32(a);
}

static float zipf_h(float x, float theta)
{
    float L = orc_ln_f32(x);
    float a = theta * L;
    return orc_exp_f32(-a);
}

static zipf_t zipf_setup(double theta_d, uint64_t N)
{
    zipf_t z;
    z.theta = (float)theta_d;
    z.omt = 1.0f - z.theta;
    z.N = N;
    z.A = zipf_H(1.5f, z.omt) - 1.0f;           /* H(3/2) - h(1) */
    float xN = (float)N;
    xN = xN + 0.5f;
    z.B = zipf_H(xN, z.omt);                    /* H(N + 1/2) */
    float h2 = zipf_H(2.5f, z.omt);
    float hh = zipf_h(2.0f, z.theta);
    h2 = h2 - hh;
    z.s = 2.0f - zipf_Hinv(h2, z.omt);          /* squeeze constant */
    return z;
}

void orc_zipf_consts(double theta, uint64_t N, float out[3])
{
    zipf_t z = zipf_setup(theta, N);
    out[0] = z.A; out[1] = z.B; out[2] = z.s;
}

/* One trial with the 32-bit word w: returns 1 and sets *k on acceptance.   */
/* A draw with k >= 256 is accepted without the test: the exact rejection    */
/* chance there is below theta (theta + 1) / (24 * 256^2) of h(k), while in   */
/* binary32 the rounding of H near k is larger than h(k) itself, so the test */
/* would reject by rounding rather than by the method.                      */
static int zipf_trial(const zipf_t *z, uint32_t w, uint64_t *k_out)
{
    float U = (float)(w >> 8) * 0x1p-24f;
    float d = z->A - z->B;
    float t = U * d;
    float u = z->B + t;
    float x = zipf_Hinv(u, z->omt);
    float xr = x + 0.5f;
    float kf = floorf(xr);
    uint64_t k = kf < 1.0f ? 1u : (uint64_t)kf;
    if (k > z->N) k = z->N;
    if (k >= 256u) { *k_out = k; return 1; }
    float fk = (float)k;
    float diff = fk - x;
    if (diff <= z->s) { *k_out = k; return 1; }
    float kh = fk + 0.5f;
    float Hk = zipf_H(kh, z->omt);
    float hk = zipf_h(fk, z->theta);
    Hk = Hk - hk;
    if (u >= Hk) { *k_out = k; return 1; }
    return 0;
}

/* Draw k: trial 0 uses the word first_word, trial m >= 1 uses word          */
/* (m - 1) % 4 of block 1 + (m - 1) / 4 of the counter stream (c0, c1, c2).  */
static uint64_t zipf_draw(const zipf_t *z, uint32_t first_word, uint64_t seed,
                          uint32_t c0, uint32_t c1, uint32_t c2)
{
    uint64_t k;
    if (zipf_trial(z, first_word, &k)) return k;
    for (int m = 1; m < 64; ++m) {
        uint32_t w[4];
        philox_block(seed, c0, c1, c2, (uint32_t)(1 + (m - 1) / 4), w);
        if (zipf_trial(z, w[(m - 1) % 4], &k)) return k;
    }
    return 1;
}

/* Test helper: one Zipf(theta) trial on [1, N] for each trial word          */
/* w = (m_begin + m) << 8, m in [0, count); out[m] = k when the trial        */
/* accepts, 0 when it rejects. A trial reads bits 8-31 of its word only, so  */
/* m over [0, 2^24) enumerates every behaviour of one trial.                  */
void orc_zipf_trials(double theta, uint64_t N, uint32_t m_begin, uint32_t count, uint64_t *out)
{
    zipf_t z = zipf_setup(theta, N);
    for (uint32_t m = 0; m < count; ++m) {
        uint64_t k;
        out[m] = zipf_trial(&z, (m_begin + m) << 8, &k) ? k : 0;
    }
}

/* Test helper: count Zipf(theta) draws on [1, N] keyed by (q, 0x40000000);  */
/* trial 0 takes word 3 of block 0, as an update does.                       */
void orc_zipf_sample(double theta, uint64_t N, uint64_t seed, uint64_t count, uint64_t *out)
{
    zipf_t z = zipf_setup(theta, N);
    for (uint64_t q = 0; q < count; ++q) {
        uint32_t w[4];
        philox_block(seed, (uint32_t)q, (uint32_t)(q >> 32), 0x40000000u, 0u, w);
        out[q] = zipf_draw(&z, w[3], seed, (uint32_t)q, (uint32_t)(q >> 32), 0x40000000u);
    }
}

/* ------------------------------------------------------------------ */
/* Graph view and the per-update sampler (Algorithm 1's pair draw).   */
/* ------------------------------------------------------------------ */

typedef struct {
    uint32_t n_nodes, n_paths;
    const uint32_t *node_len;
    const uint64_t *path_off;
    const uint32_t *step_node;
    const uint8_t *step_rev;
    const int64_t *step_pos;
} orc_graph;

typedef struct {
    uint64_t g, i, j;
    int64_t d_ref;
    uint32_t path;
    uint8_t cooling, e_i, e_j, skip; /* skip: 0 valid, 1 path < 2 steps, 2 d_ref = 0 */
} orc_sample_rec;

typedef struct {
    const orc_graph *G;
    uint64_t seed;
    uint32_t T;
    zipf_t *zipf; /* per path, valid for n_p >= 2 */
} sampler_t;

static uint32_t find_path(const orc_graph *G, uint64_t g)
{
    /* largest p with off[p] <= g; paths with no steps never contain g */
    uint32_t lo = 0, hi = G->n_paths; /* off[lo] <= g < off[hi] */
    while (hi - lo > 1) {
        uint32_t mid = lo + (hi - lo) / 2;
        if (G->path_off[mid] <= g) lo = mid; else hi = mid;
    }
    return lo;
}

static int64_t endpoint_pos(const orc_graph *G, uint64_t step, int e)
{
    int64_t pos = G->step_pos[step];
    int rev = G->step_rev[step];
    int64_t len = G->node_len[G->step_node[step]];
    return pos + (((e ^ rev) & 1) ? len : 0);
}

/* Partner step j of step i on path p (n >= 2 steps) from the words w of   */
/* block 0 of counter (c0, c1, t) (Algorithm 1: the pair draw).              */
/* One power-law trial with word w: k ~ Zipf(theta) on [1, n - 1] from bits */
/* 8-31 of w, direction from bit 4 (1 = forward); accepted when the Zipf    */
/* test accepts and step i +- k lies on the path.                            */
static int partner_trial(const zipf_t *z, uint64_t n, uint64_t i, uint32_t w, uint64_t *j)
{
    uint64_t k;
    if (!zipf_trial(z, w, &k)) return 0;
    if (w & 16u) {
        if (i + k < n) { *j = i + k; return 1; }
    } else if (i >= k) {
        *j = i - k; return 1;
    }
    return 0;
}

/* Partner step j of step i on path p (n >= 2 steps) from the words w of   */
/* block 0 of counter (c0, c1, t) (Algorithm 1: the pair draw). Uniform: j = */
/* x + (x >= i), x = mulhi64(w3 << 32 | (w2 & ~15), n - 1). Power law (the   */
/* paper names only "Powerlaw"; reading: P(j) proportional to |j - i|^-theta */
/* over the path's other steps): trials with the words w3, w2 & ~15, then    */
/* the words of blocks 1, 2, ... of the counter, 64 at most; after 64       */
/* failed trials j = i + 1 (i - 1 at the last step).                         */
static uint64_t partner_step(const sampler_t *S, uint32_t p, uint64_t n, uint64_t i, int cooling,
                             const uint32_t w[4], uint32_t c0, uint32_t c1, uint32_t t)
{
    if (cooling) {
        const zipf_t *z = &S->zipf[p];
        uint64_t j;
        if (partner_trial(z, n, i, w[3], &j)) return j;
        if (partner_trial(z, n, i, w[2] & ~15u, &j)) return j;
        for (int m = 2; m < 64; ++m) {
            uint32_t x[4];
            philox_block(S->seed, c0, c1, t, (uint32_t)(1 + (m - 2) / 4), x);
            if (partner_trial(z, n, i, x[(m - 2) % 4], &j)) return j;
        }
        return i + 1 < n ? i + 1 : i - 1;
    }
    uint64_t x = mulhi64(((uint64_t)w[3] << 32) | (w[2] & ~15u), n - 1);
    return x + (x >= i);
}

/* Warp merging (Section V-B3): one control draw decides the branch for a  */
/* group of 32 consecutive updates. Reading: the cooling coin of update u   */
/* is bit 0 of w2 of update 32 floor(u / 32).                               */
static int group_coin(const sampler_t *S, uint32_t t, uint64_t u)
{
    uint64_t u0 = u & ~(uint64_t)31;
    uint32_t w[4];
    philox_block(S->seed, (uint32_t)u0, (uint32_t)(u0 >> 32), t, 0u, w);
    return (int)(w[2] & 1u);
}

/* Update u of iteration t; wm = 1 takes the cooling coin of its group.     */
static void sample_update_coin(const sampler_t *S, uint32_t t, uint64_t u, int wm, orc_sample_rec *r)
{
    const orc_graph *G = S->G;
    uint32_t c0 = (uint32_t)u, c1 = (uint32_t)(u >> 32);
    uint32_t w[4];
    philox_block(S->seed, c0, c1, t, 0u, w);
    uint64_t steps = G->path_off[G->n_paths];
    uint64_t g = mulhi64((uint64_t)w[0] | ((uint64_t)w[1] << 32), steps);
    uint32_t p = find_path(G, g);
    uint64_t off = G->path_off[p];
    uint64_t n = G->path_off[p + 1] - off;
    uint64_t i = g - off;
    int coin = wm ? group_coin(S, t, u) : (int)(w[2] & 1u);
    memset(r, 0, sizeof *r);
    r->g = g; r->path = p; r->i = i;
    r->cooling = (2ull * t >= S->T) || coin;
    r->e_i = (w[2] >> 2) & 1u;
    r->e_j = (w[2] >> 3) & 1u;
    if (n < 2) { r->skip = 1; r->j = i; return; }
    uint64_t j = partner_step(S, p, n, i, r->cooling, w, c0, c1, t);
    r->j = j;
    int64_t a = endpoint_pos(G, off + i, r->e_i);
    int64_t b = endpoint_pos(G, off + j, r->e_j);
    r->d_ref = a > b ? a - b : b - a;
    if (r->d_ref == 0) r->skip = 2;
}

static void sample_update(const sampler_t *S, uint32_t t, uint64_t u, orc_sample_rec *r)
{
    sample_update_coin(S, t, u, 0, r);
}

static int sampler_init(sampler_t *S, const orc_graph *G, uint32_t T, double theta, uint64_t seed)
{
    S->G = G; S->T = T; S->seed = seed;
    S->zipf = (zipf_t *)calloc(G->n_paths ? G->n_paths : 1, sizeof(zipf_t));
    if (!S->zipf) return -1;
    for (uint32_t p = 0; p < G->n_paths; ++p) {
        uint64_t n = G->path_off[p + 1] - G->path_off[p];
        if (n >= 2) S->zipf[p] = zipf_setup(theta, n - 1);
    }
    return 0;
}

static void sampler_free(sampler_t *S) { free(S->zipf); }

#define GRAPH_ARGS const uint32_t *node_len, uint32_t n_nodes, const uint64_t *path_off, \
    uint32_t n_paths, const uint32_t *step_node, const uint8_t *step_rev, const int64_t *step_pos
#define GRAPH_INIT orc_graph G = {n_nodes, n_paths, node_len, path_off, step_node, step_rev, step_pos}

int orc_sample(GRAPH_ARGS, uint32_t T, uint32_t t, double theta, uint64_t seed,
               uint64_t u_begin, uint64_t count, orc_sample_rec *out)
{
    GRAPH_INIT;
    sampler_t S;
    if (sampler_init(&S, &G, T, theta, seed)) return -1;
    for (uint64_t q = 0; q < count; ++q) sample_update(&S, t, u_begin + q, &out[q]);
    sampler_free(&S);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Learning-rate schedule (Algorithm 1's eta_t; annealing of Zheng).  */
/* ------------------------------------------------------------------ */

void orc_eta_schedule(uint32_t T, double eta_max, double eta_min, double *eta)
{
    if (T == 1) { eta[0] = eta_max; return; }
    double lambda = log(eta_max / eta_min) / (double)(T - 1);
    for (uint32_t t = 0; t < T; ++t) eta[t] = eta_max * exp(-lambda * (double)t);
}

/* ------------------------------------------------------------------ */
/* The update (Algorithm 1's move of both endpoints) in FP64.         */
/* ------------------------------------------------------------------ */

static void update_delta(const double vi[2], const double vj[2], double d_ref, double eta,
                         double out[4], int *moved)
{
    double dx = vi[0] - vj[0], dy = vi[1] - vj[1];
    double mag = sqrt(dx * dx + dy * dy);
    *moved = 0;
    memset(out, 0, 4 * sizeof(double));
    if (mag == 0.0) return;
    double w = 1.0 / (d_ref * d_ref);
    double mu = eta * w;
    if (mu > 1.0) mu = 1.0;
    double r = mu * (mag - d_ref) / (2.0 * mag);
    out[0] = -r * dx; out[1] = -r * dy; /* change of v_i */
    out[2] = r * dx;  out[3] = r * dy;  /* change of v_j */
    *moved = 1;
}

/* Jacobi sweep: the change every update of [u_begin, u_begin + count) of     */
/* iteration t would make to its two points, all computed from the same      */
/* frozen layout xy [n_nodes][4] = (sx, sy, ex, ey). Skipped updates give 0. */
int orc_sweep(GRAPH_ARGS, const double *xy, uint32_t T, uint32_t t, double eta,
              double theta, uint64_t seed, uint64_t u_begin, uint64_t count, double *delta)
{
    GRAPH_INIT;
    sampler_t S;
    if (sampler_init(&S, &G, T, theta, seed)) return -1;
    for (uint64_t q = 0; q < count; ++q) {
        orc_sample_rec r;
        sample_update(&S, t, u_begin + q, &r);
        double *out = delta + 4 * q;
        memset(out, 0, 4 * sizeof(double));
        if (r.skip) continue;
        uint64_t off = G.path_off[r.path];
        uint32_t ni = G.step_node[off + r.i], nj = G.step_node[off + r.j];
        double vi[2] = {xy[4 * (uint64_t)ni + 2 * r.e_i], xy[4 * (uint64_t)ni + 2 * r.e_i + 1]};
        double vj[2] = {xy[4 * (uint64_t)nj + 2 * r.e_j], xy[4 * (uint64_t)nj + 2 * r.e_j + 1]};
        int moved;
        update_delta(vi, vj, (double)r.d_ref, eta, out, &moved);
    }
    sampler_free(&S);
    return 0;
}

/* Hogwild! layout loop. Threads share xy with relaxed atomic loads/stores */
/* of each coordinate, so a concurrent update may be lost or read stale,    */
/* as in the paper's CPU and GPU executions. n_threads = 1 is sequential.   */
typedef struct {
    const sampler_t *S;
    double *xy;
    uint32_t t;
    double eta;
    uint64_t u0, u1;
    uint64_t moved;
} layout_job;

static double ld_relaxed(double *p)
{
    uint64_t bits = __atomic_load_n((uint64_t *)p, __ATOMIC_RELAXED);
    double d; memcpy(&d, &bits, 8); return d;
}

static void st_relaxed(double *p, double v)
{
    uint64_t bits; memcpy(&bits, &v, 8);
    __atomic_store_n((uint64_t *)p, bits, __ATOMIC_RELAXED);
}

static void *layout_worker(void *arg)
{
    layout_job *J = (layout_job *)arg;
    const orc_graph *G = J->S->G;
    uint64_t moved = 0;
    for (uint64_t u = J->u0; u < J->u1; ++u) {
        orc_sample_rec r;
        sample_update(J->S, J->t, u, &r);
        if (r.skip) continue;
        uint64_t off = G->path_off[r.path];
        uint32_t ni = G->step_node[off + r.i], nj = G->step_node[off + r.j];
        double *pi = J->xy + 4 * (uint64_t)ni + 2 * r.e_i;
        double *pj = J->xy + 4 * (uint64_t)nj + 2 * r.e_j;
        double vi[2] = {ld_relaxed(pi), ld_relaxed(pi + 1)};
        double vj[2] = {ld_relaxed(pj), ld_relaxed(pj + 1)};
        double d[4];
        int mv;
        update_delta(vi, vj, (double)r.d_ref, J->eta, d, &mv);
        if (!mv) continue;
        st_relaxed(pi, vi[0] + d[0]);
        st_relaxed(pi + 1, vi[1] + d[1]);
        st_relaxed(pj, vj[0] + d[2]);
        st_relaxed(pj + 1, vj[1] + d[3]);
        ++moved;
    }
    J->moved = moved;
    return NULL;
}

/* Runs iterations [t_begin, t_end) of a T-iteration schedule eta[T] with   */
/* n_updates updates each (Algorithm 1 uses 10 * S). xy is updated in place.*/
int orc_layout(GRAPH_ARGS, double *xy, uint32_t T, const double *eta, double theta,
               uint64_t seed, uint32_t t_begin, uint32_t t_end, uint64_t n_updates,
               uint32_t n_threads, uint64_t *moved_out)
{
    GRAPH_INIT;
    sampler_t S;
    if (sampler_init(&S, &G, T, theta, seed)) return -1;
    if (n_threads < 1) n_threads = 1;
    layout_job *jobs = (layout_job *)calloc(n_threads, sizeof(layout_job));
    pthread_t *th = (pthread_t *)calloc(n_threads, sizeof(pthread_t));
    uint64_t moved = 0;
    for (uint32_t t = t_begin; t < t_end; ++t) {
        for (uint32_t k = 0; k < n_threads; ++k) {
            jobs[k].S = &S; jobs[k].xy = xy; jobs[k].t = t; jobs[k].eta = eta[t];
            jobs[k].u0 = n_updates * k / n_threads;
            jobs[k].u1 = n_updates * (k + 1) / n_threads;
        }
        if (n_threads == 1) {
            layout_worker(&jobs[0]);
        } else {
            for (uint32_t k = 0; k < n_threads; ++k) pthread_create(&th[k], NULL, layout_worker, &jobs[k]);
            for (uint32_t k = 0; k < n_threads; ++k) pthread_join(th[k], NULL);
        }
        for (uint32_t k = 0; k < n_threads; ++k) moved += jobs[k].moved;
    }
    if (moved_out) *moved_out = moved;
    free(jobs); free(th);
    sampler_free(&S);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Warp-level data reuse (Section VII-D) and warp merging, sequential.  */
/* Readings (the paper forms new pairs by shuffling cached node data in */
/* a warp but does not say how their reference distance is defined; it  */
/* exists only for two steps of one path):                               */
/*  - an iteration has n_sel selections; the 32 selections of group      */
/*    G = floor(q / 32) share one path, drawn in proportion to |p| from  */
/*    block 0 of counter (G_lo, G_hi, t, 0x20000000): g = mulhi64(w0 |   */
/*    w1 << 32, S);                                                      */
/*  - selection q draws, from block 0 of its own counter (q_lo, q_hi, t, */
/*    0), its step i = mulhi64(w0 | w1 << 32, n_p), its coins and its    */
/*    partner j exactly as an update does (the group's cooling coin with */
/*    warp merging);                                                     */
/*  - with data reuse factor r, round k = 0..r-1 of lane l = q mod 32    */
/*    pairs (i, e_i) of lane l with (j, e_j) of lane m = (l + o_k) mod   */
/*    32, o_0 = 0, o_k = 1 + floor(31 w / 2^32) for the (k-1)-th word of */
/*    blocks 1, 2 of the group counter; a pair whose partner selection   */
/*    does not exist or whose path has < 2 steps is skipped;             */
/*  - order: groups in order, rounds in order, lanes in order, each      */
/*    update applied at once (a Gauss-Seidel reading of the warp's       */
/*    simultaneous round).                                               */
/* ------------------------------------------------------------------ */

typedef struct {
    uint64_t i, j;
    uint8_t cooling, e_i, e_j, valid;
} sel_t;

static uint32_t group_path(const sampler_t *S, uint32_t t, uint64_t grp)
{
    uint32_t w[4];
    philox_block(S->seed, (uint32_t)grp, (uint32_t)(grp >> 32), t, 0x20000000u, w);
    uint64_t steps = S->G->path_off[S->G->n_paths];
    return find_path(S->G, mulhi64((uint64_t)w[0] | ((uint64_t)w[1] << 32), steps));
}

static uint32_t reuse_offset(const sampler_t *S, uint32_t t, uint64_t grp, uint32_t k)
{
    if (k == 0) return 0;
    uint32_t idx = k - 1, w[4];
    philox_block(S->seed, (uint32_t)grp, (uint32_t)(grp >> 32), t, 0x20000000u | (1u + idx / 4), w);
    return 1u + (uint32_t)(((uint64_t)w[idx % 4] * 31u) >> 32);
}

static void sample_selection(const sampler_t *S, uint32_t t, uint64_t q, int wm, uint32_t p, sel_t *r)
{
    const orc_graph *G = S->G;
    uint32_t c0 = (uint32_t)q, c1 = (uint32_t)(q >> 32);
    uint32_t w[4];
    philox_block(S->seed, c0, c1, t, 0u, w);
    uint64_t n = G->path_off[p + 1] - G->path_off[p];
    int coin = wm ? group_coin(S, t, q) : (int)(w[2] & 1u);
    memset(r, 0, sizeof *r);
    r->cooling = (2ull * t >= S->T) || coin;
    r->e_i = (w[2] >> 2) & 1u;
    r->e_j = (w[2] >> 3) & 1u;
    if (n < 2) return;
    r->i = mulhi64((uint64_t)w[0] | ((uint64_t)w[1] << 32), n);
    r->j = partner_step(S, p, n, r->i, r->cooling, w, c0, c1, t);
    r->valid = 1;
}

/* The pairs of updates [u_begin, u_begin + count) with warp merging.       */
int orc_sample_wm(GRAPH_ARGS, uint32_t T, uint32_t t, double theta, uint64_t seed, int wm,
                  uint64_t u_begin, uint64_t count, orc_sample_rec *out)
{
    GRAPH_INIT;
    sampler_t S;
    if (sampler_init(&S, &G, T, theta, seed)) return -1;
    for (uint64_t q = 0; q < count; ++q) sample_update_coin(&S, t, u_begin + q, wm, &out[q]);
    sampler_free(&S);
    return 0;
}

/* The r pairs of every selection q in [q_begin, q_begin + count) of an     */
/* iteration with n_sel selections: out[(q - q_begin) r + k] for round k.    */
/* g = the global step of i; cooling is that of the partner lane's draw.     */
int orc_sample_reuse(GRAPH_ARGS, uint32_t T, uint32_t t, double theta, uint64_t seed, int wm,
                     uint32_t drf, uint64_t n_sel, uint64_t q_begin, uint64_t count,
                     orc_sample_rec *out)
{
    GRAPH_INIT;
    sampler_t S;
    if (sampler_init(&S, &G, T, theta, seed)) return -1;
    for (uint64_t c = 0; c < count; ++c) {
        uint64_t q = q_begin + c, grp = q >> 5;
        uint32_t lane = (uint32_t)(q & 31), p = group_path(&S, t, grp);
        uint64_t off = G.path_off[p];
        sel_t mine;
        sample_selection(&S, t, q, wm, p, &mine);
        for (uint32_t k = 0; k < drf; ++k) {
            uint64_t qm = (grp << 5) | ((lane + reuse_offset(&S, t, grp, k)) & 31u);
            sel_t other;
            sample_selection(&S, t, qm, wm, p, &other);
            orc_sample_rec *r = &out[c * drf + k];
            memset(r, 0, sizeof *r);
            r->g = off + mine.i; r->i = mine.i; r->j = other.j; r->path = p;
            r->cooling = other.cooling; r->e_i = mine.e_i; r->e_j = other.e_j;
            if (!(mine.valid && other.valid && q < n_sel && qm < n_sel)) { r->skip = 1; continue; }
            int64_t a = endpoint_pos(&G, off + mine.i, mine.e_i);
            int64_t b = endpoint_pos(&G, off + other.j, other.e_j);
            r->d_ref = a > b ? a - b : b - a;
            if (r->d_ref == 0) r->skip = 2;
        }
    }
    sampler_free(&S);
    return 0;
}

static int apply_pair(const orc_graph *G, double *xy, uint64_t si, int ei, uint64_t sj, int ej,
                      int64_t d, double eta)
{
    uint32_t ni = G->step_node[si], nj = G->step_node[sj];
    double *pi = xy + 4 * (uint64_t)ni + 2 * ei;
    double *pj = xy + 4 * (uint64_t)nj + 2 * ej;
    double vi[2] = {pi[0], pi[1]}, vj[2] = {pj[0], pj[1]}, dl[4];
    int moved;
    update_delta(vi, vj, (double)d, eta, dl, &moved);
    if (!moved) return 0;
    pi[0] = vi[0] + dl[0]; pi[1] = vi[1] + dl[1];
    pj[0] = vj[0] + dl[2]; pj[1] = vj[1] + dl[3];
    return 1;
}

/* Iterations [t_begin, t_end), sequential. drf = 1: n_units updates of the */
/* standard sampler (group coin with wm); drf > 1: n_units selections with  */
/* data reuse factor drf (the readings above).                              */
int orc_layout_variant(GRAPH_ARGS, double *xy, uint32_t T, const double *eta, double theta,
                       uint64_t seed, uint32_t t_begin, uint32_t t_end, uint64_t n_units, int wm,
                       uint32_t drf, uint64_t *moved_out)
{
    GRAPH_INIT;
    sampler_t S;
    if (sampler_init(&S, &G, T, theta, seed)) return -1;
    uint64_t moved = 0;
    sel_t sel[32];
    for (uint32_t t = t_begin; t < t_end; ++t) {
        if (drf <= 1) {
            for (uint64_t u = 0; u < n_units; ++u) {
                orc_sample_rec r;
                sample_update_coin(&S, t, u, wm, &r);
                if (r.skip) continue;
                uint64_t off = G.path_off[r.path];
                moved += apply_pair(&G, xy, off + r.i, r.e_i, off + r.j, r.e_j, r.d_ref, eta[t]);
            }
            continue;
        }
        for (uint64_t grp = 0; grp << 5 < n_units; ++grp) {
            uint32_t p = group_path(&S, t, grp);
            uint64_t off = G.path_off[p];
            for (uint32_t l = 0; l < 32; ++l) {
                uint64_t q = (grp << 5) | l;
                sample_selection(&S, t, q, wm, p, &sel[l]);
                if (q >= n_units) sel[l].valid = 0;
            }
            for (uint32_t k = 0; k < drf; ++k) {
                uint32_t o = reuse_offset(&S, t, grp, k);
                for (uint32_t l = 0; l < 32; ++l) {
                    const sel_t *a = &sel[l], *b = &sel[(l + o) & 31u];
                    if (!a->valid || !b->valid) continue;
                    int64_t pa = endpoint_pos(&G, off + a->i, a->e_i), pb = endpoint_pos(&G, off + b->j, b->e_j);
                    int64_t d = pa > pb ? pa - pb : pb - pa;
                    if (d == 0) continue;
                    moved += apply_pair(&G, xy, off + a->i, a->e_i, off + b->j, b->e_j, d, eta[t]);
                }
            }
        }
    }
    if (moved_out) *moved_out = moved;
    sampler_free(&S);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Sampled path stress (Eq. 2) with its 95 % confidence interval.      */
/* ------------------------------------------------------------------ */

typedef struct {
    const orc_graph *G;
    const double *xy;
    uint64_t seed;
    uint32_t per_step;
    double mean;          /* second pass only */
    uint32_t p0, p1;      /* paths handled by this job */
    double *per_path;     /* [n_paths][3] sum, sum of squared deviations, n */
    int pass;
} stress_job;

/* Stress term of sample q of path p, or -1 when d_ref = 0. */
static double stress_term(const orc_graph *G, const double *xy, uint64_t seed, uint32_t p,
                          uint64_t q, int64_t *d_out)
{
    uint64_t off = G->path_off[p], n = G->path_off[p + 1] - off;
    uint32_t c0 = (uint32_t)q, c1 = (uint32_t)(q >> 32), c2 = 0x80000000u | p;
    uint32_t w[4];
    philox_block(seed, c0, c1, c2, 0u, w);
    uint64_t i = mulhi64((uint64_t)w[0] | ((uint64_t)w[1] << 32), n);
    uint64_t x = mulhi64(((uint64_t)w[3] << 32) | (w[2] & ~15u), n - 1);
    uint64_t j = x + (x >= i);
    int ei = w[2] & 1u, ej = (w[2] >> 1) & 1u;
    int64_t a = endpoint_pos(G, off + i, ei), b = endpoint_pos(G, off + j, ej);
    int64_t d = a > b ? a - b : b - a;
    *d_out = d;
    if (d == 0) return -1.0;
    uint32_t ni = G->step_node[off + i], nj = G->step_node[off + j];
    double dx = xy[4 * (uint64_t)ni + 2 * ei] - xy[4 * (uint64_t)nj + 2 * ej];
    double dy = xy[4 * (uint64_t)ni + 2 * ei + 1] - xy[4 * (uint64_t)nj + 2 * ej + 1];
    double mag = sqrt(dx * dx + dy * dy);
    double s = (mag - (double)d) / (double)d;
    return s * s;
}

static void *stress_worker(void *arg)
{
    stress_job *J = (stress_job *)arg;
    const orc_graph *G = J->G;
    for (uint32_t p = J->p0; p < J->p1; ++p) {
        uint64_t n = G->path_off[p + 1] - G->path_off[p];
        double acc = 0.0, cnt = 0.0;
        if (n >= 2) {
            uint64_t Q = (uint64_t)J->per_step * n;
            for (uint64_t q = 0; q < Q; ++q) {
                int64_t d;
                double term = stress_term(G, J->xy, J->seed, p, q, &d);
                if (term < 0.0) continue;
                if (J->pass == 0) acc += term;
                else acc += (term - J->mean) * (term - J->mean);
                cnt += 1.0;
            }
        }
        J->per_path[3 * (uint64_t)p + (J->pass == 0 ? 0 : 1)] = acc;
        if (J->pass == 0) J->per_path[3 * (uint64_t)p + 2] = cnt;
    }
    return NULL;
}

/* out = {mean, stddev, ci95_lo, ci95_hi, n_valid, n_skipped_dref0}.        */
/* per_path (optional, [n_paths][3]): sum of terms, sum of squared          */
/* deviations from the global mean, number of valid samples.                */
/* Paths [p_begin, p_end) only; orc_sampled_stress takes all of them.      */
int orc_sampled_stress_paths(GRAPH_ARGS, const double *xy, uint32_t per_step, uint64_t seed,
                             uint32_t n_threads, uint32_t p_begin, uint32_t p_end,
                             double *out, double *per_path);

int orc_sampled_stress(GRAPH_ARGS, const double *xy, uint32_t per_step, uint64_t seed,
                       uint32_t n_threads, double *out, double *per_path)
{
    return orc_sampled_stress_paths(node_len, n_nodes, path_off, n_paths, step_node, step_rev,
                                    step_pos, xy, per_step, seed, n_threads, 0, n_paths, out,
                                    per_path);
}

int orc_sampled_stress_paths(GRAPH_ARGS, const double *xy, uint32_t per_step, uint64_t seed,
                             uint32_t n_threads, uint32_t p_begin, uint32_t p_end,
                             double *out, double *per_path)
{
    GRAPH_INIT;
    if (n_threads < 1) n_threads = 1;
    double *pp = per_path ? per_path : (double *)calloc(3 * (size_t)(n_paths ? n_paths : 1), sizeof(double));
    if (!pp) return -1;
    memset(pp, 0, 3 * (size_t)n_paths * sizeof(double));
    stress_job *jobs = (stress_job *)calloc(n_threads, sizeof(stress_job));
    pthread_t *th = (pthread_t *)calloc(n_threads, sizeof(pthread_t));
    double total = 0.0, n_valid = 0.0, n_all = 0.0, mean = 0.0, ss = 0.0;
    if (p_end > n_paths) p_end = n_paths;
    if (p_begin > p_end) p_begin = p_end;
    for (int pass = 0; pass < 2; ++pass) {
        for (uint32_t k = 0; k < n_threads; ++k) {
            stress_job *J = &jobs[k];
            J->G = &G; J->xy = xy; J->seed = seed; J->per_step = per_step; J->mean = mean;
            J->per_path = pp; J->pass = pass;
            J->p0 = p_begin + (uint32_t)((uint64_t)(p_end - p_begin) * k / n_threads);
            J->p1 = p_begin + (uint32_t)((uint64_t)(p_end - p_begin) * (k + 1) / n_threads);
        }
        if (n_threads == 1) stress_worker(&jobs[0]);
        else {
            for (uint32_t k = 0; k < n_threads; ++k) pthread_create(&th[k], NULL, stress_worker, &jobs[k]);
            for (uint32_t k = 0; k < n_threads; ++k) pthread_join(th[k], NULL);
        }
        if (pass == 0) {
            for (uint32_t p = p_begin; p < p_end; ++p) {
                uint64_t n = path_off[p + 1] - path_off[p];
                total += pp[3 * (uint64_t)p];
                n_valid += pp[3 * (uint64_t)p + 2];
                if (n >= 2) n_all += (double)per_step * (double)n;
            }
            mean = n_valid > 0 ? total / n_valid : 0.0;
        } else {
            for (uint32_t p = p_begin; p < p_end; ++p) ss += pp[3 * (uint64_t)p + 1];
        }
    }
    double sd = n_valid > 1 ? sqrt(ss / (n_valid - 1.0)) : 0.0;
    double half = n_valid > 0 ? 1.96 * sd / sqrt(n_valid) : 0.0;
    out[0] = mean; out[1] = sd; out[2] = mean - half; out[3] = mean + half;
    out[4] = n_valid; out[5] = n_all - n_valid;
    free(jobs); free(th);
    if (!per_path) free(pp);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Path stress (Eq. 1): every unordered pair of distinct steps of a path,  */
/* the mean over its endpoint combinations with d_ref > 0; the pairs with   */
/* none are left out of the count. Quadratic: small graphs only.           */
/* ------------------------------------------------------------------ */

int orc_full_stress(GRAPH_ARGS, const double *xy, double *out)
{
    GRAPH_INIT;
    double total = 0.0, pairs = 0.0;
    for (uint32_t p = 0; p < n_paths; ++p) {
        uint64_t off = path_off[p], n = path_off[p + 1] - off;
        for (uint64_t i = 0; i < n; ++i) {
            for (uint64_t j = i + 1; j < n; ++j) {
                double sum = 0.0;
                int valid = 0;
                for (int ei = 0; ei < 2; ++ei) {
                    for (int ej = 0; ej < 2; ++ej) {
                        int64_t a = endpoint_pos(&G, off + i, ei), b = endpoint_pos(&G, off + j, ej);
                        int64_t d = a > b ? a - b : b - a;
                        if (d == 0) continue;
                        uint32_t ni = step_node[off + i], nj = step_node[off + j];
                        double dx = xy[4 * (uint64_t)ni + 2 * ei] - xy[4 * (uint64_t)nj + 2 * ej];
                        double dy = xy[4 * (uint64_t)ni + 2 * ei + 1] - xy[4 * (uint64_t)nj + 2 * ej + 1];
                        double mag = sqrt(dx * dx + dy * dy);
                        double s = (mag - (double)d) / (double)d;
                        sum += s * s;
                        ++valid;
                    }
                }
                if (valid) { total += sum / valid; pairs += 1.0; }
            }
        }
    }
    out[0] = pairs > 0 ? total / pairs : 0.0;
    out[1] = pairs;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Differentiable sampled stress: Eq. 2's estimator over a fixed set of */
/* n_pairs samples, sample q drawn by counter (q_lo, q_hi, 0xC0000000,  */
/* 0): the global step g (path in proportion to |p|, step i uniform),  */
/* the partner j uniform among the path's other steps from w3 and the  */
/* upper 28 bits of w2, endpoint coins bits 0 and 1 of w2. Samples on   */
/* paths with fewer than two steps or with d_ref = 0 are left out.      */
/* F = (1 / n_valid) sum ((|v_i - v_j| - d) / d)^2, and its gradient    */
/* dF/dv_i = (2 / n_valid) t (v_i - v_j) / (d |v_i - v_j|), dF/dv_j =   */
/* -dF/dv_i with t = (|v_i - v_j| - d) / d (zero where |v_i - v_j| = 0).*/
/* ------------------------------------------------------------------ */

typedef struct {
    int valid;
    uint32_t ni, nj;
    int ei, ej;
    int64_t d;
} dpair_t;

static void dstress_pair(const orc_graph *G, uint64_t seed, uint64_t q, dpair_t *r)
{
    uint32_t w[4];
    philox_block(seed, (uint32_t)q, (uint32_t)(q >> 32), 0xC0000000u, 0u, w);
    uint64_t steps = G->path_off[G->n_paths];
    uint64_t g = mulhi64((uint64_t)w[0] | ((uint64_t)w[1] << 32), steps);
    uint32_t p = find_path(G, g);
    uint64_t off = G->path_off[p], n = G->path_off[p + 1] - off;
    r->valid = 0;
    if (n < 2) return;
    uint64_t i = g - off;
    uint64_t x = mulhi64(((uint64_t)w[3] << 32) | (w[2] & ~15u), n - 1);
    uint64_t j = x + (x >= i);
    r->ei = w[2] & 1u;
    r->ej = (w[2] >> 1) & 1u;
    int64_t a = endpoint_pos(G, off + i, r->ei), b = endpoint_pos(G, off + j, r->ej);
    r->d = a > b ? a - b : b - a;
    if (r->d == 0) return;
    r->ni = G->step_node[off + i];
    r->nj = G->step_node[off + j];
    r->valid = 1;
}

/* out = {F, n_valid} */
int orc_dstress(GRAPH_ARGS, const double *xy, uint64_t n_pairs, uint64_t seed, double *out)
{
    GRAPH_INIT;
    double sum = 0.0, cnt = 0.0;
    for (uint64_t q = 0; q < n_pairs; ++q) {
        dpair_t r;
        dstress_pair(&G, seed, q, &r);
        if (!r.valid) continue;
        double dx = xy[4 * (uint64_t)r.ni + 2 * r.ei] - xy[4 * (uint64_t)r.nj + 2 * r.ej];
        double dy = xy[4 * (uint64_t)r.ni + 2 * r.ei + 1] - xy[4 * (uint64_t)r.nj + 2 * r.ej + 1];
        double t = (sqrt(dx * dx + dy * dy) - (double)r.d) / (double)r.d;
        sum += t * t;
        cnt += 1.0;
    }
    out[0] = cnt > 0 ? sum / cnt : 0.0;
    out[1] = cnt;
    return 0;
}

/* grad[n_nodes][4] = dF / d(sx, sy, ex, ey) */
int orc_dstress_grad(GRAPH_ARGS, const double *xy, uint64_t n_pairs, uint64_t seed, double *grad)
{
    GRAPH_INIT;
    memset(grad, 0, 4 * (size_t)n_nodes * sizeof(double));
    double cnt = 0.0;
    for (uint64_t q = 0; q < n_pairs; ++q) {
        dpair_t r;
        dstress_pair(&G, seed, q, &r);
        if (r.valid) cnt += 1.0;
    }
    if (cnt == 0.0) return 0;
    for (uint64_t q = 0; q < n_pairs; ++q) {
        dpair_t r;
        dstress_pair(&G, seed, q, &r);
        if (!r.valid) continue;
        double *vi = (double *)xy + 4 * (uint64_t)r.ni + 2 * r.ei;
        double *vj = (double *)xy + 4 * (uint64_t)r.nj + 2 * r.ej;
        double dx = vi[0] - vj[0], dy = vi[1] - vj[1];
        double mag = sqrt(dx * dx + dy * dy);
        if (mag == 0.0) continue;
        double d = (double)r.d;
        double t = (mag - d) / d;
        double c = 2.0 * t / (d * mag) / cnt;
        grad[4 * (uint64_t)r.ni + 2 * r.ei] += c * dx;
        grad[4 * (uint64_t)r.ni + 2 * r.ei + 1] += c * dy;
        grad[4 * (uint64_t)r.nj + 2 * r.ej] -= c * dx;
        grad[4 * (uint64_t)r.nj + 2 * r.ej + 1] -= c * dy;
    }
    return 0;
}
