/*
 * pgsgd.h - C ABI of libpgsgd.so: path-guided SGD (PG-SGD) layout of a
 * pangenome variation graph on one NVIDIA GB300 GPU (sm_103a), and the
 * sampled path-stress metric that scores it.
 *
 * The method is the one of "Rapid GPU-Based Pangenome Graph Layout" (SC24):
 * Algorithm 1 (Section II-C) moves the two endpoints of randomly chosen
 * same-path node pairs towards their path distance, millions of times per
 * iteration, without locks (Hogwild!, Section III-A); Eq. 2 (Section VI-B)
 * scores a layout by sampling such pairs.
 *
 * Conventions for every entry point:
 *   - The return value is a status code (pgsgd_status). On failure the
 *     calling thread's message is available from pgsgd_last_error().
 *   - `cuda_stream` is a cudaStream_t passed as void* (NULL = the legacy
 *     default stream). Work is queued on it in order.
 *   - `on_device` = 1 means a pointer is CUDA device memory (for example a
 *     torch tensor's data_ptr()); 0 means host memory. Data is always copied:
 *     the library never keeps a caller's pointer after the call returns.
 *   - A graph handle must not be used from two host threads at once.
 *   - All memory the library allocates is owned by the handle and released
 *     by pgsgd_destroy().
 */
#ifndef PGSGD_H
#define PGSGD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pgsgd_status {
    PGSGD_OK = 0,
    PGSGD_EINVAL = 1,   /* bad argument or inconsistent input array */
    PGSGD_ERANGE = 2,   /* a value overflows the packed device records */
    PGSGD_ENOMEM = 3,   /* host or device allocation failed */
    PGSGD_ECUDA = 4,    /* a CUDA call or kernel failed */
    PGSGD_ETIMEOUT = 5, /* a device-side bounded wait expired */
    PGSGD_EDEVICE = 6   /* reserved: device-side checks report EINVAL / ERANGE */
} pgsgd_status;

/* Options for pgsgd_set_option / pgsgd_get_option. */
typedef enum pgsgd_option {
    /* Coordinate storage. 0 = anchored (default): a node whose start x is at
     * least 4096 in magnitude keeps an integer x anchor and FP32 x offsets
     * from it, so FP32 keeps sub-nucleotide resolution along a chromosome-
     * scale layout (|x| < 2^30); y is plain FP32 (resolution better than
     * 0.1 nt while |y| < 1e6). 1 = plain FP32 absolute coordinates. Takes
     * effect at pgsgd_set_coords. */
    PGSGD_OPT_COORD_MODE = 1,
    /* Updates per iteration = this value times the number of path steps
     * (Algorithm 1 uses 10). Default 10. */
    PGSGD_OPT_UPDATES_PER_STEP = 2,
    /* Update-kernel launch shape: threads per block (64..256, multiple of
     * 32; default 256), blocks per SM in the grid (default 32: many short
     * blocks let the block scheduler balance the two dies), and
     * updates each thread keeps in flight per loop trip (1, 2 or 4; default 0
     * = automatic: 2 with the pipelined loop, PGSGD_OPT_PIPELINE, else 1; the
     * pipelined loop at 2 ran the full chromosome layout
     * in 6.58 s against 6.74 s for 1 update per thread unpipelined with 4
     * resident blocks per SM, the next best shape of a sweep over updates per
     * thread, register budgets, grid sizes and asynchronous step reads). */
    PGSGD_OPT_BLOCK = 3,
    PGSGD_OPT_BLOCKS_PER_SM = 4,
    PGSGD_OPT_UPDATES_PER_THREAD = 5,
    /* 0 = replace the moved points (last writer wins, as in the paper's
     * kernels; the form of the write is PGSGD_OPT_STORE_MODE; default),
     * 1 = vector atomic adds of the moves. Atomic adds sum colliding
     * full-rate (mu = 1) moves, which overshoot; on small graphs under a full
     * grid that diverges, so keep 0 unless the concurrency cap makes
     * collisions rare. */
    PGSGD_OPT_ATOMIC_UPDATES = 6,
    /* 1 = after each iteration, move the x anchor of every node whose start
     * offset has drifted past 8 to the rounded start point, so the FP32
     * offsets stay small, and copy the moved anchors into the step records
     * (anchored mode; default 1). */
    PGSGD_OPT_REBASE = 7,
    /* 1 = record CUDA events around every update-kernel launch on the
     * launching stream; read them with pgsgd_timing_read. Default 0. */
    PGSGD_OPT_TIMING = 8,
    /* Concurrency cap: the update kernel's grid is shrunk so that at most this
     * many updates are in flight at once, where the resident blocks would
     * otherwise hold more (0 = no cap; -1, the default,
     * = max(64, n_nodes / 16, N / 5120) for N = PGSGD_OPT_UPDATES_PER_STEP x
     * path steps updates per iteration). A cap below one block's worth also
     * shrinks the block (whole warps, at least 64 threads) and, with the
     * automatic shape, keeps 1 update per thread below 128. Concurrent
     * updates read points that others are about to move and overwrite each
     * other's moves; measured against the sequential oracle (paired by seed):
     * 1-12 k-node graphs of 4-12 paths came out 3.4 % above its sampled
     * stress with 2048 in flight and 0.26 % at n_nodes / 16; 1-4 k-node
     * graphs of 50-90 paths 1.95 % with 2048, 0.19 % at N / 5120; the
     * 200 k-node graph 0.4 % at n_nodes / 4 and 0.3 % at n_nodes / 16 (3.9x
     * the layout time). On the 5.5 M-node graph the resident threads, not
     * the cap, bound the updates in flight. */
    PGSGD_OPT_MAX_CONCURRENT = 9,
    /* Register budget of the update kernel: the number of resident 256-thread
     * blocks per SM its registers must allow (1 = compiler's choice; the
     * compiled variants are 1, 4, 6 for 1 update per thread, 1, 3, 4 for 2
     * and 1, 2, 3 for 4; the pipelined loop: 1, 3 for 1, 1, 2, 3 for 2 and
     * 1, 2 for 4).
     * Default 0 = automatic: for the plain loop 4 at 1 update per thread and
     * 3 at 2 (no spills); for the pipelined loop 2 at 2 updates per thread
     * (98 registers, no spills); else 1. */
    PGSGD_OPT_MIN_BLOCKS = 10,
    /* L2 fetch granularity in bytes set on the current context before each
     * layout (cudaLimitMaxL2FetchGranularity; 0 = leave it unchanged, the
     * default). Every access of the path is a random 32-byte sector. */
    PGSGD_OPT_L2_FETCH = 11,
    /* How a moved point is written when atomic updates are off: 0 = plain
     * store, 1 = 64-bit atomic exchange (default). Both replace the point
     * (last writer wins, the paper's racy store); on GB300 the exchange,
     * executed at L2, ran 1.4x (5 M-node graph) to 7x (200 k-node graph)
     * faster than every plain-store form (.wb, .cg, .cs, .wt, .relaxed.gpu,
     * L1::no_allocate) in the earlier 32-byte node-record design. */
    PGSGD_OPT_STORE_MODE = 12,
    /* 1 (default) = L2 residency hints: step records are read evict-first,
     * node records read and written evict-last, so the node array stays in
     * L2 while the step records stream past. 0 = no hints. */
    PGSGD_OPT_L2_HINTS = 13,
    /* 64-byte L2 prefetch-size hint on record loads: bit 0 = step records,
     * bit 1 = node records of the update kernel; bits 2 and 3 the same for
     * the sampled-stress kernel. Default 7 (both update-kernel loads, the
     * stress kernel's step loads): without it a random 32-byte miss of the
     * update kernel was promoted to 128 bytes, and the full chromosome
     * layout ran at 14.4e9 instead of 18.6e9 updates/s; the stress kernel's
     * step hint gained 3 % and its node hint lost 8 %. */
    PGSGD_OPT_PREFETCH64 = 14,
    /* 1 = software-pipelined update loop: each thread issues a trip's
     * step-record loads, then draws the next trip's pairs while they are in
     * flight (same draws and moves; compiled for updates per thread / min
     * blocks 1/1, 1/3, 2/1, 2/2, 2/3, 4/1 and 4/2). Default -1 = automatic: the
     * pipelined loop for the plain method, the plain loop under warp
     * merging, data reuse or PGSGD_OPT_ASYNC_DEPTH, which need it (setting 1
     * with them is an error). */
    PGSGD_OPT_PIPELINE = 15,
    /* Warp merging (Section V-B3): 1 = the cooling coin of update u is bit 0
     * of w2 of update 32 floor(u / 32), so a warp's 32 consecutive updates
     * take the same branch (one control draw, shared by shuffle). Draws and
     * moves otherwise unchanged. Needs PGSGD_OPT_PIPELINE = 0. Default 0. */
    PGSGD_OPT_WARP_MERGE = 16,
    /* Warp-level data reuse (Section VII-D). Data reuse factor DRF (1, 2, 4
     * or 8; default 1 = off): every selection performs DRF updates; the 32
     * selections of a group (= a warp) share one path drawn in proportion to
     * |p| from counter (group, t, 0x20000000); selection q draws step i
     * uniformly on it and its partner j as an update does; round k pairs
     * lane l's (i, e_i) with lane (l + o_k) mod 32's (j, e_j), o_0 = 0,
     * o_k = 1 + mulhi32(word k - 1 of blocks 1, 2 of the group counter, 31).
     * Step reduction factor SRF (1..2^20, default 1): an iteration has
     * ceil(updates_per_step x S / SRF) selections (or updates, with DRF 1).
     * Both need PGSGD_OPT_PIPELINE = 0. */
    PGSGD_OPT_DRF = 17,
    PGSGD_OPT_SRF = 18,
    /* Asynchronous step-record reads: 0 = off (default); D in {2, 3, 4, 6, 8}
     * = every thread keeps the step-record reads of its next D updates in
     * flight, copied into shared memory with cp.async, so outstanding reads
     * cost no registers (one update per thread; compiled for min blocks 4,
     * and 3 or 5 at D = 4). Same draws and moves as the plain loop. Ignored
     * under warp merging and data reuse. */
    PGSGD_OPT_ASYNC_DEPTH = 19,
    /* The same for the sampled-stress kernel (pgsgd_stress): 0 = off
     * (default), D in {2, 4, 8} samples' step-record reads in flight per
     * thread. Same samples and sums. */
    PGSGD_OPT_STRESS_ASYNC = 20,
    /* Grid of the sampled-stress kernel: W in 1..8 = W whole waves of the
     * blocks that fit on the GPU at once (default 1: every block slot stays
     * busy to the end; 2.09 s against 2.15 s for the chromosome graph's
     * 4.7e10 samples), 0 = 8 blocks per SM (2.67 waves at 3 resident). */
    PGSGD_OPT_STRESS_WAVES = 21
} pgsgd_option;

/* Device-resident graph: node records, packed step records, path table. */
typedef struct pgsgd_graph pgsgd_graph;

/* Result of pgsgd_stress (Eq. 2 and the interval of Section VI-B). */
typedef struct pgsgd_stress_result {
    double mean;        /* sampled path stress: sum of terms / n_valid */
    double stddev;      /* sample standard deviation of the terms */
    double ci_lo;       /* mean - 1.96 stddev / sqrt(n_valid) */
    double ci_hi;       /* mean + 1.96 stddev / sqrt(n_valid) */
    uint64_t n_valid;   /* samples with d_ref > 0 */
    uint64_t n_skipped; /* samples with d_ref = 0 (no defined term) */
} pgsgd_stress_result;

/* One drawn update, as pgsgd_debug_sample reports it (40 bytes). */
typedef struct pgsgd_sample {
    uint64_t g;       /* global step index drawn, in [0, S) */
    uint64_t i;       /* step index of n_i within its path */
    uint64_t j;       /* step index of n_j within its path */
    int64_t d_ref;    /* path distance of the two chosen endpoints (nt) */
    uint32_t path;    /* path id */
    uint8_t cooling;  /* 1 = power-law pair, 0 = uniform pair */
    uint8_t e_i;      /* 0 = start point, 1 = end point of n_i */
    uint8_t e_j;      /* 0 = start point, 1 = end point of n_j */
    uint8_t skip;     /* 0 = valid, 1 = path has < 2 steps, 2 = d_ref = 0 */
} pgsgd_sample;

/* Graph summary for callers and benchmarks. */
typedef struct pgsgd_info {
    uint64_t n_steps;          /* S = total path steps */
    uint64_t device_bytes;     /* device memory held by the handle */
    uint64_t max_path_steps;   /* longest path in steps */
    int64_t max_path_nt;       /* longest path in nucleotides */
    uint32_t n_nodes;
    uint32_t n_paths;
    int32_t device;            /* CUDA device ordinal the graph lives on */
    int32_t sm_count;
} pgsgd_info;

/*
 * Build the device-resident graph (Section II-A: nodes with sequence lengths
 * and paths that walk them; Section V-A: only the fields the layout reads).
 *
 *   node_len[n_nodes]        sequence length of every node, >= 1
 *   path_off[n_paths + 1]    path p owns steps [path_off[p], path_off[p+1]);
 *                            path_off[0] = 0, non-decreasing (empty paths ok)
 *   step_node[S]             node id of every step, < n_nodes
 *   step_rev[S]              1 = the path traverses the node in reverse, else 0
 *   step_pos[S]              int64 nucleotide position where the step starts:
 *                            0 at a path's first step, then the previous
 *                            step's position plus its node's length
 * S = path_off[n_paths]. All five arrays are on the host (on_device = 0) or
 * all on the device (on_device = 1); they are copied and validated on the GPU.
 * Limits (PGSGD_ERANGE beyond them): n_nodes < 2^31, every step position
 * < 2^32, n_paths <= 16384. Inconsistent arrays give PGSGD_EINVAL.
 * Synchronous: returns after the graph is resident. *out receives the handle
 * (NULL on failure). The graph lives on the current CUDA device.
 */
int pgsgd_create(const uint32_t *node_len, uint32_t n_nodes,
                 const uint64_t *path_off, uint32_t n_paths,
                 const uint32_t *step_node, const uint8_t *step_rev,
                 const int64_t *step_pos, int on_device, void *cuda_stream,
                 pgsgd_graph **out);

/* Release every resource of the handle (NULL is accepted). */
int pgsgd_destroy(pgsgd_graph *g);

int pgsgd_set_option(pgsgd_graph *g, int option, int64_t value);
int pgsgd_get_option(const pgsgd_graph *g, int option, int64_t *value);
int pgsgd_info_get(const pgsgd_graph *g, pgsgd_info *out);

/*
 * Replace the layout (Algorithm 1, output L: one 2-D segment per node).
 * xy[n_nodes][4] float64 = (start x, start y, end x, end y), host or device.
 * Stored in FP32 (anchored mode: integer x anchor + FP32 x offset, which
 * needs |x| < 2^30, PGSGD_ERANGE otherwise; y in plain FP32). Queued on the
 * stream; the caller's buffer may be reused when the call returns.
 */
int pgsgd_set_coords(pgsgd_graph *g, const double *xy, int on_device, void *cuda_stream);

/* Read the layout back into xy[n_nodes][4] float64 (exact value of the
 * stored FP32 representation). Synchronous for host xy, queued for device xy. */
int pgsgd_get_coords(pgsgd_graph *g, double *xy, int on_device, void *cuda_stream);

/*
 * Run iterations [iter_begin, iter_end) of a T = iter_max iteration layout
 * (Algorithm 1): each iteration launches one update kernel of
 * N = updates_per_step * S lock-free updates at learning rate eta_t.
 *   eta      host array of iter_max rates, or NULL for the annealing of
 *            Zheng et al.: eta_t = eta_max * exp(-lambda t),
 *            lambda = ln(eta_max / eta_min) / (T - 1); every rate, given
 *            or computed, must be finite and >= 0 (PGSGD_EINVAL otherwise,
 *            before any launch)
 *   eta_max  <= 0 selects (longest path in nucleotides)^2
 *   eta_min  <= 0 selects 0.01
 *   theta    Zipf exponent of the power-law pair choice, in [0, 4]
 *   seed     Philox key; update u of iteration t draws counter (u, t, block)
 * Iterations t with 2 t >= T always take the power-law pair (cooling).
 * Running [0, k) then [k, T) gives the same draws as [0, T) (resume).
 * Requires a layout (pgsgd_set_coords). Asynchronous on the stream.
 */
int pgsgd_layout(pgsgd_graph *g, uint32_t iter_max, const double *eta,
                 double eta_max, double eta_min, double theta, uint64_t seed,
                 uint32_t iter_begin, uint32_t iter_end, void *cuda_stream);

/*
 * Sampled path stress of the current layout (Eq. 2, Section VI-B): for every
 * path p with at least two steps, samples_per_step * |p| pairs (the paper
 * uses 100): step i uniform, step j uniform among the others, a coin for
 * each endpoint; the term ((|v_i - v_j| - d_ref) / d_ref)^2 in FP32, summed
 * in FP64; samples with d_ref = 0 are left out of n. Pass seed selects the
 * sample set (Philox counter (q, 0x80000000 | p, block)).
 * per_path (optional, host, [n_paths][3] float64): sum of terms, sum of
 * squared terms, number of valid samples, per path.
 * Synchronous. Uses a per-handle device scratch buffer.
 */
int pgsgd_stress(pgsgd_graph *g, uint32_t samples_per_step, uint64_t seed,
                 pgsgd_stress_result *out, double *per_path, void *cuda_stream);

/*
 * The pair each update u in [u_begin, u_begin + count) of iteration t (of
 * iter_max) draws, written to out[count] (host). Same sampler as the update
 * kernel; no coordinate is read or written. Synchronous.
 */
int pgsgd_debug_sample(pgsgd_graph *g, uint32_t t, uint32_t iter_max, double theta,
                       uint64_t seed, uint64_t u_begin, uint64_t count,
                       pgsgd_sample *out, void *cuda_stream);

/*
 * With data reuse on (PGSGD_OPT_DRF > 1): the DRF pairs of every selection q
 * in [q_begin, q_begin + count) of iteration t, out[count][DRF] (host),
 * round k in column k: g = the global step of i, i and path as drawn by
 * selection q, j / e_j / cooling those of the round's partner lane; skip = 1
 * when the path has < 2 steps or the partner selection is past the
 * iteration's ceil(updates_per_step x S / SRF) selections. Honors
 * PGSGD_OPT_WARP_MERGE. pgsgd_debug_sample also honors it. Synchronous.
 */
int pgsgd_debug_sample_reuse(pgsgd_graph *g, uint32_t t, uint32_t iter_max, double theta,
                             uint64_t seed, uint64_t q_begin, uint64_t count,
                             pgsgd_sample *out, void *cuda_stream);

/*
 * Jacobi sweep: for every update u in [u_begin, u_begin + count) of
 * iteration t, the FP32 change it would make to its two points, computed
 * from the current (frozen) layout at learning rate eta. out[count][4] float32
 * (host) = (dx_i, dy_i, dx_j, dy_j); skipped updates give zeros. The layout
 * is not modified. Synchronous.
 */
int pgsgd_debug_sweep(pgsgd_graph *g, uint32_t t, uint32_t iter_max, double eta,
                      double theta, uint64_t seed, uint64_t u_begin, uint64_t count,
                      float *out, void *cuda_stream);

/*
 * Path stress (Eq. 1, Section VI-A) of the current layout: for every path and
 * every pair of distinct steps i < j, the mean of ((|v_i - v_j| - d) / d)^2
 * over the four endpoint combinations with d_ref > 0, averaged over the pairs
 * with at least one such combination (value, host) and their number
 * (n_pairs, host, optional). FP32 terms, FP64 sums. Work grows as
 * sum_p |p|^2: meant for small graphs and for checking the sampled metric.
 * Synchronous.
 */
int pgsgd_full_stress(pgsgd_graph *g, double *value, uint64_t *n_pairs, void *cuda_stream);

/*
 * Differentiable sampled path stress. F is Eq. 2's estimator (Section VI-B)
 * over a fixed set of n_pairs samples (sample q: Philox counter
 * (q_lo, q_hi, 0xC0000000, 0) under `seed`; path in proportion to |p|, step
 * i uniform, partner j uniform among the other steps, a coin per endpoint;
 * samples with d_ref = 0 or on paths of fewer than two steps are left out):
 *   F = (1 / n_valid) sum_q ((|v_i - v_j| - d) / d)^2
 * pgsgd_dstress writes F and n_valid (host). Synchronous.
 */
int pgsgd_dstress(pgsgd_graph *g, uint64_t n_pairs, uint64_t seed, double *value,
                  uint64_t *n_valid, void *cuda_stream);

/*
 * Hand-written backward of the same objective: grad[n_nodes][4] (float32,
 * DEVICE memory, overwritten) = scale * sum_q d(t_q^2)/d(sx, sy, ex, ey),
 * t_q = (|v_i - v_j| - d) / d; pass scale = (upstream gradient) / n_valid
 * for dF. Contributions are added with vector atomics (order not fixed).
 * Asynchronous on the stream.
 */
int pgsgd_dstress_backward(pgsgd_graph *g, uint64_t n_pairs, uint64_t seed, double scale,
                           float *grad, void *cuda_stream);

/*
 * Gradient of the single-pair stress ((|v_i - v_j| - d) / d)^2 (Algorithm 1's
 * pair stress) of every update u in [u_begin, u_begin + count) of iteration t,
 * at the current layout: out[count][4] float32 (host) =
 * (d/dx_i, d/dy_i, d/dx_j, d/dy_j); zeros where the update is skipped.
 * Together with pgsgd_debug_sweep it shows each move equals
 * -(eta / 4) times this gradient while eta / d^2 < 1. Synchronous.
 */
int pgsgd_debug_pair_grad(pgsgd_graph *g, uint32_t t, uint32_t iter_max, double theta,
                          uint64_t seed, uint64_t u_begin, uint64_t count, float *out,
                          void *cuda_stream);

/*
 * Update-kernel timing (PGSGD_OPT_TIMING = 1): total milliseconds of all
 * update-kernel launches since the last reset, measured with CUDA events on
 * the launching stream, the number of launches and the updates they ran.
 * Synchronises the recorded events. reset = 1 clears the counters after
 * reading.
 */
int pgsgd_timing_read(pgsgd_graph *g, double *total_ms, uint64_t *launches,
                      uint64_t *updates, int reset);

/*
 * Sampled path stress without any device allocation. The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc, for example code whose device memory is owned entirely by
 * another allocator or a fixed preallocated budget (an embedding framework
 * that forbids outside allocations), or code that must not allocate at the
 * point of the call. It computes the same statistic as pgsgd_stress (same
 * samples for the same seed, FP32 terms, FP64 sums) straight from the
 * caller's raw arrays, with no graph handle:
 *   node_len, path_off, step_node, step_rev, step_pos   as for pgsgd_create,
 *                        all in DEVICE memory, already valid (not checked)
 *   xy[n_nodes][4]       float64 layout in DEVICE memory
 *   out                  one pgsgd_stress_result in DEVICE memory, written by
 *                        the last kernel of the call
 * Asynchronous on cuda_stream; the caller synchronises before reading *out.
 * Scratch: a fixed file-scope device array of 96 KiB that every GPU which
 * loads the library holds until the process exits; it has room for the
 * partial sums of 4096 blocks (the grid is capped there). Limit:
 * n_paths <= 8192 (PGSGD_ERANGE beyond, with a message). Every call looks
 * up the array's device address on the current device (cudaGetSymbolAddress)
 * and sets the kernel's shared-memory limit, so it stays valid after
 * cudaDeviceReset; the first call on a device may also load the library's
 * kernels, so make that first call before any stream capture. All calls
 * share the array (each call writes every slot it reads, so nothing is
 * cleared): calls that overlap on the GPU, on any streams, race on it.
 */
int pgsgd_stress_noalloc(const uint32_t *node_len, uint32_t n_nodes,
                         const uint64_t *path_off, uint32_t n_paths,
                         const uint32_t *step_node, const uint8_t *step_rev,
                         const int64_t *step_pos, const double *xy,
                         uint32_t samples_per_step, uint64_t seed,
                         pgsgd_stress_result *out, void *cuda_stream);

/*
 * Measurement helper, no counterpart in the paper: the L2 read bandwidth of
 * the current GPU in GB/s (*gbs, host), the ceiling for graphs whose records
 * fit in L2. Allocates a `bytes` buffer (1 MiB..1 GiB; keep it below the L2
 * size), warms it into L2, then times `reps` (1..1000) passes of mode 0 =
 * streaming 16-byte vector loads (bytes counted as read) or mode 1 = random
 * 16-byte loads, each counted as the 32-byte sector it costs. Synchronous;
 * frees everything it allocated.
 */
int pgsgd_l2_bandwidth(uint64_t bytes, uint32_t reps, int mode, double *gbs, void *cuda_stream);

/*
 * Measurement helper, no counterpart in the paper: the rate of random reads
 * from HBM (*loads_per_s, host: reads of the large buffer completed per
 * second), the ceiling of a kernel bound by random record reads, as the
 * update and stress kernels are on graphs whose 16-byte step records are far
 * larger than L2 (the memory-bound random access of Section III-B).
 * Allocates a `bytes` buffer (1..64 GiB, keep it several times the L2 size)
 * of 16-byte records cut into 90 equal "paths", and times `reps` (1..100)
 * launches of blocks_per_sm (1..64) 256-thread blocks per SM over
 * 4 x records units: unit Q takes path Q mod 90 and two records uniform on it
 * from one Philox4x32-10 block, read as the step records are (16-byte load,
 * evict-first, 64-byte L2 prefetch hint). mode 0 = those two reads; mode 1 =
 * plus two random 8-byte reads from an 88 MB array kept in L2 (an update's
 * two point reads). Multiply by 32 (the sector a read touches) or 64 (the
 * DRAM access it costs with the hint) for GB/s. Synchronous; frees
 * everything it allocated. PGSGD_EINVAL for arguments out of range,
 * PGSGD_ENOMEM when the buffers cannot be allocated.
 */
int pgsgd_hbm_gather_bandwidth(uint64_t bytes, uint32_t reps, int mode, int blocks_per_sm,
                               double *loads_per_s, void *cuda_stream);

/* Message of the calling thread's last failure ("" if none). */
const char *pgsgd_last_error(void);

/* Constant name of a status code. */
const char *pgsgd_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* PGSGD_H */
