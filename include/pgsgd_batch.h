/*
 * pgsgd_batch.h - batched PG-SGD layout: many independent pangenome graphs
 * laid out together on one GPU by libpgsgd.so.
 *
 * The paper lays out one graph per run (Algorithm 1, Section II-C) and
 * observes that small graphs cannot occupy a GPU while per-iteration kernel
 * launches dominate their run time (Section IV-B). A batch keeps the method
 * of every graph exactly as in pgsgd.h (graph g draws the same pairs as
 * pgsgd_layout on g alone with g's seed: Philox counter (u, t, block) keyed
 * by that seed; its own learning-rate schedule; lock-free updates) and only
 * changes how the work of all graphs is scheduled on the GPU. Conventions
 * (status codes, streams, on_device, ownership) are those of pgsgd.h.
 */
#ifndef PGSGD_BATCH_H
#define PGSGD_BATCH_H

#include <stdint.h>

#include "pgsgd.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pgsgd_batch pgsgd_batch;

/* Options for pgsgd_batch_set_option / pgsgd_batch_get_option. */
typedef enum pgsgd_batch_option {
    /* Schedule of the work (the updates of a graph's iteration are cut into
     * chunks of PGSGD_BOPT_CHUNK consecutive update indices):
     * 0 = one kernel launch per iteration covering all graphs (default):
     *     every graph gets `lanes` blocks, lane k runs the graph's chunks
     *     k, k + lanes, ...;
     * 1 = one persistent launch for all iterations: blocks claim chunks from
     *     per-graph queues (largest graph first; a block's first warp claims
     *     its next chunk while the other warps finish the current one); the
     *     block that completes a graph's last chunk of an iteration opens its
     *     next iteration, so graphs advance independently. Synchronous: the
     *     call waits for the kernel and returns PGSGD_ETIMEOUT if a block
     *     found no claimable work for PGSGD_BOPT_TIMEOUT_MS (a stuck queue);
     * 2 = one launch per graph per iteration (the comparison point). */
    PGSGD_BOPT_MODE = 1,
    /* Modes 0 and 2: 1 (default) = capture the layout's launches once into a
     * CUDA graph and replay it on later calls with the same shape; 0 = launch
     * directly. */
    PGSGD_BOPT_CUDA_GRAPH = 2,
    /* Threads per block, 64..256 in steps of 32 (default 256). */
    PGSGD_BOPT_BLOCK = 3,
    /* Updates each thread keeps in flight: 1, 2 (default) or 4. */
    PGSGD_BOPT_UPDATES_PER_THREAD = 4,
    /* Updates per chunk, 1..2^31 (default 16384). */
    PGSGD_BOPT_CHUNK = 5,
    /* Per-graph cap on updates in flight: graph g runs at most
     * max(1, cap / (block * updates per thread)) chunks at once; a cap
     * below one block's worth runs one chunk at a time on the block's first
     * max(32, cap / updates per thread) threads, rounded down to whole warps.
     * -1 (default) = max(64, nodes of g / 16, updates of g per iteration
     * / 5120), the single-graph rule;
     * 0 = no cap. */
    PGSGD_BOPT_MAX_CONCURRENT = 6,
    /* Updates per iteration of graph g = this value times its steps
     * (default 10, Algorithm 1). */
    PGSGD_BOPT_UPDATES_PER_STEP = 7,
    /* Mode 1: the longest a block may find no claimable work before the
     * kernel gives up (milliseconds, default 10000). */
    PGSGD_BOPT_TIMEOUT_MS = 8,
    /* 1 = record CUDA events around every pgsgd_batch_layout call on its
     * stream; read with pgsgd_batch_timing_read. Default 0. */
    PGSGD_BOPT_TIMING = 9,
    /* Testing only. 1 = in mode 1 the largest graph's first iteration never
     * counts as complete, so its queue stays closed and the kernel's bounded
     * waits expire: the call must return PGSGD_ETIMEOUT after about
     * PGSGD_BOPT_TIMEOUT_MS with the GPU context still usable. Default 0. */
    PGSGD_BOPT_STALL_TEST = 10,
    /* Mode 1: resident blocks per SM in the persistent grid; 0 (default) =
     * as many as the occupancy calculator allows. */
    PGSGD_BOPT_BLOCKS_PER_SM = 11,
    /* 1 = the software-pipelined update loop (PGSGD_OPT_PIPELINE of
     * pgsgd.h) inside every chunk. Default 0. */
    PGSGD_BOPT_PIPELINE = 12,
    /* 64-byte L2 prefetch-size hints, bits as PGSGD_OPT_PREFETCH64 of
     * pgsgd.h (bits 0-1 update kernels, bits 2-3 stress kernel). Default 7. */
    PGSGD_BOPT_PREFETCH64 = 13
} pgsgd_batch_option;

typedef struct pgsgd_batch_info {
    uint64_t n_steps;          /* all graphs' steps */
    uint64_t device_bytes;     /* device memory of the packed graphs */
    uint64_t last_launches;    /* kernel launches of the last layout call */
    uint32_t n_graphs;
    uint32_t n_nodes;          /* all graphs' nodes */
    uint32_t n_paths;          /* all graphs' paths */
    uint32_t max_graph_paths;  /* most paths of one graph */
    int32_t last_grid;         /* blocks of the last layout launch (mode 0, 1) */
    int32_t reserved;
} pgsgd_batch_info;

/*
 * Build a batch of G = n_graphs graphs, each given exactly as pgsgd_create
 * takes one graph (node lengths; per path, steps with node id, orientation
 * and int64 nucleotide position), concatenated:
 *   graph_node_off[G + 1]  host; graph g owns nodes [off[g], off[g+1]) of
 *                          node_len; off[0] = 0, non-decreasing
 *   graph_path_off[G + 1]  host; graph g owns paths [off[g], off[g+1]);
 *                          off[0] = 0, non-decreasing, <= 16384 per graph
 *   node_len[V]            V = graph_node_off[G] < 2^31
 *   path_off[P + 1]        over the concatenated steps, as in pgsgd_create
 *   step_node[S]           node id LOCAL to the step's graph
 *                          (< that graph's node count; PGSGD_EINVAL otherwise)
 *   step_rev[S], step_pos[S]  as in pgsgd_create
 * node_len, path_off and the step arrays are all on the host (on_device = 0)
 * or all on the device (on_device = 1). Validation and limits are those of
 * pgsgd_create except that P may reach 2^22. Synchronous. The batch's
 * coordinates are the concatenation of the graphs' [V_g][4] layouts.
 */
int pgsgd_batch_create(uint32_t n_graphs, const uint64_t *graph_node_off,
                       const uint64_t *graph_path_off, const uint32_t *node_len,
                       const uint64_t *path_off, const uint32_t *step_node,
                       const uint8_t *step_rev, const int64_t *step_pos,
                       int on_device, void *cuda_stream, pgsgd_batch **out);

int pgsgd_batch_destroy(pgsgd_batch *b);
int pgsgd_batch_set_option(pgsgd_batch *b, int option, int64_t value);
int pgsgd_batch_get_option(const pgsgd_batch *b, int option, int64_t *value);
int pgsgd_batch_info_get(const pgsgd_batch *b, pgsgd_batch_info *out);

/* Layout of all graphs, xy[V][4] float64 as in pgsgd_set_coords (anchored
 * FP32 storage; the batch kernels keep each node's anchor fixed). */
int pgsgd_batch_set_coords(pgsgd_batch *b, const double *xy, int on_device, void *cuda_stream);
int pgsgd_batch_get_coords(pgsgd_batch *b, double *xy, int on_device, void *cuda_stream);

/*
 * Iterations [iter_begin, iter_end) of a T = iter_max layout of every graph
 * (Algorithm 1).
 *   eta    host [G][iter_max] learning rates, or NULL: per graph, the
 *          annealing of pgsgd_layout with eta_max = (graph's longest path in
 *          nucleotides)^2 and eta_min = 0.01; given rates must be finite
 *          and >= 0 (PGSGD_EINVAL otherwise, before any launch)
 *   theta  Zipf exponent in [0, 4], the same for all graphs
 *   seeds  host [G] Philox keys, one per graph
 * The call uploads its per-graph tables from the host first, so it waits for
 * work already queued on the stream; the layout itself is then queued
 * asynchronously in modes 0 and 2 and waited for in mode 1 (see
 * PGSGD_BOPT_MODE).
 */
int pgsgd_batch_layout(pgsgd_batch *b, uint32_t iter_max, const double *eta,
                       double theta, const uint64_t *seeds, uint32_t iter_begin,
                       uint32_t iter_end, void *cuda_stream);

/*
 * Sampled path stress (Eq. 2, Section VI-B) of every graph's current
 * layout: out[G] (host), each exactly the statistic pgsgd_stress computes
 * on that graph alone (same samples for the same seed, paths numbered
 * within the graph). Synchronous.
 */
int pgsgd_batch_stress(pgsgd_batch *b, uint32_t samples_per_step, uint64_t seed,
                       pgsgd_stress_result *out, void *cuda_stream);

/*
 * The pairs that updates [u_begin, u_begin + count) of iteration t draw in
 * graph `graph` under `seed`, in the graph's own step and path numbering:
 * the same records pgsgd_debug_sample gives for that graph alone. Out on
 * the host. Synchronous.
 */
int pgsgd_batch_debug_sample(pgsgd_batch *b, uint32_t graph, uint32_t t, uint32_t iter_max,
                             double theta, uint64_t seed, uint64_t u_begin, uint64_t count,
                             pgsgd_sample *out, void *cuda_stream);

/* Milliseconds, launches and updates of the layout calls timed since the
 * last reset (PGSGD_BOPT_TIMING = 1); synchronises the recorded events. */
int pgsgd_batch_timing_read(pgsgd_batch *b, double *total_ms, uint64_t *launches,
                            uint64_t *updates, int reset);

/*
 * The schedule plan, on the host only (no GPU needed): for G graphs with
 * n_updates[g] updates per iteration and n_nodes[g] nodes, rank_to_graph[G]
 * receives the order in which mode 0 lays out lanes and mode 1 scans queues
 * (the graphs whose lanes run the most sequential rounds of updates
 * first, ties by most updates, then graph index), n_chunks[g] the chunks per
 * iteration, lanes[g] the chunks graph g may run at once (0 for a graph
 * without updates) and threads[g] the threads of a block that run graph
 * g's chunks (a multiple of 32, at most block). All six arrays are host
 * arrays of n_graphs entries owned by the caller. Arguments as the options
 * of the same names.
 */
int pgsgd_batch_plan(uint32_t n_graphs, const uint64_t *n_updates, const uint64_t *n_nodes,
                     int block, int updates_per_thread, uint64_t chunk,
                     int64_t max_concurrent, uint32_t *rank_to_graph,
                     uint32_t *n_chunks, uint32_t *lanes, uint32_t *threads);

#ifdef __cplusplus
}
#endif

#endif /* PGSGD_BATCH_H */
