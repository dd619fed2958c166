/*
 * dag.h -- C ABI of libdag.so: delayed-asynchronous pull PageRank and
 * Bellman-Ford SSSP on one GB300 GPU (sm_103a).
 *
 * Method: Blanco, McMillan, Low, "Delayed Asynchronous Iterative Graph
 * Algorithms", HPEC 2021. Each worker (here: a CTA) owns a contiguous block of
 * vertices balanced by in-neighbour count (Sec. III-A), computes its vertices
 * with a pull over their in-edges, and either writes each new value straight
 * into the global array (asynchronous, Sec. I), or to a separate array read
 * only in the next iteration (synchronous, Sec. I), or to a private buffer of
 * delta values that it copies to the global array when full and at the end of
 * its block (delayed asynchronous, Sec. III and III-B). One barrier separates
 * iterations (Sec. I).
 *
 * Conventions for every entry point:
 *  - Graphs are in-edge CSR: colidx[rowptr[v] .. rowptr[v+1]) are the sources u
 *    of the edges u -> v. rowptr/colidx are int32 (m < 2^31).
 *  - rowptr, colidx and the per-edge weight / value arrays start on a 16-byte
 *    boundary (any cudaMalloc or fresh torch allocation does); the sweeps copy
 *    them with TMA bulk copies. A solve given a misaligned array returns
 *    DAG_ERR_INVALID.
 *  - Pointers named d_* are DEVICE pointers on the current CUDA device; h_*
 *    are HOST pointers. All arrays belong to the caller; the library keeps no
 *    pointer to them after the call returns, except that a plan keeps the CSR
 *    pointers it was created with (the caller keeps them alive and unchanged
 *    until dag_plan_destroy).
 *  - stream is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream). Work is enqueued on it. When a host stats pointer is given, the
 *    call waits for the stream before returning.
 *  - Return value: DAG_OK (0) or a negative DAG_ERR_* code; dag_strerror()
 *    names it and dag_last_error_message() adds detail. Arguments are checked
 *    on the host before anything is enqueued; a rejected call changes nothing.
 *  - A solve that reaches max_iters without meeting its stopping rule returns
 *    DAG_ERR_NOT_CONVERGED and still writes its last iterate.
 *  - Every device-side wait (the grid barrier between iterations, the wait
 *    for a tile's staged inputs) has a time limit; when it runs out the kernel
 *    stops, the call returns DAG_ERR_BARRIER_TIMEOUT and the CUDA context stays
 *    usable.
 */
#ifndef DAG_H
#define DAG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DAG_OK 0
#define DAG_ERR_INVALID (-1)          /* bad argument: shape, range, null, delta < 0 ... */
#define DAG_ERR_NOT_CONVERGED (-2)    /* max_iters reached; outputs hold the last iterate */
#define DAG_ERR_BARRIER_TIMEOUT (-3)  /* a grid barrier wait ran out of time */
#define DAG_ERR_CUDA (-4)             /* a CUDA runtime call failed */
#define DAG_ERR_NOMEM (-5)            /* device allocation failed */

/* Update order (Sec. I and III-B). DAG_DELAYED with delta = 0 is DAG_ASYNC. */
typedef enum { DAG_SYNC = 0, DAG_ASYNC = 1, DAG_DELAYED = 2 } dag_variant;

/* In-edge CSR, device arrays. */
typedef struct {
    int32_t n;              /* vertices, >= 1 */
    int64_t m;              /* edges, 0 <= m < 2^31 */
    const int32_t* d_rowptr; /* [n+1], rowptr[0] = 0, nondecreasing, rowptr[n] = m */
    const int32_t* d_colidx; /* [m], each in [0, n) */
} dag_csr;

/* Result of one solve (host struct). */
typedef struct {
    int32_t iters;           /* sweeps run, the one that met the stopping rule included */
    int32_t err;             /* DAG_OK, DAG_ERR_NOT_CONVERGED or DAG_ERR_BARRIER_TIMEOUT */
    double residual;         /* last sweep: L1 change (PageRank) or vertices updated (SSSP) */
    float ms;                /* device time of the solve, CUDA events around it */
    int32_t workers;         /* CTAs that held a vertex block (the paper's thread count) */
    int32_t delta;           /* buffer size used (0 for sync/async) */
    int64_t flushes;         /* buffer flushes over the whole solve (delayed only) */
    int64_t edges_processed; /* m * iters; with DAG_SSSP_FRONTIER the edges of the tiles run */
} dag_stats;

typedef struct dag_plan dag_plan; /* opaque */

/*
 * Plan: out-degrees, per-vertex data and workspace for one graph (the
 * untimed setup step: Sec. III-A's static partition is computed per launch
 * shape and cached here). d_colidx entries are checked against [0, n) on the
 * device. The plan owns its workspace and frees it in dag_plan_destroy.
 * barrier_timeout_ms <= 0 selects the default (2000 ms). Plans take their
 * device memory from a pool the library keeps per device: up to 4 GiB of
 * what destroyed plans held stays mapped for later plans (a plan built and
 * destroyed per call maps its arrays once). dag_plan_destroy waits for the
 * device (as cudaFree would) before it returns the plan's memory.
 */
int dag_plan_create(const dag_csr* csr, int32_t barrier_timeout_ms, dag_plan** out);
int dag_plan_destroy(dag_plan* plan);

/* Copies the plan's out-degree array (int32 [n]) into d_outdeg (device). */
int dag_plan_out_degree(const dag_plan* plan, int32_t* d_outdeg, void* stream);

/*
 * The static partition the sweep kernels use for `workers` CTAs (Sec. III-A):
 * h_start[p] (host, workers+1 values) is the first vertex of block p, chosen
 * so that every block carries about (n + m)/workers of the weight
 * (in-degree + 1) per vertex: h_start[p] = min { v : v + rowptr[v] >=
 * ceil(p (n+m) / workers) }. Synchronous (waits for the result).
 */
int dag_partition(dag_plan* plan, int32_t workers, int32_t* h_start);

/* Number of CTAs the persistent kernel of this (variant, delta) runs with. */
int dag_workers(dag_plan* plan, dag_variant variant, int32_t delta, int32_t* out_workers);

/*
 * Caps the CTAs (workers, Sec. III-A blocks) of later solves on this plan at
 * max_workers (0 = as many as can be resident). Fewer workers mean longer
 * blocks, i.e. more rows per CTA; the autotuner varies it.
 */
int dag_plan_set_worker_cap(dag_plan* plan, int32_t max_workers);
/* (With DAG_WARP_WORKERS the cap counts CTAs too: eight warp workers each.) */

/* Flags of dag_pagerank / dag_sssp. */
#define DAG_PR_WARM_START 1 /* start from d_rank instead of the teleport vector (PageRank) */
/*
 * How a delayed sweep reads the global array (Sec. III-C's "global reads").
 * Default: ordinary loads, which may be served from the SM's L1, with the
 * CTA's view refreshed (an acquire fence) at each of its flushes, so delta
 * sets both how often a worker publishes and how often it takes in others'
 * values. DAG_READ_COHERENT: every read goes to L2, the point where all CTAs'
 * stores meet (as fresh as the asynchronous form). DAG_READ_CACHED: ordinary
 * loads refreshed only by the grid barrier between sweeps. The asynchronous
 * form takes DAG_READ_CACHED too: its gathers then become ordinary loads (L1)
 * refreshed by the grid barrier instead of L2 loads, so a value read is at
 * most one sweep old (still as fresh as the synchronous form's) while its own
 * stores stay in place; with DAG_SSSP_FRONTIER as well.
 */
#define DAG_READ_COHERENT 2
#define DAG_READ_CACHED 4
/*
 * Local reads (Sec. III-C): a delayed sweep's CTA reads its own values that
 * are still in its buffer from the buffer, so they reach its later rows before
 * the flush. Combines with one DAG_READ_* policy for everything else.
 */
#define DAG_READ_LOCAL 8
/*
 * Own-block reads through L1 (asynchronous form only): the CTA reads values
 * of its own vertex block with ordinary loads, which may hit the SM's L1, and
 * other blocks' values through L2. Only the owning CTA writes its block and
 * its barriers order those stores before its later loads, so every value read
 * is as fresh as in the default form; results differ only by the order in
 * which concurrent CTAs' writes are seen. Helps when workers read mostly
 * their own block (a clustered graph, Sec. IV-C); the choice is left to the
 * caller (or to a tuner).
 */
#define DAG_READ_OWN_L1 16
/*
 * Frontier Bellman-Ford (dag_sssp / dag_sssp_u8, synchronous or asynchronous
 * form; the conditionally written updates of Sec. V): a merge-path tile of
 * in-edges runs in a sweep only when one of its edges' sources got a smaller
 * distance in the previous sweep (or the tile lies between such an edge and
 * the end of its target's row); sweep 0 runs every tile. Distances are those
 * of the plain sweep (the synchronous trajectory is the same, sweep for
 * sweep); dag_stats.edges_processed counts the edges actually run. The first
 * solve with a launch shape builds the out-CSR row pointers and, per edge,
 * the tile of its in-CSR position (CTA tiles also the tile ending its
 * target's row): 4n + 8m bytes on CTA tiles, 4n + 4m on warp tiles, kept in
 * the plan. DAG_ERR_INVALID for PageRank or the delayed form.
 */
#define DAG_SSSP_FRONTIER 32
/*
 * Warp workers (dag_pagerank, dag_sssp, dag_sssp_u8; every variant): the
 * worker of Sec. III-A is one warp instead of one CTA. The merge path of the
 * whole graph (rows and in-edges in vertex order) is cut into tiles of
 * dag_warp_tile_items(plan) items and each warp takes an equal run of them, so
 * workers are balanced by in-degree + 1 as Sec. III-A asks; a warp owns the
 * rows that end in its run, and a row whose in-edges span several runs gets
 * the earlier runs' partial sums at the end of the sweep. delta counts rows
 * per warp (each warp has its own buffer). No CTA-wide barrier inside a sweep.
 * The asynchronous form reads through L2 (DAG_READ_CACHED: ordinary loads,
 * refreshed by the barrier between sweeps). With DAG_SSSP_FRONTIER
 * (asynchronous Bellman-Ford only) each warp also lists its rows that got a
 * smaller distance; after a sweep whose changed rows have few out-edges (at
 * most dag_plan_set_warp_frontier_marks per warp tile, 1 by default) only the
 * warp tiles holding those out-edges run, claimed by any warp, each row they
 * touch relaxed with an atomic minimum. DAG_ERR_INVALID with DAG_READ_LOCAL,
 * DAG_READ_OWN_L1, or DAG_SSSP_FRONTIER in another form.
 */
#define DAG_WARP_WORKERS 64
/*
 * Ordered warp sweeps (asynchronous form of dag_pagerank, dag_sssp,
 * dag_sssp_u8; implies warp workers): the warps take the tiles of the whole
 * merge path in turn, tile t to warp t mod W, so a sweep visits the vertices
 * in vertex order across the GPU, one in-order stream as a single worker's
 * asynchronous sweep (Sec. I) with every warp on it, instead of one stream per
 * worker; rows spanning tiles are finished by a bounded look-back over per-tile
 * published partials. DAG_READ_CACHED selects ordinary (L1) gathers, else L2.
 * With DAG_SSSP_FRONTIER (asynchronous Bellman-Ford): the warp-tile frontier
 * whose dense sweeps give each CTA the tiles of its warps' runs (a Sec. III-A
 * block), taken by its warps in turn, a row split over tiles relaxed by each
 * tile's atomic minimum. DAG_ERR_INVALID with the synchronous or delayed form.
 */
#define DAG_WARP_ORDERED 128
/*
 * Warp tile shape of the plan's warp-worker sweeps: 32 lanes x items_per_lane
 * items (5, 7 or 11; 7 when a plan is created), a tuning choice. Shorter tiles
 * mean more tiles in flight per warp's run; longer ones, fewer merge-path
 * searches per item. DAG_ERR_INVALID for another value or a null plan.
 */
int dag_plan_set_warp_tile(dag_plan* plan, int32_t items_per_lane);
/* Items (rows + in-edges) per warp tile of the plan's warp-worker sweeps (the default shape's for NULL). */
int32_t dag_warp_tile_items(const dag_plan* plan);
/*
 * Warp-tile frontier (DAG_WARP_WORKERS | DAG_SSSP_FRONTIER): the next sweep
 * runs only the stamped warp tiles when the out-degree sum of the rows the
 * sweep lowered is at most marks_per_tile x the warp tiles; 1 when a plan is
 * created, 0 keeps every sweep dense. A tuning choice. DAG_ERR_INVALID for a
 * value outside [0, 1e6] or a null plan.
 */
int dag_plan_set_warp_frontier_marks(dag_plan* plan, float marks_per_tile);

/*
 * PageRank (Sec. IV-A; stopping rule Sec. IV):
 *   r'_v = (1-d) t_v + d ( sum_{u in in(v)} M_vu r_u + D/n ),
 * M_vu = 1/outdeg(u) when d_val is NULL, else d_val[e] (P_vu per in-edge e,
 * e.g. from dag_normalize_weights). t = d_teleport (device, n, sum 1) or 1/n
 * when NULL. D is the dangling mass, formed as T - N (T = sum t, N = mass on
 * vertices with out-edges) from the global array as each tile of rows is
 * computed. Stops after the first sweep whose sum_v |r'_v - r_v| <= tol.
 * d in (0,1), tol > 0, max_iters >= 1, delta >= 0 (counted in 32-bit vertex
 * values, Sec. III-B; delta >= rows per CTA flushes once per sweep). d_rank
 * (device, float [n]) receives r; with DAG_PR_WARM_START it also gives r^0.
 * Without it r^0 = t. FP32 values, FP64 residual and dangling sums.
 * flags: DAG_PR_WARM_START | one DAG_READ_* (delayed form; the async form takes DAG_READ_CACHED) |
 * DAG_READ_OWN_L1 (async form only).
 * A delayed sweep with 0 < delta < dag_tile_items() cuts its tiles so that
 * none completes more than delta rows, so the buffer is flushed after about
 * every delta rows (a tile's rows are computed together and flushed at its end).
 */
int dag_pagerank(dag_plan* plan, float d, double tol, dag_variant variant, int32_t delta,
                 int32_t max_iters, const float* d_teleport, const float* d_val, float* d_rank,
                 int32_t flags, dag_stats* h_stats, void* stream);

/*
 * Bellman-Ford SSSP (Sec. IV): dist'_v = min(dist_v, min over in-edges with
 * dist_u finite of dist_u + w_uv), every value stored every sweep, changed
 * or not (Sec. IV); stops after a sweep that lowered no value. d_w: uint32 weight per in-edge (device, [m]); d_dist (device,
 * uint32 [n]) receives the distances, 0xFFFFFFFF for unreachable vertices.
 * flags: DAG_READ_* (delayed form; the async form takes DAG_READ_CACHED) | DAG_READ_OWN_L1 (async form only) |
 * DAG_SSSP_FRONTIER (sync and async forms).
 */
int dag_sssp(dag_plan* plan, uint32_t src, dag_variant variant, int32_t delta, int32_t max_iters,
             const uint32_t* d_w, uint32_t* d_dist, int32_t flags, dag_stats* h_stats, void* stream);

/*
 * dag_sssp with one-byte weights (d_w8: uint8 per in-edge, device, [m]) for
 * graphs whose weights lie in [0, 255], such as those of Sec. IV's runs
 * here (w in [1, 255]): the weight stream of each sweep shrinks from 4m to m
 * bytes. Same results and errors as dag_sssp with the same weights.
 */
int dag_sssp_u8(dag_plan* plan, uint32_t src, dag_variant variant, int32_t delta, int32_t max_iters,
                const uint8_t* d_w8, uint32_t* d_dist, int32_t flags, dag_stats* h_stats, void* stream);

/* Result of a batched solve (host struct). */
typedef struct {
    int32_t sweeps;          /* sweeps the launch ran (the slowest column's) */
    int32_t err;             /* DAG_OK, DAG_ERR_NOT_CONVERGED or DAG_ERR_BARRIER_TIMEOUT */
    float ms;                /* device time */
    int32_t workers;
    int32_t delta;
    int64_t column_sweeps;   /* sum over columns of the sweeps each ran */
    int32_t graph;           /* 1: the launch was a replay of the plan's CUDA graph of its shape, 0: direct */
} dag_batch_stats;

/*
 * Batched personalized PageRank: B teleport columns in one persistent launch
 * (no counterpart in the paper; each column is the PageRank of dag_pagerank
 * with its own teleport). d_V: row-major float [n][B] (column c = teleport of
 * problem c, sum 1). d_R: row-major float [n][B], receives the ranks (r^0 = V).
 * Each column stops on its own at its first sweep with L1 change <= tol and
 * is frozen from then on. d_iters (device int32 [B]) receives each column's
 * sweep count. B in [1, 1024]. delta as in dag_pagerank (rows per CTA).
 */
int dag_ppr_batched(dag_plan* plan, float d, double tol, dag_variant variant, int32_t delta,
                    int32_t max_iters, int32_t B, const float* d_V, float* d_R, int32_t* d_iters,
                    dag_batch_stats* h_stats, void* stream);

/*
 * Batched Bellman-Ford: B sources in one persistent launch; d_src (device
 * uint32 [B]); d_D row-major uint32 [n][B] receives the distances; d_iters
 * (device int32 [B]) each column's sweep count (a column stops after a sweep
 * that lowered none of its values). B in [1, 1024].
 */
int dag_sssp_batched(dag_plan* plan, dag_variant variant, int32_t delta, int32_t max_iters, int32_t B,
                     const uint32_t* d_src, const uint32_t* d_w, uint32_t* d_D, int32_t* d_iters,
                     dag_batch_stats* h_stats, void* stream);

/* dag_sssp_batched with one-byte weights (d_w8: uint8 per in-edge, device, [m]); same results as
 * dag_sssp_batched with the same weights, a quarter of the weight stream per sweep. */
int dag_sssp_batched_u8(dag_plan* plan, dag_variant variant, int32_t delta, int32_t max_iters, int32_t B,
                        const uint32_t* d_src, const uint8_t* d_w8, uint32_t* d_D, int32_t* d_iters,
                        dag_batch_stats* h_stats, void* stream);

/*
 * Batched launches through CUDA graphs (on != 0, the default for a new plan;
 * 0 launches directly).
 * dag_ppr_batched and dag_sssp_batched then capture each launch shape (kernel,
 * grid, block, shared memory, control block) once into a graph owned by the
 * plan: the reset of the per-column control block and the one cooperative
 * kernel launch. Later calls of that shape replay it with their own arguments.
 * When capture or instantiation fails, that shape falls back to the direct
 * launch for the plan's lifetime. Results do not depend on the setting.
 * dag_plan_destroy releases the graphs. Returns DAG_OK, or DAG_ERR_INVALID
 * for a null plan.
 */
int dag_plan_set_batched_graph(dag_plan* plan, int32_t on);
/*
 * Kernel of the plan's batched synchronous and asynchronous solves with 32,
 * 64, 128 or 256 columns: on (1, when a plan is created) a warp owns all B
 * columns (B / 32 per lane, one vector access each) and an eighth of each
 * merge-path tile, so a source vertex's B values are gathered by one warp in
 * one burst; off (0), and always for other column counts and the delayed
 * form, each warp owns 32 columns and the CTA's warps walk every edge
 * together. Results agree within rounding (the same sweep; sums may be added
 * in another order). DAG_ERR_INVALID for a null plan.
 */
int dag_plan_set_batched_wide(dag_plan* plan, int32_t on);

/*
 * Out-edge CSR of the plan's graph (for the adjoint pull). d_out_rowptr
 * (device int32 [n+1]), d_out_colidx (device int32 [m]: targets v of u's
 * out-edges, ascending), d_perm (device int32 [m]): in-edge index of each
 * out-edge, so that out-edge k is in-edge d_perm[k].
 */
int dag_transpose(dag_plan* plan, int32_t* d_out_rowptr, int32_t* d_out_colidx, int32_t* d_perm,
                  void* stream);

/*
 * Row normalisation of raw edge weights into the transition matrix: d_s[u] =
 * sum of d_w over u's out-edges (device float [n]), d_val[e] = d_w[e] /
 * d_s[src(e)] (device float [m], in-edge order). d_w > 0 expected. (M_vu of
 * dag_pagerank; no counterpart in the paper.) The first call on a plan sorts
 * its edges by source once and keeps that order in the plan (4 (n + m) bytes
 * more, freed by dag_plan_destroy); every call then runs asynchronously on
 * the stream. Each d_s[u] is summed in a fixed order: repeated calls on the
 * same weights give the same bits.
 */
int dag_normalize_weights(dag_plan* plan, const float* d_w, float* d_val, float* d_s, void* stream);

/*
 * d_out[k] = d_src[d_idx[k]] for k < m (device arrays; d_idx in range is the
 * caller's duty). Puts per-edge values into out-edge order with
 * dag_transpose's d_perm, e.g. d_val_out for dag_pagerank_adjoint.
 */
int dag_gather_f32(const float* d_src, const int32_t* d_idx, int64_t m, float* d_out, void* stream);

/*
 * PageRank adjoint (no counterpart in the paper): for a loss with dL/dr = c,
 * solves lambda = c + d M^T lambda + d g (sum_v lambda_v)/n (g: vertices with
 * no out-edges) by the same sweep (variant, delta) pulled over the out-edge
 * CSR held by out_plan (a plan created on dag_transpose's output), with
 * d_val_out[k] = P of out-edge k. Stops at L1 change <= tol * ||c||_1. Then
 * (with d_rank the forward result, d_s the normaliser, d_val the in-edge P):
 *   d_grad_w[e] = d r_u (lambda_v - (M^T lambda)_u) / s_u  for in-edge e = (u -> v),
 *   d_grad_t[v] = (1 - d) lambda_v.
 * d_lambda (device float [n], nullable) receives lambda. flags: the read path
 * of the adjoint sweep, as for dag_pagerank (one DAG_READ_* for the delayed
 * form, DAG_READ_CACHED or DAG_READ_OWN_L1 for the asynchronous form,
 * DAG_WARP_WORKERS, DAG_WARP_ORDERED); 0 for the default. Every form deflates
 * the slow error mode along the all-ones vector after each sweep short of the
 * stopping rule (the iteration operator maps 1 to d 1), which leaves the fixed
 * point unchanged.
 */
int dag_pagerank_adjoint(dag_plan* in_plan, dag_plan* out_plan, float d, double tol, dag_variant variant,
                         int32_t delta, int32_t max_iters, const float* d_val, const float* d_val_out,
                         const float* d_s, const float* d_rank, const float* d_c, float* d_grad_w,
                         float* d_grad_t, float* d_lambda, int32_t flags, dag_stats* h_stats, void* stream);

/*
 * PageRank with no device allocation. This is an interface convenience with
 * no counterpart in the paper. It is for callers that cannot call cudaMalloc
 * at solve time, for instance an application whose device memory is owned by
 * its own pool allocator, or a latency-bound service that cannot accept
 * cudaMalloc's implicit device synchronisation. It computes what dag_pagerank
 * computes for the in-edge CSR *csr (same arguments; val is not supported),
 * without a plan. Its scratch (out-degrees, state buffers, control block,
 * partition) lives in one fixed device array of about 17 MiB inside the
 * library, which every GPU that loads the library keeps until exit.
 *  - Limits: n <= DAG_NOALLOC_MAX_N and m <= DAG_NOALLOC_MAX_M; a larger
 *    graph returns DAG_ERR_INVALID and changes nothing.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current and keeps it for the
 *    process. A device reset
 *    (cudaDeviceReset) invalidates the kept address: after one, this entry
 *    point must not be called again in the same process.
 *  - The call checks the CSR on the device (rowptr order, colidx range) and
 *    returns DAG_ERR_INVALID for a bad one.
 *  - All calls share the array, and it keeps the previous call's contents
 *    (each call clears what it needs zeroed). Calls whose GPU work overlaps,
 *    for instance on two streams, race on it: serialise them.
 *  - The call waits for `stream` and reads its status back to the host, so
 *    it cannot be captured into a CUDA graph; h_stats->ms is left 0.
 */
#define DAG_NOALLOC_MAX_N (1 << 20)
#define DAG_NOALLOC_MAX_M (1 << 24)
int dag_pagerank_noalloc(const dag_csr* csr, float d, double tol, dag_variant variant, int32_t delta,
                         int32_t max_iters, const float* d_teleport, float* d_rank, dag_stats* h_stats,
                         void* stream);

/*
 * Measurement aid (no counterpart in the paper): the time of one pass that
 * streams d_idx[0..m) and gathers d_x[d_idx[e]] (device arrays; every index
 * must lie in [0, n), which the caller guarantees, e.g. a plan's colidx),
 * four gathers in flight per thread, nothing else. coherent != 0 gathers with
 * gpu-scope relaxed loads (as the asynchronous sweep), else with ordinary
 * loads (as the synchronous and delayed sweeps). *h_ms receives the mean over
 * `repeats` passes. This is the ceiling a sweep's gathers cannot beat.
 */
int dag_probe_gather(const int32_t* d_idx, int64_t m, const float* d_x, int32_t n, int32_t coherent,
                     int32_t repeats, float* h_ms, void* stream);

/*
 * Access matrix of the static partition into `workers` blocks (Sec. IV-C,
 * Fig. 5): d_counts[i * workers + j] (device uint64 [workers^2]) = number of
 * in-edge reads made while computing block i's vertices of vertices owned by
 * block j, i.e. edges u -> v with v in block i and u in block j. The diagonal
 * counts a block's reads of its own values. 1 <= workers <= 4096.
 */
int dag_access_matrix(dag_plan* plan, int32_t workers, uint64_t* d_counts, void* stream);

/*
 * Status of the plan's last single-vector solve (dag_pagerank, dag_sssp,
 * dag_sssp_u8, the adjoint's out_plan) without waiting for it: enqueues on
 * `stream` a copy of {err (DAG_OK or DAG_ERR_BARRIER_TIMEOUT), converged
 * (0/1), sweeps run} into d_status (device int32 [3]). For callers that launch
 * solves back to back with h_stats = NULL and check them afterwards.
 */
int dag_plan_last_status(const dag_plan* plan, int32_t* d_status, void* stream);

/*
 * Row sharding across GPUs (one process per GPU, every GPU holding the whole
 * graph in its own plan): the static partition of Sec. III-A at GPU
 * granularity (dag_partition with one block per GPU) gives each GPU a row
 * range; a synchronous sweep (Sec. I) is one dag_*_sweep_rows call per GPU
 * on the whole previous iterate, followed by an exchange of the new row
 * ranges (an all-gather) and of the two FP64 sums (an all-reduce) between
 * the GPUs. No counterpart in the paper beyond its synchronous sweep.
 *
 * PageRank keeps the state x of the sweeps: x_v = r_v / outdeg(v) for a
 * vertex with out-edges, r_v for one without. dag_rank_to_state converts r
 * into x (d_r, d_x device float [n]) and, when d_linked_mass (device double)
 * is given, writes the mass on vertices with out-edges N = sum r_v there;
 * dag_state_to_rank converts back. Both enqueue on `stream`, no wait.
 */
int dag_rank_to_state(const dag_plan* plan, const float* d_r, float* d_x, double* d_linked_mass, void* stream);
int dag_state_to_rank(const dag_plan* plan, const float* d_x, float* d_r, void* stream);
/*
 * One synchronous PageRank sweep (the row update of dag_pagerank) of rows
 * [row_lo, row_hi) from the whole previous iterate d_x_in (state form, device
 * float [n]): d_x_out[row_lo .. row_hi) receive the new states (the rest of
 * d_x_out is not touched). teleport_total = sum of d_teleport (1 when NULL,
 * uniform); linked_mass = N of d_x_in's iterate (the dangling mass is
 * teleport_total - linked_mass). d_sums (device double [2]) receives the
 * range's sum |r' - r| and its N of the new iterate. No wait; the sweep's
 * grid barrier is bounded as in every solve.
 */
int dag_pagerank_sweep_rows(dag_plan* plan, float d, int32_t row_lo, int32_t row_hi, const float* d_teleport,
                            double teleport_total, double linked_mass, const float* d_x_in, float* d_x_out,
                            double* d_sums, void* stream);
/*
 * One synchronous Bellman-Ford sweep of rows [row_lo, row_hi) with one-byte
 * weights: d_dist_out[v] = min(d_dist_in[v], min over in-edges of
 * d_dist_in[u] + w) for v in the range; d_sums[0] = rows lowered (FP64).
 */
int dag_sssp_sweep_rows(dag_plan* plan, int32_t row_lo, int32_t row_hi, const uint8_t* d_w8,
                        const uint32_t* d_dist_in, uint32_t* d_dist_out, double* d_sums, void* stream);

/* Items (rows + in-edges) per merge-path tile of the sweeps, the unit the
 * frontier runs or skips; fixed when the library is compiled. */
int32_t dag_tile_items(void);

/* Names an error code. Never NULL. */
const char* dag_strerror(int code);
/* Detail of the last error raised on the calling host thread ("" if none). */
const char* dag_last_error_message(void);

/*
 * Test hook for the failure path: when nonzero, the next solve on this plan
 * makes CTA 0 leave before its first grid barrier, so the others' bounded
 * waits run out (after timeout_ms) and the call returns
 * DAG_ERR_BARRIER_TIMEOUT. Resets itself after one solve.
 */
int dag_debug_skip_barrier_once(dag_plan* plan, int32_t timeout_ms);

/*
 * Test hook for the staging waits of the asynchronous sweep: the next
 * asynchronous solve on this plan announces 16 more bytes than it copies for
 * CTA 0's first tile, so that tile's bounded wait runs out (after timeout_ms)
 * and the call returns DAG_ERR_BARRIER_TIMEOUT. Resets itself after one
 * asynchronous solve.
 */
int dag_debug_stall_staging_once(dag_plan* plan, int32_t timeout_ms);

#ifdef __cplusplus
}
#endif

#endif /* DAG_H */
