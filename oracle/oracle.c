/*
 * CPU oracle for delayed-asynchronous pull PageRank and Bellman-Ford SSSP.
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this library. It shares no code with the CUDA path
 * (the two meet only in the seeded input generators).
 *
 * Everything here is plain and serial unless it says otherwise, in fp64 for
 * PageRank and exact unsigned integers for SSSP, following the paper's steps:
 *
 *  - Sync (Sec. I, Sec. III-B with delta = "infinity"): every vertex is computed
 *    from the previous iteration's values; results go to a separate array.
 *  - Delayed asynchronous with P workers and buffer delta (Sec. III, III-B):
 *    vertices are split into P contiguous blocks balanced by in-neighbour count
 *    (Sec. III-A); each worker computes its rows in order, reading only the
 *    global array (the "global read" form, Sec. III-C), and appends results to a
 *    private buffer that it copies into the global array when it holds delta
 *    values or when the worker has finished its block. delta = 0 writes each
 *    value straight away: the asynchronous algorithm (Sec. III-B).
 *    The P workers run in a fixed round-robin: in each tick every worker with
 *    rows left computes one row from the global array as it stood at the start
 *    of the tick; writes and flushes made in a tick are visible from the next.
 *    With P = 1 this is exactly Gauss-Seidel (delta = 0) or exactly Jacobi
 *    (delta >= n), which the tests use as pins.
 *  - PageRank (Sec. IV-A: a pull update that combines in-neighbour scores):
 *      r'_v = (1-d) t_v + d * ( sum_{u in in(v)} M_vu r_u + D/n ),
 *    M_vu = 1/outdeg(u) (or a given per-edge P_vu), t the teleport vector
 *    (uniform 1/n when absent) and D the dangling mass, spread uniformly. The
 *    paper does not say how D is formed. Here it is what the vertices with
 *    out-edges leave of the total: D = T - N, T = sum_v t_v, N = sum of r over
 *    vertices with out-edges, read from the global array as it stands when the
 *    row is computed (sync: the previous iterate). At the fixed point, and on
 *    every exact sync iterate from sum r0 = T, this equals the sum of r over the
 *    vertices without out-edges, so the fixed point and the sync trajectory are
 *    those of the plain definition; an in-place sweep, though, no longer carries
 *    an error in the total mass from one sweep to the next.
 *    Termination (Sec. IV): stop after the first sweep whose total absolute
 *    change sum_v |r'_v - r_v| is <= tol; "iters" counts the sweeps run,
 *    that last one included.
 *  - Bellman-Ford (Sec. IV): d'_v = min(d_v, min_{u in in(v), d_u < INF} d_u + w_uv),
 *    stop after a sweep that changed nothing. Every sweep stores every value,
 *    changed or not (Sec. IV).
 *  - Dijkstra's algorithm (binary heap) gives the exact distances.
 *  - The PageRank adjoint (no counterpart in the paper; the plain definition of
 *    the gradient of a linear fixed point) and its edge/teleport gradients.
 *  - orc_*_threads: the paper's own CPU scheme with OpenMP threads, FP32 scores,
 *    timed as the CPU baseline. Its results are checked like the GPU's.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <omp.h>

#define ORC_INF 0xFFFFFFFFu

/* ------------------------------------------------------------------------- */
/* Graph helpers                                                              */
/* ------------------------------------------------------------------------- */

/* outdeg[u] = number of edges u -> v, i.e. occurrences of u among all in-lists. */
void orc_out_degree(int32_t n, const int32_t* rowptr, const int32_t* colidx, int32_t* outdeg)
{
    memset(outdeg, 0, (size_t)n * sizeof(int32_t));
    for (int32_t v = 0; v < n; ++v)
        for (int32_t e = rowptr[v]; e < rowptr[v + 1]; ++e) outdeg[colidx[e]] += 1;
}

/*
 * Static contiguous partition into P blocks, balanced by in-neighbour count
 * (Sec. III-A). Each vertex weighs (in-degree + 1): its in-edges plus its own
 * store. start[p] is the first vertex whose cumulative weight before it,
 * v + rowptr[v], reaches ceil(p * (n + m) / P); start[0] = 0, start[P] = n.
 */
void orc_partition(int32_t n, const int32_t* rowptr, int32_t P, int32_t* start)
{
    int64_t total = (int64_t)n + rowptr[n];
    int32_t v = 0;
    start[0] = 0;
    for (int32_t p = 1; p < P; ++p) {
        int64_t target = ((int64_t)p * total + P - 1) / P;
        while (v < n && (int64_t)v + rowptr[v] < target) ++v;
        start[p] = v;
    }
    start[P] = n;
}

/* ------------------------------------------------------------------------- */
/* PageRank                                                                   */
/* ------------------------------------------------------------------------- */

typedef struct {
    int32_t n;
    const int32_t* rowptr;
    const int32_t* colidx;
    const double* val;    /* P_vu per in-edge, or NULL for 1/outdeg(u) */
    const int32_t* outdeg;
    double d;
    const double* tele;   /* NULL: uniform 1/n */
    double T;             /* sum of tele (1 when uniform) */
} pr_problem;

/* One row of the PageRank map, reading r; in-neighbours u in [lo, hi) are read
 * from buf instead (a worker's own unflushed values, Sec. III-C local reads). */
static double pr_row_view(const pr_problem* q, const double* r, const double* buf, int32_t lo, int32_t hi,
                          double D, int32_t v)
{
    double s = 0.0;
    for (int32_t e = q->rowptr[v]; e < q->rowptr[v + 1]; ++e) {
        int32_t u = q->colidx[e];
        double m_vu = q->val ? q->val[e] : 1.0 / (double)q->outdeg[u];
        s += m_vu * ((u >= lo && u < hi) ? buf[u] : r[u]);
    }
    double t = q->tele ? q->tele[v] : 1.0 / (double)q->n;
    return (1.0 - q->d) * t + q->d * (s + D / (double)q->n);
}

/* One row of the PageRank map, reading r. */
static double pr_row(const pr_problem* q, const double* r, double D, int32_t v)
{
    double s = 0.0;
    for (int32_t e = q->rowptr[v]; e < q->rowptr[v + 1]; ++e) {
        int32_t u = q->colidx[e];
        double m_vu = q->val ? q->val[e] : 1.0 / (double)q->outdeg[u];
        s += m_vu * r[u];
    }
    double t = q->tele ? q->tele[v] : 1.0 / (double)q->n;
    return (1.0 - q->d) * t + q->d * (s + D / (double)q->n);
}

/* N: the mass held by vertices that have out-edges. */
static double linked_mass(const pr_problem* q, const double* r)
{
    double N = 0.0;
    for (int32_t u = 0; u < q->n; ++u)
        if (q->outdeg[u] != 0) N += r[u];
    return N;
}

static double teleport_total(int32_t n, const double* tele)
{
    if (!tele) return 1.0;
    double T = 0.0;
    for (int32_t v = 0; v < n; ++v) T += tele[v];
    return T;
}

/*
 * Synchronous PageRank: r <- F(r) into a second array each sweep.
 * r holds r^0 on entry and the last iterate on exit. res_hist (nullable, length
 * max_iters) receives each sweep's L1 change. Returns 0 when converged, 1 when
 * max_iters sweeps ran without reaching tol, -1 on allocation failure.
 */
int orc_pagerank_sync(int32_t n, const int32_t* rowptr, const int32_t* colidx, const double* val,
                      double d, const double* tele, double tol, int32_t max_iters,
                      double* r, int32_t* iters, double* res_hist)
{
    int32_t* outdeg = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    double* nxt = (double*)malloc((size_t)n * sizeof(double));
    if (!outdeg || !nxt) { free(outdeg); free(nxt); return -1; }
    orc_out_degree(n, rowptr, colidx, outdeg);
    pr_problem q = {n, rowptr, colidx, val, outdeg, d, tele, teleport_total(n, tele)};
    int rc = 1;
    int32_t it = 0;
    while (it < max_iters) {
        double D = q.T - linked_mass(&q, r);
        double res = 0.0;
        for (int32_t v = 0; v < n; ++v) {
            nxt[v] = pr_row(&q, r, D, v);
            res += fabs(nxt[v] - r[v]);
        }
        memcpy(r, nxt, (size_t)n * sizeof(double));
        if (res_hist) res_hist[it] = res;
        ++it;
        if (res <= tol) { rc = 0; break; }
    }
    *iters = it;
    free(outdeg); free(nxt);
    return rc;
}

/*
 * orc_pagerank_sync with its rows computed by `threads` OpenMP threads. Each
 * row of a synchronous sweep reads only the previous iterate, so the rows are
 * independent and every iterate equals the serial one; only the order in
 * which the sums N and the residual are added differs (a few ulps). For the
 * fixed point of large graphs, where the serial loop takes minutes.
 */
int orc_pagerank_sync_par(int32_t n, const int32_t* rowptr, const int32_t* colidx, const double* val,
                          double d, const double* tele, double tol, int32_t max_iters, int32_t threads,
                          double* r, int32_t* iters)
{
    int32_t* outdeg = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    double* nxt = (double*)malloc((size_t)n * sizeof(double));
    if (!outdeg || !nxt) { free(outdeg); free(nxt); return -1; }
    orc_out_degree(n, rowptr, colidx, outdeg);
    pr_problem q = {n, rowptr, colidx, val, outdeg, d, tele, teleport_total(n, tele)};
    int rc = 1;
    int32_t it = 0;
    while (it < max_iters) {
        double N = 0.0, res = 0.0;
#pragma omp parallel for num_threads(threads) reduction(+ : N) schedule(static)
        for (int32_t u = 0; u < n; ++u)
            if (outdeg[u] != 0) N += r[u];
        const double D = q.T - N;
#pragma omp parallel for num_threads(threads) reduction(+ : res) schedule(dynamic, 4096)
        for (int32_t v = 0; v < n; ++v) {
            nxt[v] = pr_row(&q, r, D, v);
            res += fabs(nxt[v] - r[v]);
        }
        memcpy(r, nxt, (size_t)n * sizeof(double));
        ++it;
        if (res <= tol) { rc = 0; break; }
    }
    *iters = it;
    free(outdeg); free(nxt);
    return rc;
}

/*
 * One synchronous PageRank sweep of rows [lo, hi) only (the rows one GPU owns
 * when the rows are split across GPUs): r_out[v] = pr_row(r_in) for v in the
 * range, with the dangling mass T - N taken from the caller (N: sum of r_in
 * over vertices with out-edges, summed over every range by the caller).
 * sums[0] = sum |r_out - r_in| and sums[1] = sum of r_out over the range's
 * vertices with out-edges. Returns -1 on allocation failure.
 */
int orc_pagerank_sweep_rows(int32_t n, const int32_t* rowptr, const int32_t* colidx, const double* val, double d,
                            const double* tele, double T, double N, int32_t lo, int32_t hi, const double* r_in,
                            double* r_out, double* sums)
{
    int32_t* outdeg = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    if (!outdeg) return -1;
    orc_out_degree(n, rowptr, colidx, outdeg);
    pr_problem q = {n, rowptr, colidx, val, outdeg, d, tele, T};
    double res = 0.0, linked = 0.0;
    for (int32_t v = lo; v < hi; ++v) {
        r_out[v] = pr_row(&q, r_in, T - N, v);
        res += fabs(r_out[v] - r_in[v]);
        if (outdeg[v] != 0) linked += r_out[v];
    }
    sums[0] = res;
    sums[1] = linked;
    free(outdeg);
    return 0;
}

int orc_pagerank_delayed_view(int32_t n, const int32_t* rowptr, const int32_t* colidx, const double* val,
                              double d, const double* tele, double tol, int32_t max_iters,
                              int32_t P, int32_t delta, int32_t local_read, double* r, int32_t* iters,
                              double* res_hist);

/*
 * Delayed-asynchronous PageRank with P round-robin workers and buffer delta
 * (delta = 0: asynchronous). Same arguments and return codes as the sync form.
 */
int orc_pagerank_delayed(int32_t n, const int32_t* rowptr, const int32_t* colidx, const double* val,
                         double d, const double* tele, double tol, int32_t max_iters,
                         int32_t P, int32_t delta, double* r, int32_t* iters, double* res_hist)
{
    return orc_pagerank_delayed_view(n, rowptr, colidx, val, d, tele, tol, max_iters, P, delta, 0, r, iters,
                                     res_hist);
}

/*
 * As orc_pagerank_delayed; with local_read != 0 a worker reads its own
 * unflushed values from its buffer (the "local read" form, Sec. III-C) instead
 * of the global array. Everything else (the dangling term, other workers'
 * values) still comes from the global array.
 */
int orc_pagerank_delayed_view(int32_t n, const int32_t* rowptr, const int32_t* colidx, const double* val,
                              double d, const double* tele, double tol, int32_t max_iters,
                              int32_t P, int32_t delta, int32_t local_read, double* r, int32_t* iters,
                              double* res_hist)
{
    if (P < 1 || delta < 0) return -2;
    if (P > n) P = n;
    int32_t* outdeg = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    int32_t* start = (int32_t*)malloc(((size_t)P + 1) * sizeof(int32_t));
    int32_t* pos = (int32_t*)malloc((size_t)P * sizeof(int32_t));
    int32_t* first = (int32_t*)malloc((size_t)P * sizeof(int32_t)); /* first unflushed row */
    int32_t* cnt = (int32_t*)malloc((size_t)P * sizeof(int32_t));
    double* tick_val = (double*)malloc((size_t)P * sizeof(double));
    /* worker p's delay buffer: its unflushed values, rows first[p] .. first[p]+cnt[p]-1 */
    double* buf = (double*)malloc((size_t)n * sizeof(double));
    if (!outdeg || !start || !pos || !first || !cnt || !tick_val || !buf) {
        free(outdeg); free(start); free(pos); free(first); free(cnt); free(tick_val); free(buf);
        return -1;
    }
    orc_out_degree(n, rowptr, colidx, outdeg);
    orc_partition(n, rowptr, P, start);
    pr_problem q = {n, rowptr, colidx, val, outdeg, d, tele, teleport_total(n, tele)};
    int rc = 1;
    int32_t it = 0;
    while (it < max_iters) {
        double N = linked_mass(&q, r); /* follows every write to the global array below */
        double res = 0.0;
        int32_t left = 0;
        for (int32_t p = 0; p < P; ++p) {
            pos[p] = start[p]; first[p] = start[p]; cnt[p] = 0;
            left += start[p + 1] - start[p];
        }
        while (left > 0) {
            /* compute: every worker with rows left does one row from the global array */
            for (int32_t p = 0; p < P; ++p) {
                if (pos[p] >= start[p + 1]) continue;
                int32_t v = pos[p];
                double x = local_read ? pr_row_view(&q, r, buf, first[p], first[p] + cnt[p], q.T - N, v)
                                      : pr_row(&q, r, q.T - N, v);
                res += fabs(x - r[v]);
                tick_val[p] = x;
            }
            /* end of tick: writes (delta = 0) or buffer appends and flushes */
            for (int32_t p = 0; p < P; ++p) {
                if (pos[p] >= start[p + 1]) continue;
                int32_t v = pos[p]++;
                --left;
                if (delta == 0) {
                    if (outdeg[v]) N += tick_val[p] - r[v];
                    r[v] = tick_val[p];
                    first[p] = v + 1;
                    continue;
                }
                buf[v] = tick_val[p];
                cnt[p] += 1;
                if (cnt[p] == delta || pos[p] == start[p + 1]) {
                    for (int32_t k = 0; k < cnt[p]; ++k) {
                        int32_t x = first[p] + k;
                        if (outdeg[x]) N += buf[x] - r[x];
                        r[x] = buf[x];
                    }
                    first[p] += cnt[p];
                    cnt[p] = 0;
                }
            }
        }
        if (res_hist) res_hist[it] = res;
        ++it;
        if (res <= tol) { rc = 0; break; }
    }
    *iters = it;
    free(outdeg); free(start); free(pos); free(first); free(cnt); free(tick_val); free(buf);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Bellman-Ford SSSP                                                          */
/* ------------------------------------------------------------------------- */

/* Bellman-Ford row; in-neighbours in [lo, hi) are read from buf (local reads, Sec. III-C). */
static uint32_t bf_row_view(const int32_t* rowptr, const int32_t* colidx, const uint32_t* w,
                            const uint32_t* dist, const uint32_t* buf, int32_t lo, int32_t hi, int32_t v)
{
    uint32_t best = dist[v];
    for (int32_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
        int32_t u = colidx[e];
        uint32_t du = (u >= lo && u < hi) ? buf[u] : dist[u];
        if (du == ORC_INF) continue;
        uint64_t cand = (uint64_t)du + w[e];
        if (cand >= ORC_INF) cand = ORC_INF - 1u;
        if (cand < best) best = (uint32_t)cand;
    }
    return best;
}

static uint32_t bf_row(const int32_t* rowptr, const int32_t* colidx, const uint32_t* w,
                       const uint32_t* dist, int32_t v)
{
    uint32_t best = dist[v];
    for (int32_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
        uint32_t du = dist[colidx[e]];
        if (du == ORC_INF) continue;
        uint64_t cand = (uint64_t)du + w[e];
        if (cand >= ORC_INF) cand = ORC_INF - 1u; /* a finite path stays finite (never hit on test sizes) */
        if (cand < best) best = (uint32_t)cand;
    }
    return best;
}

/*
 * Synchronous Bellman-Ford from src. dist receives the distances (INF for
 * unreachable). updates (nullable, length max_iters) receives the number of
 * vertices whose value decreased in each sweep. Returns 0 when a sweep changed
 * nothing within max_iters sweeps, else 1.
 */
int orc_sssp_sync(int32_t n, const int32_t* rowptr, const int32_t* colidx, const uint32_t* w,
                  uint32_t src, int32_t max_iters, uint32_t* dist, int32_t* iters, int64_t* updates)
{
    uint32_t* nxt = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
    if (!nxt) return -1;
    for (int32_t v = 0; v < n; ++v) dist[v] = ORC_INF;
    dist[src] = 0;
    int rc = 1;
    int32_t it = 0;
    while (it < max_iters) {
        int64_t changed = 0;
        for (int32_t v = 0; v < n; ++v) {
            nxt[v] = bf_row(rowptr, colidx, w, dist, v);
            if (nxt[v] < dist[v]) ++changed;
        }
        memcpy(dist, nxt, (size_t)n * sizeof(uint32_t));
        if (updates) updates[it] = changed;
        ++it;
        if (changed == 0) { rc = 0; break; }
    }
    *iters = it;
    free(nxt);
    return rc;
}

/* Delayed-asynchronous Bellman-Ford (delta = 0: asynchronous), P round-robin workers. */
/*
 * One synchronous Bellman-Ford sweep of rows [lo, hi) only:
 * d_out[v] = min(d_in[v], min over in-edges with d_in[u] finite of d_in[u] + w)
 * for v in the range. Returns the number of rows lowered.
 */
int64_t orc_sssp_sweep_rows(int32_t n, const int32_t* rowptr, const int32_t* colidx, const uint32_t* w, int32_t lo,
                            int32_t hi, const uint32_t* d_in, uint32_t* d_out)
{
    (void)n;
    int64_t changed = 0;
    for (int32_t v = lo; v < hi; ++v) {
        uint32_t best = d_in[v];
        for (int32_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
            const uint32_t du = d_in[colidx[e]];
            if (du != ORC_INF && du + w[e] < best) best = du + w[e];
        }
        d_out[v] = best;
        if (best < d_in[v]) ++changed;
    }
    return changed;
}

int orc_sssp_delayed_view(int32_t n, const int32_t* rowptr, const int32_t* colidx, const uint32_t* w,
                          uint32_t src, int32_t max_iters, int32_t P, int32_t delta, int32_t local_read,
                          uint32_t* dist, int32_t* iters, int64_t* updates);

int orc_sssp_delayed(int32_t n, const int32_t* rowptr, const int32_t* colidx, const uint32_t* w,
                     uint32_t src, int32_t max_iters, int32_t P, int32_t delta,
                     uint32_t* dist, int32_t* iters, int64_t* updates)
{
    return orc_sssp_delayed_view(n, rowptr, colidx, w, src, max_iters, P, delta, 0, dist, iters, updates);
}

/* As orc_sssp_delayed; local_read != 0: a worker reads its own unflushed values (Sec. III-C). */
int orc_sssp_delayed_view(int32_t n, const int32_t* rowptr, const int32_t* colidx, const uint32_t* w,
                          uint32_t src, int32_t max_iters, int32_t P, int32_t delta, int32_t local_read,
                          uint32_t* dist, int32_t* iters, int64_t* updates)
{
    if (P < 1 || delta < 0) return -2;
    if (P > n) P = n;
    int32_t* start = (int32_t*)malloc(((size_t)P + 1) * sizeof(int32_t));
    int32_t* pos = (int32_t*)malloc((size_t)P * sizeof(int32_t));
    int32_t* first = (int32_t*)malloc((size_t)P * sizeof(int32_t));
    int32_t* cnt = (int32_t*)malloc((size_t)P * sizeof(int32_t));
    uint32_t* tick_val = (uint32_t*)malloc((size_t)P * sizeof(uint32_t));
    uint32_t* buf = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
    if (!start || !pos || !first || !cnt || !tick_val || !buf) {
        free(start); free(pos); free(first); free(cnt); free(tick_val); free(buf);
        return -1;
    }
    orc_partition(n, rowptr, P, start);
    for (int32_t v = 0; v < n; ++v) dist[v] = ORC_INF;
    dist[src] = 0;
    int rc = 1;
    int32_t it = 0;
    while (it < max_iters) {
        int64_t changed = 0;
        int32_t left = 0;
        for (int32_t p = 0; p < P; ++p) {
            pos[p] = start[p]; first[p] = start[p]; cnt[p] = 0;
            left += start[p + 1] - start[p];
        }
        while (left > 0) {
            for (int32_t p = 0; p < P; ++p) {
                if (pos[p] >= start[p + 1]) continue;
                int32_t v = pos[p];
                uint32_t x = local_read ? bf_row_view(rowptr, colidx, w, dist, buf, first[p], first[p] + cnt[p], v)
                                        : bf_row(rowptr, colidx, w, dist, v);
                if (x < dist[v]) ++changed;
                tick_val[p] = x;
            }
            for (int32_t p = 0; p < P; ++p) {
                if (pos[p] >= start[p + 1]) continue;
                int32_t v = pos[p]++;
                --left;
                if (delta == 0) {
                    dist[v] = tick_val[p];
                    first[p] = v + 1;
                    continue;
                }
                buf[v] = tick_val[p];
                cnt[p] += 1;
                if (cnt[p] == delta || pos[p] == start[p + 1]) {
                    for (int32_t k = 0; k < cnt[p]; ++k) dist[first[p] + k] = buf[first[p] + k];
                    first[p] += cnt[p];
                    cnt[p] = 0;
                }
            }
        }
        if (updates) updates[it] = changed;
        ++it;
        if (changed == 0) { rc = 0; break; }
    }
    *iters = it;
    free(start); free(pos); free(first); free(cnt); free(tick_val); free(buf);
    return rc;
}

/* Dijkstra's algorithm with a binary heap over the out-edges (built here from the in-CSR). */
int orc_dijkstra(int32_t n, const int32_t* rowptr, const int32_t* colidx, const uint32_t* w,
                 uint32_t src, uint32_t* dist)
{
    int64_t m = rowptr[n];
    int64_t* optr = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    int32_t* odst = (int32_t*)malloc((size_t)(m ? m : 1) * sizeof(int32_t));
    uint32_t* ow = (uint32_t*)malloc((size_t)(m ? m : 1) * sizeof(uint32_t));
    int64_t* fill = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    /* heap of (dist, vertex) with lazy deletion: at most m + 1 entries */
    uint64_t* heap = (uint64_t*)malloc((size_t)(m + 1) * sizeof(uint64_t));
    if (!optr || !odst || !ow || !fill || !heap) {
        free(optr); free(odst); free(ow); free(fill); free(heap);
        return -1;
    }
    for (int64_t e = 0; e < m; ++e) optr[colidx[e] + 1] += 1;
    for (int32_t u = 0; u < n; ++u) optr[u + 1] += optr[u];
    for (int32_t u = 0; u < n; ++u) fill[u] = optr[u];
    for (int32_t v = 0; v < n; ++v)
        for (int32_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
            int32_t u = colidx[e];
            odst[fill[u]] = v;
            ow[fill[u]] = w[e];
            fill[u] += 1;
        }
    for (int32_t v = 0; v < n; ++v) dist[v] = ORC_INF;
    dist[src] = 0;
    int64_t hs = 0;
    heap[hs++] = ((uint64_t)0 << 32) | src;
    while (hs > 0) {
        uint64_t top = heap[0];
        heap[0] = heap[--hs];
        for (int64_t i = 0;;) { /* sift down */
            int64_t l = 2 * i + 1, r = l + 1, s = i;
            if (l < hs && heap[l] < heap[s]) s = l;
            if (r < hs && heap[r] < heap[s]) s = r;
            if (s == i) break;
            uint64_t t = heap[i]; heap[i] = heap[s]; heap[s] = t;
            i = s;
        }
        uint32_t du = (uint32_t)(top >> 32), u = (uint32_t)(top & 0xFFFFFFFFu);
        if (du != dist[u]) continue; /* stale entry */
        for (int64_t k = optr[u]; k < optr[u + 1]; ++k) {
            uint64_t cand = (uint64_t)du + ow[k];
            int32_t v = odst[k];
            if (cand < dist[v]) {
                dist[v] = (uint32_t)cand;
                int64_t i = hs++;
                heap[i] = (cand << 32) | (uint32_t)v;
                while (i > 0) { /* sift up */
                    int64_t pnt = (i - 1) / 2;
                    if (heap[pnt] <= heap[i]) break;
                    uint64_t t = heap[i]; heap[i] = heap[pnt]; heap[pnt] = t;
                    i = pnt;
                }
            }
        }
    }
    free(optr); free(odst); free(ow); free(fill); free(heap);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Weighted PageRank: normalisation, adjoint, gradients                       */
/* ------------------------------------------------------------------------- */

/* s[u] = sum of w over the out-edges of u; val[e] = w[e] / s[colidx[e]] (column-stochastic M). */
void orc_normalize(int32_t n, const int32_t* rowptr, const int32_t* colidx, const double* w,
                   double* val, double* s)
{
    for (int32_t u = 0; u < n; ++u) s[u] = 0.0;
    for (int32_t v = 0; v < n; ++v)
        for (int32_t e = rowptr[v]; e < rowptr[v + 1]; ++e) s[colidx[e]] += w[e];
    for (int32_t v = 0; v < n; ++v)
        for (int32_t e = rowptr[v]; e < rowptr[v + 1]; ++e) val[e] = w[e] / s[colidx[e]];
}

/*
 * Adjoint of r = d (M r + (1/n) 1 g^T r) + (1-d) t for a loss with dL/dr = c:
 *   lambda = c + d M^T lambda + d g (sum_v lambda_v) / n,
 * solved by Jacobi sweeps in fp64 until the L1 change is <= tol * ||c||_1.
 * (M^T lambda)_u = sum over edges u -> v of M_vu lambda_v, formed by scattering
 * along the in-CSR. Returns 0 when converged, 1 otherwise.
 */
int orc_pagerank_adjoint(int32_t n, const int32_t* rowptr, const int32_t* colidx, const double* val,
                         double d, const double* c, double tol, int32_t max_iters,
                         double* lambda, int32_t* iters)
{
    int32_t* outdeg = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    double* mt = (double*)malloc((size_t)n * sizeof(double));
    double* nxt = (double*)malloc((size_t)n * sizeof(double));
    if (!outdeg || !mt || !nxt) { free(outdeg); free(mt); free(nxt); return -1; }
    orc_out_degree(n, rowptr, colidx, outdeg);
    double cnorm = 0.0;
    for (int32_t v = 0; v < n; ++v) { lambda[v] = c[v]; cnorm += fabs(c[v]); }
    int rc = 1;
    int32_t it = 0;
    while (it < max_iters) {
        double S = 0.0;
        for (int32_t v = 0; v < n; ++v) { S += lambda[v]; mt[v] = 0.0; }
        for (int32_t v = 0; v < n; ++v)
            for (int32_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
                int32_t u = colidx[e];
                double m_vu = val ? val[e] : 1.0 / (double)outdeg[u];
                mt[u] += m_vu * lambda[v];
            }
        double res = 0.0;
        for (int32_t u = 0; u < n; ++u) {
            nxt[u] = c[u] + d * mt[u] + (outdeg[u] == 0 ? d * S / (double)n : 0.0);
            res += fabs(nxt[u] - lambda[u]);
        }
        memcpy(lambda, nxt, (size_t)n * sizeof(double));
        ++it;
        if (res <= tol * cnorm) { rc = 0; break; }
    }
    *iters = it;
    free(outdeg); free(mt); free(nxt);
    return rc;
}

/*
 * Gradients of L through r (weighted PageRank with M_vu = w_uv / s_u):
 *   dL/dw_uv = d r_u (lambda_v - (M^T lambda)_u) / s_u   (per in-edge e = (u -> v)),
 *   dL/dt_v  = (1 - d) lambda_v.
 */
void orc_pagerank_grads(int32_t n, const int32_t* rowptr, const int32_t* colidx, const double* val,
                        const double* s, double d, const double* r, const double* lambda,
                        double* grad_w, double* grad_t)
{
    double* mt = (double*)calloc((size_t)n, sizeof(double));
    for (int32_t v = 0; v < n; ++v)
        for (int32_t e = rowptr[v]; e < rowptr[v + 1]; ++e) mt[colidx[e]] += val[e] * lambda[v];
    for (int32_t v = 0; v < n; ++v)
        for (int32_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
            int32_t u = colidx[e];
            grad_w[e] = d * r[u] * (lambda[v] - mt[u]) / s[u];
        }
    for (int32_t v = 0; v < n; ++v) grad_t[v] = (1.0 - d) * lambda[v];
    free(mt);
}

/* ------------------------------------------------------------------------- */
/* The paper's CPU scheme with OpenMP threads (timed CPU baseline)            */
/* ------------------------------------------------------------------------- */

static inline float ld_f(const float* p) { float x; __atomic_load(p, &x, __ATOMIC_RELAXED); return x; }
static inline void st_f(float* p, float x) { __atomic_store(p, &x, __ATOMIC_RELAXED); }
static inline double ld_d(const double* p) { double x; __atomic_load(p, &x, __ATOMIC_RELAXED); return x; }
static inline void st_d(double* p, double x) { __atomic_store(p, &x, __ATOMIC_RELAXED); }
static inline uint32_t ld_u(const uint32_t* p) { return __atomic_load_n(p, __ATOMIC_RELAXED); }
static inline void st_u(uint32_t* p, uint32_t x) { __atomic_store_n(p, x, __ATOMIC_RELAXED); }

/*
 * PageRank with T OpenMP threads, the paper's scheme: static blocks balanced by
 * in-neighbour count, FP32 scores, one barrier per iteration. variant 0 = sync
 * (two arrays), 1 = async (in place), 2 = delayed with buffer delta. The
 * dangling term uses the same D = 1 - N as the serial forms: sync takes N from
 * the previous iterate; async and delayed publish each thread's change of N in
 * a padded per-thread slot when they write to the global array, and re-read the
 * sum of the slots every 64 rows (async) or at each flush (delayed). r receives
 * the result; seconds the wall time of the iterations (setup excluded).
 */
int orc_pagerank_threads(int32_t variant, int32_t n, const int32_t* rowptr, const int32_t* colidx,
                         float d, double tol, int32_t max_iters, int32_t T, int32_t delta,
                         float* r, int32_t* iters, double* seconds)
{
    if (T < 1) return -2;
    if (T > n) T = n;
    if (variant == 2 && delta <= 0) variant = 1;
    const int32_t PAD = 8; /* doubles per slot: one 64-byte line */
    int32_t* outdeg = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    float* inv = (float*)malloc((size_t)n * sizeof(float));
    float* a = (float*)malloc((size_t)n * sizeof(float));
    float* b = (float*)malloc((size_t)n * sizeof(float));
    int32_t* start = (int32_t*)malloc(((size_t)T + 1) * sizeof(int32_t));
    double* part = (double*)calloc(2 * (size_t)T, sizeof(double));
    double* slot = (double*)calloc((size_t)T * PAD, sizeof(double));
    if (!outdeg || !inv || !a || !b || !start || !part || !slot) {
        free(outdeg); free(inv); free(a); free(b); free(start); free(part); free(slot);
        return -1;
    }
    orc_out_degree(n, rowptr, colidx, outdeg);
    orc_partition(n, rowptr, T, start);
    for (int32_t u = 0; u < n; ++u) { inv[u] = outdeg[u] ? 1.0f / (float)outdeg[u] : 0.0f; a[u] = 1.0f / (float)n; }
    double N0 = 0.0;
    for (int32_t u = 0; u < n; ++u) if (outdeg[u]) N0 += a[u];
    int32_t done_iters = 0, converged = 0;
    double t0 = omp_get_wtime();
#pragma omp parallel num_threads(T)
    {
        int32_t p = omp_get_thread_num();
        int32_t lo = start[p], hi = start[p + 1];
        float* buf = (variant == 2) ? (float*)malloc((size_t)(delta > 0 ? delta : 1) * sizeof(float)) : NULL;
        float* cur = a;
        float* nxt = b;
        double Nstart = N0;
        for (int32_t it = 0; it < max_iters; ++it) {
            double res = 0.0, nmass = 0.0, dN = 0.0;
            double N = Nstart;
            float* dst = (variant == 0) ? nxt : cur;
            int32_t bstart = lo, bcnt = 0;
            for (int32_t v = lo; v < hi; ++v) {
                if (variant == 1 && ((v - lo) & 63) == 0) {
                    N = Nstart;
                    for (int32_t q = 0; q < T; ++q) N += ld_d(&slot[q * PAD]);
                }
                float base = (1.0f - d) / (float)n + d * (float)((1.0 - N) / (double)n);
                float s = 0.0f;
                for (int32_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
                    int32_t u = colidx[e];
                    s += ld_f(&cur[u]) * inv[u];
                }
                float x = base + d * s;
                float old = ld_f(&cur[v]);
                res += fabs((double)x - (double)old);
                if (outdeg[v]) nmass += x;
                if (variant == 2) {
                    buf[bcnt++] = x;
                    if (bcnt == delta) {
                        for (int32_t k = 0; k < bcnt; ++k) {
                            if (outdeg[bstart + k]) dN += (double)buf[k] - (double)ld_f(&cur[bstart + k]);
                            st_f(&cur[bstart + k], buf[k]);
                        }
                        st_d(&slot[p * PAD], dN);
                        N = Nstart;
                        for (int32_t q = 0; q < T; ++q) N += ld_d(&slot[q * PAD]);
                        bstart += bcnt; bcnt = 0;
                    }
                } else {
                    if (variant == 1 && outdeg[v]) {
                        dN += (double)x - (double)old;
                        st_d(&slot[p * PAD], dN);
                    }
                    st_f(&dst[v], x);
                }
            }
            if (variant == 2)
                for (int32_t k = 0; k < bcnt; ++k) st_f(&cur[bstart + k], buf[k]);
            part[2 * p] = res; part[2 * p + 1] = nmass;
#pragma omp barrier
            double tot = 0.0, nm = 0.0;
            for (int32_t q = 0; q < T; ++q) { tot += part[2 * q]; nm += part[2 * q + 1]; }
            Nstart = nm;
            if (variant == 0) { float* t = cur; cur = nxt; nxt = t; }
#pragma omp barrier
            slot[p * PAD] = 0.0;
#pragma omp barrier
            if (tot <= tol) {
                if (p == 0) { done_iters = it + 1; converged = 1; }
                break;
            }
            if (p == 0) done_iters = it + 1;
        }
        if (p == 0) memcpy(r, cur, (size_t)n * sizeof(float));
        free(buf);
    }
    *seconds = omp_get_wtime() - t0;
    *iters = done_iters;
    free(outdeg); free(inv); free(a); free(b); free(start); free(part); free(slot);
    return converged ? 0 : 1;
}

/* Bellman-Ford with T OpenMP threads, the paper's scheme (same variants as above). */
int orc_sssp_threads(int32_t variant, int32_t n, const int32_t* rowptr, const int32_t* colidx,
                     const uint32_t* w, uint32_t src, int32_t max_iters, int32_t T, int32_t delta,
                     uint32_t* dist, int32_t* iters, double* seconds)
{
    if (T < 1) return -2;
    if (T > n) T = n;
    if (variant == 2 && delta <= 0) variant = 1;
    uint32_t* a = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
    uint32_t* b = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
    int32_t* start = (int32_t*)malloc(((size_t)T + 1) * sizeof(int32_t));
    int64_t* part = (int64_t*)calloc((size_t)T, sizeof(int64_t));
    if (!a || !b || !start || !part) { free(a); free(b); free(start); free(part); return -1; }
    orc_partition(n, rowptr, T, start);
    for (int32_t v = 0; v < n; ++v) a[v] = b[v] = ORC_INF;
    a[src] = b[src] = 0;
    int32_t done_iters = 0, converged = 0;
    double t0 = omp_get_wtime();
#pragma omp parallel num_threads(T)
    {
        int32_t p = omp_get_thread_num();
        int32_t lo = start[p], hi = start[p + 1];
        uint32_t* buf = (variant == 2) ? (uint32_t*)malloc((size_t)(delta > 0 ? delta : 1) * sizeof(uint32_t)) : NULL;
        uint32_t* cur = a;
        uint32_t* nxt = b;
        for (int32_t it = 0; it < max_iters; ++it) {
            int64_t changed = 0;
            uint32_t* dst = (variant == 0) ? nxt : cur;
            int32_t bstart = lo, bcnt = 0;
            for (int32_t v = lo; v < hi; ++v) {
                uint32_t old = ld_u(&cur[v]);
                uint32_t best = old;
                for (int32_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
                    uint32_t du = ld_u(&cur[colidx[e]]);
                    if (du == ORC_INF) continue;
                    uint32_t cand = du + w[e];
                    if (cand < best) best = cand;
                }
                if (best < old) ++changed;
                if (variant == 2) {
                    buf[bcnt++] = best;
                    if (bcnt == delta) {
                        for (int32_t k = 0; k < bcnt; ++k) st_u(&cur[bstart + k], buf[k]);
                        bstart += bcnt; bcnt = 0;
                    }
                } else {
                    st_u(&dst[v], best);
                }
            }
            if (variant == 2)
                for (int32_t k = 0; k < bcnt; ++k) st_u(&cur[bstart + k], buf[k]);
            part[p] = changed;
#pragma omp barrier
            int64_t tot = 0;
            for (int32_t q = 0; q < T; ++q) tot += part[q];
            if (variant == 0) { uint32_t* t = cur; cur = nxt; nxt = t; }
#pragma omp barrier
            if (tot == 0) {
                if (p == 0) { done_iters = it + 1; converged = 1; }
                break;
            }
            if (p == 0) done_iters = it + 1;
        }
        if (p == 0) memcpy(dist, cur, (size_t)n * sizeof(uint32_t));
        free(buf);
    }
    *seconds = omp_get_wtime() - t0;
    *iters = done_iters;
    free(a); free(b); free(start); free(part);
    return converged ? 0 : 1;
}
