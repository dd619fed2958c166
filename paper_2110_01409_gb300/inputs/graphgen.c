/*
 * Seeded synthetic graph generators (host C, OpenMP).
 *
 * This file is the one source of inputs shared by the CPU oracle and the CUDA
 * path. It holds no PageRank or Bellman-Ford arithmetic: it only draws edges,
 * removes self-loops and duplicates, and lays the result out as an in-edge CSR
 * (row v lists the sources u of the edges u->v, ascending), which is the layout
 * a pull-style sweep reads (Sec. III-A: each vertex value is computed by one
 * worker from its in-neighbours).
 *
 * Randomness is counter-based: every draw is SplitMix64 (Steele, Lea and Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014) applied to a
 * key built from (seed, edge index, level), so the output does not depend on
 * the thread count or the machine.
 *
 * Graph families (stand-ins for the GAP graphs of Table II, which are not
 * available here):
 *   - RMAT (Chakrabarti, Zhan, Faloutsos 2004): stands in for Kron;
 *   - Erdos-Renyi G(n, m) with uniform endpoints: stands in for Urand;
 *   - banded: 15 edges to targets within +-1024 of the source (wrapping modulo
 *     n) plus 1 uniform edge; stands in for Web's diagonal clustering
 *     (Sec. IV-C, Fig. 5).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <omp.h>

static inline uint64_t sm64(uint64_t z)
{
    z += 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* One counter-based draw for (seed, a, b). */
static inline uint64_t gg_hash3(uint64_t seed, uint64_t a, uint64_t b)
{
    return sm64(sm64(sm64(seed) ^ a) ^ (b * 0xd1342543de82ef95ULL + 1));
}

/* Uniform double in [0, 1) from the top 53 bits. */
static inline double u01(uint64_t h) { return (double)(h >> 11) * (1.0 / 9007199254740992.0); }

/* Uniform integer in [0, n) by the multiply-high of a 32-bit draw (n < 2^32). */
static inline uint32_t below(uint64_t h, uint32_t n) { return (uint32_t)(((h >> 32) * (uint64_t)n) >> 32); }

/* ------------------------------------------------------------------------- */
/* Edge list -> deduplicated in-edge CSR                                      */
/* ------------------------------------------------------------------------- */

typedef struct {
    int32_t n;
    int64_t m;
    int32_t* rowptr; /* n+1 */
    int32_t* colidx; /* m   */
} gg_graph;

static int cmp_i32(const void* a, const void* b)
{
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

static void sort_row(int32_t* p, int64_t len)
{
    if (len < 32) {
        for (int64_t i = 1; i < len; ++i) {
            int32_t v = p[i];
            int64_t j = i - 1;
            while (j >= 0 && p[j] > v) { p[j + 1] = p[j]; --j; }
            p[j + 1] = v;
        }
    } else {
        qsort(p, (size_t)len, sizeof(int32_t), cmp_i32);
    }
}

/* Builds the in-edge CSR of the edge list (src[e] -> dst[e]) with self-loops and
 * duplicate pairs removed and each row sorted ascending. Frees nothing it was
 * given. Returns 0, or -1 when memory runs out or the result has >= 2^31 edges. */
static int build_in_csr(int32_t n, int64_t E, const uint32_t* src, const uint32_t* dst, gg_graph* g)
{
    int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    if (!cnt) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < E; ++e) {
        if (src[e] != dst[e]) {
#pragma omp atomic
            cnt[dst[e] + 1]++;
        }
    }
    for (int32_t v = 0; v < n; ++v) cnt[v + 1] += cnt[v];
    int64_t total = cnt[n];
    int32_t* col = (int32_t*)malloc((size_t)(total ? total : 1) * sizeof(int32_t));
    int64_t* cur = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    if (!col || !cur) { free(cnt); free(col); free(cur); return -1; }
    memcpy(cur, cnt, (size_t)n * sizeof(int64_t));
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < E; ++e) {
        if (src[e] != dst[e]) {
            int64_t pos;
#pragma omp atomic capture
            pos = cur[dst[e]]++;
            col[pos] = (int32_t)src[e];
        }
    }
    free(cur);
    /* sort + dedup each row in place; keep the new length in cnt-derived array */
    int64_t* keep = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
    if (!keep) { free(cnt); free(col); return -1; }
#pragma omp parallel for schedule(dynamic, 1024)
    for (int32_t v = 0; v < n; ++v) {
        int32_t* p = col + cnt[v];
        int64_t len = cnt[v + 1] - cnt[v];
        sort_row(p, len);
        int64_t k = 0;
        for (int64_t i = 0; i < len; ++i)
            if (k == 0 || p[i] != p[k - 1]) p[k++] = p[i];
        keep[v + 1] = k;
    }
    keep[0] = 0;
    for (int32_t v = 0; v < n; ++v) keep[v + 1] += keep[v];
    int64_t m = keep[n];
    if (m >= ((int64_t)1 << 31)) { free(cnt); free(col); free(keep); return -1; }
    int32_t* rowptr = (int32_t*)malloc(((size_t)n + 1) * sizeof(int32_t));
    int32_t* colidx = (int32_t*)malloc((size_t)(m ? m : 1) * sizeof(int32_t));
    if (!rowptr || !colidx) { free(cnt); free(col); free(keep); free(rowptr); free(colidx); return -1; }
#pragma omp parallel for schedule(dynamic, 1024)
    for (int32_t v = 0; v < n; ++v) {
        memcpy(colidx + keep[v], col + cnt[v], (size_t)(keep[v + 1] - keep[v]) * sizeof(int32_t));
    }
    for (int32_t v = 0; v <= n; ++v) rowptr[v] = (int32_t)keep[v];
    free(cnt); free(col); free(keep);
    g->n = n; g->m = m; g->rowptr = rowptr; g->colidx = colidx;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Public entry points (called through ctypes)                                */
/* ------------------------------------------------------------------------- */

void gg_free(gg_graph* g)
{
    if (!g) return;
    free(g->rowptr); free(g->colidx);
    g->rowptr = NULL; g->colidx = NULL;
}

/* Copies a built graph into caller buffers and frees it. */
void gg_take(gg_graph* g, int32_t* rowptr_out, int32_t* colidx_out)
{
    memcpy(rowptr_out, g->rowptr, ((size_t)g->n + 1) * sizeof(int32_t));
    if (g->m) memcpy(colidx_out, g->colidx, (size_t)g->m * sizeof(int32_t));
    gg_free(g);
}

/* RMAT: n = 2^scale, edge_factor * n draws; each draw descends `scale` levels,
 * choosing the quadrant [a b; c d] (rows = source bit, columns = target bit). */
int gg_rmat(int32_t scale, int32_t edge_factor, double a, double b, double c, uint64_t seed, gg_graph* g)
{
    if (scale < 1 || scale > 30 || edge_factor < 1) return -2;
    int32_t n = (int32_t)1 << scale;
    int64_t E = (int64_t)n * edge_factor;
    uint32_t* src = (uint32_t*)malloc((size_t)E * sizeof(uint32_t));
    uint32_t* dst = (uint32_t*)malloc((size_t)E * sizeof(uint32_t));
    if (!src || !dst) { free(src); free(dst); return -1; }
    const double ab = a + b, abc = a + b + c;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < E; ++e) {
        uint32_t s = 0, t = 0;
        for (int32_t l = 0; l < scale; ++l) {
            double u = u01(gg_hash3(seed, (uint64_t)e, (uint64_t)l));
            uint32_t bs = 0, bt = 0;
            if (u < a) { bs = 0; bt = 0; }
            else if (u < ab) { bs = 0; bt = 1; }
            else if (u < abc) { bs = 1; bt = 0; }
            else { bs = 1; bt = 1; }
            s = (s << 1) | bs;
            t = (t << 1) | bt;
        }
        src[e] = s; dst[e] = t;
    }
    int rc = build_in_csr(n, E, src, dst, g);
    free(src); free(dst);
    return rc;
}

/* Erdos-Renyi G(n, m): m = n * avg_degree draws with independent uniform endpoints. */
int gg_erdos_renyi(int32_t n, int32_t avg_degree, uint64_t seed, gg_graph* g)
{
    if (n < 1 || avg_degree < 1) return -2;
    int64_t E = (int64_t)n * avg_degree;
    uint32_t* src = (uint32_t*)malloc((size_t)E * sizeof(uint32_t));
    uint32_t* dst = (uint32_t*)malloc((size_t)E * sizeof(uint32_t));
    if (!src || !dst) { free(src); free(dst); return -1; }
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < E; ++e) {
        src[e] = below(gg_hash3(seed, (uint64_t)e, 0), (uint32_t)n);
        dst[e] = below(gg_hash3(seed, (uint64_t)e, 1), (uint32_t)n);
    }
    int rc = build_in_csr(n, E, src, dst, g);
    free(src); free(dst);
    return rc;
}

/* Banded: for each source s, `local` edges to s + o (mod n) with o uniform in
 * [-band, band] \ {0}, plus `longrange` edges to uniform targets. */
int gg_banded(int32_t n, int32_t local, int32_t band, int32_t longrange, uint64_t seed, gg_graph* g)
{
    if (n < 1 || local < 0 || band < 1 || longrange < 0 || local + longrange < 1) return -2;
    int32_t per = local + longrange;
    int64_t E = (int64_t)n * per;
    uint32_t* src = (uint32_t*)malloc((size_t)E * sizeof(uint32_t));
    uint32_t* dst = (uint32_t*)malloc((size_t)E * sizeof(uint32_t));
    if (!src || !dst) { free(src); free(dst); return -1; }
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < n; ++s) {
        for (int32_t j = 0; j < per; ++j) {
            int64_t e = s * per + j;
            uint64_t h = gg_hash3(seed, (uint64_t)s, (uint64_t)j);
            int64_t t;
            if (j < local) {
                int64_t o = (int64_t)below(h, (uint32_t)(2 * band)) - band; /* [-band, band-1] */
                if (o >= 0) o += 1;                                          /* [-band,-1] U [1,band] */
                t = ((s + o) % n + n) % n;
            } else {
                t = below(h, (uint32_t)n);
            }
            src[e] = (uint32_t)s; dst[e] = (uint32_t)t;
        }
    }
    int rc = build_in_csr(n, E, src, dst, g);
    free(src); free(dst);
    return rc;
}

/* Graph from an explicit edge list (small test graphs). */
int gg_from_edges(int32_t n, int64_t E, const int32_t* src, const int32_t* dst, gg_graph* g)
{
    if (n < 1 || E < 0) return -2;
    for (int64_t e = 0; e < E; ++e)
        if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n) return -2;
    return build_in_csr(n, E, (const uint32_t*)src, (const uint32_t*)dst, g);
}

/* Per-in-edge integer weights in [1, 255] keyed by (seed, source, target). */
void gg_weights_u32(int32_t n, const int32_t* rowptr, const int32_t* colidx, uint64_t seed, uint32_t* w)
{
#pragma omp parallel for schedule(dynamic, 1024)
    for (int32_t v = 0; v < n; ++v)
        for (int32_t e = rowptr[v]; e < rowptr[v + 1]; ++e)
            w[e] = 1u + (uint32_t)(gg_hash3(seed, (uint64_t)colidx[e], (uint64_t)v) % 255u);
}

/* Per-in-edge float weights in (0, 1] keyed by (seed, source, target): (k+1)/2^24, k in [0, 2^24). */
void gg_weights_f32(int32_t n, const int32_t* rowptr, const int32_t* colidx, uint64_t seed, float* w)
{
#pragma omp parallel for schedule(dynamic, 1024)
    for (int32_t v = 0; v < n; ++v)
        for (int32_t e = rowptr[v]; e < rowptr[v + 1]; ++e)
            w[e] = (float)((gg_hash3(seed, (uint64_t)colidx[e], (uint64_t)v) >> 40) + 1) * (1.0f / 16777216.0f);
}

/* `count` raw 64-bit draws for (seed, stream): used for sources, seed sets and targets. */
void gg_draws(uint64_t seed, uint64_t stream, int64_t count, uint64_t* out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < count; ++i) out[i] = gg_hash3(seed, stream, (uint64_t)i);
}
