// Warp tiles shared by the warp-worker sweeps (sweep_warp.cu) and the
// warp-tile frontier Bellman-Ford (sweep_warp_frontier.cu): per-warp shared
// buffers, the staged inputs of a warp tile, its fetch (edge stream, weights,
// gathers issued ahead), the merge-path walk with a shuffle segmented scan,
// and the bounded wait on a partial another warp publishes.
#pragma once

#include <climits>
#include <cstdint>

#include "sweep_common.cuh"

namespace dag {

// Warp tile shapes: items per lane (odd: fewer bank conflicts in the walk);
// the plan picks one (dag_plan_set_warp_tile), WIPT_DEFAULT unless told.
constexpr int WIPT_DEFAULT = 7;
constexpr int WWARPS = NWARP;        // warps per CTA (block reductions and the grid barrier are per CTA)
constexpr int WMINBLOCKS = 4;        // CTAs per SM the register budget is sized for
constexpr int LIVE_EVERY = 8;        // async / delayed PageRank: a warp reads and adds to the live sum every 8
                                     // tiles (1,792 items, the CTA-tile kernels' tile), not every tile

template <int WTILE>
struct WarpShared {
    int end[WWARPS][WTILE + 1];      // tile-relative row ends (+ sentinel)
    uint32_t val[WWARPS][WTILE];     // edge terms of the tile
    uint32_t sum[WWARPS][WTILE];     // per-row reduction of the tile
    double red0[NWARP];
    double red1[NWARP];
    double res, gprev, T;
};

// Inputs of the next warp tile, loaded while the current one is walked.
template <int WIPT>
struct WStage {
    int a0, b0, NA, NB;
    int rp0;              // rowptr[a0]: the tile starts inside row a0 when b0 > rp0
    int re0;              // rowptr[a0 + lane + 1]: the end of the tile's row `lane` (lane < NA)
    uint32_t term[WIPT];  // edge terms: gathered value, combined with the edge's weight / value
    uint32_t xo;          // old value of row a0 + lane
    float dg;             // its out-degree (PageRank)
    long long gs;         // one stripe of the live global sum (async / delayed PageRank)
};

template <int MODE, int WIPT>
__device__ __forceinline__ void wfetch(WStage<WIPT>& st, const SweepParams& p, const uint32_t* xin, int t, int lane, int rmode,
                                       bool live, uint64_t pol_edge, uint64_t pol_vertex)
{
    constexpr bool BF = MODE == MODE_BF || MODE == MODE_BF8;
    st.a0 = p.tile_row[t];
    st.b0 = p.tile_nz[t];
    st.NA = p.tile_row[t + 1] - st.a0;
    st.NB = p.tile_nz[t + 1] - st.b0;
    st.rp0 = (int)ld_vertex_b32(p.rowptr + st.a0, pol_vertex);
    st.re0 = lane < st.NA ? (int)ld_vertex_b32(p.rowptr + st.a0 + lane + 1, pol_vertex) : 0;
    int col[WIPT];
    uint32_t aux[WIPT];
#pragma unroll
    for (int q = 0; q < WIPT; ++q) {
        const int j = lane + 32 * q;
        col[q] = -1;
        aux[q] = 0u;
        if (j < st.NB) {
            col[q] = (int)ld_edge_b32(p.colidx + st.b0 + j, pol_edge);
            if constexpr (MODE == MODE_BF) aux[q] = ld_edge_b32(p.w + st.b0 + j, pol_edge);
            if constexpr (MODE == MODE_BF8) aux[q] = ld_edge_u8(p.w8 + st.b0 + j, pol_edge);
            if constexpr (MODE == MODE_PRW || MODE == MODE_ADJ) aux[q] = ld_edge_b32(p.val + st.b0 + j, pol_edge);
        }
    }
#pragma unroll
    for (int q = 0; q < WIPT; ++q) {
        uint32_t term = Op<MODE>::identity();
        if (col[q] >= 0) {
            const uint32_t xv = rmode == READ_COHERENT ? ld_relaxed_keep_b32(xin + col[q], pol_vertex)
                                                       : ld_weak_keep_b32(xin + col[q], pol_vertex);
            if constexpr (BF) term = relax(xv, aux[q]);
            else if constexpr (MODE == MODE_PR) term = xv;
            else term = __float_as_uint(__uint_as_float(aux[q]) * __uint_as_float(xv));
        }
        st.term[q] = term;
    }
    st.xo = 0u;
    st.dg = 0.0f;
    if (lane < st.NA) {  // only this warp writes its rows, so a value loaded ahead is still the current one
        st.xo = ld_weak_keep_b32(xin + st.a0 + lane, pol_vertex);
        if constexpr (!BF) st.dg = __uint_as_float(ld_vertex_b32(p.degf + st.a0 + lane, pol_vertex));
    }
    if (live) st.gs = ld_relaxed_i64(&p.sync->stripe[lane * GSTRIDE]);
}

// Tile-relative row ends of a staged tile into end[0 .. NA] (sentinel INT_MAX at NA): the first 32 came
// with the tile's fetch, the rest (a tile of mostly empty rows) are loaded here.
template <int WIPT>
__device__ __forceinline__ void wstage_ends(int* end, const WStage<WIPT>& st, const SweepParams& p, int lane,
                                            uint64_t pol_vertex)
{
    if (lane < st.NA) end[lane] = st.re0 - st.b0;
    for (int i = lane + 32; i < st.NA; i += 32) end[i] = (int)ld_vertex_b32(p.rowptr + st.a0 + i + 1, pol_vertex) - st.b0;
    if (lane == 0) end[st.NA] = INT_MAX;
}

// One warp tile's merge path, warp segmented scan and per-row sums into
// sum[0 .. NA). carry: the partial of the row continuing from the previous
// tile; returns the partial of row NA (continuing into the next tile).
template <int MODE, int WIPT>
__device__ __forceinline__ uint32_t wwalk(const int* end, const uint32_t* val, uint32_t* sum, int NA, int NB,
                                          uint32_t carry, int lane)
{
    using O = Op<MODE>;
    const int L = NA + NB;
    const int k0 = min(lane * WIPT, L);
    int lo = max(0, k0 - NB), hi = min(k0, NA);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (end[mid] <= k0 - 1 - mid) lo = mid + 1;
        else hi = mid;
    }
    int i = lo, j = k0 - lo;
    const int i_start = i;
    bool emitted = false;
    uint32_t acc = lane == 0 ? carry : O::identity();
    int re = end[i];
#pragma unroll
    for (int q = 0; q < WIPT; ++q) {
        if (k0 + q < L) {
            if (re <= j) {
                sum[i] = acc;
                emitted = true;
                acc = O::identity();
                ++i;
                re = end[i];
            } else {
                acc = O::combine(acc, val[j]);
                ++j;
            }
        }
    }
    // inclusive segmented scan of (row in progress, partial) over the lanes
    const int key = i;
    uint32_t sv = acc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t ov = __shfl_up_sync(0xffffffffu, sv, o);
        const int ok = __shfl_up_sync(0xffffffffu, key, o);
        if (lane >= o && ok == key) sv = O::combine(sv, ov);
    }
    const uint32_t cin = __shfl_up_sync(0xffffffffu, sv, 1);
    const int kprev = __shfl_up_sync(0xffffffffu, key, 1);
    if (lane > 0 && emitted && kprev == i_start) sum[i_start] = O::combine(sum[i_start], cin);
    return __shfl_sync(0xffffffffu, sv, 31);
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// The partial that warp k published for sweep `stamp` (waits, bounded); false
// when the wait ran out or another CTA recorded an error.
__device__ __forceinline__ bool wait_published(const unsigned long long* pub, int k, unsigned stamp, SyncBlock* sb,
                                               long long timeout_ns, uint32_t* out)
{
    const unsigned long long t0 = globaltimer_ns();
    unsigned spins = 0;
    for (;;) {
        const unsigned long long v = ld_relaxed_u64(pub + k);
        if ((unsigned)(v >> 32) == stamp) {
            *out = (uint32_t)v;
            return true;
        }
        if (ld_relaxed_i32(&sb->err) != 0) return false;
        if ((++spins & 15u) == 0 && (long long)(globaltimer_ns() - t0) > timeout_ns) {
            atomicCAS(&sb->err, 0, DAG_ERR_BARRIER_TIMEOUT);
            return false;
        }
        __nanosleep(64);
    }
}

}  // namespace dag
