// Warp-worker pull sweep: PageRank (plain and weighted), its adjoint and
// Bellman-Ford in the synchronous, asynchronous and delayed-asynchronous
// forms, with one warp per worker and no CTA-wide barrier inside a sweep.
//
// Paper mapping (Blanco, McMillan, Low, HPEC 2021):
//  * worker = one warp. The merge path of the whole graph (rows and in-edges
//    in vertex order, Merrill & Garland) is cut into warp tiles of WTILE items
//    and every worker takes an equal run of consecutive tiles, so each carries
//    the same in-degree + 1 weight (Sec. III-A's balance) and owns the rows
//    whose end item lies in its run (contiguous in vertex order). A row whose
//    in-edges span two runs (a hub, or a cut inside a row) is owned by the run
//    that ends it; the earlier runs' partial sums reach it at the end of the
//    sweep through a bounded look-back (below);
//  * pull update of each owned vertex from its in-neighbours (Sec. III-A);
//  * sync: values go to the second array (Sec. I); async: values are written
//    in place as soon as a warp tile completes them (Sec. I); delayed: values
//    go to the warp's buffer in shared memory and reach the global array when
//    it holds >= delta values or the run is done (Sec. III, III-B); reads come
//    from the global array (the "global read" form, Sec. III-C);
//  * one grid barrier per iteration (Sec. I) and the stopping rules of Sec. IV.
//
// Why warps: the CTA-tile kernels (sweep.cu, sweep_tma.cu) stop all eight
// warps at three barriers per 1,792-item tile, so each tile waits for its
// slowest gather; here each warp walks its own 224-item tiles with a
// shuffle-only segmented scan and issues the next tile's edge stream and
// gathers before walking the current one, so the SM's 32 warps keep their
// gathers in flight independently.
//
// Row straddling two runs. At the end of its run a warp publishes the partial
// of the row it leaves unfinished (one 64-bit word: sweep stamp and value).
// A warp whose run starts inside a row holds back that row's value and, after
// its own run, adds the partials published by the preceding warps back to the
// one where the row starts (several when a hub spans whole runs); each wait is
// bounded by the launch's timeout. The row then gets its new value like any
// other, so every row is computed once per sweep; only its write comes at the
// end of the sweep.
#include <algorithm>
#include <climits>
#include <cstdint>

#include "sweep_warp.cuh"

namespace dag {

template <int MODE, int VAR, int WIPT>
__global__ void __launch_bounds__(NT, WMINBLOCKS) sweep_warp_kernel(const SweepParams p)
{
    constexpr int WTILE = 32 * WIPT;
    using O = Op<MODE>;
    constexpr bool BF = MODE == MODE_BF || MODE == MODE_BF8;
    constexpr bool SYNC = VAR == DAG_SYNC;
    constexpr bool ASYNC = VAR == DAG_ASYNC;
    constexpr bool DELAYED = VAR == DAG_DELAYED;
    constexpr bool LIVE_G = !SYNC && !BF;  // async/delayed PageRank-type: live global sum
    constexpr unsigned FULL = 0xffffffffu;

    __shared__ WarpShared<WTILE> sh;
    extern __shared__ __align__(16) uint32_t w_buf[];  // delayed: p.buf_cap values per warp

    const int c = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wl = tid >> 5;
    const int w = c * WWARPS + wl;  // this worker
    SyncBlock* sb = p.sync;
    unsigned long long bar_target = 0;
    uint32_t* X0 = (uint32_t*)p.x0;
    uint32_t* X1 = (uint32_t*)p.x1;
    const int row_lo = p.cta_row[w], row_hi = p.cta_row[w + 1];  // rows whose end item lies in the run
    const int t_lo = p.cta_tile[w], t_hi = p.cta_tile[w + 1];
    int* end = sh.end[wl];
    uint32_t* val = sh.val[wl];
    uint32_t* sum = sh.sum[wl];
    uint32_t* buf = w_buf + (size_t)wl * (DELAYED ? p.buf_cap : 0);
    // the run starts inside a row: its first row waits for the earlier runs' partials
    const bool mid0 = t_lo < t_hi && p.tile_nz[t_lo] > p.rowptr[p.tile_row[t_lo]];
    const bool head = mid0 && row_hi > row_lo;

    // ---------------- initial values, a grid-stride pass (a row-range sweep is given them) ----------------
    if (!p.shard) {
        double gpart = 0.0, tpart = 0.0;
        init_values<MODE>(p, X0, gpart, tpart);
        if constexpr (!BF) {
            block_sum2(sh, gpart, tpart);
            if (tid == 0) {
                atomicAdd(&sb->acc_g[2], gpart);
                atomicAdd(&sb->T, tpart);
            }
        }
    }
    if (p.skip_barrier_cta0 && c == 0) return;  // test hook: the others' waits must run out
    if (!p.shard && !grid_barrier(sb, p.nblocks, bar_target, p.timeout_ns)) return;

    double T = 1.0;
    if (tid == 0 && !BF) {
        sh.T = p.shard ? p.shard_T : ld_relaxed_f64(&sb->T);
        sh.gprev = p.shard ? p.shard_N : ld_relaxed_f64(&sb->acc_g[2]);
    }
    __syncthreads();
    if constexpr (!BF) T = (MODE == MODE_ADJ || p.base || p.shard) ? sh.T : 1.0;  // a uniform teleport sums to 1
    double gprev = BF ? 0.0 : sh.gprev;
    AdjOffset A{gprev, 0.0, 0.0f, 0.0, 0.0, 0};  // adjoint: sum lambda, deflation offset
    LiveSum L{};
    if constexpr (LIVE_G) L = live_sum_setup<MODE>(p, T, gprev);
    const double tol = (MODE == MODE_ADJ) ? p.tol * T : p.tol;
    // gathers: sync reads the previous iterate with ordinary loads; async reads the live array
    // in L2 (DAG_READ_CACHED: ordinary loads, refreshed by the grid barrier); delayed per p.read_mode
    const int rmode = SYNC ? READ_CACHED : ASYNC ? (p.read_mode == READ_CACHED ? READ_CACHED : READ_COHERENT)
                                                  : p.read_mode;
    const uint64_t pol_edge = policy_evict_first();
    const uint64_t pol_vertex = policy_evict_last();
    long long flushes = 0;
    int it = 0;
    bool converged = false;
    double last_res = 0.0;

    for (; it < p.max_iters; ++it) {
        const int slot = it % 3;
        const unsigned stamp = (unsigned)it + 1u;
        const uint32_t* xin = SYNC ? ((it & 1) ? X1 : X0) : X0;
        uint32_t* xout = SYNC ? ((it & 1) ? X0 : X1) : X0;
        // per-lane partial sums in FP32 (few rows each); FP64 from the block reduction on
        float res_part = 0.0f, g_part = 0.0f, dg_part = 0.0f;
        uint32_t carry = O::identity();
        bool head_pending = head;
        uint32_t head_part = O::identity();
        int buf_first = row_lo + (head ? 1 : 0), buf_cnt = 0;
        float gt = 0.0f;
        if constexpr (SYNC && !BF)
            gt = (MODE == MODE_ADJ) ? (float)((double)p.g_coef * gprev) : (float)((double)p.g_coef * (T - gprev));

        WStage<WIPT> nx;
        if (t_lo < t_hi) wfetch<MODE, WIPT>(nx, p, xin, t_lo, lane, rmode, LIVE_G, pol_edge, pol_vertex);
        for (int t = t_lo; t < t_hi; ++t) {
            const int a0 = nx.a0, b0 = nx.b0, NA = nx.NA, NB = nx.NB;
            const uint32_t pf_xo = nx.xo;
            const float pf_dg = nx.dg;
            if constexpr (LIVE_G) {  // the global term, from the live sum read with every LIVE_EVERY-th tile
                if (((t - t_lo) & (LIVE_EVERY - 1)) == 0) gt = live_term<MODE>(L, warp_sum(nx.gs));
            }
            __syncwarp();  // the previous tile's epilogue is done with end / val / sum
#pragma unroll
            for (int q = 0; q < WIPT; ++q) {
                const int j = lane + 32 * q;
                if (j < NB) val[j] = nx.term[q];
            }
            wstage_ends<WIPT>(end, nx, p, lane, pol_vertex);
            if (t + 1 < t_hi)
                wfetch<MODE, WIPT>(nx, p, xin, t + 1, lane, rmode, LIVE_G && ((t + 1 - t_lo) & (LIVE_EVERY - 1)) == 0,
                             pol_edge, pol_vertex);
            __syncwarp();
            carry = wwalk<MODE, WIPT>(end, val, sum, NA, NB, carry, lane);
            __syncwarp();

            // -------- new values of the rows this tile completed --------
            const int skip = (head_pending && NA > 0) ? 1 : 0;  // the run's first row waits for the look-back
            if (skip && lane == 0) head_part = sum[0];
            head_pending = head_pending && NA == 0;
            // rows lane + 32 k: the first came with the tile, the others' inputs are loaded together
            uint32_t xo_k[WIPT];
            float dg_k[WIPT];
            xo_k[0] = pf_xo;
            dg_k[0] = pf_dg;
#pragma unroll
            for (int k = 1; k < WIPT; ++k) {
                const int r = lane + 32 * k;
                xo_k[k] = 0u;
                dg_k[k] = 0.0f;
                if (r < NA) {
                    xo_k[k] = ld_weak_b32(xin + a0 + r);
                    if constexpr (!BF) dg_k[k] = ld_stream_f32(p.degf + a0 + r);
                }
            }
            // the adjoint's base terms c_v, all of the tile's loads in flight together (a load per row
            // ahead of its update would wait once per row)
            float bv_k[WIPT];
            if constexpr (MODE == MODE_ADJ) {
#pragma unroll
                for (int k = 0; k < WIPT; ++k) bv_k[k] = lane + 32 * k < NA ? row_base<MODE>(p, a0 + lane + 32 * k) : 0.0f;
            }
#pragma unroll
            for (int k = 0; k < WIPT; ++k) {
                const int r = lane + 32 * k;
                if (r >= NA || (k == 0 && lane == 0 && skip)) continue;
                const int v = a0 + r;
                float bv;
                if constexpr (MODE == MODE_ADJ) bv = bv_k[k];
                else bv = row_base<MODE>(p, v);
                const uint32_t xnew =
                    row_update_b<MODE>(p, v, sum[r], xo_k[k], dg_k[k], gt, bv, A.off_f, res_part, g_part, dg_part);
                if constexpr (SYNC) st_weak_b32(xout + v, xnew);
                else if constexpr (ASYNC) st_relaxed_b32(X0 + v, xnew);
                else buf[v - buf_first] = xnew;
            }
            if constexpr (ASYNC && LIVE_G) {
                if (((t - t_lo) & (LIVE_EVERY - 1)) == LIVE_EVERY - 1) {  // this warp's change of N
                    const float s = warp_sum(dg_part);
                    dg_part = 0.0f;
                    if (lane == 0 && s != 0.0f) live_add(sb, w % GSTRIPES, s, L.S);
                }
            }
            if constexpr (DELAYED) {
                buf_cnt += NA - skip;
                if (buf_cnt >= p.delta || t == t_hi - 1 || (p.buf_clamped && buf_cnt > p.buf_cap - WTILE)) {
                    __syncwarp();  // the buffer's values are written
                    for (int k = lane; k < buf_cnt; k += 32) st_relaxed_b32(X0 + buf_first + k, buf[k]);
                    if constexpr (LIVE_G) {
                        const float s = warp_sum(dg_part);
                        dg_part = 0.0f;
                        __syncwarp();
                        if (lane == 0 && s != 0.0f) {
                            __threadfence();  // this warp's flushed values before its share of N
                            live_add(sb, w % GSTRIPES, s, L.S);
                        }
                    }
                    if (lane == 0) {
                        // refresh this SM's view: later ordinary loads see what other workers published
                        if (rmode == READ_CACHED_REFRESH) asm volatile("fence.acq_rel.gpu;" ::: "memory");
                        ++flushes;
                    }
                    buf_first += buf_cnt;
                    buf_cnt = 0;
                    __syncwarp();  // the buffer is free again
                }
            }
        }  // tiles

        // -------- the row this run leaves unfinished, and the one it started inside --------
        if (lane == 0) st_relaxed_u64(p.wpub + w, ((unsigned long long)stamp << 32) | carry);
        if (head) {
            uint32_t s = __shfl_sync(FULL, head_part, 0);
            bool ok = true;
            for (int k = w - 1; k >= 0; --k) {
                uint32_t pk = 0u;
                if (lane == 0) ok = wait_published(p.wpub, k, stamp, sb, p.timeout_ns, &pk);
                ok = __shfl_sync(FULL, ok, 0);
                pk = __shfl_sync(FULL, pk, 0);
                if (!ok) break;
                s = O::combine(s, pk);
                // the row starts in run k unless run k ends no row and itself starts inside the row
                const int tk0 = p.cta_tile[k], tk1 = p.cta_tile[k + 1];
                const bool k_emits = p.cta_row[k + 1] > p.cta_row[k];
                const bool k_mid = tk0 >= tk1 || p.tile_nz[tk0] > p.rowptr[p.tile_row[tk0]];
                if (k_emits || !k_mid) break;
            }
            if (ok && lane == 0) {
                const int v = row_lo;
                const uint32_t xo = ld_weak_b32(xin + v);
                const float dg = BF ? 0.0f : p.degf[v];
                if constexpr (LIVE_G) gt = live_term<MODE>(L, stripes_total(sb));  // the live term as the row is computed
                const uint32_t xnew = row_update<MODE>(p, v, s, xo, dg, gt, A.off_f, res_part, g_part, dg_part);
                if constexpr (SYNC) st_weak_b32(xout + v, xnew);
                else st_relaxed_b32(X0 + v, xnew);
            }
        }
        if constexpr (LIVE_G) {  // the rest of this warp's change of N
            const float s = warp_sum(dg_part);
            dg_part = 0.0f;
            if (lane == 0 && s != 0.0f) live_add(sb, w % GSTRIPES, s, L.S);
        }

        // -------- end of sweep: residual, barrier, stopping rule --------
        double res_d = (double)res_part, g_d = (double)g_part;
        block_sum2(sh, res_d, g_d);
        if (tid == 0) {
            if (res_d != 0.0) atomicAdd(&sb->acc_res[slot], res_d);
            if ((SYNC || MODE == MODE_ADJ) && !BF && g_d != 0.0) atomicAdd(&sb->acc_g[slot], g_d);
        }
        if (!grid_barrier(sb, p.nblocks, bar_target, p.timeout_ns)) return;
        if (tid == 0) {
            sh.res = ld_relaxed_f64(&sb->acc_res[slot]);
            sh.gprev = ld_relaxed_f64(&sb->acc_g[slot]);
            if (c == 0) {
                const int dead = (it + 2) % 3;  // read by everyone before this barrier
                sb->acc_res[dead] = 0.0;
                sb->acc_g[dead] = 0.0;
            }
        }
        __syncthreads();
        last_res = sh.res;
        gprev = sh.gprev;
        if (last_res <= tol) {
            converged = true;
            ++it;
            break;
        }
        if constexpr (MODE == MODE_ADJ) adjoint_deflate(p, A, gprev, SYNC);  // the slow mode along 1, as an offset
    }

    // ---------------- output, a grid-stride pass (a row-range sweep leaves them in x1) ----------------
    if (!p.shard) {
        const uint32_t* xf = SYNC ? ((it & 1) ? X1 : X0) : X0;
        write_output<MODE>(p, xf, A.off_f);
    }
    if (lane == 0 && flushes) atomicAdd((unsigned long long*)&sb->flushes, (unsigned long long)flushes);
    if (tid == 0 && c == 0) {
        sb->iters = it;
        sb->residual = last_res;
        sb->converged = converged ? 1 : 0;
    }
}

// ---------------------------------------------------------------------------
// Ordered warp sweep (asynchronous form, DAG_WARP_ORDERED): the warps take the
// tiles of the whole merge path in turn instead of each walking a run of its
// own, tile t to warp t mod W, so at any moment the GPU works on one window of
// W consecutive tiles and a sweep visits the vertices in order across the GPU:
// one in-order stream, as a single thread's asynchronous sweep (Sec. I) with
// every warp on it. A row whose in-edges
// span tiles is finished with a decoupled look-back over per-tile published
// partials (Merrill & Garland's single-pass scan): every tile publishes the
// partial of the row it leaves unfinished at once (inclusive when that row
// starts inside the tile, else an aggregate, upgraded to inclusive later), and
// the tile that ends a row begun earlier adds the published partials back to
// the first inclusive one, 32 tiles per step (one per lane). A warp resolves
// its tile's look-back after walking its next tile, by when the tiles before
// it have published (a tile publishes before its warp resolves anything
// older, so the lowest pending tile can always finish); each wait is bounded
// by the launch's timeout.
// ---------------------------------------------------------------------------
constexpr unsigned TPUB_INCL = 0x80000000u;  // the published value is the row's partial from its start

// The word tile j published in sweep `stamp` (waits, bounded); false when the wait ran out or another CTA
// recorded an error.
__device__ __forceinline__ bool wait_tile(const unsigned long long* pub, int j, unsigned stamp, SyncBlock* sb,
                                          long long timeout_ns, unsigned long long* out)
{
    const unsigned long long t0 = globaltimer_ns();
    unsigned spins = 0;
    for (;;) {
        const unsigned long long v = ld_relaxed_u64(pub + j);
        if (((unsigned)(v >> 32) & ~TPUB_INCL) == stamp) {
            *out = v;
            return true;
        }
        if (ld_relaxed_i32(&sb->err) != 0) return false;
        if ((++spins & 15u) == 0 && (long long)(globaltimer_ns() - t0) > timeout_ns) {
            atomicCAS(&sb->err, 0, DAG_ERR_BARRIER_TIMEOUT);
            return false;
        }
        __nanosleep(32);
    }
}

template <int MODE, int WIPT>
__global__ void __launch_bounds__(NT, WMINBLOCKS) sweep_ordered_kernel(const SweepParams p)
{
    using O = Op<MODE>;
    constexpr int WTILE = 32 * WIPT;
    constexpr bool BF = MODE == MODE_BF || MODE == MODE_BF8;
    constexpr bool LIVE_G = !BF;
    constexpr unsigned FULL = 0xffffffffu;
    (void)WTILE;

    __shared__ WarpShared<32 * WIPT> sh;
    const int c = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wl = tid >> 5;
    const int w = c * WWARPS + wl;
    const int W = p.nblocks * WWARPS, T = p.ntiles;  // warp w takes tiles w, w + W, w + 2W, ...
    SyncBlock* sb = p.sync;
    unsigned long long bar_target = 0;
    uint32_t* X = (uint32_t*)p.x0;
    unsigned long long* pub = p.wpub;  // [T]
    int* end = sh.end[wl];
    uint32_t* val = sh.val[wl];
    uint32_t* sum = sh.sum[wl];

    // ---------------- initial values (any thread any row: nothing reads them before the barrier) ----------------
    {
        double gpart = 0.0, tpart = 0.0;
        init_values<MODE>(p, X, gpart, tpart);
        if constexpr (!BF) {
            block_sum2(sh, gpart, tpart);
            if (tid == 0) {
                atomicAdd(&sb->acc_g[2], gpart);
                atomicAdd(&sb->T, tpart);
            }
        }
    }
    if (p.skip_barrier_cta0 && c == 0) return;  // test hook: the others' waits must run out
    if (!grid_barrier(sb, p.nblocks, bar_target, p.timeout_ns)) return;

    double T_tot = 1.0;
    if (tid == 0 && !BF) {
        sh.T = ld_relaxed_f64(&sb->T);
        sh.gprev = ld_relaxed_f64(&sb->acc_g[2]);
    }
    __syncthreads();
    if constexpr (!BF) T_tot = (MODE == MODE_ADJ || p.base) ? sh.T : 1.0;
    LiveSum L{};
    if constexpr (LIVE_G) L = live_sum_setup<MODE>(p, T_tot, sh.gprev);
    AdjOffset A{BF ? 0.0 : sh.gprev, 0.0, 0.0f, 0.0, 0.0, 0};  // adjoint: sum lambda, deflation offset
    const double tol = (MODE == MODE_ADJ) ? p.tol * T_tot : p.tol;
    const int rmode = p.read_mode == READ_CACHED ? READ_CACHED : READ_COHERENT;
    const uint64_t pol_edge = policy_evict_first();
    const uint64_t pol_vertex = policy_evict_last();
    int it = 0;
    bool converged = false;
    double last_res = 0.0;

    for (; it < p.max_iters; ++it) {
        const int slot = it % 3;
        const unsigned stamp = (unsigned)it + 1u;
        float res_part = 0.0f, g_part = 0.0f, dg_part = 0.0f;
        float gt = 0.0f;
        // the look-back this warp still owes (warp-uniform): tile, its first row, the tile's partial of it,
        // whether the row ends in the tile (else the tile's published aggregate is upgraded), its inputs
        int pend_t = -1, pend_row = 0, pend_fin = 0;
        uint32_t pend_val = 0u, pend_xo = 0u;
        float pend_dg = 0.0f;
        bool ok = true;

        // Adds the partials published by the tiles before pend_t back to the first inclusive one, then
        // finishes the pending row or publishes the tile's inclusive partial. The warp looks back 32
        // tiles at a time, one per lane (lane i reads tile hi - i), as in a single-pass scan's look-back:
        // the nearest inclusive entry ends the walk, the partials after it are reduced over the lanes.
        auto resolve = [&]() {
            if (pend_t < 0) return;
            uint32_t C = O::identity();
            for (int hi = pend_t - 1; ok;) {
                const int j = hi - lane;
                unsigned long long v = 0ull;
                bool got = true;
                if (j >= 0) got = wait_tile(pub, j, stamp, sb, p.timeout_ns, &v);
                ok = __all_sync(FULL, got) != 0;
                if (!ok) break;
                const unsigned incl = __ballot_sync(FULL, j >= 0 && (((unsigned)(v >> 32)) & TPUB_INCL) != 0);
                const int stop = incl ? __ffs(incl) - 1 : 31;  // the nearest inclusive entry, else the whole window
                uint32_t mine = (j >= 0 && lane <= stop) ? (uint32_t)v : O::identity();
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) mine = O::combine(mine, __shfl_xor_sync(FULL, mine, o));
                C = O::combine(C, mine);
                if (incl || hi < 32) break;  // tile 0 is always inclusive, so the walk ends by then
                hi -= 32;
            }
            if (ok && lane == 0) {
                const uint32_t total = O::combine(C, pend_val);
                if (pend_fin) {
                    const uint32_t xnew =
                        row_update<MODE>(p, pend_row, total, pend_xo, pend_dg, gt, A.off_f, res_part, g_part, dg_part);
                    st_relaxed_b32(X + pend_row, xnew);
                } else {
                    st_relaxed_u64(pub + pend_t, ((unsigned long long)(stamp | TPUB_INCL) << 32) | total);
                }
            }
            pend_t = -1;
        };

        WStage<WIPT> nx;
        int k = 0;  // this warp's tiles so far in the sweep
        if (w < T) wfetch<MODE, WIPT>(nx, p, X, w, lane, rmode, LIVE_G, pol_edge, pol_vertex);
        for (int t = w; t < T && ok; t += W, ++k) {
            const int a0 = nx.a0, b0 = nx.b0, NA = nx.NA, NB = nx.NB;
            const bool cont = b0 > nx.rp0;  // the tile starts inside row a0
            const uint32_t pf_xo = nx.xo;
            const float pf_dg = nx.dg;
            if constexpr (LIVE_G) {
                if ((k & (LIVE_EVERY - 1)) == 0) gt = live_term<MODE>(L, warp_sum(nx.gs));
            }
            __syncwarp();
#pragma unroll
            for (int q = 0; q < WIPT; ++q) {
                const int j = lane + 32 * q;
                if (j < NB) val[j] = nx.term[q];
            }
            wstage_ends<WIPT>(end, nx, p, lane, pol_vertex);
            if (t + W < T)
                wfetch<MODE, WIPT>(nx, p, X, t + W, lane, rmode, LIVE_G && ((k + 1) & (LIVE_EVERY - 1)) == 0,
                                   pol_edge, pol_vertex);
            __syncwarp();
            const uint32_t trail = wwalk<MODE, WIPT>(end, val, sum, NA, NB, O::identity(), lane);
            __syncwarp();
            // the partial of the row left unfinished: inclusive unless the tile lies inside a row begun before
            const bool incl = NA > 0 || !cont;
            if (lane == 0)
                st_relaxed_u64(pub + t, ((unsigned long long)(stamp | (incl ? TPUB_INCL : 0u)) << 32) | trail);

            // -------- rows this tile completed (its first one, begun before, waits for the look-back) --------
            const int skip = (cont && NA > 0) ? 1 : 0;
            const uint32_t first_sum = __shfl_sync(FULL, NA > 0 ? sum[0] : 0u, 0);
            uint32_t xo_k[WIPT];
            float dg_k[WIPT];
            xo_k[0] = pf_xo;
            dg_k[0] = pf_dg;
#pragma unroll
            for (int q = 1; q < WIPT; ++q) {
                const int r = lane + 32 * q;
                xo_k[q] = 0u;
                dg_k[q] = 0.0f;
                if (r < NA) {
                    xo_k[q] = ld_weak_b32(X + a0 + r);
                    if constexpr (!BF) dg_k[q] = ld_stream_f32(p.degf + a0 + r);
                }
            }
            float bv_k[WIPT];  // the adjoint's base terms c_v, loaded together
            if constexpr (MODE == MODE_ADJ) {
#pragma unroll
                for (int q = 0; q < WIPT; ++q) bv_k[q] = lane + 32 * q < NA ? row_base<MODE>(p, a0 + lane + 32 * q) : 0.0f;
            }
#pragma unroll
            for (int q = 0; q < WIPT; ++q) {
                const int r = lane + 32 * q;
                if (r >= NA || (q == 0 && lane == 0 && skip)) continue;
                const int v = a0 + r;
                float bv;
                if constexpr (MODE == MODE_ADJ) bv = bv_k[q];
                else bv = row_base<MODE>(p, v);
                const uint32_t xnew =
                    row_update_b<MODE>(p, v, sum[r], xo_k[q], dg_k[q], gt, bv, A.off_f, res_part, g_part, dg_part);
                st_relaxed_b32(X + v, xnew);
            }
            // -------- the previous tile's look-back, then this tile's becomes pending --------
            resolve();
            if (cont) {
                pend_t = t;
                pend_row = a0;
                pend_fin = NA > 0 ? 1 : 0;
                pend_val = NA > 0 ? first_sum : trail;
                pend_xo = __shfl_sync(FULL, pf_xo, 0);
                pend_dg = __shfl_sync(FULL, pf_dg, 0);
            }
            if constexpr (LIVE_G) {
                if ((k & (LIVE_EVERY - 1)) == LIVE_EVERY - 1) {  // this warp's change of N
                    const float s = warp_sum(dg_part);
                    dg_part = 0.0f;
                    if (lane == 0 && s != 0.0f) live_add(sb, w % GSTRIPES, s, L.S);
                }
            }
        }  // tiles
        resolve();
        if constexpr (LIVE_G) {
            const float s = warp_sum(dg_part);
            dg_part = 0.0f;
            if (lane == 0 && s != 0.0f) live_add(sb, w % GSTRIPES, s, L.S);
        }

        // -------- end of sweep: residual, barrier, stopping rule --------
        double res_d = (double)res_part, g_d = (double)g_part;
        block_sum2(sh, res_d, g_d);
        if (tid == 0 && res_d != 0.0) atomicAdd(&sb->acc_res[slot], res_d);
        if (MODE == MODE_ADJ && tid == 0 && g_d != 0.0) atomicAdd(&sb->acc_g[slot], g_d);
        if (!grid_barrier(sb, p.nblocks, bar_target, p.timeout_ns)) return;
        if (tid == 0) {
            sh.res = ld_relaxed_f64(&sb->acc_res[slot]);
            if (MODE == MODE_ADJ) sh.gprev = ld_relaxed_f64(&sb->acc_g[slot]);
            if (c == 0) {
                const int dead = (it + 2) % 3;  // read by everyone before this barrier
                sb->acc_res[dead] = 0.0;
                sb->acc_g[dead] = 0.0;
            }
        }
        __syncthreads();
        last_res = sh.res;
        if (last_res <= tol) {
            converged = true;
            ++it;
            break;
        }
        if constexpr (MODE == MODE_ADJ) adjoint_deflate(p, A, sh.gprev, false);  // the slow mode along 1, as an offset
    }

    // ---------------- output ----------------
    write_output<MODE>(p, X, A.off_f);
    if (tid == 0 && c == 0) {
        sb->iters = it;
        sb->residual = last_res;
        sb->converged = converged ? 1 : 0;
    }
}

const void* sweep_ordered_kernel_ptr(int mode, int ipt)
{
#define DAG_ORD_ROW(I)                                                                                        \
    {(const void*)sweep_ordered_kernel<MODE_PR, I>, (const void*)sweep_ordered_kernel<MODE_PRW, I>,         \
     (const void*)sweep_ordered_kernel<MODE_ADJ, I>, (const void*)sweep_ordered_kernel<MODE_BF, I>,         \
     (const void*)sweep_ordered_kernel<MODE_BF8, I>}
    static const void* const table[3][5] = {DAG_ORD_ROW(5), DAG_ORD_ROW(7), DAG_ORD_ROW(11)};
#undef DAG_ORD_ROW
    const int k = ipt == 5 ? 0 : ipt == 7 ? 1 : ipt == 11 ? 2 : -1;
    return k < 0 ? nullptr : table[k][mode];
}

// Kernel of (mode, variant, items per lane); nullptr for a shape not built.
const void* sweep_warp_kernel_ptr(int mode, int variant, int ipt)
{
#define DAG_WARP_ROW(M, I)                                                                                    \
    {(const void*)sweep_warp_kernel<M, DAG_SYNC, I>, (const void*)sweep_warp_kernel<M, DAG_ASYNC, I>,       \
     (const void*)sweep_warp_kernel<M, DAG_DELAYED, I>}
#define DAG_WARP_SHAPE(I) \
    {DAG_WARP_ROW(MODE_PR, I), DAG_WARP_ROW(MODE_PRW, I), DAG_WARP_ROW(MODE_ADJ, I), DAG_WARP_ROW(MODE_BF, I), \
     DAG_WARP_ROW(MODE_BF8, I)}
    static const void* const table[3][5][3] = {DAG_WARP_SHAPE(5), DAG_WARP_SHAPE(7), DAG_WARP_SHAPE(11)};
#undef DAG_WARP_SHAPE
#undef DAG_WARP_ROW
    const int k = ipt == 5 ? 0 : ipt == 7 ? 1 : ipt == 11 ? 2 : -1;
    return k < 0 ? nullptr : table[k][mode][variant];
}

// Launch shape of a warp-worker sweep: CTAs resident at once (cooperative
// launch), warps = CTAs * WWARPS workers, and the delayed form's buffer of
// min(delta - 1 + WTILE, rows of the longest run) values per warp, clamped to
// what fits in shared memory (flushed when the next tile might not fit).
enum WarpKind { WARP_RUNS = 0, WARP_ORDERED = 1, WARP_FRONTIER = 2 };

static const void* warp_kernel(int kind, int mode, int variant, int ipt, bool ordered = false)
{
    if (kind == WARP_ORDERED) return sweep_ordered_kernel_ptr(mode, ipt);
    if (kind == WARP_FRONTIER) return sweep_warp_frontier_kernel_ptr(mode, ipt, ordered);
    return sweep_warp_kernel_ptr(mode, variant, ipt);
}

static int warp_shape(dag_plan* plan, int mode, int variant, int delta, int* nb_out, int* cap_out, int* clamped_out,
                      Partition** part_out, cudaStream_t s, int kind, bool ordered = false)
{
    const int WTILE = 32 * plan->warp_ipt;
    const void* k = warp_kernel(kind, mode, variant, plan->warp_ipt, ordered);
    if (!k) return set_error(DAG_ERR_INVALID, "no warp tile of that shape");
    cudaFuncAttributes fa{};
    DAG_CUDA(cudaFuncGetAttributes(&fa, k));
    int max_dyn = 0;
    DAG_CUDA(cudaDeviceGetAttribute(&max_dyn, cudaDevAttrMaxSharedMemoryPerBlockOptin, plan->device));
    const long long max_cap = ((long long)max_dyn - (long long)fa.sharedSizeBytes) / (4LL * WWARPS);
    int cap = 0, clamped = 0, nb = 0;
    Partition* part = nullptr;
    auto resident = [&](int cap_elems, int* out) -> int {
        const size_t dyn = (size_t)WWARPS * (size_t)cap_elems * 4;
        DAG_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
        DAG_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
        int per_sm = 0;
        DAG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NT, dyn));
        if (per_sm < 1) return set_error(DAG_ERR_INVALID, "warp sweep cannot be resident with this delta");
        const int rc = set_l1_carveout(k, plan->device, NT, fa.sharedSizeBytes, dyn, per_sm);
        if (rc) return rc;
        int n_cta = per_sm * plan->num_sms;
        if (plan->worker_cap > 0) n_cta = std::min(n_cta, plan->worker_cap);  // the cap counts CTAs
        *out = n_cta;
        return DAG_OK;
    };
    int rc = resident(0, &nb);
    if (rc) return rc;
    bool settled = false;  // CTAs per SM only fall, so a few passes settle the shape
    for (int iter = 0; iter < 6 && !settled; ++iter) {
        rc = get_warp_partition(plan, nb * WWARPS, WTILE, &part, s);
        if (rc) return rc;
        settled = true;
        if (variant != DAG_DELAYED) break;
        const long long want = std::min((long long)delta - 1 + WTILE, (long long)std::max(part->max_rows, 1));
        const long long need = std::min(want, max_cap);
        clamped = need < want ? 1 : 0;
        if (clamped && need < WTILE + 1) return set_error(DAG_ERR_INVALID, "delay buffer does not fit in shared memory");
        cap = (int)std::max(need, 1LL);
        int nb2 = 0;
        rc = resident(cap, &nb2);
        if (rc) return rc;
        if (nb2 < nb) {
            nb = nb2;
            settled = false;
        }
    }
    if (!settled) return set_error(DAG_ERR_INVALID, "warp sweep launch shape did not settle");
    *nb_out = nb;
    *cap_out = cap;
    *clamped_out = clamped;
    *part_out = part;
    return DAG_OK;
}

// The frontier maps of the warp partition a frontier solve of this plan would use (built once, outside the
// timed solve, as the CTA-tile frontier's are).
int warp_frontier_maps(dag_plan* plan, int mode, cudaStream_t s)
{
    int nb = 0, cap = 0, clamped = 0;
    Partition* part = nullptr;
    int rc = warp_shape(plan, mode, DAG_ASYNC, 0, &nb, &cap, &clamped, &part, s, WARP_FRONTIER);
    if (rc) return rc;
    return frontier_maps(plan, part, s, false);
}

int launch_warp_sweep(dag_plan* plan, int mode, int variant, int delta, SweepParams& p, cudaStream_t s,
                      int* out_nblocks)
{
    if (p.local_read || p.own_l1) return set_error(DAG_ERR_INVALID, "local and own-block reads run the CTA-tile sweeps");
    const bool ordered = p.ordered != 0;
    if (ordered && variant != DAG_ASYNC)
        return set_error(DAG_ERR_INVALID, "ordered warp sweeps run the asynchronous form (delta 0)");
    if (p.frontier && (variant != DAG_ASYNC || (mode != MODE_BF && mode != MODE_BF8)))
        return set_error(DAG_ERR_INVALID, "the warp-tile frontier runs the asynchronous Bellman-Ford form");
    const int kind = p.frontier ? WARP_FRONTIER : ordered ? WARP_ORDERED : WARP_RUNS;
    int nb = 0, cap = 0, clamped = 0;
    Partition* part = nullptr;
    int rc = warp_shape(plan, mode, variant, delta, &nb, &cap, &clamped, &part, s, kind, ordered);
    if (rc) return rc;
    if (kind == WARP_ORDERED && !part->tpub)
        DAG_CUDA(cudaMalloc(&part->tpub, (size_t)part->tiles * sizeof(unsigned long long)));
    if (p.frontier) {
        rc = frontier_maps(plan, part, s, false);
        if (rc) return rc;
        p.fr_orow = plan->fr_orow;
        p.fr_otile = part->fr_otile;
        p.fr_oend = part->fr_oend;
        p.fr_act = part->fr_act;
        p.fr_alist = part->fr_alist;
        p.fr_chg = part->fr_chg;
        p.fr_glist = part->fr_glist;
        p.fr_gchg = part->fr_gchg;
        p.fr_sparse = plan->fr_sparse_warp;
        DAG_CUDA(cudaMemsetAsync(part->fr_act, 0, (size_t)std::max(part->tiles, 1) * sizeof(int), s));
    }
    p.nblocks = nb;
    p.delta = (variant == DAG_DELAYED) ? delta : 0;
    p.buf_cap = cap;
    p.buf_clamped = clamped;
    p.cta_row = part->cta_row;
    p.cta_tile = part->cta_tile;
    p.tile_row = part->tile_row;
    p.tile_nz = part->tile_nz;
    p.wpub = kind == WARP_ORDERED ? part->tpub : part->wpub;
    p.ntiles = part->tiles;
    p.sync = plan->sync;
    p.timeout_ns = plan->timeout_ns;
    p.skip_barrier_cta0 = 0;
    p.stall_fill = 0;
    if (plan->skip_barrier_once) {
        p.skip_barrier_cta0 = 1;
        p.timeout_ns = plan->skip_timeout_ns;
        plan->skip_barrier_once = 0;
    }
    DAG_CUDA(cudaMemsetAsync(plan->sync, 0, sizeof(SyncBlock), s));
    // stamps of an earlier solve must not pass for this one's
    DAG_CUDA(cudaMemsetAsync(p.wpub, 0,
                             (size_t)(kind == WARP_ORDERED ? part->tiles : part->nblocks) * sizeof(unsigned long long),
                             s));
    const void* k = warp_kernel(kind, mode, variant, plan->warp_ipt, ordered);
    const size_t dyn = (size_t)WWARPS * (size_t)cap * 4;
    DAG_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    void* args[] = {(void*)&p};
    DAG_CUDA(cudaLaunchCooperativeKernel(k, dim3(nb), dim3(NT), args, dyn, s));
    *out_nblocks = nb * WWARPS;
    return DAG_OK;
}

// One synchronous sweep over rows [lo, hi) of the plan's graph (row sharding
// across GPUs, rowshard.py): x_in is the whole previous iterate, the new
// values of the range go to x_out[lo, hi), and d_sums receives {sum |r' - r|
// over the range (PageRank; Bellman-Ford: rows lowered), sum of r' over the
// range's vertices with out-edges (PageRank)} in FP64. The range's merge path
// is cut into warp tiles and warp runs as in a whole sweep.
__global__ void k_copy_sums(const SyncBlock* sb, double* out)
{
    out[0] = sb->acc_res[0];
    out[1] = sb->acc_g[0];
}

int sweep_rows(dag_plan* plan, int mode, int lo, int hi, SweepParams& p, double* d_sums, cudaStream_t s)
{
    const int WTILE = 32 * plan->warp_ipt;
    const void* k = sweep_warp_kernel_ptr(mode, DAG_SYNC, plan->warp_ipt);
    cudaFuncAttributes fa{};
    DAG_CUDA(cudaFuncGetAttributes(&fa, k));
    DAG_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 0));
    int per_sm = 0;
    DAG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NT, 0));
    if (per_sm < 1) return set_error(DAG_ERR_INVALID, "row sweep cannot be resident");
    int nb = per_sm * plan->num_sms;
    if (plan->worker_cap > 0) nb = std::min(nb, plan->worker_cap);
    Partition* part = nullptr;
    int rc = get_warp_partition_range(plan, nb * WWARPS, WTILE, lo, hi, &part, s);
    if (rc) return rc;
    p.nblocks = nb;
    p.max_iters = 1;
    p.tol = 0.0;
    p.delta = 0;
    p.buf_cap = 0;
    p.buf_clamped = 0;
    p.shard = 1;
    p.cta_row = part->cta_row;
    p.cta_tile = part->cta_tile;
    p.tile_row = part->tile_row;
    p.tile_nz = part->tile_nz;
    p.wpub = part->wpub;
    p.sync = plan->sync;
    p.timeout_ns = plan->timeout_ns;
    DAG_CUDA(cudaMemsetAsync(plan->sync, 0, sizeof(SyncBlock), s));
    DAG_CUDA(cudaMemsetAsync(part->wpub, 0, (size_t)part->nblocks * sizeof(unsigned long long), s));
    void* args[] = {(void*)&p};
    DAG_CUDA(cudaLaunchCooperativeKernel(k, dim3(nb), dim3(NT), args, 0, s));
    k_copy_sums<<<1, 1, 0, s>>>(plan->sync, d_sums);
    DAG_CUDA(cudaGetLastError());
    return DAG_OK;
}

}  // namespace dag

extern "C" int dag_plan_set_warp_tile(dag_plan* plan, int32_t items_per_lane)
{
    if (!plan) return dag::set_error(DAG_ERR_INVALID, "null plan");
    if (!dag::sweep_warp_kernel_ptr(dag::MODE_PR, DAG_SYNC, items_per_lane))
        return dag::set_error(DAG_ERR_INVALID, "items per lane must be 5, 7 or 11");
    plan->warp_ipt = items_per_lane;
    return DAG_OK;
}

extern "C" int32_t dag_warp_tile_items(const dag_plan* plan)
{
    return 32 * (plan ? plan->warp_ipt : dag::WIPT_DEFAULT);
}

extern "C" int dag_plan_set_warp_frontier_marks(dag_plan* plan, float marks_per_tile)
{
    if (!plan) return dag::set_error(DAG_ERR_INVALID, "null plan");
    if (!(marks_per_tile >= 0.0f) || !(marks_per_tile <= 1.0e6f))
        return dag::set_error(DAG_ERR_INVALID, "marks per tile must lie in [0, 1e6]");
    plan->fr_sparse_warp = marks_per_tile;
    return DAG_OK;
}
