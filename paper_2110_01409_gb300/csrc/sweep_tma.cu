// Asynchronous pull sweep (Sec. I; delta = 0 of the delayed method, Sec. III-B)
// of PageRank, weighted PageRank, the PageRank adjoint and Bellman-Ford, with
// TMA-staged tiles.
//
// The asynchronous form reads the live state with relaxed gpu-scope loads,
// which L2 serves, so its gathers gain nothing from L1; what it needs is
// gathers in flight long enough to cover L2 latency. So a tile's contiguous
// inputs (edge stream, row ends, weights or values, the first NT rows' old
// values and out-degrees) are copied by the TMA engine (cp.async.bulk) two
// tiles ahead into a three-slot shared-memory ring, completing on one
// mbarrier per slot, and the tile's gathers are issued a whole tile ahead from
// the staged edge stream. The walk, scan and row update are those of the
// register-staged kernel (sweep_common.cuh). Every wait on a ring mbarrier is
// bounded by the launch's timeout: when one runs out the CTA records
// DAG_ERR_BARRIER_TIMEOUT, waits (bounded) for its own copies and leaves, and
// the other CTAs' grid-barrier waits end on the recorded error.
//
// Own block through L1 (DAG_READ_OWN_L1): only the owning CTA writes its
// vertices, and its barriers order its stores before its later loads, so an
// ordinary load of its own vertices is as fresh as a gpu-scope one; with the
// flag set those gathers use ordinary loads and may hit in L1.
#include <cstdint>

#include "sweep_common.cuh"

namespace dag {

// Ring layout (dynamic shared memory). Every copy starts at the 16-byte
// boundary at or below its first element and ends at the one at or above its
// last, so it stays inside the 16-byte granules that hold the wanted elements
// (arrays are 16-byte aligned; the launch checks).
template <int MODE>
struct Ring {
    static constexpr bool BF = MODE == MODE_BF || MODE == MODE_BF8;
    static constexpr int CR_INTS = TILE + 12;  // edge stream + row ends (a tile's rows + edges <= TILE) + slack
    static constexpr int OLD_INTS = NT + 8;    // old values of the tile's first NT rows + slack
    static constexpr int AUX_BYTES = MODE == MODE_PR ? 0 : MODE == MODE_BF8 ? TILE + 32 : (TILE + 8) * 4;
    static constexpr int DEG_INTS = BF ? 0 : OLD_INTS;
    static constexpr int OFF_CR = 0;
    static constexpr int OFF_OLD = OFF_CR + RING * CR_INTS * 4;
    static constexpr int OFF_DEG = OFF_OLD + RING * OLD_INTS * 4;
    static constexpr int OFF_AUX = OFF_DEG + RING * DEG_INTS * 4;
    static constexpr int BYTES = OFF_AUX + 2 * AUX_BYTES;  // weights: two slots, consumed before barrier (A)
    static_assert(CR_INTS % 4 == 0 && OLD_INTS % 4 == 0 && AUX_BYTES % 16 == 0, "16-byte slot sizes");
};

// Where tile t's inputs sit inside its slot (element offsets) and how much each
// copy moves. Every thread derives the same numbers from the tile's
// merge-path coordinates.
struct TileGeo {
    int a0, b0, NA, NB;
    int c_n;   // edge-stream elements copied (multiple of 4): at most NB + 6
    int r_n;   // row-end elements copied (multiple of 4): at most NA + 6
    int nold;  // rows whose old value / out-degree is staged: min(NA, NT)
    int o_n;   // old-value elements copied (multiple of 4): at most nold + 6
    __device__ __forceinline__ int col_off() const { return b0 & 3; }
    __device__ __forceinline__ int rend_off() const { return c_n + ((a0 + 1) & 3); }
    __device__ __forceinline__ int old_off() const { return a0 & 3; }
};

__device__ __forceinline__ TileGeo tile_geo(const SweepParams& p, int t)
{
    TileGeo g;
    g.a0 = p.tile_row[t];
    g.b0 = p.tile_nz[t];
    g.NA = p.tile_row[t + 1] - g.a0;
    g.NB = p.tile_nz[t + 1] - g.b0;
    g.c_n = g.NB ? ((g.b0 + g.NB + 3) & ~3) - (g.b0 & ~3) : 0;
    g.r_n = g.NA ? ((g.a0 + g.NA + 4) & ~3) - ((g.a0 + 1) & ~3) : 0;
    g.nold = g.NA < NT ? g.NA : NT;
    g.o_n = g.nold ? ((g.a0 + g.nold + 3) & ~3) - (g.a0 & ~3) : 0;
    return g;
}

template <int MODE>
__device__ __forceinline__ int aux_off(const TileGeo& g)
{
    return MODE == MODE_BF8 ? (g.b0 & 15) : (g.b0 & 3);
}

template <int MODE>
__device__ __forceinline__ int aux_bytes(const TileGeo& g)
{
    if constexpr (MODE == MODE_PR) return 0;
    else if constexpr (MODE == MODE_BF8) return g.NB ? ((g.b0 + g.NB + 15) & ~15) - (g.b0 & ~15) : 0;
    else return 4 * g.c_n;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.u32 %0, 1, 0, P;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Waits for the phase of a ring mbarrier with the given parity, bounded by
// timeout_ns of the global timer.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, uint32_t parity, long long timeout_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if ((long long)(globaltimer_ns() - t0) > timeout_ns) return false;
    }
    return true;
}

__device__ __forceinline__ void tma_load(void* dst, const void* src, uint32_t bytes, unsigned long long* bar,
                                         uint64_t pol)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}

// Lane 0 of warp 1 adds the warps' shares of the last tile's change of the
// live sum N to this CTA's stripe (one atomic per tile instead of one per
// warp: the stripe lines are read by every CTA each tile) and clears them.
template <class SH>
__device__ __forceinline__ void flush_dg(SH& sh, SyncBlock* sb, int c, int S)
{
    if (threadIdx.x == 32) {
        float tot = 0.0f;
#pragma unroll
        for (int k = 0; k < NWARP; ++k) {
            tot += sh.dgw[k];
            sh.dgw[k] = 0.0f;
        }
        live_add(sb, c % GSTRIPES, tot, S);
    }
}

// Thread 0: starts the copies of tile t into the ring slot of fill q.
template <int MODE>
__device__ __forceinline__ void issue_fill(unsigned char* ring, unsigned long long* bars, uint32_t q,
                                           const SweepParams& p, const uint32_t* x, int t, uint64_t pol_edge,
                                           uint64_t pol_vertex)
{
    using R = Ring<MODE>;
    const TileGeo g = tile_geo(p, t);
    const int s3 = (int)(q % RING), s2 = (int)(q & 1u);
    int* cr = (int*)(ring + R::OFF_CR) + s3 * R::CR_INTS;
    const int ab = aux_bytes<MODE>(g);
    uint32_t bytes = 4u * (uint32_t)(g.c_n + g.r_n) + (uint32_t)ab + 4u * (uint32_t)g.o_n * (R::BF ? 1u : 2u);
    if (p.stall_fill && q == 0 && blockIdx.x == 0) bytes += 16u;  // test hook: this phase never completes
    unsigned long long* bar = &bars[s3];
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // earlier generic accesses of the slot first
    mbar_expect_tx(bar, bytes);
    if (g.c_n) tma_load(cr, p.colidx + (g.b0 & ~3), 4u * g.c_n, bar, pol_edge);
    if (g.r_n) tma_load(cr + g.c_n, p.rowptr + ((g.a0 + 1) & ~3), 4u * g.r_n, bar, pol_vertex);
    if constexpr (MODE != MODE_PR) {
        unsigned char* aux = ring + R::OFF_AUX + s2 * R::AUX_BYTES;
        if (ab) {
            if constexpr (MODE == MODE_BF8) tma_load(aux, p.w8 + (g.b0 & ~15), (uint32_t)ab, bar, pol_edge);
            else if constexpr (MODE == MODE_BF) tma_load(aux, p.w + (g.b0 & ~3), (uint32_t)ab, bar, pol_edge);
            else tma_load(aux, p.val + (g.b0 & ~3), (uint32_t)ab, bar, pol_edge);
        }
    }
    if (g.o_n) {
        uint32_t* old = (uint32_t*)(ring + R::OFF_OLD) + s3 * R::OLD_INTS;
        tma_load(old, x + (g.a0 & ~3), 4u * g.o_n, bar, pol_vertex);
        if constexpr (!R::BF) {
            uint32_t* deg = (uint32_t*)(ring + R::OFF_DEG) + s3 * R::OLD_INTS;
            tma_load(deg, p.degf + (g.a0 & ~3), 4u * g.o_n, bar, pol_vertex);
        }
    }
}

// Issues the gathers of a tile's edges from the staged edge stream.
__device__ __forceinline__ void gather_tile(uint32_t (&term)[IPT], const int* col, int NB, const uint32_t* x, int tid,
                                            uint64_t pol_vertex, int own_lo, int own_n)
{
#pragma unroll
    for (int k = 0; k < IPT; ++k) {
        const int j = tid + k * NT;
        uint32_t xv = 0u;
        if (j < NB) {
            const int u = col[j];
            xv = (unsigned)(u - own_lo) < (unsigned)own_n ? ld_weak_keep_b32(x + u, pol_vertex)
                                                          : ld_relaxed_keep_b32(x + u, pol_vertex);
        }
        term[k] = xv;
    }
}

// Edge term of the walk from a gathered value and the edge's weight / value.
template <int MODE>
__device__ __forceinline__ uint32_t edge_term(uint32_t xv, const unsigned char* aux, int k)
{
    if constexpr (MODE == MODE_BF8) return relax(xv, (uint32_t)aux[k]);
    else if constexpr (MODE == MODE_BF) return relax(xv, ((const uint32_t*)aux)[k]);
    else if constexpr (MODE == MODE_PR) return xv;
    else return __float_as_uint(__uint_as_float(((const uint32_t*)aux)[k]) * __uint_as_float(xv));
}

// FRONTIER (Bellman-Ford): after a sweep whose changed rows feed few tiles,
// only the tiles stamped for the next sweep run (see active_tiles /
// mark_out_tiles), and the ring is filled along that list.
template <int MODE, bool FRONTIER>
__global__ void __launch_bounds__(NT, MINBLOCKS) sweep_tma_kernel(const SweepParams p)
{
    using R = Ring<MODE>;
    constexpr bool BF = MODE == MODE_BF || MODE == MODE_BF8;
    static_assert(!FRONTIER || BF, "frontier: Bellman-Ford only");
    constexpr bool LIVE_G = !BF;  // PageRank-type: live global sum

    __shared__ SweepShared<false> sh;
    extern __shared__ __align__(128) unsigned char ring[];  // tile staging ring

    const int c = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    SyncBlock* sb = p.sync;
    unsigned long long bar_target = 0;
    uint32_t* X = (uint32_t*)p.x0;
    const int row_lo = p.cta_row[c], row_hi = p.cta_row[c + 1];
    const int tile_lo = p.cta_tile[c], tile_hi = p.cta_tile[c + 1];

    if (tid == 0) {
        for (int s = 0; s < RING; ++s) mbar_init(&sh.fill_bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        sh.abort = 0;
        sh.nchg = 0;
        for (int k = 0; k < NWARP; ++k) sh.dgw[k] = 0.0f;
    }

    // ---------------- initial values (a grid-stride pass, init_values) ----------------
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

    double T = 1.0;
    if (tid == 0 && !BF) {
        sh.T = ld_relaxed_f64(&sb->T);
        sh.gprev = ld_relaxed_f64(&sb->acc_g[2]);
    }
    __syncthreads();
    if constexpr (!BF) T = (MODE == MODE_ADJ || p.base) ? sh.T : 1.0;  // a uniform teleport sums to 1 exactly
    LiveSum L{};
    if constexpr (LIVE_G) L = live_sum_setup<MODE>(p, T, sh.gprev);
    AdjOffset A{sh.gprev, 0.0, 0.0f, 0.0, 0.0, 0};  // adjoint: sum lambda, deflation offset
    const double tol = (MODE == MODE_ADJ) ? p.tol * T : p.tol;

    // Gathers that take ordinary loads (L1): the CTA's own block with DAG_READ_OWN_L1 (as fresh as L2: only
    // this CTA writes it), every vertex with DAG_READ_CACHED (a view refreshed by the grid barrier, so a value
    // is at most one sweep old, which the stopping rule tolerates: a sweep that changes nothing read fresh values)
    const bool cached = p.read_mode == READ_CACHED;
    const int own_lo = cached ? 0 : row_lo, own_n = cached ? p.n : p.own_l1 ? row_hi - row_lo : 0;
    const uint64_t pol_edge = policy_evict_first();
    const uint64_t pol_vertex = policy_evict_last();
    int it = 0;
    bool converged = false;
    double last_res = 0.0;
    uint32_t qbase = 0;  // ring fills of earlier sweeps (the i-th tile of a sweep is fill qbase + i)
    int edges_done = 0;        // frontier: edges of the tiles this CTA claimed in a shared sweep (thread 0)
    int marks = 0;             // frontier: out-degree sum of this thread's changed rows in the sweep (<= m)
    bool dense = true;         // frontier: this sweep runs every tile

    for (; it < p.max_iters; ++it) {
        const int slot = it % 3;
        // per-thread partial sums in FP32 (few rows each); FP64 from the block reduction on
        float res_part = 0.0f, g_part = 0.0f, dg_part = 0.0f;
        uint32_t carry = Op<MODE>::identity();  // thread 0: partial of the row continuing into the next tile

        // Tiles of this sweep. Own sweeps: the CTA's own range, in order, with the
        // carry of a row passed from tile to tile. Shared sweeps (frontier, after a
        // sweep that changed few rows): the CTAs claim tiles of the sweep's list one
        // at a time, so a thin frontier is spread over all of them; every row
        // write is then an atomicMin (a partial row is as valid a relaxation as a
        // whole one) and own-block L1 reads are off (any CTA may write any row).
        const bool shared = FRONTIER && !dense;
        const int own_n_sweep = (shared && !cached) ? 0 : own_n;
        int next_own = tile_lo;  // own sweeps: the next tile to hand out
        const int list_cnt = shared ? ld_relaxed_i32(&sb->fr_cnt[slot]) : 0;
        if constexpr (FRONTIER) {
            __syncthreads();  // the previous sweep's marks are done with sh.nchg
            if (tid == 0) sh.nchg = 0;
        }
        // thread 0: the tile of ring position q, or -1 when the sweep has no more
        auto pick = [&]() -> int {
            if (!shared) return next_own < tile_hi ? next_own++ : -1;
            const int k = atomicAdd(&sb->fr_head[slot], 1);
            return k < list_cnt ? p.fr_glist[k] : -1;
        };

        // Pipeline: tile t+2's inputs are being copied and tile t+1's gathers are in
        // flight while tile t is walked, scanned and finished.
        uint32_t term[IPT];  // gathered values of the next tile
        long long gs = 0;    // warp 0: one stripe of the live global sum for the next tile
        if (tid == 0) {
            for (int k = 0; k < 2; ++k) {
                const int t = pick();
                sh.tq[(qbase + k) % RING] = t;
                if (t >= 0) issue_fill<MODE>(ring, sh.fill_bar, qbase + k, p, X, t, pol_edge, pol_vertex);
            }
        }
        __syncthreads();  // the first two tiles are known
        if (sh.tq[qbase % RING] >= 0) {
            const TileGeo g0 = tile_geo(p, sh.tq[qbase % RING]);
            if (mbar_wait(&sh.fill_bar[qbase % RING], (qbase / RING) & 1u, p.timeout_ns)) {
                const int* cr = (const int*)(ring + R::OFF_CR) + (qbase % RING) * R::CR_INTS;
                gather_tile(term, cr + g0.col_off(), g0.NB, X, tid, pol_vertex, own_lo, own_n_sweep);
            } else {
                sh.abort = 1;
                atomicCAS(&sb->err, 0, DAG_ERR_BARRIER_TIMEOUT);
#pragma unroll
                for (int k = 0; k < IPT; ++k) term[k] = 0u;
            }
            if constexpr (LIVE_G) {
                if (warp == 0) gs = ld_relaxed_i64(&sb->stripe[lane * GSTRIDE]);
            }
        }

        uint32_t ntl = 0;  // tiles run in this sweep (ring positions used)
        for (;; ++ntl) {
            const uint32_t q = qbase + ntl;
            const int t = sh.tq[q % RING];
            if (t < 0) break;
            const TileGeo g = tile_geo(p, t);
            const int a0 = g.a0, b0 = g.b0, NA = g.NA, NB = g.NB;
            const int* rend = (const int*)(ring + R::OFF_CR) + (q % RING) * R::CR_INTS + g.rend_off();
            // -------- tile t's edge terms into shared memory --------
            {
                const unsigned char* aux = ring + R::OFF_AUX + (q & 1u) * R::AUX_BYTES;
                const int ao = aux_off<MODE>(g);
#pragma unroll
                for (int k = 0; k < IPT; ++k) {
                    const int jj = tid + k * NT;
                    if (jj < NB) sh.val[jj] = edge_term<MODE>(term[k], aux, ao + jj);
                }
                if constexpr (LIVE_G) {
                    if (warp == 0) {  // the tile's global term, formed once
                        const long long G = warp_sum(gs);
                        if (lane == 0) sh.gt = live_term<MODE>(L, G);
                    }
                }
            }
            __syncthreads();  // (A) tile staged; every thread is done with the previous tile
            if constexpr (LIVE_G) flush_dg(sh, sb, c, L.S);  // the previous tile's change of N, one atomic per CTA

            const int t1 = sh.tq[(q + 1) % RING];  // the next tile (known since the previous tile)
            const bool more = t1 >= 0;
            const float gt = LIVE_G ? sh.gt : 0.0f;
            if constexpr (FRONTIER) {
                if (tid == 0 && shared) {
                    carry = Op<MODE>::identity();  // a claimed tile starts afresh
                    edges_done += NB;
                }
            }
            // -------- the copies of the tile after next, the next tile's gathers --------
            if (tid == 0) {
                const int t2 = more ? pick() : -1;
                sh.tq[(q + 2) % RING] = t2;  // the slot of tile i-1, which nobody reads any more
                if (t2 >= 0) issue_fill<MODE>(ring, sh.fill_bar, q + 2, p, X, t2, pol_edge, pol_vertex);
            }
            if (more) {
                const TileGeo g1 = tile_geo(p, t1);
                const uint32_t q1 = q + 1;
                if (mbar_wait(&sh.fill_bar[q1 % RING], (q1 / RING) & 1u, p.timeout_ns)) {
                    const int* cr1 = (const int*)(ring + R::OFF_CR) + (q1 % RING) * R::CR_INTS;
                    gather_tile(term, cr1 + g1.col_off(), g1.NB, X, tid, pol_vertex, own_lo, own_n_sweep);
                } else {
                    sh.abort = 1;
                    atomicCAS(&sb->err, 0, DAG_ERR_BARRIER_TIMEOUT);
#pragma unroll
                    for (int k = 0; k < IPT; ++k) term[k] = 0u;
                }
                if constexpr (LIVE_G) {
                    if (warp == 0) gs = ld_relaxed_i64(&sb->stripe[lane * GSTRIDE]);
                }
            }

            // -------- merge-path walk over this thread's IPT items, block segmented scan --------
            const WalkOut w = walk_tile<MODE, false>(sh, [&](int i) { return rend[i] - b0; }, NA, NB, carry);
            __syncthreads();  // (B) warp run totals visible; sh.tq of the tile after next written
            if (sh.abort) {   // a staging wait ran out (error recorded): drain own copies, leave
                if (tid == 0) {
                    if (more) (void)mbar_wait(&sh.fill_bar[(q + 1) % RING], ((q + 1) / RING) & 1u, p.timeout_ns);
                    if (sh.tq[(q + 2) % RING] >= 0)
                        (void)mbar_wait(&sh.fill_bar[(q + 2) % RING], ((q + 2) / RING) & 1u, p.timeout_ns);
                }
                return;  // the other CTAs' barrier waits end on the recorded error
            }
            const uint32_t E_last = finish_scan<MODE>(sh, w);
            if (tid == 0) {
                if (!shared) {
                    carry = E_last;  // partial of row NA for the next tile
                } else if constexpr (FRONTIER) {
                    if (E_last != Op<MODE>::identity()) {  // the row continuing into another tile: relax it now
                        const int v = a0 + NA;
                        const uint32_t old = atomicMin(X + v, E_last);
                        if (E_last < old) {
                            res_part += 1.0f;
                            p.fr_gchg[atomicAdd(&sb->fr_nchg[slot], 1)] = v;
                            marks += p.fr_orow[v + 1] - p.fr_orow[v];
                        }
                    }
                }
            }
            __syncthreads();  // (C) row sums final

            // -------- epilogue: new values of the rows this tile completed --------
            const uint32_t* old = (const uint32_t*)(ring + R::OFF_OLD) + (q % RING) * R::OLD_INTS + g.old_off();
            const uint32_t* degs = (const uint32_t*)(ring + R::OFF_DEG) + (q % RING) * R::DEG_INTS + g.old_off();
#pragma unroll
            for (int k = 0; k < IPT; ++k) {
                const int r = tid + k * NT;
                if (r >= NA) break;
                const int v = a0 + r;
                if constexpr (FRONTIER) {
                    if (shared) {
                        const uint32_t sum = sh.rowsum[r];
                        const uint32_t prev = atomicMin(X + v, sum);
                        if (sum < prev) {
                            res_part += 1.0f;
                            p.fr_gchg[atomicAdd(&sb->fr_nchg[slot], 1)] = v;
                            marks += p.fr_orow[v + 1] - p.fr_orow[v];
                        }
                        continue;
                    }
                }
                uint32_t xo_bits;
                float dg = 0.0f;
                if (k == 0) {  // the first NT rows' inputs came with the tile
                    xo_bits = old[r];
                    if constexpr (!BF) dg = __uint_as_float(degs[r]);
                } else {
                    xo_bits = ld_relaxed_b32(X + v);
                    if constexpr (!BF) dg = ld_stream_f32(p.degf + v);
                }
                const uint32_t xnew = row_update<MODE>(p, v, sh.rowsum[r], xo_bits, dg, gt, A.off_f, res_part, g_part,
                                                       dg_part);
                if constexpr (FRONTIER)  // the row goes on the CTA's list; its marks are counted at the sweep's end
                    log_changed(p.fr_chg + row_lo, &sh.nchg, xnew < xo_bits, v, epilogue_lanes(NA, k));
                st_relaxed_b32(X + v, xnew);
            }
            if constexpr (LIVE_G) {  // this tile's change of N: one share per warp, added after barrier (A)
                const float s = warp_sum(dg_part);
                dg_part = 0.0f;
                if (lane == 0) sh.dgw[warp] = s;
            }
        }  // tiles
        qbase += ntl;
        if constexpr (LIVE_G) {
            __syncthreads();  // the last tile's shares
            flush_dg(sh, sb, c, L.S);
        }

        // -------- end of sweep: residual, barrier, stopping rule (frontier: tile marks) --------
        if constexpr (FRONTIER) {
            if (!shared) {  // an own sweep's changed rows are on the CTA's list (a shared sweep counted them)
                __syncthreads();
                marks += changed_marks(p.fr_chg + row_lo, sh.nchg, p.fr_orow);
            }
        }
        double res_d = (double)res_part, g_d = FRONTIER ? (double)marks : (double)g_part;  // marks: exact in FP64
        marks = 0;
        block_sum2(sh, res_d, g_d);
        if (tid == 0 && res_d != 0.0) atomicAdd(&sb->acc_res[slot], res_d);
        if (MODE == MODE_ADJ && tid == 0 && g_d != 0.0) atomicAdd(&sb->acc_g[slot], g_d);
        if (FRONTIER && tid == 0) {
            if (g_d != 0.0) atomicAdd(&sb->acc_g[slot], g_d);
            // edges of the tiles run: an own sweep runs all of the CTA's tiles
            const int e = shared ? edges_done : p.tile_nz[tile_hi] - p.tile_nz[tile_lo];
            if (e) atomicAdd((unsigned long long*)&sb->edges, (unsigned long long)e);
            edges_done = 0;
        }
        if (!grid_barrier(sb, p.nblocks, bar_target, p.timeout_ns)) return;
        if (tid == 0) {
            sh.res = ld_relaxed_f64(&sb->acc_res[slot]);
            if (FRONTIER || MODE == MODE_ADJ) sh.gprev = ld_relaxed_f64(&sb->acc_g[slot]);
            if (FRONTIER) sh.cnt[0] = ld_relaxed_i32(&sb->fr_nchg[slot]);
            if (c == 0) {
                const int dead = (it + 2) % 3;  // read by everyone before this barrier
                sb->acc_res[dead] = 0.0;
                sb->acc_g[dead] = 0.0;
                sb->fr_cnt[dead] = 0;
                sb->fr_head[dead] = 0;
                sb->fr_nchg[dead] = 0;
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
        if constexpr (FRONTIER) {
            // sparse next sweep: stamp the tiles the changed rows feed, publish them in one list, run that
            const bool was_shared = shared;
            const int gchg_cnt = sh.cnt[0];
            dense = sh.gprev > FR_SPARSE * (double)p.cta_tile[p.nblocks];
            if (!dense) {
                if (was_shared)
                    mark_out_tiles(p.fr_gchg, gchg_cnt, p.fr_orow, p.fr_otile, p.fr_oend, p.fr_act, it,
                                   c * NWARP + warp, p.nblocks * NWARP);
                else
                    mark_out_tiles(p.fr_chg + row_lo, sh.nchg, p.fr_orow, p.fr_otile, p.fr_oend, p.fr_act, it,
                                   warp, NWARP);
                if (!grid_barrier(sb, p.nblocks, bar_target, p.timeout_ns)) return;
                publish_tiles(sh, p.fr_act, it + 1, tile_lo, tile_hi, p.fr_glist, &sb->fr_cnt[(it + 1) % 3]);
                if (!grid_barrier(sb, p.nblocks, bar_target, p.timeout_ns)) return;
            }
        }
    }

    // ---------------- output (a grid-stride pass, write_output) ----------------
    write_output<MODE>(p, X, A.off_f);
    if (tid == 0 && c == 0) {
        sb->iters = it;
        sb->residual = last_res;
        sb->converged = converged ? 1 : 0;
    }
}

const void* sweep_tma_kernel_ptr(int mode, bool frontier)
{
    switch (mode) {
    case MODE_PR: return (const void*)sweep_tma_kernel<MODE_PR, false>;
    case MODE_PRW: return (const void*)sweep_tma_kernel<MODE_PRW, false>;
    case MODE_ADJ: return (const void*)sweep_tma_kernel<MODE_ADJ, false>;
    case MODE_BF: return frontier ? (const void*)sweep_tma_kernel<MODE_BF, true> : (const void*)sweep_tma_kernel<MODE_BF, false>;
    default: return frontier ? (const void*)sweep_tma_kernel<MODE_BF8, true> : (const void*)sweep_tma_kernel<MODE_BF8, false>;
    }
}

size_t sweep_tma_ring_bytes(int mode)
{
    switch (mode) {
    case MODE_PR: return Ring<MODE_PR>::BYTES;
    case MODE_PRW: return Ring<MODE_PRW>::BYTES;
    case MODE_ADJ: return Ring<MODE_ADJ>::BYTES;
    case MODE_BF: return Ring<MODE_BF>::BYTES;
    default: return Ring<MODE_BF8>::BYTES;
    }
}

}  // namespace dag
