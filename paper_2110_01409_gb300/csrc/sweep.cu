// Persistent pull-sweep kernels: PageRank (plain and weighted), the PageRank
// adjoint, and Bellman-Ford, each in the synchronous, asynchronous and
// delayed-asynchronous forms. This file holds the register-staged kernel that
// runs the synchronous and delayed forms, and the launch logic of all three;
// the asynchronous form runs the TMA-staged kernel of sweep_tma.cu.
//
// Paper mapping (Blanco, McMillan, Low, HPEC 2021):
//  * worker = one CTA owning a contiguous vertex block balanced by in-degree
//    (Sec. III-A); the block is fixed for the whole solve;
//  * pull update of each owned vertex from its in-neighbours (Sec. III-A);
//  * sync: values go to a second array that is read only after the barrier
//    (Sec. I); async: values are written in place as soon as they are
//    computed (Sec. I); delayed: values go to a shared-memory buffer of the
//    CTA, copied to the global array when it holds >= delta values or the
//    block is finished (Sec. III, III-B); reads always come from the global
//    array (the "global read" form, Sec. III-C);
//  * one grid barrier per iteration (Sec. I) and the stopping rules of Sec. IV.
//
// GPU specifics. The synchronous form reads the previous iterate with
// ordinary loads, which may hit in L1 (no CTA writes that array during the
// sweep). The asynchronous form reads the live array with relaxed gpu-scope
// loads, served by L2 where all CTAs' stores meet, so every value is the
// latest written. The delayed form reads with ordinary loads too: a CTA's
// view of other blocks may then lag until its next flush, where an acquire
// fence refreshes it. The delay delta thus sets both how often a worker
// publishes its values and how often it takes in everyone else's; between
// refreshes the gathers keep their L1 hits, which in-place coherent reads
// give up. The edge stream (colidx, weights) bypasses L1. Rows completed by a
// tile are contiguous, so flushes are coalesced stores of consecutive values.
//
// Per tile: all loads (edge stream, gathers, row ends, the rows' old values)
// are issued in one staging phase into registers; after barrier (A) each
// thread walks its IPT items of the merge path; after barrier (B) each thread
// takes the carry of a row begun by earlier threads from a block segmented
// prefix over the warps' run totals and finishes the rows it ends. A delayed
// flush is copied out between (A) and (B) of the following tile, so it costs
// no barrier. This kernel keeps its shared memory small (about 22 KB per CTA
// plus the delay buffer) because its gathers of the previous iterate or of the
// SM's view of the live array are ordinary loads that live off L1 hits.
#include <algorithm>
#include <climits>
#include <cstdint>
#include <functional>
#include <type_traits>

#include "sweep_common.cuh"

namespace dag {

constexpr int RP = 2;  // epilogue rows per thread whose inputs are loaded with the tile

// Registers of a tile being loaded ahead of use.
template <int MODE>
struct Stage {
    int a0, b0, NA, NB;
    int col[IPT];        // edge stream (source ids)
    uint32_t aux[IPT];   // per-edge weight / value
    uint32_t term[IPT];  // gathered edge terms
    int rend[IPT];       // tile-relative row ends
    uint32_t pfx[RP];    // old values of the first RP * NT rows
    float pfd[RP];       // their out-degrees
    long long gs;        // one stripe of the live global sum (warp 0)
};

// Issues the coalesced loads of tile t (everything except the gathers).
template <int MODE>
__device__ __forceinline__ void stage_issue(Stage<MODE>& st, const SweepParams& p, const uint32_t* xin, int t, int tid,
                                            bool weak, uint64_t pol_edge, uint64_t pol_vertex)
{
    constexpr bool BF = MODE == MODE_BF || MODE == MODE_BF8;
    st.a0 = p.tile_row[t];
    st.b0 = p.tile_nz[t];
    st.NA = p.tile_row[t + 1] - st.a0;
    st.NB = p.tile_nz[t + 1] - st.b0;
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
        const int j = tid + q * NT;
        st.col[q] = 0;
        st.aux[q] = 0;
        if (j < st.NB) {
            st.col[q] = (int)ld_edge_b32(p.colidx + st.b0 + j, pol_edge);
            if constexpr (MODE == MODE_BF) st.aux[q] = ld_edge_b32(p.w + st.b0 + j, pol_edge);
            if constexpr (MODE == MODE_BF8) st.aux[q] = ld_edge_u8(p.w8 + st.b0 + j, pol_edge);
            if constexpr (MODE == MODE_PRW || MODE == MODE_ADJ) st.aux[q] = ld_edge_b32(p.val + st.b0 + j, pol_edge);
        }
    }
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
        const int i = tid + q * NT;
        st.rend[q] = (i < st.NA) ? (int)ld_vertex_b32(p.rowptr + st.a0 + i + 1, pol_vertex) - st.b0 : 0;
    }
#pragma unroll
    for (int k = 0; k < RP; ++k) {
        const int r = tid + k * NT;
        st.pfx[k] = 0u;
        st.pfd[k] = 0.0f;
        if (r < st.NA) {
            st.pfx[k] = weak ? ld_weak_keep_b32(xin + st.a0 + r, pol_vertex)
                             : ld_relaxed_keep_b32(xin + st.a0 + r, pol_vertex);
            if constexpr (!BF) st.pfd[k] = __uint_as_float(ld_vertex_b32(p.degf + st.a0 + r, pol_vertex));
        }
    }
}

// Issues tile t's gathers of the state vector (sync: previous iterate; delayed:
// this SM's view of the live array, or the array in L2 with DAG_READ_COHERENT).
// lbuf/lbase/lcnt: the CTA's own unflushed rows [lbase, lbase + lcnt), read from
// shared memory instead of the global array (local reads, Sec. III-C); lcnt = 0
// reads everything from the global array.
template <int MODE>
__device__ __forceinline__ void stage_gather(Stage<MODE>& st, const uint32_t* xin, int tid, bool weak,
                                             uint64_t pol_vertex, const uint32_t* lbuf, int lbase, int lcnt)
{
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
        const int j = tid + q * NT;
        uint32_t term = 0u;
        if (j < st.NB) {
            const unsigned off = (unsigned)(st.col[q] - lbase);
            const uint32_t xv = off < (unsigned)lcnt ? lbuf[off]
                              : weak ? ld_weak_keep_b32(xin + st.col[q], pol_vertex)
                                     : ld_relaxed_keep_b32(xin + st.col[q], pol_vertex);
            if constexpr (MODE == MODE_BF || MODE == MODE_BF8) term = relax(xv, st.aux[q]);
            else if constexpr (MODE == MODE_PR) term = xv;
            else term = __float_as_uint(__uint_as_float(st.aux[q]) * __uint_as_float(xv));
        }
        st.term[q] = term;
    }
}

// FRONTIER (Bellman-Ford, synchronous form): after a sweep whose changed rows
// feed few tiles (marks <= FR_SPARSE * tiles) only the tiles stamped for the
// next sweep run (see active_tiles / mark_out_tiles), otherwise all do; the
// rows a sweep changes are copied into the other array at the start of the
// next, so both arrays agree on every row a skipped tile leaves alone.
template <int MODE, int VAR, bool FRONTIER>
__global__ void __launch_bounds__(NT, MINBLOCKS) sweep_kernel(const SweepParams p)
{
    using O = Op<MODE>;
    static_assert(!FRONTIER || ((MODE == MODE_BF || MODE == MODE_BF8) && VAR == DAG_SYNC), "frontier: sync BF");
    constexpr bool BF = MODE == MODE_BF || MODE == MODE_BF8;
    constexpr bool SYNC = VAR == DAG_SYNC;
    constexpr bool DELAYED = VAR == DAG_DELAYED;
    constexpr bool LIVE_G = !SYNC && !BF;  // async/delayed PageRank-type: live global sum

    __shared__ SweepShared<true> sh;
    extern __shared__ uint32_t s_buf[];  // delay buffer (DELAYED)

    const int c = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    SyncBlock* sb = p.sync;
    unsigned long long bar_target = 0;
    uint32_t* X0 = (uint32_t*)p.x0;
    uint32_t* X1 = (uint32_t*)p.x1;
    const int row_lo = p.cta_row[c];
    const int tile_lo = p.cta_tile[c], tile_hi = p.cta_tile[c + 1];

    // ---------------- initial values (a grid-stride pass, init_values) ----------------
    {
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
    if (!grid_barrier(sb, p.nblocks, bar_target, p.timeout_ns)) return;

    double T = 1.0;
    if (tid == 0 && !BF) {
        sh.T = ld_relaxed_f64(&sb->T);
        sh.gprev = ld_relaxed_f64(&sb->acc_g[2]);
    }
    __syncthreads();
    if constexpr (!BF) {
        // uniform teleport sums to 1 exactly; a given vector (or ||c||_1) as summed
        T = (MODE == MODE_ADJ || p.base) ? sh.T : 1.0;
    }
    double gprev = BF ? 0.0 : sh.gprev;
    LiveSum L{};
    if constexpr (LIVE_G) L = live_sum_setup<MODE>(p, T, gprev);
    AdjOffset A{gprev, 0.0, 0.0f, 0.0, 0.0, 0};  // adjoint: sum lambda, deflation offset
    const double tol = (MODE == MODE_ADJ) ? p.tol * T : p.tol;

    // sync reads the previous iterate with ordinary loads; async reads the live
    // array coherently (L2); delayed follows p.read_mode
    const bool weak = SYNC || (DELAYED && p.read_mode != READ_COHERENT);
    const uint64_t pol_edge = policy_evict_first();
    const uint64_t pol_vertex = policy_evict_last();
    int buf_first = row_lo, buf_cnt = 0;
    long long flushes = 0;
    long long edges_done = 0;  // frontier: edges of the tiles this CTA ran (thread 0)
    long long marks = 0;       // frontier: out-degree sum of this thread's changed rows in the sweep
    bool dense = true;         // frontier: this sweep runs every tile
    if (tid == 0) sh.nchg = 0;
    int it = 0;
    bool converged = false;
    double last_res = 0.0;

    for (; it < p.max_iters; ++it) {
        const int slot = it % 3;
        const uint32_t* xin = SYNC ? ((it & 1) ? X1 : X0) : X0;
        uint32_t* xout = SYNC ? ((it & 1) ? X0 : X1) : X0;
        // per-thread partial sums in FP32 (few rows each); FP64 from the block reduction on
        float res_part = 0.0f, g_part = 0.0f, dg_part = 0.0f;
        uint32_t carry = O::identity();  // thread 0: partial of the row continuing into the next tile
        bool flush_pending = false;      // delayed: the buffer is copied out during the next tile's walk
        float gterm = 0.0f;
        if constexpr (SYNC && !BF) {
            gterm = (MODE == MODE_ADJ) ? (float)((double)p.g_coef * gprev)
                                       : (float)((double)p.g_coef * (T - gprev));
        }

        // Tiles of this sweep: all of the CTA's, or (frontier) the stamped ones.
        int ntl = tile_hi - tile_lo;
        if constexpr (FRONTIER) {
            // the rows changed in the previous sweep take their new value in this sweep's output too
            for (int k = tid; k < sh.nchg; k += NT) {
                const int v = p.fr_chg[row_lo + k];
                st_weak_b32(xout + v, ld_weak_b32(xin + v));
            }
            __syncthreads();
            if (tid == 0) sh.nchg = 0;
            if (!dense) ntl = active_tiles(sh, p.fr_act, it, tile_lo, tile_hi, p.fr_alist);
        }
        auto tile_at = [&](int i) { return (FRONTIER && !dense) ? p.fr_alist[tile_lo + i] : tile_lo + i; };
        int t_prev = -2;  // frontier: the tile run before, for the carry

        // Software pipeline: while tile t is walked, tile t+1's edge stream,
        // row ends and old values are in flight (issued after barrier A of t)
        // and its gathers too (issued before barrier C of t).
        Stage<MODE> nx;
        if (ntl > 0) {
            stage_issue<MODE>(nx, p, xin, tile_at(0), tid, weak, pol_edge, pol_vertex);
            stage_gather<MODE>(nx, xin, tid, weak, pol_vertex, s_buf, 0, 0);
            if constexpr (LIVE_G) {
                if (warp == 0) nx.gs = ld_relaxed_i64(&sb->stripe[lane * GSTRIDE]);
            }
        }

        for (int i = 0; i <= ntl; ++i) {
            // One pass per tile, plus one extra pass (i == ntl) that only completes a pending flush.
            const bool real = i < ntl;
            const int a0 = real ? nx.a0 : 0, b0 = real ? nx.b0 : 0;
            const int NA = real ? nx.NA : 0, NB = real ? nx.NB : 0;
            uint32_t pf_x[RP];
            float pf_d[RP];
            // -------- tile t into shared memory --------
            if (real) {
#pragma unroll
                for (int q = 0; q < IPT; ++q) {
                    const int jj = tid + q * NT;
                    if (jj < NB) sh.val[jj] = nx.term[q];
                    if (jj < NA) sh.rowend[jj] = nx.rend[q];
                }
#pragma unroll
                for (int k = 0; k < RP; ++k) { pf_x[k] = nx.pfx[k]; pf_d[k] = nx.pfd[k]; }
                if constexpr (LIVE_G) {
                    if (warp == 0) {  // the tile's global term, formed once
                        const long long G = warp_sum(nx.gs);
                        if (lane == 0) sh.gt = live_term<MODE>(L, G);
                    }
                }
            }
            if (tid == 0) sh.rowend[NA] = INT_MAX;
            __syncthreads();  // (A) tile staged; every thread is done with the previous tile

            // -------- delayed: copy out the buffer filled by the previous tiles --------
            if constexpr (DELAYED) {
                if (flush_pending) {
                    for (int k = tid; k < buf_cnt; k += NT) st_relaxed_b32(X0 + buf_first + k, s_buf[k]);
                    if constexpr (!BF) {
                        const float s = warp_sum(dg_part);
                        dg_part = 0.0f;
                        __syncwarp();
                        if (lane == 0 && s != 0.0f) {
                            __threadfence();  // this warp's flushed values before its share of N
                            live_add(sb, c % GSTRIPES, s, L.S);
                        }
                    }
                    if (tid == 0) {
                        // refresh this SM's view: later ordinary loads see what other CTAs published
                        if (p.read_mode == READ_CACHED_REFRESH) asm volatile("fence.acq_rel.gpu;" ::: "memory");
                        ++flushes;
                    }
                    buf_first += buf_cnt;  // every thread keeps the same copy of the buffer state
                    buf_cnt = 0;
                    flush_pending = false;
                }
            }
            if (!real) break;
            const bool more = i + 1 < ntl;
            if constexpr (FRONTIER) {
                const int t = tile_at(i);
                if (tid == 0 && t != t_prev + 1) carry = O::identity();  // the row before was not run
                t_prev = t;
                if (tid == 0) edges_done += NB;
            }
            if (more) stage_issue<MODE>(nx, p, xin, tile_at(i + 1), tid, weak, pol_edge, pol_vertex);
            float gt = gterm;
            if constexpr (LIVE_G) {
                gt = sh.gt;
                if (warp == 0 && more) nx.gs = ld_relaxed_i64(&sb->stripe[lane * GSTRIDE]);
            }

            // -------- merge-path walk over this thread's IPT items, block segmented scan --------
            const WalkOut w = walk_tile<MODE, true>(sh, [&](int i) { return sh.rowend[i]; }, NA, NB, carry);
            __syncthreads();  // (B) warp run totals visible
            const uint32_t E_last = finish_scan<MODE>(sh, w);
            if (tid == 0) carry = E_last;  // partial of row NA for the next tile
            if (more)
                stage_gather<MODE>(nx, xin, tid, weak, pol_vertex, s_buf, buf_first,
                                   (DELAYED && p.local_read) ? buf_cnt : 0);
            __syncthreads();  // (C) row sums final

            // -------- epilogue: new values of the rows this tile completed --------
#pragma unroll
            for (int k = 0; k < IPT; ++k) {
                const int r = tid + k * NT;
                if (r >= NA) break;
                const int v = a0 + r;
                const uint32_t sum = sh.rowsum[r];
                uint32_t xo_bits;
                float dg = 0.0f;
                if (k < RP) {
                    xo_bits = pf_x[k < RP ? k : 0];
                    dg = pf_d[k < RP ? k : 0];
                } else {
                    xo_bits = weak ? ld_weak_b32(xin + v) : ld_relaxed_b32(xin + v);
                    if constexpr (!BF) dg = ld_stream_f32(p.degf + v);
                }
                const uint32_t xnew = row_update<MODE>(p, v, sum, xo_bits, dg, gt, A.off_f, res_part, g_part, dg_part);
                if constexpr (FRONTIER)  // the row goes on the CTA's list; its marks are counted at the sweep's end
                    log_changed(p.fr_chg + row_lo, &sh.nchg, xnew < xo_bits, v, epilogue_lanes(NA, k));
                if constexpr (SYNC) st_weak_b32(xout + v, xnew);
                else if constexpr (DELAYED) s_buf[v - buf_first] = xnew;
                else st_relaxed_b32(xout + v, xnew);
            }
            if constexpr (DELAYED) {
                buf_cnt += NA;
                // flush at delta, at the block end, or (buffer clamped to what fits) when the next tile might not fit
                if (buf_cnt >= p.delta || i == ntl - 1 || (p.buf_clamped && buf_cnt > p.buf_cap - TILE))
                    flush_pending = true;
            }
        }  // tiles

        if constexpr (DELAYED) {
            buf_first = row_lo;
            buf_cnt = 0;
        }

        // -------- end of sweep: residual, barrier, stopping rule (frontier: tile marks) --------
        if constexpr (FRONTIER) {
            __syncthreads();  // the CTA's list of changed rows is complete
            marks += changed_marks(p.fr_chg + row_lo, sh.nchg, p.fr_orow);
        }
        double res_d = (double)res_part, g_d = FRONTIER ? (double)marks : (double)g_part;  // marks: exact in FP64
        marks = 0;
        block_sum2(sh, res_d, g_d);
        if (tid == 0) {
            if (res_d != 0.0) atomicAdd(&sb->acc_res[slot], res_d);
            if ((FRONTIER || (SYNC && !BF) || MODE == MODE_ADJ) && g_d != 0.0) atomicAdd(&sb->acc_g[slot], g_d);
            if (FRONTIER && edges_done) atomicAdd((unsigned long long*)&sb->edges, (unsigned long long)edges_done);
            edges_done = 0;
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
        if constexpr (FRONTIER) {
            // sparse next sweep: stamp the tiles the changed rows feed, publish, run only those
            dense = gprev > FR_SPARSE * (double)p.cta_tile[p.nblocks];
            if (!dense) {
                mark_out_tiles(p.fr_chg + row_lo, sh.nchg, p.fr_orow, p.fr_otile, p.fr_oend, p.fr_act, it, warp,
                               NWARP);
                if (!grid_barrier(sb, p.nblocks, bar_target, p.timeout_ns)) return;
            }
        }
    }

    // ---------------- output (a grid-stride pass, write_output) ----------------
    {
        const uint32_t* xf = SYNC ? ((it & 1) ? X1 : X0) : X0;
        write_output<MODE>(p, xf, A.off_f);
    }
    if (tid == 0) {
        if (flushes) atomicAdd((unsigned long long*)&sb->flushes, (unsigned long long)flushes);
        if (c == 0) {
            sb->iters = it;
            sb->residual = last_res;
            sb->converged = converged ? 1 : 0;
        }
    }
}

using KernelFn = void (*)(const SweepParams);

// The kernel a solve of (mode, variant) runs; frontier: the Bellman-Ford
// kernels that run only the tiles whose inputs changed (sync and async forms).
static KernelFn kernel_for(int mode, int variant, bool frontier)
{
    const bool bf = mode == MODE_BF || mode == MODE_BF8;
    if (variant == DAG_ASYNC) return (KernelFn)sweep_tma_kernel_ptr(mode, frontier && bf);
    if (frontier && bf && variant == DAG_SYNC)
        return mode == MODE_BF ? sweep_kernel<MODE_BF, DAG_SYNC, true> : sweep_kernel<MODE_BF8, DAG_SYNC, true>;
    static const KernelFn table[5][2] = {
        {sweep_kernel<MODE_PR, DAG_SYNC, false>, sweep_kernel<MODE_PR, DAG_DELAYED, false>},
        {sweep_kernel<MODE_PRW, DAG_SYNC, false>, sweep_kernel<MODE_PRW, DAG_DELAYED, false>},
        {sweep_kernel<MODE_ADJ, DAG_SYNC, false>, sweep_kernel<MODE_ADJ, DAG_DELAYED, false>},
        {sweep_kernel<MODE_BF, DAG_SYNC, false>, sweep_kernel<MODE_BF, DAG_DELAYED, false>},
        {sweep_kernel<MODE_BF8, DAG_SYNC, false>, sweep_kernel<MODE_BF8, DAG_DELAYED, false>},
    };
    return table[mode][variant == DAG_DELAYED ? 1 : 0];
}

// The sweep kernel of (mode, variant), for launches that build their own
// parameters (the allocation-free entry point).
const void* sweep_kernel_ptr(int mode, int variant) { return (const void*)kernel_for(mode, variant, false); }

size_t sweep_ring_bytes(int mode, int variant) { return variant == DAG_ASYNC ? sweep_tma_ring_bytes(mode) : 0; }

// Without a preference the driver may keep whatever L1/shared split an earlier
// kernel needed (up to the largest shared share), which leaves L1 small and
// makes a sweep's speed depend on what ran before it.
int set_l1_carveout(const void* k, int device, int threads, size_t static_smem, size_t dyn, int per_sm)
{
    int max_sm = 0, reserved = 0;
    DAG_CUDA(cudaDeviceGetAttribute(&max_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device));
    DAG_CUDA(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, device));
    const size_t need = (size_t)per_sm * (static_smem + dyn + (size_t)reserved);
    int pct = max_sm > 0 ? (int)((need * 100 + (size_t)max_sm - 1) / (size_t)max_sm) : 100;
    pct = pct < 1 ? 1 : (pct > 100 ? 100 : pct);
    DAG_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, pct));
    int got = 0;
    DAG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&got, k, threads, dyn));
    if (got < per_sm) DAG_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    return DAG_OK;
}

// CTAs of a (mode, variant) sweep that fit on the GPU at once, with each kernel
// such a solve may run (plain, and frontier for Bellman-Ford) configured for
// that residency: dynamic shared memory and L1/shared carveout.
int max_workers(dag_plan* plan, int mode, int variant, int buf_cap_elems, int* out)
{
    const void* ks[2] = {(const void*)kernel_for(mode, variant, false), (const void*)kernel_for(mode, variant, true)};
    const int nk = ks[1] != ks[0] ? 2 : 1;
    size_t dyn = sweep_ring_bytes(mode, variant) + ((variant == DAG_DELAYED) ? (size_t)buf_cap_elems * 4 : 0);
    int max_dyn = 0;
    DAG_CUDA(cudaDeviceGetAttribute(&max_dyn, cudaDevAttrMaxSharedMemoryPerBlockOptin, plan->device));
    cudaFuncAttributes fa{};
    int per_sm = INT_MAX;
    for (int i = 0; i < nk; ++i) {
        cudaFuncAttributes fi;
        DAG_CUDA(cudaFuncGetAttributes(&fi, ks[i]));
        if (dyn + fi.sharedSizeBytes > (size_t)max_dyn)
            return set_error(DAG_ERR_INVALID, "delta too large: the delay buffer does not fit in shared memory");
        if (i == 0 || fi.sharedSizeBytes > fa.sharedSizeBytes) fa = fi;
        DAG_CUDA(cudaFuncSetAttribute(ks[i], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
        DAG_CUDA(cudaFuncSetAttribute(ks[i], cudaFuncAttributePreferredSharedMemoryCarveout, 100));
        int ps = 0;
        DAG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, ks[i], NT, dyn));
        per_sm = std::min(per_sm, ps);
    }
    if (per_sm < 1) return set_error(DAG_ERR_INVALID, "sweep kernel cannot be resident with this delta");
    if (variant == DAG_ASYNC) {
        // The TMA kernel's streams and coherent gathers bypass L1, but its own-block gathers and
        // epilogue loads still use it: keep the CTAs' shared memory within the share that leaves
        // 32 KB of the opt-in maximum to L1 (about 60 KB of L1 on this part), which fits four CTAs
        // of the one-byte-weight and plain PageRank rings and three of the four-byte ones (with
        // four of those, L1 drops under 30 KB and the sweep slowed by 25%).
        int max_sm = 0, reserved = 0;
        DAG_CUDA(cudaDeviceGetAttribute(&max_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, plan->device));
        DAG_CUDA(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, plan->device));
        const size_t per_cta = fa.sharedSizeBytes + dyn + (size_t)reserved;
        const size_t budget = max_sm > (32 << 10) ? (size_t)max_sm - (32 << 10) : (size_t)max_sm;
        while (per_sm > 1 && (size_t)per_sm * per_cta > budget) --per_sm;
    }
    for (int i = 0; i < nk; ++i) {
        const int rc = set_l1_carveout(ks[i], plan->device, NT, fa.sharedSizeBytes, dyn, per_sm);
        if (rc) return rc;
    }
    *out = per_sm * plan->num_sms;
    return DAG_OK;
}

// Launch shape of a sweep: CTA count and delay-buffer capacity. A delayed
// sweep's buffer holds at most min(delta - 1 + TILE, rows of the largest block)
// values (a flush empties it once it reaches delta after a tile), and at most
// what fits in shared memory beside the kernel's static share (then it is
// clamped: flushed when the next tile might not fit). Fewer CTAs mean longer
// blocks, so the shape is settled by a short fixed-point loop; `partition`
// builds the static partition of Sec. III-A for a CTA count and returns its
// largest block's row count.
int settle_shape(dag_plan* plan, int mode, int variant, int delta,
                 const std::function<int(int nblocks, int* max_rows)>& partition, int* nb_out, int* cap_out,
                 int* clamped_out)
{
    int nb = 0;
    int rc = max_workers(plan, mode, variant, 0, &nb);
    if (rc) return rc;
    if (plan->worker_cap > 0 && nb > plan->worker_cap) nb = plan->worker_cap;
    int cap = 0, clamped = 0;
    long long max_cap = 0;  // largest buffer (values) one CTA can hold beside its static shared memory
    {
        int max_dyn = 0;
        cudaFuncAttributes fa;
        DAG_CUDA(cudaDeviceGetAttribute(&max_dyn, cudaDevAttrMaxSharedMemoryPerBlockOptin, plan->device));
        DAG_CUDA(cudaFuncGetAttributes(&fa, sweep_kernel_ptr(mode, variant)));
        max_cap = ((long long)max_dyn - (long long)fa.sharedSizeBytes - (long long)sweep_ring_bytes(mode, variant)) / 4;
    }
    bool settled = false;  // CTAs per SM only fall (4, 3, 2, 1), so a few passes settle the shape
    for (int iter = 0; iter < 6 && !settled; ++iter) {
        int max_rows = 0;
        rc = partition(nb, &max_rows);
        if (rc) return rc;
        settled = true;
        if (variant != DAG_DELAYED) break;
        const long long want = std::min((long long)delta - 1 + TILE, (long long)max_rows);
        const long long need = std::min(want, max_cap);  // a larger buffer does not fit: it flushes when full
        clamped = need < want ? 1 : 0;
        cap = (int)(need < 1 ? 1 : need);
        int nb2 = 0;
        rc = max_workers(plan, mode, variant, cap, &nb2);
        if (rc) return rc;
        if (nb2 < nb) {
            nb = nb2;
            settled = false;
        }
    }
    if (!settled) return set_error(DAG_ERR_INVALID, "sweep launch shape did not settle");
    *nb_out = nb;
    *cap_out = cap;
    *clamped_out = clamped;
    return DAG_OK;
}

// Launch shape and the plan's cached partition for it (a delayed sweep with
// delta below a tile's items gets tiles of at most delta rows).
int sweep_shape(dag_plan* plan, int mode, int variant, int delta, int* nb_out, int* cap_out, Partition** part_out,
                cudaStream_t s, int* clamped_out)
{
    Partition* part = nullptr;
    int clamped = 0;
    auto build = [&](int nb, int* max_rows) {
        const int rc = get_partition(plan, nb, &part, s, delayed_row_cap(variant, delta));
        if (rc == DAG_OK) *max_rows = part->max_rows;
        return rc;
    };
    const int rc = settle_shape(plan, mode, variant, delta, build, nb_out, cap_out, &clamped);
    if (rc) return rc;
    *part_out = part;
    if (clamped_out) *clamped_out = clamped;
    return DAG_OK;
}

int launch_sweep(dag_plan* plan, int mode, int variant, int delta, SweepParams& p, cudaStream_t s,
                 int* out_nblocks)
{
    if (p.warp) return launch_warp_sweep(plan, mode, variant, delta, p, s, out_nblocks);
    int nb = 0, cap = 0, clamped = 0;
    Partition* part = nullptr;
    int rc = sweep_shape(plan, mode, variant, delta, &nb, &cap, &part, s, &clamped);
    if (rc) return rc;
    p.nblocks = nb;
    p.delta = (variant == DAG_DELAYED) ? delta : 0;
    p.buf_cap = cap;
    p.buf_clamped = clamped;
    p.cta_row = part->cta_row;
    p.cta_tile = part->cta_tile;
    p.tile_row = part->tile_row;
    p.tile_nz = part->tile_nz;
    p.sync = plan->sync;
    p.timeout_ns = plan->timeout_ns;
    p.skip_barrier_cta0 = 0;
    p.stall_fill = 0;
    if (plan->stall_staging_once && variant == DAG_ASYNC) {
        p.stall_fill = 1;
        p.timeout_ns = plan->skip_timeout_ns;
        plan->stall_staging_once = 0;
    }
    if (plan->skip_barrier_once) {
        p.skip_barrier_cta0 = 1;
        p.timeout_ns = plan->skip_timeout_ns;
        plan->skip_barrier_once = 0;
    }
    if (p.frontier) {
        const int frc = frontier_maps(plan, part, s);
        if (frc) return frc;
        p.fr_orow = plan->fr_orow;
        p.fr_otile = part->fr_otile;
        p.fr_oend = part->fr_oend;
        p.fr_act = part->fr_act;
        p.fr_alist = part->fr_alist;
        p.fr_chg = part->fr_chg;
        p.fr_glist = part->fr_glist;
        p.fr_gchg = part->fr_gchg;
        DAG_CUDA(cudaMemsetAsync(part->fr_act, 0, (size_t)std::max(part->tiles, 1) * sizeof(int), s));
    }
    // the asynchronous form's tile copies are TMA bulk copies from 16-byte boundaries of these arrays
    for (const void* a : {(const void*)p.rowptr, (const void*)p.colidx, (const void*)p.w, (const void*)p.w8,
                          (const void*)p.val, (const void*)p.degf, (const void*)p.x0, (const void*)p.x1})
        if (((uintptr_t)a & 15u) != 0)
            return set_error(DAG_ERR_INVALID, "graph, weight and state arrays must be 16-byte aligned");
    DAG_CUDA(cudaMemsetAsync(plan->sync, 0, sizeof(SyncBlock), s));
    KernelFn k = kernel_for(mode, variant, p.frontier != 0);
    void* args[] = {(void*)&p};
    size_t dyn = sweep_ring_bytes(mode, variant) + ((variant == DAG_DELAYED) ? (size_t)cap * 4 : 0);
    DAG_CUDA(cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    DAG_CUDA(cudaLaunchCooperativeKernel((const void*)k, dim3(nb), dim3(NT), args, dyn, s));
    *out_nblocks = nb;
    return DAG_OK;
}

}  // namespace dag
