// Frontier Bellman-Ford on warp tiles: the asynchronous sweep of Sec. I with
// the conditionally written updates of Sec. V (DAG_WARP_WORKERS together with
// DAG_SSSP_FRONTIER, dag_sssp / dag_sssp_u8).
//
// Dense sweeps are the warp-worker sweep (sweep_warp.cu): every warp walks
// its run of warp tiles, owns the rows that end in it and finishes a row that
// straddles runs with the bounded look-back over published partials. Each
// warp also keeps the list of its rows that got a smaller distance, and the
// sweep's total of their out-degrees (the tile flags they would set) goes
// through the grid reduction with the residual. When that total is at most
// fr_sparse per warp tile, the sweeps turn sparse: the lowered rows set the
// flag of every warp tile holding one of their out-edges (fr_otile, the in-CSR
// position of each out-edge), and a sparse sweep runs only flagged tiles, in
// tile order (warps claim the tile ids 32 at a time). A tile's flag is taken
// (exchanged for 0) before the tile reads its inputs, and a row a sparse tile
// lowers flags its out-edges' tiles at once, after a fence: a tile further on
// in the same sweep then runs with the new value, and a tile already taken is
// flagged again for the next sweep, so no lowered value goes unpropagated. A
// sparse tile relaxes its rows with atomicMin: a row that the tile holds only
// part of (its first or last one) gets the minimum over that part, which is as
// valid a relaxation as the whole row's (every other in-edge's source kept
// its value since its tile last ran). A sweep that lowers no distance ends the
// solve, as in Sec. IV; one grid barrier per sweep, one more when the sweeps
// turn sparse.
//
// Dense sweeps gather through L2 (relaxed loads) or, with DAG_READ_CACHED,
// with ordinary loads refreshed by every grid barrier (a tile that read a
// value older than a change of the same sweep is flagged by that change);
// sparse sweeps always gather through L2, after the fence that orders them
// behind the flags they took.
#include <algorithm>
#include <climits>
#include <cstdint>

#include "sweep_warp.cuh"

namespace dag {

// Sets to s + 1 the flag of the warp tile of every out-edge of the rows list[first], list[first + stride], ...
// (one warp per row, its lanes over the row's out-edges).
__device__ __forceinline__ void stamp_edge_tiles(const int* list, int cnt, const int* orow, const int* otile, int* act,
                                                 int s, int first, int stride, int lane)
{
    for (int k = first; k < cnt; k += stride) {
        const int v = list[k];
        const int e1 = orow[v + 1];
        for (int e = orow[v] + lane; e < e1; e += 32) act[otile[e]] = s + 1;
    }
}

// ORD: dense sweeps on the CTA's tiles in turn (DAG_WARP_ORDERED), else on each warp's run.
template <int MODE, int WIPT, bool ORD>
__global__ void __launch_bounds__(NT, WMINBLOCKS) sweep_warp_frontier_kernel(const SweepParams p)
{
    static_assert(MODE == MODE_BF || MODE == MODE_BF8, "frontier: Bellman-Ford only");
    constexpr int WTILE = 32 * WIPT;
    using O = Op<MODE>;
    constexpr unsigned FULL = 0xffffffffu;
    (void)WTILE;

    __shared__ WarpShared<32 * WIPT> sh;
    __shared__ int s_cnt;  // ordered dense sweeps: rows on the CTA's list of lowered rows
    const int c = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wl = tid >> 5;
    const int w = c * WWARPS + wl;
    SyncBlock* sb = p.sync;
    unsigned long long bar_target = 0;
    uint32_t* X = (uint32_t*)p.x0;
    const int row_lo = p.cta_row[w], row_hi = p.cta_row[w + 1];
    const int t_lo = p.cta_tile[w], t_hi = p.cta_tile[w + 1];
    int* end = sh.end[wl];
    uint32_t* val = sh.val[wl];
    uint32_t* sum = sh.sum[wl];
    int* own_chg = p.fr_chg + row_lo;  // dense sweeps: this warp's changed rows (its own, so at most row_hi - row_lo)
    // ordered dense sweeps: the CTA's tiles [T0, T1) (its warps' runs together), taken by its warps in turn, and
    // its list of lowered rows (a row split over k of its tiles may appear k times: at most rows + tiles entries)
    const int T0 = p.cta_tile[c * WWARPS], T1 = p.cta_tile[c * WWARPS + WWARPS];
    int* cta_chg = p.fr_gchg + (p.cta_row[c * WWARPS] + T0);
    const bool mid0 = t_lo < t_hi && p.tile_nz[t_lo] > p.rowptr[p.tile_row[t_lo]];
    const bool head = mid0 && row_hi > row_lo;

    {
        double unused_n = 0.0, unused_t = 0.0;
        init_values<MODE>(p, X, unused_n, unused_t);
    }
    if (p.skip_barrier_cta0 && c == 0) return;  // test hook: the others' waits must run out
    if (!grid_barrier(sb, p.nblocks, bar_target, p.timeout_ns)) return;

    const int rmode = p.read_mode == READ_CACHED ? READ_CACHED : READ_COHERENT;
    const uint64_t pol_edge = policy_evict_first();
    const uint64_t pol_vertex = policy_evict_last();
    const double sparse_marks = (double)p.fr_sparse * (double)p.ntiles;
    int it = 0;
    bool converged = false, dense = true;
    double last_res = 0.0;
    int own_cnt = 0;  // rows on own_chg after a dense sweep (warp-uniform)

    for (; it < p.max_iters; ++it) {
        const int slot = it % 3;
        const unsigned stamp = (unsigned)it + 1u;
        float res_part = 0.0f, unused_g = 0.0f, unused_dg = 0.0f;
        long long marks = 0;  // this lane's share of the out-degree sum of the rows lowered in the sweep
        long long edges = 0;  // lane 0: edges of the tiles this warp ran
        bool ok = true;

        if (ORD && dense) {
            // ---------------- dense sweep, ordered: the CTA's tiles, its warps taking them in turn ----------------
            // A row whose in-edges all lie in one tile gets min(old, sum) from that tile alone; a row split over
            // tiles gets each tile's partial with an atomic minimum (as valid a relaxation as the whole row's),
            // so no tile waits for another.
            if (tid == 0) s_cnt = 0;
            __syncthreads();
            WStage<WIPT> nx;
            if (T0 + wl < T1) wfetch<MODE, WIPT>(nx, p, X, T0 + wl, lane, rmode, false, pol_edge, pol_vertex);
            for (int t = T0 + wl; t < T1; t += WWARPS) {
                const int a0 = nx.a0, b0 = nx.b0, NA = nx.NA, NB = nx.NB;
                const bool cont = b0 > nx.rp0;  // the tile starts inside row a0
                const uint32_t pf_xo = nx.xo;
                __syncwarp();
#pragma unroll
                for (int q = 0; q < WIPT; ++q) {
                    const int j = lane + 32 * q;
                    if (j < NB) val[j] = nx.term[q];
                }
                wstage_ends<WIPT>(end, nx, p, lane, pol_vertex);
                if (t + WWARPS < T1)
                    wfetch<MODE, WIPT>(nx, p, X, t + WWARPS, lane, rmode, false, pol_edge, pol_vertex);
                __syncwarp();
                const uint32_t trail = wwalk<MODE, WIPT>(end, val, sum, NA, NB, O::identity(), lane);
                __syncwarp();
                if (lane == 0) edges += NB;
                uint32_t xo_k[WIPT];
                xo_k[0] = pf_xo;
#pragma unroll
                for (int k = 1; k < WIPT; ++k) {
                    const int r = lane + 32 * k;
                    xo_k[k] = r < NA ? ld_weak_b32(X + a0 + r) : 0u;
                }
#pragma unroll
                for (int k = 0; k <= WIPT; ++k) {
                    const int r = lane + 32 * k;
                    if (32 * k > NA) break;  // warp-uniform
                    bool changed = false;
                    const int v = a0 + r;
                    if (r < NA) {
                        const uint32_t sv = sum[r];
                        const uint32_t xo = xo_k[k < WIPT ? k : 0];
                        if (r == 0 && cont) {  // the rest of a row begun in an earlier tile
                            if (sv != INF && sv < xo) changed = sv < atomicMin(X + v, sv);
                        } else if (sv < xo) {  // a whole row: only this tile writes it in a dense sweep
                            st_relaxed_b32(X + v, sv);
                            changed = true;
                        }
                    } else if (r == NA && v < p.n && trail != INF) {  // the start of a row ending in a later tile
                        if (trail < ld_weak_b32(X + v)) changed = trail < atomicMin(X + v, trail);
                    }
                    const unsigned bal = __ballot_sync(FULL, changed);
                    if (bal == 0u) continue;
                    if (changed) res_part += 1.0f;
                    int base = 0;
                    if (lane == 0) base = atomicAdd(&s_cnt, __popc(bal));
                    base = __shfl_sync(FULL, base, 0);
                    if (changed) cta_chg[base + __popc(bal & ((1u << lane) - 1u))] = v;
                }
            }
            __syncthreads();  // the CTA's list is complete
            own_cnt = s_cnt;
            for (int k = wl * 32 + lane; k < own_cnt; k += NT) {
                const int v = cta_chg[k];
                marks += p.fr_orow[v + 1] - p.fr_orow[v];
            }
        } else if (!ORD && dense) {
            // ---------------- dense sweep: the warp's run, in order ----------------
            own_cnt = 0;
            uint32_t carry = O::identity();
            bool head_pending = head;
            uint32_t head_part = O::identity();
            WStage<WIPT> nx;
            if (t_lo < t_hi) wfetch<MODE, WIPT>(nx, p, X, t_lo, lane, rmode, false, pol_edge, pol_vertex);
            for (int t = t_lo; t < t_hi; ++t) {
                const int a0 = nx.a0, b0 = nx.b0, NA = nx.NA, NB = nx.NB;
                const uint32_t pf_xo = nx.xo;
                __syncwarp();
#pragma unroll
                for (int q = 0; q < WIPT; ++q) {
                    const int j = lane + 32 * q;
                    if (j < NB) val[j] = nx.term[q];
                }
                wstage_ends<WIPT>(end, nx, p, lane, pol_vertex);
                if (t + 1 < t_hi) wfetch<MODE, WIPT>(nx, p, X, t + 1, lane, rmode, false, pol_edge, pol_vertex);
                __syncwarp();
                carry = wwalk<MODE, WIPT>(end, val, sum, NA, NB, carry, lane);
                __syncwarp();
                const int skip = (head_pending && NA > 0) ? 1 : 0;  // the run's first row waits for the look-back
                if (skip && lane == 0) head_part = sum[0];
                head_pending = head_pending && NA == 0;
                uint32_t xo_k[WIPT];
                xo_k[0] = pf_xo;
#pragma unroll
                for (int k = 1; k < WIPT; ++k) {
                    const int r = lane + 32 * k;
                    xo_k[k] = r < NA ? ld_weak_b32(X + a0 + r) : 0u;
                }
#pragma unroll
                for (int k = 0; k < WIPT; ++k) {
                    const int r = lane + 32 * k;
                    if (32 * k >= NA) break;  // warp-uniform: no lane has a row in this or a later slot
                    bool changed = false;
                    if (r < NA && !(k == 0 && lane == 0 && skip)) {
                        const uint32_t xnew =
                            row_update<MODE>(p, a0 + r, sum[r], xo_k[k], 0.0f, 0.0f, 0.0f, res_part, unused_g, unused_dg);
                        changed = xnew < xo_k[k];
                        st_relaxed_b32(X + a0 + r, xnew);
                    }
                    const unsigned bal = __ballot_sync(FULL, changed);
                    if (changed) own_chg[own_cnt + __popc(bal & ((1u << lane) - 1u))] = a0 + r;
                    own_cnt += __popc(bal);
                }
            }
            if (lane == 0) edges += (long long)(p.tile_nz[t_hi] - p.tile_nz[t_lo]);
            // the row this run leaves unfinished, and the one it started inside (as in the warp-worker sweep)
            if (lane == 0) st_relaxed_u64(p.wpub + w, ((unsigned long long)stamp << 32) | carry);
            if (head) {
                uint32_t s = __shfl_sync(FULL, head_part, 0);
                for (int k = w - 1; k >= 0; --k) {
                    uint32_t pk = 0u;
                    if (lane == 0) ok = wait_published(p.wpub, k, stamp, sb, p.timeout_ns, &pk);
                    ok = __shfl_sync(FULL, ok, 0) != 0;
                    pk = __shfl_sync(FULL, pk, 0);
                    if (!ok) break;
                    s = O::combine(s, pk);
                    const int tk0 = p.cta_tile[k], tk1 = p.cta_tile[k + 1];
                    const bool k_emits = p.cta_row[k + 1] > p.cta_row[k];
                    const bool k_mid = tk0 >= tk1 || p.tile_nz[tk0] > p.rowptr[p.tile_row[tk0]];
                    if (k_emits || !k_mid) break;
                }
                if (ok) {
                    bool changed = false;
                    if (lane == 0) {
                        const uint32_t xo = ld_weak_b32(X + row_lo);
                        const uint32_t xnew = row_update<MODE>(p, row_lo, s, xo, 0.0f, 0.0f, 0.0f, res_part, unused_g,
                                                               unused_dg);
                        changed = xnew < xo;
                        st_relaxed_b32(X + row_lo, xnew);
                    }
                    changed = __shfl_sync(FULL, changed, 0) != 0;
                    if (changed && lane == 0) own_chg[own_cnt] = row_lo;
                    own_cnt += changed ? 1 : 0;
                }
            }
            __syncwarp();  // the list's entries before the lanes read them
            for (int k = lane; k < own_cnt; k += 32) {
                const int v = own_chg[k];
                marks += p.fr_orow[v + 1] - p.fr_orow[v];
            }
        } else {
            // ---------------- sparse sweep: the flagged tiles, in tile order ----------------
            // Warps claim the tile ids 32 at a time in increasing order; a flagged tile's flag is taken
            // (exchanged for 0) before its inputs are read, so a flag set later by a lowered input is kept for
            // a later claim or the next sweep, and one set earlier is seen with the value that set it.
            unsigned bits = 0u;
            int base = 0;
            auto next_tile = [&]() -> int {
                for (;;) {
                    if (bits) {
                        const int b = __ffs(bits) - 1;
                        bits &= bits - 1u;
                        return base + b;
                    }
                    int b0 = 0;
                    if (lane == 0) b0 = atomicAdd(&sb->fr_head[slot], 32);
                    b0 = __shfl_sync(FULL, b0, 0);
                    if (b0 >= p.ntiles) return -1;
                    base = b0;
                    const int t = b0 + lane;
                    bool mine = false;
                    if (t < p.ntiles && ld_relaxed_i32(p.fr_act + t) != 0) mine = atomicExch(p.fr_act + t, 0) != 0;
                    bits = __ballot_sync(FULL, mine);
                    if (bits) __threadfence();  // the flags' setters' lowered values before this warp's reads
                }
            };
            int t = next_tile();
            WStage<WIPT> nx;
            if (t >= 0) wfetch<MODE, WIPT>(nx, p, X, t, lane, READ_COHERENT, false, pol_edge, pol_vertex);
            while (t >= 0) {
                const int a0 = nx.a0, b0 = nx.b0, NA = nx.NA, NB = nx.NB;
                const uint32_t pf_xo = nx.xo;
                const int tn = next_tile();
                __syncwarp();
#pragma unroll
                for (int q = 0; q < WIPT; ++q) {
                    const int j = lane + 32 * q;
                    if (j < NB) val[j] = nx.term[q];
                }
                wstage_ends<WIPT>(end, nx, p, lane, pol_vertex);
                if (tn >= 0) wfetch<MODE, WIPT>(nx, p, X, tn, lane, READ_COHERENT, false, pol_edge, pol_vertex);
                __syncwarp();
                const uint32_t trail = wwalk<MODE, WIPT>(end, val, sum, NA, NB, O::identity(), lane);
                __syncwarp();
                if (lane == 0) edges += NB;
                // rows of the tile (the first may be partial), then the partial of the row it leaves unfinished;
                // a value read here may be older than the latest (never lower), so only a smaller sum is sent.
                // A lowered row flags the tiles of its out-edges at once (after a fence, so that a warp that
                // takes the flag reads the lowered value).
#pragma unroll
                for (int k = 0; k <= WIPT; ++k) {
                    const int r = lane + 32 * k;
                    if (32 * k > NA) break;  // warp-uniform
                    bool changed = false;
                    const int v = a0 + r;
                    uint32_t cand = INF, seen = 0u;
                    if (r < NA) {
                        cand = sum[r];
                        seen = k == 0 ? pf_xo : ld_relaxed_b32(X + v);
                    } else if (r == NA && v < p.n) {  // the row continuing into the next tile
                        cand = trail;
                        seen = ld_relaxed_b32(X + v);
                    }
                    if (cand != INF && cand < seen) {
                        const uint32_t old = atomicMin(X + v, cand);
                        changed = cand < old;
                    }
                    unsigned bal = __ballot_sync(FULL, changed);
                    if (bal == 0u) continue;
                    __threadfence();
                    if (changed) {
                        res_part += 1.0f;
                        marks += p.fr_orow[v + 1] - p.fr_orow[v];
                    }
                    while (bal) {
                        const int ld = __ffs(bal) - 1;
                        bal &= bal - 1u;
                        const int u = __shfl_sync(FULL, v, ld);
                        const int e1 = p.fr_orow[u + 1];
                        for (int e = p.fr_orow[u] + lane; e < e1; e += 32) st_relaxed_b32(p.fr_act + p.fr_otile[e], 1u);
                    }
                }
                t = tn;
            }
        }

        // ---------------- end of sweep: rows lowered, marks, edges; barrier; stopping rule ----------------
        double res_d = (double)res_part, g_d = (double)marks;  // marks: exact in FP64
        block_sum2(sh, res_d, g_d);
        if (lane == 0 && edges) atomicAdd((unsigned long long*)&sb->edges, (unsigned long long)edges);
        if (tid == 0) {
            if (res_d != 0.0) atomicAdd(&sb->acc_res[slot], res_d);
            if (g_d != 0.0) atomicAdd(&sb->acc_g[slot], g_d);
        }
        if (!grid_barrier(sb, p.nblocks, bar_target, p.timeout_ns)) return;
        if (tid == 0) {
            sh.res = ld_relaxed_f64(&sb->acc_res[slot]);
            sh.gprev = ld_relaxed_f64(&sb->acc_g[slot]);
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
        if (last_res <= 0.0) {
            converged = true;
            ++it;
            break;
        }
        const bool was_dense = dense;
        dense = sh.gprev > sparse_marks;
        if (!dense && was_dense) {
            // into the sparse phase: the rows the dense sweep lowered flag the tiles of their out-edges (a sparse
            // sweep's lowered rows flagged theirs as they went)
            if (ORD)
                stamp_edge_tiles(cta_chg, own_cnt, p.fr_orow, p.fr_otile, p.fr_act, 0, wl, WWARPS, lane);
            else
                stamp_edge_tiles(own_chg, own_cnt, p.fr_orow, p.fr_otile, p.fr_act, 0, 0, 1, lane);
            if (!grid_barrier(sb, p.nblocks, bar_target, p.timeout_ns)) return;
        }
    }

    write_output<MODE>(p, X);
    if (tid == 0 && c == 0) {
        sb->iters = it;
        sb->residual = last_res;
        sb->converged = converged ? 1 : 0;
    }
}

const void* sweep_warp_frontier_kernel_ptr(int mode, int ipt, bool ordered)
{
    if (mode != MODE_BF && mode != MODE_BF8) return nullptr;
#define DAG_WF(I) \
    {(const void*)sweep_warp_frontier_kernel<MODE_BF, I, false>, (const void*)sweep_warp_frontier_kernel<MODE_BF, I, true>, \
     (const void*)sweep_warp_frontier_kernel<MODE_BF8, I, false>, (const void*)sweep_warp_frontier_kernel<MODE_BF8, I, true>}
    static const void* const table[3][4] = {DAG_WF(5), DAG_WF(7), DAG_WF(11)};
#undef DAG_WF
    const int k = ipt == 5 ? 0 : ipt == 7 ? 1 : ipt == 11 ? 2 : -1;
    return k < 0 ? nullptr : table[k][(mode == MODE_BF8 ? 2 : 0) + (ordered ? 1 : 0)];
}

}  // namespace dag
