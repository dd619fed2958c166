// Device pieces shared by the two sweep kernels (sweep.cu: register-staged
// tiles, used by the synchronous and delayed forms; sweep_tma.cu: TMA-staged
// tiles, used by the asynchronous form): the per-mode reduction, the
// Bellman-Ford relaxation, block reductions, the merge-path walk of one tile
// with its block segmented scan, and the row update of PageRank (Sec. IV-A),
// its adjoint and Bellman-Ford.
#pragma once

#include <climits>

#include "dag_internal.cuh"

namespace dag {

template <int MODE>
struct Op;
template <>
struct Op<MODE_PR> {
    static __device__ __forceinline__ uint32_t identity() { return 0u; }  // +0.0f
    static __device__ __forceinline__ uint32_t combine(uint32_t a, uint32_t b)
    {
        return __float_as_uint(__uint_as_float(a) + __uint_as_float(b));
    }
};
template <>
struct Op<MODE_PRW> : Op<MODE_PR> {};
template <>
struct Op<MODE_ADJ> : Op<MODE_PR> {};
template <>
struct Op<MODE_BF> {
    static __device__ __forceinline__ uint32_t identity() { return INF; }
    static __device__ __forceinline__ uint32_t combine(uint32_t a, uint32_t b) { return a < b ? a : b; }
};
template <>
struct Op<MODE_BF8> : Op<MODE_BF> {};

// dist_u + w, INF when dist_u is INF; a finite sum that would reach INF stays
// finite at INF - 1 (cannot happen for n * 255 < 2^32).
__device__ __forceinline__ uint32_t relax(uint32_t du, uint32_t w)
{
    if (du == INF) return INF;
    uint32_t s = du + w;
    return (s < du || s == INF) ? INF - 1u : s;
}

// Shared memory of one sweep CTA. ROWEND: the tile's row ends live here (the
// register-staged kernel); the TMA kernel reads them from its staging ring.
template <bool ROWEND>
struct SweepShared {
    uint32_t val[TILE];                  // edge terms of the tile
    int rowend[ROWEND ? TILE + 1 : 1];   // tile-relative row end offsets (+ sentinel)
    uint32_t rowsum[TILE];               // per-row reduction of the tile
    int wkey[NWARP];                     // row in progress after each warp's last lane
    int wfirst[NWARP];                   // row in progress after each warp's first lane
    uint32_t wval[NWARP];                // warp-local inclusive run total at the last lane
    double red0[NWARP];
    double red1[NWARP];
    float gt;                            // the tile's global (dangling) term from the live sum
    int abort;                           // a bounded wait of this CTA ran out (TMA kernel)
    int nchg;                            // frontier: rows of this CTA changed in the sweep
    int cnt[NWARP];                      // frontier: per-warp counts of the active-tile scan
    int tq[RING];                        // TMA kernel: the tile of each ring slot (-1: none)
    float dgw[NWARP];                    // TMA kernel: the warps' shares of a tile's change of N
    double res;                          // broadcast of the sweep residual
    double gprev;                        // broadcast of the previous sweep's global sum
    double T;                            // broadcast of the teleport total / ||c||_1
    alignas(8) unsigned long long fill_bar[RING];  // staging-ring mbarriers (TMA kernel)
};

// Block sum of two doubles; the result is valid in thread 0.
template <class SH>
__device__ __forceinline__ void block_sum2(SH& sh, double& a, double& b)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    a = warp_sum(a);
    b = warp_sum(b);
    if (lane == 0) { sh.red0[warp] = a; sh.red1[warp] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        a = 0.0; b = 0.0;
        for (int k = 0; k < NWARP; ++k) { a += sh.red0[k]; b += sh.red1[k]; }
    }
    __syncthreads();
}

// A thread's part of one tile's merge path (Merrill & Garland): IPT items from
// diagonal tid * IPT, rows 0..NA-1 and edges 0..NB-1 of the tile, row ends from
// rowend(i) (tile-relative, i < NA; with SENTINEL, rowend(NA) is INT_MAX too,
// which saves a compare per step). Rows it ends get their partial in
// sh.rowsum; the row in progress after its last item is (key, sv) after the
// warp-level segmented scan, whose warp summaries go to sh.wkey / wval / wfirst.
// The caller places barrier (B) after this.
struct WalkOut {
    int i_start;  // first row this thread touches
    int key;      // row in progress after its last item
    uint32_t sv;  // warp-inclusive run total of that row
    bool emitted; // it ended at least one row
};

template <int MODE, bool SENTINEL, class SH, class RE>
__device__ __forceinline__ WalkOut walk_tile(SH& sh, const RE& rowend, int NA, int NB, uint32_t carry)
{
    using O = Op<MODE>;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int L = NA + NB;
    const int k0 = min(tid * IPT, L);
    int lo = max(0, k0 - NB), hi = min(k0, NA);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (rowend(mid) <= k0 - 1 - mid) lo = mid + 1;
        else hi = mid;
    }
    WalkOut w;
    int i = lo, j = k0 - lo;
    w.i_start = i;
    w.emitted = false;
    uint32_t acc = (tid == 0) ? carry : O::identity();
    int re = (SENTINEL || i < NA) ? rowend(i) : INT_MAX;
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
        if (k0 + q < L) {
            if (re <= j) {
                sh.rowsum[i] = acc;
                w.emitted = true;
                acc = O::identity();
                ++i;
                re = (SENTINEL || i < NA) ? rowend(i) : INT_MAX;
            } else {
                acc = O::combine(acc, sh.val[j]);
                ++j;
            }
        }
    }
    // segmented scan of (row in progress, partial) within the warp
    w.key = i;
    uint32_t sv = acc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t ov = __shfl_up_sync(0xffffffffu, sv, o);
        const int ok = __shfl_up_sync(0xffffffffu, w.key, o);
        if (lane >= o && ok == w.key) sv = O::combine(sv, ov);
    }
    w.sv = sv;
    if (lane == 31) { sh.wkey[warp] = w.key; sh.wval[warp] = sv; }
    if (lane == 0) sh.wfirst[warp] = w.key;
    return w;
}

// After barrier (B): the carry of a row begun by earlier threads, from a
// segmented scan over the warps' run totals (in every warp), added to the
// first row this thread ended. Returns the partial of the row that continues
// into the next tile (the same value in every thread).
template <int MODE, class SH>
__device__ __forceinline__ uint32_t finish_scan(SH& sh, const WalkOut& w)
{
    using O = Op<MODE>;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t E;  // run total ending at warp w's last lane, over all earlier warps
    {
        const int wl = lane < NWARP ? lane : NWARP - 1;
        const int wk = sh.wkey[wl];
        const bool head = lane == 0 || sh.wfirst[wl] != wk || sh.wkey[wl > 0 ? wl - 1 : 0] != wk;
        E = sh.wval[wl];
        int hd = head ? 1 : 0;
#pragma unroll
        for (int o = 1; o < NWARP; o <<= 1) {
            const uint32_t oe = __shfl_up_sync(0xffffffffu, E, o);
            const int oh = __shfl_up_sync(0xffffffffu, hd, o);
            if (lane >= o && !hd) E = O::combine(E, oe);
            if (lane >= o) hd |= oh;
        }
    }
    const uint32_t E_prev = __shfl_sync(0xffffffffu, E, warp > 0 ? warp - 1 : 0);
    const int key_prev = warp > 0 ? sh.wkey[warp - 1] : -1;
    const int k_first = __shfl_sync(0xffffffffu, w.key, 0);
    const uint32_t pre = (warp > 0 && key_prev == k_first) ? E_prev : O::identity();
    const uint32_t S = (w.key == k_first) ? O::combine(w.sv, pre) : w.sv;
    uint32_t cin = __shfl_up_sync(0xffffffffu, S, 1);
    if (lane == 0) cin = (warp > 0) ? E_prev : O::identity();
    if (tid > 0 && w.emitted) sh.rowsum[w.i_start] = O::combine(sh.rowsum[w.i_start], cin);
    return __shfl_sync(0xffffffffu, E, NWARP - 1);  // whole warp takes part
}

// ---------------------------------------------------------------------------
// Frontier Bellman-Ford (tiles that run only when an input changed). Every
// sweep counts the tile marks its changed rows would cause (their out-degree
// sum). When that is at most FR_SPARSE per tile, each CTA stamps s + 1 on the
// tiles from every out-edge of its changed rows to the tile ending that edge's
// target row, an extra grid barrier publishes the stamps, and sweep s + 1 runs
// only the tiles with act[t] == s + 1; otherwise (changes that reach nearly
// every tile anyway) sweep s + 1 runs every tile and nothing is marked.
// Sweep 0 runs every tile.
// ---------------------------------------------------------------------------
constexpr double FR_SPARSE = 4.0;  // measured: below ~5 marks per tile, tiles start to be skipped

// This CTA's tiles that run in sweep s, in order, into alist[tile_lo ...];
// returns their count (the same in every thread).
template <class SH>
__device__ __forceinline__ int active_tiles(SH& sh, const int* act, int s, int tile_lo, int tile_hi, int* alist)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int total = 0;
    for (int base = tile_lo; base < tile_hi; base += NT) {
        const int t = base + tid;
        const bool on = t < tile_hi && act[t] == s;
        const unsigned bal = __ballot_sync(0xffffffffu, on);
        if (lane == 0) sh.cnt[warp] = __popc(bal);
        __syncthreads();
        int before = 0, all = 0;
#pragma unroll
        for (int k = 0; k < NWARP; ++k) {
            before += k < warp ? sh.cnt[k] : 0;
            all += sh.cnt[k];
        }
        if (on) alist[tile_lo + total + before + __popc(bal & ((1u << lane) - 1u))] = t;
        total += all;
        __syncthreads();  // the list is complete and sh.cnt free again
    }
    return total;
}

// Stamps s + 1 on the tiles that the rows in chg[0 .. nchg) feed: one warp per
// changed row (rows first, first + stride, ...), its lanes over the row's
// out-edges. A CTA's own list: first = warp, stride = NWARP; a list shared by
// the grid: first = blockIdx * NWARP + warp, stride = gridDim * NWARP.
__device__ __forceinline__ void mark_out_tiles(const int* chg, int nchg, const int* orow, const int* otile,
                                               const int* oend, int* act, int s, int first, int stride)
{
    const int lane = threadIdx.x & 31;
    for (int k = first; k < nchg; k += stride) {
        const int v = chg[k];
        const int e1 = orow[v + 1];
        for (int e = orow[v] + lane; e < e1; e += 32) {
            const int t1 = oend[e];
            for (int t = otile[e]; t <= t1; ++t) act[t] = s + 1;
        }
    }
}

// The lanes of this warp whose epilogue row tid + k * NT is below NA (a
// prefix of the warp; the caller's lane is one of them).
__device__ __forceinline__ unsigned epilogue_lanes(int NA, int k)
{
    const int rem = NA - ((int)threadIdx.x & ~31) - k * NT;
    return rem >= 32 ? 0xffffffffu : (1u << rem) - 1u;
}

// Appends row v to the CTA's list of changed rows when `changed` (one shared
// atomic per warp; the order within the list is free). Every lane of `lanes`
// calls it.
__device__ __forceinline__ void log_changed(int* list, int* cnt, bool changed, int v, unsigned lanes)
{
    const int lane = threadIdx.x & 31;
    const unsigned bal = __ballot_sync(lanes, changed);
    if (bal == 0u) return;
    const int leader = __ffs(bal) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(cnt, __popc(bal));
    base = __shfl_sync(lanes, base, leader);
    if (changed) list[base + __popc(bal & ((1u << lane) - 1u))] = v;
}

// This thread's share of the out-degree sum of the rows in list[0 .. cnt)
// (the tile marks they would cause), read once at the end of a sweep so that
// the loads are all in flight together instead of in each tile's epilogue.
__device__ __forceinline__ int changed_marks(const int* list, int cnt, const int* orow)
{
    int s = 0;
    for (int k = threadIdx.x; k < cnt; k += NT) {
        const int v = list[k];
        s += orow[v + 1] - orow[v];
    }
    return s;
}

// Appends this CTA's tiles stamped s to the grid's list glist[0 .. *gcnt)
// (one atomic per chunk of NT tiles; the order within the list is free).
template <class SH>
__device__ __forceinline__ void publish_tiles(SH& sh, const int* act, int s, int tile_lo, int tile_hi, int* glist,
                                              int* gcnt)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int base = tile_lo; base < tile_hi; base += NT) {
        const int t = base + tid;
        const bool on = t < tile_hi && act[t] == s;
        const unsigned bal = __ballot_sync(0xffffffffu, on);
        if (lane == 0) sh.cnt[warp] = __popc(bal);
        __syncthreads();
        int before = 0, all = 0;
#pragma unroll
        for (int k = 0; k < NWARP; ++k) {
            before += k < warp ? sh.cnt[k] : 0;
            all += sh.cnt[k];
        }
        __syncthreads();  // everyone has read sh.cnt
        if (tid == 0) sh.cnt[0] = all ? atomicAdd(gcnt, all) : 0;
        __syncthreads();
        if (on) glist[sh.cnt[0] + before + __popc(bal & ((1u << lane) - 1u))] = t;
        __syncthreads();  // sh.cnt free again
    }
}

// ---------------------------------------------------------------------------
// Live global sum N of the asynchronous and delayed sweeps (PageRank: the mass
// on rows with out-edges, so that T - N is the dangling mass every row
// receives, Sec. IV-A; adjoint: the sum of lambda), read by every tile. It is
// kept in 64-bit fixed point with unit 2^-S: the stripes hold its change since
// the start of the solve, added with integer atomics, and a reader sums them
// with integer shuffles. No tile does FP64 arithmetic then (FP64 issues at a
// small fraction of the FP32 rate on this part), and the sum does not depend
// on the order in which the adds land. S is chosen once per solve so that the
// bound 4 T / (1 - d) on |N| stays below 2^62 units.
// ---------------------------------------------------------------------------
struct LiveSum {
    int S;           // the unit is 2^-S
    long long base;  // PageRank: T - N(0); adjoint: N(0); in units
    float scale;     // g_coef * 2^-S
};

// T: the teleport total (adjoint: ||c||_1); N0: N at the start of the solve.
template <int MODE>
__device__ __forceinline__ LiveSum live_sum_setup(const SweepParams& p, double T, double N0)
{
    LiveSum L;
    int ex;
    (void)frexp(4.0 * fmax(T, 1e-30) / fmax(1.0 - (double)p.d, 1e-3), &ex);  // the bound is below 2^ex
    L.S = min(90, 62 - ex);
    const double unit = ldexp(1.0, L.S);
    L.base = __double2ll_rn(((MODE == MODE_ADJ) ? N0 : T - N0) * unit);
    L.scale = (float)((double)p.g_coef / unit);
    return L;
}

// f in units of 2^-S, rounded to nearest (ties away from zero), by integer
// operations on its bits: |f| = m * 2^(e - 150) for the 24-bit significand m.
// Subnormals (below any unit used here) give 0.
__device__ __forceinline__ long long live_units(float f, int S)
{
    const uint32_t b = __float_as_uint(f);
    const int e = (int)((b >> 23) & 0xffu);
    if (e == 0) return 0;
    const long long m = (long long)((b & 0x7fffffu) | 0x800000u);
    const int sh = e - 150 + S;
    long long r;
    if (sh >= 0) r = sh < 39 ? m << sh : (1LL << 62);  // past the bound: saturate
    else r = sh >= -24 ? ((m >> (-sh - 1)) + 1) >> 1 : 0;
    return (b >> 31) ? -r : r;
}

// Adds f (a change of N) to stripe k.
__device__ __forceinline__ void live_add(SyncBlock* sb, int k, float f, int S)
{
    const long long u = live_units(f, S);
    if (u != 0) atomicAdd((unsigned long long*)&sb->stripe[k * GSTRIDE], (unsigned long long)u);
}

// The global term of a tile from the stripe sum G (the change of N): PageRank
// g_coef (T - N), adjoint g_coef N. The 64-bit value is converted as
// hi * 2^32 + lo (two exact-or-rounded 32-bit conversions, one rounded sum).
template <int MODE>
__device__ __forceinline__ float live_term(const LiveSum& L, long long G)
{
    const long long v = (MODE == MODE_ADJ) ? L.base + G : L.base - G;
    const float f = (float)(int)(v >> 32) * 4294967296.0f + (float)(uint32_t)v;
    return L.scale * f;
}

// Adjoint deflation. The adjoint's iteration operator B = d M^T + d g 1^T / n
// has B 1 = d 1 (every column of M sums to 1 over a vertex's out-edges, and a
// dangling vertex gets d (sum lambda)/n), so the error's component along 1
// decays only at rate d per sweep. After each sweep that did not meet the
// stopping rule every value is shifted by d / (1 - d) times the sweep's mean
// change: for the synchronous sweep this replaces B by B + 1 w^T with
// w^T 1 = -d, which keeps B's other eigenvalues, sends the one of 1 to 0 and
// leaves the fixed point where it was (a Wielandt deflation of the known
// eigenpair (d, 1)); the in-place forms take the same step with their own
// contraction rate (adjoint_deflate). The shift is applied as an offset
// (AdjOffset, below), not to the array.

// The adjoint keeps its deflation shifts as one offset: the array holds
// lambda - aoff (aoff the sum of the shifts so far), so a shift is one add to
// a scalar every CTA computes alike instead of a pass over all n values and a
// grid barrier. A row's update from the held values: with lambda_v = x_v + aoff
// and every out-edge value row of M^T summing to 1,
//   lambda'_u = c_u + d (sum + aoff) = c_u + d sum + d aoff (u with out-edges),
//   lambda'_u = c_u + d (sum x + n aoff) / n = c_u + gt + d aoff (dangling u),
// so x'_u = lambda'_u - aoff = c_u - (1 - d) aoff + d sum (+ gt when dangling),
// gt the global term of the held values; (M^T lambda)_u = sum + aoff for u
// with out-edges. Changes, the residual and the live sum are those of the held
// values; the sum of lambda is theirs plus n aoff; the output adds aoff back.
struct AdjOffset {
    double sum;    // sum lambda as the sweep starts (held values + n aoff)
    double off;    // aoff
    float off_f;   // aoff in FP32 for the row updates
    double dprev;  // the previous sweep's mean change
    double sprev;  // the previous shift
    int steps;     // shifts so far
};

// After a sweep short of the stopping rule: the shift of the slow mode from the
// sweep's sum of the held values (exact FP64 grid sum, the same in every CTA).
// A sweep multiplies the mean error e by rho: d for the synchronous sweep, so
// its mean change is (rho - 1) e and the shift that cancels the error after the
// sweep is rho / (1 - rho) times the mean change. An in-place sweep reuses
// values it has already lowered, so its rho is below d and d's shift would
// overshoot (the mean error then alternates in sign and can grow). Its rho is
// estimated from the response to the previous shift s: the mean changes
// satisfy delta_k = rho (delta_{k-1} + s) - s, so rho = (delta_k + s) /
// (delta_{k-1} + s), clamped to [0, d].
__device__ __forceinline__ void adjoint_deflate(const SweepParams& p, AdjOffset& A, double held_sum, bool jacobi)
{
    const double n = (double)p.n, d = (double)p.d;
    const double sum_new = held_sum + n * A.off;
    const double delta = (sum_new - A.sum) / n;
    double rho = d;
    if (!jacobi && A.steps > 0) {
        const double den = A.dprev + A.sprev;
        const double r = den != 0.0 ? (delta + A.sprev) / den : d;
        rho = fmin(fmax(r, 0.0), d);
    }
    const double shift = rho / (1.0 - rho) * delta;
    A.off += shift;
    A.off_f = (float)A.off;
    A.sum = sum_new + n * shift;
    A.dprev = delta;
    A.sprev = shift;
    ++A.steps;
}

// Initial values of all n rows as a grid-stride pass (any thread any row:
// nothing reads them before the grid barrier that follows; a pass over the
// worker's own rows would leave the grid waiting for the workers whose blocks
// hold thousands of rows without in-edges), four rows' inputs loaded before
// any is stored. PageRank: x = r0 / outdeg (r0 on vertices without
// out-edges), gpart += r0 over vertices with out-edges (N(0)), tpart += t (T);
// the adjoint: lambda0 = c (or the warm start), gpart += lambda0, tpart += |c|;
// Bellman-Ford: 0 at the source, INF elsewhere.
template <int MODE>
__device__ __forceinline__ void init_values(const SweepParams& p, uint32_t* X, double& gpart, double& tpart)
{
    constexpr bool BF = MODE == MODE_BF || MODE == MODE_BF8;
    const long long stride = (long long)gridDim.x * blockDim.x, n = p.n;
    const float inv_n = 1.0f / (float)p.n;
    for (long long v0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; v0 < n; v0 += 4 * stride) {
        if constexpr (BF) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const long long v = v0 + q * stride;
                if (v < n) X[v] = (v == (long long)p.src) ? 0u : INF;
            }
        } else {
            float t[4], r0[4], dg[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const long long v = v0 + q * stride;
                t[q] = inv_n;
                r0[q] = 0.0f;
                dg[q] = 0.0f;
                if (v < n) {
                    if (MODE == MODE_ADJ || p.base) t[q] = p.base[v];
                    r0[q] = p.init ? p.init[v] : t[q];
                    if constexpr (MODE != MODE_ADJ) dg[q] = p.degf[v];
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const long long v = v0 + q * stride;
                if (v >= n) continue;
                if constexpr (MODE == MODE_ADJ) {
                    X[v] = __float_as_uint(r0[q]);
                    gpart += (double)r0[q];
                    tpart += fabs((double)t[q]);
                } else {
                    X[v] = __float_as_uint((MODE == MODE_PR && dg[q] > 0.0f) ? r0[q] / dg[q] : r0[q]);
                    if (dg[q] > 0.0f) gpart += (double)r0[q];
                    tpart += (double)t[q];
                }
            }
        }
    }
}

// The caller's output from the final state x as a grid-stride pass (after the
// last grid barrier every value is final), four values in flight per thread:
// distances, lambda and the weighted form's r as they are, PageRank's
// x = r / outdeg back to r.
template <int MODE>
__device__ __forceinline__ void write_output(const SweepParams& p, const uint32_t* x, float aoff = 0.0f)
{
    constexpr bool RAW = MODE == MODE_BF || MODE == MODE_BF8 || MODE == MODE_ADJ || MODE == MODE_PRW;
    const long long stride = (long long)gridDim.x * blockDim.x, n = p.n;
    for (long long v0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; v0 < n; v0 += 4 * stride) {
        uint32_t a[4];
        float dg[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const long long v = v0 + q * stride;
            a[q] = v < n ? ld_relaxed_b32(x + v) : 0u;
            dg[q] = (!RAW && v < n) ? p.degf[v] : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const long long v = v0 + q * stride;
            if (v >= n) continue;
            if constexpr (MODE == MODE_ADJ) ((float*)p.out)[v] = __uint_as_float(a[q]) + aoff;  // AdjOffset
            else if constexpr (RAW) ((uint32_t*)p.out)[v] = a[q];
            else ((float*)p.out)[v] = dg[q] > 0.0f ? __uint_as_float(a[q]) * dg[q] : __uint_as_float(a[q]);
        }
    }
}

// Sum of the live sum's stripes read by one thread: all loads issued before
// any is added, so the thread waits for one L2 round trip, not one per stripe.
__device__ __forceinline__ long long stripes_total(const SyncBlock* sb)
{
    long long a[GSTRIPES];
#pragma unroll
    for (int k = 0; k < GSTRIPES; ++k) a[k] = ld_relaxed_i64(&sb->stripe[k * GSTRIDE]);
    long long G = 0;
#pragma unroll
    for (int k = 0; k < GSTRIPES; ++k) G += a[k];
    return G;
}

// The base term of row v: c_v for the adjoint, (1 - d) t_v for PageRank with a
// teleport vector, (1 - d) / n without one (Bellman-Ford: none).
template <int MODE>
__device__ __forceinline__ float row_base(const SweepParams& p, int v)
{
    if constexpr (MODE == MODE_ADJ) return ld_stream_f32(p.base + v);
    else if constexpr (MODE == MODE_BF || MODE == MODE_BF8) return 0.0f;
    else return p.base ? p.base_scale * ld_stream_f32(p.base + v) : p.uniform_base;
}

// New value of row v from its pull sum, old value and base term bv (row_base;
// PageRank: x = r/outdeg with dg = outdeg; adjoint: lambda; Bellman-Ford:
// dist), with the residual and global-sum contributions.
template <int MODE>
__device__ __forceinline__ uint32_t row_update_b(const SweepParams& p, int v, uint32_t sum, uint32_t xo_bits,
                                                 float dg, float gt, float bv, float aoff, float& res_part,
                                                 float& g_part, float& dg_part)
{
    constexpr bool BF = MODE == MODE_BF || MODE == MODE_BF8;
    if constexpr (BF) {
        const uint32_t xnew = sum < xo_bits ? sum : xo_bits;
        if (xnew < xo_bits) res_part += 1.0f;
        return xnew;
    } else {
        const float xo = __uint_as_float(xo_bits);
        float rnew, rold;
        if constexpr (MODE == MODE_ADJ) {
            rold = xo;
            // held values (AdjOffset): x' = c - (1 - d) aoff + d sum (+ gt when dangling)
            rnew = (bv - (1.0f - p.d) * aoff) + p.d * __uint_as_float(sum) + (dg == 0.0f ? gt : 0.0f);
            g_part += rnew;
            dg_part += rnew - rold;
            if (p.aux_out) p.aux_out[v] = __uint_as_float(sum) + (dg > 0.0f ? aoff : 0.0f);
        } else {
            rold = (MODE == MODE_PR && dg > 0.0f) ? xo * dg : xo;
            rnew = bv + p.d * __uint_as_float(sum) + gt;
            if (dg > 0.0f) {
                g_part += rnew;
                dg_part += rnew - rold;
            }
        }
        res_part += fabsf(rnew - rold);
        // x = r / outdeg; __fdividef (2 ulp) has no special-value path, and the
        // quotient of a dangling row (dg = 0) is discarded by the select
        return __float_as_uint((MODE == MODE_PR && dg > 0.0f) ? __fdividef(rnew, dg) : rnew);
    }
}

// row_update_b with the base term loaded here (aoff: the adjoint's offset, 0 for the other modes).
template <int MODE>
__device__ __forceinline__ uint32_t row_update(const SweepParams& p, int v, uint32_t sum, uint32_t xo_bits, float dg,
                                               float gt, float aoff, float& res_part, float& g_part, float& dg_part)
{
    return row_update_b<MODE>(p, v, sum, xo_bits, dg, gt, row_base<MODE>(p, v), aoff, res_part, g_part, dg_part);
}

}  // namespace dag
