// Persistent pull-sweep kernels: PageRank (plain and weighted), the PageRank
// adjoint, and Bellman-Ford, each in the synchronous, asynchronous and
// delayed-asynchronous forms.
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
// GPU specifics: in-place forms read the shared state with relaxed gpu-scope
// loads (served by L2, where all CTAs' stores meet), the synchronous form
// with ordinary loads that may hit in L1; the edge stream (colidx, weights)
// bypasses L1. Rows completed by a tile are contiguous, so flushes are
// coalesced stores of consecutive values.
#include <climits>
#include <type_traits>

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

// dist_u + w, INF when dist_u is INF; a finite sum that would reach INF stays
// finite at INF - 1 (cannot happen for n * 255 < 2^32).
__device__ __forceinline__ uint32_t relax(uint32_t du, uint32_t w)
{
    if (du == INF) return INF;
    uint32_t s = du + w;
    return (s < du || s == INF) ? INF - 1u : s;
}

struct SweepShared {
    uint32_t val[TILE];        // gathered edge terms of the tile
    int rowend[TILE + 1];      // tile-relative row end offsets (+ sentinel)
    uint32_t rowsum[TILE];     // per-row reduction of the tile
    uint32_t scan[NT];         // per-thread inclusive segmented scan of carries
    int wkey[NWARP];
    uint32_t wval[NWARP];
    uint32_t wscan[NWARP];
    double red0[NWARP];
    double red1[NWARP];
    double dgw[NWARP];
    double G;                  // live global sum read at the tile start
    double res;                // broadcast of the sweep residual
    double gprev;              // broadcast of the previous sweep's global sum
    double T;                  // broadcast of the teleport total / ||c||_1
};

// Block sum of two doubles; the result is valid in thread 0.
__device__ __forceinline__ void block_sum2(SweepShared& sh, double& a, double& b)
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

template <int MODE, int VAR>
__global__ void __launch_bounds__(NT) sweep_kernel(const SweepParams p)
{
    using O = Op<MODE>;
    constexpr bool BF = MODE == MODE_BF;
    constexpr bool SYNC = VAR == DAG_SYNC;
    constexpr bool DELAYED = VAR == DAG_DELAYED;
    constexpr bool LIVE_G = !SYNC && !BF;  // async/delayed PageRank-type: live global sum

    __shared__ SweepShared sh;
    extern __shared__ uint32_t s_buf[];  // delay buffer (DELAYED)

    const int c = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    SyncBlock* sb = p.sync;
    unsigned long long bar_target = 0;
    uint32_t* X0 = (uint32_t*)p.x0;
    uint32_t* X1 = (uint32_t*)p.x1;
    const int row_lo = p.cta_row[c], row_hi = p.cta_row[c + 1];
    const int tile_lo = p.cta_tile[c], tile_hi = p.cta_tile[c + 1];
    const float inv_n = 1.0f / (float)p.n;

    // ---------------- initial values of the owned rows ----------------
    {
        double gpart = 0.0, tpart = 0.0;
        for (int v = row_lo + tid; v < row_hi; v += NT) {
            if constexpr (BF) {
                X0[v] = (v == (int)p.src) ? 0u : INF;
            } else if constexpr (MODE == MODE_ADJ) {
                float cv = p.base[v];
                float l0 = p.init ? p.init[v] : cv;
                X0[v] = __float_as_uint(l0);
                gpart += (double)l0;
                tpart += fabs((double)cv);
            } else {
                float t = p.base ? p.base[v] : inv_n;
                float r0 = p.init ? p.init[v] : t;
                float dg = p.degf[v];
                float x = (MODE == MODE_PR && dg > 0.0f) ? r0 / dg : r0;
                X0[v] = __float_as_uint(x);
                if (dg > 0.0f) gpart += (double)r0;
                tpart += (double)t;
            }
        }
        if constexpr (!BF) {
            block_sum2(sh, gpart, tpart);
            if (tid == 0) {
                atomicAdd(&sb->acc_g[2], gpart);
                atomicAdd(&sb->T, tpart);
                if (LIVE_G) atomicAdd(&sb->stripe[(c % GSTRIPES) * GSTRIDE], gpart);
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
    const double tol = (MODE == MODE_ADJ) ? p.tol * T : p.tol;

    int buf_first = row_lo, buf_cnt = 0;
    long long flushes = 0;
    int it = 0;
    bool converged = false;
    double last_res = 0.0;

    for (; it < p.max_iters; ++it) {
        const int slot = it % 3;
        const uint32_t* xin = SYNC ? ((it & 1) ? X1 : X0) : X0;
        uint32_t* xout = SYNC ? ((it & 1) ? X0 : X1) : X0;
        double res_part = 0.0, g_part = 0.0, dg_part = 0.0;
        uint32_t carry = O::identity();  // partial of the row that continues into the next tile
        bool publish = false;            // async: a tile's change of G waits in sh.dgw
        // global term of this sweep (sync) or of this tile (async/delayed)
        float gterm = 0.0f;
        if constexpr (SYNC && !BF) {
            gterm = (MODE == MODE_ADJ) ? (float)((double)p.g_coef * gprev)
                                       : (float)((double)p.g_coef * (T - gprev));
        }

        for (int t = tile_lo; t < tile_hi; ++t) {
            const int a0 = p.tile_row[t], b0 = p.tile_nz[t];
            const int NA = p.tile_row[t + 1] - a0, NB = p.tile_nz[t + 1] - b0;
            const int L = NA + NB;

            if constexpr (LIVE_G) {
                if (warp == 0) {
                    double gs = ld_relaxed_f64(&sb->stripe[lane * GSTRIDE]);
                    gs = warp_sum(gs);
                    if (lane == 0) sh.G = gs;
                }
            }
            // -------- stage the tile: row ends, then gathered edge terms --------
            for (int i = tid; i < NA; i += NT) sh.rowend[i] = ld_stream_i32(p.rowptr + a0 + i + 1) - b0;
            if (tid == 0) sh.rowend[NA] = INT_MAX;
            {
                int col[IPT];
                uint32_t aux[IPT];
#pragma unroll
                for (int q = 0; q < IPT; ++q) {
                    const int j = tid + q * NT;
                    col[q] = 0;
                    aux[q] = 0;
                    if (j < NB) {
                        col[q] = ld_stream_i32(p.colidx + b0 + j);
                        if constexpr (BF) aux[q] = ld_stream_u32(p.w + b0 + j);
                        if constexpr (MODE == MODE_PRW || MODE == MODE_ADJ)
                            aux[q] = __float_as_uint(ld_stream_f32(p.val + b0 + j));
                    }
                }
#pragma unroll
                for (int q = 0; q < IPT; ++q) {
                    const int j = tid + q * NT;
                    if (j < NB) {
                        uint32_t xv = SYNC ? ld_weak_b32(xin + col[q]) : ld_relaxed_b32(xin + col[q]);
                        uint32_t term;
                        if constexpr (BF) term = relax(xv, aux[q]);
                        else if constexpr (MODE == MODE_PR) term = xv;
                        else term = __float_as_uint(__uint_as_float(aux[q]) * __uint_as_float(xv));
                        sh.val[j] = term;
                    }
                }
            }
            __syncthreads();  // (A) tile staged

            if constexpr (VAR == DAG_ASYNC && !BF) {
                if (publish && tid == 0) {
                    double s = 0.0;
                    for (int k = 0; k < NWARP; ++k) s += sh.dgw[k];
                    atomicAdd(&sb->stripe[(c % GSTRIPES) * GSTRIDE], s);
                }
                publish = false;
            }

            // -------- merge-path walk over this thread's IPT items --------
            const int k0 = min(tid * IPT, L);
            int lo = max(0, k0 - NB), hi = min(k0, NA);
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (sh.rowend[mid] <= k0 - 1 - mid) lo = mid + 1;
                else hi = mid;
            }
            int i = lo, j = k0 - lo;
            const int i_start = i;
            bool emitted = false;
            uint32_t acc = (tid == 0) ? carry : O::identity();
            int re = sh.rowend[i];
#pragma unroll
            for (int q = 0; q < IPT; ++q) {
                if (k0 + q < L) {
                    if (re <= j) {
                        sh.rowsum[i] = acc;
                        emitted = true;
                        acc = O::identity();
                        ++i;
                        re = sh.rowend[i];
                    } else {
                        acc = O::combine(acc, sh.val[j]);
                        ++j;
                    }
                }
            }
            // -------- block segmented scan of (row in progress, partial) --------
            const int key = i;
            uint32_t sv = acc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t ov = __shfl_up_sync(0xffffffffu, sv, o);
                const int ok = __shfl_up_sync(0xffffffffu, key, o);
                if (lane >= o && ok == key) sv = O::combine(sv, ov);
            }
            if (lane == 31) { sh.wkey[warp] = key; sh.wval[warp] = sv; }
            __syncthreads();  // (B)
            if (warp == 0) {
                const int wk = lane < NWARP ? sh.wkey[lane] : INT_MAX - lane;
                uint32_t wv = lane < NWARP ? sh.wval[lane] : O::identity();
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t ov = __shfl_up_sync(0xffffffffu, wv, o);
                    const int ok = __shfl_up_sync(0xffffffffu, wk, o);
                    if (lane >= o && ok == wk) wv = O::combine(wv, ov);
                }
                if (lane < NWARP) sh.wscan[lane] = wv;
            }
            __syncthreads();  // (C)
            {
                const int k_first = __shfl_sync(0xffffffffu, key, 0);
                if (warp > 0 && key == k_first && sh.wkey[warp - 1] == key)
                    sv = O::combine(sv, sh.wscan[warp - 1]);
            }
            sh.scan[tid] = sv;
            __syncthreads();  // (D)
            if (tid > 0 && emitted) sh.rowsum[i_start] = O::combine(sh.rowsum[i_start], sh.scan[tid - 1]);
            if (tid == 0) carry = sh.scan[NT - 1];
            __syncthreads();  // (E) row sums final

            // -------- epilogue: new values of the rows this tile completed --------
            float gt = gterm;
            if constexpr (LIVE_G) {
                gt = (MODE == MODE_ADJ) ? (float)((double)p.g_coef * sh.G)
                                        : (float)((double)p.g_coef * (T - sh.G));
            }
            for (int r = tid; r < NA; r += NT) {
                const int v = a0 + r;
                const uint32_t sum = sh.rowsum[r];
                uint32_t xnew;
                if constexpr (BF) {
                    const uint32_t old = SYNC ? ld_weak_b32(xin + v) : ld_relaxed_b32(xin + v);
                    xnew = sum < old ? sum : old;
                    if (xnew < old) res_part += 1.0;
                } else {
                    const float xo = __uint_as_float(SYNC ? ld_weak_b32(xin + v) : ld_relaxed_b32(xin + v));
                    const float dg = ld_stream_f32(p.degf + v);
                    float rnew;
                    float rold;
                    if constexpr (MODE == MODE_ADJ) {
                        rold = xo;
                        rnew = ld_stream_f32(p.base + v) + p.d * __uint_as_float(sum) + (dg == 0.0f ? gt : 0.0f);
                        g_part += (double)rnew;
                        dg_part += (double)rnew - (double)rold;
                        if (p.aux_out) p.aux_out[v] = __uint_as_float(sum);
                    } else {
                        rold = (MODE == MODE_PR && dg > 0.0f) ? xo * dg : xo;
                        const float bv = p.base ? p.base_scale * ld_stream_f32(p.base + v) : p.uniform_base;
                        rnew = bv + p.d * __uint_as_float(sum) + gt;
                        if (dg > 0.0f) {
                            g_part += (double)rnew;
                            dg_part += (double)rnew - (double)rold;
                        }
                    }
                    res_part += fabs((double)rnew - (double)rold);
                    xnew = __float_as_uint((MODE == MODE_PR && dg > 0.0f) ? rnew / dg : rnew);
                }
                if constexpr (SYNC) st_weak_b32(xout + v, xnew);
                else if constexpr (DELAYED) s_buf[v - buf_first] = xnew;
                else st_relaxed_b32(xout + v, xnew);
            }

            if constexpr (VAR == DAG_ASYNC && !BF) {
                const double s = warp_sum(dg_part);
                dg_part = 0.0;
                if (lane == 0) sh.dgw[warp] = s;
                publish = true;  // summed by thread 0 after the next barrier point
            }
            if constexpr (DELAYED) {
                buf_cnt += NA;
                if (buf_cnt >= p.delta || t == tile_hi - 1) {
                    double s = 0.0;
                    if constexpr (!BF) s = warp_sum(dg_part);
                    dg_part = 0.0;
                    if (lane == 0) sh.dgw[warp] = s;
                    __syncthreads();  // buffer complete
                    for (int k = tid; k < buf_cnt; k += NT) st_relaxed_b32(X0 + buf_first + k, s_buf[k]);
                    if constexpr (!BF) {
                        if (tid == 0) {
                            double tot = 0.0;
                            for (int k = 0; k < NWARP; ++k) tot += sh.dgw[k];
                            atomicAdd(&sb->stripe[(c % GSTRIPES) * GSTRIDE], tot);
                        }
                    }
                    buf_first += buf_cnt;
                    buf_cnt = 0;
                    ++flushes;
                    __syncthreads();  // buffer free again
                }
            }
        }  // tiles

        if constexpr (VAR == DAG_ASYNC && !BF) {
            __syncthreads();
            if (publish && tid == 0) {
                double s = 0.0;
                for (int k = 0; k < NWARP; ++k) s += sh.dgw[k];
                atomicAdd(&sb->stripe[(c % GSTRIPES) * GSTRIDE], s);
            }
        }
        if constexpr (DELAYED) buf_first = row_lo;

        // -------- end of sweep: residual, barrier, stopping rule --------
        block_sum2(sh, res_part, g_part);
        if (tid == 0) {
            if (res_part != 0.0) atomicAdd(&sb->acc_res[slot], res_part);
            if (SYNC && !BF && g_part != 0.0) atomicAdd(&sb->acc_g[slot], g_part);
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
    }

    // ---------------- output of the owned rows ----------------
    {
        const uint32_t* xf = SYNC ? ((it & 1) ? X1 : X0) : X0;
        for (int v = row_lo + tid; v < row_hi; v += NT) {
            const uint32_t x = ld_relaxed_b32(xf + v);
            if constexpr (BF || MODE == MODE_ADJ || MODE == MODE_PRW) {
                ((uint32_t*)p.out)[v] = x;
            } else {
                const float dg = p.degf[v];
                ((float*)p.out)[v] = dg > 0.0f ? __uint_as_float(x) * dg : __uint_as_float(x);
            }
        }
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

static KernelFn kernel_for(int mode, int variant)
{
    static const KernelFn table[4][3] = {
        {sweep_kernel<MODE_PR, DAG_SYNC>, sweep_kernel<MODE_PR, DAG_ASYNC>, sweep_kernel<MODE_PR, DAG_DELAYED>},
        {sweep_kernel<MODE_PRW, DAG_SYNC>, sweep_kernel<MODE_PRW, DAG_ASYNC>, sweep_kernel<MODE_PRW, DAG_DELAYED>},
        {sweep_kernel<MODE_ADJ, DAG_SYNC>, sweep_kernel<MODE_ADJ, DAG_ASYNC>, sweep_kernel<MODE_ADJ, DAG_DELAYED>},
        {sweep_kernel<MODE_BF, DAG_SYNC>, sweep_kernel<MODE_BF, DAG_ASYNC>, sweep_kernel<MODE_BF, DAG_DELAYED>},
    };
    return table[mode][variant];
}

// Elements of dynamic shared memory a delayed sweep needs for buffer size
// delta: up to delta - 1 buffered rows plus one tile's rows.
int sweep_buffer_cap(dag_plan* plan, int delta, int* cap)
{
    long long c = (long long)delta - 1 + TILE;
    if (c > plan->n) c = plan->n;
    if (c < 1) c = 1;
    *cap = (int)c;
    return DAG_OK;
}

int max_workers(dag_plan* plan, int mode, int variant, int buf_cap_elems, int* out)
{
    KernelFn k = kernel_for(mode, variant);
    size_t dyn = (variant == DAG_DELAYED) ? (size_t)buf_cap_elems * 4 : 0;
    int max_dyn = 0;
    DAG_CUDA(cudaDeviceGetAttribute(&max_dyn, cudaDevAttrMaxSharedMemoryPerBlockOptin, plan->device));
    if (dyn + sizeof(SweepShared) > (size_t)max_dyn)
        return set_error(DAG_ERR_INVALID, "delta too large: the delay buffer does not fit in shared memory");
    DAG_CUDA(cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    int per_sm = 0;
    DAG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k, NT, dyn));
    if (per_sm < 1) return set_error(DAG_ERR_INVALID, "sweep kernel cannot be resident with this delta");
    *out = per_sm * plan->num_sms;
    return DAG_OK;
}

int launch_sweep(dag_plan* plan, int mode, int variant, int delta, SweepParams& p, cudaStream_t s,
                 int* out_nblocks)
{
    int cap = 0;
    if (variant == DAG_DELAYED) sweep_buffer_cap(plan, delta, &cap);
    int nb = 0;
    int rc = max_workers(plan, mode, variant, cap, &nb);
    if (rc) return rc;
    Partition* part = nullptr;
    rc = get_partition(plan, nb, &part, s);
    if (rc) return rc;
    if (variant == DAG_DELAYED && cap > part->max_rows + TILE) cap = part->max_rows + TILE;
    p.nblocks = nb;
    p.delta = (variant == DAG_DELAYED) ? delta : 0;
    p.buf_cap = cap;
    p.cta_row = part->cta_row;
    p.cta_tile = part->cta_tile;
    p.tile_row = part->tile_row;
    p.tile_nz = part->tile_nz;
    p.sync = plan->sync;
    p.timeout_ns = plan->timeout_ns;
    p.skip_barrier_cta0 = 0;
    if (plan->skip_barrier_once) {
        p.skip_barrier_cta0 = 1;
        p.timeout_ns = plan->skip_timeout_ns;
        plan->skip_barrier_once = 0;
    }
    DAG_CUDA(cudaMemsetAsync(plan->sync, 0, sizeof(SyncBlock), s));
    KernelFn k = kernel_for(mode, variant);
    void* args[] = {(void*)&p};
    size_t dyn = (variant == DAG_DELAYED) ? (size_t)cap * 4 : 0;
    DAG_CUDA(cudaLaunchCooperativeKernel((const void*)k, dim3(nb), dim3(NT), args, dyn, s));
    *out_nblocks = nb;
    return DAG_OK;
}

}  // namespace dag
