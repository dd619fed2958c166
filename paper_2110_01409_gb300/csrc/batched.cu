// Batched personalized PageRank and batched Bellman-Ford in one persistent
// launch (no counterpart in the paper: each column is an independent problem
// solved with the paper's sweep, Sec. III; columns stop on their own).
//
// State X is row-major [n][B]: the B values of a vertex are contiguous, so an
// in-edge gathers one contiguous slice of B values. A CTA owns a vertex block
// (Sec. III-A partition) and holds one warp per 32-column chunk; every warp
// walks the CTA's merge-path tiles in vertex order, one lane per column. A
// column that met its stopping rule is frozen (not read, not written) for the
// rest of the launch, and a warp whose 32 columns are all frozen skips the
// tile. In the delayed form the "worker" of Sec. III-B is a (CTA, column
// chunk) pair: each warp buffers delta rows of its 32 columns in shared
// memory and copies them out when the buffer is full or its block is done.
#include <climits>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "dag_internal.cuh"

namespace dag {

struct BatchParams {
    int n;
    int B;
    int nblocks;
    const int* rowptr;
    const int* colidx;
    const uint32_t* w;
    const uint8_t* w8;     // one-byte weights (BF8), else nullptr
    const float* degf;
    const float* V;        // PPR teleports [n][B]
    const uint32_t* src;   // BF sources [B]
    float d;
    float g_coef;
    double tol;
    int max_iters;
    int delta;             // rows per warp buffer (delayed)
    uint32_t* X0;          // [n][B] (the caller's output array)
    uint32_t* X1;          // [n][B] workspace (sync)
    const int* cta_row;
    const int* cta_tile;
    const int* tile_row;
    const int* tile_nz;
    SyncBlock* sb;
    double* acc_res;       // [3][B]
    double* acc_g;         // [3][B]
    double* gl;            // [B] live non-dangling mass (async / delayed PPR)
    double* T;             // [B] teleport totals
    int* iters;            // [B] sweeps of each column (output)
    long long timeout_ns;
};

constexpr int BU = 8;  // edges gathered per warp before accumulating

template <bool BF>
__device__ __forceinline__ uint32_t b_ident()
{
    return BF ? INF : 0u;
}

template <bool BF>
__device__ __forceinline__ uint32_t b_comb(uint32_t a, uint32_t b)
{
    if constexpr (BF) return a < b ? a : b;
    else return __float_as_uint(__uint_as_float(a) + __uint_as_float(b));
}

__device__ __forceinline__ uint32_t b_relax(uint32_t du, uint32_t w)
{
    if (du == INF) return INF;
    uint32_t s = du + w;
    return (s < du || s == INF) ? INF - 1u : s;
}

template <bool BF, int VAR, bool W8 = false>
__global__ void batched_kernel(const BatchParams p)
{
    constexpr bool SYNC = VAR == DAG_SYNC;
    constexpr bool DELAYED = VAR == DAG_DELAYED;
    constexpr bool LIVE = !SYNC && !BF;
    extern __shared__ __align__(16) uint32_t smem[];
    int* s_col = (int*)smem;
    int* s_end = s_col + TILE;
    uint32_t* s_w = (uint32_t*)(s_end + TILE + 1);
    uint32_t* s_buf = s_w + (BF ? TILE : 0);  // per warp: delta rows x 32 columns

    const int B = p.B;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int col = warp * 32 + lane;
    const bool colok = col < B;
    const int cb = blockIdx.x;
    const int row_lo = p.cta_row[cb], row_hi = p.cta_row[cb + 1];
    const int tile_lo = p.cta_tile[cb], tile_hi = p.cta_tile[cb + 1];
    unsigned long long bar = 0;
    uint32_t* mybuf = s_buf + (size_t)warp * (DELAYED ? p.delta : 0) * 32;

    // ---------------- initial values ----------------
    {
        float gpart = 0.0f, tpart = 0.0f;  // per-lane partials over the block; FP64 in the atomics
        uint32_t s0 = BF && colok ? p.src[col] : 0u;
        // four rows' inputs loaded before any is stored (the stores could alias the inputs, so the
        // compiler would not overlap them itself)
        for (int v0 = row_lo; colok && v0 < row_hi; v0 += 4) {
            if constexpr (BF) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int v = v0 + q;
                    if (v < row_hi) p.X0[(size_t)v * B + col] = ((uint32_t)v == s0) ? 0u : INF;
                }
            } else {
                float t[4], dg[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int v = v0 + q;
                    t[q] = v < row_hi ? p.V[(size_t)v * B + col] : 0.0f;
                    dg[q] = v < row_hi ? p.degf[v] : 0.0f;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int v = v0 + q;
                    if (v >= row_hi) continue;
                    p.X0[(size_t)v * B + col] = __float_as_uint(dg[q] > 0.0f ? t[q] / dg[q] : t[q]);
                    if (dg[q] > 0.0f) gpart += t[q];
                    tpart += t[q];
                }
            }
        }
        if (!BF && colok) {
            if (tpart != 0.0f) atomicAdd(&p.T[col], (double)tpart);
            if (gpart != 0.0f) {
                atomicAdd(&p.acc_g[2 * B + col], (double)gpart);
                if (LIVE) atomicAdd(&p.gl[col], (double)gpart);
            }
        }
    }
    if (!grid_barrier(p.sb, p.nblocks, bar, p.timeout_ns)) return;
    double Tc = 0.0, gprev = 0.0;
    if (!BF && colok) {
        Tc = ld_relaxed_f64(&p.T[col]);
        gprev = ld_relaxed_f64(&p.acc_g[2 * B + col]);
    }
    bool active = colok;
    int last_it = 0;  // sweeps this column ran (same value in every CTA)
    int it = 0;
    for (; it < p.max_iters; ++it) {
        const int slot = it % 3;
        const uint32_t* xin = SYNC ? ((it & 1) ? p.X1 : p.X0) : p.X0;
        uint32_t* xout = SYNC ? ((it & 1) ? p.X0 : p.X1) : p.X0;
        float res = 0.0f, gsum = 0.0f, dg_acc = 0.0f;  // per-lane partials; FP64 in the atomics
        uint32_t carry = b_ident<BF>();
        int buf_first = row_lo, buf_cnt = 0;
        const bool warp_active = __any_sync(0xffffffffu, active);
        float gt = 0.0f;
        if (SYNC && !BF) gt = (float)((double)p.g_coef * (Tc - gprev));

        for (int t = tile_lo; t < tile_hi; ++t) {
            const int a0 = p.tile_row[t], b0 = p.tile_nz[t];
            const int NA = p.tile_row[t + 1] - a0, NB = p.tile_nz[t + 1] - b0;
            __syncthreads();  // previous tile's staging no longer read
            for (int i = threadIdx.x; i < NA; i += blockDim.x) s_end[i] = ld_stream_i32(p.rowptr + a0 + i + 1) - b0;
            if (threadIdx.x == 0) s_end[NA] = INT_MAX;
            for (int j = threadIdx.x; j < NB; j += blockDim.x) {
                s_col[j] = ld_stream_i32(p.colidx + b0 + j);
                if constexpr (BF && W8) s_w[j] = (uint32_t)p.w8[b0 + j];
                else if constexpr (BF) s_w[j] = ld_stream_u32(p.w + b0 + j);
            }
            __syncthreads();
            if (!warp_active) continue;
            if constexpr (LIVE) {
                if (active) gt = (float)((double)p.g_coef * (Tc - ld_relaxed_f64(&p.gl[col])));
            }
            uint32_t acc = carry;
            int i = 0;
            int re = s_end[0];
            // the inputs of the row being accumulated (old value, teleport entry, out-degree), loaded when
            // the row starts so that they arrive while its edges are gathered; only this lane writes the
            // row's value in this column, so a value loaded early is still the current one
            uint32_t pre_old = 0u;
            float pre_v = 0.0f, pre_dg = 0.0f;
            auto preload = [&](int r) {
                if (r >= NA || !active) return;
                const int v = a0 + r;
                const size_t k = (size_t)v * B + col;
                pre_old = SYNC ? ld_weak_b32(xin + k) : ld_relaxed_b32(xin + k);
                if constexpr (!BF) {
                    pre_v = ld_stream_f32(p.V + k);
                    pre_dg = p.degf[v];
                }
            };
            preload(0);
            auto finish_row = [&](int r, uint32_t sum) {
                const int v = a0 + r;
                if (!active) return;
                const size_t k = (size_t)v * B + col;
                uint32_t xnew;
                if constexpr (BF) {
                    const uint32_t old = pre_old;
                    xnew = sum < old ? sum : old;
                    if (xnew < old) res += 1.0f;
                } else {
                    const float xo = __uint_as_float(pre_old);
                    const float dg = pre_dg;
                    const float rold = dg > 0.0f ? xo * dg : xo;
                    const float rnew = (1.0f - p.d) * pre_v + p.d * __uint_as_float(sum) + gt;
                    res += fabsf(rnew - rold);
                    if (dg > 0.0f) {
                        gsum += rnew;
                        dg_acc += rnew - rold;
                    }
                    xnew = __float_as_uint(dg > 0.0f ? __fdividef(rnew, dg) : rnew);  // 2 ulp, no special-value path
                }
                if constexpr (SYNC) st_weak_b32(xout + k, xnew);
                else if constexpr (DELAYED) mybuf[(v - buf_first) * 32 + lane] = xnew;
                else st_relaxed_b32(xout + k, xnew);
            };
            auto maybe_flush = [&](bool force) {
                if constexpr (DELAYED) {
                    if (buf_cnt > 0 && (buf_cnt >= p.delta || force)) {
                        __syncwarp();
                        if (active)
                            for (int q = 0; q < buf_cnt; ++q)
                                st_relaxed_b32(p.X0 + (size_t)(buf_first + q) * B + col, mybuf[q * 32 + lane]);
                        if (LIVE && active && dg_acc != 0.0f) {
                            atomicAdd(&p.gl[col], (double)dg_acc);
                            dg_acc = 0.0f;
                        }
                        buf_first += buf_cnt;
                        buf_cnt = 0;
                        __syncwarp();
                        if (LIVE && active) gt = (float)((double)p.g_coef * (Tc - ld_relaxed_f64(&p.gl[col])));
                    }
                }
            };
            for (int j0 = 0; j0 < NB; j0 += BU) {
                uint32_t xv[BU];
#pragma unroll
                for (int u = 0; u < BU; ++u) {
                    const int j = j0 + u;
                    xv[u] = 0u;
                    if (j < NB && active) {
                        const size_t k = (size_t)s_col[j] * B + col;
                        xv[u] = SYNC ? ld_weak_b32(xin + k) : ld_relaxed_b32(xin + k);
                    }
                }
#pragma unroll
                for (int u = 0; u < BU; ++u) {
                    const int j = j0 + u;
                    if (j < NB) {
                        while (re <= j) {
                            finish_row(i, acc);
                            if constexpr (DELAYED) { ++buf_cnt; maybe_flush(false); }
                            acc = b_ident<BF>();
                            ++i;
                            re = s_end[i];
                            preload(i);
                        }
                        uint32_t term;
                        if constexpr (BF) term = b_relax(xv[u], s_w[j]);
                        else term = xv[u];
                        acc = b_comb<BF>(acc, term);
                    }
                }
            }
            while (i < NA) {
                finish_row(i, acc);
                if constexpr (DELAYED) { ++buf_cnt; maybe_flush(false); }
                acc = b_ident<BF>();
                ++i;
                preload(i);
            }
            carry = acc;
            if constexpr (DELAYED) maybe_flush(t == tile_hi - 1);
            if constexpr (VAR == DAG_ASYNC && !BF) {
                if (active && dg_acc != 0.0f) {
                    atomicAdd(&p.gl[col], (double)dg_acc);
                    dg_acc = 0.0f;
                }
            }
        }
        // ---- end of sweep ----
        if (active) {
            if (res != 0.0f) atomicAdd(&p.acc_res[slot * B + col], (double)res);
            if (SYNC && !BF && gsum != 0.0f) atomicAdd(&p.acc_g[slot * B + col], (double)gsum);
        }
        if (!grid_barrier(p.sb, p.nblocks, bar, p.timeout_ns)) return;
        int still = 0;
        if (active) {
            const double r = ld_relaxed_f64(&p.acc_res[slot * B + col]);
            if (SYNC && !BF) gprev = ld_relaxed_f64(&p.acc_g[slot * B + col]);
            if (r <= p.tol) {
                active = false;
                last_it = it + 1;
                if (cb == 0) p.iters[col] = it + 1;
            } else {
                still = 1;
            }
        }
        if (cb == 0 && colok) {
            const int dead = (it + 2) % 3;
            p.acc_res[dead * B + col] = 0.0;
            p.acc_g[dead * B + col] = 0.0;
        }
        if (!__syncthreads_or(still)) { ++it; break; }
    }
    if (cb == 0 && active) p.iters[col] = it;  // not converged: ran them all
    if (active) last_it = it;
    {
        // every CTA holds all B columns and reads the same sums, so CTA 0 sees the outcome
        const int any_active = __syncthreads_or(active ? 1 : 0);
        if (cb == 0 && threadIdx.x == 0) {
            p.sb->iters = it;
            p.sb->converged = any_active ? 0 : 1;
        }
    }

    // ---------------- output: r = x * outdeg, from the buffer of each column's last sweep ----------------
    if (!colok) return;
    const uint32_t* xf = (SYNC && (last_it & 1)) ? p.X1 : p.X0;
    for (int v0 = row_lo; v0 < row_hi; v0 += 4) {  // four rows in flight
        uint32_t x[4];
        float dg[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int v = v0 + q;
            x[q] = v < row_hi ? ld_relaxed_b32(xf + (size_t)v * B + col) : 0u;
            dg[q] = (!BF && v < row_hi) ? p.degf[v] : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int v = v0 + q;
            if (v >= row_hi) continue;
            if constexpr (BF) p.X0[(size_t)v * B + col] = x[q];
            else p.X0[(size_t)v * B + col] =
                __float_as_uint(dg[q] > 0.0f ? __uint_as_float(x[q]) * dg[q] : __uint_as_float(x[q]));
        }
    }
}

// ---------------------------------------------------------------------------
// Wide batched sweep (synchronous and asynchronous forms, B = 32 CPL columns,
// CPL in {1, 2, 4, 8}). The kernel above gives each warp 32 columns and walks
// every edge of a tile with all eight warps in lock step, so a source row of
// B values is fetched as eight 128-byte slices by eight warps and each tile
// waits for the slowest of them. Here a warp owns all B columns (CPL per lane,
// one vector access each) and an eighth of each merge-path tile: it gathers a
// source's whole row as one burst and walks its share of the tile's rows and
// edges on its own. A row split between two warps' shares is finished after
// the tile's barrier from the shares' partials (kept in shared memory), and a
// row continuing into the next tile carries its partial there.
// ---------------------------------------------------------------------------
template <int CPL>
__device__ __forceinline__ void ld_cols(const uint32_t* a, uint32_t (&o)[CPL], bool coherent)
{
    if constexpr (CPL == 8) {
        if (coherent) {
            asm volatile("ld.relaxed.gpu.global.v4.b32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(o[0]), "=r"(o[1]), "=r"(o[2]), "=r"(o[3]) : "l"(a) : "memory");
            asm volatile("ld.relaxed.gpu.global.v4.b32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(o[4]), "=r"(o[5]), "=r"(o[6]), "=r"(o[7]) : "l"(a + 4) : "memory");
        } else {
            const uint4 u = *(const uint4*)a, w = *(const uint4*)(a + 4);
            o[0] = u.x; o[1] = u.y; o[2] = u.z; o[3] = u.w; o[4] = w.x; o[5] = w.y; o[6] = w.z; o[7] = w.w;
        }
    } else if constexpr (CPL == 4) {
        if (coherent) {
            asm volatile("ld.relaxed.gpu.global.v4.b32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(o[0]), "=r"(o[1]), "=r"(o[2]), "=r"(o[3]) : "l"(a) : "memory");
        } else {
            const uint4 u = *(const uint4*)a;
            o[0] = u.x; o[1] = u.y; o[2] = u.z; o[3] = u.w;
        }
    } else if constexpr (CPL == 2) {
        if (coherent) {
            asm volatile("ld.relaxed.gpu.global.v2.b32 {%0, %1}, [%2];" : "=r"(o[0]), "=r"(o[1]) : "l"(a) : "memory");
        } else {
            const uint2 u = *(const uint2*)a;
            o[0] = u.x; o[1] = u.y;
        }
    } else {
        o[0] = coherent ? ld_relaxed_b32(a) : *a;
    }
}

// Stores the lane's CPL values (all of them when every column runs, else only the running ones).
template <int CPL>
__device__ __forceinline__ void st_cols(uint32_t* a, const uint32_t (&v)[CPL], unsigned run, bool coherent)
{
    constexpr unsigned ALL = (1u << CPL) - 1u;
    if (run == ALL && CPL >= 2) {
        if constexpr (CPL == 8) {
            if (coherent) {
                asm volatile("st.relaxed.gpu.global.v4.b32 [%0], {%1, %2, %3, %4};"
                             ::"l"(a), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]) : "memory");
                asm volatile("st.relaxed.gpu.global.v4.b32 [%0], {%1, %2, %3, %4};"
                             ::"l"(a + 4), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]) : "memory");
            } else {
                *(uint4*)a = make_uint4(v[0], v[1], v[2], v[3]);
                *(uint4*)(a + 4) = make_uint4(v[4], v[5], v[6], v[7]);
            }
            return;
        } else if constexpr (CPL == 4) {
            if (coherent)
                asm volatile("st.relaxed.gpu.global.v4.b32 [%0], {%1, %2, %3, %4};"
                             ::"l"(a), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]) : "memory");
            else *(uint4*)a = make_uint4(v[0], v[1], v[2], v[3]);
            return;
        } else if constexpr (CPL == 2) {
            if (coherent) asm volatile("st.relaxed.gpu.global.v2.b32 [%0], {%1, %2};" ::"l"(a), "r"(v[0]), "r"(v[1]) : "memory");
            else *(uint2*)a = make_uint2(v[0], v[1]);
            return;
        }
    }
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
        if (!((run >> q) & 1u)) continue;
        if (coherent) st_relaxed_b32(a + q, v[q]);
        else a[q] = v[q];
    }
}

constexpr int WIDE_WARPS = 8;  // warps per CTA of the wide kernel
constexpr int WIDE_U = 1;      // edges whose rows a warp gathers before accumulating: the warps in flight hide the
                               // latency (measured at B = 256: 1 edge and 3 CTAs per SM beat 2, 4, 6 and 8 edges
                               // at 2 CTAs, and 4 CTAs, whose 64 registers spill)

template <bool BF, int VAR, bool W8, int CPL>
__global__ void __launch_bounds__(NT, 3) batched_wide_kernel(const BatchParams p)
{
    constexpr bool SYNC = VAR == DAG_SYNC;
    constexpr bool LIVE = !SYNC && !BF;
    constexpr unsigned ALL = (1u << CPL) - 1u;
    constexpr int B = 32 * CPL;
    static_assert(VAR != DAG_DELAYED, "the delayed form runs the column-chunk kernel");
    extern __shared__ __align__(16) uint32_t smem[];
    int* s_col = (int*)smem;                            // [TILE] the tile's edge sources
    int* s_end = s_col + TILE;                          // [TILE + 4] tile-relative row ends (+ sentinel)
    uint32_t* s_w = (uint32_t*)(s_end + TILE + 4);      // [TILE] weights (Bellman-Ford)
    uint32_t* s_part = s_w + (BF ? TILE : 0);           // [WIDE_WARPS][B] each share's trailing partial
    uint32_t* s_carry = s_part + WIDE_WARPS * B;        // [2][B] the partial carried into a tile
    double* s_T = (double*)(s_carry + 2 * B);           // [B] teleport totals (PageRank)
    double* s_g = s_T + B;                              // [B] mass on linked vertices, last sweep (synchronous)
    float* s_red = (float*)(s_g + B);                   // [WIDE_WARPS][B] the warps' per-column sums of a sweep
    float* s_dg = s_red + WIDE_WARPS * B;               // [B] the CTA's change of the live mass (asynchronous)
    int* s_last = (int*)(s_dg + B);                     // [B] sweeps each column ran
    __shared__ int s_i0[WIDE_WARPS], s_head[WIDE_WARPS], s_ends[WIDE_WARPS], s_tcont;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, tid = threadIdx.x;
    const int cb = blockIdx.x, c0 = lane * CPL;
    const int row_lo = p.cta_row[cb], row_hi = p.cta_row[cb + 1];
    const int tile_lo = p.cta_tile[cb], tile_hi = p.cta_tile[cb + 1];
    unsigned long long bar = 0;
    uint32_t srcv[CPL];
#pragma unroll
    for (int q = 0; q < CPL; ++q) srcv[q] = BF ? p.src[c0 + q] : 0u;

    // ---------------- initial values (the CTA's rows, a warp per row, CPL columns per lane) ----------------
    {
        float gpart[CPL], tpart[CPL];
#pragma unroll
        for (int q = 0; q < CPL; ++q) gpart[q] = tpart[q] = 0.0f;
        for (int v = row_lo + warp; v < row_hi; v += WIDE_WARPS) {
            uint32_t x[CPL];
            if constexpr (BF) {
#pragma unroll
                for (int q = 0; q < CPL; ++q) x[q] = ((uint32_t)v == srcv[q]) ? 0u : INF;
            } else {
                uint32_t t[CPL];
                ld_cols<CPL>((const uint32_t*)p.V + (size_t)v * B + c0, t, false);
                const float dg = p.degf[v];
#pragma unroll
                for (int q = 0; q < CPL; ++q) {
                    const float tv = __uint_as_float(t[q]);
                    x[q] = __float_as_uint(dg > 0.0f ? tv / dg : tv);
                    if (dg > 0.0f) gpart[q] += tv;
                    tpart[q] += tv;
                }
            }
            st_cols<CPL>(p.X0 + (size_t)v * B + c0, x, ALL, false);
        }
        if constexpr (!BF) {
#pragma unroll
            for (int q = 0; q < CPL; ++q) {
                if (tpart[q] != 0.0f) atomicAdd(&p.T[c0 + q], (double)tpart[q]);
                if (gpart[q] != 0.0f) {
                    atomicAdd(&p.acc_g[2 * B + c0 + q], (double)gpart[q]);
                    if (LIVE) atomicAdd(&p.gl[c0 + q], (double)gpart[q]);
                }
            }
        }
    }
    if (!grid_barrier(p.sb, p.nblocks, bar, p.timeout_ns)) return;
    for (int c = tid; c < B; c += NT) {
        if constexpr (!BF) {
            s_T[c] = ld_relaxed_f64(&p.T[c]);
            s_g[c] = ld_relaxed_f64(&p.acc_g[2 * B + c]);
        }
        s_last[c] = 0;
        s_dg[c] = 0.0f;
    }
    __syncthreads();
    unsigned act = ALL;  // this lane's columns still running (the same in every warp and CTA)
    int it = 0;
    for (; it < p.max_iters; ++it) {
        const int slot = it % 3;
        const uint32_t* xin = SYNC ? ((it & 1) ? p.X1 : p.X0) : p.X0;
        uint32_t* xout = SYNC ? ((it & 1) ? p.X0 : p.X1) : p.X0;
        float res[CPL], gsum[CPL], dga[CPL], gt[CPL];
#pragma unroll
        for (int q = 0; q < CPL; ++q) {
            res[q] = gsum[q] = dga[q] = 0.0f;
            gt[q] = (SYNC && !BF) ? (float)((double)p.g_coef * (s_T[c0 + q] - s_g[c0 + q])) : 0.0f;
        }
        // the new values of tile row i from its sum acc
        auto finish_row = [&](int a0, int i, const uint32_t (&acc)[CPL]) {
            const int v = a0 + i;
            const size_t base = (size_t)v * B + c0;
            uint32_t old[CPL], xn[CPL];
            ld_cols<CPL>(xin + base, old, !SYNC);
            if constexpr (BF) {
#pragma unroll
                for (int q = 0; q < CPL; ++q) {
                    xn[q] = acc[q] < old[q] ? acc[q] : old[q];
                    if (((act >> q) & 1u) && xn[q] < old[q]) res[q] += 1.0f;
                }
            } else {
                uint32_t tv[CPL];
                ld_cols<CPL>((const uint32_t*)p.V + base, tv, false);
                const float dg = p.degf[v];
#pragma unroll
                for (int q = 0; q < CPL; ++q) {
                    const float xo = __uint_as_float(old[q]);
                    const float rold = dg > 0.0f ? xo * dg : xo;
                    const float rnew = (1.0f - p.d) * __uint_as_float(tv[q]) + p.d * __uint_as_float(acc[q]) + gt[q];
                    if ((act >> q) & 1u) {
                        res[q] += fabsf(rnew - rold);
                        if (dg > 0.0f) {
                            gsum[q] += rnew;
                            dga[q] += rnew - rold;
                        }
                    }
                    xn[q] = __float_as_uint(dg > 0.0f ? __fdividef(rnew, dg) : rnew);  // 2 ulp, no special-value path
                }
            }
            st_cols<CPL>(xout + base, xn, act, !SYNC);
        };
        const bool any = __syncthreads_or(act != 0u) != 0;  // (the same in every CTA)
        int cbuf = 0;
        for (int t = tile_lo; any && t < tile_hi; ++t) {
            const int a0 = p.tile_row[t], b0 = p.tile_nz[t];
            const int NA = p.tile_row[t + 1] - a0, NB = p.tile_nz[t + 1] - b0;
            __syncthreads();  // the previous tile's buffers are no longer read
            for (int i = tid; i < NA; i += NT) s_end[i] = ld_stream_i32(p.rowptr + a0 + i + 1) - b0;
            if (tid == 0) {
                s_end[NA] = INT_MAX;
                s_tcont = b0 > ld_stream_i32(p.rowptr + a0) ? 1 : 0;  // the tile starts inside row a0
            }
            for (int j = tid; j < NB; j += NT) {
                s_col[j] = ld_stream_i32(p.colidx + b0 + j);
                if constexpr (BF && W8) s_w[j] = (uint32_t)p.w8[b0 + j];
                else if constexpr (BF) s_w[j] = ld_stream_u32(p.w + b0 + j);
            }
            __syncthreads();
            if constexpr (LIVE) {
#pragma unroll
                for (int q = 0; q < CPL; ++q)
                    if ((act >> q) & 1u) gt[q] = (float)((double)p.g_coef * (s_T[c0 + q] - ld_relaxed_f64(&p.gl[c0 + q])));
            }
            // this warp's share of the tile: merge-path diagonals [d0, d1)
            const int L = NA + NB;
            const int d0 = (int)((long long)warp * L / WIDE_WARPS), d1 = (int)((long long)(warp + 1) * L / WIDE_WARPS);
            auto search = [&](int d) -> int {  // rows completed before diagonal d
                int lo = max(0, d - NB), hi = min(d, NA);
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (s_end[mid] <= d - 1 - mid) lo = mid + 1;
                    else hi = mid;
                }
                return lo;
            };
            const int i0 = search(d0), i1 = search(d1);
            const int j0 = d0 - i0, j1 = d1 - i1;
            const bool head = i0 == 0 ? (s_tcont != 0 || j0 > 0) : j0 > s_end[i0 - 1];
            bool pending = head;  // the share's first row began before it: finished after the barrier
            uint32_t acc[CPL], headp[CPL];
#pragma unroll
            for (int q = 0; q < CPL; ++q) acc[q] = headp[q] = b_ident<BF>();
            int i = i0;
            bool head_done = false;
            auto row_end = [&]() {
                if (pending) {
#pragma unroll
                    for (int q = 0; q < CPL; ++q) headp[q] = acc[q];
                    pending = false;
                    head_done = true;
                } else {
                    finish_row(a0, i, acc);
                }
#pragma unroll
                for (int q = 0; q < CPL; ++q) acc[q] = b_ident<BF>();
                ++i;
            };
            for (int jb = j0; jb < j1; jb += WIDE_U) {
                const int nu = min(WIDE_U, j1 - jb);
                uint32_t xv[WIDE_U][CPL];
#pragma unroll
                for (int u = 0; u < WIDE_U; ++u)
                    if (u < nu) ld_cols<CPL>(xin + (size_t)s_col[jb + u] * B + c0, xv[u], !SYNC);
#pragma unroll
                for (int u = 0; u < WIDE_U; ++u) {
                    if (u >= nu) break;
                    const int e = jb + u;
                    while (i < i1 && s_end[i] <= e) row_end();
                    const uint32_t we = BF ? s_w[e] : 0u;
#pragma unroll
                    for (int q = 0; q < CPL; ++q)
                        acc[q] = b_comb<BF>(acc[q], BF ? b_relax(xv[u][q], we) : xv[u][q]);
                }
            }
            while (i < i1) row_end();
            // the share's trailing partial, and how its first row relates to the shares before it
#pragma unroll
            for (int q = 0; q < CPL; ++q) s_part[warp * B + c0 + q] = acc[q];
            if (lane == 0) {
                s_i0[warp] = i0;
                s_head[warp] = head ? 1 : 0;
                s_ends[warp] = i1 > i0 ? 1 : 0;
            }
            __syncthreads();
            // a row begun in earlier shares: theirs back to the one where it starts (or the tile's carry)
            auto gather_back = [&](int w_from, uint32_t (&tot)[CPL]) {
                int w2 = w_from;
                for (;; --w2) {
                    if (w2 < 0) {
#pragma unroll
                        for (int q = 0; q < CPL; ++q) tot[q] = b_comb<BF>(tot[q], s_carry[cbuf * B + c0 + q]);
                        break;
                    }
#pragma unroll
                    for (int q = 0; q < CPL; ++q) tot[q] = b_comb<BF>(tot[q], s_part[w2 * B + c0 + q]);
                    if (s_ends[w2] || !s_head[w2]) break;
                }
            };
            if (head_done) {
                uint32_t tot[CPL];
#pragma unroll
                for (int q = 0; q < CPL; ++q) tot[q] = headp[q];
                gather_back(warp - 1, tot);
                finish_row(a0, i0, tot);
            }
            if (warp == WIDE_WARPS - 1) {  // the partial carried into the next tile (identity when none)
                uint32_t tot[CPL];
#pragma unroll
                for (int q = 0; q < CPL; ++q) tot[q] = b_ident<BF>();
                gather_back(WIDE_WARPS - 1, tot);
#pragma unroll
                for (int q = 0; q < CPL; ++q) s_carry[(cbuf ^ 1) * B + c0 + q] = tot[q];
            }
            cbuf ^= 1;
            if constexpr (LIVE) {  // the tile's change of the live mass: the CTA's shares, then one atomic each
#pragma unroll
                for (int q = 0; q < CPL; ++q) {
                    if (dga[q] != 0.0f) atomicAdd(&s_dg[c0 + q], dga[q]);
                    dga[q] = 0.0f;
                }
                __syncthreads();
                for (int c = tid; c < B; c += NT) {
                    const float v = s_dg[c];
                    if (v != 0.0f) {
                        atomicAdd(&p.gl[c], (double)v);
                        s_dg[c] = 0.0f;
                    }
                }
            }
        }
        // ---- end of sweep: per-column sums (the CTA's warps added in a fixed order, so that the synchronous
        // form is deterministic; then one FP64 atomic each), barrier, stopping rules ----
        auto cta_sum = [&](const float (&part)[CPL], double* dst) {
            __syncthreads();  // s_red is free
#pragma unroll
            for (int q = 0; q < CPL; ++q) s_red[warp * B + c0 + q] = part[q];
            __syncthreads();
            for (int c = tid; c < B; c += NT) {
                float v = 0.0f;
#pragma unroll
                for (int w2 = 0; w2 < WIDE_WARPS; ++w2) v += s_red[w2 * B + c];
                if (v != 0.0f) atomicAdd(&dst[c], (double)v);
            }
        };
        cta_sum(res, p.acc_res + slot * B);
        if constexpr (SYNC && !BF) cta_sum(gsum, p.acc_g + slot * B);
        if (!grid_barrier(p.sb, p.nblocks, bar, p.timeout_ns)) return;
#pragma unroll
        for (int q = 0; q < CPL; ++q) {
            if (!((act >> q) & 1u)) continue;
            const int c = c0 + q;
            const double r = ld_relaxed_f64(&p.acc_res[slot * B + c]);
            if (SYNC && !BF && warp == 0) s_g[c] = ld_relaxed_f64(&p.acc_g[slot * B + c]);
            if (r <= p.tol) {
                act &= ~(1u << q);
                if (warp == 0) {
                    s_last[c] = it + 1;
                    if (cb == 0) p.iters[c] = it + 1;
                }
            }
        }
        if (cb == 0) {
            const int dead = (it + 2) % 3;
            for (int c = tid; c < B; c += NT) {
                p.acc_res[dead * B + c] = 0.0;
                p.acc_g[dead * B + c] = 0.0;
            }
        }
        if (!__syncthreads_or(act != 0u)) {
            ++it;
            break;
        }
    }
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < CPL; ++q)
            if ((act >> q) & 1u) {  // not converged: ran them all
                s_last[c0 + q] = it;
                if (cb == 0) p.iters[c0 + q] = it;
            }
    }
    {
        const int any_active = __syncthreads_or(act != 0u ? 1 : 0);
        if (cb == 0 && tid == 0) {
            p.sb->iters = it;
            p.sb->converged = any_active ? 0 : 1;
        }
    }

    // ---------------- output: r = x * outdeg, from the buffer of each column's last sweep ----------------
    for (int v = row_lo + warp; v < row_hi; v += WIDE_WARPS) {
        uint32_t x[CPL];
        const size_t base = (size_t)v * B + c0;
        if constexpr (SYNC) {
#pragma unroll
            for (int q = 0; q < CPL; ++q) x[q] = ld_relaxed_b32(((s_last[c0 + q] & 1) ? p.X1 : p.X0) + base + q);
        } else {
            ld_cols<CPL>(p.X0 + base, x, true);
        }
        if constexpr (!BF) {
            const float dg = p.degf[v];
#pragma unroll
            for (int q = 0; q < CPL; ++q) x[q] = __float_as_uint(dg > 0.0f ? __uint_as_float(x[q]) * dg : __uint_as_float(x[q]));
        }
        st_cols<CPL>(p.X0 + base, x, ALL, false);
    }
}

using BKernel = void (*)(const BatchParams);

// The wide kernel of (is_bf, variant) for B = 32 * cpl columns; nullptr when it does not apply (the delayed
// form, or a column count that is not 32, 64, 128 or 256).
static BKernel wide_kernel_for(int is_bf, int variant, int B)
{
    if (variant == DAG_DELAYED || B % 32 != 0) return nullptr;
    const int cpl = B / 32;
    const int ci = cpl == 1 ? 0 : cpl == 2 ? 1 : cpl == 4 ? 2 : cpl == 8 ? 3 : -1;
    if (ci < 0) return nullptr;
#define DAG_WIDE(BFV, W8V, VAR) \
    {batched_wide_kernel<BFV, VAR, W8V, 1>, batched_wide_kernel<BFV, VAR, W8V, 2>, batched_wide_kernel<BFV, VAR, W8V, 4>, \
     batched_wide_kernel<BFV, VAR, W8V, 8>}
    static const BKernel table[3][2][4] = {{DAG_WIDE(false, false, DAG_SYNC), DAG_WIDE(false, false, DAG_ASYNC)},
                                           {DAG_WIDE(true, false, DAG_SYNC), DAG_WIDE(true, false, DAG_ASYNC)},
                                           {DAG_WIDE(true, true, DAG_SYNC), DAG_WIDE(true, true, DAG_ASYNC)}};
#undef DAG_WIDE
    return table[is_bf][variant == DAG_SYNC ? 0 : 1][ci];
}

// is_bf: 0 PPR, 1 Bellman-Ford with four-byte weights, 2 with one-byte weights
static BKernel bkernel_for(int is_bf, int variant)
{
    static const BKernel table[3][3] = {
        {batched_kernel<false, DAG_SYNC>, batched_kernel<false, DAG_ASYNC>, batched_kernel<false, DAG_DELAYED>},
        {batched_kernel<true, DAG_SYNC>, batched_kernel<true, DAG_ASYNC>, batched_kernel<true, DAG_DELAYED>},
        {batched_kernel<true, DAG_SYNC, true>, batched_kernel<true, DAG_ASYNC, true>,
         batched_kernel<true, DAG_DELAYED, true>},
    };
    return table[is_bf][variant];
}

// ---------------------------------------------------------------------------
// CUDA graphs of batched launches (dag_plan_set_batched_graph). A launch shape
// (kernel, grid, block, shared memory, control block) is captured once into a
// graph of two nodes: the reset of the control block and the cooperative
// kernel. Every call replays it with its own kernel arguments. Capture runs on
// a private stream (the caller's may be the legacy default stream, which
// cannot be captured); when capture or instantiation fails, the shape is
// marked and its calls launch directly. The cache sits here, keyed by plan,
// and is released by dag_plan_destroy.
// ---------------------------------------------------------------------------
struct BatchGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t knode = nullptr;  // the kernel node, whose arguments each call sets
    bool failed = false;              // capture or instantiation failed: launch directly
};
using ShapeKey = std::tuple<const void*, int, int, size_t, size_t, const void*>;
struct PlanGraphs {
    bool on = true;  // graphs are the default for every plan
    std::map<ShapeKey, BatchGraph> shapes;
};
static std::mutex g_graph_mu;
static std::map<const dag_plan*, PlanGraphs> g_graphs;

static bool batched_graph_on(const dag_plan* plan)
{
    std::lock_guard<std::mutex> lk(g_graph_mu);
    auto it = g_graphs.find(plan);
    return it == g_graphs.end() || it->second.on;  // on unless the plan turned it off
}

// Records the reset and the kernel launch into bg (nothing runs); on any
// failure bg.failed is set and the error state cleared.
static void capture_shape(BatchGraph& bg, const void* k, int nb, int threads, size_t dyn, void* bsync,
                          size_t cbytes, void** args)
{
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        bg.failed = true;
        return;
    }
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    cudaGraphNode_t kn = nullptr;
    const cudaError_t e0 = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e0 != cudaSuccess) set_error(DAG_OK, std::string("batched graph: begin capture: ") + cudaGetErrorString(e0));
    if (e0 == cudaSuccess) {
        const cudaError_t e1 = cudaMemsetAsync(bsync, 0, cbytes, cs);
        const cudaError_t e2 = cudaLaunchCooperativeKernel(k, dim3(nb), dim3(threads), args, dyn, cs);
        const cudaError_t e3 = cudaStreamEndCapture(cs, &g);  // ends capture mode whatever happened
        cudaError_t e4 = cudaErrorUnknown;
        if (e1 == cudaSuccess && e2 == cudaSuccess && e3 == cudaSuccess && g) e4 = cudaGraphInstantiate(&ex, g, 0);
        const cudaError_t bad = e1 != cudaSuccess ? e1 : e2 != cudaSuccess ? e2 : e3 != cudaSuccess ? e3 : e4;
        if (bad != cudaSuccess)  // recorded for dag_last_error_message; the call itself launches directly
            set_error(DAG_OK, std::string("batched graph: capture (memset, launch, end, instantiate ") +
                                  std::to_string((int)e1) + " " + std::to_string((int)e2) + " " +
                                  std::to_string((int)e3) + " " + std::to_string((int)e4) + "): " +
                                  cudaGetErrorString(bad));
        if (e4 == cudaSuccess) {
            size_t cnt = 0;
            if (cudaGraphGetNodes(g, nullptr, &cnt) == cudaSuccess && cnt > 0) {
                std::vector<cudaGraphNode_t> nodes(cnt);
                if (cudaGraphGetNodes(g, nodes.data(), &cnt) == cudaSuccess) {
                    for (size_t i = 0; i < cnt; ++i) {
                        cudaGraphNodeType t;
                        if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel)
                            kn = nodes[i];
                    }
                }
            }
        }
    }
    cudaStreamDestroy(cs);
    if (!kn && ex) {
        size_t cnt = 0;
        cudaGraphGetNodes(g, nullptr, &cnt);
        std::string types;
        std::vector<cudaGraphNode_t> nodes(cnt);
        if (cnt) cudaGraphGetNodes(g, nodes.data(), &cnt);
        for (size_t i = 0; i < cnt; ++i) {
            cudaGraphNodeType t;
            cudaGraphNodeGetType(nodes[i], &t);
            types += " " + std::to_string((int)t);
        }
        set_error(DAG_OK, "batched graph: no kernel node among " + std::to_string(cnt) + " nodes:" + types);
    }
    if (!kn) {
        if (ex) cudaGraphExecDestroy(ex);
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        bg.failed = true;
        return;
    }
    bg.graph = g;
    bg.exec = ex;
    bg.knode = kn;
}

// One batched launch on stream s through the plan's graph of this shape
// (captured on first use), or directly when the shape cannot be captured.
static cudaError_t graph_launch(dag_plan* plan, const void* k, int nb, int threads, size_t dyn, size_t cbytes,
                                void** args, cudaStream_t s, bool* replayed)
{
    *replayed = false;
    std::lock_guard<std::mutex> lk(g_graph_mu);
    BatchGraph& bg = g_graphs[plan].shapes[ShapeKey(k, nb, threads, dyn, cbytes, plan->bsync)];
    if (!bg.exec && !bg.failed) capture_shape(bg, k, nb, threads, dyn, plan->bsync, cbytes, args);
    if (!bg.failed) {
        cudaKernelNodeParams kp{};
        kp.func = const_cast<void*>(k);
        kp.gridDim = dim3(nb);
        kp.blockDim = dim3(threads);
        kp.sharedMemBytes = (unsigned)dyn;
        kp.kernelParams = args;
        kp.extra = nullptr;
        // the replay must run with this call's arguments: if they cannot be set, or the graph
        // cannot be launched, nothing was enqueued, and the shape launches directly from now on
        const cudaError_t ep = cudaGraphExecKernelNodeSetParams(bg.exec, bg.knode, &kp);
        const cudaError_t el = ep == cudaSuccess ? cudaGraphLaunch(bg.exec, s) : ep;
        if (el == cudaSuccess) {
            *replayed = true;
            return cudaSuccess;
        }
        set_error(DAG_OK, std::string("batched graph: replay: ") + cudaGetErrorString(el));
        cudaGetLastError();
        bg.failed = true;
    }
    const cudaError_t e = cudaMemsetAsync(plan->bsync, 0, cbytes, s);
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel(k, dim3(nb), dim3(threads), args, dyn, s);
}

void release_batched_graphs(const dag_plan* plan)
{
    std::lock_guard<std::mutex> lk(g_graph_mu);
    auto it = g_graphs.find(plan);
    if (it == g_graphs.end()) return;
    for (auto& kv : it->second.shapes) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
    }
    g_graphs.erase(it);
}

int launch_batched(dag_plan* plan, int is_bf, int variant, int delta, int max_iters, int B, float d, double tol,
                   const void* V_or_src, const uint32_t* w, void* out, int* iters, dag_batch_stats* st,
                   cudaStream_t s)
{
    const int n = plan->n;
    const int W = (B + 31) / 32;
    const int threads = W * 32;
    if (is_bf) {
        // sources must be vertices of the graph
        std::vector<uint32_t> hs(B);
        DAG_CUDA(cudaMemcpyAsync(hs.data(), V_or_src, (size_t)B * 4, cudaMemcpyDeviceToHost, s));
        DAG_CUDA(cudaStreamSynchronize(s));
        for (int c = 0; c < B; ++c)
            if (hs[c] >= (uint32_t)n) return set_error(DAG_ERR_INVALID, "source outside [0, n)");
    }
    const int dl = (variant == DAG_DELAYED) ? delta : 0;
    size_t dyn = (size_t)(2 * TILE + 1 + (is_bf ? TILE : 0)) * 4 + (size_t)W * dl * 32 * 4;
    BKernel k = bkernel_for(is_bf, variant);
    int threads_launch = threads;
    // the wide kernel's vector accesses want 16-byte aligned column arrays (rows of B values are)
    const bool aligned16 = ((uintptr_t)out & 15u) == 0 && (is_bf || ((uintptr_t)V_or_src & 15u) == 0);
    if (BKernel kw = (plan->batched_wide && aligned16) ? wide_kernel_for(is_bf, variant, B) : nullptr) {
        k = kw;
        threads_launch = NT;
        // s_col, s_end, s_w, the shares' partials, the carries; then FP64 T and linked mass, FP32 sums, last sweeps
        dyn = (size_t)(2 * TILE + 4 + (is_bf ? TILE : 0) + (WIDE_WARPS + 2) * B) * 4 +
              (size_t)B * (16 + 4 * WIDE_WARPS + 4 + 4);
    }
    int max_dyn = 0;
    DAG_CUDA(cudaDeviceGetAttribute(&max_dyn, cudaDevAttrMaxSharedMemoryPerBlockOptin, plan->device));
    if (dyn > (size_t)max_dyn)
        return set_error(DAG_ERR_INVALID, "delta too large for the batched delay buffers in shared memory");
    DAG_CUDA(cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    int per_sm = 0;
    DAG_CUDA(cudaFuncSetAttribute((const void*)k, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    DAG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k, threads_launch, dyn));
    if (per_sm < 1) return set_error(DAG_ERR_INVALID, "batched kernel cannot be resident");
    {
        cudaFuncAttributes fa;
        DAG_CUDA(cudaFuncGetAttributes(&fa, (const void*)k));
        const int rc = set_l1_carveout((const void*)k, plan->device, threads_launch, fa.sharedSizeBytes, dyn, per_sm);
        if (rc) return rc;
    }
    int nb = per_sm * plan->num_sms;
    if (plan->worker_cap > 0 && nb > plan->worker_cap) nb = plan->worker_cap;
    Partition* part = nullptr;
    int rc = get_partition(plan, nb, &part, s, 0);
    if (rc) return rc;
    // workspace: X1 (sync) and the per-column control block
    size_t xbytes = (variant == DAG_SYNC) ? (size_t)n * B * 4 : 0;
    if (xbytes > plan->bx_bytes) {
        cudaFree(plan->bx);
        plan->bx = nullptr;
        plan->bx_bytes = 0;
        if (cudaMalloc(&plan->bx, xbytes) != cudaSuccess) {
            cudaGetLastError();
            return set_error(DAG_ERR_NOMEM, "batched workspace allocation failed");
        }
        plan->bx_bytes = xbytes;
    }
    size_t cbytes = sizeof(SyncBlock) + (size_t)B * (3 + 3 + 1 + 1) * sizeof(double);
    if (cbytes > plan->bsync_bytes) {
        cudaFree(plan->bsync);
        plan->bsync = nullptr;
        plan->bsync_bytes = 0;
        if (cudaMalloc(&plan->bsync, cbytes) != cudaSuccess) {
            cudaGetLastError();
            return set_error(DAG_ERR_NOMEM, "batched control allocation failed");
        }
        plan->bsync_bytes = cbytes;
    }
    const bool use_graph = batched_graph_on(plan);
    if (!use_graph) DAG_CUDA(cudaMemsetAsync(plan->bsync, 0, cbytes, s));  // the graph holds its own reset
    BatchParams p{};
    p.n = n;
    p.B = B;
    p.nblocks = nb;
    p.rowptr = plan->rowptr;
    p.colidx = plan->colidx;
    p.w = is_bf == 1 ? w : nullptr;
    p.w8 = is_bf == 2 ? (const uint8_t*)w : nullptr;
    p.degf = plan->degf;
    p.V = is_bf ? nullptr : (const float*)V_or_src;
    p.src = is_bf ? (const uint32_t*)V_or_src : nullptr;
    p.d = d;
    p.g_coef = d / (float)n;
    p.tol = is_bf ? 0.0 : tol;
    p.max_iters = max_iters;
    p.delta = dl;
    p.X0 = (uint32_t*)out;
    p.X1 = (uint32_t*)plan->bx;
    p.cta_row = part->cta_row;
    p.cta_tile = part->cta_tile;
    p.tile_row = part->tile_row;
    p.tile_nz = part->tile_nz;
    p.sb = (SyncBlock*)plan->bsync;
    double* base = (double*)((char*)plan->bsync + sizeof(SyncBlock));
    p.acc_res = base;
    p.acc_g = base + 3 * B;
    p.gl = base + 6 * B;
    p.T = base + 7 * B;
    p.iters = iters;
    p.timeout_ns = plan->timeout_ns;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (st) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, s);
    }
    void* args[] = {(void*)&p};
    bool replayed = false;
    cudaError_t le = use_graph ? graph_launch(plan, (const void*)k, nb, threads_launch, dyn, cbytes, args, s, &replayed)
                               : cudaLaunchCooperativeKernel((const void*)k, dim3(nb), dim3(threads_launch), args, dyn, s);
    if (le != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        return cuda_check(le, "batched cooperative launch");
    }
    if (!st) return DAG_OK;
    cudaEventRecord(e1, s);
    SyncBlock sb;
    DAG_CUDA(cudaMemcpyAsync(&sb, plan->bsync, sizeof(SyncBlock), cudaMemcpyDeviceToHost, s));
    std::vector<int> hit(B);
    DAG_CUDA(cudaMemcpyAsync(hit.data(), iters, (size_t)B * sizeof(int), cudaMemcpyDeviceToHost, s));
    DAG_CUDA(cudaStreamSynchronize(s));
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int rc2 = DAG_OK;
    if (sb.err) rc2 = sb.err;
    else if (!sb.converged) rc2 = DAG_ERR_NOT_CONVERGED;
    long long colsw = 0;
    for (int c = 0; c < B; ++c) colsw += hit[c];
    st->sweeps = sb.iters;
    st->err = rc2;
    st->ms = ms;
    st->workers = nb;
    st->delta = dl;
    st->column_sweeps = colsw;
    st->graph = replayed ? 1 : 0;
    if (rc2 == DAG_ERR_BARRIER_TIMEOUT) set_error(rc2, "grid barrier wait ran out of time");
    return rc2;
}

}  // namespace dag

extern "C" int dag_plan_set_batched_wide(dag_plan* plan, int32_t on)
{
    if (!plan) return dag::set_error(DAG_ERR_INVALID, "null plan");
    plan->batched_wide = on != 0;
    return DAG_OK;
}

extern "C" int dag_plan_set_batched_graph(dag_plan* plan, int32_t on)
{
    if (!plan) return dag::set_error(DAG_ERR_INVALID, "null plan");
    std::lock_guard<std::mutex> lk(dag::g_graph_mu);
    dag::g_graphs[plan].on = on != 0;
    return DAG_OK;
}
