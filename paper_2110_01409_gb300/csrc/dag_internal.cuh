// Internal declarations shared by the libdag.so translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/dag.h"

namespace dag {

// ---------------------------------------------------------------------------
// Launch shape of the persistent sweep kernels.
// A CTA walks its vertex block in merge-path tiles of TILE items, where an item
// is either one in-edge or one row end (Merrill & Garland, "Merge-based
// parallel sparse matrix-vector multiplication", SC 2016). Tiles follow vertex
// order, so the rows a tile completes are contiguous and a delay buffer of
// consecutive rows can be flushed with coalesced stores.
// ---------------------------------------------------------------------------
#ifndef DAG_NT
#define DAG_NT 256
#endif
#ifndef DAG_IPT
#define DAG_IPT 7
#endif
#ifndef DAG_MINBLOCKS
#define DAG_MINBLOCKS 4
#endif
constexpr int NT = DAG_NT;        // threads per CTA
constexpr int IPT = DAG_IPT;      // items per thread per tile (odd: fewer bank conflicts in the walk)
constexpr int MINBLOCKS = DAG_MINBLOCKS;  // CTAs per SM the register budget is sized for
constexpr int TILE = NT * IPT;    // items per tile
constexpr int NWARP = NT / 32;
constexpr int RING = 3;           // tile staging slots of the sweep kernel (tiles t, t+1, t+2)
constexpr int GSTRIPES = 32;      // stripes of the live dangling/global-sum accumulator
constexpr int GSTRIDE = 16;       // 8-byte words between stripes: one 128-byte L2 line each, since
                                  // atomics to stripes sharing a line serialise on it

enum Mode { MODE_PR = 0, MODE_PRW = 1, MODE_ADJ = 2, MODE_BF = 3, MODE_BF8 = 4 };  // BF8: uint8 weights

// How the delayed form reads other blocks' values (see dag.h, DAG_READ_*).
enum ReadMode { READ_CACHED_REFRESH = 0, READ_COHERENT = 1, READ_CACHED = 2 };

constexpr uint32_t INF = 0xFFFFFFFFu;

// Default time limit of every device-side wait (grid barrier, staging ring).
constexpr long long DEFAULT_TIMEOUT_NS = 2000000000LL;

// Device-side control block of one solve (lives in the plan's workspace,
// zeroed before each launch).
struct __align__(128) SyncBlock {
    unsigned long long arrive;   // grid-barrier arrivals, monotone within a launch
    int err;                     // first error (DAG_ERR_*), 0 while fine
    int iters;                   // sweeps run
    double residual;             // last sweep's residual
    long long flushes;           // delay-buffer flushes
    int converged;
    int pad0;
    double T;                    // teleport total (PageRank)
    double acc_res[3];           // per-sweep residual sums, slot = sweep % 3 (init = slot 2)
    double acc_g[3];             // per-sweep global sums (N for PageRank, sum lambda for the adjoint)
    long long edges;             // edges processed (frontier sweeps)
    int fr_cnt[3];               // frontier, shared sweeps: tiles in the sweep's list, slot = sweep % 3
    int fr_head[3];              //   tiles claimed so far
    int fr_nchg[3];              //   rows logged as changed
    int pad2[3];
    alignas(128) long long stripe[GSTRIPES * GSTRIDE];  // live global sum, fixed point (async / delayed)
};

// Parameters of one sweep launch.
struct SweepParams {
    int n;
    int nblocks;
    const int* rowptr;
    const int* colidx;
    const float* val;       // per-edge P (PRW, ADJ)
    const uint32_t* w;      // per-edge weight (BF)
    const uint8_t* w8;      // per-edge weight, one byte (BF8)
    const float* degf;      // out-degree as float (PR, PRW: dangling when 0; ADJ: row length of out-CSR)
    const float* base;      // per-row base vector: teleport (PR/PRW) or c (ADJ); NULL = uniform
    float base_scale;       // (1-d) for PageRank, 1 for the adjoint
    float uniform_base;     // base when `base` is NULL: (1-d)/n
    float d;
    float g_coef;           // d/n: weight of the global term per row
    double tol;
    int max_iters;
    int delta;              // delayed buffer size (rows); 0 for sync/async
    int buf_cap;            // delay buffer capacity (elements of dynamic shared memory)
    int buf_clamped;        // 1: capacity below delta - 1 + TILE (shared memory limit): flush when full
    uint32_t src;           // BF source
    // state (two buffers for sync)
    void* x0;
    void* x1;
    // partition
    const int* cta_row;     // [nblocks+1]
    const int* cta_tile;    // [nblocks+1]
    const int* tile_row;    // [tiles+1]
    const int* tile_nz;     // [tiles+1]
    // control
    SyncBlock* sync;
    long long timeout_ns;
    int skip_barrier_cta0;  // test hook
    int stall_fill;         // test hook: CTA 0's first staging wait cannot complete
    int read_mode;          // ReadMode (delayed form)
    int local_read;         // delayed form: read own unflushed rows from the buffer (Sec. III-C)
    int own_l1;             // async form: own block through L1, other blocks through L2
    // frontier Bellman-Ford: a tile runs in sweep s only when fr_act[tile] == s
    int frontier;
    const int* fr_orow;     // out-CSR row pointers [n+1]
    const int* fr_otile;    // per out-edge: tile of its in-CSR position
    const int* fr_oend;     // per out-edge: tile that ends its target's row
    int* fr_act;            // [tiles] sweep stamp of the last mark (zero before the first sweep)
    int* fr_alist;          // [tiles] the CTAs' active tiles of the current sweep
    int* fr_chg;            // [n] the CTAs' rows that changed in the current sweep
    int* fr_glist;          // [tiles] shared sweeps: the tiles any CTA may claim
    int* fr_gchg;           // [n + tiles] shared sweeps: rows logged as changed (a row may repeat)
    float fr_sparse;        // warp-tile frontier: a sweep is sparse after one whose marks <= fr_sparse per tile
    // warp workers (sweep_warp.cu): cta_row / cta_tile hold each warp's first row / tile
    int warp;                     // 1: one worker per warp
    int ordered;                  // 1: warps take the tiles of the whole merge path in turn (async form)
    int ntiles;                   //    tiles of that merge path; wpub then holds one word per tile
    int shard;                    // 1: one synchronous sweep of a row range, x0 / x1 given (sweep_rows)
    double shard_T, shard_N;      //    teleport total and mass on vertices with out-edges of x0's iterate
    unsigned long long* wpub;     // [warps] partial of the row each run leaves unfinished, with its sweep stamp
    // init / output
    const float* init;      // warm start (PR) or nullptr
    void* out;              // float r / lambda, or uint32 dist
    float* aux_out;         // ADJ: (M^T lambda)_u of the last sweep, nullable
};

// Partition of one launch shape, cached per plan.
struct Partition {
    int nblocks = 0;
    int row_cap = 0;          // > 0: a tile completes at most this many rows (delayed sweeps, small delta)
    int tiles = 0;
    int max_rows = 0;
    int* cta_row = nullptr;   // device [nblocks+1]
    int* cta_tile = nullptr;  // device [nblocks+1]
    int* tile_row = nullptr;  // device [tiles+1]
    int* tile_nz = nullptr;   // device [tiles+1]
    // frontier maps (built on first use)
    int* fr_otile = nullptr;  // device [m]
    int* fr_oend = nullptr;   // device [m]
    int* fr_act = nullptr;    // device [tiles]
    int* fr_alist = nullptr;  // device [tiles]
    int* fr_chg = nullptr;    // device [n]
    int* fr_glist = nullptr;  // device [tiles]
    int* fr_gchg = nullptr;   // device [n + tiles]
    unsigned long long* wpub = nullptr;  // warp workers: [nblocks] published partials
    unsigned long long* tpub = nullptr;  // ordered warp sweeps: [tiles] published partials (built on first use)
};

}  // namespace dag

struct dag_plan {
    int n = 0;
    long long m = 0;
    const int* rowptr = nullptr;
    const int* colidx = nullptr;
    int device = 0;
    int num_sms = 0;
    long long timeout_ns = dag::DEFAULT_TIMEOUT_NS;
    int skip_barrier_once = 0;
    int stall_staging_once = 0;
    long long skip_timeout_ns = 0;
    int worker_cap = 0;       // > 0: at most this many CTAs per solve (more rows per CTA)
    int warp_ipt = 7;         // items per lane of the warp-worker tiles (5, 7 or 11)
    float fr_sparse_warp = 1.0f;  // warp-tile frontier: marks per tile at or below which the next sweep is sparse
    bool batched_wide = true;     // batched sync / async solves of 32, 64, 128 or 256 columns: the wide kernel
    // per-vertex data
    int* outdeg = nullptr;    // [n]
    float* degf = nullptr;    // [n]
    // workspace
    void* x0 = nullptr;       // [n] 4-byte values
    void* x1 = nullptr;       // [n]
    dag::SyncBlock* sync = nullptr;
    float* scratch_f = nullptr; // [n] float scratch (adjoint aux)
    int* fr_orow = nullptr;   // [n+1] out-CSR row pointers (frontier sweeps, built on first use)
    int* nw_perm = nullptr;   // [m] in-edge of each out-edge, targets ascending (weight normalisation, first use)
    int* nw_hubs = nullptr;   // sources of more than NW_HUB out-edges (summed by a whole block)
    int nw_nhubs = 0;
    void* grad_coef = nullptr;  // [n] float2 (d r_u / s_u, (M^T lambda)_u) of the edge gradients, first use
    std::map<long long, dag::Partition> parts;  // key: nblocks | row_cap << 32
    std::map<std::tuple<int, int, int, int>, dag::Partition> range_parts;  // (warps, tile, lo, hi)
    // batched workspace (grown on demand)
    void* bx = nullptr;
    size_t bx_bytes = 0;
    void* bsync = nullptr;
    size_t bsync_bytes = 0;
};

namespace dag {

// error plumbing (api.cu)
int set_error(int code, const std::string& msg);
int cuda_check(cudaError_t e, const char* what);
#define DAG_CUDA(call)                                            \
    do {                                                          \
        cudaError_t e__ = (call);                                 \
        if (e__ != cudaSuccess) return ::dag::cuda_check(e__, #call); \
    } while (0)

// plan.cu
int get_partition(dag_plan* plan, int nblocks, Partition** out, cudaStream_t s, int row_cap);

// The frontier maps of a partition (and the plan's out-CSR row pointers), built once.
int frontier_maps(dag_plan* plan, Partition* part, cudaStream_t s, bool with_end = true);
int max_workers(dag_plan* plan, int mode, int variant, int buf_cap_elems, int* out);

// sweep.cu
int launch_sweep(dag_plan* plan, int mode, int variant, int delta, SweepParams& p, cudaStream_t s,
                 int* out_nblocks);
int sweep_shape(dag_plan* plan, int mode, int variant, int delta, int* nb_out, int* cap_out, Partition** part_out,
                cudaStream_t s, int* clamped_out = nullptr);
// The launch-shape rule of sweep_shape with the partition built by the caller
// (`partition(nblocks, &max_rows)`), for launches without a plan's workspace.
int settle_shape(dag_plan* plan, int mode, int variant, int delta,
                 const std::function<int(int nblocks, int* max_rows)>& partition, int* nb_out, int* cap_out,
                 int* clamped_out);
// Rows a tile of a delayed sweep may complete (0: no cap): a buffer of delta
// rows can only be flushed at a tile end.
inline int delayed_row_cap(int variant, int delta) { return (variant == DAG_DELAYED && delta > 0 && delta < TILE) ? delta : 0; }

const void* sweep_kernel_ptr(int mode, int variant);
// Dynamic shared memory of a sweep launch in front of the delay buffer: the
// TMA kernel's tile staging ring (asynchronous form), 0 for the other forms.
size_t sweep_ring_bytes(int mode, int variant);

// sweep_tma.cu: the asynchronous form's TMA-staged kernel and its ring size.
const void* sweep_tma_kernel_ptr(int mode, bool frontier);
size_t sweep_tma_ring_bytes(int mode);
// Smallest shared-memory carveout of kernel k that keeps per_sm CTAs of
// (static_smem + dyn) bytes resident; the rest of the SM's array is L1.
int set_l1_carveout(const void* k, int device, int threads, size_t static_smem, size_t dyn, int per_sm);

// Warp workers: the whole merge path cut into tiles of `tile` items, warp w
// of W taking tiles [floor(w T / W), floor((w+1) T / W)); cta_tile / cta_row
// hold each warp's first tile / first owned row (the partition's nblocks is W).
int get_warp_partition(dag_plan* plan, int W, int tile, Partition** out, cudaStream_t s);
// The same over the merge path of rows [lo, hi) only (row-range sweeps).
int get_warp_partition_range(dag_plan* plan, int W, int tile, int lo, int hi, Partition** out, cudaStream_t s);
int sweep_rows(dag_plan* plan, int mode, int lo, int hi, SweepParams& p, double* d_sums, cudaStream_t s);
// sweep_warp.cu
const void* sweep_warp_kernel_ptr(int mode, int variant, int ipt);
const void* sweep_ordered_kernel_ptr(int mode, int ipt);
const void* sweep_warp_frontier_kernel_ptr(int mode, int ipt, bool ordered);
int warp_frontier_maps(dag_plan* plan, int mode, cudaStream_t s);
int launch_warp_sweep(dag_plan* plan, int mode, int variant, int delta, SweepParams& p, cudaStream_t s,
                      int* out_nblocks);

// plan.cu kernels reused by the allocation-free entry point (noalloc.cu)
__global__ void k_check_rowptr(const int* rowptr, int n, long long m, int* bad);
__global__ void k_out_degree(const int* colidx, long long m, int n, int* outdeg, int* bad);
__global__ void k_degf(const int* outdeg, float* degf, int n);
__global__ void k_cta_rows(const int* rowptr, int n, long long total, int P, int* cta_row, int row_w);
constexpr int CT_THREADS = 1024;  // threads of k_cta_tiles (one CTA)
__global__ void k_cta_tiles(const int* rowptr, const int* cta_row, int P, int* cta_tile, int* max_rows);
__global__ void k_tile_coords(const int* rowptr, int n, long long m, const int* cta_row, const int* cta_tile,
                              int P, int tiles, int* tile_row, int* tile_nz);

// batched.cu
int launch_batched(dag_plan* plan, int is_bf, int variant, int delta, int max_iters, int B, float d,
                   double tol, const void* V_or_src, const uint32_t* w, void* out, int* iters,
                   dag_batch_stats* st, cudaStream_t s);

// adjoint.cu
int launch_edge_grad(dag_plan* in_plan, float d, const float* val, const float* s_norm, const float* rank,
                     const float* lambda, const float* mt, float* grad_w, float* grad_t, cudaStream_t st);
int launch_transpose(dag_plan* plan, int* out_rowptr, int* out_colidx, int* perm, cudaStream_t s);
int launch_normalize(dag_plan* plan, const float* w, float* val, float* s_out, cudaStream_t s);

}  // namespace dag

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
#ifdef __CUDACC__
namespace dag {

__device__ __forceinline__ int ld_stream_i32(const int* p)
{
    int v;
    asm volatile("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float ld_stream_f32(const float* p)
{
    float v;
    asm volatile("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ uint32_t ld_stream_u32(const uint32_t* p)
{
    uint32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
// L2 eviction policies. The per-edge streams (colidx, weights, edge values) are
// read once per sweep and are larger than L2: they go first, so that the
// per-vertex arrays every tile rereads (row ends, out-degrees, the state
// vector) stay resident in L2 across sweeps.
__device__ __forceinline__ uint64_t policy_evict_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_last()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint32_t ld_edge_b32(const void* p, uint64_t pol)
{
    uint32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ uint32_t ld_edge_u8(const uint8_t* p, uint64_t pol)
{
    uint32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.u8 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ uint32_t ld_vertex_b32(const void* p, uint64_t pol)
{
    uint32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ uint32_t ld_weak_keep_b32(const void* p, uint64_t pol)
{
    uint32_t v;
    asm volatile("ld.global.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_relaxed_keep_b32(const void* p, uint64_t pol)
{
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol) : "memory");
    return v;
}
// Weak load: may hit in L1. Used for the previous iterate in the synchronous
// form (no CTA writes it during the sweep) and for the delayed form's view of
// the live array, which may lag other CTAs' flushes until this SM's next
// acquire (a flush or the grid barrier).
__device__ __forceinline__ uint32_t ld_weak_b32(const void* p)
{
    uint32_t v;
    asm volatile("ld.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// Relaxed gpu-scope load: served by L2, the point of coherence, so it sees
// other CTAs' latest stores. Used by the in-place (async / delayed) forms.
__device__ __forceinline__ uint32_t ld_relaxed_b32(const void* p)
{
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_b32(void* p, uint32_t v)
{
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_weak_b32(void* p, uint32_t v)
{
    asm volatile("st.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ double ld_relaxed_f64(const double* p)
{
    double v;
    asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ long long ld_relaxed_i64(const long long* p)
{
    long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed_i32(const int* p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier for a co-resident (cooperative) grid. Arrivals count up
// monotonically; after its k-th barrier a CTA waits for k * nblocks arrivals.
// The wait is bounded: past timeout_ns, or when another CTA has already
// recorded an error, it records DAG_ERR_BARRIER_TIMEOUT (first error wins) and
// returns false. Every thread of the CTA gets the same answer.
__device__ __forceinline__ bool grid_barrier(SyncBlock* sb, unsigned nblocks, unsigned long long& target,
                                             long long timeout_ns)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        target += nblocks;
        __threadfence();
        atomicAdd(&sb->arrive, 1ULL);
        int ok = 1;
        unsigned long long t0 = globaltimer_ns();
        unsigned spins = 0;
        while (ld_acquire_u64(&sb->arrive) < target) {
            if (ld_relaxed_i32(&sb->err) != 0) { ok = 0; break; }
            if ((++spins & 31u) == 0 && (long long)(globaltimer_ns() - t0) > timeout_ns) {
                atomicCAS(&sb->err, 0, DAG_ERR_BARRIER_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(100);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace dag
#endif
