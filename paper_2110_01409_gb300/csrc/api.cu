// C ABI entry points of libdag.so (declared in include/dag.h): argument
// checks, launch of the persistent sweep, timing and status read-back.
#include <cmath>
#include <cstdio>
#include <string>

#include "dag_internal.cuh"
#include "devmem.cuh"

namespace dag {

static thread_local std::string g_last_error;

int set_error(int code, const std::string& msg)
{
    g_last_error = msg;
    return code;
}

int cuda_check(cudaError_t e, const char* what)
{
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return DAG_ERR_NOMEM;
    return DAG_ERR_CUDA;
}

namespace {

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    bool on = false;
    void start(cudaStream_t s, bool want)
    {
        on = want;
        if (!on) return;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, s);
    }
    void stop(cudaStream_t s)
    {
        if (on) cudaEventRecord(b, s);
    }
    float ms()
    {
        float x = 0.0f;
        if (on) cudaEventElapsedTime(&x, a, b);
        return x;
    }
    ~Timer()
    {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

// Reads the device status of a finished solve into h (waits for the stream).
int finish_solve(dag_plan* plan, int nblocks, int delta, Timer& tm, cudaStream_t s, dag_stats* h, bool frontier = false)
{
    SyncBlock sb;
    DAG_CUDA(cudaMemcpyAsync(&sb, plan->sync, sizeof(SyncBlock), cudaMemcpyDeviceToHost, s));
    DAG_CUDA(cudaStreamSynchronize(s));
    DAG_CUDA(cudaGetLastError());
    int rc = DAG_OK;
    if (sb.err) rc = sb.err;
    else if (!sb.converged) rc = DAG_ERR_NOT_CONVERGED;
    if (h) {
        h->iters = sb.iters;
        h->err = rc;
        h->residual = sb.residual;
        h->ms = tm.ms();
        h->workers = nblocks;
        h->delta = delta;
        h->flushes = sb.flushes;
        h->edges_processed = frontier ? sb.edges : (long long)sb.iters * plan->m;
    }
    if (rc == DAG_ERR_BARRIER_TIMEOUT) set_error(rc, "grid barrier wait ran out of time");
    else if (rc == DAG_ERR_NOT_CONVERGED) set_error(rc, "max_iters reached before the stopping rule");
    return rc;
}

int read_mode_of(int flags)
{
    if (flags & DAG_READ_COHERENT) return READ_COHERENT;
    if (flags & DAG_READ_CACHED) return READ_CACHED;
    return READ_CACHED_REFRESH;
}

int check_variant(int variant, int delta, int max_iters)
{
    if (variant < DAG_SYNC || variant > DAG_DELAYED) return set_error(DAG_ERR_INVALID, "unknown variant");
    if (delta < 0) return set_error(DAG_ERR_INVALID, "delta must be >= 0");
    if (max_iters < 1) return set_error(DAG_ERR_INVALID, "max_iters must be >= 1");
    return DAG_OK;
}

}  // namespace
}  // namespace dag

using namespace dag;

extern "C" const char* dag_strerror(int code)
{
    switch (code) {
    case DAG_OK: return "ok";
    case DAG_ERR_INVALID: return "invalid argument";
    case DAG_ERR_NOT_CONVERGED: return "not converged within max_iters";
    case DAG_ERR_BARRIER_TIMEOUT: return "grid barrier timeout";
    case DAG_ERR_CUDA: return "CUDA error";
    case DAG_ERR_NOMEM: return "out of device memory";
    default: return "unknown error";
    }
}

extern "C" const char* dag_last_error_message(void) { return g_last_error.c_str(); }

extern "C" int dag_workers(dag_plan* plan, dag_variant variant, int32_t delta, int32_t* out_workers)
{
    if (!plan || !out_workers) return set_error(DAG_ERR_INVALID, "null argument");
    int rc = check_variant(variant, delta, 1);
    if (rc) return rc;
    if (variant == DAG_DELAYED && delta == 0) variant = DAG_ASYNC;
    int nb = 0, cap = 0;
    Partition* part = nullptr;
    rc = sweep_shape(plan, MODE_PR, variant, delta, &nb, &cap, &part, 0);
    if (rc) return rc;
    *out_workers = nb;
    return DAG_OK;
}

extern "C" int dag_pagerank(dag_plan* plan, float d, double tol, dag_variant variant, int32_t delta,
                            int32_t max_iters, const float* d_teleport, const float* d_val, float* d_rank,
                            int32_t flags, dag_stats* h_stats, void* stream)
{
    if (!plan || !d_rank) return set_error(DAG_ERR_INVALID, "null argument");
    if (!(d > 0.0f && d < 1.0f)) return set_error(DAG_ERR_INVALID, "d must lie in (0, 1)");
    if (!(tol > 0.0) || std::isnan(tol)) return set_error(DAG_ERR_INVALID, "tol must be > 0");
    if (flags & DAG_SSSP_FRONTIER) return set_error(DAG_ERR_INVALID, "the frontier is a Bellman-Ford flag");
    int rc = check_variant(variant, delta, max_iters);
    if (rc) return rc;
    int var = variant;
    if (var == DAG_DELAYED && delta == 0) var = DAG_ASYNC;
    cudaStream_t s = (cudaStream_t)stream;
    SweepParams p{};
    p.n = plan->n;
    p.rowptr = plan->rowptr;
    p.colidx = plan->colidx;
    p.val = d_val;
    p.degf = plan->degf;
    p.base = d_teleport;
    p.base_scale = 1.0f - d;
    p.uniform_base = (1.0f - d) / (float)plan->n;
    p.d = d;
    p.g_coef = d / (float)plan->n;
    p.tol = tol;
    p.max_iters = max_iters;
    p.x0 = plan->x0;
    p.x1 = plan->x1;
    p.init = (flags & DAG_PR_WARM_START) ? d_rank : nullptr;
    p.out = d_rank;
    p.read_mode = read_mode_of(flags);
    p.local_read = (flags & DAG_READ_LOCAL) ? 1 : 0;
    p.own_l1 = (flags & DAG_READ_OWN_L1) ? 1 : 0;
    p.warp = (flags & (DAG_WARP_WORKERS | DAG_WARP_ORDERED)) ? 1 : 0;
    p.ordered = (flags & DAG_WARP_ORDERED) ? 1 : 0;
    Timer tm;
    tm.start(s, h_stats != nullptr);
    int nb = 0;
    rc = launch_sweep(plan, d_val ? MODE_PRW : MODE_PR, var, delta, p, s, &nb);
    if (rc) return rc;
    tm.stop(s);
    if (!h_stats) return DAG_OK;
    return finish_solve(plan, nb, var == DAG_DELAYED ? delta : 0, tm, s, h_stats);
}

namespace dag {
namespace {
int sssp_impl(dag_plan* plan, uint32_t src, int variant, int delta, int max_iters, const uint32_t* w,
              const uint8_t* w8, uint32_t* dist, int flags, dag_stats* h_stats, cudaStream_t s)
{
    if (!plan || !dist || (plan->m > 0 && !w && !w8)) return set_error(DAG_ERR_INVALID, "null argument");
    if (src >= (uint32_t)plan->n) return set_error(DAG_ERR_INVALID, "source outside [0, n)");
    int rc = check_variant(variant, delta, max_iters);
    if (rc) return rc;
    int var = variant;
    if (var == DAG_DELAYED && delta == 0) var = DAG_ASYNC;
    SweepParams p{};
    p.n = plan->n;
    p.rowptr = plan->rowptr;
    p.colidx = plan->colidx;
    p.w = w;
    p.w8 = w8;
    p.degf = plan->degf;
    p.tol = 0.0;
    p.max_iters = max_iters;
    p.src = src;
    p.x0 = plan->x0;
    p.x1 = plan->x1;
    p.out = dist;
    p.read_mode = read_mode_of(flags);
    p.local_read = (flags & DAG_READ_LOCAL) ? 1 : 0;
    p.own_l1 = (flags & DAG_READ_OWN_L1) ? 1 : 0;
    p.frontier = (flags & DAG_SSSP_FRONTIER) ? 1 : 0;
    p.warp = (flags & (DAG_WARP_WORKERS | DAG_WARP_ORDERED)) ? 1 : 0;
    p.ordered = (flags & DAG_WARP_ORDERED) ? 1 : 0;
    if (p.frontier && var == DAG_DELAYED)
        return set_error(DAG_ERR_INVALID, "the frontier runs the synchronous and asynchronous forms (delta 0)");
    if (p.frontier && p.warp && var != DAG_ASYNC)
        return set_error(DAG_ERR_INVALID, "the warp-tile frontier runs the asynchronous form");
    if (p.frontier) {  // the frontier maps of this launch shape are built (once) outside the timed solve
        if (p.warp) {
            rc = warp_frontier_maps(plan, w8 ? MODE_BF8 : MODE_BF, s);
        } else {
            int nb0 = 0, cap0 = 0;
            Partition* part = nullptr;
            rc = sweep_shape(plan, w8 ? MODE_BF8 : MODE_BF, var, delta, &nb0, &cap0, &part, s);
            if (rc == DAG_OK) rc = frontier_maps(plan, part, s);
        }
        if (rc) return rc;
    }
    Timer tm;
    tm.start(s, h_stats != nullptr);
    int nb = 0;
    rc = launch_sweep(plan, w8 ? MODE_BF8 : MODE_BF, var, delta, p, s, &nb);
    if (rc) return rc;
    tm.stop(s);
    if (!h_stats) return DAG_OK;
    return finish_solve(plan, nb, var == DAG_DELAYED ? delta : 0, tm, s, h_stats, p.frontier != 0);
}
}  // namespace
}  // namespace dag

extern "C" int32_t dag_tile_items(void) { return TILE; }

namespace dag {
__global__ void k_copy_status(const SyncBlock* sb, int32_t* out)
{
    out[0] = sb->err;
    out[1] = sb->converged;
    out[2] = sb->iters;
}
}  // namespace dag

extern "C" int dag_plan_last_status(const dag_plan* plan, int32_t* d_status, void* stream)
{
    if (!plan || !d_status) return set_error(DAG_ERR_INVALID, "null argument");
    k_copy_status<<<1, 1, 0, (cudaStream_t)stream>>>(plan->sync, d_status);
    DAG_CUDA(cudaGetLastError());
    return DAG_OK;
}

extern "C" int dag_sssp(dag_plan* plan, uint32_t src, dag_variant variant, int32_t delta, int32_t max_iters,
                        const uint32_t* d_w, uint32_t* d_dist, int32_t flags, dag_stats* h_stats, void* stream)
{
    if (plan && plan->m > 0 && !d_w) return set_error(DAG_ERR_INVALID, "null weights");
    return sssp_impl(plan, src, variant, delta, max_iters, d_w, nullptr, d_dist, flags, h_stats, (cudaStream_t)stream);
}

extern "C" int dag_sssp_u8(dag_plan* plan, uint32_t src, dag_variant variant, int32_t delta, int32_t max_iters,
                           const uint8_t* d_w8, uint32_t* d_dist, int32_t flags, dag_stats* h_stats, void* stream)
{
    if (plan && plan->m > 0 && !d_w8) return set_error(DAG_ERR_INVALID, "null weights");
    return sssp_impl(plan, src, variant, delta, max_iters, nullptr, d_w8, d_dist, flags, h_stats,
                     (cudaStream_t)stream);
}

extern "C" int dag_pagerank_adjoint(dag_plan* in_plan, dag_plan* out_plan, float d, double tol,
                                    dag_variant variant, int32_t delta, int32_t max_iters, const float* d_val,
                                    const float* d_val_out, const float* d_s, const float* d_rank,
                                    const float* d_c, float* d_grad_w, float* d_grad_t, float* d_lambda,
                                    int32_t flags, dag_stats* h_stats, void* stream)
{
    if (!in_plan || !out_plan || !d_c || !d_rank || !d_s) return set_error(DAG_ERR_INVALID, "null argument");
    if (in_plan->n != out_plan->n || in_plan->m != out_plan->m)
        return set_error(DAG_ERR_INVALID, "in_plan and out_plan describe different graphs");
    if (in_plan->m > 0 && (!d_val_out || (d_grad_w && !d_val)))
        return set_error(DAG_ERR_INVALID, "null edge values");
    if (!(d > 0.0f && d < 1.0f)) return set_error(DAG_ERR_INVALID, "d must lie in (0, 1)");
    if (!(tol > 0.0)) return set_error(DAG_ERR_INVALID, "tol must be > 0");
    if (flags & (DAG_PR_WARM_START | DAG_SSSP_FRONTIER | DAG_READ_LOCAL))
        return set_error(DAG_ERR_INVALID, "flag not taken by the adjoint");
    int rc = check_variant(variant, delta, max_iters);
    if (rc) return rc;
    int var = variant;
    if (var == DAG_DELAYED && delta == 0) var = DAG_ASYNC;
    cudaStream_t s = (cudaStream_t)stream;
    float* lam = d_lambda;
    float* lam_tmp = nullptr;
    if (!lam) {
        DAG_CUDA(dev_alloc(&lam_tmp, (size_t)in_plan->n * sizeof(float)));
        lam = lam_tmp;
    }
    SweepParams p{};
    p.n = out_plan->n;
    p.rowptr = out_plan->rowptr;
    p.colidx = out_plan->colidx;
    p.val = d_val_out;
    p.degf = in_plan->degf;  // forward out-degree = out-CSR row length: dangling test
    p.base = d_c;
    p.base_scale = 1.0f;
    p.d = d;
    p.g_coef = d / (float)out_plan->n;
    p.tol = tol;
    p.max_iters = max_iters;
    p.x0 = out_plan->x0;
    p.x1 = out_plan->x1;
    p.out = lam;
    p.aux_out = in_plan->scratch_f;  // (M^T lambda)_u of the last sweep
    p.read_mode = read_mode_of(flags);
    p.own_l1 = (flags & DAG_READ_OWN_L1) ? 1 : 0;
    p.warp = (flags & (DAG_WARP_WORKERS | DAG_WARP_ORDERED)) ? 1 : 0;
    p.ordered = (flags & DAG_WARP_ORDERED) ? 1 : 0;
    Timer tm;
    tm.start(s, true);
    int nb = 0;
    rc = launch_sweep(out_plan, MODE_ADJ, var, delta, p, s, &nb);
    if (rc) {
        if (lam_tmp) dev_free(lam_tmp);
        return rc;
    }
    rc = launch_edge_grad(in_plan, d, d_val, d_s, d_rank, lam, in_plan->scratch_f, d_grad_w, d_grad_t, s);
    tm.stop(s);
    int rc2 = finish_solve(out_plan, nb, var == DAG_DELAYED ? delta : 0, tm, s, h_stats);
    if (lam_tmp) dev_free(lam_tmp);
    return rc ? rc : rc2;
}

extern "C" int dag_ppr_batched(dag_plan* plan, float d, double tol, dag_variant variant, int32_t delta,
                               int32_t max_iters, int32_t B, const float* d_V, float* d_R, int32_t* d_iters,
                               dag_batch_stats* h_stats, void* stream)
{
    if (!plan || !d_V || !d_R || !d_iters) return set_error(DAG_ERR_INVALID, "null argument");
    if (B < 1 || B > 1024) return set_error(DAG_ERR_INVALID, "B must lie in [1, 1024]");
    if (!(d > 0.0f && d < 1.0f)) return set_error(DAG_ERR_INVALID, "d must lie in (0, 1)");
    if (!(tol > 0.0)) return set_error(DAG_ERR_INVALID, "tol must be > 0");
    int rc = check_variant(variant, delta, max_iters);
    if (rc) return rc;
    int var = variant;
    if (var == DAG_DELAYED && delta == 0) var = DAG_ASYNC;
    return launch_batched(plan, 0, var, delta, max_iters, B, d, tol, d_V, nullptr, d_R, d_iters, h_stats,
                          (cudaStream_t)stream);
}

namespace dag {
namespace {
int sssp_batched_impl(dag_plan* plan, int variant, int delta, int max_iters, int B, const uint32_t* d_src,
                      const void* d_w, int wbytes, uint32_t* d_D, int32_t* d_iters, dag_batch_stats* h_stats,
                      cudaStream_t s)
{
    if (!plan || !d_src || !d_D || !d_iters || (plan->m > 0 && !d_w))
        return set_error(DAG_ERR_INVALID, "null argument");
    if (B < 1 || B > 1024) return set_error(DAG_ERR_INVALID, "B must lie in [1, 1024]");
    int rc = check_variant(variant, delta, max_iters);
    if (rc) return rc;
    int var = variant;
    if (var == DAG_DELAYED && delta == 0) var = DAG_ASYNC;
    return launch_batched(plan, wbytes == 1 ? 2 : 1, var, delta, max_iters, B, 0.0f, 0.0, d_src,
                          (const uint32_t*)d_w, d_D, d_iters, h_stats, s);
}
}  // namespace
}  // namespace dag

extern "C" int dag_sssp_batched(dag_plan* plan, dag_variant variant, int32_t delta, int32_t max_iters, int32_t B,
                                const uint32_t* d_src, const uint32_t* d_w, uint32_t* d_D, int32_t* d_iters,
                                dag_batch_stats* h_stats, void* stream)
{
    return sssp_batched_impl(plan, variant, delta, max_iters, B, d_src, d_w, 4, d_D, d_iters, h_stats,
                             (cudaStream_t)stream);
}

extern "C" int dag_sssp_batched_u8(dag_plan* plan, dag_variant variant, int32_t delta, int32_t max_iters, int32_t B,
                                   const uint32_t* d_src, const uint8_t* d_w8, uint32_t* d_D, int32_t* d_iters,
                                   dag_batch_stats* h_stats, void* stream)
{
    return sssp_batched_impl(plan, variant, delta, max_iters, B, d_src, d_w8, 1, d_D, d_iters, h_stats,
                             (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// Row-range sweeps (row sharding across GPUs) and the state conversions
// ---------------------------------------------------------------------------
namespace dag {
__global__ void k_rank_to_state(const float* r, const float* degf, int n, float* x, double* linked)
{
    double part = 0.0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const float dg = degf[v];
        x[v] = dg > 0.0f ? r[v] / dg : r[v];
        if (dg > 0.0f) part += (double)r[v];
    }
    if (linked) {
        part = warp_sum(part);
        if ((threadIdx.x & 31) == 0 && part != 0.0) atomicAdd(linked, part);
    }
}
__global__ void k_state_to_rank(const float* x, const float* degf, int n, float* r)
{
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const float dg = degf[v];
        r[v] = dg > 0.0f ? x[v] * dg : x[v];
    }
}
}  // namespace dag

extern "C" int dag_rank_to_state(const dag_plan* plan, const float* d_r, float* d_x, double* d_linked_mass,
                                 void* stream)
{
    if (!plan || !d_r || !d_x) return set_error(DAG_ERR_INVALID, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    if (d_linked_mass) DAG_CUDA(cudaMemsetAsync(d_linked_mass, 0, sizeof(double), s));
    k_rank_to_state<<<1024, 256, 0, s>>>(d_r, plan->degf, plan->n, d_x, d_linked_mass);
    DAG_CUDA(cudaGetLastError());
    return DAG_OK;
}

extern "C" int dag_state_to_rank(const dag_plan* plan, const float* d_x, float* d_r, void* stream)
{
    if (!plan || !d_r || !d_x) return set_error(DAG_ERR_INVALID, "null argument");
    k_state_to_rank<<<1024, 256, 0, (cudaStream_t)stream>>>(d_x, plan->degf, plan->n, d_r);
    DAG_CUDA(cudaGetLastError());
    return DAG_OK;
}

extern "C" int dag_pagerank_sweep_rows(dag_plan* plan, float d, int32_t row_lo, int32_t row_hi,
                                       const float* d_teleport, double teleport_total, double linked_mass,
                                       const float* d_x_in, float* d_x_out, double* d_sums, void* stream)
{
    if (!plan || !d_x_in || !d_x_out || !d_sums) return set_error(DAG_ERR_INVALID, "null argument");
    if (row_lo < 0 || row_lo > row_hi || row_hi > plan->n) return set_error(DAG_ERR_INVALID, "bad row range");
    if (!(d > 0.0f && d < 1.0f)) return set_error(DAG_ERR_INVALID, "d must lie in (0, 1)");
    SweepParams p{};
    p.n = plan->n;
    p.rowptr = plan->rowptr;
    p.colidx = plan->colidx;
    p.degf = plan->degf;
    p.base = d_teleport;
    p.base_scale = 1.0f - d;
    p.uniform_base = (1.0f - d) / (float)plan->n;
    p.d = d;
    p.g_coef = d / (float)plan->n;
    p.x0 = (void*)d_x_in;
    p.x1 = d_x_out;
    p.shard_T = teleport_total;
    p.shard_N = linked_mass;
    return sweep_rows(plan, MODE_PR, row_lo, row_hi, p, d_sums, (cudaStream_t)stream);
}

extern "C" int dag_sssp_sweep_rows(dag_plan* plan, int32_t row_lo, int32_t row_hi, const uint8_t* d_w8,
                                   const uint32_t* d_dist_in, uint32_t* d_dist_out, double* d_sums, void* stream)
{
    if (!plan || !d_dist_in || !d_dist_out || !d_sums || (plan->m > 0 && !d_w8))
        return set_error(DAG_ERR_INVALID, "null argument");
    if (row_lo < 0 || row_lo > row_hi || row_hi > plan->n) return set_error(DAG_ERR_INVALID, "bad row range");
    SweepParams p{};
    p.n = plan->n;
    p.rowptr = plan->rowptr;
    p.colidx = plan->colidx;
    p.w8 = d_w8;
    p.degf = plan->degf;
    p.x0 = (void*)d_dist_in;
    p.x1 = d_dist_out;
    return sweep_rows(plan, MODE_BF8, row_lo, row_hi, p, d_sums, (cudaStream_t)stream);
}
