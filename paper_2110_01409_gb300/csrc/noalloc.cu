// PageRank without any device allocation (dag_pagerank_noalloc).
//
// Some callers cannot call cudaMalloc when they solve: an application whose
// device memory is owned up front by its own pool allocator (a cudaMalloc
// behind its back would break its budget), or a latency-bound service that
// cannot accept cudaMalloc's implicit device synchronisation and unbounded
// latency on the solve path. dag_pagerank needs a plan, and creating one
// allocates workspace. This entry point instead keeps all its scratch (out-
// degrees, the two state buffers, the solve's control block and the vertex
// partition) in one fixed, file-scope device array, and takes only the
// caller's inputs and outputs.
//
// The array is a static __device__ variable, so every GPU that loads this
// library holds it (about 17 MiB) until the process exits. Host code cannot
// use the variable's name as a device address: its device address is looked
// up once per device with cudaGetSymbolAddress, on that device's first call,
// and cached. All calls share the array and it keeps the last call's
// contents, so each call clears what must start at zero; two calls whose work
// overlaps on the GPU (for example on two streams) race on it. The paper has
// no counterpart of this entry point: it is an interface convenience.
#include <algorithm>
#include <mutex>

#include <cstdint>

#include "dag_internal.cuh"

namespace dag {
namespace {

constexpr long long NA_MAX_N = DAG_NOALLOC_MAX_N;
constexpr long long NA_MAX_M = DAG_NOALLOC_MAX_M;
constexpr int NA_MAX_CTAS = 8192;
constexpr long long NA_MAX_TILES = (NA_MAX_N + NA_MAX_M) / TILE + NA_MAX_CTAS + 1;

constexpr size_t al(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t OFF_SYNC = 0;
constexpr size_t OFF_FLAGS = OFF_SYNC + al(sizeof(SyncBlock));                  // bad, tiles, max_rows
constexpr size_t OFF_OUTDEG = OFF_FLAGS + al(4 * sizeof(int));
constexpr size_t OFF_DEGF = OFF_OUTDEG + al(NA_MAX_N * sizeof(int));
constexpr size_t OFF_X0 = OFF_DEGF + al(NA_MAX_N * sizeof(float));
constexpr size_t OFF_X1 = OFF_X0 + al(NA_MAX_N * 4);
constexpr size_t OFF_CTA_ROW = OFF_X1 + al(NA_MAX_N * 4);
constexpr size_t OFF_CTA_TILE = OFF_CTA_ROW + al((NA_MAX_CTAS + 1) * sizeof(int));
constexpr size_t OFF_TILE_ROW = OFF_CTA_TILE + al((NA_MAX_CTAS + 1) * sizeof(int));
constexpr size_t OFF_TILE_NZ = OFF_TILE_ROW + al((NA_MAX_TILES + 1) * sizeof(int));
constexpr size_t SCRATCH_BYTES = OFF_TILE_NZ + al((NA_MAX_TILES + 1) * sizeof(int));

}  // namespace
}  // namespace dag

// The fixed scratch of dag_pagerank_noalloc (one copy per device).
static __device__ __align__(256) unsigned char g_noalloc_scratch[dag::SCRATCH_BYTES];

namespace dag {
namespace {

std::mutex g_scratch_mu;
unsigned char* g_scratch_ptr[128] = {nullptr};

// Device address of the scratch array on `device` (the current device),
// looked up on the first call for that device.
int scratch_for_device(int device, unsigned char** out)
{
    if (device < 0 || device >= 128) return set_error(DAG_ERR_INVALID, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_ptr[device]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_check(e, "cudaGetSymbolAddress(no-alloc scratch)");
        g_scratch_ptr[device] = (unsigned char*)ptr;
    }
    *out = g_scratch_ptr[device];
    return DAG_OK;
}

}  // namespace
}  // namespace dag

using namespace dag;

extern "C" int dag_pagerank_noalloc(const dag_csr* csr, float d, double tol, dag_variant variant, int32_t delta,
                                    int32_t max_iters, const float* d_teleport, float* d_rank, dag_stats* h_stats,
                                    void* stream)
{
    if (!csr || !d_rank) return set_error(DAG_ERR_INVALID, "null argument");
    if (csr->n < 1 || csr->m < 0) return set_error(DAG_ERR_INVALID, "need n >= 1 and m >= 0");
    if ((long long)csr->n > NA_MAX_N || csr->m > NA_MAX_M)
        return set_error(DAG_ERR_INVALID, "graph too large for the no-alloc scratch (n <= 2^20 and m <= 2^24)");
    if (!csr->d_rowptr || (csr->m > 0 && !csr->d_colidx)) return set_error(DAG_ERR_INVALID, "null CSR array");
    if (!(d > 0.0f && d < 1.0f)) return set_error(DAG_ERR_INVALID, "d must lie in (0, 1)");
    if (!(tol > 0.0)) return set_error(DAG_ERR_INVALID, "tol must be > 0");
    if (variant < DAG_SYNC || variant > DAG_DELAYED) return set_error(DAG_ERR_INVALID, "unknown variant");
    if (delta < 0 || max_iters < 1) return set_error(DAG_ERR_INVALID, "need delta >= 0 and max_iters >= 1");
    if ((((uintptr_t)csr->d_rowptr | (uintptr_t)csr->d_colidx) & 15u) != 0)
        return set_error(DAG_ERR_INVALID, "rowptr and colidx must be 16-byte aligned");
    int var = variant;
    if (var == DAG_DELAYED && delta == 0) var = DAG_ASYNC;

    int device = 0;
    DAG_CUDA(cudaGetDevice(&device));
    unsigned char* base = nullptr;
    int rc = scratch_for_device(device, &base);
    if (rc) return rc;
    const int n = csr->n;
    const long long m = csr->m;
    const int* rowptr = csr->d_rowptr;
    const int* colidx = csr->d_colidx;
    SyncBlock* sync = (SyncBlock*)(base + OFF_SYNC);
    int* flags = (int*)(base + OFF_FLAGS);  // [0] bad CSR, [1] tiles, [2] largest block
    int* outdeg = (int*)(base + OFF_OUTDEG);
    float* degf = (float*)(base + OFF_DEGF);
    int* cta_row = (int*)(base + OFF_CTA_ROW);
    int* cta_tile = (int*)(base + OFF_CTA_TILE);
    int* tile_row = (int*)(base + OFF_TILE_ROW);
    int* tile_nz = (int*)(base + OFF_TILE_NZ);
    cudaStream_t s = (cudaStream_t)stream;

    // the previous call's contents stay in the array: clear what counts from zero
    DAG_CUDA(cudaMemsetAsync(flags, 0, 4 * sizeof(int), s));
    DAG_CUDA(cudaMemsetAsync(outdeg, 0, (size_t)n * sizeof(int), s));
    k_check_rowptr<<<(n + 1 + 255) / 256, 256, 0, s>>>(rowptr, n, m, flags);
    if (m > 0) k_out_degree<<<2048, 256, 0, s>>>(colidx, m, n, outdeg, flags);
    k_degf<<<(n + 255) / 256, 256, 0, s>>>(outdeg, degf, n);
    DAG_CUDA(cudaGetLastError());

    // launch shape: dag_pagerank's rule (settle_shape), with the partition built in the scratch array
    dag_plan shape;  // host-side description only (device and SM count)
    shape.device = device;
    shape.n = n;
    shape.m = m;
    DAG_CUDA(cudaDeviceGetAttribute(&shape.num_sms, cudaDevAttrMultiProcessorCount, device));
    int host_flags[4] = {0, 0, 0, 0};
    auto build = [&](int nb, int* max_rows) -> int {
        if (nb > NA_MAX_CTAS) return set_error(DAG_ERR_INVALID, "more CTAs than the no-alloc scratch holds");
        k_cta_rows<<<(nb + 1 + 255) / 256, 256, 0, s>>>(rowptr, n, (long long)n + m, nb, cta_row, 1);
        k_cta_tiles<<<1, CT_THREADS, 0, s>>>(rowptr, cta_row, nb, cta_tile, flags + 2);
        DAG_CUDA(cudaMemcpyAsync(flags + 1, cta_tile + nb, sizeof(int), cudaMemcpyDeviceToDevice, s));
        DAG_CUDA(cudaMemcpyAsync(host_flags, flags, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
        DAG_CUDA(cudaStreamSynchronize(s));
        if (host_flags[0]) return set_error(DAG_ERR_INVALID, "invalid CSR (rowptr order or colidx range)");
        *max_rows = host_flags[2];
        return DAG_OK;
    };
    shape.worker_cap = NA_MAX_CTAS;
    int nb = 0, cap = 0, clamped = 0;
    rc = settle_shape(&shape, MODE_PR, var, delta, build, &nb, &cap, &clamped);
    if (rc) return rc;
    const int tiles = host_flags[1];
    if (tiles > NA_MAX_TILES) return set_error(DAG_ERR_INVALID, "partition exceeds the no-alloc scratch");
    k_tile_coords<<<(tiles + 1 + 255) / 256, 256, 0, s>>>(rowptr, n, m, cta_row, cta_tile, nb, tiles, tile_row,
                                                           tile_nz);
    DAG_CUDA(cudaGetLastError());

    SweepParams p{};
    p.n = n;
    p.nblocks = nb;
    p.rowptr = rowptr;
    p.colidx = colidx;
    p.degf = degf;
    p.base = d_teleport;
    p.base_scale = 1.0f - d;
    p.uniform_base = (1.0f - d) / (float)n;
    p.d = d;
    p.g_coef = d / (float)n;
    p.tol = tol;
    p.max_iters = max_iters;
    p.delta = (var == DAG_DELAYED) ? delta : 0;
    p.buf_cap = cap;
    p.buf_clamped = clamped;
    p.x0 = base + OFF_X0;
    p.x1 = base + OFF_X1;
    p.cta_row = cta_row;
    p.cta_tile = cta_tile;
    p.tile_row = tile_row;
    p.tile_nz = tile_nz;
    p.sync = sync;
    p.timeout_ns = DEFAULT_TIMEOUT_NS;
    p.out = d_rank;
    DAG_CUDA(cudaMemsetAsync(sync, 0, sizeof(SyncBlock), s));
    const void* k = sweep_kernel_ptr(MODE_PR, var);
    size_t dyn = sweep_ring_bytes(MODE_PR, var) + ((var == DAG_DELAYED) ? (size_t)cap * 4 : 0);
    DAG_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    void* args[] = {(void*)&p};
    DAG_CUDA(cudaLaunchCooperativeKernel(k, dim3(nb), dim3(NT), args, dyn, s));
    SyncBlock sb;
    DAG_CUDA(cudaMemcpyAsync(&sb, sync, sizeof(SyncBlock), cudaMemcpyDeviceToHost, s));
    DAG_CUDA(cudaStreamSynchronize(s));
    int out = DAG_OK;
    if (sb.err) out = sb.err;
    else if (!sb.converged) out = DAG_ERR_NOT_CONVERGED;
    if (h_stats) {
        h_stats->iters = sb.iters;
        h_stats->err = out;
        h_stats->residual = sb.residual;
        h_stats->ms = 0.0f;  // no events: creating them is itself a resource allocation
        h_stats->workers = nb;
        h_stats->delta = (var == DAG_DELAYED) ? delta : 0;
        h_stats->flushes = sb.flushes;
        h_stats->edges_processed = (long long)sb.iters * m;
    }
    if (out == DAG_ERR_BARRIER_TIMEOUT) set_error(out, "grid barrier wait ran out of time");
    else if (out == DAG_ERR_NOT_CONVERGED) set_error(out, "max_iters reached before the stopping rule");
    return out;
}
