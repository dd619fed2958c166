// Access-matrix instrumentation (Sec. IV-C, Fig. 5): how often the workers of
// the static partition read each other's values. Counting, no floating point.
#include "dag_internal.cuh"

namespace dag {

// Access matrix (Sec. IV-C, Fig. 5): counts[i * P + j] = in-edge reads by block i
// (the owner of the row) of vertices owned by block j, for the static
// partition into P blocks. One CUDA block per merge-path tile of that
// partition; the tile's rows all belong to one block.
__global__ void __launch_bounds__(NT) k_access_matrix(const int* rowptr, const int* colidx, const int* cta_row,
                                                      const int* cta_tile, const int* tile_row, const int* tile_nz,
                                                      int P, unsigned long long* counts)
{
    extern __shared__ unsigned long long s_hist[];  // [P]
    int* s_start = (int*)(s_hist + P);              // [P + 1] block starts
    const int t = blockIdx.x;
    for (int i = threadIdx.x; i < P; i += NT) s_hist[i] = 0ull;
    for (int i = threadIdx.x; i <= P; i += NT) s_start[i] = cta_row[i];
    // owning block of this tile: last p with cta_tile[p] <= t
    int lo = 0, hi = P - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cta_tile[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    const int owner = lo;
    __syncthreads();
    const int b0 = tile_nz[t], b1 = tile_nz[t + 1];
    for (int e = b0 + threadIdx.x; e < b1; e += NT) {
        const int u = colidx[e];
        int a = 0, b = P - 1;  // block of u: last p with start[p] <= u
        while (a < b) {
            const int mid = (a + b + 1) >> 1;
            if (s_start[mid] <= u) a = mid;
            else b = mid - 1;
        }
        atomicAdd(&s_hist[a], 1ull);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < P; i += NT)
        if (s_hist[i]) atomicAdd(&counts[(size_t)owner * P + i], s_hist[i]);
}

}  // namespace dag

extern "C" int dag_access_matrix(dag_plan* plan, int32_t workers, uint64_t* d_counts, void* stream)
{
    using namespace dag;
    if (!plan || !d_counts || workers < 1 || workers > 4096) return set_error(DAG_ERR_INVALID, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    Partition* part = nullptr;
    int rc = get_partition(plan, workers, &part, s, 0);
    if (rc) return rc;
    DAG_CUDA(cudaMemsetAsync(d_counts, 0, (size_t)workers * workers * sizeof(unsigned long long), s));
    if (part->tiles == 0) return DAG_OK;
    const size_t smem = (size_t)workers * sizeof(unsigned long long) + (size_t)(workers + 1) * sizeof(int);
    if (smem > 48 * 1024)
        DAG_CUDA(cudaFuncSetAttribute((const void*)k_access_matrix, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    k_access_matrix<<<part->tiles, NT, smem, s>>>(plan->rowptr, plan->colidx, part->cta_row, part->cta_tile,
                                                  part->tile_row, part->tile_nz, workers,
                                                  (unsigned long long*)d_counts);
    DAG_CUDA(cudaGetLastError());
    return DAG_OK;
}
