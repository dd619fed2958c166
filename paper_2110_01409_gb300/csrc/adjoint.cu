// Gradients of a loss through weighted PageRank, after the adjoint solve
// (no counterpart in the paper). With M_vu = w_uv / s_u, r the forward fixed
// point and lambda the adjoint (lambda = c + d M^T lambda + d g sum(lambda)/n):
//   dL/dw_uv = d r_u (lambda_v - (M^T lambda)_u) / s_u,   dL/dt_v = (1 - d) lambda_v.
// A pass over the vertices packs each source's two factors, d r_u / s_u and
// (M^T lambda)_u, into one 8-byte pair; then one pass over the in-edges in the
// caller's (in-CSR) order, one gather per edge: each CTA walks its vertex
// block tile by tile and finds an edge's row by binary search over the tile's
// row ends in shared memory.
#include <climits>

#include "dag_internal.cuh"
#include "devmem.cuh"

namespace dag {

__global__ void k_grad_coef(const float* s_norm, const float* rank, const float* mt, float d, int n, float2* coef)
{
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u < n) coef[u] = make_float2(d * rank[u] / s_norm[u], mt[u]);  // s_u = 0: u is no edge's source
}

__global__ void __launch_bounds__(NT) k_edge_grad(const int* rowptr, const int* colidx, const int* cta_tile,
                                                  const int* tile_row, const int* tile_nz, const float2* coef,
                                                  const float* lambda, float* grad_w)
{
    __shared__ int s_end[TILE + 1];
    const int c = blockIdx.x;
    for (int t = cta_tile[c]; t < cta_tile[c + 1]; ++t) {
        const int a0 = tile_row[t], b0 = tile_nz[t];
        const int NA = tile_row[t + 1] - a0, NB = tile_nz[t + 1] - b0;
        __syncthreads();
        for (int i = threadIdx.x; i < NA; i += NT) s_end[i] = rowptr[a0 + i + 1] - b0;
        if (threadIdx.x == 0) s_end[NA] = INT_MAX;  // the row still open at the tile's end
        __syncthreads();
        for (int j = threadIdx.x; j < NB; j += NT) {
            // row of edge j: first i with s_end[i] > j
            int lo = 0, hi = NA;
            while (lo < hi) {
                int mid = (lo + hi) >> 1;
                if (s_end[mid] > j) hi = mid;
                else lo = mid + 1;
            }
            const int e = b0 + j;
            const float2 cf = coef[colidx[e]];
            grad_w[e] = cf.x * (lambda[a0 + lo] - cf.y);
        }
    }
}

__global__ void k_teleport_grad(const float* lambda, float one_minus_d, float* grad_t, int n)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) grad_t[v] = one_minus_d * lambda[v];
}

int launch_edge_grad(dag_plan* plan, float d, const float* val, const float* s_norm, const float* rank,
                     const float* lambda, const float* mt, float* grad_w, float* grad_t, cudaStream_t st)
{
    (void)val;
    const int P = plan->num_sms * 4;
    Partition* part = nullptr;
    int rc = get_partition(plan, P, &part, st, 0);
    if (rc) return rc;
    if (grad_w && plan->m > 0) {
        if (!plan->grad_coef) DAG_CUDA(dev_alloc(&plan->grad_coef, (size_t)plan->n * sizeof(float2)));
        k_grad_coef<<<(plan->n + 255) / 256, 256, 0, st>>>(s_norm, rank, mt, d, plan->n, (float2*)plan->grad_coef);
        k_edge_grad<<<P, NT, 0, st>>>(plan->rowptr, plan->colidx, part->cta_tile, part->tile_row, part->tile_nz,
                                      (const float2*)plan->grad_coef, lambda, grad_w);
    }
    if (grad_t) k_teleport_grad<<<(plan->n + 255) / 256, 256, 0, st>>>(lambda, 1.0f - d, grad_t, plan->n);
    DAG_CUDA(cudaGetLastError());
    return DAG_OK;
}

}  // namespace dag
