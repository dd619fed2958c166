// Gather-rate probe (measurement aid): the throughput ceiling of a sweep's
// dominant memory pattern on this GPU. Each thread streams the graph's column
// indices and gathers x[colidx[e]] from the state vector, four gathers in
// flight per thread, with no merge-path tiles, barriers, stores or reductions.
// A sweep cannot gather faster than this, so "probe time / sweep time" says
// how close the sweep is to its real bound. That bound is the L2 sector rate
// of random 4-byte gathers, far below the HBM copy bandwidth.
#include "dag_internal.cuh"

namespace dag {

template <bool COHERENT>
__global__ void __launch_bounds__(256) k_gather_probe(const int* idx, long long m, const uint32_t* x, float* sink)
{
    float s = 0.0f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const uint64_t pol_edge = policy_evict_first();
    const uint64_t pol_vertex = policy_evict_last();
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < m; e += 4 * stride) {
        int u[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const long long f = e + q * stride;
            u[q] = f < m ? (int)ld_edge_b32(idx + f, pol_edge) : -1;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (u[q] >= 0) {
                const uint32_t v = COHERENT ? ld_relaxed_keep_b32(x + u[q], pol_vertex)
                                            : ld_weak_keep_b32(x + u[q], pol_vertex);
                s += __uint_as_float(v);
            }
        }
    }
    sink[blockIdx.x * (long long)blockDim.x + threadIdx.x] = s;
}

}  // namespace dag

using namespace dag;

extern "C" int dag_probe_gather(const int32_t* d_idx, int64_t m, const float* d_x, int32_t n, int32_t coherent,
                                int32_t repeats, float* h_ms, void* stream)
{
    if (!d_idx || !d_x || !h_ms || m < 1 || n < 1 || repeats < 1) return set_error(DAG_ERR_INVALID, "bad argument");
    int dev = 0, sms = 0;
    DAG_CUDA(cudaGetDevice(&dev));
    DAG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8, threads = 256;
    float* sink = nullptr;
    DAG_CUDA(cudaMalloc(&sink, (size_t)blocks * threads * sizeof(float)));
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    auto launch = [&]() {
        if (coherent) k_gather_probe<true><<<blocks, threads, 0, s>>>(d_idx, m, (const uint32_t*)d_x, sink);
        else k_gather_probe<false><<<blocks, threads, 0, s>>>(d_idx, m, (const uint32_t*)d_x, sink);
    };
    launch();  // warm-up
    cudaEventRecord(a, s);
    for (int r = 0; r < repeats; ++r) launch();
    cudaEventRecord(b, s);
    cudaError_t e = cudaEventSynchronize(b);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(sink);
    if (e != cudaSuccess) return cuda_check(e, "gather probe");
    DAG_CUDA(cudaGetLastError());
    *h_ms = ms / repeats;
    return DAG_OK;
}
