// Device memory of the library's plans: one stream-ordered pool per device that
// keeps up to POOL_KEEP bytes of freed memory for later allocations, so a plan
// built and destroyed per call (the end-to-end path) maps its arrays once
// instead of paying cudaMalloc and cudaFree (an implicit device synchronisation)
// on every call. Allocations are made on a private stream and waited for, so
// the memory is ready for any stream when dev_alloc returns; dev_free returns
// memory whose users have all finished (the caller has waited for them).
#include <mutex>

#include "dag_internal.cuh"
#include "devmem.cuh"

namespace dag {
namespace {

constexpr unsigned long long POOL_KEEP = 4ull << 30;
constexpr int MAX_DEVICES = 128;

struct DevicePool {
    cudaMemPool_t pool = nullptr;
    cudaStream_t stream = nullptr;
};

std::mutex g_pool_mu;
DevicePool g_pool[MAX_DEVICES];

cudaError_t current_pool(DevicePool** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    DevicePool& d = g_pool[dev];
    if (!d.pool) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return e;
        unsigned long long keep = POOL_KEEP;
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        cudaStream_t st = nullptr;
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return e;
        }
        d.pool = pool;
        d.stream = st;
    }
    *out = &d;
    return cudaSuccess;
}

}  // namespace

cudaError_t dev_alloc(void** p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0) return cudaSuccess;  // as cudaMalloc: no memory, a null pointer
    DevicePool* d = nullptr;
    cudaError_t e = current_pool(&d);
    if (e != cudaSuccess) return e;
    e = cudaMallocFromPoolAsync(p, bytes, d->pool, d->stream);
    if (e != cudaSuccess) {
        *p = nullptr;
        return e;
    }
    e = cudaStreamSynchronize(d->stream);
    if (e != cudaSuccess) {
        cudaFreeAsync(*p, d->stream);
        *p = nullptr;
    }
    return e;
}

cudaError_t dev_free(void* p)
{
    if (!p) return cudaSuccess;
    DevicePool* d = nullptr;
    cudaError_t e = current_pool(&d);
    if (e != cudaSuccess) return e;
    return cudaFreeAsync(p, d->stream);
}

}  // namespace dag
