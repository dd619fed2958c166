// Device memory of the plans (devmem.cu): a per-device pool that keeps freed
// memory for the next plan. dev_alloc's memory is ready for any stream;
// dev_free takes memory that no work still uses.
#pragma once
#include <cstddef>

#include <cuda_runtime.h>

namespace dag {

cudaError_t dev_alloc(void** p, size_t bytes);
cudaError_t dev_free(void* p);
template <class T>
inline cudaError_t dev_alloc(T** p, size_t bytes)
{
    return dev_alloc(reinterpret_cast<void**>(p), bytes);
}

}  // namespace dag
