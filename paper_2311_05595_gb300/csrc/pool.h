// Device memory of the library: one stream-ordered pool per device.
//
// Handles and serving buffers allocate from it and free back into it. Freed
// memory stays reserved in the pool (release threshold: unlimited), so a
// design rebuilt after eviction reuses it without new driver mappings, and
// a free never synchronises the device while other streams run.
// tosolve_trim_pool returns the unused part to the driver.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

namespace tos {

// Allocates bytes on stream st from the current device's pool.
cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t st);
// Returns p to the pool, ordered after the work issued on st.
cudaError_t pool_free(void* p, cudaStream_t st);

}  // namespace tos
