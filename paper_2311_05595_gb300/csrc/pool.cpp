// The library's device-memory pool (see pool.h).
#include "pool.h"

#include <cstdint>
#include <mutex>

#include "../../include/tosolve.h"

namespace tos {
namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
cudaMemPool_t g_pool[kMaxDevices] = {};

cudaError_t pool_of_current(cudaMemPool_t* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_pool[dev] == nullptr) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) return e;
    uint64_t keep = UINT64_MAX;
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
      cudaMemPoolDestroy(pool);
      return e;
    }
    g_pool[dev] = pool;
  }
  *out = g_pool[dev];
  return cudaSuccess;
}

}  // namespace

cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t st) {
  *p = nullptr;
  cudaMemPool_t pool = nullptr;
  cudaError_t e = pool_of_current(&pool);
  if (e != cudaSuccess) return e;
  e = cudaMallocFromPoolAsync(p, bytes, pool, st);
  if (e == cudaErrorMemoryAllocation) {
    // memory reserved by the pool but unused (freed by evicted designs, in
    // pieces of other sizes) goes back to the driver; then one more try
    cudaGetLastError();
    cudaMemPoolTrimTo(pool, 0);
    e = cudaMallocFromPoolAsync(p, bytes, pool, st);
  }
  return e;
}

cudaError_t pool_free(void* p, cudaStream_t st) {
  if (p == nullptr) return cudaSuccess;
  return cudaFreeAsync(p, st);
}

}  // namespace tos

extern "C" tosolve_status tosolve_trim_pool(size_t keep_bytes) {
  cudaMemPool_t pool = nullptr;
  if (tos::pool_of_current(&pool) != cudaSuccess) return TOSOLVE_ECUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return TOSOLVE_ECUDA;
  return cudaMemPoolTrimTo(pool, keep_bytes) == cudaSuccess ? TOSOLVE_OK : TOSOLVE_ECUDA;
}
