// Compliance c_r = f_r^T u_r over the free DOFs without any device
// allocation: the per-block partial sums that tosolve_compliance_grad keeps
// in its handle's workspace live here in one fixed device array instead.
//
// Who needs it: callers that may not allocate device memory at the time they
// evaluate the compliance -- a plug-in that works only inside buffers its
// host application hands it (the application's allocator owns the free HBM),
// or a latency-critical loop in which a cudaMalloc, which can synchronise the
// whole device, would stall every other stream.  Such a caller also cannot
// create a tosolve handle at that point, so this entry point takes plain
// device pointers and needs no handle.
//
// The array is shared by every call on a device and keeps what the last call
// wrote.  Each call writes every partial sum it later reads, so nothing has
// to start at zero; calls whose kernels overlap on the GPU (different streams
// with no ordering between them) overwrite each other's partial sums and
// race.

#include <cuda_runtime.h>

#include <mutex>

#include "../../include/tosolve.h"
#include "internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kParts = 608;  // blocks per load case at most
constexpr int kMaxDevices = 64;
static_assert(TOSOLVE_NOALLOC_MAX_RHS * kParts * sizeof(double) == TOSOLVE_NOALLOC_SCRATCH_BYTES,
              "scratch size stated in the header");

static __device__ __align__(256) double g_noalloc_part[TOSOLVE_NOALLOC_MAX_RHS * kParts];

std::mutex g_mu;
double* g_part_ptr[kMaxDevices] = {};

__device__ __forceinline__ double block_total(double v) {
  __shared__ double red[kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kThreads / 32; ++w) s += red[w];
  return s;
}

// grid (parts, nrhs): block b of load case r sums f_r[d] u_r[d] over the free
// DOFs d = b*256 + t + k*parts*256 and stores it as part[r*kParts + b].
__global__ void __launch_bounds__(kThreads) k_noalloc_partial(long ndof, const uint8_t* __restrict__ mask,
                                                              const double* __restrict__ f,
                                                              const double* __restrict__ u,
                                                              double* __restrict__ part) {
  const int r = blockIdx.y;
  const double* fr = f + (size_t)r * ndof;
  const double* ur = u + (size_t)r * ndof;
  double s = 0.0;
  for (long d = blockIdx.x * (long)kThreads + threadIdx.x; d < ndof; d += (long)gridDim.x * kThreads)
    if (!mask[d]) s += fr[d] * ur[d];
  s = block_total(s);
  if (threadIdx.x == 0) part[r * kParts + blockIdx.x] = s;
}

// grid nrhs: c[r] = sum of the parts partial sums of load case r, fixed order.
__global__ void __launch_bounds__(kThreads) k_noalloc_total(const double* __restrict__ part, int parts,
                                                            double* __restrict__ c) {
  const int r = blockIdx.x;
  double v = 0.0;
  for (int t = threadIdx.x; t < parts; t += kThreads) v += part[r * kParts + t];
  v = block_total(v);
  if (threadIdx.x == 0) c[r] = v;
}

// Device address of the array on the current device.  Outside a stream
// capture it is looked up afresh on every call (a context torn down by
// cudaDeviceReset and created again reloads the module at a new address);
// during a capture, where the lookup may not run, the address of the last
// call made outside capture on that device is used.
cudaError_t part_address(cudaStream_t st, double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(st, &cs);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_mu);
  if (cs == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_part);
    if (e != cudaSuccess) return e;
    g_part_ptr[dev] = static_cast<double*>(p);
  } else if (g_part_ptr[dev] == nullptr) {
    return cudaErrorStreamCaptureUnsupported;
  }
  *out = g_part_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" tosolve_status tosolve_compliance_noalloc(const double* f_dev, const double* u_dev,
                                                     const uint8_t* mask_dev, size_t ndof, int nrhs,
                                                     double* c_dev, void* cuda_stream) {
  if (f_dev == nullptr || u_dev == nullptr || mask_dev == nullptr || c_dev == nullptr) {
    tos::set_last_error("tosolve_compliance_noalloc: f, u, mask or c is NULL");
    return TOSOLVE_EINVAL;
  }
  if (ndof < 1 || ndof > ((size_t)1 << 62)) {
    tos::set_last_error("tosolve_compliance_noalloc: ndof must be in 1..2^62");
    return TOSOLVE_EINVAL;
  }
  if (nrhs < 1 || nrhs > TOSOLVE_NOALLOC_MAX_RHS) {
    tos::set_last_error(
        "tosolve_compliance_noalloc: nrhs must be in 1..TOSOLVE_NOALLOC_MAX_RHS (16): the partial sums "
        "live in a fixed device array of 16 x 608 doubles");
    return TOSOLVE_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  double* part = nullptr;
  cudaError_t e = part_address(st, &part);
  if (e != cudaSuccess) {
    tos::set_last_error(e == cudaErrorStreamCaptureUnsupported
                            ? "tosolve_compliance_noalloc: the first call on a device (and the first after a "
                              "context reset) must come before any stream capture"
                            : "tosolve_compliance_noalloc: cudaGetSymbolAddress of the scratch array failed");
    cudaGetLastError();
    return TOSOLVE_ECUDA;
  }
  const size_t blocks = (ndof + kThreads - 1) / kThreads;
  const int parts = (int)(blocks < (size_t)kParts ? blocks : (size_t)kParts);
  k_noalloc_partial<<<dim3(parts, nrhs), kThreads, 0, st>>>((long)ndof, mask_dev, f_dev, u_dev, part);
  k_noalloc_total<<<nrhs, kThreads, 0, st>>>(part, parts, c_dev);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    tos::set_last_error("tosolve_compliance_noalloc: kernel launch failed");
    return TOSOLVE_ECUDA;
  }
  return TOSOLVE_OK;
}
