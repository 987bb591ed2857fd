// Arithmetic-throughput and launch-latency probe for the FP64 / FP32 paths.
//
// The elasticity solve runs its outer Krylov iteration, true residual,
// compliance and gradient in FP64, so the FP64 issue rate of the part bounds
// those kernels.  This program measures, with CUDA events after warm-up:
//   * DFMA and FFMA throughput over the whole GPU and on one SM,
//   * DMMA (mma.sync m8n8k4 f64) throughput,
//   * back-to-back launch latency (plain stream and CUDA graph),
//   * a cooperative grid-wide barrier.
// It prints one JSON object.  Every loop has a fixed trip count; no kernel
// waits on another.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <cstdio>
#include <cstdlib>

namespace cg = cooperative_groups;

#define CK(x)                                                                  \
  do {                                                                         \
    cudaError_t e_ = (x);                                                      \
    if (e_ != cudaSuccess) {                                                   \
      fprintf(stderr, "CUDA error %s at %s:%d\n", cudaGetErrorString(e_),      \
              __FILE__, __LINE__);                                             \
      exit(1);                                                                 \
    }                                                                          \
  } while (0)

template <typename T, int NACC>
__global__ void fma_chain(T* out, int iters, T a, T b) {
  T acc[NACC];
#pragma unroll
  for (int i = 0; i < NACC; ++i) acc[i] = (T)(threadIdx.x * 1e-3 + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < NACC; ++i) acc[i] = fma(acc[i], a, b);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < NACC; ++i) s += acc[i];
  if (s == (T)-1.2345) out[blockIdx.x] = s;  // keeps the chain alive
}

template <int NACC>
__global__ void dmma_chain(double* out, int iters) {
  double a = 1.0 + threadIdx.x * 1e-9, b = 0.5;
  double c0[NACC], c1[NACC];
#pragma unroll
  for (int i = 0; i < NACC; ++i) { c0[i] = i; c1[i] = -i; }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < NACC; ++i) {
      asm volatile(
          "mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, "
          "{%3}, {%0,%1};\n"
          : "+d"(c0[i]), "+d"(c1[i])
          : "d"(a), "d"(b));
    }
  }
  double s = 0;
#pragma unroll
  for (int i = 0; i < NACC; ++i) s += c0[i] + c1[i];
  if (s == -1.2345) out[blockIdx.x] = s;
}

__global__ void empty_kernel(int* p) {
  if (p != nullptr && threadIdx.x == 1023 && blockIdx.x == 1 << 30) p[0] = 1;
}

__global__ void grid_sync_loop(int iters, int* p) {
  cg::grid_group g = cg::this_grid();
  for (int i = 0; i < iters; ++i) g.sync();
  if (p != nullptr && g.thread_rank() == 0) p[0] = iters;
}

static float time_ms(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, a, b));
  return ms;
}

template <typename T>
static double fma_rate(int blocks, int threads, int iters, T* out) {
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  for (int w = 0; w < 2; ++w)
    fma_chain<T, 8><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-6);
  CK(cudaEventRecord(e0));
  fma_chain<T, 8><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-6);
  CK(cudaEventRecord(e1));
  CK(cudaEventSynchronize(e1));
  double ms = time_ms(e0, e1);
  double flops = 2.0 * 8.0 * (double)iters * blocks * threads;
  CK(cudaEventDestroy(e0));
  CK(cudaEventDestroy(e1));
  return flops / (ms * 1e-3);
}

static double dmma_rate(int blocks, int threads, int iters, double* out) {
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  for (int w = 0; w < 2; ++w) dmma_chain<4><<<blocks, threads>>>(out, iters);
  CK(cudaEventRecord(e0));
  dmma_chain<4><<<blocks, threads>>>(out, iters);
  CK(cudaEventRecord(e1));
  CK(cudaEventSynchronize(e1));
  double ms = time_ms(e0, e1);
  double warps = (double)blocks * threads / 32.0;
  double flops = 512.0 * 4.0 * (double)iters * warps;
  CK(cudaEventDestroy(e0));
  CK(cudaEventDestroy(e1));
  return flops / (ms * 1e-3);
}

int main() {
  int dev = 0;
  CK(cudaSetDevice(dev));
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, dev));
  const int sms = prop.multiProcessorCount;
  double* dout = nullptr;
  float* fout = nullptr;
  CK(cudaMalloc(&dout, sizeof(double) * 65536));
  CK(cudaMalloc(&fout, sizeof(float) * 65536));

  double dfma_full = fma_rate<double>(sms * 4, 256, 4096, dout);
  double dfma_sm = fma_rate<double>(1, 1024, 2048, dout);
  double ffma_full = fma_rate<float>(sms * 8, 256, 16384, fout);
  double ffma_sm = fma_rate<float>(1, 1024, 16384, fout);
  double dmma_full = dmma_rate(sms * 4, 256, 2048, dout);
  double dmma_sm = dmma_rate(1, 1024, 1024, dout);

  cudaStream_t s;
  CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const int NL = 2000;
  for (int i = 0; i < 100; ++i) empty_kernel<<<sms, 128, 0, s>>>(nullptr);
  CK(cudaEventRecord(e0, s));
  for (int i = 0; i < NL; ++i) empty_kernel<<<sms, 128, 0, s>>>(nullptr);
  CK(cudaEventRecord(e1, s));
  CK(cudaEventSynchronize(e1));
  double us_stream = time_ms(e0, e1) * 1e3 / NL;

  cudaGraph_t g;
  cudaGraphExec_t ge;
  const int NG = 200;
  CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  for (int i = 0; i < NG; ++i) empty_kernel<<<sms, 128, 0, s>>>(nullptr);
  CK(cudaStreamEndCapture(s, &g));
  CK(cudaGraphInstantiate(&ge, g, 0));
  for (int i = 0; i < 3; ++i) CK(cudaGraphLaunch(ge, s));
  CK(cudaEventRecord(e0, s));
  for (int i = 0; i < 10; ++i) CK(cudaGraphLaunch(ge, s));
  CK(cudaEventRecord(e1, s));
  CK(cudaEventSynchronize(e1));
  double us_graph = time_ms(e0, e1) * 1e3 / (10.0 * NG);

  int nb_per_sm = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb_per_sm, grid_sync_loop,
                                                   256, 0));
  double us_gsync = -1.0;
  if (nb_per_sm >= 1) {
    int iters = 2000;
    int* pn = nullptr;
    void* args[] = {&iters, &pn};
    CK(cudaLaunchCooperativeKernel((void*)grid_sync_loop, dim3(sms), dim3(256),
                                   args, 0, s));
    CK(cudaEventRecord(e0, s));
    CK(cudaLaunchCooperativeKernel((void*)grid_sync_loop, dim3(sms), dim3(256),
                                   args, 0, s));
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    us_gsync = time_ms(e0, e1) * 1e3 / iters;
  }
  CK(cudaDeviceSynchronize());

  printf(
      "{\"gpu\": \"%s\", \"sms\": %d, "
      "\"dfma_tflops\": %.4f, \"dfma_one_sm_gflops\": %.3f, "
      "\"ffma_tflops\": %.3f, \"ffma_one_sm_gflops\": %.2f, "
      "\"dmma_tflops\": %.4f, \"dmma_one_sm_gflops\": %.3f, "
      "\"launch_us_stream\": %.3f, \"launch_us_graph\": %.3f, "
      "\"grid_sync_us\": %.3f}\n",
      prop.name, sms, dfma_full * 1e-12, dfma_sm * 1e-9,
      ffma_full * 1e-12, ffma_sm * 1e-9, dmma_full * 1e-12, dmma_sm * 1e-9,
      us_stream, us_graph, us_gsync);
  CK(cudaGraphExecDestroy(ge));
  CK(cudaGraphDestroy(g));
  CK(cudaFree(dout));
  CK(cudaFree(fout));
  return 0;
}
