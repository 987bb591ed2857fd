// Finest-level operator of the TF32 preconditioner on the 5th-generation
// tensor cores (tcgen05): the stacked subcell contraction of Eq. matrixK_mr,
//     Y_e = [K^(e_1); ...; K^(e_m)] u_e        (m*24 x 24 times 24),
//     y_e = sum_i w_{e,i} Y_e[i*24 : i*24+24],
// for a tile of 128 elements per CTA, then a deterministic node gather.
//
// Tile shape: M = 128 elements (TMEM lanes), N = 24 m stacked subcell rows
// rounded up to a multiple of 16 (TMEM columns), K = 24 element DOFs padded
// to 32 (four kind::tf32 MMAs of K = 8).  A (element DOFs) and B (stacked
// table, constant) sit in shared memory in the no-swizzle K-major
// core-matrix layout (8 rows x 16 bytes per core matrix, LBO = 128 B along
// K, SBO = 1024 B along M/N); the FP32 accumulator lives in TMEM and is read
// back with tcgen05.ld for the weighted reduce over subcells.  One thread
// issues the MMAs; completion is signalled through an mbarrier whose wait is
// bounded (on timeout the kernel raises an error flag, waits once more,
// frees its TMEM and returns).
#include <cstdint>
#include <mutex>

#include "internal.cuh"

namespace tos {
namespace {

constexpr int kTcM = 128;
constexpr int kTcK = 32;
constexpr int kTcCols = 256;
constexpr int kTcASize = 16384;  // 128 x 32 fp32
constexpr int kTcBSize = 32768;  // <= 256 x 32 fp32
constexpr long kTcSpin = 1L << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Byte offset of element (row, k) in the no-swizzle K-major layout.
__device__ __forceinline__ uint32_t kmaj_off(int row, int k) {
  return (uint32_t)((row >> 3) * 1024 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

// Shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte
// offsets in 16-byte units, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFF) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFF) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t phase) {
  uint32_t done = 0;
  for (long it = 0; it < kTcSpin && !done; ++it)
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(phase)
        : "memory");
  return done != 0;
}

__global__ void __launch_bounds__(kTcM, 1)
    k_tc_stacked(int ex, int ey, int ez, int m, int Lx, int Ly, const float* __restrict__ v,
                 const float* __restrict__ w32, const float* __restrict__ KT,
                 float* __restrict__ Ye, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem;
  unsigned char* sB = smem + kTcASize;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int N = ((24 * m + 15) / 16) * 16;
  const long E = (long)ex * ey * ez;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(kTcCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // B: row n = i*24 + R, column k: K^(e_i)[R][k] (tables are symmetric)
  for (int t = tid; t < N * kTcK; t += blockDim.x) {
    const int n = t / kTcK, k = t % kTcK;
    float x = 0.f;
    if (n < 24 * m && k < 24) x = KT[(n / 24) * 576 + (n % 24) * 24 + k];
    *(float*)(sB + kmaj_off(n, k)) = to_tf32(x);
  }
  for (int t = tid; t < kTcM * kTcK; t += blockDim.x) *(float*)(sA + kmaj_off(t / kTcK, t % kTcK)) = 0.f;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
                         ((uint32_t)(kTcM >> 4) << 24);
  const uint32_t aaddr = smem_u32(sA), baddr = smem_u32(sB);
  uint32_t phase = 0;
  bool failed = false;
  const long ntiles = (E + kTcM - 1) / kTcM;
  for (long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long e = tile * kTcM + tid;
    // gather u_e: element nodes (ix, iy, iz) in {0,1}^3, local node a = ix + 2 iy + 4 iz
    if (e < E) {
      const int exi = e % ex, eyi = (e / ex) % ey, ezi = e / ((long)ex * ey);
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const long node = (exi + (a & 1)) + (long)Lx * ((eyi + ((a >> 1) & 1)) + (long)Ly * (ezi + (a >> 2)));
#pragma unroll
        for (int c = 0; c < 3; ++c) *(float*)(sA + kmaj_off(tid, 3 * a + c)) = to_tf32(v[3 * node + c]);
      }
    } else {
#pragma unroll
      for (int k = 0; k < 24; ++k) *(float*)(sA + kmaj_off(tid, k)) = 0.f;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
#pragma unroll
      for (int s = 0; s < kTcK / 8; ++s) {
        const uint64_t ad = smem_desc(aaddr + 256 * s, 128, 1024);
        const uint64_t bd = smem_desc(baddr + 256 * s, 128, 1024);
        const uint32_t acc = s > 0 ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&mbar))
          : "memory");
    }
    const bool ok = mbar_wait(&mbar, phase);
    if (__syncthreads_or(!ok)) {  // block-uniform decision
      failed = true;
      if (tid == 0) atomicExch(err, 1);
      break;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    float y[24];
#pragma unroll
    for (int r = 0; r < 24; ++r) y[r] = 0.f;
    for (int i = 0; i < m; ++i) {
      const float wi = (e < E) ? w32[e * m + i] : 0.f;
      uint32_t q[24];
      const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(i * 24);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]),
            "=r"(q[7]), "=r"(q[8]), "=r"(q[9]), "=r"(q[10]), "=r"(q[11]), "=r"(q[12]), "=r"(q[13]),
            "=r"(q[14]), "=r"(q[15])
          : "r"(ta));
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                   : "=r"(q[16]), "=r"(q[17]), "=r"(q[18]), "=r"(q[19]), "=r"(q[20]), "=r"(q[21]),
                     "=r"(q[22]), "=r"(q[23])
                   : "r"(ta + 16));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int r = 0; r < 24; ++r) y[r] += wi * __uint_as_float(q[r]);
    }
    if (e < E) {
      float4* dst = (float4*)(Ye + e * 24);
#pragma unroll
      for (int r = 0; r < 6; ++r) dst[r] = make_float4(y[4 * r], y[4 * r + 1], y[4 * r + 2], y[4 * r + 3]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  if (failed) mbar_wait(&mbar, phase);  // let an MMA still in flight finish
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols));
}

// Node gather of the element results (fixed order: deterministic), fused
// with the V-cycle update.  Fixed DOFs have identity rows: y = v there.
//   mode 0 (residual):  out = b - y
//   mode 1 (smoother):  out = v + omega D^-1 (b - y)
//   mode 2 (apply):     out = y
__global__ void k_tc_gather(int ex, int ey, int ez, int Lx, int Ly, int Lz, const float* __restrict__ Ye,
                            const uint8_t* __restrict__ mask, const float* __restrict__ b,
                            const float* __restrict__ v, const float* __restrict__ dinv, float omega,
                            int mode, float* __restrict__ out) {
  const long nn = (long)Lx * Ly * Lz;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < 3 * nn; t += (long)gridDim.x * blockDim.x) {
    const long node = t / 3;
    const int c = t % 3;
    const int i = node % Lx, j = (node / Lx) % Ly, l = node / ((long)Lx * Ly);
    float y = 0.f;
#pragma unroll
    for (int a = 0; a < 8; ++a) {  // the element in which this node is local node a
      const int exi = i - (a & 1), eyi = j - ((a >> 1) & 1), ezi = l - (a >> 2);
      if (exi >= 0 && exi < ex && eyi >= 0 && eyi < ey && ezi >= 0 && ezi < ez)
        y += Ye[(exi + (long)ex * (eyi + (long)ey * ezi)) * 24 + 3 * a + c];
    }
    const long d = 3 * node + c;
    if (mask[d]) y = v[d];
    float o;
    if (mode == 0)
      o = b[d] - y;
    else if (mode == 1)
      o = v[d] + omega * dinv[d] * (b[d] - y);
    else
      o = y;
    out[d] = o;
  }
}

// Element-major FP32 copy of the subcell weights for the tensor-core tiles.
__global__ void k_weights_elem(int ex, int ey, int ez, int n, const double* __restrict__ w, int Dx, int Dy,
                               float* __restrict__ w32) {
  const int m = n * n * n;
  const long total = (long)ex * ey * ez * m;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const long e = t / m;
    const int s = t % m;
    const int exi = e % ex, eyi = (e / ex) % ey, ezi = e / ((long)ex * ey);
    const int a = s % n, b = (s / n) % n, c = s / (n * n);
    w32[t] = (float)w[(n * exi + a) + (long)Dx * ((n * eyi + b) + (long)Dy * (n * ezi + c))];
  }
}

__global__ void k_mask_fp32(long n, const uint8_t* __restrict__ mask, float* __restrict__ x) {
  for (long d = blockIdx.x * (long)blockDim.x + threadIdx.x; d < n; d += (long)gridDim.x * blockDim.x)
    if (mask[d]) x[d] = 0.f;
}

}  // namespace

void launch_mask_fp32(const Level& L, float* x, cudaStream_t st) {
  const long n = L.ndof;
  long g = (n + 255) / 256;
  if (g > 4096) g = 4096;
  k_mask_fp32<<<(int)g, 256, 0, st>>>(n, L.mask, x);
}

bool tc_supported(int n) { return n * n * n * 24 <= kTcCols && n >= 1; }

cudaError_t launch_tc_apply(const Level& L0, int m, const float* v, const float* w32, const float* KT,
                            float* Ye, int* err, int sms, cudaStream_t st) {
  const long E = (long)L0.ex * L0.ey * L0.ez;
  const long ntiles = (E + kTcM - 1) / kTcM;
  const size_t sm = kTcASize + kTcBSize;
  static std::once_flag attr;  // handles may be created from several threads
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(attr, [sm] {
    attr_err = cudaFuncSetAttribute(k_tc_stacked, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  });
  if (attr_err != cudaSuccess) return attr_err;
  const long cap = 2L * sms;  // two CTAs per SM: 2 x 256 TMEM columns fit in 512
  const int g = (int)(ntiles < cap ? ntiles : cap);
  k_tc_stacked<<<g, kTcM, sm, st>>>(L0.ex, L0.ey, L0.ez, m, L0.Lx, L0.Ly, v, w32, KT, Ye, err);
  return cudaGetLastError();
}

void launch_tc_gather(const Level& L0, const float* Ye, const float* b, const float* v, const float* dinv,
                      float omega, int mode, float* out, cudaStream_t st) {
  const long n = 3L * L0.nn;
  long g = (n + 255) / 256;
  if (g > 4096) g = 4096;
  k_tc_gather<<<(int)g, 256, 0, st>>>(L0.ex, L0.ey, L0.ez, L0.Lx, L0.Ly, L0.Lz, Ye, L0.mask, b, v, dinv,
                                      omega, mode, out);
}

void launch_weights_elem(const Level& L0, int n, const double* w, int Dx, int Dy, float* w32,
                         cudaStream_t st) {
  const long total = (long)L0.ex * L0.ey * L0.ez * n * n * n;
  long g = (total + 255) / 256;
  if (g > 4096) g = 4096;
  k_weights_elem<<<(int)g, 256, 0, st>>>(L0.ex, L0.ey, L0.ez, n, w, Dx, Dy, w32);
}

}  // namespace tos
