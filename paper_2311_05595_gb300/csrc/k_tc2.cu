// Finest-level operator of the tensor-core preconditioners for triquadratic
// (Lagrange degree 2) elements: the stacked subcell contraction of
// Eq. matrixK_mr (Sec. 3.3),
//     Z_e = [K^(e_1); ...; K^(e_m)] u_e        (81 m x 81 times 81),
//     y_e = sum_i w_{e,i} Z_e[81 i : 81 i + 81],
// on the tcgen05 tensor cores, then a deterministic node gather.
//
// Orientation: M = 128 elements of a tile (TMEM lanes), N = a chunk of the
// stacked subcell rows (TMEM columns), K = the 81 element DOFs padded to 88
// (TF32) or 96 (16-bit operands).  With the elements on the lanes, the
// weighted reduce over subcells is thread-local in the epilogue: thread e
// reads its lane's columns and accumulates w_{e,i} Z[i, r] into 81
// registers, so no cross-lane reduction and a fixed summation order.
//
// Operand modes:
//   TF32     one product, TF32 operands (10-bit mantissas), kind::tf32;
//   BF16     one product, BF16 operands (7-bit), kind::f16;
//   BF16X3   split pairs a = a_hi + a_lo of BF16 (about 16 bits each side)
//            and three products a_hi b_hi + a_lo b_hi + a_hi b_lo;
//   F16X3    split pairs of FP16 (about 22 bits each side), three products;
//            FP16 has a narrow exponent range, so each element's vector is
//            scaled by a power of two to a maximum below 1 (the table by one
//            global power of two), and the epilogue scales back exactly.
// A multigrid smoother on high-contrast triquadratic meshes needs about 20
// bits of operator accuracy (a single rounding to 10 bits stalls the outer
// iteration); F16X3 gives that at the FP16 tensor rate.
//
// Operands sit in shared memory in the no-swizzle K-major core-matrix layout
// (8 rows x 16 bytes per core matrix; LBO = 128 bytes between core matrices
// along K, SBO = (K / elements-per-16-bytes) * 128 bytes between 8-row
// groups).  A split operand row is [hi (KP) | lo (KP)]; each MMA of the
// three products points its descriptors at the K-slices it pairs.  The
// stacked table is constant: it is laid out once, at create, in exactly that
// shared-memory image, chunk by chunk, and each chunk is moved by one 1D bulk
// copy (TMA) completing on an mbarrier.
//
// Warp roles (256 threads, one CTA per SM, persistent over element tiles):
//   warp 0     allocates the 512 TMEM columns; lane 0 streams table chunks
//              into a ring of B stages;
//   warp 1     lane 0 issues the MMAs of each chunk into one of two TMEM
//              accumulators and commits their completion to mbarriers;
//   warps 2-5  epilogue: read the accumulator of each chunk (tcgen05.ld),
//              weighted reduce over subcells, store y_e;
//   warps 6-7  gather u_e of the next tile (fixed DOFs as zero), minus its
//              least-squares rigid motion, into one of two A buffers, two
//              elements per thread.
// Every mbarrier wait is bounded; a timeout raises the error flag and a
// shared abort flag that ends every role, the MMA thread waits for its last
// commit and the producer for its copies in flight, and the TMEM is freed.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cmath>
#include <cstdint>
#include <mutex>
#include <vector>

#include "internal.cuh"

namespace tos {
namespace {

constexpr int kTm = 128;            // elements per tile
constexpr int kThreads = 256;       // 8 warps (two per SM sub-partition: up to 255 registers)
constexpr int kTmemCols = 512;      // two accumulators of up to 256 columns
constexpr long kSpin2 = 1L << 22;   // bound of every mbarrier wait

enum Mode : int { kTF32 = 0, kBF16 = 1, kBF16X3 = 2, kF16X3 = 3 };

template <int MD>
struct Opnd {
  static constexpr bool kSplit = MD == kBF16X3 || MD == kF16X3;
  static constexpr bool kScaled = MD == kF16X3;
  static constexpr int kEs = MD == kTF32 ? 4 : 2;          // bytes per element
  static constexpr int kKc = 16 / kEs;                     // elements per 16-byte core-matrix row
  static constexpr int kKstep = MD == kTF32 ? 8 : 16;      // K of one MMA
  static constexpr int kNch = MD == kTF32 ? 192 : (kSplit ? 128 : 256);  // stacked rows per chunk
  static constexpr int kStages = MD == kBF16 ? 3 : 2;      // B ring
  static constexpr int kParts = kSplit ? 2 : 1;            // hi (and lo) K-slices per row
  static constexpr int kProducts = kSplit ? 3 : 1;
  // operand format in the instruction descriptor: TF32 2, BF16 1, F16 0
  static constexpr uint32_t kFmt = MD == kTF32 ? 2u : (MD == kF16X3 ? 0u : 1u);
};

template <int MD, int D, int M>
struct Shape {
  using O = Opnd<MD>;
  static constexpr int KP = (D + O::kKstep - 1) / O::kKstep * O::kKstep;  // padded K of one part
  static constexpr int KR = KP * O::kParts;                                 // K extent of a row
  static constexpr int ROWS = D * M;                                        // stacked rows
  static constexpr int NCH = O::kNch;
  static constexpr int NC = (ROWS + NCH - 1) / NCH;                         // chunks
  static constexpr int LASTN = ROWS - (NC - 1) * NCH;
  static constexpr int LASTNP = (LASTN + 15) / 16 * 16;                     // MMA N of the last
  static constexpr int KS = KP / O::kKstep;                                 // MMAs of one product
  static constexpr uint32_t SBO = (uint32_t)(KR / O::kKc) * 128u;
  static constexpr uint32_t ABYTES = (uint32_t)kTm * KR * O::kEs;
  static constexpr uint32_t BBYTES = (uint32_t)NCH * KR * O::kEs;
  static constexpr size_t SMEM = 2 * (size_t)ABYTES + (size_t)O::kStages * BBYTES;
  static constexpr int YS = 84;  // stride of y_e in the result buffer: the 81 DOFs of the 27-node layout
};

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFF) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFF) >> 4) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version; base offset 0, no swizzle
  return d;
}

__device__ __forceinline__ bool try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(su32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Bounded wait that also gives up when another role raised the abort flag.
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  for (long it = 0; it < kSpin2; ++it) {
    if (try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
  }
  *abort_flag = 1;
  return false;
}

// Bounded wait that ignores the abort flag (draining copies or MMAs in flight).
__device__ __forceinline__ void drain_wait(uint64_t* bar, uint32_t parity) {
  for (long it = 0; it < kSpin2; ++it)
    if (try_wait(bar, parity)) return;
}

__device__ __forceinline__ void arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}

__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}

__device__ __forceinline__ uint32_t tf32_bits(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}
__device__ __forceinline__ uint32_t pack2(__half lo, __half hi) {
  return (uint32_t)__half_as_ushort(lo) | ((uint32_t)__half_as_ushort(hi) << 16);
}

// The 16-bit (hi, lo) pair of x: hi = x rounded, lo = the rest rounded (the
// difference x - hi is exact in FP32).
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& h, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(x);
  l = __float2bfloat16_rn(x - __bfloat162float(h));
}
__device__ __forceinline__ void split_f16(float x, __half& h, __half& l) {
  h = __float2half_rn(x);
  l = __float2half_rn(x - __half2float(h));
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&q)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]), "=r"(q[7]),
        "=r"(q[8]), "=r"(q[9]), "=r"(q[10]), "=r"(q[11]), "=r"(q[12]), "=r"(q[13]), "=r"(q[14]),
        "=r"(q[15]), "=r"(q[16]), "=r"(q[17]), "=r"(q[18]), "=r"(q[19]), "=r"(q[20]), "=r"(q[21]),
        "=r"(q[22]), "=r"(q[23]), "=r"(q[24]), "=r"(q[25]), "=r"(q[26]), "=r"(q[27]), "=r"(q[28]),
        "=r"(q[29]), "=r"(q[30]), "=r"(q[31])
      : "r"(taddr));
}

struct Tc2Args {
  int ex, ey, Lx, Ly;
  long E;                     // elements to apply (the list's length when there is a list)
  const int* list;            // element ids, or null: 0 .. E-1
  const uint32_t* slm;        // per listed element, its slaved local nodes (mixed meshes), or null
  const float* v;             // level-0 vector, 3 per lattice node
  const uint8_t* mask;        // per DOF, 1 = fixed
  const float* w32;           // E x M subcell weights, element-major
  const unsigned char* img;   // stacked table, NC chunks of BBYTES in the smem image layout
  float tscale;               // F16X3: the table's power-of-two scale to undo (else 1)
  float* Y;                   // E x YS element results
  int* err;
};

// The element's nodes on the degree-2 lattice: D = 81, the 27 nodes of a
// triquadratic element (a = ax + 3 (ay + 3 az)); D = 24, the 8 vertices of a
// trilinear element of a mixed mesh (v = vx + 2 (vy + 2 vz)), whose
// results go to the vertex positions of the 27-node layout of Y.
template <int D>
struct Elem;
template <>
struct Elem<81> {
  static constexpr int NN = 27;
  __host__ __device__ static constexpr int off(int a, int d) { return d == 0 ? a % 3 : (d == 1 ? (a / 3) % 3 : a / 9); }
  __host__ __device__ static constexpr int pos(int a, int d) { return off(a, d) - 1; }  // reference position
  __host__ __device__ static constexpr int out(int r) { return r; }
  static constexpr float kRot = 1.f / 36.f;  // 1 / (sum |x|^2 - sum x_d^2) over the nodes
};
template <>
struct Elem<24> {
  static constexpr int NN = 8;
  __host__ __device__ static constexpr int off(int v, int d) { return 2 * ((v >> d) & 1); }
  __host__ __device__ static constexpr int pos(int v, int d) { return off(v, d) - 1; }
  __host__ __device__ static constexpr int out(int r) {
    return 3 * (off(r / 3, 0) + 3 * (off(r / 3, 1) + 3 * off(r / 3, 2))) + r % 3;
  }
  static constexpr float kRot = 1.f / 16.f;
};
template <int D>
__device__ __forceinline__ long elem_lattice_node(int exi, int eyi, int ezi, int a, int Lx, int Ly) {
  return (2 * exi + Elem<D>::off(a, 0)) + (long)Lx * ((2 * eyi + Elem<D>::off(a, 1)) + (long)Ly * (2 * ezi + Elem<D>::off(a, 2)));
}

// Mixed meshes: a slaved local node of a triquadratic element carries the
// linear interpolation of the vertices of its edge, face or cell (u = T_e
// u, from the element's own vertices), and the element's result is folded
// back (y <- T_e^T y): T_e^T K^(e) T_e applied without forming it.
__device__ __forceinline__ void expand_slaved(float* u, uint32_t msk) {
#pragma unroll
  for (int a = 0; a < 27; ++a) {
    const int ax = a % 3, ay = (a / 3) % 3, az = a / 9;
    if (((ax | ay | az) & 1) == 0) continue;  // vertices are never slaved
    if (!((msk >> a) & 1u)) continue;
    const int nx = ax == 1 ? 2 : 1, ny = ay == 1 ? 2 : 1, nz = az == 1 ? 2 : 1;
    const float wgt = 1.f / (float)(nx * ny * nz);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float acc = 0.f;
#pragma unroll
      for (int kz = 0; kz < 2; ++kz)
#pragma unroll
        for (int ky = 0; ky < 2; ++ky)
#pragma unroll
          for (int kx = 0; kx < 2; ++kx) {
            if (kx >= nx || ky >= ny || kz >= nz) continue;
            const int px = ax == 1 ? 2 * kx : ax, py = ay == 1 ? 2 * ky : ay, pz = az == 1 ? 2 * kz : az;
            acc += u[3 * (px + 3 * (py + 3 * pz)) + c];
          }
      u[3 * a + c] = wgt * acc;
    }
  }
}
__device__ __forceinline__ void fold_slaved(float* y, uint32_t msk) {
#pragma unroll
  for (int a = 0; a < 27; ++a) {
    const int ax = a % 3, ay = (a / 3) % 3, az = a / 9;
    if (((ax | ay | az) & 1) == 0) continue;
    if (!((msk >> a) & 1u)) continue;
    const int nx = ax == 1 ? 2 : 1, ny = ay == 1 ? 2 : 1, nz = az == 1 ? 2 : 1;
    const float wgt = 1.f / (float)(nx * ny * nz);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float v = wgt * y[3 * a + c];
#pragma unroll
      for (int kz = 0; kz < 2; ++kz)
#pragma unroll
        for (int ky = 0; ky < 2; ++ky)
#pragma unroll
          for (int kx = 0; kx < 2; ++kx) {
            if (kx >= nx || ky >= ny || kz >= nz) continue;
            const int px = ax == 1 ? 2 * kx : ax, py = ay == 1 ? 2 * ky : ay, pz = az == 1 ? 2 * kz : az;
            y[3 * (px + 3 * (py + 3 * pz)) + c] += v;
          }
      y[3 * a + c] = 0.f;
    }
  }
}

// u_e minus its least-squares rigid motion t + omega x over the element's
// nodes at reference positions x_a (the 27 points of {-1, 0, 1}^3, or the 8
// vertices {-1, 1}^3).  Every subcell matrix
// annihilates rigid motions (they carry no strain), so K^(e_i) u_e is
// unchanged in exact arithmetic, but the rounded operands then carry an
// error relative to the element's deformation instead of its displacement:
// a smooth multigrid correction is locally almost rigid, and rounding it
// whole would leave spurious forces of the rounding unit times |K| |u|.
// For these symmetric node sets sum_a x_a = 0 and sum_a x_a x_a^T = s I
// (s = 18 resp. 8), so t is the mean and omega = sum_a x_a x u_a / (3 s - s).
template <int D>
__device__ __forceinline__ void deflate_rigid(float* u) {
  constexpr int NN = Elem<D>::NN;
  float t[3] = {0.f, 0.f, 0.f}, om[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int nd = 0; nd < NN; ++nd) {
    const float px = (float)Elem<D>::pos(nd, 0), py = (float)Elem<D>::pos(nd, 1), pz = (float)Elem<D>::pos(nd, 2);
    const float ux = u[3 * nd], uy = u[3 * nd + 1], uz = u[3 * nd + 2];
    t[0] += ux;
    t[1] += uy;
    t[2] += uz;
    om[0] += py * uz - pz * uy;
    om[1] += pz * ux - px * uz;
    om[2] += px * uy - py * ux;
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    t[c] *= 1.f / (float)NN;
    om[c] *= Elem<D>::kRot;
  }
#pragma unroll
  for (int nd = 0; nd < NN; ++nd) {
    const float px = (float)Elem<D>::pos(nd, 0), py = (float)Elem<D>::pos(nd, 1), pz = (float)Elem<D>::pos(nd, 2);
    u[3 * nd] -= t[0] + (om[1] * pz - om[2] * py);
    u[3 * nd + 1] -= t[1] + (om[2] * px - om[0] * pz);
    u[3 * nd + 2] -= t[2] + (om[0] * py - om[1] * px);
  }
}

// One element row of the A operand: 16-byte groups g of kKc elements in
// the no-swizzle layout (a split row holds the hi part in K [0, KP) and the
// lo part in [KP, 2 KP)).  Returns the power of two the row was scaled by.
template <int MD, int KP>
__device__ __forceinline__ float store_row(const float* u, unsigned char* dstrow) {
  using O = Opnd<MD>;
  float s = 1.f;
  if constexpr (O::kScaled) {  // largest magnitude into [0.5, 1): FP16's range
    float mx = 0.f;
#pragma unroll
    for (int k = 0; k < KP; ++k) mx = fmaxf(mx, fabsf(u[k]));
    int ex2 = 0;
    frexpf(mx, &ex2);
    s = ldexpf(1.f, ex2);
  }
  const float is = 1.f / s;  // exact: a power of two
#pragma unroll
  for (int g = 0; g < KP / O::kKc; ++g) {
    if constexpr (MD == kTF32) {
      uint4 val;
      val.x = tf32_bits(u[4 * g + 0]);
      val.y = tf32_bits(u[4 * g + 1]);
      val.z = tf32_bits(u[4 * g + 2]);
      val.w = tf32_bits(u[4 * g + 3]);
      *reinterpret_cast<uint4*>(dstrow + 128 * g) = val;
    } else if constexpr (MD == kBF16) {
      uint4 val;
      val.x = pack2(__float2bfloat16_rn(u[8 * g + 0]), __float2bfloat16_rn(u[8 * g + 1]));
      val.y = pack2(__float2bfloat16_rn(u[8 * g + 2]), __float2bfloat16_rn(u[8 * g + 3]));
      val.z = pack2(__float2bfloat16_rn(u[8 * g + 4]), __float2bfloat16_rn(u[8 * g + 5]));
      val.w = pack2(__float2bfloat16_rn(u[8 * g + 6]), __float2bfloat16_rn(u[8 * g + 7]));
      *reinterpret_cast<uint4*>(dstrow + 128 * g) = val;
    } else {
      uint32_t hw[4], lw[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if constexpr (MD == kBF16X3) {
          __nv_bfloat16 h0, l0, h1, l1;
          split_bf16(u[8 * g + 2 * q], h0, l0);
          split_bf16(u[8 * g + 2 * q + 1], h1, l1);
          hw[q] = pack2(h0, h1);
          lw[q] = pack2(l0, l1);
        } else {
          __half h0, l0, h1, l1;
          split_f16(u[8 * g + 2 * q] * is, h0, l0);
          split_f16(u[8 * g + 2 * q + 1] * is, h1, l1);
          hw[q] = pack2(h0, h1);
          lw[q] = pack2(l0, l1);
        }
      }
      *reinterpret_cast<uint4*>(dstrow + 128 * g) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
      *reinterpret_cast<uint4*>(dstrow + 128 * (g + KP / O::kKc)) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
  }
  return s;
}

template <int MD, int D, int M>
__global__ void __launch_bounds__(kThreads, 1) k_tc2_apply(Tc2Args a) {
  using S = Shape<MD, D, M>;
  using O = Opnd<MD>;
  constexpr int NS = O::kStages;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem;                  // 2 x ABYTES
  unsigned char* sB = smem + 2 * S::ABYTES;  // NS x BBYTES
  __shared__ __align__(8) uint64_t bfull[NS], bempty[NS], afull[2], aempty[2], tfull[2], tempty[2], sfull[2],
      mdone;
  __shared__ float rscale[2][kTm];  // F16X3: the power of two each element row was scaled by
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long ntiles = (a.E + kTm - 1) / kTm;
  const long ntl = (long)blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 32) {
    for (int s = 0; s < NS; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bfull[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bempty[s])));
    }
    for (int s = 0; s < 2; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&afull[s])), "r"(kTm));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&aempty[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&tfull[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&tempty[s])), "r"(kTm));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&sfull[s])), "r"(kTm));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&mdone)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_flag = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    // ---- producer: table chunks into the B ring ----
    if (lane == 0) {
      long q = 0;
      const long nq = ntl * S::NC;
      for (; q < nq; ++q) {
        const int s = (int)(q % NS), c = (int)(q % S::NC);
        if (!wait_or_abort(&bempty[s], (uint32_t)(((q / NS) & 1) ^ 1), &abort_flag)) break;
        const uint32_t bytes = c == S::NC - 1 ? (uint32_t)(S::LASTNP / 8) * S::SBO : S::BBYTES;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(&bfull[s])),
                     "r"(bytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                su32(sB + (size_t)s * S::BBYTES)),
            "l"(a.img + (size_t)c * S::BBYTES), "r"(bytes), "r"(su32(&bfull[s]))
            : "memory");
      }
      if (q < nq) {  // aborted: let the copies in flight land before the CTA exits
        atomicExch(a.err, 1);
        for (long p = q - 1; p >= 0 && p >= q - NS; --p) drain_wait(&bfull[p % NS], (uint32_t)((p / NS) & 1));
      }
    }
  } else if (warp == 1) {
    // ---- MMA issue ----
    if (lane == 0) {
      const uint32_t abase = su32(sA), bbase = su32(sB);
      bool ok = true;
      for (long j = 0; j < ntl && ok; ++j) {
        const int ab = (int)(j & 1);
        ok = wait_or_abort(&afull[ab], (uint32_t)((j >> 1) & 1), &abort_flag);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        for (int c = 0; c < S::NC; ++c) {
          const long q = j * S::NC + c;
          const int s = (int)(q % NS), acc = (int)(q & 1);
          ok = wait_or_abort(&bfull[s], (uint32_t)((q / NS) & 1), &abort_flag) &&
               wait_or_abort(&tempty[acc], (uint32_t)(((q >> 1) & 1) ^ 1), &abort_flag);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t n = c == S::NC - 1 ? (uint32_t)S::LASTNP : (uint32_t)S::NCH;
          const uint32_t idesc = (1u << 4) | (O::kFmt << 7) | (O::kFmt << 10) | ((n >> 3) << 17) |
                                 ((uint32_t)(kTm >> 4) << 24);
          const uint32_t dt = tmem + (uint32_t)(acc * 256);
          const uint32_t ao = abase + (uint32_t)ab * S::ABYTES, bo = bbase + (uint32_t)s * S::BBYTES;
#pragma unroll
          for (int t = 0; t < O::kProducts * S::KS; ++t) {
            // products: a_hi b_hi, a_lo b_hi, a_hi b_lo (K-slice t % KS of each part)
            const int pr = t / S::KS, ks = t % S::KS;
            const int apart = pr == 1 ? 1 : 0, bpart = pr == 2 ? 1 : 0;
            const uint64_t ad = sdesc(ao + 256u * (apart * S::KS + ks), 128u, S::SBO);
            const uint64_t bd = sdesc(bo + 256u * (bpart * S::KS + ks), 128u, S::SBO);
            const uint32_t accum = t > 0 ? 1u : 0u;
            if constexpr (MD == kTF32)
              asm volatile(
                  "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                  " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
                  "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
            else
              asm volatile(
                  "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                  " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
                  "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
          }
          commit(&bempty[s]);   // the B stage is free once these MMAs are done
          commit(&tfull[acc]);  // and the accumulator is ready for the epilogue
        }
        if (!ok) break;
        commit(&aempty[ab]);  // all chunks of the tile are issued: A buffer free when done
      }
      if (!ok) atomicExch(a.err, 1);
      // every MMA issued above has completed before the TMEM is freed
      commit(&mdone);
      drain_wait(&mdone, 0);
    }
  } else if (warp < 6) {
    // ---- epilogue: weighted reduce over subcells ----
    const int quarter = warp & 3;  // a warp reads the TMEM lanes of its sub-partition
    const int row = 32 * quarter + lane;
    const uint32_t tl = tmem + ((uint32_t)(32 * quarter) << 16);
    for (long j = 0; j < ntl; ++j) {
      const long ei = (blockIdx.x + j * gridDim.x) * (long)kTm + row;
      const bool live = ei < a.E;
      const long e = !live ? 0 : (a.list != nullptr ? (long)a.list[ei] : ei);
      float sc = a.tscale;
      if constexpr (O::kScaled) {
        // the gather of this tile published the row scales before its
        // arrival; the buffer is not rewritten before this tile's MMAs end
        if (!__all_sync(0xffffffffu, wait_or_abort(&sfull[j & 1], (uint32_t)((j >> 1) & 1), &abort_flag))) {
          atomicExch(a.err, 1);
          break;
        }
        sc *= rscale[j & 1][row];
      }
      float w[M];
#pragma unroll
      for (int i = 0; i < M; ++i) w[i] = live ? __ldg(a.w32 + e * M + i) : 0.f;
      float y[D];
#pragma unroll
      for (int r = 0; r < D; ++r) y[r] = 0.f;
      bool ok = true;
#pragma unroll
      for (int c = 0; c < S::NC; ++c) {
        const long q = j * S::NC + c;
        const int acc = (int)(q & 1);
        ok = __all_sync(0xffffffffu, wait_or_abort(&tfull[acc], (uint32_t)((q >> 1) & 1), &abort_flag));
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        constexpr int G = S::NCH / 32;
        const int ng = c == S::NC - 1 ? (S::LASTN + 31) / 32 : G;
#pragma unroll
        for (int g = 0; g < G; ++g) {
          if (g < ng) {
            uint32_t qv[32];
            tmem_ld32(tl + (uint32_t)(acc * 256 + 32 * g), qv);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int t = 0; t < 32; ++t) {
              const int col = c * S::NCH + 32 * g + t;
              if (col < S::ROWS) y[col % D] = fmaf(w[col / D], __uint_as_float(qv[t]), y[col % D]);
            }
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        arrive(&tempty[acc]);
      }
      if (!ok) {
        atomicExch(a.err, 1);
        break;
      }
      if (live) {
        if constexpr (D == 81) {
          if (a.slm != nullptr) fold_slaved(y, a.slm[ei]);
          float4* dst = reinterpret_cast<float4*>(a.Y + e * S::YS);
#pragma unroll
          for (int t = 0; t < S::YS / 4; ++t) {
            const int r = 4 * t;
            dst[t] = make_float4(r < D ? sc * y[r] : 0.f, r + 1 < D ? sc * y[r + 1] : 0.f,
                                 r + 2 < D ? sc * y[r + 2] : 0.f, r + 3 < D ? sc * y[r + 3] : 0.f);
          }
        } else {  // the vertex positions of the 27-node layout (the others are slaved)
          float* dst = a.Y + e * S::YS;
#pragma unroll
          for (int r = 0; r < D; ++r) dst[Elem<D>::out(r)] = sc * y[r];
        }
      }
    }
  } else {
    // ---- gather u_e of each tile into an A buffer ----
    for (long j = 0; j < ntl; ++j) {
      const int ab = (int)(j & 1);
      if (!wait_or_abort(&aempty[ab], (uint32_t)(((j >> 1) & 1) ^ 1), &abort_flag)) {
        atomicExch(a.err, 1);
        break;
      }
#pragma unroll 1
      for (int rr = 0; rr < 2; ++rr) {
        const int row = 32 * (warp - 6) + lane + 64 * rr;
        const long ei = (blockIdx.x + j * gridDim.x) * (long)kTm + row;
        float u[S::KP];
#pragma unroll
        for (int k = 0; k < S::KP; ++k) u[k] = 0.f;
        if (ei < a.E) {
          const long e = a.list != nullptr ? (long)a.list[ei] : ei;
          const int exi = (int)(e % a.ex), eyi = (int)((e / a.ex) % a.ey), ezi = (int)(e / ((long)a.ex * a.ey));
#pragma unroll
          for (int nd = 0; nd < D / 3; ++nd) {
            const long d0 = 3 * elem_lattice_node<D>(exi, eyi, ezi, nd, a.Lx, a.Ly);
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) {
              const float x = __ldg(a.v + d0 + cc);
              u[3 * nd + cc] = __ldg(a.mask + d0 + cc) ? 0.f : x;
            }
          }
          if constexpr (D == 81)
            if (a.slm != nullptr) expand_slaved(u, a.slm[ei]);
          deflate_rigid<D>(u);
        }
        unsigned char* dstrow = sA + (size_t)ab * S::ABYTES + (size_t)(row >> 3) * S::SBO + (row & 7) * 16;
        const float s = store_row<MD, S::KP>(u, dstrow);
        if constexpr (O::kScaled) {
          rscale[ab][row] = s;
          arrive(&sfull[ab]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
        arrive(&afull[ab]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// The stacked table in the shared-memory image of its chunks: chunk c, row
// n (stacked row c * nch + n = 81 i + R: row R of subcell i), K column k (an
// element DOF; the subcell matrices are symmetric); zero padding beyond the
// table.  Single modes round once (TF32 to nearest with ties away, BF16 to
// nearest even); split modes store hi in columns [0, kp) and lo in
// [kp, 2 kp), FP16 after scaling the table by tinv (a power of two).
__global__ void k_tc2_image(int mode, int D, int m, int nch, int kp, int parts, int kc, uint32_t sbo, double tinv,
                            const double* __restrict__ tab, unsigned char* __restrict__ img, long total) {
  const int es = mode == kTF32 ? 4 : 2;
  const int kr = kp * parts;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const int k = (int)(t % kp);
    const long rowg = t / kp;
    const int c = (int)(rowg / nch), n = (int)(rowg % nch);
    const long gr = (long)c * nch + n;
    double x = 0.0;
    if (gr < (long)D * m && k < D) {
      const long i = gr / D, R = gr % D;
      x = tab[(i * D + R) * D + k];
    }
    auto at = [&](int kk) {
      return (size_t)c * nch * kr * es + (size_t)(n >> 3) * sbo + (size_t)(kk / kc) * 128 + (size_t)(n & 7) * 16 +
             (size_t)(kk % kc) * es;
    };
    if (mode == kTF32) {
      *reinterpret_cast<uint32_t*>(img + at(k)) = tf32_bits((float)x);
    } else if (mode == kBF16) {
      *reinterpret_cast<__nv_bfloat16*>(img + at(k)) = __double2bfloat16(x);
    } else if (mode == kBF16X3) {
      const __nv_bfloat16 h = __double2bfloat16(x);
      *reinterpret_cast<__nv_bfloat16*>(img + at(k)) = h;
      *reinterpret_cast<__nv_bfloat16*>(img + at(k + kp)) = __double2bfloat16(x - (double)__bfloat162float(h));
    } else {
      const double xs = x * tinv;
      const __half h = __double2half(xs);
      *reinterpret_cast<__half*>(img + at(k)) = h;
      *reinterpret_cast<__half*>(img + at(k + kp)) = __double2half(xs - (double)__half2float(h));
    }
  }
}

// y_n = sum of y_e over the elements containing node n (fixed order), then
//   mode 0: out = b - y;  mode 1: out = v + omega D^-1 (b - y);  mode 2: out = y.
// Fixed DOFs are identity rows: y = v there.
template <int YS>
__global__ void k_tc2_gather(int Lx, int Ly, int Lz, int ex, int ey, int ez, const float* __restrict__ Y,
                             const float* __restrict__ b, const float* __restrict__ v,
                             const float* __restrict__ dinv, const uint8_t* __restrict__ mask, float omega,
                             int mode, float* __restrict__ out) {
  const long nn = (long)Lx * Ly * Lz;
  for (long node = blockIdx.x * (long)blockDim.x + threadIdx.x; node < nn; node += (long)gridDim.x * blockDim.x) {
    const int i = (int)(node % Lx), j = (int)((node / Lx) % Ly), l = (int)(node / ((long)Lx * Ly));
    const int co[3] = {i, j, l}, ext[3] = {ex, ey, ez};
    int e0[3], e1[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {  // elements along the axis holding lattice coordinate co
      const int c = co[ax];
      if (c & 1) {
        e0[ax] = e1[ax] = c >> 1;
      } else {
        e0[ax] = (c >> 1) - 1 < 0 ? 0 : (c >> 1) - 1;
        e1[ax] = (c >> 1) > ext[ax] - 1 ? ext[ax] - 1 : (c >> 1);
      }
    }
    const bool all_fixed = mask[3 * node] && mask[3 * node + 1] && mask[3 * node + 2];
    float y[3] = {0.f, 0.f, 0.f};
    for (int ez_ = e0[2]; !all_fixed && ez_ <= e1[2]; ++ez_)
      for (int ey_ = e0[1]; ey_ <= e1[1]; ++ey_)
        for (int ex_ = e0[0]; ex_ <= e1[0]; ++ex_) {
          const long e = ex_ + (long)ex * (ey_ + (long)ey * ez_);
          const int la = (i - 2 * ex_) + 3 * ((j - 2 * ey_) + 3 * (l - 2 * ez_));
          const float* ye = Y + e * YS + 3 * la;
          y[0] += ye[0];
          y[1] += ye[1];
          y[2] += ye[2];
        }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const long d = 3 * node + c;
      const float yc = mask[d] ? v[d] : y[c];
      if (mode == 0) out[d] = b[d] - yc;
      else if (mode == 1) out[d] = v[d] + omega * dinv[d] * (b[d] - yc);
      else out[d] = yc;
    }
  }
}

template <int MD, int D, int M>
cudaError_t run_apply(const Level& L0, long count, const int* list, const uint32_t* slm, const float* v,
                      const float* w32, const unsigned char* img, float tscale, float* Y, int* err, int sms,
                      cudaStream_t st) {
  using S = Shape<MD, D, M>;
  static std::once_flag once;  // handles may be created from several threads
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(k_tc2_apply<MD, D, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
  });
  if (attr != cudaSuccess) return attr;
  if (count <= 0) return cudaSuccess;
  Tc2Args a;
  a.ex = L0.ex;
  a.ey = L0.ey;
  a.Lx = L0.Lx;
  a.Ly = L0.Ly;
  a.E = count;
  a.list = list;
  a.slm = slm;
  a.v = v;
  a.mask = L0.mask;
  a.w32 = w32;
  a.img = img;
  a.tscale = tscale;
  a.Y = Y;
  a.err = err;
  const long ntiles = (count + kTm - 1) / kTm;
  const int g = (int)(ntiles < sms ? ntiles : sms);
  k_tc2_apply<MD, D, M><<<g, kThreads, S::SMEM, st>>>(a);
  return cudaGetLastError();
}

template <int MD, int D>
size_t image_bytes_for(int m) {
  switch (m) {
    case 1: return (size_t)Shape<MD, D, 1>::NC * Shape<MD, D, 1>::BBYTES;
    case 8: return (size_t)Shape<MD, D, 8>::NC * Shape<MD, D, 8>::BBYTES;
    case 27: return (size_t)Shape<MD, D, 27>::NC * Shape<MD, D, 27>::BBYTES;
    default: return 0;
  }
}

template <int MD, int D>
cudaError_t apply_for(int m, const Level& L0, long count, const int* list, const uint32_t* slm, const float* v,
                      const float* w32, const unsigned char* img, float tscale, float* Y, int* err, int sms,
                      cudaStream_t st) {
  if (m == 27) return run_apply<MD, D, 27>(L0, count, list, slm, v, w32, img, tscale, Y, err, sms, st);
  if (m == 8) return run_apply<MD, D, 8>(L0, count, list, slm, v, w32, img, tscale, Y, err, sms, st);
  if (m == 1) return run_apply<MD, D, 1>(L0, count, list, slm, v, w32, img, tscale, Y, err, sms, st);
  return cudaErrorInvalidValue;
}

template <int D>
cudaError_t apply_mode(int mode, int m, const Level& L0, long count, const int* list, const uint32_t* slm,
                       const float* v, const float* w32, const unsigned char* img, float tscale, float* Y, int* err,
                       int sms, cudaStream_t st) {
  switch (mode) {
    case kTF32: return apply_for<kTF32, D>(m, L0, count, list, slm, v, w32, img, tscale, Y, err, sms, st);
    case kBF16: return apply_for<kBF16, D>(m, L0, count, list, slm, v, w32, img, tscale, Y, err, sms, st);
    case kBF16X3: return apply_for<kBF16X3, D>(m, L0, count, list, slm, v, w32, img, tscale, Y, err, sms, st);
    case kF16X3: return apply_for<kF16X3, D>(m, L0, count, list, slm, v, w32, img, tscale, Y, err, sms, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int MD, int D>
void image_for(int m, const double* tab, double tinv, unsigned char* img, cudaStream_t st) {
  using S = Shape<MD, D, 1>;
  using O = Opnd<MD>;
  const size_t bytes = image_bytes_for<MD, D>(m);
  // one thread per (chunk row, K column of one part)
  const long total = (long)(bytes / O::kEs / O::kParts);
  long g = (total + 255) / 256;
  if (g > 4096) g = 4096;
  k_tc2_image<<<(int)g, 256, 0, st>>>(MD, D, m, O::kNch, S::KP, O::kParts, O::kKc, S::SBO, tinv, tab, img, total);
}

template <int D>
size_t image_bytes_mode(int mode, int m) {
  switch (mode) {
    case kTF32: return image_bytes_for<kTF32, D>(m);
    case kBF16: return image_bytes_for<kBF16, D>(m);
    case kBF16X3: return image_bytes_for<kBF16X3, D>(m);
    case kF16X3: return image_bytes_for<kF16X3, D>(m);
    default: return 0;
  }
}

}  // namespace

bool tc2_supported(int n) { return n >= 1 && n <= 3; }

size_t tc2_image_bytes(int mode, int m, int dofs) {
  return dofs == 24 ? image_bytes_mode<24>(mode, m) : image_bytes_mode<81>(mode, m);
}

size_t tc2_result_stride() { return (size_t)Shape<kTF32, 81, 1>::YS; }

float tc2_table_scale(int mode, const double* tab_host, size_t count) {
  if (mode != kF16X3) return 1.f;
  double mx = 0.0;
  for (size_t t = 0; t < count; ++t) mx = std::fmax(mx, std::fabs(tab_host[t]));
  if (!(mx > 0.0)) return 1.f;
  int ex2 = 0;
  std::frexp(mx, &ex2);  // mx / 2^ex2 in [0.5, 1)
  return (float)std::ldexp(1.0, ex2);
}

void launch_tc2_image(int mode, int m, int dofs, const double* tab, float tscale, unsigned char* img,
                      cudaStream_t st) {
  const double tinv = 1.0 / (double)tscale;
  if (dofs == 24) {
    switch (mode) {
      case kTF32: image_for<kTF32, 24>(m, tab, tinv, img, st); break;
      case kBF16: image_for<kBF16, 24>(m, tab, tinv, img, st); break;
      case kBF16X3: image_for<kBF16X3, 24>(m, tab, tinv, img, st); break;
      default: image_for<kF16X3, 24>(m, tab, tinv, img, st); break;
    }
    return;
  }
  switch (mode) {
    case kTF32: image_for<kTF32, 81>(m, tab, tinv, img, st); break;
    case kBF16: image_for<kBF16, 81>(m, tab, tinv, img, st); break;
    case kBF16X3: image_for<kBF16X3, 81>(m, tab, tinv, img, st); break;
    default: image_for<kF16X3, 81>(m, tab, tinv, img, st); break;
  }
}

cudaError_t launch_tc2_apply(const TcOp& tc, const Level& L0, const float* v, cudaStream_t st) {
  if (L0.el2 != nullptr) {  // mixed mesh: triquadratic elements with their slaved nodes, then trilinear ones
    cudaError_t e = apply_mode<81>(tc.mode, tc.m, L0, L0.ne2, L0.el2, L0.sl2, v, tc.w32, tc.img, tc.tscale, tc.Y2,
                                   tc.err, tc.sms, st);
    if (e != cudaSuccess) return e;
    return apply_mode<24>(tc.mode, tc.m, L0, L0.ne1, L0.el1, nullptr, v, tc.w32, tc.img1, tc.tscale1, tc.Y2,
                          tc.err, tc.sms, st);
  }
  const long E = (long)L0.ex * L0.ey * L0.ez;
  return apply_mode<81>(tc.mode, tc.m, L0, E, nullptr, nullptr, v, tc.w32, tc.img, tc.tscale, tc.Y2, tc.err,
                        tc.sms, st);
}

void launch_tc2_gather(const Level& L0, const float* Y, const float* b, const float* v, const float* dinv,
                       float omega, int mode, float* out, cudaStream_t st) {
  long g = (L0.nn + 255) / 256;
  if (g > 8192) g = 8192;
  k_tc2_gather<Shape<kTF32, 81, 1>::YS><<<(int)g, 256, 0, st>>>(L0.Lx, L0.Ly, L0.Lz, L0.ex, L0.ey, L0.ez, Y, b,
                                                                 v, dinv, L0.mask, omega, mode, out);
}

}  // namespace tos
