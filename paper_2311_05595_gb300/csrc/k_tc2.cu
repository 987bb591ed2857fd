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
// weighted reduce over subcells is thread-local in the epilogue: the rows
// are stacked DOF-major (all subcells of output DOF r together), so thread e
// reads the columns of one output at a time and forms sum_i w_{e,i} Z[i, r]
// in a fixed order, with no cross-lane reduction.
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
// Work unit: a pair of 128-element tiles, so each table chunk brought to
// shared memory serves 256 elements (two MMAs per K-slice, two TMEM
// accumulators).  Warp roles (192 threads, one CTA per SM, persistent over
// work units):
//   warp 0     allocates the 512 TMEM columns; lane 0 brings each unit's A
//              tiles and streams table chunks into a ring of B stages;
//   warp 1     lane 0 issues the MMAs of each chunk into one of two TMEM
//              accumulators and commits their completion to mbarriers;
//   warps 2-5  epilogue: read each 32-column group of the accumulator
//              (tcgen05.ld), weighted sum over its subcells, store the
//              output DOF.
// The (unit, chunk) work items are split evenly over one CTA per SM, so
// every SM works and the CTAs start at different chunks (the chunks'
// outputs are independent) instead of all streaming the same chunk from L2
// at the same moment.
// The A operand rows (u_e with fixed DOFs as zero, slaved nodes expanded,
// minus the least-squares rigid motion, scaled and split) are assembled by
// a separate high-occupancy kernel, k_tc2_pack, straight into the
// shared-memory image of their tiles: the scattered gathers then hide their
// latency behind thousands of threads, and the producer moves a pair's two
// A tiles with one bulk copy.
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

constexpr int kTm = 128;            // elements per tile (TMEM lanes of one MMA)
constexpr int kPair = 2;            // tiles per work unit: each table chunk serves both
constexpr int kUnit = kPair * kTm;  // elements per work unit
constexpr int kThreads = 192;       // 6 warps, one per role below
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
  static constexpr int kStages = MD == kBF16 ? 3 : 2;      // B ring
  static constexpr int kParts = kSplit ? 2 : 1;            // hi (and lo) K-slices per row
  static constexpr int kProducts = kSplit ? 3 : 1;
  // operand format in the instruction descriptor: TF32 2, BF16 1, F16 0
  static constexpr uint32_t kFmt = MD == kTF32 ? 2u : (MD == kF16X3 ? 0u : 1u);
};

// Stacked rows are DOF-major and unpadded: chunk c holds the OPC outputs
// r = c OPC + o (OPC = 128 / M, at most 128), output o's M subcell rows at
// columns [M o, M o + M) of the chunk, then zero rows up to NCH (a multiple
// of 16, the MMA's N).  Every accumulator has a 128-column TMEM slot.  Where
// M divides 32 every 32-column group holds whole outputs; otherwise (M = 27:
// four outputs in 112 columns instead of one per 32) an output may straddle
// two groups and the epilogue keeps a partial sum per output of the chunk.
template <int MD, int D, int M>
struct Shape {
  using O = Opnd<MD>;
  static constexpr int KP = (D + O::kKstep - 1) / O::kKstep * O::kKstep;  // padded K of one part
  static constexpr int KR = KP * O::kParts;                                 // K extent of a row
  static constexpr int OPC = M >= 128 ? 1 : 128 / M;                        // outputs per chunk
  static constexpr int NCH = (OPC * M + 15) / 16 * 16;                      // rows of a chunk (MMA N)
  static constexpr int NC = (D + OPC - 1) / OPC;                            // chunks
  static constexpr int LASTO = D - (NC - 1) * OPC;                          // outputs of the last
  static constexpr int LASTN = LASTO * M;
  static constexpr int LASTNP = (LASTN + 15) / 16 * 16;                     // MMA N of the last
  static constexpr int NG = (NCH + 31) / 32;                                // 32-column groups of a chunk
  static constexpr bool kWhole = 32 % M == 0;                               // groups hold whole outputs
  static constexpr int KS = KP / O::kKstep;                                 // MMAs of one product
  static constexpr uint32_t SBO = (uint32_t)(KR / O::kKc) * 128u;
  static constexpr uint32_t ABYTES = (uint32_t)kTm * KR * O::kEs;
  static constexpr uint32_t BBYTES = (uint32_t)NCH * KR * O::kEs;
  static constexpr size_t SMEM = (size_t)kPair * ABYTES + (size_t)O::kStages * BBYTES;
};
constexpr int kAccCols = 128;  // TMEM columns of one accumulator slot

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
  long E;                     // elements to apply (the list's length when there is a list)
  const int* list;            // element ids, or null: 0 .. E-1
  const unsigned char* apack; // the packed A tiles (k_tc2_pack), tile t at t * ABYTES
  const float* escale;        // F16X3: per listed element, the power of two its row was scaled by
  const float* w32;           // E x M subcell weights, element-major
  const unsigned char* img;   // stacked table, NC chunks of BBYTES in the smem image layout
  float tscale;               // F16X3: the table's power-of-two scale to undo (else 1)
  float* Y;                   // element results, DOF-major: Y[r * Ey + e] (r of the 27-node layout)
  long Ey;                    // elements of the level (the stride of Y)
  int* err;
};

struct PackArgs {
  int ex, ey, Lx, Ly;
  long E, rows;               // listed elements; rows packed (whole work units)
  const int* list;
  const uint32_t* slm;
  const float* v;             // level-0 vector, 3 per lattice node
  const uint8_t* mask;        // per DOF, 1 = fixed
  unsigned char* apack;
  float* escale;
  long pblocks;               // blocks that pack rows; the others multiply trilinear elements
  long E1;                    // trilinear elements of a mixed mesh (L0.el1 order), or 0
  const int* list1;
  const float* K1;            // their FP32 packed vertex blocks (kQ1Sym each)
  float* Y;                   // element results, DOF-major: Y[r * Ey + e]
  long Ey;
};

// The element's nodes on the degree-2 lattice: D = 81, the 27 nodes of a
// triquadratic element (a = ax + 3 (ay + 3 az)), the rows of the stacked
// contraction; D = 24, the 8 vertices of a trilinear element of a mixed mesh
// (v = vx + 2 (vy + 2 vz)), whose FP32 products go to the vertex positions
// of the 27-node layout of Y.
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
  __host__ __device__ static constexpr int off(int v, int d) { return 2 * ((v >> d) & 1); }
  __host__ __device__ static constexpr int out(int r) {
    return 3 * (off(r / 3, 0) + 3 * (off(r / 3, 1) + 3 * off(r / 3, 2))) + r % 3;
  }
};
template <int D>
__device__ __forceinline__ long elem_lattice_node(int exi, int eyi, int ezi, int a, int Lx, int Ly) {
  return (2 * exi + Elem<D>::off(a, 0)) + (long)Lx * ((2 * eyi + Elem<D>::off(a, 1)) + (long)Ly * (2 * ezi + Elem<D>::off(a, 2)));
}

// Mixed meshes: a slaved local node of a triquadratic element carries the
// linear interpolation of the vertices of its edge, face or cell (u = T_e
// u, from the element's own vertices).  The results are folded back after
// assembly, y <- T^T y on the node lattice: the constraint T is local to each
// element, so sum_e T_e^T y_e = T^T sum_e y_e, and T_e^T K^(e) T_e is
// applied without forming it.
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


// u_e minus its least-squares rigid motion t + omega x over the element's
// nodes at reference positions x_a (the 27 points of {-1, 0, 1}^3).  Every
// subcell matrix
// annihilates rigid motions (they carry no strain), so K^(e_i) u_e is
// unchanged in exact arithmetic, but the rounded operands then carry an
// error relative to the element's deformation instead of its displacement:
// a smooth multigrid correction is locally almost rigid, and rounding it
// whole would leave spurious forces of the rounding unit times |K| |u|.
// For this symmetric node set sum_a x_a = 0 and sum_a x_a x_a^T = s I
// (s = 18), so t is the mean and omega = sum_a x_a x u_a / (3 s - s).
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

// Trilinear elements of a mixed mesh: y_e = K^(e) u_e on their 24 vertex
// DOFs in FP32 on the CUDA cores.  With 576 products per element (against
// 27 x 6561 for a triquadratic one) the tensor-core pipeline would spend
// these elements in its fixed latencies; here the FP32 matrices are the
// packed upper triangles of the elements' vertex blocks (k_q1v_compact32,
// after each refresh), 1.2 KB per element.  A warp takes four consecutive
// listed elements: their matrices go to shared memory by asynchronous
// 16-byte copies (no registers held), lane 8 s + q gathers vertex q of
// element s (fixed DOFs as zero), then forms its vertex's three rows
// (columns, by symmetry) in a fixed order and writes them to their places
// in the 27-node layout of Y.  Blocks blk = 0 .. nblk-1 of 128 threads; the
// row packing of the triquadratic elements launches these blocks beside its
// own, so that the two latency-bound gathers overlap.
constexpr int kQ1Warps = 4;
constexpr int kQ1PerWarp = 4;
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void q1v_rows(const PackArgs& a, long blk, long nblk) {
  __shared__ __align__(16) float ks[kQ1Warps][kQ1PerWarp * kQ1Sym];
  __shared__ float us[kQ1Warps][kQ1PerWarp][24];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, sub = lane >> 3, vq = lane & 7;
  const long stride = nblk * kQ1Warps * kQ1PerWarp;
  for (long t0 = (blk * kQ1Warps + w) * kQ1PerWarp; t0 < a.E1; t0 += stride) {  // warp-uniform
    const int nel = a.E1 - t0 < kQ1PerWarp ? (int)(a.E1 - t0) : kQ1PerWarp;
    const float4* src = reinterpret_cast<const float4*>(a.K1 + t0 * kQ1Sym);
    float4* dst = reinterpret_cast<float4*>(ks[w]);
    for (int q = lane; q < nel * (kQ1Sym / 4); q += 32) cp_async16(dst + q, src + q);
    asm volatile("cp.async.commit_group;" ::: "memory");
    const bool live = sub < nel;
    int e = 0;
    if (live) {
      e = a.list1[t0 + sub];
      const int exi = e % a.ex, eyi = (e / a.ex) % a.ey, ezi = e / (a.ex * a.ey);
      const long d = 3 * elem_lattice_node<24>(exi, eyi, ezi, vq, a.Lx, a.Ly);
      float vd[3];
      uint8_t md[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        vd[c] = a.v[d + c];
        md[c] = a.mask[d + c];
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) us[w][sub][3 * vq + c] = md[c] ? 0.f : vd[c];
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncwarp();
    if (live) {
      const float* km = ks[w] + sub * kQ1Sym;
      const float* um = us[w][sub];
#pragma unroll
      for (int c3 = 0; c3 < 3; ++c3) {
        // entry (min, max) of the packed rows: along column c < r the index
        // steps by 23 - c, along row r (c >= r) by 1
        const int r = 3 * vq + c3;
        float acc = 0.f;
        int idx = r;  // (0, r)
#pragma unroll
        for (int c = 0; c < 24; ++c) {
          acc += km[idx] * um[c];
          idx += c < r ? 23 - c : 1;
        }
        a.Y[(long)Elem<24>::out(r) * a.Ey + e] = acc;
      }
    }
    __syncwarp();
  }
}
__global__ void __launch_bounds__(32 * kQ1Warps, 8) k_q1v_apply32(PackArgs a) { q1v_rows(a, blockIdx.x, gridDim.x); }

// One element's A row per thread, written into the image of its tile
// (whole work units: rows past the list are zeros).
template <int MD, int D>
__global__ void __launch_bounds__(128) k_tc2_pack(PackArgs a) {
  using S = Shape<MD, D, 1>;  // the row layout does not depend on M
  using O = Opnd<MD>;
  if constexpr (D == 81) {
    if ((long)blockIdx.x >= a.pblocks) {  // the trilinear elements' products
      q1v_rows(a, (long)blockIdx.x - a.pblocks, (long)gridDim.x - a.pblocks);
      return;
    }
  }
  for (long ei = blockIdx.x * (long)blockDim.x + threadIdx.x; ei < a.rows; ei += a.pblocks * blockDim.x) {
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
        for (int cc = 0; cc < 3; ++cc) u[3 * nd + cc] = __ldg(a.mask + d0 + cc) ? 0.f : __ldg(a.v + d0 + cc);
      }
      if constexpr (D == 81)
        if (a.slm != nullptr) expand_slaved(u, a.slm[ei]);
      deflate_rigid<D>(u);
    }
    const long tile = ei / kTm;
    const int lrow = (int)(ei % kTm);
    unsigned char* dstrow = a.apack + (size_t)tile * S::ABYTES + (size_t)(lrow >> 3) * S::SBO + (lrow & 7) * 16;
    const float sv = store_row<MD, S::KP>(u, dstrow);
    if constexpr (O::kScaled) a.escale[ei] = sv;
  }
}

template <int MD, int D, int M>
__global__ void __launch_bounds__(kThreads, 1) k_tc2_apply(Tc2Args a) {
  using S = Shape<MD, D, M>;
  using O = Opnd<MD>;
  constexpr int NS = O::kStages;
  static_assert(kThreads == 6 * 32, "one warp per role: producer, MMA, 4 epilogue");
  static_assert(S::NCH <= kAccCols && 2 * 2 * kAccCols <= kTmemCols, "two accumulator buffers of a tile pair");
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem;                        // the pair's two A tiles
  unsigned char* sB = smem + kPair * S::ABYTES;    // NS x BBYTES
  __shared__ __align__(8) uint64_t bfull[NS], bempty[NS], afull, aempty, tfull[2], tempty[2], mdone;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // Work items are (unit, chunk) pairs in unit order; CTA b takes the
  // contiguous range [i0, i1), which touches ntl units (segments): every SM
  // works, and the CTAs start at different chunks.
  const long nunits = (a.E + kUnit - 1) / kUnit;
  const long nitems = nunits * S::NC;
  const long i0 = (long)blockIdx.x * nitems / gridDim.x, i1 = ((long)blockIdx.x + 1) * nitems / gridDim.x;
  const long u0 = i0 / S::NC;
  const long ntl = i1 > i0 ? (i1 - 1) / S::NC - u0 + 1 : 0;
  auto segment = [&](long j, long& unit, int& c0, int& c1) {  // chunks [c0, c1) of unit u0 + j
    unit = u0 + j;
    c0 = unit == u0 ? (int)(i0 - unit * S::NC) : 0;
    c1 = (unit + 1) * S::NC <= i1 ? S::NC : (int)(i1 - unit * S::NC);
  };

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
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&afull)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&aempty)));
    for (int s = 0; s < 2; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&tfull[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&tempty[s])), "r"(kTm));
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
    // ---- producer: each unit's A tiles, then its table chunks into the B ring ----
    if (lane == 0) {
      long q = 0, j = 0;
      bool ok = true;
      for (; j < ntl && ok; ++j) {
        if (!(ok = wait_or_abort(&aempty, (uint32_t)((j & 1) ^ 1), &abort_flag))) break;
        long unit;
        int c0, c1;
        segment(j, unit, c0, c1);
        const uint32_t abytes = (uint32_t)kPair * S::ABYTES;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(&afull)), "r"(abytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                su32(sA)),
            "l"(a.apack + (size_t)unit * abytes), "r"(abytes), "r"(su32(&afull))
            : "memory");
        for (int c = c0; c < c1; ++c, ++q) {
          const int s = (int)(q % NS);
          const int cc = c;
          if (!(ok = wait_or_abort(&bempty[s], (uint32_t)(((q / NS) & 1) ^ 1), &abort_flag))) break;
          const uint32_t bytes = cc == S::NC - 1 ? (uint32_t)(S::LASTNP / 8) * S::SBO : S::BBYTES;
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(&bfull[s])),
                       "r"(bytes)
                       : "memory");
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                  su32(sB + (size_t)s * S::BBYTES)),
              "l"(a.img + (size_t)cc * S::BBYTES), "r"(bytes), "r"(su32(&bfull[s]))
              : "memory");
        }
      }
      if (!ok) {  // aborted: let the copies in flight land before the CTA exits
        atomicExch(a.err, 1);
        for (long p = q - 1; p >= 0 && p >= q - NS; --p) drain_wait(&bfull[p % NS], (uint32_t)((p / NS) & 1));
        if (j > 0) drain_wait(&afull, (uint32_t)((j - 1) & 1));
      }
    }
  } else if (warp == 1) {
    // ---- MMA issue: each chunk against both tiles of the pair ----
    if (lane == 0) {
      const uint32_t abase = su32(sA), bbase = su32(sB);
      bool ok = true;
      long q = 0;
      for (long j = 0; j < ntl && ok; ++j) {
        long unit;
        int c0, c1;
        segment(j, unit, c0, c1);
        ok = wait_or_abort(&afull, (uint32_t)(j & 1), &abort_flag);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        for (int c = c0; c < c1; ++c, ++q) {
          const int s = (int)(q % NS), acc = (int)(q & 1);
          ok = wait_or_abort(&bfull[s], (uint32_t)((q / NS) & 1), &abort_flag) &&
               wait_or_abort(&tempty[acc], (uint32_t)(((q >> 1) & 1) ^ 1), &abort_flag);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t n = c == S::NC - 1 ? (uint32_t)S::LASTNP : (uint32_t)S::NCH;
          const uint32_t idesc = (1u << 4) | (O::kFmt << 7) | (O::kFmt << 10) | ((n >> 3) << 17) |
                                 ((uint32_t)(kTm >> 4) << 24);
          const uint32_t bo = bbase + (uint32_t)s * S::BBYTES;
#pragma unroll
          for (int tt = 0; tt < kPair; ++tt) {
            const uint32_t dt = tmem + (uint32_t)(acc * 2 * kAccCols + tt * kAccCols);
            const uint32_t ao = abase + (uint32_t)tt * S::ABYTES;
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
          }
          commit(&bempty[s]);   // the B stage is free once these MMAs are done
          commit(&tfull[acc]);  // and the accumulators are ready for the epilogue
        }
        if (!ok) break;
        commit(&aempty);  // all chunks of the pair issued: its A tiles are free when done
      }
      if (!ok) atomicExch(a.err, 1);
      // every MMA issued above has completed before the TMEM is freed
      commit(&mdone);
      drain_wait(&mdone, 0);
    }
  } else {
    // ---- epilogue: weighted sum over the subcells of each output DOF ----
    const int quarter = warp & 3;  // a warp reads the TMEM lanes of its sub-partition
    const int lrow = 32 * quarter + lane;
    const uint32_t tl = tmem + ((uint32_t)(32 * quarter) << 16);
    long q = 0;
    for (long j = 0; j < ntl; ++j) {
      long unit;
      int c0, c1;
      segment(j, unit, c0, c1);
      long ei[kPair], e[kPair];
      bool live[kPair];
      float w[kPair][M];
#pragma unroll
      for (int tt = 0; tt < kPair; ++tt) {
        ei[tt] = unit * (long)kUnit + tt * kTm + lrow;
        live[tt] = ei[tt] < a.E;
        e[tt] = !live[tt] ? 0 : (a.list != nullptr ? (long)a.list[ei[tt]] : ei[tt]);
        float sc = a.tscale;
        if constexpr (O::kScaled) sc *= live[tt] ? a.escale[ei[tt]] : 0.f;
#pragma unroll
        for (int i = 0; i < M; ++i) w[tt][i] = live[tt] ? sc * __ldg(a.w32 + e[tt] * M + i) : 0.f;
      }
      bool ok = true;
#pragma unroll 1
      for (int c = c0; c < c1; ++c, ++q) {
        const int acc = (int)(q & 1);
        ok = __all_sync(0xffffffffu, wait_or_abort(&tfull[acc], (uint32_t)((q >> 1) & 1), &abort_flag));
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int cc = c;
        const int ng = cc == S::NC - 1 ? (S::LASTN + 31) / 32 : S::NG;
#pragma unroll
        for (int tt = 0; tt < kPair; ++tt) {
          const uint32_t ta = tl + (uint32_t)(acc * 2 * kAccCols + tt * kAccCols);
          if constexpr (S::kWhole) {
#pragma unroll 1
            for (int g = 0; g < ng; ++g) {
              uint32_t qv[32];
              tmem_ld32(ta + 32 * g, qv);
              asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
              for (int o = 0; o < 32 / M; ++o) {
                float v = 0.f;
#pragma unroll
                for (int i = 0; i < M; ++i) v = fmaf(w[tt][i], __uint_as_float(qv[o * M + i]), v);
                const int r = cc * S::OPC + (32 * g) / M + o;
                if (live[tt] && r < D) a.Y[(long)Elem<D>::out(r) * a.Ey + e[tt]] = v;
              }
            }
          } else {
            // partial sums of the chunk's outputs, each over i = 0 .. M-1 in order
            float part[S::OPC];
#pragma unroll
            for (int o = 0; o < S::OPC; ++o) part[o] = 0.f;
#pragma unroll
            for (int g = 0; g < S::NG; ++g) {
              if (g < ng) {
                uint32_t qv[32];
                tmem_ld32(ta + 32 * g, qv);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int t = 0; t < 32; ++t) {
                  const int col = 32 * g + t;
                  if (col < S::OPC * M) part[col / M] = fmaf(w[tt][col % M], __uint_as_float(qv[t]), part[col / M]);
                }
              }
            }
#pragma unroll
            for (int o = 0; o < S::OPC; ++o) {
              const int r = cc * S::OPC + o;
              if (live[tt] && r < D) a.Y[(long)Elem<D>::out(r) * a.Ey + e[tt]] = part[o];
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
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// The stacked table in the shared-memory image of its chunks: chunk c, row
// n = m o + i (o < opc) is row R = c opc + o of subcell i, rows n >= m opc
// and R >= D are zero; K column k (an element DOF; the subcell matrices are
// symmetric); zero padding beyond the table.  Single modes round once (TF32 to nearest with ties away, BF16 to
// nearest even); split modes store hi in columns [0, kp) and lo in
// [kp, 2 kp), FP16 after scaling the table by tinv (a power of two).
__global__ void k_tc2_image(int mode, int D, int m, int opc, int nch, int kp, int parts, int kc, uint32_t sbo,
                            double tinv, const double* __restrict__ tab, unsigned char* __restrict__ img,
                            long total) {
  const int es = mode == kTF32 ? 4 : 2;
  const int kr = kp * parts;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const int k = (int)(t % kp);
    const long rowg = t / kp;
    const int c = (int)(rowg / nch), n = (int)(rowg % nch);
    double x = 0.0;
    const int R = c * opc + n / m, i = n % m;
    if (n < m * opc && R < D && k < D) x = tab[((long)i * D + R) * D + k];
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

// The per-DOF result of an operator gather, y the assembled A v at DOF d
// (fixed DOFs are identity rows: y = v there):
//   mode 0: out = b - y;  mode 1: out = v + omega D^-1 (b - y);  mode 2: out = y;
//   mode 3: a Chebyshev step (ChebStep).
__device__ __forceinline__ void gather_out(int mode, long d, float y, const float* __restrict__ b,
                                           const float* __restrict__ v, const float* __restrict__ dinv,
                                           const uint8_t* __restrict__ mask, float omega, float* __restrict__ out,
                                           const ChebStep& cs) {
  const float yc = mask[d] ? v[d] : y;
  if (mode == 0) {
    out[d] = b[d] - yc;
  } else if (mode == 1) {
    out[d] = v[d] + omega * dinv[d] * (b[d] - yc);
  } else if (mode == 3) {
    const float* co = static_cast<const float*>(cs.coef);
    const float c1 = cs.ci < 0 ? 0.f : co[2 * cs.ci], c2 = cs.ci < 0 ? 1.f : co[2 * cs.ci + 1];
    const float vd = v[d];
    const float dp = cs.dprev ? static_cast<const float*>(cs.dprev)[d] : vd;
    const float o = vd + c1 * dp + c2 * dinv[d] * (b[d] - yc);
    static_cast<float*>(cs.dout)[d] = o - vd;
    out[d] = o;
  } else {
    out[d] = yc;
  }
}

// y_n = sum of y_e over the elements containing node n (fixed order), then
// gather_out.  On a mixed mesh (slv != null) the vertices and the slaved
// nodes also keep their raw assembled y in yraw for k_tc2_fold, which
// finishes the vertices.
__global__ void k_tc2_gather(int Lx, int Ly, int Lz, int ex, int ey, int ez, const float* __restrict__ Y,
                             const float* __restrict__ b, const float* __restrict__ v,
                             const float* __restrict__ dinv, const uint8_t* __restrict__ mask, float omega,
                             int mode, float* __restrict__ out, ChebStep cs, const uint8_t* __restrict__ slv,
                             float* __restrict__ yraw) {
  const long nn = (long)Lx * Ly * Lz;
  const long Ey = (long)ex * ey * ez;
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
    const bool slaved = slv != nullptr && slv[node];
    const bool vertex = slv != nullptr && !((i | j | l) & 1);  // finished by k_tc2_fold
    const bool skip = !slaved && mask[3 * node] && mask[3 * node + 1] && mask[3 * node + 2];
    float y[3] = {0.f, 0.f, 0.f};
    // the (at most) 2 x 2 x 2 elements, unrolled with predicates so that all
    // their loads are in flight together; summed in the order z, y, x
#pragma unroll
    for (int kz = 0; kz < 2; ++kz)
#pragma unroll
      for (int ky = 0; ky < 2; ++ky)
#pragma unroll
        for (int kx = 0; kx < 2; ++kx) {
          const int ex_ = e0[0] + kx, ey_ = e0[1] + ky, ez_ = e0[2] + kz;
          if (skip || ex_ > e1[0] || ey_ > e1[1] || ez_ > e1[2]) continue;
          const long e = ex_ + (long)ex * (ey_ + (long)ey * ez_);
          const int la = (i - 2 * ex_) + 3 * ((j - 2 * ey_) + 3 * (l - 2 * ez_));
          const float* ye = Y + (long)(3 * la) * Ey + e;  // DOF-major: coalesced along x
          y[0] += ye[0];
          y[1] += ye[Ey];
          y[2] += ye[2 * Ey];
        }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const long d = 3 * node + c;
      if (slaved || vertex) yraw[d] = y[c];
      if (!vertex) gather_out(mode, d, y[c], b, v, dinv, mask, omega, out, cs);
    }
  }
}

// Mixed meshes: y <- T^T y at the vertices of the node lattice: each adds
// 2^-q times the raw y of every slaved neighbour (q = the neighbour's
// coordinates off the vertex: edge, face or cell midpoint), then
// gather_out.  vnb[t] holds vertex t's slaved neighbours as bits k = (dx + 1)
// + 3 (dy + 1) + 9 (dz + 1) (fixed at set-up).  Slaved nodes are fixed DOFs
// (identity rows); every other node was finished by the gather.  One thread
// per vertex.
__global__ void k_tc2_fold(int Lx, int Ly, int Lz, const uint32_t* __restrict__ vnb, const float* __restrict__ yr,
                           const float* __restrict__ b, const float* __restrict__ v,
                           const float* __restrict__ dinv, const uint8_t* __restrict__ mask, float omega, int mode,
                           float* __restrict__ out, ChebStep cs) {
  const int Vx = (Lx + 1) / 2, Vy = (Ly + 1) / 2, Vz = (Lz + 1) / 2;
  const long nv = (long)Vx * Vy * Vz;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < nv; t += (long)gridDim.x * blockDim.x) {
    const int i = 2 * (int)(t % Vx), j = 2 * (int)((t / Vx) % Vy), l = 2 * (int)(t / ((long)Vx * Vy));
    const long node = i + (long)Lx * (j + (long)Ly * l);
    float y[3] = {yr[3 * node], yr[3 * node + 1], yr[3 * node + 2]};
    const uint32_t nb = vnb[t];
#pragma unroll
    for (int k = 0; k < 27; ++k) {
      if (!((nb >> k) & 1u)) continue;
      const int dx = k % 3 - 1, dy = (k / 3) % 3 - 1, dz = k / 9 - 1;
      const int q = (dx != 0) + (dy != 0) + (dz != 0);
      const float w = q == 1 ? 0.5f : (q == 2 ? 0.25f : 0.125f);
      const long sn = node + dx + (long)Lx * (dy + (long)Ly * dz);
      y[0] += w * yr[3 * sn];
      y[1] += w * yr[3 * sn + 1];
      y[2] += w * yr[3 * sn + 2];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) gather_out(mode, 3 * node + c, y[c], b, v, dinv, mask, omega, out, cs);
  }
}

// FP32 packed upper triangles (row by row, kQ1Sym entries) of the trilinear
// elements' 24 x 24 vertex blocks, read from their slots of the level's FP64
// element matrices (packed symmetric 81 x 81 when sym, else full).
__global__ void k_q1v_compact32(long E1, const int* __restrict__ list, const double* __restrict__ K64, int sym,
                                float* __restrict__ K1) {
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < E1 * kQ1Sym; q += (long)gridDim.x * blockDim.x) {
    const long t = q / kQ1Sym;
    int rem = (int)(q % kQ1Sym), R = 0;
    while (rem >= 24 - R) {
      rem -= 24 - R;
      ++R;
    }
    const int C = R + rem;
    const int a = Elem<24>::out(R), b = Elem<24>::out(C);
    const long e = list[t];
    K1[q] = (float)(sym ? K64[e * (long)kPS2 + sym2_idx(a, b)] : K64[e * (long)kDD2 + (long)a * 81 + b]);
  }
}

// Arguments of the trilinear products (PackArgs fields), in blocks of their own.
void set_q1v(PackArgs& pa, const TcOp& tc, const Level& L0, const float* v) {
  pa.ex = L0.ex;
  pa.ey = L0.ey;
  pa.Lx = L0.Lx;
  pa.Ly = L0.Ly;
  pa.v = v;
  pa.mask = L0.mask;
  pa.E1 = L0.ne1;
  pa.list1 = L0.el1;
  pa.K1 = tc.K1v;
  pa.Y = tc.Y2;
  pa.Ey = (long)L0.ex * L0.ey * L0.ez;
}
long q1v_blocks(const TcOp& tc, long E1) {
  long g = (E1 + kQ1Warps * kQ1PerWarp - 1) / (kQ1Warps * kQ1PerWarp);
  return g > 8L * tc.sms ? 8L * tc.sms : g;
}

// tri: the row packing also launches the trilinear elements' products
// (mixed meshes, D = 81).
template <int MD, int D, int M>
cudaError_t run_apply(const TcOp& tc, const Level& L0, long count, const int* list, const uint32_t* slm,
                      const float* v, const unsigned char* img, float tscale, int stages, bool tri,
                      cudaStream_t st) {
  using S = Shape<MD, D, M>;
  static std::once_flag once;  // handles may be created from several threads
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(k_tc2_apply<MD, D, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
  });
  if (attr != cudaSuccess) return attr;
  if (count <= 0) return cudaSuccess;
  const long nunits = (count + kUnit - 1) / kUnit;
  PackArgs pa;
  set_q1v(pa, tc, L0, v);
  if (!tri) pa.E1 = 0;
  pa.E = count;
  pa.rows = nunits * kUnit;
  pa.list = list;
  pa.slm = slm;
  pa.apack = tc.apack;
  pa.escale = tc.escale;
  long gp = (pa.rows + 127) / 128;
  if (gp > 16L * tc.sms) gp = 16L * tc.sms;
  pa.pblocks = gp;
  const long gt = D == 81 && pa.E1 > 0 ? q1v_blocks(tc, pa.E1) : 0;
  if (stages & 1) k_tc2_pack<MD, D><<<(int)(gp + gt), 128, 0, st>>>(pa);
  if (!(stages & 2)) return cudaGetLastError();
  Tc2Args a;
  a.E = count;
  a.list = list;
  a.apack = tc.apack;
  a.escale = tc.escale;
  a.w32 = tc.w32;
  a.img = img;
  a.tscale = tscale;
  a.Y = tc.Y2;
  a.Ey = (long)L0.ex * L0.ey * L0.ez;
  a.err = tc.err;
  // (unit, chunk) work items split evenly over one CTA per SM; a table of few
  // chunks (n_mr = 1 or 2) keeps whole units per CTA, where a second unit's
  // A tiles would cost more than the balance gains
  const long nitems = nunits * S::NC;
  const long per = S::NC >= 12 ? nitems : nunits;
  const int g = (int)(per < tc.sms ? per : tc.sms);
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
cudaError_t apply_for(const TcOp& tc, const Level& L0, long count, const int* list, const uint32_t* slm,
                      const float* v, const unsigned char* img, float tscale, int stages, bool tri,
                      cudaStream_t st) {
  if (tc.m == 27) return run_apply<MD, D, 27>(tc, L0, count, list, slm, v, img, tscale, stages, tri, st);
  if (tc.m == 8) return run_apply<MD, D, 8>(tc, L0, count, list, slm, v, img, tscale, stages, tri, st);
  if (tc.m == 1) return run_apply<MD, D, 1>(tc, L0, count, list, slm, v, img, tscale, stages, tri, st);
  return cudaErrorInvalidValue;
}

template <int D>
cudaError_t apply_mode(const TcOp& tc, const Level& L0, long count, const int* list, const uint32_t* slm,
                       const float* v, const unsigned char* img, float tscale, int stages, bool tri,
                       cudaStream_t st) {
  switch (tc.mode) {
    case kTF32: return apply_for<kTF32, D>(tc, L0, count, list, slm, v, img, tscale, stages, tri, st);
    case kBF16: return apply_for<kBF16, D>(tc, L0, count, list, slm, v, img, tscale, stages, tri, st);
    case kBF16X3: return apply_for<kBF16X3, D>(tc, L0, count, list, slm, v, img, tscale, stages, tri, st);
    case kF16X3: return apply_for<kF16X3, D>(tc, L0, count, list, slm, v, img, tscale, stages, tri, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int MD, int D, int M>
void image_for_m(const double* tab, double tinv, unsigned char* img, cudaStream_t st) {
  using S = Shape<MD, D, M>;
  using O = Opnd<MD>;
  // one thread per (chunk row, K column of one part)
  const long total = (long)S::NC * S::NCH * S::KP;
  long g = (total + 255) / 256;
  if (g > 4096) g = 4096;
  k_tc2_image<<<(int)g, 256, 0, st>>>(MD, D, M, S::OPC, S::NCH, S::KP, O::kParts, O::kKc, S::SBO, tinv, tab, img,
                                      total);
}
template <int MD, int D>
void image_for(int m, const double* tab, double tinv, unsigned char* img, cudaStream_t st) {
  if (m == 27) image_for_m<MD, D, 27>(tab, tinv, img, st);
  else if (m == 8) image_for_m<MD, D, 8>(tab, tinv, img, st);
  else if (m == 1) image_for_m<MD, D, 1>(tab, tinv, img, st);
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

size_t tc2_image_bytes(int mode, int m) { return image_bytes_mode<81>(mode, m); }

size_t tc2_result_stride() { return 84; }  // floats per element of the result buffer (81 used)

float tc2_table_scale(int mode, const double* tab_host, size_t count) {
  if (mode != kF16X3) return 1.f;
  double mx = 0.0;
  for (size_t t = 0; t < count; ++t) mx = std::fmax(mx, std::fabs(tab_host[t]));
  if (!(mx > 0.0)) return 1.f;
  int ex2 = 0;
  std::frexp(mx, &ex2);  // mx / 2^ex2 in [0.5, 1)
  return (float)std::ldexp(1.0, ex2);
}

void launch_tc2_image(int mode, int m, const double* tab, float tscale, unsigned char* img, cudaStream_t st) {
  const double tinv = 1.0 / (double)tscale;
  switch (mode) {
    case kTF32: image_for<kTF32, 81>(m, tab, tinv, img, st); break;
    case kBF16: image_for<kBF16, 81>(m, tab, tinv, img, st); break;
    case kBF16X3: image_for<kBF16X3, 81>(m, tab, tinv, img, st); break;
    default: image_for<kF16X3, 81>(m, tab, tinv, img, st); break;
  }
}

cudaError_t launch_tc2_apply(const TcOp& tc, const Level& L0, const float* v, cudaStream_t st, int part,
                             int stages) {
  if (L0.el2 != nullptr) {  // mixed mesh: triquadratic elements with their slaved nodes, trilinear ones
    const bool tri = part != 0 && (stages & 2) && L0.ne1 > 0;
    // the whole operator: the trilinear products ride on the row packing
    const bool fused = tri && part < 0 && (stages & 1) && L0.ne2 > 0;
    if (part != 1) {
      const cudaError_t e = apply_mode<81>(tc, L0, L0.ne2, L0.el2, L0.sl2, v, tc.img, tc.tscale, stages, fused, st);
      if (e != cudaSuccess) return e;
    }
    if (tri && !fused) {
      PackArgs pa{};
      set_q1v(pa, tc, L0, v);
      k_q1v_apply32<<<(int)q1v_blocks(tc, pa.E1), 32 * kQ1Warps, 0, st>>>(pa);
    }
    return cudaGetLastError();
  }
  if (part == 1) return cudaSuccess;  // no trilinear elements
  const long E = (long)L0.ex * L0.ey * L0.ez;
  return apply_mode<81>(tc, L0, E, nullptr, nullptr, v, tc.img, tc.tscale, stages, false, st);
}

void launch_q1v_compact32(const Level& L0, const double* K64, float* K1v, cudaStream_t st) {
  if (L0.ne1 <= 0) return;
  long g = (L0.ne1 * kQ1Sym + 255) / 256;
  if (g > 8192) g = 8192;
  k_q1v_compact32<<<(int)g, 256, 0, st>>>(L0.ne1, L0.el1, K64, L0.sym ? 1 : 0, K1v);
}

size_t tc2_pack_bytes(int mode, long E) {
  const long units = (E + kUnit - 1) / kUnit;
  size_t per_tile = 0;
  switch (mode) {
    case kTF32: per_tile = Shape<kTF32, 81, 1>::ABYTES; break;
    case kBF16: per_tile = Shape<kBF16, 81, 1>::ABYTES; break;
    case kBF16X3: per_tile = Shape<kBF16X3, 81, 1>::ABYTES; break;
    default: per_tile = Shape<kF16X3, 81, 1>::ABYTES; break;
  }
  return (size_t)units * kPair * per_tile;
}

void launch_tc2_gather(const Level& L0, const float* Y, const float* b, const float* v, const float* dinv,
                       float omega, int mode, float* out, cudaStream_t st, const ChebStep* cs) {
  long g = (L0.nn + 255) / 256;
  if (g > 8192) g = 8192;
  const ChebStep c = cs ? *cs : ChebStep{};
  k_tc2_gather<<<(int)g, 256, 0, st>>>(L0.Lx, L0.Ly, L0.Lz, L0.ex, L0.ey, L0.ez, Y, b, v, dinv, L0.mask, omega,
                                       mode, out, c, L0.slv, L0.yraw);
  if (L0.slv != nullptr) {  // mixed mesh: fold the slaved nodes onto the vertices and finish them
    const long nv = (long)((L0.Lx + 1) / 2) * ((L0.Ly + 1) / 2) * ((L0.Lz + 1) / 2);
    long gv = (nv + 255) / 256;
    if (gv > 8192) gv = 8192;
    k_tc2_fold<<<(int)gv, 256, 0, st>>>(L0.Lx, L0.Ly, L0.Lz, L0.vnb, L0.yraw, b, v, dinv, L0.mask, omega, mode,
                                        out, c);
  }
}

}  // namespace tos
