// Solve kernels: the 27-point block-stencil operator apply (K u, Sec. 3.3
// Eq. matrixK_mr assembled per node), the multigrid cycle of Algorithm 1
// (damped Jacobi smoothing, linear-interpolation transfer, dense coarse
// solve), and the FP64 preconditioned CG of Sec. 7.2 with fused vector
// updates and deterministic reductions (warp shuffles, then a fixed-order
// sum of per-block partials done by the last block to finish).
#include <type_traits>

#include "internal.cuh"

namespace tos {

template <typename T>
LevelView<T> view(const Level& L);
template <>
LevelView<double> view<double>(const Level& L) {
  return LevelView<double>{L.Lx, L.Ly, L.Lz, L.nn, L.S64, L.dinv64, L.mask, L.err, L.sms, L.tl, L.tcnt};
}
template <>
LevelView<float> view<float>(const Level& L) {
  return LevelView<float>{L.Lx, L.Ly, L.Lz, L.nn, L.S32, L.dinv32, L.mask, L.err, L.sms, L.tl, L.tcnt};
}
template <>
LevelView<dfloat> view<dfloat>(const Level& L) {
  return LevelView<dfloat>{L.Lx, L.Ly, L.Lz, L.nn, L.S32, L.dinv32, L.mask, L.err, L.sms, L.tl, L.tcnt};
}

namespace {

// Stencil kernels.  The operator is streamed tile by tile (32 nodes x 243
// coefficients, one contiguous block, see internal.cuh) into a ring of
// kStages shared-memory buffers by 1D bulk copies (TMA) that complete on an
// mbarrier, so the coefficient stream -- nearly all of the kernel's DRAM
// traffic -- runs ahead of the arithmetic instead of stalling each thread on
// its own loads.  A block of 288 threads (9 warps) is persistent over its
// tiles.  The operand vector is read from global memory (L1/L2: each value
// is used by 27 neighbours and 3 rows).
constexpr int kTileThreads = 9 * kTN;  // 3 rows x 3 neighbour planes
// FP64 tiles take one more warp: the 9 (plane, row) partials would sit
// 3/2/2/2 on the SM's four sub-partitions, and FP64 issue is the scarce
// resource, so the last partial is split over two warps (sub-partitions 0
// and 1): 90/61/61/58 FP64 instructions per tile become 76/76/61/58.
template <typename T>
constexpr int tile_threads() { return std::is_same<T, double>::value ? kTileThreads + 32 : kTileThreads; }
constexpr int kStages = 3;
constexpr long kTileSpin = 1L << 22;  // bound of every mbarrier wait

template <typename T>
constexpr uint32_t tile_bytes() { return 243u * kTN * (uint32_t)sizeof(op_t<T>); }
template <typename T>
constexpr size_t tile_smem() { return (size_t)kStages * tile_bytes<T>() + kStages * sizeof(uint64_t); }
// Blocks of the tile kernels resident per SM (shared-memory bound).
template <typename T>
constexpr int tile_blocks_per_sm() { return sizeof(op_t<T>) == 4 ? 2 : 1; }

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void tile_issue(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool tile_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done = 0;
  for (long it = 0; it < kTileSpin && !done; ++it)
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
  return done != 0;
}

// Operand loads through the read-only path.  They are volatile asm so that
// the compiler issues all of a row's loads, in order, before the products
// that consume them: left to itself it schedules each load next to its use
// and the row then waits on one load at a time.
__device__ __forceinline__ float ld_nc(const float* p) {
  float v;
  asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ double ld_nc(const double* p) {
  double v;
  asm volatile("ld.global.nc.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ dfloat ld_nc(const dfloat* p) {
  float h, l;
  asm volatile("ld.global.nc.v2.f32 {%0, %1}, [%2];" : "=f"(h), "=f"(l) : "l"(p));
  return dfloat(h, l);
}

// Partial of row r of (A x) at node over the 9 neighbours in z-plane g
// (o = 9g .. 9g+8), from the tile's coefficients sb (shared memory);
// ld(nb, c) loads component c of the operand at node nb.  Neighbours outside
// the lattice are clamped onto it (their coefficients are zero), so there is
// no branch.
template <typename T>
struct Partial { using type = T; };
template <>
struct Partial<dfloat> { using type = Dot2; };
template <typename T>
using partial_t = typename Partial<T>::type;

template <typename T, typename LD>
__device__ __forceinline__ T plane_row(const LevelView<T>& V, const op_t<T>* __restrict__ sb, long node,
                                       int i, int j, int l, int r, int g, LD ld, int qlo = 0, int qhi = 9) {
  const long sx[3] = {i > 0 ? -1L : 0L, 0L, i + 1 < V.Lx ? 1L : 0L};
  const long sy[3] = {j > 0 ? -(long)V.Lx : 0L, 0L, j + 1 < V.Ly ? (long)V.Lx : 0L};
  const long zoff = g == 0 ? (l > 0 ? -(long)V.Lx * V.Ly : 0L) : g == 1 ? 0L
                                                                   : (l + 1 < V.Lz ? (long)V.Lx * V.Ly : 0L);
  // Three accumulators, each product fused into one of them: 27 FMAs per
  // partial (FP64 issue is the scarce resource on this part), with three
  // independent dependency chains per thread.
  T acc[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    if (q < qlo || q >= qhi) continue;  // warp-uniform: neighbours [qlo, qhi) only
    const long nb = node + sx[q % 3] + sy[q / 3] + zoff;
    const op_t<T>* s = sb + ((9 * g + q) * 9 + 3 * r) * kTN;
    T& a = acc[q % 3];
    a = fma(s[0], ld(nb, 0), a);
    a = fma(s[kTN], ld(nb, 1), a);
    a = fma(s[2 * kTN], ld(nb, 2), a);
  }
  return (acc[0] + acc[1]) + acc[2];
}

// The same with FP32 coefficients and float-pair operands, summed by Dot2
// (every product and addition error kept): the result carries about twice
// FP32's precision at a few FP32 operations per coefficient.
template <typename LD>
__device__ __forceinline__ Dot2 plane_row(const LevelView<dfloat>& V, const float* __restrict__ sb,
                                          long node, int i, int j, int l, int r, int g, LD ld,
                                          int qlo = 0, int qhi = 9) {
  const long sx[3] = {i > 0 ? -1L : 0L, 0L, i + 1 < V.Lx ? 1L : 0L};
  const long sy[3] = {j > 0 ? -(long)V.Lx : 0L, 0L, j + 1 < V.Ly ? (long)V.Lx : 0L};
  const long zoff = g == 0 ? (l > 0 ? -(long)V.Lx * V.Ly : 0L) : g == 1 ? 0L
                                                                   : (l + 1 < V.Lz ? (long)V.Lx * V.Ly : 0L);
  Dot2 acc[3];
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    if (q < qlo || q >= qhi) continue;
    const long nb = node + sx[q % 3] + sy[q / 3] + zoff;
    const float* s = sb + ((9 * g + q) * 9 + 3 * r) * kTN;
    acc[q % 3].add(s[0], ld(nb, 0));
    acc[q % 3].add(s[kTN], ld(nb, 1));
    acc[q % 3].add(s[2 * kTN], ld(nb, 2));
  }
  acc[0].add(acc[1]);
  acc[0].add(acc[2]);
  return acc[0];
}

template <typename P>
__device__ __forceinline__ P sum3(P a, P b, P c) { return (a + b) + c; }
__device__ __forceinline__ dfloat sum3(Dot2 a, const Dot2& b, const Dot2& c) {
  a.add(b);
  a.add(c);
  return a.value();
}

// Runs row(node, r, y) with y = (A x)_{node, r} for every node of the tiles
// this block owns (entries blockIdx.x, +gridDim.x, ... of the tile order
// V.tl).  Thread 0 keeps kStages tile copies in flight; a stage is refilled
// once every warp is done with it.  Warp w = 3g + r computes, for the tile's
// 32 nodes, the part of row r that comes from the neighbours in z-plane g;
// the three parts meet in shared memory and the g = 0 warps finish the rows.
// Tiles past the first *V.tcnt of the order hold fixed DOFs only, whose rows
// are identity rows: the g = 0 warps pass y = x without reading the tile.
// Every wait is bounded: if a copy does not land in time the block sets
// *V.err, waits (bounded) for its other copies and stops; the result is then
// invalid and the host reports the error.
template <bool kOrd, typename T, typename LD, typename ROW>
__device__ __forceinline__ void for_each_row(const LevelView<T>& V, LD ld, ROW row) {
  extern __shared__ __align__(128) unsigned char tsm[];
  using O = op_t<T>;
  using PT = partial_t<T>;
  constexpr uint32_t kBytes = tile_bytes<T>();
  constexpr bool kSplit = tile_threads<T>() > kTileThreads;
  // partials double-buffered by tile parity: the combine of tile k (warps of
  // plane 0) overlaps the other warps' start on tile k + 1
  __shared__ PT parts[2][3][kTileThreads / 3];
  __shared__ PT tail[2][kSplit ? kTN : 1];  // second half of the (g 2, row 2) partial
  O* sbuf = reinterpret_cast<O*>(tsm);
  uint64_t* bars = reinterpret_cast<uint64_t*>(tsm + (size_t)kStages * kBytes);
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const bool extra = kSplit && w == 9;  // the tenth warp: plane 2, row 2, neighbours 5..8
  const int g = extra ? 2 : w / 3, r = extra ? 2 : w % 3, rl = 32 * r + lane;
  const int qlo = extra ? 5 : 0, qhi = (kSplit && w == 8) ? 5 : 9;
  const long ntiles = ((long)V.nn + kTN - 1) / kTN;
  const long nact = kOrd ? *V.tcnt : ntiles;
  auto tile_at = [&](long q) { return kOrd ? (long)V.tl[q] : q; };
  const long nk = (long)blockIdx.x < nact ? (nact - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const char* gsrc = reinterpret_cast<const char*>(V.S);
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[s])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0)
    for (long k = 0; k < kStages && k < nk; ++k)
      tile_issue(tsm + k * kBytes, gsrc + (size_t)tile_at(blockIdx.x + k * gridDim.x) * kBytes, kBytes,
                 &bars[k]);
  long k = 0;
  for (; k < nk; ++k) {
    const int s = (int)(k % kStages);
    // every thread waits (bounded) for the tile; a timeout is agreed on at
    // the barrier below, so a warp that finished combining the previous
    // tile does not hold the others back
    const bool got = tile_wait(&bars[s], (uint32_t)((k / kStages) & 1));
    const long node = tile_at(blockIdx.x + k * gridDim.x) * kTN + lane;
    const bool live = node < V.nn;
    const int i = node % V.Lx, j = (node / V.Lx) % V.Ly, l = node / ((long)V.Lx * V.Ly);
    const int pb = (int)(k & 1);
    if (live) {
      const PT part = plane_row(V, sbuf + (size_t)s * 243 * kTN + lane, node, i, j, l, r, g, ld, qlo, qhi);
      if (extra) tail[pb][lane] = part;
      else parts[pb][g][rl] = part;
    }
    // stage s is free; the three parts are in (a timed-out tile's are never
    // combined).  Buffer pb is written again by tile k + 2, after the next
    // tile's barrier, which the combining warps reach only once they have
    // read it.
    if (__syncthreads_or(!got)) break;
    if (tid == 0 && k + kStages < nk) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tile_issue(tsm + (size_t)s * kBytes,
                 gsrc + (size_t)tile_at(blockIdx.x + (k + kStages) * gridDim.x) * kBytes, kBytes, &bars[s]);
    }
    if (g == 0 && !extra && live) {
      if constexpr (kSplit) {
        const PT p2 = r == 2 ? parts[pb][2][rl] + tail[pb][lane] : parts[pb][2][rl];
        row(node, r, sum3(parts[pb][0][rl], parts[pb][1][rl], p2));
      } else {
        row(node, r, sum3(parts[pb][0][rl], parts[pb][1][rl], parts[pb][2][rl]));
      }
    }
  }
  if (k < nk && tid == 0) {  // timed out: flag, then let the copies in flight land
    atomicExch(V.err, 1);
    for (long q = k; q < nk && q < k + kStages; ++q)
      tile_wait(&bars[q % kStages], (uint32_t)((q / kStages) & 1));
  }
  if (!kOrd || k < nk) return;
  if (g == 0 && !extra)  // tiles of fixed DOFs only: identity rows
    for (long q = nact + blockIdx.x; q < ntiles; q += gridDim.x) {
      const long node = tile_at(q) * kTN + lane;
      if (node < V.nn) row(node, r, (T)ld(node, r));
    }
}

// Threads per block of the vector kernels (one DOF or node per thread).
constexpr int kRowThreads = 192;

#define DOF_LOOP(ndof)                                                             \
  for (long d = blockIdx.x * (long)blockDim.x + threadIdx.x; d < (ndof);           \
       d += (long)gridDim.x * blockDim.x)

#define NODE_LOOP(nn)                                                              \
  for (long node = blockIdx.x * (long)blockDim.x + threadIdx.x; node < (nn);       \
       node += (long)gridDim.x * blockDim.x)

// Deterministic block sum of one double (result valid in thread 0).
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;
}

// Sum of np partials in a fixed order (L2 reads: the partials were written
// by other SMs during this launch); broadcast to the whole block.
__device__ __forceinline__ double reduce_parts(const double* part, int np) {
  __shared__ double bc;
  double v = 0.0;
  for (int t = threadIdx.x; t < np; t += blockDim.x) v += __ldcg(part + t);
  v = block_sum(v);
  if (threadIdx.x == 0) bc = v;
  __syncthreads();
  const double r = bc;
  __syncthreads();
  return r;
}

// Thread 0 of every block has written the block's partial(s); returns true
// in the single block that finishes last (threadfence + counter: no block
// ever waits on another).  That block then owns the final reduction and
// resets the counter for the next launch.
__device__ __forceinline__ bool last_block(unsigned* cnt) {
  __shared__ unsigned flag;
  if (threadIdx.x == 0) {
    __threadfence();
    flag = (atomicAdd(cnt, 1u) == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (flag) __threadfence();
  return flag != 0;
}

__device__ __forceinline__ void set_cond(cudaGraphConditionalHandle hc, int use_cond, unsigned v) {
  if (use_cond) cudaGraphSetConditional(hc, v);
}

// ---- multigrid cycle ------------------------------------------------------

template <typename T, bool kOrd>
__global__ void __launch_bounds__(tile_threads<T>(), tile_blocks_per_sm<T>()) k_vc_pre(LevelView<T> V, const T* __restrict__ b,
                                                        const T* __restrict__ v, T* __restrict__ r_out) {
  for_each_row<kOrd>(V, [&](long nb, int c) { return ld_nc(v + 3 * nb + c); }, [&](long node, int r, T y) {
    const long d = 3 * node + r;
    r_out[d] = b[d] - y;
  });
}

// Weighted sum with FP32 weights (the transfer weights are powers of 1/2,
// exact in FP32): plain for FP64 / FP32, compensated (Dot2) for float pairs.
template <typename T>
struct Acc {
  T s = T(0);
  __device__ __forceinline__ void add(float w, T x) { s += (T)w * x; }
  __device__ __forceinline__ T value() const { return s; }
};
template <>
struct Acc<dfloat> {
  Dot2 d;
  __device__ __forceinline__ void add(float w, dfloat x) { d.add(w, x); }
  __device__ __forceinline__ dfloat value() const { return d.value(); }
};

// b_H = M_H P^T r_h: each coarse node gathers the 3x3x3 fine nodes around its
// coincident fine node with weights (1, 1/2) per axis; also v_H = omega
// D_H^-1 b_H (the next level's first smoothing step) unless H is coarsest.
template <typename T>
__global__ void k_vc_restrict(int Lxf, int Lyf, int Lzf, int Lxc, int Lyc, int Lzc,
                              const uint8_t* __restrict__ maskc, const T* __restrict__ rf,
                              T* __restrict__ bc, const op_t<T>* __restrict__ dinvc, T omega,
                              T* __restrict__ vc) {
  const long nnc = (long)Lxc * Lyc * Lzc;
  NODE_LOOP(nnc) {
    const int I = node % Lxc, J = (node / Lxc) % Lyc, K = node / ((long)Lxc * Lyc);
    Acc<T> a[3];
    for (int dz = -1; dz <= 1; ++dz) {
      const int l = 2 * K + dz;
      if (l < 0 || l >= Lzf) continue;
      const float wz = dz ? 0.5f : 1.f;
      for (int dy = -1; dy <= 1; ++dy) {
        const int j = 2 * J + dy;
        if (j < 0 || j >= Lyf) continue;
        const float wyz = wz * (dy ? 0.5f : 1.f);
        for (int dx = -1; dx <= 1; ++dx) {
          const int i = 2 * I + dx;
          if (i < 0 || i >= Lxf) continue;
          const float wgt = wyz * (dx ? 0.5f : 1.f);
          const long f = i + (long)Lxf * (j + (long)Lyf * l);
          a[0].add(wgt, rf[3 * f]);
          a[1].add(wgt, rf[3 * f + 1]);
          a[2].add(wgt, rf[3 * f + 2]);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const long d = 3 * node + c;
      const T bv = maskc[d] ? T(0) : a[c].value();
      bc[d] = bv;
      if (vc != nullptr) vc[d] = omega * dinvc[d] * bv;
    }
  }
}

// v_h += M_h P z_H (trilinear interpolation between the node lattices).
template <typename T>
__global__ void k_vc_prolong(int Lxf, int Lyf, int Lzf, int Lxc, int Lyc,
                             const uint8_t* __restrict__ maskf, const T* __restrict__ zc,
                             T* __restrict__ v) {
  const long nnf = (long)Lxf * Lyf * Lzf;
  NODE_LOOP(nnf) {
    const int i = node % Lxf, j = (node / Lxf) % Lyf, l = node / ((long)Lxf * Lyf);
    const int I0 = i >> 1, I1 = (i + 1) >> 1, J0 = j >> 1, J1 = (j + 1) >> 1, K0 = l >> 1,
              K1 = (l + 1) >> 1;
    Acc<T> a0, a1, a2;
    for (int K = K0; K <= K1; ++K) {
      const float wz = (K0 == K1) ? 1.f : 0.5f;
      for (int J = J0; J <= J1; ++J) {
        const float wyz = wz * ((J0 == J1) ? 1.f : 0.5f);
        for (int I = I0; I <= I1; ++I) {
          const float wgt = wyz * ((I0 == I1) ? 1.f : 0.5f);
          const long c = I + (long)Lxc * (J + (long)Lyc * K);
          a0.add(wgt, zc[3 * c]);
          a1.add(wgt, zc[3 * c + 1]);
          a2.add(wgt, zc[3 * c + 2]);
        }
      }
    }
    if (!maskf[3 * node]) v[3 * node] += a0.value();
    if (!maskf[3 * node + 1]) v[3 * node + 1] += a1.value();
    if (!maskf[3 * node + 2]) v[3 * node + 2] += a2.value();
  }
}

// Post-smoothing: z = v + omega D^-1 (b - A v).
template <typename T, bool kOrd>
__global__ void __launch_bounds__(tile_threads<T>(), tile_blocks_per_sm<T>()) k_vc_post(LevelView<T> V, T omega, const T* __restrict__ b,
                                                         const T* __restrict__ v, T* __restrict__ z) {
  for_each_row<kOrd>(V, [&](long nb, int c) { return ld_nc(v + 3 * nb + c); }, [&](long node, int r, T y) {
    const long d = 3 * node + r;
    z[d] = v[d] + omega * V.dinv[d] * (b[d] - y);
  });
}

// The same last smoothing step at the finest level, fused with the PCG
// reduction that follows it (k_cg_dots_rz): partial r^T z and z^T q over
// the rows this block writes; the last block forms beta.
template <typename T, bool kOrd>
__global__ void __launch_bounds__(tile_threads<T>(), tile_blocks_per_sm<T>())
    k_vc_post_dots(LevelView<T> V, T omega, const T* __restrict__ b, const T* __restrict__ v,
                   T* __restrict__ z, CgDots cd) {
  double a = 0.0, c = 0.0;
  for_each_row<kOrd>(V, [&](long nb, int cc) { return ld_nc(v + 3 * nb + cc); }, [&](long node, int r, T y) {
    const long d = 3 * node + r;
    const T zt = v[d] + omega * V.dinv[d] * (b[d] - y);
    z[d] = zt;
    const double zv = (double)zt;
    a += cd.r[d] * zv;
    c += zv * cd.q[d];
  });
  a = block_sum(a);
  c = block_sum(c);
  if (threadIdx.x == 0) {
    cd.part_rz[blockIdx.x] = a;
    cd.part_zq[blockIdx.x] = c;
  }
  if (!last_block(cd.cnt)) return;
  const double rz_new = reduce_parts(cd.part_rz, gridDim.x);
  const double zq = reduce_parts(cd.part_zq, gridDim.x);
  if (threadIdx.x == 0) {
    DevState* ds = cd.ds;
    ds->beta = (ds->iter == 0) ? 0.0 : -ds->alpha * zq / ds->rz;
    ds->rz_next = rz_new;
    *cd.cnt = 0u;
  }
}

// Coarsest level: z = A_c^{-1} b in FP64, one warp per row.
template <typename T>
__global__ void k_coarse_solve(int n, const double* __restrict__ Ainv, const T* __restrict__ b,
                               T* __restrict__ z) {
  const int lane = threadIdx.x & 31;
  const long warp = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5;
  const long nw = ((long)gridDim.x * blockDim.x) >> 5;
  for (long row = warp; row < n; row += nw) {
    const double* a = Ainv + row * n;
    double s = 0.0;
    for (int c = lane; c < n; c += 32) s += a[c] * (double)b[c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) z[row] = (T)s;
  }
}

// Solve parameters from device memory (so a recorded graph keeps the
// latest rtol / maxit): params = {rtol^2, maxit}.
__global__ void k_set_params(DevState* __restrict__ ds, const double* __restrict__ params) {
  if (threadIdx.x == 0) {
    ds->tol2 = params[0];
    ds->maxit = (int)params[1];
  }
}

template <typename T>
__global__ void k_smooth0(long n, T omega, const op_t<T>* __restrict__ dinv, const T* __restrict__ b,
                          T* __restrict__ v) {
  DOF_LOOP(n) v[d] = omega * dinv[d] * b[d];
}

// ---- FP64 preconditioned CG -------------------------------------------------

__global__ void k_cg_prep(int nn, const uint8_t* __restrict__ mask, double* __restrict__ f,
                          double* __restrict__ u, double* __restrict__ part) {
  double s = 0.0;
  DOF_LOOP(3L * nn) {
    const bool fx = mask[d] != 0;
    const double fv = fx ? 0.0 : f[d];
    f[d] = fv;
    if (fx) u[d] = 0.0;
    s += fv * fv;
  }
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// r = f - K u (FP64) with partial ||r||^2.  mode 1 (before the loop): also
// b0 = (T) r, v0 = omega D0^-1 b0, and the last block runs the initial
// convergence test (||f||^2 from part_ff) and sets the loop condition;
// mode 2 (after the loop): the last block stores the true residual.
template <typename T, bool kOrd>
__global__ void __launch_bounds__(tile_threads<double>())
    k_cg_residual(LevelView<double> V, const double* __restrict__ f, const double* __restrict__ u,
                  double* __restrict__ rv, T* __restrict__ b0, const op_t<T>* __restrict__ dinv0,
                  T omega, T* __restrict__ v0, double* part, const double* part_ff, int np_ff,
                  int mode, DevState* __restrict__ ds, unsigned* cnt, cudaGraphConditionalHandle hc,
                  int use_cond) {
  double s = 0.0;
  for_each_row<kOrd>(V, [&](long nb, int c) { return ld_nc(u + 3 * nb + c); }, [&](long node, int r, double y) {
    const long d = 3 * node + r;
    const double rd = f[d] - y;
    rv[d] = rd;
    if (mode == 1) {
      const T bt = (T)rd;
      b0[d] = bt;
      if (dinv0 != nullptr) v0[d] = omega * dinv0[d] * bt;  // no smoothing level when L = 1
    }
    s += rd * rd;
  });
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
  if (!last_block(cnt)) return;
  const double rr = reduce_parts(part, gridDim.x);
  if (mode == 1) {
    const double ff = reduce_parts(part_ff, np_ff);
    if (threadIdx.x == 0) {
      ds->ff = ff;
      ds->rr = rr;
      ds->iter = 0;
      ds->status = ds->coarse_status ? (int)TOSOLVE_EBREAKDOWN : 0;
      if (!(rr == rr)) ds->status = TOSOLVE_EBREAKDOWN;
      const bool conv = (rr <= ds->tol2 * ff) || ff == 0.0;
      ds->converged = conv;
      set_cond(hc, use_cond, (conv || ds->status || ds->tile_status || ds->maxit <= 0) ? 0u : 1u);
    }
  } else if (threadIdx.x == 0) {
    ds->rr_true = rr;
  }
  if (threadIdx.x == 0) *cnt = 0u;
}

// Partial r^T z and z^T q; the last block forms the flexible (Polak-Ribiere)
// coefficient, valid for a preconditioner evaluated in lower precision:
//   beta = z_{k+1}^T (r_{k+1} - r_k) / (z_k^T r_k) = -alpha_k z_{k+1}^T q_k / rz_k.
template <typename T>
__global__ void k_cg_dots_rz(int nn, const double* __restrict__ r, const T* __restrict__ z,
                             const double* __restrict__ q, double* part_rz, double* part_zq,
                             DevState* __restrict__ ds, unsigned* cnt) {
  double a = 0.0, b = 0.0;
  DOF_LOOP(3L * nn) {
    const double zv = (double)z[d];
    a += r[d] * zv;
    b += zv * q[d];
  }
  a = block_sum(a);
  b = block_sum(b);
  if (threadIdx.x == 0) {
    part_rz[blockIdx.x] = a;
    part_zq[blockIdx.x] = b;
  }
  if (!last_block(cnt)) return;
  const double rz_new = reduce_parts(part_rz, gridDim.x);
  const double zq = reduce_parts(part_zq, gridDim.x);
  if (threadIdx.x == 0) {
    ds->beta = (ds->iter == 0) ? 0.0 : -ds->alpha * zq / ds->rz;
    ds->rz_next = rz_new;
    *cnt = 0u;
  }
}

template <typename T>
__global__ void k_cg_dir(int nn, const T* __restrict__ z, double* __restrict__ p,
                         const DevState* __restrict__ ds) {
  const bool first = ds->iter == 0;
  const double beta = ds->beta;
  DOF_LOOP(3L * nn) {
    const double zv = (double)z[d];
    p[d] = first ? zv : zv + beta * p[d];
  }
}

// q = K p (FP64) and partial p^T q; the last block forms alpha = rz / p^T q
// (a non-positive or non-finite value is a breakdown).
template <bool kOrd>
__global__ void __launch_bounds__(tile_threads<double>())
    k_cg_apply(LevelView<double> V, const double* __restrict__ p, double* __restrict__ q, double* part,
               DevState* __restrict__ ds, unsigned* cnt) {
  double s = 0.0;
  for_each_row<kOrd>(V, [&](long nb, int c) { return ld_nc(p + 3 * nb + c); }, [&](long node, int r, double y) {
    const long d = 3 * node + r;
    q[d] = y;
    s += p[d] * y;
  });
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
  if (!last_block(cnt)) return;
  const double pq = reduce_parts(part, gridDim.x);
  if (threadIdx.x == 0) {
    const double rz = ds->rz_next;
    const double alpha = rz / pq;
    const bool ok = (pq > 0.0) && (alpha == alpha) && (fabs(alpha) < 1e300);
    ds->alpha = ok ? alpha : 0.0;
    ds->rz = rz;
    if (!ok) ds->status = TOSOLVE_EBREAKDOWN;
    *cnt = 0u;
  }
}

// The same two CG steps when the operator was applied by another kernel
// (element-form levels): y holds K u (residual) or K p (= q, apply).
template <typename T>
__global__ void k_cg_residual_y(int nn, const double* __restrict__ f, double* __restrict__ yr,
                                T* __restrict__ b0, const op_t<T>* __restrict__ dinv0, T omega,
                                T* __restrict__ v0, double* part, const double* part_ff, int np_ff,
                                int mode, DevState* __restrict__ ds, unsigned* cnt,
                                cudaGraphConditionalHandle hc, int use_cond) {
  double s = 0.0;
  DOF_LOOP(3L * nn) {
    const double rd = f[d] - yr[d];
    yr[d] = rd;
    if (mode == 1) {
      const T bt = (T)rd;
      b0[d] = bt;
      if (dinv0 != nullptr) v0[d] = omega * dinv0[d] * bt;
    }
    s += rd * rd;
  }
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
  if (!last_block(cnt)) return;
  const double rr = reduce_parts(part, gridDim.x);
  if (mode == 1) {
    const double ff = reduce_parts(part_ff, np_ff);
    if (threadIdx.x == 0) {
      ds->ff = ff;
      ds->rr = rr;
      ds->iter = 0;
      ds->status = ds->coarse_status ? (int)TOSOLVE_EBREAKDOWN : 0;
      if (!(rr == rr)) ds->status = TOSOLVE_EBREAKDOWN;
      const bool conv = (rr <= ds->tol2 * ff) || ff == 0.0;
      ds->converged = conv;
      set_cond(hc, use_cond, (conv || ds->status || ds->tile_status || ds->maxit <= 0) ? 0u : 1u);
    }
  } else if (threadIdx.x == 0) {
    ds->rr_true = rr;
  }
  if (threadIdx.x == 0) *cnt = 0u;
}

__global__ void k_cg_apply_y(int nn, const double* __restrict__ p, const double* __restrict__ q,
                             double* part, DevState* __restrict__ ds, unsigned* cnt) {
  double s = 0.0;
  DOF_LOOP(3L * nn) s += p[d] * q[d];
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
  if (!last_block(cnt)) return;
  const double pq = reduce_parts(part, gridDim.x);
  if (threadIdx.x == 0) {
    const double rz = ds->rz_next;
    const double alpha = rz / pq;
    const bool ok = (pq > 0.0) && (alpha == alpha) && (fabs(alpha) < 1e300);
    ds->alpha = ok ? alpha : 0.0;
    ds->rz = rz;
    if (!ok) ds->status = TOSOLVE_EBREAKDOWN;
    *cnt = 0u;
  }
}

// u += alpha p, r -= alpha q, b0 = (T) r, v0 = omega D0^-1 b0, partial
// ||r||^2; the last block runs the convergence test and sets the loop
// condition (stop on convergence, breakdown or maxit).
template <typename T>
__global__ void k_cg_update(int nn, double* __restrict__ u, double* __restrict__ r,
                            const double* __restrict__ p, const double* __restrict__ q,
                            T* __restrict__ b0, const op_t<T>* __restrict__ dinv0, T omega,
                            T* __restrict__ v0, double* part_rr, DevState* __restrict__ ds,
                            unsigned* cnt, cudaGraphConditionalHandle hc, int use_cond) {
  const double alpha = ds->alpha;
  double s = 0.0;
  DOF_LOOP(3L * nn) {
    u[d] += alpha * p[d];
    const double rv = r[d] - alpha * q[d];
    r[d] = rv;
    const T bt = (T)rv;
    b0[d] = bt;
    if (dinv0 != nullptr) v0[d] = omega * dinv0[d] * bt;  // no smoothing level when L = 1
    s += rv * rv;
  }
  s = block_sum(s);
  if (threadIdx.x == 0) part_rr[blockIdx.x] = s;
  if (!last_block(cnt)) return;
  const double rr = reduce_parts(part_rr, gridDim.x);
  if (threadIdx.x == 0) {
    ds->rr = rr;
    ds->iter += 1;
    if (!(rr == rr)) ds->status = TOSOLVE_EBREAKDOWN;
    const bool conv = rr <= ds->tol2 * ds->ff;
    ds->converged = conv;
    set_cond(hc, use_cond, (conv || ds->status || ds->tile_status || ds->iter >= ds->maxit) ? 0u : 1u);
    *cnt = 0u;
  }
}

// ---- inner FP32 PCG ----------------------------------------------------------
// Each outer (FP64) iteration may precondition with a few iterations of PCG
// in FP32 on the level-0 operator of the preconditioner, each of those
// preconditioned by one V-cycle: a stronger preconditioner for the outer
// flexible CG, whose FP64 operator apply then runs far fewer times.  The
// inner coefficients use the same flexible form as the outer loop.

// The vector kernels of the inner iteration stride over the DOFs four at a
// time, loading all four before any store, so that each thread has four
// independent loads in flight (the reductions' grids are capped at kMaxPart
// blocks, about fourteen DOFs per thread on a 1.6 M DOF level); a thread
// visits its DOFs in the same order as a plain grid-stride loop.
constexpr int kU = 4;
#define DOF_LOOP_U(ndof)                                                               \
  for (long d0 = blockIdx.x * (long)blockDim.x + threadIdx.x, sd = (long)gridDim.x * blockDim.x; \
       d0 < (ndof); d0 += kU * sd)

// ri = b0 (the outer residual in FP32); e = 0.
__global__ void k_in_init(long n, const float* __restrict__ b0, float* __restrict__ ri, float* __restrict__ e) {
  DOF_LOOP(n) {
    ri[d] = b0[d];
    e[d] = 0.f;
  }
}

// rho = ri^T z and zq = z^T qi (qi = A p of the previous inner iteration);
// the last block forms beta = -alpha zq / rho_old (0 on the first).
__global__ void k_in_rz(long n, const float* __restrict__ ri, const float* __restrict__ z,
                        const float* __restrict__ qi, int first, double* part_a, double* part_b,
                        DevState* __restrict__ ds, unsigned* cnt) {
  // each thread's few dozen terms in FP32 (FP64 issue is scarce here), the
  // block and grid sums in FP64; the inner CG runs in FP32 throughout
  float fa = 0.f, fb = 0.f;
  DOF_LOOP_U(n) {
    float zv[kU], rv[kU], qv[kU];
#pragma unroll
    for (int q = 0; q < kU; ++q) {
      const long d = d0 + q * sd;
      zv[q] = d < n ? z[d] : 0.f;
      rv[q] = d < n ? ri[d] : 0.f;
      qv[q] = d < n && !first ? qi[d] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < kU; ++q) {
      if (d0 + q * sd >= n) break;
      fa = fmaf(rv[q], zv[q], fa);
      if (!first) fb = fmaf(zv[q], qv[q], fb);
    }
  }
  double a = block_sum((double)fa);
  double b = block_sum((double)fb);
  if (threadIdx.x == 0) {
    part_a[blockIdx.x] = a;
    part_b[blockIdx.x] = b;
  }
  if (!last_block(cnt)) return;
  const double rz = reduce_parts(part_a, gridDim.x);
  const double zq = reduce_parts(part_b, gridDim.x);
  if (threadIdx.x == 0) {
    const double beta = first ? 0.0 : -ds->in_alpha * zq / ds->in_rho;
    ds->in_beta = (beta == beta && fabs(beta) < 1e30) ? beta : 0.0;
    ds->in_rho_next = rz;
    *cnt = 0u;
  }
}

__global__ void k_in_dir(long n, const float* __restrict__ z, float* __restrict__ pi, int first,
                         const DevState* __restrict__ ds) {
  const float beta = (float)ds->in_beta;
  DOF_LOOP_U(n) {
    float zv[kU], pv[kU];
#pragma unroll
    for (int q = 0; q < kU; ++q) {
      const long d = d0 + q * sd;
      zv[q] = d < n ? z[d] : 0.f;
      pv[q] = d < n && !first ? pi[d] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < kU; ++q) {
      const long d = d0 + q * sd;
      if (d < n) pi[d] = first ? zv[q] : zv[q] + beta * pv[q];
    }
  }
}

// sigma = pi^T qi; the last block forms alpha = rho / sigma.  A
// non-positive or non-finite sigma (rounding on a nearly converged inner
// system) keeps the inner solution: alpha = 0, except on the first inner
// iteration, where alpha = 1 leaves the V-cycle's output as the result.
__global__ void k_in_pq(long n, const float* __restrict__ pi, const float* __restrict__ qi, int first,
                        double* part, DevState* __restrict__ ds, unsigned* cnt) {
  float fs = 0.f;
  DOF_LOOP_U(n) {
    float pv[kU], qv[kU];
#pragma unroll
    for (int q = 0; q < kU; ++q) {
      const long d = d0 + q * sd;
      pv[q] = d < n ? pi[d] : 0.f;
      qv[q] = d < n ? qi[d] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < kU; ++q) {
      if (d0 + q * sd >= n) break;
      fs = fmaf(pv[q], qv[q], fs);
    }
  }
  const double s = block_sum((double)fs);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
  if (!last_block(cnt)) return;
  const double sig = reduce_parts(part, gridDim.x);
  if (threadIdx.x == 0) {
    const double rz = ds->in_rho_next;
    const double alpha = rz / sig;
    const bool ok = sig > 0.0 && alpha == alpha && fabs(alpha) < 1e30;
    ds->in_alpha = ok ? alpha : (first ? 1.0 : 0.0);
    ds->in_rho = rz;
    *cnt = 0u;
  }
}

// e += alpha pi; unless last: ri -= alpha qi, b0 = ri, v0 = omega D^-1 ri
// (the next V-cycle's input and its first smoothing step); last: z0 = e.
__global__ void k_in_update(long n, float* __restrict__ e, float* __restrict__ ri, const float* __restrict__ pi,
                            const float* __restrict__ qi, float* __restrict__ b0, const float* __restrict__ dinv0,
                            float omega, float* __restrict__ v0, float* __restrict__ z0, int last,
                            const DevState* __restrict__ ds) {
  const float a = (float)ds->in_alpha;
  DOF_LOOP_U(n) {
    float ev[kU], pv[kU], rv[kU], qv[kU], dv[kU];
#pragma unroll
    for (int q = 0; q < kU; ++q) {
      const long d = d0 + q * sd;
      const bool in = d < n;
      ev[q] = in ? e[d] : 0.f;
      pv[q] = in ? pi[d] : 0.f;
      rv[q] = in && !last ? ri[d] : 0.f;
      qv[q] = in && !last ? qi[d] : 0.f;
      dv[q] = in && !last ? dinv0[d] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < kU; ++q) {
      const long d = d0 + q * sd;
      if (d >= n) break;
      const float evn = ev[q] + a * pv[q];
      if (last) {
        z0[d] = evn;
      } else {
        e[d] = evn;
        const float r = rv[q] - a * qv[q];
        ri[d] = r;
        b0[d] = r;
        v0[d] = omega * dv[q] * r;
      }
    }
  }
}

// Diagnostic: y = A x in the level's stored precision, FP64 in and out.
template <typename T, bool kOrd>
__global__ void __launch_bounds__(tile_threads<T>(), tile_blocks_per_sm<T>()) k_apply_diag(LevelView<T> V, const double* __restrict__ x,
                                                            double* __restrict__ y) {
  for_each_row<kOrd>(V, [&](long nb, int c) { return (T)ld_nc(x + 3 * nb + c); },
               [&](long node, int r, T v) { y[3 * node + r] = (double)v; });
}

template <typename A, typename B>
__global__ void k_cast(size_t n, const A* __restrict__ a, B* __restrict__ b) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    b[t] = (B)a[t];
}

inline int grid_nodes(long nn) { return parts_for(nn); }

// Grid of a tile kernel over level L: persistent blocks, at most as many as
// are resident at once (and at most kMaxPart, the partial-sum capacity).
// Launches the stencil kernel variant that follows the level's tile order
// (kOrd = true, only while a suppression leaves tiles of fixed DOFs) or the
// plain index order.
#define TILE_ORD(V, ...)                  \
  do {                                    \
    if ((V).tl != nullptr) {              \
      constexpr bool kOrd = true;         \
      __VA_ARGS__;                        \
    } else {                              \
      constexpr bool kOrd = false;        \
      __VA_ARGS__;                        \
    }                                     \
  } while (0)

template <typename T>
int tile_grid(const Level& L) {
  const long nt = ((long)L.nn + kTN - 1) / kTN;
  long g = (long)tile_blocks_per_sm<T>() * L.sms;
  if (g > nt) g = nt;
  if (g > kMaxPart) g = kMaxPart;
  return g < 1 ? 1 : (int)g;
}

template <typename T>
const op_t<T>* dinv_of(const Level& L);
template <>
const double* dinv_of<double>(const Level& L) { return L.dinv64; }
template <>
const float* dinv_of<float>(const Level& L) { return L.dinv32; }
template <>
const float* dinv_of<dfloat>(const Level& L) { return L.dinv32; }

template <typename T>
constexpr int vt_code() {
  return std::is_same<T, double>::value ? kVtF64 : (std::is_same<T, float>::value ? kVtF32 : kVtDF);
}
template <typename T>
const void* elem_op(const Level& L) {
  return std::is_same<T, double>::value ? (const void*)L.K64 : (const void*)L.K32;
}

// ---- Chebyshev smoothing: lambda_max(D^-1 A) by Lanczos at set-up --------
// Lanczos on the symmetric D^-1/2 A D^-1/2, written in the unscaled vectors
// p = D^-1/2 q (alpha_j = p_j^T A p_j, s = D^-1 A p_j - alpha_j p_j - beta_j
// p_{j-1}, beta_{j+1} = (s^T D s)^1/2, p_{j+1} = s / beta_{j+1}), from the
// Weyl vector frac(d phi) - 1/2 (0 at fixed DOFs) normalised in the D-norm.
// The operator is the level's own smoothing operator in its vector type.
// Every reduction is FP64 in a fixed order.  State in lz: alpha_j at j,
// beta_j at kLzMax + j, then the D-norm, the estimate and theta.
constexpr int kLzMax = 16;
constexpr int kLzNrm = 2 * kLzMax, kLzLmax = kLzNrm + 1, kLzTheta = kLzNrm + 2;
constexpr double kGolden = 0.6180339887498949;

template <typename T>
__global__ void k_lz_start(long n, const uint8_t* __restrict__ mask, const T* __restrict__ dinv, T* __restrict__ p,
                           double* __restrict__ part, unsigned* cnt, double* __restrict__ lz) {
  double s = 0.0;
  DOF_LOOP(n) {
    double x = (double)d * kGolden;
    x = mask[d] ? 0.0 : x - floor(x) - 0.5;
    const T xt = (T)x;
    p[d] = xt;
    s += (double)xt * (double)xt / (double)dinv[d];
  }
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
  if (!last_block(cnt)) return;
  const double tot = reduce_parts(part, gridDim.x);
  if (threadIdx.x == 0) {
    lz[kLzNrm] = sqrt(tot);
    *cnt = 0u;
  }
}

template <typename T>
__global__ void k_lz_scale(long n, T* __restrict__ p, const double* __restrict__ lz) {
  const T inv = (T)(1.0 / lz[kLzNrm]);
  DOF_LOOP(n) p[d] *= inv;
}

// alpha_j = p^T y (y = A p)
template <typename T>
__global__ void k_lz_alpha(long n, const T* __restrict__ p, const T* __restrict__ y, double* __restrict__ part,
                           unsigned* cnt, double* __restrict__ lz, int j) {
  double s = 0.0;
  DOF_LOOP(n) s += (double)p[d] * (double)y[d];
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
  if (!last_block(cnt)) return;
  const double tot = reduce_parts(part, gridDim.x);
  if (threadIdx.x == 0) {
    lz[j] = tot;
    *cnt = 0u;
  }
}

// q <- s = D^-1 y - alpha_j p - beta_j q (q holds p_{j-1}), beta_{j+1}
template <typename T>
__global__ void k_lz_next(long n, const T* __restrict__ p, const T* __restrict__ y, T* __restrict__ q,
                          const T* __restrict__ dinv, double* __restrict__ part, unsigned* cnt,
                          double* __restrict__ lz, int j) {
  const T alpha = (T)lz[j], beta = j == 0 ? T(0) : (T)lz[kLzMax + j];
  double s = 0.0;
  DOF_LOOP(n) {
    const T sv = dinv[d] * y[d] - alpha * p[d] - beta * q[d];
    q[d] = sv;
    s += (double)sv * (double)sv / (double)dinv[d];
  }
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
  if (!last_block(cnt)) return;
  const double tot = reduce_parts(part, gridDim.x);
  if (threadIdx.x == 0) {
    lz[kLzMax + j + 1] = sqrt(tot);
    *cnt = 0u;
  }
}

// p_{j+1} = s / beta_{j+1}, and q takes p_j
template <typename T>
__global__ void k_lz_swap(long n, T* __restrict__ p, T* __restrict__ q, const double* __restrict__ lz, int j) {
  const T inv = (T)(1.0 / lz[kLzMax + j + 1]);
  DOF_LOOP(n) {
    const T t = p[d];
    p[d] = q[d] * inv;
    q[d] = t;
  }
}

// Number of eigenvalues below x of the symmetric tridiagonal matrix with
// diagonal a[0..k) and off-diagonal b[1..k) (Sturm sequence of the LDL^T
// pivots).
__device__ int sturm_below(const double* a, const double* b, int k, double x) {
  int c = 0;
  double q = a[0] - x;
  for (int i = 0;; ++i) {
    if (q == 0.0) q = -1e-300;
    c += q < 0.0;
    if (i + 1 == k) break;
    q = a[i + 1] - x - b[i + 1] * b[i + 1] / q;
  }
  return c;
}

// The largest Ritz value by bisection on the Sturm count, then the
// Chebyshev interval [0.3 hi, hi], hi = 1.1 lambda, and the coefficients of
// steps 2..k (Saad, Algorithm 12.1 on D^-1 A): c1 = rho_i rho_{i-1} and
// c2 = 2 rho_i / delta, stored as (c1, c2 theta) because the level's D^-1 is
// divided by theta afterwards (the first step is then D^-1 r with weight 1).
__global__ void k_lz_finish(int steps, int degree, double* __restrict__ lz, double* __restrict__ c64,
                            float* __restrict__ c32) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double* a = lz;
  const double* b = lz + kLzMax;  // b[i] couples i - 1 and i
  double lo = a[0], hi = a[0];
  for (int i = 0; i < steps; ++i) {
    const double r = (i > 0 ? fabs(b[i]) : 0.0) + (i + 1 < steps ? fabs(b[i + 1]) : 0.0);
    lo = fmin(lo, a[i] - r);
    hi = fmax(hi, a[i] + r);
  }
  for (int it = 0; it < 200 && hi - lo > 1e-15 * fmax(fabs(hi), 1.0); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (sturm_below(a, b, steps, mid) <= steps - 1) lo = mid;
    else hi = mid;
  }
  const double lam = 0.5 * (lo + hi);
  const double top = 1.1 * lam, bot = 0.3 * top;
  const double theta = 0.5 * (top + bot), delta = 0.5 * (top - bot), sigma = theta / delta;
  double rho = 1.0 / sigma;
  for (int i = 1; i < degree; ++i) {
    const double rn = 1.0 / (2.0 * sigma - rho);
    c64[2 * (i - 1)] = rn * rho;
    c64[2 * (i - 1) + 1] = 2.0 * rn / delta * theta;
    c32[2 * (i - 1)] = (float)(rn * rho);
    c32[2 * (i - 1) + 1] = (float)(2.0 * rn / delta * theta);
    rho = rn;
  }
  lz[kLzLmax] = lam;
  lz[kLzTheta] = theta;
}

template <typename T>
__global__ void k_lz_scale_dinv(long n, T* __restrict__ dinv, const double* __restrict__ lz) {
  const T inv = (T)(1.0 / lz[kLzTheta]);
  DOF_LOOP(n) dinv[d] *= inv;
}

// One V-cycle from level l down (Algorithm 1).  With dots (finest level
// only) the last smoothing step also forms the PCG reduction when it is a
// stencil kernel; returns whether it did.
template <typename T>
bool vcycle_rec(Level* lv, int l, int L, T omega, const double* Ainv, const TcOp& tc,
                cudaStream_t st, const CgDots* dots) {
  Level& F = lv[l];
  if (l == L - 1) {
    const int n = F.ndof;
    int g = (n * 32 + kBS - 1) / kBS;
    if (g > 1024) g = 1024;
    k_coarse_solve<T><<<g, kBS, 0, st>>>(n, Ainv, (const T*)F.b, (T*)F.z);
    return false;
  }
  Level& C = lv[l + 1];
  const LevelView<T> V = view<T>(F);
  const bool c_coarsest = (l + 1 == L - 1);
  const bool use_tc = tc.on && l == 0;
  // element-form levels: out = f(A v) in gather mode `mode` (the degree-2
  // stacked contraction on tensor cores at level 0 when it is on)
  auto elem_op_step = [&](int mode, void* out, const ChebStep* cs) {
    if constexpr (std::is_same<T, float>::value) {
      if (use_tc && tc.deg >= 2) {
        launch_tc2_apply(tc, F, (const float*)F.v, st);
        launch_tc2_gather(F, tc.Y2, (const float*)F.b, (const float*)F.v, F.dinv32, (float)omega, mode,
                          (float*)out, st, cs);
        return;
      }
    }
    launch_q2_op(vt_code<T>(), F, elem_op<T>(F), F.Y, F.b, F.v, dinv_of<T>(F), (double)omega, mode, out, F.sms,
                 st, cs);
  };
  const bool elem_form = F.k >= 2 && (!use_tc || tc.deg >= 2);
  const void* coef = std::is_same<T, double>::value ? (const void*)F.cheb64 : (const void*)F.cheb32;
  if (elem_form && F.cheb > 0) {
    // Chebyshev: v holds the first step from 0 (D^-1 b / theta, formed with
    // the coarse right-hand side); steps 2..k, then the residual
    for (int i = 2; i <= F.cheb; ++i) {
      ChebStep cs;
      cs.dprev = i == 2 ? nullptr : F.d;
      cs.dout = F.d;
      cs.coef = coef;
      cs.ci = i - 2;
      elem_op_step(3, F.v, &cs);
    }
    elem_op_step(0, F.r, nullptr);
  } else if constexpr (std::is_same<T, float>::value) {
    if (use_tc && tc.deg >= 2) {  // r = b - A v, A v from the degree-2 stacked contraction
      elem_op_step(0, F.r, nullptr);
    } else if (use_tc) {  // r = b - A v with A v from the tensor-core stacked contraction
      launch_tc_apply(F, tc.m, (const float*)F.v, tc.w32, tc.KT, tc.Ye, tc.err, tc.sms, st);
      launch_tc_gather(F, tc.Ye, (const float*)F.b, (const float*)F.v, F.dinv32, (float)omega, 0,
                       (float*)F.r, st);
    }
  }
  if (elem_form && F.cheb > 0) {
    // residual formed above
  } else if (F.k >= 2 && !use_tc)
    launch_q2_op(vt_code<T>(), F, elem_op<T>(F), F.Y, F.b, F.v, dinv_of<T>(F), (double)omega, 0, F.r,
                 F.sms, st);
  else if (!use_tc)
    TILE_ORD(V, (k_vc_pre<T, kOrd><<<tile_grid<T>(F), tile_threads<T>(), tile_smem<T>(), st>>>(
                    V, (const T*)F.b, (const T*)F.v, (T*)F.r)));
  if (C.ptab != nullptr)  // the coarse shape functions and their transpose
    launch_s2_restrict(vt_code<T>(), F, C, C.ptab, c_coarsest ? nullptr : dinv_of<T>(C), (double)omega,
                       c_coarsest ? nullptr : C.v, st);
  else
    k_vc_restrict<T><<<grid_nodes(C.nn), kRowThreads, 0, st>>>(
        F.Lx, F.Ly, F.Lz, C.Lx, C.Ly, C.Lz, C.mask, (const T*)F.r, (T*)C.b,
        c_coarsest ? nullptr : dinv_of<T>(C), omega, c_coarsest ? nullptr : (T*)C.v);
  vcycle_rec<T>(lv, l + 1, L, omega, Ainv, tc, st, nullptr);
  if (C.ptab != nullptr)
    launch_s2_prolong(vt_code<T>(), F, C, C.ptab, st);
  else
    k_vc_prolong<T><<<grid_nodes(F.nn), kRowThreads, 0, st>>>(F.Lx, F.Ly, F.Lz, C.Lx, C.Ly, F.mask,
                                                              (const T*)C.z, (T*)F.v);
  if (elem_form && F.cheb > 0) {  // Chebyshev post-smoothing: k steps from the corrected v, the last into z
    for (int i = 1; i <= F.cheb; ++i) {
      ChebStep cs;
      cs.dprev = i == 1 ? nullptr : F.d;
      cs.dout = F.d;
      cs.coef = coef;
      cs.ci = i == 1 ? -1 : i - 2;
      elem_op_step(3, i == F.cheb ? F.z : F.v, &cs);
    }
    return false;
  }
  if constexpr (std::is_same<T, float>::value) {
    if (use_tc && tc.deg >= 2) {  // z = v + omega D^-1 (b - A v)
      elem_op_step(1, F.z, nullptr);
      return false;
    }
    if (use_tc) {  // z = v + omega D^-1 (b - A v)
      launch_tc_apply(F, tc.m, (const float*)F.v, tc.w32, tc.KT, tc.Ye, tc.err, tc.sms, st);
      launch_tc_gather(F, tc.Ye, (const float*)F.b, (const float*)F.v, F.dinv32, (float)omega, 1,
                       (float*)F.z, st);
      return false;
    }
  }
  if (F.k >= 2) {
    launch_q2_op(vt_code<T>(), F, elem_op<T>(F), F.Y, F.b, F.v, dinv_of<T>(F), (double)omega, 1, F.z,
                 F.sms, st);
    return false;
  }
  if (dots != nullptr) {
    TILE_ORD(V, (k_vc_post_dots<T, kOrd><<<tile_grid<T>(F), tile_threads<T>(), tile_smem<T>(), st>>>(
                    V, omega, (const T*)F.b, (const T*)F.v, (T*)F.z, *dots)));
    return true;
  }
  TILE_ORD(V, (k_vc_post<T, kOrd><<<tile_grid<T>(F), tile_threads<T>(), tile_smem<T>(), st>>>(
                  V, omega, (const T*)F.b, (const T*)F.v, (T*)F.z)));
  return false;
}

}  // namespace

// Runs BODY with T bound to the vector type of vt.
#define VT_DISPATCH(vt, BODY)                 \
  do {                                        \
    if ((vt) == kVtF64) {                     \
      using T = double;                       \
      BODY;                                   \
    } else if ((vt) == kVtF32) {              \
      using T = float;                        \
      BODY;                                   \
    } else {                                  \
      using T = dfloat;                       \
      BODY;                                   \
    }                                         \
  } while (0)

bool launch_vcycle(int vt, Level* lv, int L, double omega, int gamma, const double* Ainv,
                   const TcOp& tc, cudaStream_t st, const CgDots* dots) {
  (void)gamma;
  bool fused = false;
  VT_DISPATCH(vt, fused = vcycle_rec<T>(lv, 0, L, (T)omega, Ainv, tc, st, dots));
  return fused;
}

void launch_inner_pcg(Level* lv, int L, double omega, const double* Ainv, const TcOp& tc, const InnerPcg& in,
                      double* part_a, double* part_b, DevState* ds, unsigned* cnt, cudaStream_t st) {
  Level& L0 = lv[0];
  const long n = L0.ndof;
  const int g = parts_for(L0.nn);  // blocks of the reductions (<= kMaxPart partials)
  const int gv = (int)((n + kU * kRowThreads - 1) / (kU * kRowThreads));  // the others: one pass
  float* b0 = (float*)L0.b;
  float* v0 = (float*)L0.v;
  float* z0 = (float*)L0.z;
  k_in_init<<<g, kRowThreads, 0, st>>>(n, b0, in.ri, in.e);
  for (int it = 0; it < in.its; ++it) {
    const int first = it == 0, last = it == in.its - 1;
    vcycle_rec<float>(lv, 0, L, (float)omega, Ainv, tc, st, nullptr);  // z0 = M^-1 b0
    k_in_rz<<<g, kRowThreads, 0, st>>>(n, in.ri, z0, in.qi, first, part_a, part_b, ds, cnt);
    k_in_dir<<<gv, kRowThreads, 0, st>>>(n, z0, in.pi, first, ds);
    if (tc.on && tc.deg >= 2) {  // qi = A pi on the tensor cores
      launch_tc2_apply(tc, L0, in.pi, st);
      launch_tc2_gather(L0, tc.Y2, in.pi, in.pi, L0.dinv32, 0.f, 2, in.qi, st);
    } else {  // the FP32 element matrices
      launch_q2_op(kVtF32, L0, L0.K32, L0.Y, nullptr, in.pi, nullptr, 0.0, 2, in.qi, L0.sms, st);
    }
    k_in_pq<<<g, kRowThreads, 0, st>>>(n, in.pi, in.qi, first, part_a, ds, cnt);
    k_in_update<<<gv, kRowThreads, 0, st>>>(n, in.e, in.ri, in.pi, in.qi, b0, L0.dinv32, (float)omega, v0, z0,
                                            last, ds);
  }
}

void launch_set_params(DevState* ds, const double* params, cudaStream_t st) {
  k_set_params<<<1, 32, 0, st>>>(ds, params);
}

void launch_cheb_setup(int vt, Level* lv, int L, const TcOp& tc, int steps, double* part, unsigned* cnt,
                       double* lz, double* lmax_out, cudaStream_t st) {
  for (int l = 0; l + 1 < L; ++l) {
    Level& F = lv[l];
    if (F.cheb <= 0) continue;
    auto run = [&](auto tag) {
      using T = decltype(tag);
      const long n = F.ndof;
      int g = (int)((n + kRowThreads - 1) / kRowThreads);
      if (g > kMaxPart) g = kMaxPart;
      T* P = (T*)F.v;
      T* Q = (T*)F.d;
      T* Y = (T*)F.r;
      T* dinv = const_cast<T*>(dinv_of<T>(F));
      const bool use_tc = tc.on && l == 0 && tc.deg >= 2;
      k_lz_start<T><<<g, kRowThreads, 0, st>>>(n, F.mask, dinv, P, part, cnt, lz);
      k_lz_scale<T><<<g, kRowThreads, 0, st>>>(n, P, lz);
      cudaMemsetAsync(Q, 0, (size_t)n * sizeof(T), st);
      for (int j = 0; j < steps; ++j) {
        if constexpr (std::is_same<T, float>::value) {
          if (use_tc) {
            launch_tc2_apply(tc, F, P, st);
            launch_tc2_gather(F, tc.Y2, nullptr, P, F.dinv32, 0.f, 2, Y, st);
          }
        }
        if (!use_tc)
          launch_q2_op(vt_code<T>(), F, elem_op<T>(F), F.Y, nullptr, P, dinv, 0.0, 2, Y, F.sms, st);
        k_lz_alpha<T><<<g, kRowThreads, 0, st>>>(n, P, Y, part, cnt, lz, j);
        if (j + 1 < steps) {
          k_lz_next<T><<<g, kRowThreads, 0, st>>>(n, P, Y, Q, dinv, part, cnt, lz, j);
          k_lz_swap<T><<<g, kRowThreads, 0, st>>>(n, P, Q, lz, j);
        }
      }
      k_lz_finish<<<1, 32, 0, st>>>(steps, F.cheb, lz, F.cheb64, F.cheb32);
      if (lmax_out != nullptr) cudaMemcpyAsync(lmax_out + l, lz + kLzLmax, sizeof(double), cudaMemcpyDeviceToDevice, st);
      k_lz_scale_dinv<T><<<g, kRowThreads, 0, st>>>(n, dinv, lz);
    };
    if (vt == kVtF64) run(double());
    else run(float());
  }
}

void launch_smooth0(int vt, const Level& L0, double omega, cudaStream_t st) {
  const int g = parts_for(L0.nn);
  VT_DISPATCH(vt, (k_smooth0<T><<<g, kRowThreads, 0, st>>>(L0.ndof, (T)omega, dinv_of<T>(L0),
                                                           (const T*)L0.b, (T*)L0.v)));
}

void launch_cg_prep(const Level& L0, double* f, double* u, double* part, int np, cudaStream_t st) {
  k_cg_prep<<<np, kRowThreads, 0, st>>>(L0.nn, L0.mask, f, u, part);
}

void launch_cg_residual(int vt, const Level& L0, double omega, const double* f, const double* u,
                        double* r, int mode, double* part, const double* part_ff, int np,
                        DevState* ds, unsigned* cnt, cudaGraphConditionalHandle hc, int use_cond,
                        cudaStream_t st) {
  if (L0.k >= 2) {  // r = K u by elements, then the residual step
    launch_q2_op(kVtF64, L0, L0.K64, L0.Y, nullptr, u, nullptr, 0.0, 2, r, L0.sms, st);
    VT_DISPATCH(vt, (k_cg_residual_y<T><<<np, kRowThreads, 0, st>>>(
                        L0.nn, f, r, (T*)L0.b, dinv_of<T>(L0), (T)omega, (T*)L0.v, part, part_ff, np,
                        mode, ds, cnt, hc, use_cond)));
    return;
  }
  const LevelView<double> V0 = view<double>(L0);
  VT_DISPATCH(vt, TILE_ORD(V0, (k_cg_residual<T, kOrd><<<tile_grid<double>(L0), tile_threads<double>(),
                                                         tile_smem<double>(), st>>>(
                                   V0, f, u, r, (T*)L0.b, dinv_of<T>(L0), (T)omega, (T*)L0.v, part,
                                   part_ff, np, mode, ds, cnt, hc, use_cond))));
}

void launch_cg_dots_rz(int vt, const Level& L0, const double* r, const double* q, double* part_rz,
                       double* part_zq, int np, DevState* ds, unsigned* cnt, cudaStream_t st) {
  VT_DISPATCH(vt, (k_cg_dots_rz<T><<<np, kRowThreads, 0, st>>>(L0.nn, r, (const T*)L0.z, q, part_rz,
                                                               part_zq, ds, cnt)));
}

void launch_cg_dir(int vt, const Level& L0, double* p, int np, const DevState* ds,
                   cudaStream_t st) {
  VT_DISPATCH(vt, (k_cg_dir<T><<<np, kRowThreads, 0, st>>>(L0.nn, (const T*)L0.z, p, ds)));
}

void launch_cg_apply(const Level& L0, const double* p, double* q, double* part, int np, DevState* ds,
                     unsigned* cnt, cudaStream_t st) {
  if (L0.k >= 2) {
    launch_q2_op(kVtF64, L0, L0.K64, L0.Y, nullptr, p, nullptr, 0.0, 2, q, L0.sms, st);
    k_cg_apply_y<<<np, kRowThreads, 0, st>>>(L0.nn, p, q, part, ds, cnt);
    return;
  }
  const LevelView<double> V0 = view<double>(L0);
  TILE_ORD(V0, (k_cg_apply<kOrd><<<tile_grid<double>(L0), tile_threads<double>(), tile_smem<double>(), st>>>(
                   V0, p, q, part, ds, cnt)));
}

void launch_cg_update(int vt, const Level& L0, double omega, double* u, double* r, const double* p,
                      const double* q, double* part_rr, int np, DevState* ds, unsigned* cnt,
                      cudaGraphConditionalHandle hc, int use_cond, cudaStream_t st) {
  VT_DISPATCH(vt, (k_cg_update<T><<<np, kRowThreads, 0, st>>>(
                      L0.nn, u, r, p, q, (T*)L0.b, dinv_of<T>(L0), (T)omega, (T*)L0.v, part_rr,
                      ds, cnt, hc, use_cond)));
}

void launch_apply_diag(int vt, const Level& L, const double* x, double* y, cudaStream_t st) {
  if (L.k >= 2) {
    if (vt == kVtF64) {  // FP64 in and out: no staging
      launch_q2_op(kVtF64, L, L.K64, L.Y, nullptr, x, nullptr, 0.0, 2, y, L.sms, st);
      return;
    }
    // through the level's preconditioner vectors, whose type is vt (the
    // caller checks that vt is the handle's preconditioner arithmetic)
    const size_t nd = L.ndof;
    launch_vec_in(vt, nd, x, L.v, st);
    launch_q2_op(vt, L, L.K32, L.Y, nullptr, L.v, nullptr, 0.0, 2, L.r, L.sms, st);
    launch_vec_out(vt, nd, L.r, y, st);
    return;
  }
  VT_DISPATCH(vt, TILE_ORD(view<T>(L), (k_apply_diag<T, kOrd><<<tile_grid<T>(L), tile_threads<T>(),
                                                                   tile_smem<T>(), st>>>(view<T>(L), x, y))));
}

template <typename T, bool kOrd>
cudaError_t allow_tile_smem() {
  const int b = (int)tile_smem<T>();
  const int b64 = (int)tile_smem<double>();
  cudaError_t e = cudaFuncSetAttribute(k_vc_pre<T, kOrd>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_vc_post<T, kOrd>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_vc_post_dots<T, kOrd>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_apply_diag<T, kOrd>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_cg_residual<T, kOrd>, cudaFuncAttributeMaxDynamicSharedMemorySize, b64);
  return e;
}

cudaError_t configure_tile_kernels() {
  cudaError_t e = allow_tile_smem<double, false>();
  if (e == cudaSuccess) e = allow_tile_smem<float, false>();
  if (e == cudaSuccess) e = allow_tile_smem<dfloat, false>();
  if (e == cudaSuccess) e = allow_tile_smem<double, true>();
  if (e == cudaSuccess) e = allow_tile_smem<float, true>();
  if (e == cudaSuccess) e = allow_tile_smem<dfloat, true>();
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_cg_apply<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tile_smem<double>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_cg_apply<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tile_smem<double>());
  return e;
}

void launch_cast(bool to_fp64, size_t n, const void* a, void* b, bool src_fp64, cudaStream_t st) {
  const int g = (int)((n + kBS - 1) / kBS < 4096 ? (n + kBS - 1) / kBS : 4096);
  if (to_fp64) {
    if (src_fp64)
      k_cast<double, double><<<g, kBS, 0, st>>>(n, (const double*)a, (double*)b);
    else
      k_cast<float, double><<<g, kBS, 0, st>>>(n, (const float*)a, (double*)b);
  } else {
    if (src_fp64)
      k_cast<double, float><<<g, kBS, 0, st>>>(n, (const double*)a, (float*)b);
    else
      k_cast<float, float><<<g, kBS, 0, st>>>(n, (const float*)a, (float*)b);
  }
}

void launch_vec_in(int vt, size_t n, const double* a, void* b, cudaStream_t st) {
  const int g = (int)((n + kBS - 1) / kBS < 4096 ? (n + kBS - 1) / kBS : 4096);
  VT_DISPATCH(vt, (k_cast<double, T><<<g, kBS, 0, st>>>(n, a, (T*)b)));
}

void launch_vec_out(int vt, size_t n, const void* a, double* b, cudaStream_t st) {
  const int g = (int)((n + kBS - 1) / kBS < 4096 ? (n + kBS - 1) / kBS : 4096);
  VT_DISPATCH(vt, (k_cast<T, double><<<g, kBS, 0, st>>>(n, (const T*)a, b)));
}

}  // namespace tos
