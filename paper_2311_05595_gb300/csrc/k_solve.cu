// Solve kernels: the 27-point block-stencil operator apply (K u, Sec. 3.3
// Eq. matrixK_mr assembled per node), the multigrid cycle of Algorithm 1
// (damped Jacobi smoothing, linear-interpolation transfer, dense coarse
// solve), and the FP64 preconditioned CG of Sec. 7.2 with fused vector
// updates and deterministic two-stage reductions (warp shuffles, then a
// fixed-order sum of per-block partials).
#include "internal.cuh"

namespace tos {

template <typename T>
LevelView<T> view(const Level& L);
template <>
LevelView<double> view<double>(const Level& L) {
  return LevelView<double>{L.Lx, L.Ly, L.Lz, L.nn, L.S64, L.dinv64, L.mask};
}
template <>
LevelView<float> view<float>(const Level& L) {
  return LevelView<float>{L.Lx, L.Ly, L.Lz, L.nn, L.S32, L.dinv32, L.mask};
}

namespace {

// y = (A x)_node for the three DOFs of one node; ld(nb, x0, x1, x2) loads
// the operand at neighbour node nb.
template <typename T, typename LD>
__device__ __forceinline__ void stencil_node(const LevelView<T>& V, long node, int i, int j, int l,
                                             LD ld, T& y0, T& y1, T& y2) {
  y0 = y1 = y2 = T(0);
  const size_t nn = V.nn;
#pragma unroll
  for (int o = 0; o < 27; ++o) {
    const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
    const int ii = i + dx, jj = j + dy, ll = l + dz;
    if (ii < 0 || ii >= V.Lx || jj < 0 || jj >= V.Ly || ll < 0 || ll >= V.Lz) continue;
    const long nb = node + dx + (long)V.Lx * (dy + (long)V.Ly * dz);
    T x0, x1, x2;
    ld(nb, x0, x1, x2);
    const T* s = V.S + (size_t)o * 9 * nn + node;
    y0 += s[0] * x0 + s[nn] * x1 + s[2 * nn] * x2;
    y1 += s[3 * nn] * x0 + s[4 * nn] * x1 + s[5 * nn] * x2;
    y2 += s[6 * nn] * x0 + s[7 * nn] * x1 + s[8 * nn] * x2;
  }
}

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

// Sum of np partials, computed identically by every block (fixed order);
// the result is broadcast to all threads of the block.
__device__ __forceinline__ double reduce_parts(const double* __restrict__ part, int np) {
  __shared__ double bc;
  double v = 0.0;
  for (int t = threadIdx.x; t < np; t += blockDim.x) v += part[t];
  v = block_sum(v);
  if (threadIdx.x == 0) bc = v;
  __syncthreads();
  const double r = bc;
  __syncthreads();
  return r;
}

#define NODE_LOOP(nn)                                                              \
  for (long node = blockIdx.x * (long)blockDim.x + threadIdx.x; node < (nn);       \
       node += (long)gridDim.x * blockDim.x)

#define NODE_IJL(V)                                                                \
  const int i = node % (V).Lx, j = (node / (V).Lx) % (V).Ly,                       \
            l = node / ((long)(V).Lx * (V).Ly)

// ---- multigrid cycle ------------------------------------------------------

// Pre-smoothing from a zero guess and the residual, fused:
// v = omega D^-1 b, r = b - A v.
template <typename T>
__global__ void k_vc_pre(LevelView<T> V, T omega, const T* __restrict__ b, T* __restrict__ v,
                         T* __restrict__ r) {
  NODE_LOOP(V.nn) {
    NODE_IJL(V);
    T y0, y1, y2;
    stencil_node(V, node, i, j, l,
                 [&](long nb, T& x0, T& x1, T& x2) {
                   x0 = omega * V.dinv[3 * nb] * b[3 * nb];
                   x1 = omega * V.dinv[3 * nb + 1] * b[3 * nb + 1];
                   x2 = omega * V.dinv[3 * nb + 2] * b[3 * nb + 2];
                 },
                 y0, y1, y2);
    const T b0 = b[3 * node], b1 = b[3 * node + 1], b2 = b[3 * node + 2];
    v[3 * node] = omega * V.dinv[3 * node] * b0;
    v[3 * node + 1] = omega * V.dinv[3 * node + 1] * b1;
    v[3 * node + 2] = omega * V.dinv[3 * node + 2] * b2;
    r[3 * node] = b0 - y0;
    r[3 * node + 1] = b1 - y1;
    r[3 * node + 2] = b2 - y2;
  }
}

// r_H = M_H P^T r_h: each coarse node gathers the 3x3x3 fine nodes around its
// coincident fine node with weights (1, 1/2) per axis.
template <typename T>
__global__ void k_vc_restrict(int Lxf, int Lyf, int Lzf, int Lxc, int Lyc, int Lzc,
                              const uint8_t* __restrict__ maskc, const T* __restrict__ rf,
                              T* __restrict__ bc) {
  const long nnc = (long)Lxc * Lyc * Lzc;
  NODE_LOOP(nnc) {
    const int I = node % Lxc, J = (node / Lxc) % Lyc, K = node / ((long)Lxc * Lyc);
    T a0 = 0, a1 = 0, a2 = 0;
    for (int dz = -1; dz <= 1; ++dz) {
      const int l = 2 * K + dz;
      if (l < 0 || l >= Lzf) continue;
      const T wz = dz ? T(0.5) : T(1);
      for (int dy = -1; dy <= 1; ++dy) {
        const int j = 2 * J + dy;
        if (j < 0 || j >= Lyf) continue;
        const T wyz = wz * (dy ? T(0.5) : T(1));
        for (int dx = -1; dx <= 1; ++dx) {
          const int i = 2 * I + dx;
          if (i < 0 || i >= Lxf) continue;
          const T wgt = wyz * (dx ? T(0.5) : T(1));
          const long f = i + (long)Lxf * (j + (long)Lyf * l);
          a0 += wgt * rf[3 * f];
          a1 += wgt * rf[3 * f + 1];
          a2 += wgt * rf[3 * f + 2];
        }
      }
    }
    bc[3 * node] = maskc[3 * node] ? T(0) : a0;
    bc[3 * node + 1] = maskc[3 * node + 1] ? T(0) : a1;
    bc[3 * node + 2] = maskc[3 * node + 2] ? T(0) : a2;
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
    T a0 = 0, a1 = 0, a2 = 0;
    for (int K = K0; K <= K1; ++K) {
      const T wz = (K0 == K1) ? T(1) : T(0.5);
      for (int J = J0; J <= J1; ++J) {
        const T wyz = wz * ((J0 == J1) ? T(1) : T(0.5));
        for (int I = I0; I <= I1; ++I) {
          const T wgt = wyz * ((I0 == I1) ? T(1) : T(0.5));
          const long c = I + (long)Lxc * (J + (long)Lyc * K);
          a0 += wgt * zc[3 * c];
          a1 += wgt * zc[3 * c + 1];
          a2 += wgt * zc[3 * c + 2];
        }
      }
    }
    if (!maskf[3 * node]) v[3 * node] += a0;
    if (!maskf[3 * node + 1]) v[3 * node + 1] += a1;
    if (!maskf[3 * node + 2]) v[3 * node + 2] += a2;
  }
}

// Post-smoothing: z = v + omega D^-1 (b - A v).
template <typename T>
__global__ void k_vc_post(LevelView<T> V, T omega, const T* __restrict__ b, const T* __restrict__ v,
                          T* __restrict__ z) {
  NODE_LOOP(V.nn) {
    NODE_IJL(V);
    T y0, y1, y2;
    stencil_node(V, node, i, j, l,
                 [&](long nb, T& x0, T& x1, T& x2) {
                   x0 = v[3 * nb];
                   x1 = v[3 * nb + 1];
                   x2 = v[3 * nb + 2];
                 },
                 y0, y1, y2);
    z[3 * node] = v[3 * node] + omega * V.dinv[3 * node] * (b[3 * node] - y0);
    z[3 * node + 1] = v[3 * node + 1] + omega * V.dinv[3 * node + 1] * (b[3 * node + 1] - y1);
    z[3 * node + 2] = v[3 * node + 2] + omega * V.dinv[3 * node + 2] * (b[3 * node + 2] - y2);
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

// ---- FP64 preconditioned CG -------------------------------------------------

__global__ void k_cg_prep(int nn, const uint8_t* __restrict__ mask, const double* __restrict__ fin,
                          const double* __restrict__ uin, double* __restrict__ f,
                          double* __restrict__ u, double* __restrict__ part) {
  double s = 0.0;
  NODE_LOOP(nn) {
    for (int c = 0; c < 3; ++c) {
      const long d = 3 * node + c;
      const bool fx = mask[d] != 0;
      const double fv = fx ? 0.0 : fin[d];
      f[d] = fv;
      u[d] = fx ? 0.0 : uin[d];
      s += fv * fv;
    }
  }
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// r = f - K u (FP64), optional cast of r into the preconditioner input b0,
// partial ||r||^2.
template <typename T>
__global__ void k_cg_residual(LevelView<double> V, const double* __restrict__ f,
                              const double* __restrict__ u, double* __restrict__ r,
                              T* __restrict__ b0, double* __restrict__ part) {
  double s = 0.0;
  NODE_LOOP(V.nn) {
    NODE_IJL(V);
    double y0, y1, y2;
    stencil_node(V, node, i, j, l,
                 [&](long nb, double& x0, double& x1, double& x2) {
                   x0 = u[3 * nb];
                   x1 = u[3 * nb + 1];
                   x2 = u[3 * nb + 2];
                 },
                 y0, y1, y2);
    const double r0 = f[3 * node] - y0, r1 = f[3 * node + 1] - y1, r2 = f[3 * node + 2] - y2;
    r[3 * node] = r0;
    r[3 * node + 1] = r1;
    r[3 * node + 2] = r2;
    if (b0 != nullptr) {
      b0[3 * node] = (T)r0;
      b0[3 * node + 1] = (T)r1;
      b0[3 * node + 2] = (T)r2;
    }
    s += r0 * r0 + r1 * r1 + r2 * r2;
  }
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__device__ __forceinline__ void set_cond(cudaGraphConditionalHandle hc, int use_cond, unsigned v) {
  if (use_cond) cudaGraphSetConditional(hc, v);
}

__global__ void k_cg_check_init(const double* __restrict__ part_ff, const double* __restrict__ part_rr,
                                int np, DevState* __restrict__ ds, cudaGraphConditionalHandle hc,
                                int use_cond) {
  const double ff = reduce_parts(part_ff, np);
  const double rr = reduce_parts(part_rr, np);
  if (threadIdx.x == 0) {
    ds->ff = ff;
    ds->rr = rr;
    ds->iter = 0;
    ds->status = ds->coarse_status ? (int)TOSOLVE_EBREAKDOWN : 0;
    const bool conv = (rr <= ds->tol2 * ff) || ff == 0.0;
    ds->converged = conv;
    if (!(rr == rr)) ds->status = TOSOLVE_EBREAKDOWN;
    set_cond(hc, use_cond, (conv || ds->status || ds->maxit <= 0) ? 0u : 1u);
  }
}

template <typename T>
__global__ void k_cg_dots_rz(int nn, const double* __restrict__ r, const T* __restrict__ z,
                             const double* __restrict__ q, double* __restrict__ part_rz,
                             double* __restrict__ part_zq) {
  double a = 0.0, b = 0.0;
  NODE_LOOP(nn) {
    for (int c = 0; c < 3; ++c) {
      const double zv = (double)z[3 * node + c];
      a += r[3 * node + c] * zv;
      b += zv * q[3 * node + c];
    }
  }
  a = block_sum(a);
  b = block_sum(b);
  if (threadIdx.x == 0) {
    part_rz[blockIdx.x] = a;
    part_zq[blockIdx.x] = b;
  }
}

// Flexible (Polak-Ribiere) direction update, which stays valid for a
// preconditioner evaluated in lower precision:
//   beta = z_{k+1}^T (r_{k+1} - r_k) / (z_k^T r_k) = -alpha_k z_{k+1}^T q_k / rz_k.
template <typename T>
__global__ void k_cg_dir(int nn, const double* __restrict__ part_rz, const double* __restrict__ part_zq,
                         int np, const T* __restrict__ z, double* __restrict__ p,
                         DevState* __restrict__ ds) {
  const double rz_new = reduce_parts(part_rz, np);
  const double zq = reduce_parts(part_zq, np);
  const bool first = ds->iter == 0;
  const double beta = first ? 0.0 : -ds->alpha * zq / ds->rz;
  NODE_LOOP(nn) {
    for (int c = 0; c < 3; ++c) {
      const double zv = (double)z[3 * node + c];
      p[3 * node + c] = first ? zv : zv + beta * p[3 * node + c];
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ds->rz_next = rz_new;
    ds->beta = beta;
  }
}

__global__ void k_cg_apply(LevelView<double> V, const double* __restrict__ p, double* __restrict__ q,
                           double* __restrict__ part) {
  double s = 0.0;
  NODE_LOOP(V.nn) {
    NODE_IJL(V);
    double y0, y1, y2;
    stencil_node(V, node, i, j, l,
                 [&](long nb, double& x0, double& x1, double& x2) {
                   x0 = p[3 * nb];
                   x1 = p[3 * nb + 1];
                   x2 = p[3 * nb + 2];
                 },
                 y0, y1, y2);
    q[3 * node] = y0;
    q[3 * node + 1] = y1;
    q[3 * node + 2] = y2;
    s += p[3 * node] * y0 + p[3 * node + 1] * y1 + p[3 * node + 2] * y2;
  }
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

template <typename T>
__global__ void k_cg_update(int nn, const double* __restrict__ part_pq, int np, double* __restrict__ u,
                            double* __restrict__ r, const double* __restrict__ p,
                            const double* __restrict__ q, T* __restrict__ b0,
                            double* __restrict__ part_rr, DevState* __restrict__ ds) {
  const double pq = reduce_parts(part_pq, np);
  const double rz = ds->rz_next;
  const double alpha = rz / pq;
  const bool ok = (pq > 0.0) && (alpha == alpha) && (fabs(alpha) < 1e300);
  double s = 0.0;
  if (ok) {
    NODE_LOOP(nn) {
      for (int c = 0; c < 3; ++c) {
        const long d = 3 * node + c;
        u[d] += alpha * p[d];
        const double rv = r[d] - alpha * q[d];
        r[d] = rv;
        b0[d] = (T)rv;
        s += rv * rv;
      }
    }
  }
  s = block_sum(s);
  if (threadIdx.x == 0) part_rr[blockIdx.x] = s;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ds->alpha = alpha;
    ds->rz = rz;
    if (!ok) ds->status = TOSOLVE_EBREAKDOWN;
  }
}

__global__ void k_cg_check(const double* __restrict__ part_rr, int np, DevState* __restrict__ ds,
                           cudaGraphConditionalHandle hc, int use_cond) {
  const double rr = reduce_parts(part_rr, np);
  if (threadIdx.x == 0) {
    ds->rr = rr;
    ds->iter += 1;
    if (!(rr == rr)) ds->status = TOSOLVE_EBREAKDOWN;
    const bool conv = rr <= ds->tol2 * ds->ff;
    ds->converged = conv;
    set_cond(hc, use_cond, (conv || ds->status || ds->iter >= ds->maxit) ? 0u : 1u);
  }
}

__global__ void k_cg_final(const double* __restrict__ part_rr, int np, DevState* __restrict__ ds) {
  const double rr = reduce_parts(part_rr, np);
  if (threadIdx.x == 0) ds->rr_true = rr;
}

// Diagnostic: y = A x in the level's stored precision, FP64 in and out.
template <typename T>
__global__ void k_apply_diag(LevelView<T> V, const double* __restrict__ x, double* __restrict__ y) {
  NODE_LOOP(V.nn) {
    NODE_IJL(V);
    T y0, y1, y2;
    stencil_node(V, node, i, j, l,
                 [&](long nb, T& x0, T& x1, T& x2) {
                   x0 = (T)x[3 * nb];
                   x1 = (T)x[3 * nb + 1];
                   x2 = (T)x[3 * nb + 2];
                 },
                 y0, y1, y2);
    y[3 * node] = y0;
    y[3 * node + 1] = y1;
    y[3 * node + 2] = y2;
  }
}

template <typename A, typename B>
__global__ void k_cast(size_t n, const A* __restrict__ a, B* __restrict__ b) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    b[t] = (B)a[t];
}

inline int grid_nodes(long nn) {
  long g = (nn + kBS - 1) / kBS;
  if (g < 1) g = 1;
  return (int)(g < kMaxPart ? g : kMaxPart);
}

template <typename T>
void vcycle_rec(Level* lv, int l, int L, T omega, const double* Ainv, cudaStream_t st) {
  Level& F = lv[l];
  if (l == L - 1) {
    const int n = F.ndof;
    int g = (n * 32 + kBS - 1) / kBS;
    if (g > 1024) g = 1024;
    k_coarse_solve<T><<<g, kBS, 0, st>>>(n, Ainv, (const T*)F.b, (T*)F.z);
    return;
  }
  Level& C = lv[l + 1];
  const LevelView<T> V = view<T>(F);
  k_vc_pre<T><<<grid_nodes(F.nn), kBS, 0, st>>>(V, omega, (const T*)F.b, (T*)F.v, (T*)F.r);
  k_vc_restrict<T><<<grid_nodes(C.nn), kBS, 0, st>>>(F.Lx, F.Ly, F.Lz, C.Lx, C.Ly, C.Lz, C.mask,
                                                     (const T*)F.r, (T*)C.b);
  vcycle_rec<T>(lv, l + 1, L, omega, Ainv, st);
  k_vc_prolong<T><<<grid_nodes(F.nn), kBS, 0, st>>>(F.Lx, F.Ly, F.Lz, C.Lx, C.Ly, F.mask,
                                                    (const T*)C.z, (T*)F.v);
  k_vc_post<T><<<grid_nodes(F.nn), kBS, 0, st>>>(V, omega, (const T*)F.b, (const T*)F.v, (T*)F.z);
}

}  // namespace

void launch_vcycle(bool fp64, Level* lv, int L, double omega, int gamma, const double* Ainv,
                   cudaStream_t st) {
  (void)gamma;
  if (fp64)
    vcycle_rec<double>(lv, 0, L, omega, Ainv, st);
  else
    vcycle_rec<float>(lv, 0, L, (float)omega, Ainv, st);
}

void launch_cg_prep(const Level& L0, const double* fin, const double* uin, double* f, double* u,
                    double* part, int np, cudaStream_t st) {
  k_cg_prep<<<np, kBS, 0, st>>>(L0.nn, L0.mask, fin, uin, f, u, part);
}

void launch_cg_residual(bool fp64, const Level& L0, const double* f, const double* u, double* r,
                        void* b0, double* part, int np, cudaStream_t st) {
  if (fp64)
    k_cg_residual<double><<<np, kBS, 0, st>>>(view<double>(L0), f, u, r, (double*)b0, part);
  else
    k_cg_residual<float><<<np, kBS, 0, st>>>(view<double>(L0), f, u, r, (float*)b0, part);
}

void launch_cg_check_init(double* part_ff, double* part_rr, int np, DevState* ds,
                          cudaGraphConditionalHandle hc, int use_cond, cudaStream_t st) {
  k_cg_check_init<<<1, kBS, 0, st>>>(part_ff, part_rr, np, ds, hc, use_cond);
}

void launch_cg_dots_rz(bool fp64, const Level& L0, const double* r, const void* z, const double* q,
                       double* part_rz, double* part_zq, int np, cudaStream_t st) {
  if (fp64)
    k_cg_dots_rz<double><<<np, kBS, 0, st>>>(L0.nn, r, (const double*)z, q, part_rz, part_zq);
  else
    k_cg_dots_rz<float><<<np, kBS, 0, st>>>(L0.nn, r, (const float*)z, q, part_rz, part_zq);
}

void launch_cg_dir(bool fp64, const Level& L0, const double* part_rz, const double* part_zq, int np,
                   const void* z, double* p, DevState* ds, cudaStream_t st) {
  if (fp64)
    k_cg_dir<double><<<np, kBS, 0, st>>>(L0.nn, part_rz, part_zq, np, (const double*)z, p, ds);
  else
    k_cg_dir<float><<<np, kBS, 0, st>>>(L0.nn, part_rz, part_zq, np, (const float*)z, p, ds);
}

void launch_cg_apply(const Level& L0, const double* p, double* q, double* part, int np,
                     cudaStream_t st) {
  k_cg_apply<<<np, kBS, 0, st>>>(view<double>(L0), p, q, part);
}

void launch_cg_update(bool fp64, const Level& L0, const double* part_pq, int np, double* u,
                      double* r, const double* p, const double* q, void* b0, double* part_rr,
                      DevState* ds, cudaStream_t st) {
  if (fp64)
    k_cg_update<double><<<np, kBS, 0, st>>>(L0.nn, part_pq, np, u, r, p, q, (double*)b0, part_rr, ds);
  else
    k_cg_update<float><<<np, kBS, 0, st>>>(L0.nn, part_pq, np, u, r, p, q, (float*)b0, part_rr, ds);
}

void launch_cg_check(const double* part_rr, int np, DevState* ds, cudaGraphConditionalHandle hc,
                     int use_cond, cudaStream_t st) {
  k_cg_check<<<1, kBS, 0, st>>>(part_rr, np, ds, hc, use_cond);
}

void launch_cg_final(const double* part_rr, int np, DevState* ds, cudaStream_t st) {
  k_cg_final<<<1, kBS, 0, st>>>(part_rr, np, ds);
}

void launch_apply_diag(bool fp64, const Level& L, const double* x, double* y, cudaStream_t st) {
  if (fp64)
    k_apply_diag<double><<<grid_nodes(L.nn), kBS, 0, st>>>(view<double>(L), x, y);
  else
    k_apply_diag<float><<<grid_nodes(L.nn), kBS, 0, st>>>(view<float>(L), x, y);
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

}  // namespace tos
