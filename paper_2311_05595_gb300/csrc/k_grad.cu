// Objective and sensitivities of Sec. 3.4: compliance c = f^T u, the subcell
// strain energies s_{e,i} = u_e^T K^(e_i) u_e with the density derivative
// -p rho^(p-1) (E0 - Emin) s_{e,i}, and the chain rule through the filter
// (dc/dx = H^T dc/drho).  All FP64.
#include "internal.cuh"

namespace tos {
namespace {

// One thread per (element, subcell): gather the 24 element DOFs and form
// the quadratic form with the symmetric subcell table row by row.
__global__ void k_energy_grad(int ex, int ey, int ez, int n, int Lx, int Ly,
                              const double* __restrict__ u, const double* __restrict__ tabsym,
                              const double* __restrict__ rho, double penal, double dE, int Dx,
                              int Dy, int first, double* __restrict__ g) {
  const int m = n * n * n;
  const long E = (long)ex * ey * ez;
  const long total = E * m;
  // subcell-major: the lanes of a warp share the subcell s (its 300-entry
  // table is read once per warp) and take consecutive elements
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total;
       t += (long)gridDim.x * blockDim.x) {
    const long e = t % E;
    const int s = (int)(t / E);
    const int exi = e % ex, eyi = (e / ex) % ey, ezi = e / ((long)ex * ey);
    double ue[kEdofQ1];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const long node = (exi + (a & 1)) + (long)Lx * ((eyi + ((a >> 1) & 1)) + (long)Ly * (ezi + (a >> 2)));
      ue[3 * a] = u[3 * node];
      ue[3 * a + 1] = u[3 * node + 1];
      ue[3 * a + 2] = u[3 * node + 2];
    }
    const double* K = tabsym + (size_t)s * kSym;
    double en = 0.0;
    int idx = 0;
#pragma unroll
    for (int R = 0; R < kEdofQ1; ++R) {
      double acc = 0.5 * K[idx] * ue[R];
      ++idx;
#pragma unroll
      for (int C = R + 1; C < kEdofQ1; ++C, ++idx) acc += K[idx] * ue[C];
      en += ue[R] * acc;
    }
    en *= 2.0;
    const int a = s % n, b = (s / n) % n, c = s / (n * n);
    const long cell = (n * exi + a) + (long)Dx * ((n * eyi + b) + (long)Dy * (n * ezi + c));
    const double gv = -penal * simp_pow(rho[cell], penal - 1.0) * dE * en;
    g[cell] = first ? gv : g[cell] + gv;
  }
}

__global__ void k_scale(size_t n, const double* __restrict__ a, const double* __restrict__ s,
                        double* __restrict__ out) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    out[t] = a[t] * s[t];
}

// (H^T g)_k = sum_i (w_ik / w_i) g_i = sum_offsets w_o * (g_i / w_i): the
// gather form of the transpose (the Gaussian weights are symmetric in the
// offset), so no atomics and a fixed summation order.
__global__ void k_filter_T(int Dx, int Dy, int Dz, int noff, const int4* __restrict__ off,
                           const double* __restrict__ wgt, const double* __restrict__ gt,
                           double* __restrict__ gx) {
  const long N = (long)Dx * Dy * Dz;
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < N; c += (long)gridDim.x * blockDim.x) {
    const int cx = c % Dx, cy = (c / Dx) % Dy, cz = c / ((long)Dx * Dy);
    double s = 0.0;
    for (int o = 0; o < noff; ++o) {
      const int4 d = off[o];
      const int X = cx + d.x, Y = cy + d.y, Z = cz + d.z;
      if (X >= 0 && X < Dx && Y >= 0 && Y < Dy && Z >= 0 && Z < Dz)
        s += wgt[o] * gt[X + (long)Dx * (Y + (long)Dy * Z)];
    }
    gx[c] = s;
  }
}

// (P^T gt)_j for the design-grid projection: sum over the density cells i
// within r of design cell j of wt(dist) * gt_i, gt = g / w_i (gather form,
// fixed order).  The neighbour decision rounds as in the forward kernel.
__device__ __forceinline__ double pdist2(int jx, int jy, int jz, int d, int cx, int cy, int cz, int n) {
  const double tx = __dsub_rn(__ddiv_rn(jx + 0.5, (double)d), __ddiv_rn(cx + 0.5, (double)n));
  const double ty = __dsub_rn(__ddiv_rn(jy + 0.5, (double)d), __ddiv_rn(cy + 0.5, (double)n));
  const double tz = __dsub_rn(__ddiv_rn(jz + 0.5, (double)d), __ddiv_rn(cz + 0.5, (double)n));
  return __dadd_rn(__dadd_rn(__dmul_rn(tx, tx), __dmul_rn(ty, ty)), __dmul_rn(tz, tz));
}

__global__ void k_proj_T(ProjGrid P, const double* __restrict__ gt, double* __restrict__ gx) {
  const long G = (long)P.Gx * P.Gy * P.Gz;
  const int Rn = (int)ceil(P.r * P.n) + 1;
  const double r2 = P.r * P.r * (1.0 + 1e-12), s2 = 2.0 * (P.r / 3.0) * (P.r / 3.0);
  for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < G; j += (long)gridDim.x * blockDim.x) {
    const int jx = j % P.Gx, jy = (j / P.Gx) % P.Gy, jz = j / ((long)P.Gx * P.Gy);
    const int bx = (int)floor((jx + 0.5) / P.d * P.n - 0.5), by = (int)floor((jy + 0.5) / P.d * P.n - 0.5),
              bz = (int)floor((jz + 0.5) / P.d * P.n - 0.5);
    double s = 0.0;
    for (int cz = max(bz - Rn, 0); cz <= min(bz + Rn + 1, P.Dz - 1); ++cz)
      for (int cy = max(by - Rn, 0); cy <= min(by + Rn + 1, P.Dy - 1); ++cy)
        for (int cx = max(bx - Rn, 0); cx <= min(bx + Rn + 1, P.Dx - 1); ++cx) {
          const double q = pdist2(jx, jy, jz, P.d, cx, cy, cz, P.n);
          if (q > r2) continue;
          s += exp(-q / s2) * gt[cx + (long)P.Dx * (cy + (long)P.Dy * cz)];
        }
    gx[j] = s;
  }
}

__device__ __forceinline__ double block_sum_g(double v) {
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

__global__ void k_dot_masked(long ndof, const uint8_t* __restrict__ mask, const double* __restrict__ f,
                             const double* __restrict__ u, double* __restrict__ part) {
  double s = 0.0;
  for (long d = blockIdx.x * (long)blockDim.x + threadIdx.x; d < ndof; d += (long)gridDim.x * blockDim.x)
    if (!mask[d]) s += f[d] * u[d];
  s = block_sum_g(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_sum_to(const double* __restrict__ part, int np, double* __restrict__ out) {
  double v = 0.0;
  for (int t = threadIdx.x; t < np; t += blockDim.x) v += part[t];
  v = block_sum_g(v);
  if (threadIdx.x == 0) *out = v;
}

inline int grid_for(long n, int cap = 4096) {
  long g = (n + kBS - 1) / kBS;
  if (g < 1) g = 1;
  return (int)(g < cap ? g : cap);
}

}  // namespace

void launch_energy_grad(const Level& L0, int n, const double* u, const double* tabsym,
                        const double* rho, double penal, double dE, int Dx, int Dy, bool first,
                        double* g_rho, cudaStream_t st) {
  const long total = (long)L0.ex * L0.ey * L0.ez * n * n * n;
  k_energy_grad<<<grid_for(total, 8192), kBS, 0, st>>>(L0.ex, L0.ey, L0.ez, n, L0.Lx, L0.Ly, u,
                                                       tabsym, rho, penal, dE, Dx, Dy, first ? 1 : 0,
                                                       g_rho);
}

void launch_scale(size_t n, const double* a, const double* s, double* out, cudaStream_t st) {
  k_scale<<<grid_for((long)n), kBS, 0, st>>>(n, a, s, out);
}

void launch_proj_T(const ProjGrid& P, const double* gt, double* gx, cudaStream_t st) {
  k_proj_T<<<grid_for((long)P.Gx * P.Gy * P.Gz), kBS, 0, st>>>(P, gt, gx);
}

void launch_filter_T(int Dx, int Dy, int Dz, int noff, const int4* off, const double* wgt,
                     const double* gt, double* gx, cudaStream_t st) {
  k_filter_T<<<grid_for((long)Dx * Dy * Dz), kBS, 0, st>>>(Dx, Dy, Dz, noff, off, wgt, gt, gx);
}

void launch_compliance(const Level& L0, const uint8_t* fixed, const double* f, const double* u,
                       double* part, int np, DevState* ds, cudaStream_t st) {
  k_dot_masked<<<np, kBS, 0, st>>>((long)L0.ndof, fixed, f, u, part);
  k_sum_to<<<1, kBS, 0, st>>>(part, np, &ds->c);
}

}  // namespace tos
