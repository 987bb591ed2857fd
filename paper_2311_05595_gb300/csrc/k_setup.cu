// Setup kernels: the stacked subcell stiffness table (Sec. 3.3), the density
// filter (Sec. 2.2 / 3.2), SIMP weights (Eq. matrixK), and the per-design
// multigrid refresh of Sec. 7.2 (every level's operator and the coarsest
// level's direct solve, here its explicit inverse, are rebuilt for each new
// density field; the level structure itself is built once).
#include <cooperative_groups.h>

#include <algorithm>
#include <functional>
#include <mutex>

#include "internal.cuh"

namespace cg = cooperative_groups;

namespace tos {
namespace {

// 1D trilinear factors on [-1, 1]: phi_0 = (1 - t)/2, phi_1 = (1 + t)/2.
__device__ __forceinline__ double phi(int a, double t) { return a ? 0.5 * (1.0 + t) : 0.5 * (1.0 - t); }
__device__ __forceinline__ double dphi(int a) { return a ? 0.5 : -0.5; }

// K^(e_i) = int_{subcell i} lambda d_i N_a d_j N_b + mu d_j N_a d_i N_b
//                          + mu delta_ij grad N_a . grad N_b   (E = 1),
// the tensor form of int B^T D B, integrated with 2x2x2 Gauss points per
// subcell (exact for the trilinear element).  One block per subcell.
__global__ void k_subcell_table(int n, double nu, double h, double* __restrict__ tab) {
  __shared__ double g[8][8][3];  // [gauss point][node][direction], physical
  const int sub = blockIdx.x;
  const int sa = sub % n, sb = (sub / n) % n, sc = sub / (n * n);
  const double half = 1.0 / n;
  const double gp = 1.0 / sqrt(3.0);
  const int tid = threadIdx.x;
  if (tid < 64) {
    const int q = tid >> 3, node = tid & 7;
    const double xi = -1.0 + (2 * sa + 1) * half + half * ((q & 1) ? gp : -gp);
    const double eta = -1.0 + (2 * sb + 1) * half + half * ((q & 2) ? gp : -gp);
    const double zeta = -1.0 + (2 * sc + 1) * half + half * ((q & 4) ? gp : -gp);
    const int ix = node & 1, iy = (node >> 1) & 1, iz = node >> 2;
    const double s = 2.0 / h;
    g[q][node][0] = s * dphi(ix) * phi(iy, eta) * phi(iz, zeta);
    g[q][node][1] = s * phi(ix, xi) * dphi(iy) * phi(iz, zeta);
    g[q][node][2] = s * phi(ix, xi) * phi(iy, eta) * dphi(iz);
  }
  __syncthreads();
  const double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  const double mu = 1.0 / (2.0 * (1.0 + nu));
  const double wq = half * half * half * (0.125 * h * h * h);  // GL weights are 1
  for (int t = tid; t < kEdofQ1 * kEdofQ1; t += blockDim.x) {
    const int R = t / kEdofQ1, C = t % kEdofQ1;
    const int a = R / 3, i = R % 3, b = C / 3, j = C % 3;
    double acc = 0.0;
    for (int q = 0; q < 8; ++q) {
      const double* ga = g[q][a];
      const double* gb = g[q][b];
      double v = lam * ga[i] * gb[j] + mu * ga[j] * gb[i];
      if (i == j) v += mu * (ga[0] * gb[0] + ga[1] * gb[1] + ga[2] * gb[2]);
      acc += v;
    }
    tab[(size_t)sub * kEdofQ1 * kEdofQ1 + t] = wq * acc;
  }
}

__global__ void k_symmetrize(int m, const double* __restrict__ tab, double* __restrict__ tabsym) {
  const int s = blockIdx.x;
  for (int t = threadIdx.x; t < kEdofQ1 * kEdofQ1; t += blockDim.x) {
    const int R = t / kEdofQ1, C = t % kEdofQ1;
    if (R <= C) tabsym[(size_t)s * kSym + sym_index(R, C)] = tab[(size_t)s * kEdofQ1 * kEdofQ1 + t];
  }
}

// Polynomial coefficients of one 1D factor: value (deriv = 0) or derivative.
__device__ __forceinline__ void poly1(int a, int deriv, double c[2]) {
  if (deriv) { c[0] = a ? 0.5 : -0.5; c[1] = 0.0; }
  else { c[0] = 0.5; c[1] = a ? 0.5 : -0.5; }
}

// Coefficient of xi^k (k = 0..2) of the product of two degree-1 factors.
__device__ __forceinline__ double prod_coef(const double u[2], const double v[2], int k) {
  if (k == 0) return u[0] * v[0];
  if (k == 1) return u[0] * v[1] + u[1] * v[0];
  return u[1] * v[1];
}

// Moment basis of the trilinear element: the integrand of the element
// matrix, in reference coordinates, is sum_alpha C_alpha xi^alpha with
// alpha in {0,1,2}^3, so K^(e) = (h/2) sum_alpha M_alpha C_alpha with
// M_alpha = int_e w(xi) xi^alpha dxi.  Thread per (alpha, upper entry).
__global__ void k_moment_basis(double nu, double* __restrict__ cmom) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 27 * kSym) return;
  const int alpha = t / kSym, e = t % kSym;
  int R = 0;
  while (sym_index(R, kEdofQ1 - 1) < e) ++R;
  const int C = R + (e - sym_index(R, R));
  const int al[3] = {alpha % 3, (alpha / 3) % 3, alpha / 9};
  const int a = R / 3, i = R % 3, b = C / 3, j = C % 3;
  const int na[3] = {a & 1, (a >> 1) & 1, a >> 2};
  const int nb[3] = {b & 1, (b >> 1) & 1, b >> 2};
  // T(p, s) = coefficient of xi^alpha in d_p N_a * d_s N_b
  auto T = [&](int p, int s) {
    double v = 1.0;
    for (int ax = 0; ax < 3; ++ax) {
      double u[2], w[2];
      poly1(na[ax], p == ax, u);
      poly1(nb[ax], s == ax, w);
      v *= prod_coef(u, w, al[ax]);
    }
    return v;
  };
  const double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  const double mu = 1.0 / (2.0 * (1.0 + nu));
  double v = lam * T(i, j) + mu * T(j, i);
  if (i == j) v += mu * (T(0, 0) + T(1, 1) + T(2, 2));
  cmom[t] = v;
}

__global__ void k_filter_init(int Dx, int Dy, int Dz, int noff, const int4* __restrict__ off,
                              const double* __restrict__ wgt, double* __restrict__ invom) {
  const long N = (long)Dx * Dy * Dz;
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < N; c += (long)gridDim.x * blockDim.x) {
    const int cx = c % Dx, cy = (c / Dx) % Dy, cz = c / ((long)Dx * Dy);
    double s = 0.0;
    for (int o = 0; o < noff; ++o) {
      const int4 d = off[o];
      const int x = cx + d.x, y = cy + d.y, z = cz + d.z;
      if (x >= 0 && x < Dx && y >= 0 && y < Dy && z >= 0 && z < Dz) s += wgt[o];
    }
    invom[c] = 1.0 / s;
  }
}

// Projection from a coarser design grid (Eq. projdsgn, d_mr < n_mr): the
// filter weights between density-cell centres (c + 1/2) / n and design-cell
// centres (j + 1/2) / d, in element units, neighbours at dist <= r.  The
// squared distance is formed with explicit rounding (no fused operations)
// in the same order as the definition, so the neighbour decision is the
// same as a plain FP64 evaluation of it.
__device__ __forceinline__ double cell_dist2(int jx, int jy, int jz, int d, int cx, int cy, int cz, int n) {
  const double tx = __dsub_rn(__ddiv_rn(jx + 0.5, (double)d), __ddiv_rn(cx + 0.5, (double)n));
  const double ty = __dsub_rn(__ddiv_rn(jy + 0.5, (double)d), __ddiv_rn(cy + 0.5, (double)n));
  const double tz = __dsub_rn(__ddiv_rn(jz + 0.5, (double)d), __ddiv_rn(cz + 0.5, (double)n));
  return __dadd_rn(__dadd_rn(__dmul_rn(tx, tx), __dmul_rn(ty, ty)), __dmul_rn(tz, tz));
}

// Sum over the design cells within r of density cell c of wt(dist) * v_j
// (v = nullptr: of wt alone).
__device__ __forceinline__ double proj_row(const ProjGrid& P, long c, const double* __restrict__ v) {
  const int cx = c % P.Dx, cy = (c / P.Dx) % P.Dy, cz = c / ((long)P.Dx * P.Dy);
  const int bx = (int)floor((cx + 0.5) / P.n * P.d - 0.5), by = (int)floor((cy + 0.5) / P.n * P.d - 0.5),
            bz = (int)floor((cz + 0.5) / P.n * P.d - 0.5);
  const double r2 = P.r * P.r * (1.0 + 1e-12), s2 = 2.0 * (P.r / 3.0) * (P.r / 3.0);
  double s = 0.0;
  for (int jz = max(bz - P.R, 0); jz <= min(bz + P.R + 1, P.Gz - 1); ++jz)
    for (int jy = max(by - P.R, 0); jy <= min(by + P.R + 1, P.Gy - 1); ++jy)
      for (int jx = max(bx - P.R, 0); jx <= min(bx + P.R + 1, P.Gx - 1); ++jx) {
        const double q = cell_dist2(jx, jy, jz, P.d, cx, cy, cz, P.n);
        if (q > r2) continue;
        const double wt = exp(-q / s2);
        s += v ? wt * v[jx + (long)P.Gx * (jy + (long)P.Gy * jz)] : wt;
      }
  return s;
}

__global__ void k_proj_init(ProjGrid P, double* __restrict__ invom) {
  const long N = (long)P.Dx * P.Dy * P.Dz;
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < N; c += (long)gridDim.x * blockDim.x)
    invom[c] = 1.0 / proj_row(P, c, nullptr);
}

__global__ void k_proj_fwd(ProjGrid P, const double* __restrict__ invom, const double* __restrict__ x,
                           double Emin, double dE, double penal, double* __restrict__ rho,
                           double* __restrict__ w) {
  const long N = (long)P.Dx * P.Dy * P.Dz;
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < N; c += (long)gridDim.x * blockDim.x) {
    const double r = proj_row(P, c, x) * invom[c];
    rho[c] = r;
    w[c] = Emin + simp_pow(r, penal) * dE;
  }
}

// rho_i = sum_j (w_ij / w_i) x_j (Eq. filter_weights / projdsgn) and the
// SIMP weight w_i = Emin + rho_i^p (E0 - Emin) (Eq. matrixK), fused.
__global__ void k_filter_fwd(int Dx, int Dy, int Dz, int noff, const int4* __restrict__ off,
                             const double* __restrict__ wgt, const double* __restrict__ invom,
                             const double* __restrict__ x, double Emin, double dE, double penal,
                             double* __restrict__ rho, double* __restrict__ w) {
  const long N = (long)Dx * Dy * Dz;
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < N; c += (long)gridDim.x * blockDim.x) {
    const int cx = c % Dx, cy = (c / Dx) % Dy, cz = c / ((long)Dx * Dy);
    double s = 0.0;
    for (int o = 0; o < noff; ++o) {
      const int4 d = off[o];
      const int X = cx + d.x, Y = cy + d.y, Z = cz + d.z;
      if (X >= 0 && X < Dx && Y >= 0 && Y < Dy && Z >= 0 && Z < Dz)
        s += wgt[o] * x[X + (long)Dx * (Y + (long)Dy * Z)];
    }
    const double r = s * invom[c];
    rho[c] = r;
    w[c] = Emin + simp_pow(r, penal) * dE;
  }
}

// Fine-level element matrices, Eq. matrixK_mr: K^(e) = sum_i w_{e,i} K^(e_i),
// upper triangle.  A block handles epb consecutive elements (their weights
// staged in shared memory); consecutive threads write consecutive entries.
// FP64 accumulation.
// Elements of z-layers [ze0, ze0 + nlayers) (a slab); Ke is indexed from the
// slab's first element.
template <typename T>
__global__ void k_elem_direct(int ex, int ey, int ze0, int nlayers, int n, int epb,
                              const double* __restrict__ w, int Dx, int Dy,
                              const double* __restrict__ tabsym, T* __restrict__ Ke) {
  extern __shared__ double ws[];  // epb * m
  const int m = n * n * n;
  const long E = (long)ex * ey * nlayers;
  const long e0 = (long)blockIdx.x * epb;
  for (int t = threadIdx.x; t < epb * m; t += blockDim.x) {
    const int q = t / m, s = t % m;
    const long e = e0 + q;
    double v = 0.0;
    if (e < E) {
      const int exi = e % ex, eyi = (e / ex) % ey, ezi = ze0 + (int)(e / ((long)ex * ey));
      const int a = s % n, b = (s / n) % n, c = s / (n * n);
      v = w[(n * exi + a) + (long)Dx * ((n * eyi + b) + (long)Dy * (n * ezi + c))];
    }
    ws[t] = v;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < epb * kSym; t += blockDim.x) {
    const int q = t / kSym, k = t % kSym;
    const long e = e0 + q;
    if (e >= E) continue;
    const double* wq = ws + q * m;
    double acc = 0.0;
    for (int s = 0; s < m; ++s) acc += wq[s] * tabsym[(size_t)s * kSym + k];
    Ke[e * kSym + k] = (T)acc;
  }
}

// Coarse-level element matrices from the density field: a level-l element
// covers N^3 density cells; K^(e) = (h/2) sum_alpha M_alpha C_alpha with the
// 27 polynomial moments M_alpha of the cellwise-constant weights.  This is
// Eq. matrixK_mr with N^3 subcells evaluated exactly through the moments.
//
// Moments are separable: for each row of cells along x, three sums
// sum_a w mu_k(a) (3 FMAs per cell), then 27 products with mu_l(b) mu_m(c)
// per row.  mu_k(a) = int over the a-th of N intervals of xi^k.
template <typename Acc>
__device__ __forceinline__ void row_moments(const double* __restrict__ w, long rowbase, int N,
                                            int b, int c, const Acc* mu0, const Acc* mu1,
                                            const Acc* mu2, Acc acc[27]) {
  Acc s0 = 0, s1 = 0, s2 = 0;
  for (int a = 0; a < N; ++a) {
    const Acc wv = (Acc)w[rowbase + a];
    s0 += wv * mu0[a];
    s1 += wv * mu1[a];
    s2 += wv * mu2[a];
  }
  const Acc sx[3] = {s0, s1, s2};
  const Acc my[3] = {mu0[b], mu1[b], mu2[b]};
  const Acc mz[3] = {mu0[c], mu1[c], mu2[c]};
#pragma unroll
  for (int gz = 0; gz < 3; ++gz)
#pragma unroll
    for (int gy = 0; gy < 3; ++gy)
#pragma unroll
      for (int gx = 0; gx < 3; ++gx) acc[gx + 3 * (gy + 3 * gz)] += sx[gx] * my[gy] * mz[gz];
}

template <typename Acc>
__device__ __forceinline__ void fill_mu(int N, Acc* mu0, Acc* mu1, Acc* mu2) {
  for (int a = threadIdx.x; a < N; a += blockDim.x) {
    const double t0 = -1.0 + 2.0 * a / N, t1 = -1.0 + 2.0 * (a + 1) / N;
    mu0[a] = (Acc)(t1 - t0);
    mu1[a] = (Acc)(0.5 * (t1 * t1 - t0 * t0));
    mu2[a] = (Acc)((t1 * t1 * t1 - t0 * t0 * t0) / 3.0);
  }
}

// Moments of small elements (N <= 4): one thread per element.
template <typename Acc>
__global__ void k_moments_thread(int ex, int ey, int ze0, int nlayers, int N,
                                 const double* __restrict__ w, int Dx, int Dy, Acc* __restrict__ M) {
  __shared__ Acc mu[3][4];
  fill_mu<Acc>(N, mu[0], mu[1], mu[2]);
  __syncthreads();
  const long E = (long)ex * ey * nlayers;
  const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (e >= E) return;
  const int exi = e % ex, eyi = (e / ex) % ey, ezi = ze0 + (int)(e / ((long)ex * ey));
  Acc acc[27];
#pragma unroll
  for (int q = 0; q < 27; ++q) acc[q] = 0;
  for (int c = 0; c < N; ++c)
    for (int b = 0; b < N; ++b) {
      const long rowbase = (N * exi) + (long)Dx * ((N * eyi + b) + (long)Dy * (N * ezi + c));
      row_moments<Acc>(w, rowbase, N, b, c, mu[0], mu[1], mu[2], acc);
    }
#pragma unroll
  for (int q = 0; q < 27; ++q) M[e * 27 + q] = acc[q];
}

// Moments of larger elements: one block per element, one thread per row of
// cells, warp-shuffle then shared-memory reduction (fixed order).
template <typename Acc>
__global__ void k_moments_block(int ex, int ey, int ze0, int N, const double* __restrict__ w, int Dx,
                                int Dy, Acc* __restrict__ M) {
  __shared__ Acc mu[3][1024];
  __shared__ Acc red[32][27];
  const long e = blockIdx.x;
  const int exi = e % ex, eyi = (e / ex) % ey, ezi = ze0 + (int)(e / ((long)ex * ey));
  const int tid = threadIdx.x;
  fill_mu<Acc>(N, mu[0], mu[1], mu[2]);
  __syncthreads();
  Acc acc[27];
#pragma unroll
  for (int q = 0; q < 27; ++q) acc[q] = 0;
  for (long rr = tid; rr < (long)N * N; rr += blockDim.x) {
    const int b = rr % N, c = rr / N;
    const long rowbase = (N * exi) + (long)Dx * ((N * eyi + b) + (long)Dy * (N * ezi + c));
    row_moments<Acc>(w, rowbase, N, b, c, mu[0], mu[1], mu[2], acc);
  }
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int q = 0; q < 27; ++q) {
    Acc v = acc[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][q] = v;
  }
  __syncthreads();
  if (tid < 27) {
    Acc s = 0;
    for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) s += red[wi][tid];
    M[e * 27 + tid] = s;
  }
}

// K^(e) = (h/2) M_e C for 32 elements per block: C (27 x 300) staged once in
// shared memory, consecutive threads write consecutive entries.
template <typename T, typename Acc>
__global__ void k_moments_to_ke(long E, double h, const Acc* __restrict__ M,
                                const double* __restrict__ cmom, T* __restrict__ Ke) {
  extern __shared__ unsigned char smraw[];
  Acc* cm = (Acc*)smraw;       // 27 * kSym
  Acc* Ms = cm + 27 * kSym;    // 32 * 27
  const long e0 = blockIdx.x * 32L;
  const int ne = (int)min(32L, E - e0);
  for (int t = threadIdx.x; t < 27 * kSym; t += blockDim.x) cm[t] = (Acc)cmom[t];
  for (int t = threadIdx.x; t < ne * 27; t += blockDim.x) Ms[t] = M[e0 * 27 + t];
  __syncthreads();
  const Acc half = (Acc)(0.5 * h);
  for (int o = threadIdx.x; o < ne * kSym; o += blockDim.x) {
    const int q = o / kSym, k = o % kSym;
    const Acc* Mq = Ms + q * 27;
    Acc s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
    for (int a = 0; a < 27; a += 3) {
      s0 += Mq[a] * cm[a * kSym + k];
      s1 += Mq[a + 1] * cm[(a + 1) * kSym + k];
      s2 += Mq[a + 2] * cm[(a + 2) * kSym + k];
    }
    Ke[(e0 + q) * kSym + k] = (T)(half * ((s0 + s1) + s2));
  }
}

// Node-centred assembly of the 27-point block stencil from the element
// matrices around each node (gather, fixed order: deterministic).  One
// thread per (neighbour block o, node), node fastest, so each of its 9
// stores is coalesced.  Fixed DOFs get identity rows and zero columns; the
// centre block also writes the inverse diagonal.
// Nodes of z-layers [l0, l1); Ke holds the elements of layers from ze0 on
// (every element these nodes touch).
template <typename T>
__global__ void k_assemble(int ex, int ey, int ez, int Lx, int Ly, int Lz, int l0, int l1, int ze0,
                           const T* __restrict__ Ke, const uint8_t* __restrict__ mask,
                           T* __restrict__ S, T* __restrict__ dinv) {
  const long nsl = (long)Lx * Ly * (l1 - l0);
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < 27 * nsl;
       t += (long)gridDim.x * blockDim.x) {
    const int o = (int)(t / nsl);
    const long node = t % nsl + (long)Lx * Ly * l0;
    const int i = node % Lx, j = (node / Lx) % Ly, l = node / ((long)Lx * Ly);
    const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
    const int ii = i + dx, jj = j + dy, ll = l + dz;
    const bool valid = ii >= 0 && ii < Lx && jj >= 0 && jj < Ly && ll >= 0 && ll < Lz;
    double acc[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) acc[q] = 0.0;
    if (valid) {
      const int x0 = max(dx == 1 ? i : i - 1, 0), x1 = min(dx == -1 ? i - 1 : i, ex - 1);
      const int y0 = max(dy == 1 ? j : j - 1, 0), y1 = min(dy == -1 ? j - 1 : j, ey - 1);
      const int z0 = max(dz == 1 ? l : l - 1, 0), z1 = min(dz == -1 ? l - 1 : l, ez - 1);
      for (int ez_ = z0; ez_ <= z1; ++ez_)
        for (int ey_ = y0; ey_ <= y1; ++ey_)
          for (int ex_ = x0; ex_ <= x1; ++ex_) {
            const long e = ex_ + (long)ex * (ey_ + (long)ey * (ez_ - ze0));
            const int a = (i - ex_) + 2 * ((j - ey_) + 2 * (l - ez_));
            const int b = (ii - ex_) + 2 * ((jj - ey_) + 2 * (ll - ez_));
            const T* base = Ke + e * kSym;
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
              for (int c = 0; c < 3; ++c) {
                const int R = 3 * a + r, C = 3 * b + c;
                acc[3 * r + c] += (double)base[R <= C ? sym_index(R, C) : sym_index(C, R)];
              }
          }
    }
    const long nb = valid ? node + dx + (long)Lx * (dy + (long)Ly * dz) : node;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const bool fr = mask[3 * node + r] != 0;
        const bool fc = valid ? (mask[3 * nb + c] != 0) : true;
        double v = acc[3 * r + c];
        if (fr || fc) v = (o == 13 && r == c) ? 1.0 : 0.0;
        S[op_idx(node, o * 9 + 3 * r + c)] = (T)v;
        if (o == 13 && r == c) dinv[3 * node + r] = (T)(1.0 / v);
      }
  }
}

__global__ void k_to_fp32(size_t n, const double* __restrict__ a, float* __restrict__ b) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    b[t] = (float)a[t];
}

__global__ void k_coarse_dense(int Lx, int Ly, int Lz, const double* __restrict__ S, double* __restrict__ A) {
  const long nn = (long)Lx * Ly * Lz;
  const long n = 3 * nn;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < nn * 27; t += (long)gridDim.x * blockDim.x) {
    const long node = t % nn;
    const int o = t / nn;
    const int i = node % Lx, j = (node / Lx) % Ly, l = node / ((long)Lx * Ly);
    const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
    const int ii = i + dx, jj = j + dy, ll = l + dz;
    if (ii < 0 || ii >= Lx || jj < 0 || jj >= Ly || ll < 0 || ll >= Lz) continue;
    const long nb = node + dx + (long)Lx * (dy + (long)Ly * dz);
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c)
        A[(3 * node + r) * n + 3 * nb + c] = S[op_idx(node, o * 9 + 3 * r + c)];
  }
}

// The coarsest level's direct solve (Sec. 7.2) as an explicit FP64 inverse,
// formed by blocked symmetric Gauss-Jordan sweeps in one cooperative launch.
// The V-cycle's coarse solve is then one dense matrix-vector product spread
// over many SMs.
//
// Sweeping the pivot block K of a symmetric matrix, with P = A_KK:
//   A_IJ <- A_IJ - A_IK P^{-1} A_KJ   (I, J outside K)
//   A_IK <- A_IK P^{-1},  A_KJ <- P^{-1} A_KJ,  A_KK <- -P^{-1}.
// Sweeping every block in turn leaves -A^{-1}.  The pivot blocks are the
// Schur complements a block Cholesky factorisation meets, so for an SPD
// matrix they are SPD and no pivoting is needed; a non-positive scalar pivot
// sets the status flag (the matrix is not SPD).
//
// FP64 on this part issues one warp instruction per ~64 cycles per SM
// sub-partition with a ~64-cycle dependent latency, and a reciprocal takes
// ~400 cycles, so the launch is latency-bound at coarse sizes of a few
// hundred DOFs, by the chain of scalar pivots.  The pivots of each B x B
// pivot block (B = 16 up to 640 DOFs, else 32) are swept in shared memory
// with two block barriers per pivot, the reciprocal on a warp of its own,
// each entry's update formed while the reciprocal is in flight.  One block
// looks ahead: in each update phase it updates the next pivot block first
// and sweeps it while the other blocks update the rest, so the pivot sweeps
// overlap the updates.  The block-row phase and the update (16x16 tiles of
// the lower triangle, operands staged in shared memory, both halves written
// so the matrix stays exactly symmetric) spread over every SM.  Grid
// barriers: one to symmetrise, two per pivot block.
constexpr int kCT = 16;   // output tile of the update

// Lower-triangle tile index -> (ti, tj) with tj <= ti.
__device__ __forceinline__ void tri_tile(int tile, int& ti, int& tj) {
  int t = 0;
  while ((t + 1) * (t + 2) / 2 <= tile) ++t;
  ti = t;
  tj = tile - t * (t + 1) / 2;
}

// Sweeps the scalar pivots 0..nb-1 of the B x B block p (lower triangle
// current, identity past nb) into -P^{-1}, then mirrors it.  All threads of
// the block call it; the lower-triangle entries sit on warps 0..6 (ei, ek),
// warp 7 forms the reciprocals.
template <int B>
__device__ __forceinline__ void sweep_pivots(double (*p)[B + 1], int nb, const int* ei, const int* ek,
                                             double* rcp, int* status) {
  constexpr int kLow = B * (B + 1) / 2;
  constexpr int kWk = 224;
  constexpr int kM = (kLow + kWk - 1) / kWk;
  const int tid = threadIdx.x;
  for (int j = 0; j < nb; ++j) {
    // Every entry's new value is fma(x, r, y) with r = 1 / p_jj:
    // p_ik - p_ij p_kj r off row and column j, p_ik r on them, -r at the
    // pivot. x and y are formed while the reciprocal is in flight, so the
    // update after the barrier is one FMA per entry and no warp diverges.
    double ux[kM], uy[kM];
#pragma unroll
    for (int m = 0; m < kM; ++m) {
      ux[m] = 0.0;
      uy[m] = 0.0;
      if (ei[m] >= 0) {
        const int i = ei[m], k = ek[m];
        const double pik = p[i][k];
        const double pij = i >= j ? p[i][j] : p[j][i];
        const double pkj = k >= j ? p[k][j] : p[j][k];
        const bool off = i != j && k != j, piv = i == j && k == j;
        ux[m] = off ? -(pij * pkj) : (piv ? -1.0 : pik);
        uy[m] = off ? pik : 0.0;
      }
    }
    if (tid == kWk) {
      double d = p[j][j];
      if (!(d > 0.0)) {
        atomicExch(status, 1);
        d = 1.0;
      }
      *rcp = 1.0 / d;
    }
    __syncthreads();
    const double r = *rcp;
#pragma unroll
    for (int m = 0; m < kM; ++m)
      if (ei[m] >= 0) p[ei[m]][ek[m]] = fma(ux[m], r, uy[m]);
    __syncthreads();
  }
  for (int t = tid; t < B * B; t += blockDim.x) {
    const int i = t / B, k = t % B;
    if (k > i) p[i][k] = p[k][i];
  }
  __syncthreads();
}

template <int B>
__global__ void __launch_bounds__(256) k_coarse_sweep(int n, double* __restrict__ A,
                                                      double* __restrict__ W,
                                                      double* __restrict__ V,
                                                      double* __restrict__ Pg,
                                                      double* __restrict__ Ainv,
                                                      int* __restrict__ status) {
  cg::grid_group grid = cg::this_grid();
  __shared__ double p[B][B + 1];      // -P^{-1} of the current pivot block
  __shared__ double rcp;              // reciprocal of the current scalar pivot
  __shared__ double sa[kCT][B + 1];   // staged W rows (tile i side)
  __shared__ double sb[kCT][B + 1];   // staged V rows (tile j side)
  const int tid = threadIdx.x, bd = blockDim.x;
  const long gtid = blockIdx.x * (long)bd + tid, gstride = (long)gridDim.x * bd;
  const int ty = tid / kCT, tx = tid % kCT;  // 16 x 16 threads
  const int nblk = (n + B - 1) / B;
  const int look = gridDim.x - 1;            // the look-ahead block
  constexpr int kLow = B * (B + 1) / 2;
  constexpr int kWk = 224;
  constexpr int kM = (kLow + kWk - 1) / kWk;
  int ei[kM], ek[kM];
#pragma unroll
  for (int m = 0; m < kM; ++m) {
    const int e = tid + kWk * m;
    ei[m] = -1;
    ek[m] = 0;
    if (tid < kWk && e < kLow) {
      int ii = (int)((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f);
      while ((ii + 1) * (ii + 2) / 2 <= e) ++ii;
      while (ii * (ii + 1) / 2 > e) --ii;
      ei[m] = ii;
      ek[m] = e - ii * (ii + 1) / 2;
    }
  }
  // The operator's lower triangle, mirrored: exactly symmetric from here on.
  for (long t = gtid; t < (long)n * n; t += gstride) {
    const int i = (int)(t / n), j = (int)(t % n);
    if (j > i) A[(size_t)i * n + j] = A[(size_t)j * n + i];
  }
  grid.sync();
  const int nt = (n + kCT - 1) / kCT;
  for (int kb = 0; kb < nblk; ++kb) {
    const int k0 = kb * B, nb = min(B, n - k0);
    // (A) -P^{-1} of this pivot block: swept by every block for the first
    // one, published by the look-ahead block for the others
    if (kb == 0) {
      for (int t = tid; t < B * B; t += bd) {
        const int i = t / B, j = t % B;
        p[i][j] = (i < nb && j < nb) ? A[(size_t)(k0 + i) * n + k0 + j] : (i == j ? 1.0 : 0.0);
      }
      __syncthreads();
      sweep_pivots<B>(p, nb, ei, ek, &rcp, status);
    } else {
      for (int t = tid; t < B * B; t += bd) p[t / B][t % B] = Pg[t];
      __syncthreads();
    }
    // (B) rows I outside K: W_I = A_IK P^{-1} = -A_IK p, V_I = A_IK
    for (long t = gtid; t < (long)(n - nb) * nb; t += gstride) {
      const int ii = (int)(t / nb), c = (int)(t % nb);
      const int i = ii < k0 ? ii : ii + nb;
      const double* Ar = A + (size_t)i * n + k0;
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
      int q = 0;
      for (; q + 3 < nb; q += 4) {
        s0 += Ar[q] * p[q][c];
        s1 += Ar[q + 1] * p[q + 1][c];
        s2 += Ar[q + 2] * p[q + 2][c];
        s3 += Ar[q + 3] * p[q + 3][c];
      }
      for (; q < nb; ++q) s0 += Ar[q] * p[q][c];
      W[(size_t)i * B + c] = -((s0 + s1) + (s2 + s3));
      V[(size_t)i * B + c] = Ar[c];
    }
    grid.sync();
    // (C) the sweep's update over the lower 16x16 tiles, both halves
    // written. The look-ahead block takes the tiles of the next pivot block
    // (rows and columns [k1, k1 + nb1), k1 a multiple of 16), keeps them in
    // shared memory and sweeps them while the others update the rest.
    const bool ahead = kb + 1 < nblk;
    const int k1 = k0 + B, nb1 = ahead ? min(B, n - k1) : 0;
    const int tl0 = k1 / kCT, tl1 = (k1 + nb1 + kCT - 1) / kCT;
    auto tile_update = [&](int ti, int tj, bool keep) {
      const int i0 = ti * kCT, j0 = tj * kCT;
      __syncthreads();
      for (int t = tid; t < kCT * B; t += bd) {
        const int r = t / B, q = t % B;
        const int gi = i0 + r, gj = j0 + r;
        sa[r][q] = (gi < n && q < nb && (gi < k0 || gi >= k0 + nb)) ? W[(size_t)gi * B + q] : 0.0;
        sb[r][q] = (gj < n && q < nb && (gj < k0 || gj >= k0 + nb)) ? V[(size_t)gj * B + q] : 0.0;
      }
      __syncthreads();
      const int i = i0 + ty, j = j0 + tx;
      if (i < n && j < n && (ti != tj || j <= i)) {
        const bool iK = i >= k0 && i < k0 + nb, jK = j >= k0 && j < k0 + nb;
        double v;
        if (!iK && !jK) {
          double s0 = 0.0, s1 = 0.0;
#pragma unroll
          for (int q = 0; q < B; q += 2) {
            s0 += sa[ty][q] * sb[tx][q];
            s1 += sa[ty][q + 1] * sb[tx][q + 1];
          }
          v = A[(size_t)i * n + j] - (s0 + s1);
        } else if (!iK) {
          v = sa[ty][j - k0];                    // A_IK <- W_I
        } else if (!jK) {
          v = W[(size_t)j * B + (i - k0)];       // A_KJ <- W_J^T
        } else {
          v = p[i - k0][j - k0];                 // A_KK <- -P^{-1}
        }
        A[(size_t)i * n + j] = v;
        if (i != j) A[(size_t)j * n + i] = v;
        if (keep) {                              // entries of the next pivot block
          p[i - k1][j - k1] = v;
          p[j - k1][i - k1] = v;
        }
      }
    };
    if (ahead && blockIdx.x == look) {
      // the next block's tiles lie outside K, so they never read p: it is
      // reused for P_{k+1}
      __syncthreads();
      for (int t = tid; t < B * B; t += bd) {
        const int i = t / B, j = t % B;
        if (i >= nb1 || j >= nb1) p[i][j] = (i == j ? 1.0 : 0.0);
      }
      for (int ti = tl0; ti < tl1; ++ti)
        for (int tj = tl0; tj <= ti; ++tj) tile_update(ti, tj, true);
      __syncthreads();
      sweep_pivots<B>(p, nb1, ei, ek, &rcp, status);
      for (int t = tid; t < B * B; t += bd) Pg[t] = p[t / B][t % B];
    } else {
      const int workers = ahead ? gridDim.x - 1 : gridDim.x;
      for (int tile = blockIdx.x; tile < nt * (nt + 1) / 2; tile += workers) {
        int ti, tj;
        tri_tile(tile, ti, tj);
        if (ahead && ti >= tl0 && ti < tl1 && tj >= tl0 && tj < tl1) continue;
        tile_update(ti, tj, false);
      }
    }
    grid.sync();
  }
  for (long t = gtid; t < (long)n * n; t += gstride) Ainv[t] = -A[t];
}

// Pivot block of the coarse sweeps for an n x n coarse operator.
inline int coarse_pivot_block(int n) { return n <= 640 ? 16 : 32; }

inline int grid_for(long n, int bs = kBS, int cap = 4096) {
  long g = (n + bs - 1) / bs;
  if (g < 1) g = 1;
  return (int)(g < cap ? g : cap);
}

}  // namespace

void launch_subcell_table(int n, double nu, double h, double* tab, cudaStream_t st) {
  k_subcell_table<<<n * n * n, 256, 0, st>>>(n, nu, h, tab);
}

void launch_symmetrize(int m, const double* tab, double* tabsym, cudaStream_t st) {
  k_symmetrize<<<m, 256, 0, st>>>(m, tab, tabsym);
}

void launch_moment_basis(double nu, double* cmom, cudaStream_t st) {
  k_moment_basis<<<(27 * kSym + 255) / 256, 256, 0, st>>>(nu, cmom);
}

void launch_filter_init(int Dx, int Dy, int Dz, int noff, const int4* off, const double* wgt,
                        double* invom, cudaStream_t st) {
  k_filter_init<<<grid_for((long)Dx * Dy * Dz), kBS, 0, st>>>(Dx, Dy, Dz, noff, off, wgt, invom);
}

void launch_proj_init(const ProjGrid& P, double* invom, cudaStream_t st) {
  k_proj_init<<<grid_for((long)P.Dx * P.Dy * P.Dz), kBS, 0, st>>>(P, invom);
}

void launch_proj_fwd(const ProjGrid& P, const double* invom, const double* x, double Emin, double dE,
                     double penal, double* rho, double* w, cudaStream_t st) {
  k_proj_fwd<<<grid_for((long)P.Dx * P.Dy * P.Dz), kBS, 0, st>>>(P, invom, x, Emin, dE, penal, rho, w);
}

void launch_filter_fwd(int Dx, int Dy, int Dz, int noff, const int4* off, const double* wgt,
                       const double* invom, const double* x, double Emin, double dE,
                       double penal, double* rho, double* w, cudaStream_t st) {
  k_filter_fwd<<<grid_for((long)Dx * Dy * Dz), kBS, 0, st>>>(Dx, Dy, Dz, noff, off, wgt, invom, x,
                                                             Emin, dE, penal, rho, w);
}

void launch_elem_direct(bool fp64, const Level& L, int ze0, int ze1, int n, const double* w, int Dx,
                        int Dy, const double* tabsym, void* Ke, cudaStream_t st) {
  const long E = (long)L.ex * L.ey * (ze1 - ze0);
  const int m = n * n * n;
  int epb = 4096 / m;
  if (epb > 32) epb = 32;
  if (epb < 1) epb = 1;
  const long g = (E + epb - 1) / epb;
  const size_t sm = (size_t)epb * m * sizeof(double);
  if (fp64)
    k_elem_direct<double><<<g, 256, sm, st>>>(L.ex, L.ey, ze0, ze1 - ze0, n, epb, w, Dx, Dy, tabsym,
                                              (double*)Ke);
  else
    k_elem_direct<float><<<g, 256, sm, st>>>(L.ex, L.ey, ze0, ze1 - ze0, n, epb, w, Dx, Dy, tabsym,
                                             (float*)Ke);
}

void launch_elem_moments(bool fp64, const Level& L, int ze0, int ze1, const double* w, int Dx, int Dy,
                         const double* cmom, void* Mscr, void* Ke, cudaStream_t st) {
  const long E = (long)L.ex * L.ey * (ze1 - ze0);
  const int N = L.nsub;
  const long gk = (E + 31) / 32;
  if (fp64) {
    double* M = (double*)Mscr;
    if (N <= 4)
      k_moments_thread<double><<<(E + 127) / 128, 128, 0, st>>>(L.ex, L.ey, ze0, ze1 - ze0, N, w, Dx,
                                                                Dy, M);
    else
      k_moments_block<double><<<E, N * N >= 256 ? 256 : 64, 0, st>>>(L.ex, L.ey, ze0, N, w, Dx, Dy, M);
    const size_t sm = (size_t)(27 * kSym + 32 * 27) * sizeof(double);
    static std::once_flag attr;  // handles may be created from several threads
    std::call_once(attr, [sm] {
      cudaFuncSetAttribute(k_moments_to_ke<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sm);
    });
    k_moments_to_ke<double, double><<<gk, 256, sm, st>>>(E, L.h, M, cmom, (double*)Ke);
  } else {
    float* M = (float*)Mscr;
    if (N <= 4)
      k_moments_thread<float><<<(E + 127) / 128, 128, 0, st>>>(L.ex, L.ey, ze0, ze1 - ze0, N, w, Dx,
                                                               Dy, M);
    else
      k_moments_block<float><<<E, N * N >= 256 ? 256 : 64, 0, st>>>(L.ex, L.ey, ze0, N, w, Dx, Dy, M);
    const size_t sm = (size_t)(27 * kSym + 32 * 27) * sizeof(float);
    static std::once_flag attr;  // handles may be created from several threads
    std::call_once(attr, [sm] {
      cudaFuncSetAttribute(k_moments_to_ke<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sm);
    });
    k_moments_to_ke<float, float><<<gk, 256, sm, st>>>(E, L.h, M, cmom, (float*)Ke);
  }
}

void launch_assemble(bool fp64, const Level& L, int l0, int l1, int ze0, const void* Ke, void* S,
                     void* dinv, cudaStream_t st) {
  const int g = grid_for((long)L.Lx * L.Ly * (l1 - l0) * 27, 128, 65536);
  if (fp64)
    k_assemble<double><<<g, 128, 0, st>>>(L.ex, L.ey, L.ez, L.Lx, L.Ly, L.Lz, l0, l1, ze0,
                                          (const double*)Ke, L.mask, (double*)S, (double*)dinv);
  else
    k_assemble<float><<<g, 128, 0, st>>>(L.ex, L.ey, L.ez, L.Lx, L.Ly, L.Lz, l0, l1, ze0,
                                         (const float*)Ke, L.mask, (float*)S, (float*)dinv);
}

void for_each_slab(const Level& L, size_t scratch_bytes, size_t elem_bytes,
                   const std::function<void(int, int, int, int)>& fn) {
  const size_t layer = (size_t)L.ex * L.ey * elem_bytes;
  int C = L.Lz;  // node layers per slab
  if ((size_t)L.ez * layer > scratch_bytes) {
    const size_t fit = scratch_bytes / layer;  // element layers that fit
    C = fit >= 2 ? (int)(fit - 1) : 1;
  }
  for (int l0 = 0; l0 < L.Lz; l0 += C) {
    const int l1 = std::min(l0 + C, L.Lz);
    const int ze0 = std::max(l0 - 1, 0), ze1 = std::min(l1, L.ez);
    fn(l0, l1, ze0, ze1);
  }
}

void launch_to_fp32(size_t n, const double* a, float* b, cudaStream_t st) {
  k_to_fp32<<<grid_for((long)n), kBS, 0, st>>>(n, a, b);
}

void launch_coarse_dense(const Level& L, double* A, cudaStream_t st) {
  k_coarse_dense<<<grid_for((long)L.nn * 27), kBS, 0, st>>>(L.Lx, L.Ly, L.Lz, L.S64, A);
}

int coarse_sweep_grid() {
  int dev = 0, sms = 0, per16 = 0, per32 = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per16, k_coarse_sweep<16>, 256, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per32, k_coarse_sweep<32>, 256, 0);
  // one block per SM (co-resident as long as one block fits, checked here)
  if (per16 < 1 || per32 < 1) return 0;
  return sms;
}

cudaError_t launch_coarse_invert(int n, double* A, double* W, double* V, double* Pg, double* Ainv,
                                 int* status, int grid, cudaStream_t st) {
  if (grid < 2) return cudaErrorInvalidConfiguration;  // one block looks ahead
  void* args[] = {&n, &A, &W, &V, &Pg, &Ainv, &status};
  void* fn = coarse_pivot_block(n) == 16 ? (void*)k_coarse_sweep<16> : (void*)k_coarse_sweep<32>;
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(256), args, 0, st);
}

}  // namespace tos
