// Triquadratic (Lagrange degree 2) elements: every step of the path for
// k = 2, in element form.
//
// The level operators of a degree-2 hierarchy are kept as element matrices
// K^(e) (81 x 81, full, FP64 and optionally an FP32 copy) instead of node
// stencils: a degree-2 node couples to up to 125 lattice nodes, and on this
// GPU the element form reads fewer bytes per apply than that stencil would.
// An apply is two kernels: Y_e = K^(e) u_e for every element (u gathered
// with the fixed DOFs zeroed), then a node gather y_n = sum of the Y_e of the
// elements containing n (fixed order: deterministic), with identity rows at
// fixed DOFs.  The gather also finishes the multigrid smoothing steps.
//
// Element conventions: reference [-1,1]^3, K = 3 equispaced nodes per axis,
// local node a = ax + 3 (ay + 3 az) at lattice node (2 ex + ax, 2 ey + ay,
// 2 ez + az), DOF 3a + c.  Sec. 2.1 (Lagrange elements), Sec. 3.3
// (Eq. matrixK_mr: K^(e) = sum_i w_i K^(e_i) over the element's n^3
// subcells), Sec. 2.3 (linear interpolation between node lattices).
#include <mutex>
#include <type_traits>

#include "internal.cuh"

namespace tos {
namespace {

constexpr int kK = 3;               // nodes per axis
constexpr int kNE = kK * kK * kK;   // 27 nodes
constexpr int kD = 3 * kNE;         // 81 DOFs
constexpr int kDD = kD * kD;        // 6561
constexpr int kP = 2 * kK - 1;      // 5 monomial powers per axis
constexpr int kNM = kP * kP * kP;   // 125 moments

// An element of degree K (2 or 3) on its node lattice: K + 1 nodes per axis.
// The degree-3 element appears only on the finest level of a hierarchy,
// whose next level is the degree-2 mesh of the same elements.
template <int K>
struct Deg {
  static constexpr int NA = K + 1;
  static constexpr int NE = NA * NA * NA;
  static constexpr int D = 3 * NE;
  static constexpr int DD = D * D;
  static constexpr int TB = (D + 31) / 32 * 32;  // threads of the element apply
};

// 1D Lagrange basis on the nodes -1, 0, 1: value and derivative of basis j.
__host__ __device__ __forceinline__ double lag(int j, double x) {
  return j == 0 ? 0.5 * x * (x - 1.0) : (j == 1 ? 1.0 - x * x : 0.5 * x * (x + 1.0));
}
__host__ __device__ __forceinline__ double dlag(int j, double x) {
  return j == 0 ? x - 0.5 : (j == 1 ? -2.0 * x : x + 0.5);
}
// Monomial coefficients (degree <= 2) of the basis (deriv = 0) or its
// derivative (deriv = 1).
__device__ __forceinline__ void lag_coef(int j, int deriv, double c[3]) {
  if (!deriv) {
    if (j == 0) { c[0] = 0.0; c[1] = -0.5; c[2] = 0.5; }
    else if (j == 1) { c[0] = 1.0; c[1] = 0.0; c[2] = -1.0; }
    else { c[0] = 0.0; c[1] = 0.5; c[2] = 0.5; }
  } else {
    if (j == 0) { c[0] = -0.5; c[1] = 1.0; c[2] = 0.0; }
    else if (j == 1) { c[0] = 0.0; c[1] = -2.0; c[2] = 0.0; }
    else { c[0] = 0.5; c[1] = 1.0; c[2] = 0.0; }
  }
}

// Reference gradient of the 20-node serendipity shape function at lattice
// position (ax, ay, az) in 0..2 (Sec. 2.1): a vertex has
// N = (1 + x c_x)(1 + y c_y)(1 + z c_z)(x c_x + y c_y + z c_z - 2) / 8, an
// edge midpoint (one coordinate c = 0) N = (1 - t^2)(1 + ...)(1 + ...) / 4;
// face and element centres have no node (zero).
__device__ __forceinline__ void s2_grad(int ax, int ay, int az, double x, double y, double z, double g[3]) {
  const int c[3] = {ax - 1, ay - 1, az - 1};
  const double p[3] = {x, y, z};
  const int nmid = (c[0] == 0) + (c[1] == 0) + (c[2] == 0);
  g[0] = g[1] = g[2] = 0.0;
  if (nmid == 0) {
    double f[3];
    for (int q = 0; q < 3; ++q) f[q] = 1.0 + p[q] * c[q];
    const double sv = p[0] * c[0] + p[1] * c[1] + p[2] * c[2] - 2.0;
    const double prod = f[0] * f[1] * f[2];
    for (int q = 0; q < 3; ++q) {
      const double others = q == 0 ? f[1] * f[2] : (q == 1 ? f[0] * f[2] : f[0] * f[1]);
      g[q] = (c[q] * others * sv + prod * c[q]) * 0.125;
    }
  } else if (nmid == 1) {
    double f[3], df[3];
    for (int q = 0; q < 3; ++q) {
      if (c[q] == 0) { f[q] = 1.0 - p[q] * p[q]; df[q] = -2.0 * p[q]; }
      else { f[q] = 1.0 + p[q] * c[q]; df[q] = c[q]; }
    }
    g[0] = df[0] * f[1] * f[2] * 0.25;
    g[1] = f[0] * df[1] * f[2] * 0.25;
    g[2] = f[0] * f[1] * df[2] * 0.25;
  }
}

// K^(e_i) for the n^3 subcells of an element of edge h (E = 1), full 81 x 81:
// 3-point Gauss-Legendre per axis in each subcell (exact: the integrand has
// degree <= 4 per axis, for both element families).  One block per subcell.
// family 1: the serendipity element (zero rows and columns at the face and
// element centres).
__global__ void k_q2_subcell_table(int n, double nu, double h, int family, double* __restrict__ tab) {
  __shared__ double gr[27][kNE][3];  // physical gradients at the 27 points
  const int sub = blockIdx.x;
  const int sa = sub % n, sb = (sub / n) % n, sc = sub / (n * n);
  const double half = 1.0 / n;
  const double gp[3] = {-sqrt(0.6), 0.0, sqrt(0.6)};
  const double gw[3] = {5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0};
  const double s = 2.0 / h;
  for (int t = threadIdx.x; t < 27 * kNE; t += blockDim.x) {
    const int q = t / kNE, a = t % kNE;
    const int qx = q % 3, qy = (q / 3) % 3, qz = q / 9;
    const double xi = -1.0 + (2 * sa + 1) * half + half * gp[qx];
    const double eta = -1.0 + (2 * sb + 1) * half + half * gp[qy];
    const double zeta = -1.0 + (2 * sc + 1) * half + half * gp[qz];
    const int ax = a % 3, ay = (a / 3) % 3, az = a / 9;
    if (family == 1) {
      double g[3];
      s2_grad(ax, ay, az, xi, eta, zeta, g);
      gr[q][a][0] = s * g[0];
      gr[q][a][1] = s * g[1];
      gr[q][a][2] = s * g[2];
    } else {
      gr[q][a][0] = s * dlag(ax, xi) * lag(ay, eta) * lag(az, zeta);
      gr[q][a][1] = s * lag(ax, xi) * dlag(ay, eta) * lag(az, zeta);
      gr[q][a][2] = s * lag(ax, xi) * lag(ay, eta) * dlag(az, zeta);
    }
  }
  __syncthreads();
  const double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  const double mu = 1.0 / (2.0 * (1.0 + nu));
  // dx = (h/2)^3 dxi, and the subcell maps onto xi with factor 1/n per axis
  const double jac = half * half * half * (0.125 * h * h * h);
  for (int t = threadIdx.x; t < kDD; t += blockDim.x) {
    const int R = t / kD, C = t % kD;
    const int a = R / 3, i = R % 3, b = C / 3, j = C % 3;
    double acc = 0.0;
    for (int q = 0; q < 27; ++q) {
      const double wq = gw[q % 3] * gw[(q / 3) % 3] * gw[q / 9];
      const double* ga = gr[q][a];
      const double* gb = gr[q][b];
      double v = lam * ga[i] * gb[j] + mu * ga[j] * gb[i];
      if (i == j) v += mu * (ga[0] * gb[0] + ga[1] * gb[1] + ga[2] * gb[2]);
      acc += wq * v;
    }
    tab[(size_t)sub * kDD + t] = jac * acc;
  }
}

// Degree 3 (the finest level only).  1D cubic Lagrange basis on the nodes
// -1, -1/3, 1/3, 1 and its derivative (product form).
__device__ __forceinline__ double lag3(int j, double x) {
  double v = 1.0;
  const double xj = -1.0 + 2.0 * j / 3.0;
  for (int m = 0; m < 4; ++m)
    if (m != j) {
      const double xm = -1.0 + 2.0 * m / 3.0;
      v *= (x - xm) / (xj - xm);
    }
  return v;
}
__device__ __forceinline__ double dlag3(int j, double x) {
  const double xj = -1.0 + 2.0 * j / 3.0;
  double s = 0.0;
  for (int q = 0; q < 4; ++q) {
    if (q == j) continue;
    double v = 1.0 / (xj - (-1.0 + 2.0 * q / 3.0));
    for (int m = 0; m < 4; ++m)
      if (m != j && m != q) {
        const double xm = -1.0 + 2.0 * m / 3.0;
        v *= (x - xm) / (xj - xm);
      }
    s += v;
  }
  return s;
}

// Reference gradient of the 32-node serendipity shape function at lattice
// position (ax, ay, az) in 0..3 (positions -1, -1/3, 1/3, 1): a vertex has
// N = (1 + x c_x)(1 + y c_y)(1 + z c_z)(9 (x^2 + y^2 + z^2) - 19) / 64, an
// edge node with interior coordinate c = +-1/3 along axis m
// N = 9 (1 - t^2)(1 + 9 t c)(1 + ...)(1 + ...) / 64; positions with two or
// three interior coordinates have no node.
__device__ void s3_grad(int ax, int ay, int az, double x, double y, double z, double g[3]) {
  const int ix[3] = {ax, ay, az};
  const double p[3] = {x, y, z};
  double c[3];
  int inner = 0, m = 0;
  for (int q = 0; q < 3; ++q) {
    c[q] = -1.0 + 2.0 * ix[q] / 3.0;
    if (ix[q] == 1 || ix[q] == 2) { ++inner; m = q; }
  }
  g[0] = g[1] = g[2] = 0.0;
  if (inner == 0) {
    double f[3];
    for (int q = 0; q < 3; ++q) f[q] = 1.0 + p[q] * c[q];
    const double sv = 9.0 * (p[0] * p[0] + p[1] * p[1] + p[2] * p[2]) - 19.0;
    const double prod = f[0] * f[1] * f[2];
    for (int q = 0; q < 3; ++q) {
      const double others = q == 0 ? f[1] * f[2] : (q == 1 ? f[0] * f[2] : f[0] * f[1]);
      g[q] = (c[q] * others * sv + prod * 18.0 * p[q]) / 64.0;
    }
  } else if (inner == 1) {
    double f[3], df[3];
    for (int q = 0; q < 3; ++q) {
      if (q == m) {
        f[q] = (1.0 - p[q] * p[q]) * (1.0 + 9.0 * p[q] * c[q]);
        df[q] = -2.0 * p[q] * (1.0 + 9.0 * p[q] * c[q]) + (1.0 - p[q] * p[q]) * 9.0 * c[q];
      } else {
        f[q] = 1.0 + p[q] * c[q];
        df[q] = c[q];
      }
    }
    g[0] = 9.0 * df[0] * f[1] * f[2] / 64.0;
    g[1] = 9.0 * f[0] * df[1] * f[2] / 64.0;
    g[2] = 9.0 * f[0] * f[1] * df[2] / 64.0;
  }
}

// Physical gradients of the 64 degree-3 shape functions at the 4^3
// Gauss-Legendre points of every subcell: gr[((sub * 64 + q) * 64 + a) * 3 + i].
__global__ void k_q3_grads(int n, double h, int family, double* __restrict__ gr) {
  const double gp[4] = {-0.8611363115940526, -0.3399810435848563, 0.3399810435848563, 0.8611363115940526};
  const long total = (long)n * n * n * 64 * 64;
  const double half = 1.0 / n, s = 2.0 / h;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const int a = t % 64, q = (t / 64) % 64;
    const int sub = (int)(t / (64 * 64));
    const int sa = sub % n, sb = (sub / n) % n, sc = sub / (n * n);
    const double xi = -1.0 + (2 * sa + 1) * half + half * gp[q % 4];
    const double eta = -1.0 + (2 * sb + 1) * half + half * gp[(q / 4) % 4];
    const double zeta = -1.0 + (2 * sc + 1) * half + half * gp[q / 16];
    const int ax = a % 4, ay = (a / 4) % 4, az = a / 16;
    double g[3];
    if (family == 1) {
      s3_grad(ax, ay, az, xi, eta, zeta, g);
    } else {
      g[0] = dlag3(ax, xi) * lag3(ay, eta) * lag3(az, zeta);
      g[1] = lag3(ax, xi) * dlag3(ay, eta) * lag3(az, zeta);
      g[2] = lag3(ax, xi) * lag3(ay, eta) * dlag3(az, zeta);
    }
    for (int i = 0; i < 3; ++i) gr[t * 3 + i] = s * g[i];
  }
}

// K^(e_i), 192 x 192, from the gradients: 4-point Gauss-Legendre per axis
// and subcell (exact for the integrand's degree <= 6 per axis).
__global__ void k_q3_subcell_table(int n, double nu, double h, const double* __restrict__ gr,
                                   double* __restrict__ tab) {
  constexpr int kD3 = Deg<3>::D, kDD3 = Deg<3>::DD;
  const double gw[4] = {0.3478548451374538, 0.6521451548625461, 0.6521451548625461, 0.3478548451374538};
  const double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  const double mu = 1.0 / (2.0 * (1.0 + nu));
  const double half = 1.0 / n;
  const double jac = half * half * half * (0.125 * h * h * h);
  const long total = (long)n * n * n * kDD3;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const int sub = (int)(t / kDD3), ent = (int)(t % kDD3);
    const int R = ent / kD3, C = ent % kD3;
    const int a = R / 3, i = R % 3, b = C / 3, j = C % 3;
    double acc = 0.0;
    for (int q = 0; q < 64; ++q) {
      const double wq = gw[q % 4] * gw[(q / 4) % 4] * gw[q / 16];
      const double* ga = gr + ((size_t)(sub * 64 + q) * 64 + a) * 3;
      const double* gb = gr + ((size_t)(sub * 64 + q) * 64 + b) * 3;
      double v = lam * ga[i] * gb[j] + mu * ga[j] * gb[i];
      if (i == j) v += mu * (ga[0] * gb[0] + ga[1] * gb[1] + ga[2] * gb[2]);
      acc += wq * v;
    }
    tab[t] = jac * acc;
  }
}

// Moment basis: the element-matrix integrand in reference coordinates is
// sum_alpha C_alpha xi^alpha (alpha in {0..4}^3), so an element of edge h
// with cellwise-constant weights w has K^(e) = (h/2) sum_alpha M_alpha
// C_alpha, M_alpha = int_ref w(xi) xi^alpha dxi.  Thread per (alpha, entry).
__global__ void k_q2_moment_basis(double nu, double* __restrict__ cmom) {
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t >= (long)kNM * kDD) return;
  const int alpha = (int)(t / kDD), e = (int)(t % kDD);
  const int R = e / kD, C = e % kD;
  const int al[3] = {alpha % kP, (alpha / kP) % kP, alpha / (kP * kP)};
  const int a = R / 3, i = R % 3, b = C / 3, j = C % 3;
  const int na[3] = {a % 3, (a / 3) % 3, a / 9};
  const int nb[3] = {b % 3, (b / 3) % 3, b / 9};
  auto T = [&](int p, int q) {  // coefficient of xi^alpha in d_p N_a * d_q N_b
    double v = 1.0;
    for (int ax = 0; ax < 3; ++ax) {
      double u[3], w[3];
      lag_coef(na[ax], p == ax, u);
      lag_coef(nb[ax], q == ax, w);
      double c = 0.0;
      for (int r = 0; r < 3; ++r) {
        const int s = al[ax] - r;
        if (s >= 0 && s < 3) c += u[r] * w[s];
      }
      v *= c;
    }
    return v;
  };
  const double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  const double mu = 1.0 / (2.0 * (1.0 + nu));
  double v = lam * T(i, j) + mu * T(j, i);
  if (i == j) v += mu * (T(0, 0) + T(1, 1) + T(2, 2));
  cmom[t] = v;
}

// Monomial coefficients of the 20-node serendipity shape function at lattice
// position (ax, ay, az): c[e0 + 3 (e1 + 3 e2)] multiplies xi^e0 eta^e1
// zeta^e2 (each exponent <= 2); zero for face and element centres.
__device__ void s2_coef(int ax, int ay, int az, double c[27]) {
  for (int q = 0; q < 27; ++q) c[q] = 0.0;
  const int cc[3] = {ax - 1, ay - 1, az - 1};
  const int nmid = (cc[0] == 0) + (cc[1] == 0) + (cc[2] == 0);
  if (nmid >= 2) return;
  // 1D factors: (1 + c t) for a vertex coordinate, (1 - t^2) for the
  // midpoint coordinate of an edge node
  double f[3][3];
  for (int q = 0; q < 3; ++q) {
    if (cc[q] == 0) { f[q][0] = 1.0; f[q][1] = 0.0; f[q][2] = -1.0; }
    else { f[q][0] = 1.0; f[q][1] = (double)cc[q]; f[q][2] = 0.0; }
  }
  double prod[27];
  for (int e2 = 0; e2 < 3; ++e2)
    for (int e1 = 0; e1 < 3; ++e1)
      for (int e0 = 0; e0 < 3; ++e0) prod[e0 + 3 * (e1 + 3 * e2)] = f[0][e0] * f[1][e1] * f[2][e2];
  if (nmid == 1) {
    for (int q = 0; q < 27; ++q) c[q] = 0.25 * prod[q];
    return;
  }
  // vertex: times (c0 xi + c1 eta + c2 zeta - 2) / 8; (1 + c t) t = t + c t^2
  // keeps every exponent <= 2
  for (int e2 = 0; e2 < 3; ++e2)
    for (int e1 = 0; e1 < 3; ++e1)
      for (int e0 = 0; e0 < 3; ++e0) {
        const double v = prod[e0 + 3 * (e1 + 3 * e2)];
        if (v == 0.0) continue;
        c[e0 + 3 * (e1 + 3 * e2)] += -2.0 * v / 8.0;
        const int ee[3] = {e0, e1, e2};
        for (int q = 0; q < 3; ++q) {
          int up[3] = {ee[0], ee[1], ee[2]};
          up[q] += 1;
          if (up[q] <= 2) c[up[0] + 3 * (up[1] + 3 * up[2])] += cc[q] * v / 8.0;
        }
      }
}

// The moment basis of the serendipity element (as k_q2_moment_basis): the
// coefficient of xi^alpha in d_p N_a d_q N_b is a 3D convolution of the
// derivatives' coefficient arrays.  Thread per (alpha, entry).
__global__ void k_s2_moment_basis(double nu, double* __restrict__ cmom) {
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t >= (long)kNM * kDD) return;
  const int alpha = (int)(t / kDD), e = (int)(t % kDD);
  const int R = e / kD, C = e % kD;
  const int al[3] = {alpha % kP, (alpha / kP) % kP, alpha / (kP * kP)};
  const int a = R / 3, i = R % 3, b = C / 3, j = C % 3;
  double ca[27], cb[27];
  s2_coef(a % 3, (a / 3) % 3, a / 9, ca);
  s2_coef(b % 3, (b / 3) % 3, b / 9, cb);
  auto deriv = [](const double* c, int p, int e0, int e1, int e2) {  // coefficient of t^e in d_p N
    int ee[3] = {e0, e1, e2};
    ee[p] += 1;
    if (ee[p] > 2) return 0.0;
    return ee[p] * c[ee[0] + 3 * (ee[1] + 3 * ee[2])];
  };
  auto T = [&](int p, int q) {
    double v = 0.0;
    for (int x0 = 0; x0 <= 1 + (p != 0); ++x0) {
      const int y0 = al[0] - x0;
      if (y0 < 0 || y0 > 2) continue;
      for (int x1 = 0; x1 <= 2; ++x1) {
        const int y1 = al[1] - x1;
        if (y1 < 0 || y1 > 2) continue;
        for (int x2 = 0; x2 <= 2; ++x2) {
          const int y2 = al[2] - x2;
          if (y2 < 0 || y2 > 2) continue;
          v += deriv(ca, p, x0, x1, x2) * deriv(cb, q, y0, y1, y2);
        }
      }
    }
    return v;
  };
  const double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  const double mu = 1.0 / (2.0 * (1.0 + nu));
  double v = lam * T(i, j) + mu * T(j, i);
  if (i == j) v += mu * (T(0, 0) + T(1, 1) + T(2, 2));
  cmom[t] = v;
}

// mu_p(a) = integral of xi^p over the a-th of N equal intervals of [-1, 1].
__device__ __forceinline__ double mono_int(int p, int a, int N) {
  const double t0 = -1.0 + 2.0 * a / N, t1 = -1.0 + 2.0 * (a + 1) / N;
  double p0 = t0, p1 = t1;
  for (int k = 0; k < p; ++k) { p0 *= t0; p1 *= t1; }
  return (p1 - p0) / (p + 1);
}

// Moments M_alpha (125) of the weights over each element of a coarse
// degree-2 level (N^3 density cells per element), separably: for each row of
// cells along x the five sums sum_a w mu_p(a), then products with mu_q(b)
// mu_r(c).  One block per element, threads over rows, fixed-order
// reduction.
__global__ void k_q2_moments(int ex, int ey, int N, const double* __restrict__ w, int Dx, int Dy,
                             double* __restrict__ M) {
  __shared__ double red[kNM];
  const long e = blockIdx.x;
  const int exi = e % ex, eyi = (e / ex) % ey, ezi = e / ((long)ex * ey);
  for (int q = threadIdx.x; q < kNM; q += blockDim.x) red[q] = 0.0;
  __syncthreads();
  // rows handled in a fixed order by a fixed thread; partial sums per thread
  double acc[kNM];
  for (int q = 0; q < kNM; ++q) acc[q] = 0.0;
  for (long rr = threadIdx.x; rr < (long)N * N; rr += blockDim.x) {
    const int b = rr % N, c = rr / N;
    const long base = (N * exi) + (long)Dx * ((N * eyi + b) + (long)Dy * (N * ezi + c));
    double sx[kP] = {0, 0, 0, 0, 0};
    for (int a = 0; a < N; ++a) {
      const double wv = w[base + a];
      for (int p = 0; p < kP; ++p) sx[p] += wv * mono_int(p, a, N);
    }
    double my[kP], mz[kP];
    for (int p = 0; p < kP; ++p) { my[p] = mono_int(p, b, N); mz[p] = mono_int(p, c, N); }
    for (int q = 0; q < kNM; ++q) acc[q] += sx[q % kP] * my[(q / kP) % kP] * mz[q / (kP * kP)];
  }
  // fixed-order combination: thread t adds its partials in turn
  for (int t = 0; t < (int)blockDim.x; ++t) {
    if ((int)threadIdx.x == t)
      for (int q = 0; q < kNM; ++q) red[q] += acc[q];
    __syncthreads();
  }
  for (int q = threadIdx.x; q < kNM; q += blockDim.x) M[e * kNM + q] = red[q];
}

template <int K>
__device__ __forceinline__ long elem_node_k(int exi, int eyi, int ezi, int a, int Lx, int Ly) {
  constexpr int NA = K + 1;
  return (K * exi + a % NA) + (long)Lx * ((K * eyi + (a / NA) % NA) + (long)Ly * (K * ezi + a / (NA * NA)));
}
__device__ __forceinline__ long elem_node(int exi, int eyi, int ezi, int a, int Lx, int Ly) {
  return elem_node_k<2>(exi, eyi, ezi, a, Lx, Ly);
}

// Parent vertices of local node a of a 27-node element (the corners of the
// edge, face or cell whose midpoint a is), as a table in constant memory
// (read uniformly by a warp).
struct ParentTab {
  signed char p[27][8];
  unsigned char n[27];
};
constexpr ParentTab make_parent_tab() {
  ParentTab t{};
  for (int a = 0; a < 27; ++a) {
    const int ax = a % 3, ay = (a / 3) % 3, az = a / 9;
    const int nx = ax == 1 ? 2 : 1, ny = ay == 1 ? 2 : 1, nz = az == 1 ? 2 : 1;
    int k = 0;
    for (int c = 0; c < nz; ++c)
      for (int b = 0; b < ny; ++b)
        for (int q = 0; q < nx; ++q) {
          const int px = ax == 1 ? 2 * q : ax, py = ay == 1 ? 2 * b : ay, pz = az == 1 ? 2 * c : az;
          t.p[a][k++] = (signed char)(px + 3 * (py + 3 * pz));
        }
    t.n[a] = (unsigned char)k;
  }
  return t;
}
__constant__ ParentTab c_parents = make_parent_tab();

// Element matrices of a Lagrange degree-2 level by sum factorisation (any
// level: the element covers N^3 density cells of constant weight).  With
// N_a(xi) = phi_ax(xi) phi_ay(eta) phi_az(zeta), the entries of Eq.
// matrixK_mr are
//   K[(a,i),(b,j)] = (h/2) (lam F^ij_ab + mu F^ji_ab + mu delta_ij sum_s F^ss_ab),
//   F^st_ab = int_ref w d_s N_a d_t N_b = sum_alpha M_alpha prod_d c_d(alpha_d)[a_d][b_d],
// where M_alpha (alpha in {0..4}^3) are the moments of w over the reference
// element and c_d(p)[x][y] is the coefficient of xi^p in phi_x^(m) phi_y^(n)
// with m = [s = d], n = [t = d] (Sec. 2.1; the same polynomial identity as
// the moment basis, but contracted one axis at a time).  Per element: the
// moments by z-slices of cells (x, then y, then accumulated over z in a
// fixed order), then for the six pairs s <= t the contractions over
// alpha_z, alpha_y, alpha_x, then the 81 x 81 assembly (F^ts_ab = F^st_ba).
// About 6.5e4 FMAs per element instead of 27 x 6561 (subcell sum) or
// 125 x 6561 (moment basis).  Only the moments are formed in FP64: FP64
// issues at 1/64 of the FP32 rate here, so the rest runs on the FP32 pipes
// in float pairs (about 48 significant bits).  The coefficients c are
// dyadic rationals, exact in FP32, so the three contractions are
// compensated dot products (Dot2) of FP32 coefficients with float pairs;
// the slaved-node congruence (weights 1/2, 1/4, 1/8: exact scalings) and
// the assembly with lambda, mu and h/2 follow in float-pair arithmetic,
// each entry rounded to FP64 once.  Block of 512 threads per element.
constexpr int kSfMaxN = 64;
struct SfSmem {
  float cf[4][kP][9];           // c_tau(p)[x * 3 + y], tau = 2 m + n (exact)
  double mu[kP][kSfMaxN];       // mu_p(k): integral of xi^p over interval k
  double S1[kSfMaxN][kP];       // one z-slice summed along x
  double S2[kP * kP];           // the same slice summed along x and y
  double M[kNM];                // moments, alpha = ax + 5 (ay + 5 az)
  dfloat Md[kNM];               // the same as float pairs
  dfloat G[4][kP * kP][9];      // contracted over alpha_z, per z-type
  dfloat H[6][kP][81];          // contracted over alpha_y, per pair
  dfloat F[6][729];             // F^st, a = ax + 3 (ay + 3 az), entry a * 27 + b
};
__device__ __forceinline__ int sf_pair(int s, int t) {  // s <= t: 00 11 22 01 02 12
  return s == t ? s : (s == 0 ? (t == 1 ? 3 : 4) : 5);
}

__global__ void __launch_bounds__(512) k_q2_elem_sf(int ex, int ey, long E, int N, double h, double nu,
                                                   const double* __restrict__ w, int Dx, int Dy,
                                                   const int* __restrict__ list, const uint8_t* __restrict__ slv,
                                                   int Lx, int Ly, int sym, double* __restrict__ Ke) {
  extern __shared__ __align__(16) unsigned char sfraw[];
  SfSmem& S = *reinterpret_cast<SfSmem*>(sfraw);
  __shared__ unsigned slaved;  // bit a: local node a is slaved (mixed meshes)
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int t = tid; t < 4 * kP * 9; t += nt) {
    const int tau = t / (kP * 9), p = (t / 9) % kP, xy = t % 9;
    double u[3], v[3];
    lag_coef(xy / 3, tau >> 1, u);
    lag_coef(xy % 3, tau & 1, v);
    double c = 0.0;
    for (int r = 0; r < 3; ++r)
      if (p - r >= 0 && p - r < 3) c += u[r] * v[p - r];
    S.cf[tau][p][xy] = (float)c;
  }
  for (int t = tid; t < kP * N; t += nt) S.mu[t / N][t % N] = mono_int(t / N, t % N, N);
  const double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  const double mu = 1.0 / (2.0 * (1.0 + nu));
  const double hh = 0.5 * h;
  const dfloat lamd(lam), mud(mu), hhd(hh);
  __syncthreads();
  for (long idx = blockIdx.x; idx < E; idx += gridDim.x) {
    const long e = list ? (long)list[idx] : idx;
    const int exi = (int)(e % ex), eyi = (int)((e / ex) % ey), ezi = (int)(e / ((long)ex * ey));
    if (tid == 0) slaved = 0u;
    for (int q = tid; q < kNM; q += nt) S.M[q] = 0.0;
    __syncthreads();
    if (slv != nullptr && tid < kNE && slv[elem_node(exi, eyi, ezi, tid, Lx, Ly)]) atomicOr(&slaved, 1u << tid);
    // ---- moments, one z-slice of cells at a time ----
    for (int c = 0; c < N; ++c) {
      for (int t = tid; t < N * kP; t += nt) {
        const int b = t / kP, p = t % kP;
        const double* row = w + (N * exi) + (long)Dx * ((N * eyi + b) + (long)Dy * (N * ezi + c));
        double acc = 0.0;
        for (int a = 0; a < N; ++a) acc += row[a] * S.mu[p][a];
        S.S1[b][p] = acc;
      }
      __syncthreads();
      for (int t = tid; t < kP * kP; t += nt) {
        const int px = t % kP, py = t / kP;
        double acc = 0.0;
        for (int b = 0; b < N; ++b) acc += S.S1[b][px] * S.mu[py][b];
        S.S2[t] = acc;
      }
      __syncthreads();
      for (int q = tid; q < kNM; q += nt) S.M[q] += S.S2[q % (kP * kP)] * S.mu[q / (kP * kP)][c];
      __syncthreads();
    }
    for (int q = tid; q < kNM; q += nt) S.Md[q] = dfloat(S.M[q]);
    __syncthreads();
    // ---- over alpha_z: G[tz][ax + 5 ay][az * 3 + bz] ----
    for (int t = tid; t < 4 * kP * kP * 9; t += nt) {
      const int tz = t / (kP * kP * 9), xy = (t / 9) % (kP * kP), zz = t % 9;
      Dot2 acc;
      for (int pz = 0; pz < kP; ++pz) acc.add(S.cf[tz][pz][zz], S.Md[xy + kP * kP * pz]);
      S.G[tz][xy][zz] = acc.value();
    }
    __syncthreads();
    // ---- over alpha_y: H[pair][ax][(ay * 3 + by) * 9 + az * 3 + bz] ----
    for (int t = tid; t < 6 * kP * 81; t += nt) {
      const int pr = t / (kP * 81), px = (t / 81) % kP, yz = t % 81;
      const int s = pr < 3 ? pr : (pr == 5 ? 1 : 0), tt = pr < 3 ? pr : (pr == 3 ? 1 : 2);
      const int ty = 2 * (s == 1) + (tt == 1), tz = 2 * (s == 2) + (tt == 2);
      const int yy = yz / 9, zz = yz % 9;
      Dot2 acc;
      for (int py = 0; py < kP; ++py) acc.add(S.cf[ty][py][yy], S.G[tz][px + kP * py][zz]);
      S.H[pr][px][yz] = acc.value();
    }
    __syncthreads();
    // ---- over alpha_x: F[pair][a * 27 + b] ----
    for (int t = tid; t < 6 * 729; t += nt) {
      const int pr = t / 729, ab = t % 729, a = ab / 27, b = ab % 27;
      const int s = pr < 3 ? pr : (pr == 5 ? 1 : 0), tt = pr < 3 ? pr : (pr == 3 ? 1 : 2);
      const int tx = 2 * (s == 0) + (tt == 0);
      const int xx = (a % 3) * 3 + (b % 3);
      const int yz = ((a / 3) % 3 * 3 + (b / 3) % 3) * 9 + (a / 9) * 3 + (b / 9);
      Dot2 acc;
      for (int px = 0; px < kP; ++px) acc.add(S.cf[tx][px][xx], S.H[pr][px][yz]);
      S.F[pr][ab] = acc.value();
    }
    __syncthreads();
    // ---- slaved nodes (mixed meshes): T^T K T = the assembly of T_n^T F T_n ----
    // T = T_n (x) I_3 acts on the nodes alone, so the congruence is applied to
    // every 27 x 27 F^st before the assembly: the column of a slaved node s is
    // added, times 1 / (its parents), to the columns of its parent vertices and
    // cleared (thread per row, s in increasing order), then the same on rows.
    const unsigned sm = slaved;
    if (sm) {
      for (int t = tid; t < 6 * 27; t += nt) {
        dfloat* row = &S.F[t / 27][(t % 27) * 27];
        for (int a = 0; a < kNE; ++a) {
          if (!((sm >> a) & 1u)) continue;  // uniform across the block
          const int np = c_parents.n[a];
          const float sc = 1.f / (float)np;  // a power of two: the scaled pair is exact
          const dfloat v(row[a].hi * sc, row[a].lo * sc);
          for (int q = 0; q < np; ++q) row[c_parents.p[a][q]] += v;
          row[a] = dfloat(0.f, 0.f);
        }
      }
      __syncthreads();
      for (int t = tid; t < 6 * 27; t += nt) {
        dfloat* col = &S.F[t / 27][t % 27];
        for (int a = 0; a < kNE; ++a) {
          if (!((sm >> a) & 1u)) continue;
          const int np = c_parents.n[a];
          const float sc = 1.f / (float)np;
          const dfloat v(col[a * 27].hi * sc, col[a * 27].lo * sc);
          for (int q = 0; q < np; ++q) col[c_parents.p[a][q] * 27] += v;
          col[a * 27] = dfloat(0.f, 0.f);
        }
      }
      __syncthreads();
    }
    // ---- K[(a,i),(b,j)] ----
    // K is symmetric: the upper triangle R <= C is formed (u = R * 81 -
    // R (R - 1) / 2 + C - R) and stored packed (sym) or in both places
    double* out = Ke + e * (size_t)(sym ? kPS2 : kDD);
    for (int u = tid; u < kD * (kD + 1) / 2; u += nt) {
      int R = (int)((2 * kD + 1 - sqrtf((float)((2 * kD + 1) * (2 * kD + 1) - 8 * u))) * 0.5f);
      while (R > 0 && R * kD - R * (R - 1) / 2 > u) --R;
      while ((R + 1) * kD - (R + 1) * R / 2 <= u) ++R;
      const int C = R + u - (R * kD - R * (R - 1) / 2);
      const int a = R / 3, i = R % 3, b = C / 3, j = C % 3;
      const dfloat fij = i <= j ? S.F[sf_pair(i, j)][a * 27 + b] : S.F[sf_pair(j, i)][b * 27 + a];
      const dfloat fji = j <= i ? S.F[sf_pair(j, i)][a * 27 + b] : S.F[sf_pair(i, j)][b * 27 + a];
      dfloat vp = lamd * fij + mud * fji;
      if (i == j) vp += mud * (S.F[0][a * 27 + b] + S.F[1][a * 27 + b] + S.F[2][a * 27 + b]);
      const double v = (double)(hhd * vp);
      if (sym) {
        out[u] = v;
      } else {
        out[R * kD + C] = v;
        out[C * kD + R] = v;
      }
    }
    __syncthreads();
  }
}

// K^(e) = (h/2) sum_alpha M_alpha C_alpha, full 81 x 81, for kEB elements per
// block (each C_alpha entry read once per block).
constexpr int kEB = 8;
template <typename T>
__global__ void k_q2_moments_to_ke(long E, double h, const double* __restrict__ M,
                                   const double* __restrict__ cmom, T* __restrict__ Ke) {
  __shared__ double Ms[kEB][kNM];
  const long e0 = blockIdx.x * (long)kEB;
  const int ne = (int)min((long)kEB, E - e0);
  for (int t = threadIdx.x; t < ne * kNM; t += blockDim.x) Ms[t / kNM][t % kNM] = M[e0 * kNM + t];
  __syncthreads();
  for (int ent = threadIdx.x; ent < kDD; ent += blockDim.x) {
    double acc[kEB];
#pragma unroll
    for (int q = 0; q < kEB; ++q) acc[q] = 0.0;
    for (int al = 0; al < kNM; ++al) {
      const double c = cmom[(size_t)al * kDD + ent];
#pragma unroll
      for (int q = 0; q < kEB; ++q) acc[q] += Ms[q][al] * c;
    }
    for (int q = 0; q < ne; ++q) Ke[(e0 + q) * (size_t)kDD + ent] = (T)(0.5 * h * acc[q]);
  }
}

// Level-0 element matrices: K^(e) = sum_i w_{e,i} K^(e_i) over the n^3
// subcells (Eq. matrixK_mr), FP64.  Block per kEB elements.
template <int K>
__global__ void k_q2_elem(int ex, int ey, long E, int n, const double* __restrict__ w, int Dx, int Dy,
                          const double* __restrict__ tab, double* __restrict__ Ke) {
  constexpr int kDD = Deg<K>::DD;
  extern __shared__ double ws[];  // kEB * m
  const int m = n * n * n;
  const long e0 = blockIdx.x * (long)kEB;
  const int ne = (int)min((long)kEB, E - e0);
  for (int t = threadIdx.x; t < kEB * m; t += blockDim.x) {
    const int q = t / m, s = t % m;
    double v = 0.0;
    if (q < ne) {
      const long e = e0 + q;
      const int exi = e % ex, eyi = (e / ex) % ey, ezi = e / ((long)ex * ey);
      const int a = s % n, b = (s / n) % n, c = s / (n * n);
      v = w[(n * exi + a) + (long)Dx * ((n * eyi + b) + (long)Dy * (n * ezi + c))];
    }
    ws[t] = v;
  }
  __syncthreads();
  for (int ent = threadIdx.x; ent < kDD; ent += blockDim.x) {
    double acc[kEB];
#pragma unroll
    for (int q = 0; q < kEB; ++q) acc[q] = 0.0;
    for (int s = 0; s < m; ++s) {
      const double t = tab[(size_t)s * kDD + ent];
#pragma unroll
      for (int q = 0; q < kEB; ++q) acc[q] += ws[q * m + s] * t;
    }
    for (int q = 0; q < ne; ++q) Ke[(e0 + q) * (size_t)kDD + ent] = acc[q];
  }
}

// Elements along one axis that contain lattice coordinate c (degree K, e
// elements): [lo, hi].
template <int K>
__device__ __forceinline__ void elems_of(int c, int e, int& lo, int& hi) {
  if (c % K) {
    lo = hi = c / K;
  } else {
    lo = max(c / K - 1, 0);
    hi = min(c / K, e - 1);
  }
}

template <typename T>
struct Sum {
  T s = T(0);
  __device__ __forceinline__ void add(op_t<T> a, T x) { s += a * x; }
  __device__ __forceinline__ T value() const { return s; }
};
template <>
struct Sum<dfloat> {
  Dot2 d;
  __device__ __forceinline__ void add(float a, dfloat x) { d.add(a, x); }
  __device__ __forceinline__ dfloat value() const { return d.value(); }
};

// Transfers between serendipity levels by the coarse shape functions
// (prolongation v_h(x) = sum_a phi_a(x) v_H(x_a)) and their transpose.  A
// fine lattice node belongs to the coarse element min(i / 4, E - 1) along
// each axis, at local fine position f = i - 4 e in 0..4; W[a][f] (27 x 125,
// FP32: the values at the quarter points are dyadic and exact) is coarse
// shape function a there.  The restriction gathers, for each coarse node,
// the fine nodes of its elements that belong to those elements, so that it
// is exactly the transpose of the prolongation.
template <int S, typename T>
__global__ void k_s2_prolong(int Lxf, int Lyf, int Lzf, int Lxc, int Lyc, int ecx, int ecy, int ecz,
                             const float* __restrict__ W, const uint8_t* __restrict__ maskf,
                             const T* __restrict__ zc, T* __restrict__ v) {
  constexpr int FP = S + 1, NF = FP * FP * FP;
  const long nnf = (long)Lxf * Lyf * Lzf;
  for (long node = blockIdx.x * (long)blockDim.x + threadIdx.x; node < nnf;
       node += (long)gridDim.x * blockDim.x) {
    const int i = node % Lxf, j = (node / Lxf) % Lyf, l = node / ((long)Lxf * Lyf);
    const int ex = min(i / S, ecx - 1), ey = min(j / S, ecy - 1), ez = min(l / S, ecz - 1);
    const int f = (i - S * ex) + FP * ((j - S * ey) + FP * (l - S * ez));
    Sum<T> acc[3];
    for (int a = 0; a < 27; ++a) {
      const float wgt = W[a * NF + f];
      if (wgt == 0.f) continue;
      const long cn = (2 * ex + a % 3) + (long)Lxc * ((2 * ey + (a / 3) % 3) + (long)Lyc * (2 * ez + a / 9));
      acc[0].add(wgt, zc[3 * cn]);
      acc[1].add(wgt, zc[3 * cn + 1]);
      acc[2].add(wgt, zc[3 * cn + 2]);
    }
    for (int c = 0; c < 3; ++c)
      if (!maskf[3 * node + c]) v[3 * node + c] += acc[c].value();
  }
}

// Restriction, element by element: coarse element E owns the fine nodes
// with min(i / 4, E - 1) = e along each axis (so each fine node counts
// once); Y_E[a] = sum over its owned fine points f of W[a][f] r_f, then each
// coarse node adds Y over the elements that contain it (fixed order).  One
// block per coarse element at a time, 81 outputs.
template <int S, typename T>
__global__ void __launch_bounds__(96) k_s2_restrict_elem(int Lxf, int Lyf, int ecx, int ecy, long Ec,
                                                         const float* __restrict__ W, const T* __restrict__ rf,
                                                         T* __restrict__ Y) {
  constexpr int FP = S + 1, NF = FP * FP * FP;
  __shared__ T rs[NF][3];
  __shared__ float ws[27 * NF];
  for (int t = threadIdx.x; t < 27 * NF; t += blockDim.x) ws[t] = W[t];
  const int ecz = (int)(Ec / ((long)ecx * ecy));
  for (long e = blockIdx.x; e < Ec; e += gridDim.x) {
    const int ex = e % ecx, ey = (e / ecx) % ecy, ez = e / ((long)ecx * ecy);
    __syncthreads();
    for (int t = threadIdx.x; t < NF; t += blockDim.x) {
      const int fx = t % FP, fy = (t / FP) % FP, fz = t / (FP * FP);
      const int i = S * ex + fx, j = S * ey + fy, l = S * ez + fz;
      const bool own = min(i / S, ecx - 1) == ex && min(j / S, ecy - 1) == ey && min(l / S, ecz - 1) == ez;
      const long fn = i + (long)Lxf * (j + (long)Lyf * l);
      for (int c = 0; c < 3; ++c) rs[t][c] = own ? rf[3 * fn + c] : T(0);
    }
    __syncthreads();
    if (threadIdx.x < kD) {
      const int a = threadIdx.x / 3, c = threadIdx.x % 3;
      Sum<T> acc;
      for (int f = 0; f < NF; ++f) {
        const float wgt = ws[a * NF + f];
        if (wgt != 0.f) acc.add(wgt, rs[f][c]);
      }
      Y[e * kD + threadIdx.x] = acc.value();
    }
  }
}

// Lagrange degree 2 -> 2 (a coarse element spans 2 x 2 x 2 fine elements,
// 4 fine lattice intervals per axis): the coarse shape functions are products
// of 1D quadratics, so the transfers are products of 1D transfers.  Along one
// axis a fine node at offset f = 0..4 in its coarse element takes the coarse
// node at f / 2 with weight 1 when f is even, else all three with the values
// of the quadratics at -1/2 (f = 1: 3/8, 3/4, -1/8) or +1/2 (f = 3: -1/8,
// 3/4, 3/8).  Every weight and every product of three is dyadic, exact in
// FP32, and equal to the corresponding entry of the 27 x 125 table.
__device__ __forceinline__ int l2_taps(int i, int e_max, int* c, float* w) {
  const int e = min(i >> 2, e_max), f = i - 4 * e;
  if (!(f & 1)) {
    c[0] = 2 * e + (f >> 1);
    w[0] = 1.f;
    return 1;
  }
  c[0] = 2 * e;
  c[1] = 2 * e + 1;
  c[2] = 2 * e + 2;
  w[0] = f == 1 ? 0.375f : -0.125f;
  w[1] = 0.75f;
  w[2] = f == 1 ? -0.125f : 0.375f;
  return 3;
}

// v_f += (P z_c)_f at the free fine DOFs, one thread per fine node.
template <typename T>
__global__ void k_l2_prolong(int Lxf, int Lyf, int Lzf, int Lxc, int Lyc, int ecx, int ecy, int ecz,
                             const uint8_t* __restrict__ maskf, const T* __restrict__ zc, T* __restrict__ v) {
  const long nnf = (long)Lxf * Lyf * Lzf;
  for (long node = blockIdx.x * (long)blockDim.x + threadIdx.x; node < nnf;
       node += (long)gridDim.x * blockDim.x) {
    const int i = node % Lxf, j = (node / Lxf) % Lyf, l = node / ((long)Lxf * Lyf);
    int cx[3], cy[3], cz[3];
    float wx[3], wy[3], wz[3];
    const int nx = l2_taps(i, ecx - 1, cx, wx), ny = l2_taps(j, ecy - 1, cy, wy), nz = l2_taps(l, ecz - 1, cz, wz);
    Sum<T> acc[3];
    for (int c = 0; c < nz; ++c)
      for (int b = 0; b < ny; ++b) {
        const float wzy = wz[c] * wy[b];
        const long row = (long)Lxc * (cy[b] + (long)Lyc * cz[c]);
        for (int a = 0; a < nx; ++a) {
          const float wgt = wzy * wx[a];
          const T* zp = zc + 3 * (row + cx[a]);
          acc[0].add(wgt, zp[0]);
          acc[1].add(wgt, zp[1]);
          acc[2].add(wgt, zp[2]);
        }
      }
    for (int c = 0; c < 3; ++c)
      if (!maskf[3 * node + c]) v[3 * node + c] += acc[c].value();
  }
}

// Coarse-node taps of the transpose: coarse lattice index I gathers the fine
// nodes 2I - 1, 2I, 2I + 1 (weights 3/4, 1, 3/4) when I is odd (a mid-edge
// node), else 2I - 3, 2I - 1, 2I, 2I + 1, 2I + 3 (-1/8, 3/8, 1, 3/8, -1/8),
// clipped to the fine lattice: the same products as the prolongation.  Five
// fixed slots, absent ones with weight 0 on node 2I (always in range).
__device__ __forceinline__ void l2_rtaps(int I, int Lf, int (&f)[5], float (&w)[5]) {
  const bool odd = I & 1;
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const int off = odd ? (q < 3 ? q - 1 : 0) : (q == 0 ? -3 : (q == 4 ? 3 : q - 2));
    const float wq = odd ? (q == 1 ? 1.f : (q < 3 ? 0.75f : 0.f))
                         : (q == 2 ? 1.f : ((q == 1 || q == 3) ? 0.375f : -0.125f));
    const int i = 2 * I + off;
    const bool in = i >= 0 && i < Lf && wq != 0.f;
    f[q] = in ? i : 2 * I;
    w[q] = in ? wq : 0.f;
  }
}

// b_c = R r_f = P^T r_f (zero at the fixed coarse DOFs) and, unless vc is
// null, the first smoothing step v_c = omega D^-1 b_c; one thread per coarse
// node, the fine nodes in a fixed order.
template <typename T>
__global__ void k_l2_restrict(int Lxf, int Lyf, int Lzf, int Lxc, int Lyc, int Lzc, const T* __restrict__ rf,
                              const uint8_t* __restrict__ maskc, T* __restrict__ bc,
                              const op_t<T>* __restrict__ dinvc, T omega, T* __restrict__ vc) {
  const long nnc = (long)Lxc * Lyc * Lzc;
  for (long node = blockIdx.x * (long)blockDim.x + threadIdx.x; node < nnc;
       node += (long)gridDim.x * blockDim.x) {
    const int I = node % Lxc, J = (node / Lxc) % Lyc, K = node / ((long)Lxc * Lyc);
    int fx[5], fy[5], fz[5];
    float wx[5], wy[5], wz[5];
    l2_rtaps(I, Lxf, fx, wx);
    l2_rtaps(J, Lyf, fy, wy);
    l2_rtaps(K, Lzf, fz, wz);
    Sum<T> acc[3];
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      if (wz[c] == 0.f) continue;
#pragma unroll
      for (int b = 0; b < 5; ++b) {
        const float wzy = wz[c] * wy[b];
        if (wzy == 0.f) continue;
        const long row = (long)Lxf * (fy[b] + (long)Lyf * fz[c]);
#pragma unroll
        for (int a = 0; a < 5; ++a) {
          const float wgt = wzy * wx[a];
          const T* rp = rf + 3 * (row + fx[a]);
          acc[0].add(wgt, rp[0]);
          acc[1].add(wgt, rp[1]);
          acc[2].add(wgt, rp[2]);
        }
      }
    }
    for (int c = 0; c < 3; ++c) {
      const long d = 3 * node + c;
      const T bv = maskc[d] ? T(0) : acc[c].value();
      bc[d] = bv;
      if (vc != nullptr) vc[d] = omega * dinvc[d] * bv;
    }
  }
}

// The same restriction with five lanes per coarse node, one per z tap
// (six nodes per warp): each lane sums its 5 x 5 (x, y) taps and the five
// partials meet by shuffles, added in tap order.  Five times the threads of
// the one-lane form and a fifth of its dependent chain: the small coarse
// levels, whose launches are latency bound, gain most.
template <typename T>
__global__ void k_l2_restrict5(int Lxf, int Lyf, int Lzf, int Lxc, int Lyc, int Lzc, const T* __restrict__ rf,
                               const uint8_t* __restrict__ maskc, T* __restrict__ bc,
                               const op_t<T>* __restrict__ dinvc, T omega, T* __restrict__ vc) {
  const long nnc = (long)Lxc * Lyc * Lzc;
  const int lane = threadIdx.x & 31;
  const long nwarp = ((long)gridDim.x * blockDim.x) >> 5;
  for (long wg = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; wg * 6 < nnc; wg += nwarp) {
    const long node = wg * 6 + lane / 5;
    const int cz = lane % 5;
    const bool live = lane < 30 && node < nnc;
    T acc[3] = {T(0), T(0), T(0)};
    if (live) {
      const int I = node % Lxc, J = (node / Lxc) % Lyc, K = node / ((long)Lxc * Lyc);
      int fx[5], fy[5], fz[5];
      float wx[5], wy[5], wz[5];
      l2_rtaps(I, Lxf, fx, wx);
      l2_rtaps(J, Lyf, fy, wy);
      l2_rtaps(K, Lzf, fz, wz);
      float wzc = 0.f;
      int fzc = 0;
#pragma unroll
      for (int c = 0; c < 5; ++c)
        if (c == cz) {
          wzc = wz[c];
          fzc = fz[c];
        }
      if (wzc != 0.f) {
#pragma unroll
        for (int b = 0; b < 5; ++b) {
          const float wzy = wzc * wy[b];
          if (wzy == 0.f) continue;
          const long row = (long)Lxf * (fy[b] + (long)Lyf * fzc);
#pragma unroll
          for (int a = 0; a < 5; ++a) {
            const float wgt = wzy * wx[a];
            const T* rp = rf + 3 * (row + fx[a]);
            acc[0] += (T)wgt * rp[0];
            acc[1] += (T)wgt * rp[1];
            acc[2] += (T)wgt * rp[2];
          }
        }
      }
    }
    const int base = lane < 30 ? (lane / 5) * 5 : 0;
    T tot[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T sum = T(0);
#pragma unroll
      for (int k = 0; k < 5; ++k) sum += __shfl_sync(0xffffffffu, acc[c], base + k);
      tot[c] = sum;
    }
    if (live && cz == 0)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const long d = 3 * node + c;
        const T bv = maskc[d] ? T(0) : tot[c];
        bc[d] = bv;
        if (vc != nullptr) vc[d] = omega * dinvc[d] * bv;
      }
  }
}

template <typename T>
__global__ void k_s2_restrict_gather(int Lxc, int Lyc, int Lzc, int ecx, int ecy, int ecz,
                                     const T* __restrict__ Y, const uint8_t* __restrict__ maskc,
                                     T* __restrict__ bc, const op_t<T>* __restrict__ dinvc, T omega,
                                     T* __restrict__ vc) {
  const long nnc = (long)Lxc * Lyc * Lzc;
  for (long node = blockIdx.x * (long)blockDim.x + threadIdx.x; node < nnc;
       node += (long)gridDim.x * blockDim.x) {
    const int I = node % Lxc, J = (node / Lxc) % Lyc, K = node / ((long)Lxc * Lyc);
    const int x0 = (I & 1) ? I >> 1 : max((I >> 1) - 1, 0), x1 = min(I >> 1, ecx - 1);
    const int y0 = (J & 1) ? J >> 1 : max((J >> 1) - 1, 0), y1 = min(J >> 1, ecy - 1);
    const int z0 = (K & 1) ? K >> 1 : max((K >> 1) - 1, 0), z1 = min(K >> 1, ecz - 1);
    T acc[3] = {T(0), T(0), T(0)};
    for (int ez = z0; ez <= z1; ++ez)
      for (int ey = y0; ey <= y1; ++ey)
        for (int ex = x0; ex <= x1; ++ex) {
          const long e = ex + (long)ecx * (ey + (long)ecy * ez);
          const int a = (I - 2 * ex) + 3 * ((J - 2 * ey) + 3 * (K - 2 * ez));
          for (int c = 0; c < 3; ++c) acc[c] += Y[e * kD + 3 * a + c];
        }
    for (int c = 0; c < 3; ++c) {
      const long d = 3 * node + c;
      const T bv = maskc[d] ? T(0) : acc[c];
      bc[d] = bv;
      if (vc != nullptr) vc[d] = omega * dinvc[d] * bv;
    }
  }
}


// Y_e = K^(e) u_e for every element; u_e gathered with the fixed DOFs set to
// zero.  One block of 96 threads per element at a time (persistent), thread
// a < 81 computes entry a; K^(e) is symmetric, so its column a (read
// coalesced across the threads) is its row a.  An element whose 81 DOFs are
// all fixed is skipped (no row of it is ever read: the gather passes fixed
// DOFs through as identity rows), so suppressed void regions cost no
// element-matrix traffic.
// With an element list (mixed meshes: the triquadratic elements) only the
// listed elements are applied.
template <int K, typename T>
__global__ void __launch_bounds__(Deg<K>::TB) k_q2_apply(int ex, int ey, long E, int Lx, int Ly,
                                                         const op_t<T>* __restrict__ Ke,
                                                         const uint8_t* __restrict__ mask,
                                                         const T* __restrict__ u, T* __restrict__ Y,
                                                         const int* __restrict__ list) {
  constexpr int kD = Deg<K>::D, kDD = Deg<K>::DD;
  __shared__ T ue[kD];
  for (long t = blockIdx.x; t < E; t += gridDim.x) {
    const long e = list != nullptr ? (long)list[t] : t;
    const int exi = e % ex, eyi = (e / ex) % ey, ezi = e / ((long)ex * ey);
    bool free_dof = false;
    if (threadIdx.x < kD) {
      const int a = threadIdx.x / 3, c = threadIdx.x % 3;
      const long d = 3 * elem_node_k<K>(exi, eyi, ezi, a, Lx, Ly) + c;
      free_dof = mask[d] == 0;
      ue[threadIdx.x] = free_dof ? u[d] : T(0);
    }
    if (!__syncthreads_or(free_dof)) continue;  // block-uniform
    if (threadIdx.x < kD) {
      const op_t<T>* Kc = Ke + e * (size_t)kDD + threadIdx.x;
      Sum<T> acc;
#pragma unroll 9
      for (int b = 0; b < kD; ++b) acc.add(Kc[(size_t)b * kD], ue[b]);
      Y[e * kD + threadIdx.x] = acc.value();
    }
    __syncthreads();
  }
}

// The same for packed symmetric element matrices (Lagrange degree 2, kPS2
// per element: the upper triangle row by row): each element's packed matrix
// is brought into shared memory by one bulk copy (a two-stage ring, so the
// next element's copy runs under this element's products), then thread a
// forms row a: half the matrix traffic of the full form.  Every wait is bounded; on a timeout the block sets *err, lets its
// copies land and stops.
constexpr long kSymSpin = 1L << 22;
__device__ __forceinline__ void sym_issue(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(bytes), "r"(b)
               : "memory");
}
__device__ __forceinline__ bool sym_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done = 0;
  const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
  for (long it = 0; it < kSymSpin && !done; ++it)
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(b), "r"(parity)
        : "memory");
  return done != 0;
}
template <typename T>
__global__ void __launch_bounds__(96) k_q2_apply_sym(int ex, int ey, long E, int Lx, int Ly,
                                                     const op_t<T>* __restrict__ Ke,
                                                     const uint8_t* __restrict__ mask, const T* __restrict__ u,
                                                     T* __restrict__ Y, const int* __restrict__ list, int* err) {
  using O = op_t<T>;
  constexpr uint32_t kBytes = (uint32_t)(kPS2 * sizeof(O));
  extern __shared__ __align__(128) unsigned char symsm[];  // 2 stages of kPS2 entries
  O* ks0 = reinterpret_cast<O*>(symsm);
  __shared__ T ue[kD];
  __shared__ int cofs[kD];  // off(b) - b: entry (b, a), b <= a, is at cofs[b] + a
  __shared__ __align__(8) uint64_t bar[2];
  const int tid = threadIdx.x;
  if (tid < kD) cofs[tid] = sym2_idx(tid, tid) - tid;
  if (tid == 0) {
    for (int q = 0; q < 2; ++q)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(&bar[q])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const long nk = (long)blockIdx.x < E ? (E - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  auto elem_at = [&](long k) {
    const long t = blockIdx.x + k * gridDim.x;
    return list != nullptr ? (long)list[t] : t;
  };
  if (tid == 0)
    for (long k = 0; k < 2 && k < nk; ++k) sym_issue(ks0 + k * kPS2, Ke + elem_at(k) * (size_t)kPS2, kBytes, &bar[k]);
  long k = 0;
  for (; k < nk; ++k) {
    const int st = (int)(k & 1);
    const long e = elem_at(k);
    const int exi = e % ex, eyi = (e / ex) % ey, ezi = e / ((long)ex * ey);
    bool free_dof = false;
    if (tid < kD) {
      const int a = tid / 3, c = tid % 3;
      const long d = 3 * elem_node(exi, eyi, ezi, a, Lx, Ly) + c;
      free_dof = mask[d] == 0;
      ue[tid] = free_dof ? u[d] : T(0);
    }
    const bool any = __syncthreads_or(free_dof) != 0;
    const bool got = sym_wait(&bar[st], (uint32_t)((k >> 1) & 1));
    if (__syncthreads_or(!got)) break;
    if (any && tid < kD) {  // an element with every DOF fixed is skipped (its rows are identity rows)
      // row a in the cyclic order b = a, a + 1, ..: every lane does 81 steps,
      // so no lane idles while the others finish (FP64 issue is the scarce
      // resource); entry (a, b) is at cofs[min] + max
      const O* ks = ks0 + st * kPS2;
      Sum<T> acc;
      int b = tid;
#pragma unroll 3
      for (int q = 0; q < kD; ++q) {
        const int lo = b < tid ? b : tid, hi = b < tid ? tid : b;
        acc.add(ks[cofs[lo] + hi], ue[b]);
        b = b + 1 == kD ? 0 : b + 1;
      }
      Y[e * kD + tid] = acc.value();
    }
    __syncthreads();  // stage st and ue are free
    if (tid == 0 && k + 2 < nk) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      sym_issue(ks0 + st * kPS2, Ke + elem_at(k + 2) * (size_t)kPS2, kBytes, &bar[st]);
    }
  }
  if (k < nk && tid == 0) {  // timed out: flag, then let the copies in flight land
    atomicExch(err, 1);
    for (long q = k; q < nk && q < k + 2; ++q) sym_wait(&bar[q & 1], (uint32_t)((q >> 1) & 1));
  }
}

// The FP32 form of the packed apply (the preconditioner's copies): the same
// two-stage ring of bulk copies, with u_e of the next element gathered while
// this one is multiplied, and row a formed in column order c = 0 .. 80 (u_c
// is then one broadcast read per warp): entry (min(a, c), max(a, c)) steps
// by 80 - c along column a above the diagonal and by 1 along row a.
__global__ void __launch_bounds__(96) k_q2_apply_sym32(int ex, int ey, long E, int Lx, int Ly,
                                                      const float* __restrict__ Ke,
                                                      const uint8_t* __restrict__ mask, const float* __restrict__ u,
                                                      float* __restrict__ Y, const int* __restrict__ list,
                                                      int* err) {
  constexpr uint32_t kBytes = (uint32_t)(kPS2 * sizeof(float));
  __shared__ __align__(128) float ks0[2][kPS2];
  __shared__ float ue[2][kD];
  __shared__ __align__(8) uint64_t bar[2];
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int q = 0; q < 2; ++q)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(&bar[q])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const long nk = (long)blockIdx.x < E ? (E - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  auto elem_at = [&](long k) {
    const long t = blockIdx.x + k * gridDim.x;
    return list != nullptr ? (long)list[t] : t;
  };
  // u_e of element k (fixed DOFs as zero) into registers; whether any is free
  auto gather = [&](long k, float& uv, bool& fr) {
    uv = 0.f;
    fr = false;
    if (k < nk && tid < kD) {
      const long e = elem_at(k);
      const int exi = e % ex, eyi = (e / ex) % ey, ezi = e / ((long)ex * ey);
      const long d = 3 * elem_node(exi, eyi, ezi, tid / 3, Lx, Ly) + tid % 3;
      const float vd = u[d];
      fr = mask[d] == 0;
      uv = fr ? vd : 0.f;
    }
  };
  if (tid == 0)
    for (long k = 0; k < 2 && k < nk; ++k) sym_issue(ks0[k], Ke + elem_at(k) * (size_t)kPS2, kBytes, &bar[k]);
  float uv;
  bool fr;
  gather(0, uv, fr);
  if (tid < kD) ue[0][tid] = uv;
  long k = 0;
  for (; k < nk; ++k) {
    const int st = (int)(k & 1);
    const bool any = __syncthreads_or(fr) != 0;  // ue[st] is complete
    float un;
    bool fn;
    gather(k + 1, un, fn);  // in flight during this element's products
    const bool got = sym_wait(&bar[st], (uint32_t)((k >> 1) & 1));
    if (__syncthreads_or(!got)) break;
    if (any && tid < kD) {  // an element with every DOF fixed is skipped (its rows are identity rows)
      const float* ks = ks0[st];
      const float* uk = ue[st];
      float acc = 0.f;
      int idx = tid;  // (0, a)
#pragma unroll
      for (int c = 0; c < kD; ++c) {
        acc = fmaf(ks[idx], uk[c], acc);
        idx += c < tid ? 80 - c : 1;
      }
      Y[elem_at(k) * kD + tid] = acc;
    }
    if (tid < kD) ue[st ^ 1][tid] = un;  // read by element k - 1, finished before the barriers above
    fr = fn;
    __syncthreads();  // stage st is free
    if (tid == 0 && k + 2 < nk) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      sym_issue(ks0[st], Ke + elem_at(k + 2) * (size_t)kPS2, kBytes, &bar[st]);
    }
  }
  if (k < nk && tid == 0) {  // timed out: flag, then let the copies in flight land
    atomicExch(err, 1);
    for (long q = k; q < nk && q < k + 2; ++q) sym_wait(&bar[q & 1], (uint32_t)((q >> 1) & 1));
  }
}

// Trilinear elements of a mixed mesh: their constrained 81 x 81 matrix is
// T_e^T K T_e with every non-vertex node slaved to the vertices, which is
// zero outside the 24 vertex DOFs, so the product needs only that block
// (24 x 24, the trilinear element's matrix).  Results go to the vertex
// positions of Y; the other positions of these elements belong to slaved
// nodes, which the gather treats as identity rows.  Four elements per
// block of 128 threads, thread r < 24 of each group computes vertex DOF r.
__device__ __forceinline__ int q1v_dof(int r) {  // vertex DOF r -> DOF of the 27-node element
  const int v = r / 3;
  return 3 * (2 * (v & 1) + 3 * (2 * ((v >> 1) & 1)) + 9 * (2 * (v >> 2))) + r % 3;
}
template <typename T>
__global__ void __launch_bounds__(128) k_q1v_apply(int ex, int ey, long E1, int Lx, int Ly,
                                                   const op_t<T>* __restrict__ Ke,
                                                   const uint8_t* __restrict__ mask, const T* __restrict__ u,
                                                   T* __restrict__ Y, const int* __restrict__ list, int sym) {
  __shared__ T ue[4][24];
  const int grp = threadIdx.x >> 5, r = threadIdx.x & 31;
  for (long t0 = (long)blockIdx.x * 4; t0 < E1; t0 += (long)gridDim.x * 4) {
    const long t = t0 + grp;
    const bool live = t < E1 && r < 24;
    long e = 0;
    int dr = 0;
    if (live) {
      e = list[t];
      const int exi = e % ex, eyi = (e / ex) % ey, ezi = e / ((long)ex * ey);
      dr = q1v_dof(r);
      const long d = 3 * elem_node(exi, eyi, ezi, dr / 3, Lx, Ly) + dr % 3;
      ue[grp][r] = mask[d] ? T(0) : u[d];
    }
    __syncthreads();
    if (live) {
      const op_t<T>* Kr = Ke + e * (size_t)(sym ? kPS2 : kDD);
      Sum<T> acc;
#pragma unroll 4
      for (int c = 0; c < 24; ++c)  // symmetric: column dr is row dr
        acc.add(Kr[sym ? sym2_idx(q1v_dof(c), dr) : q1v_dof(c) * kD + dr], ue[grp][c]);
      Y[e * kD + dr] = acc.value();
    }
    __syncthreads();
  }
}

// Serendipity elements: only the 20 (degree 2) or 32 (degree 3) lattice
// positions with at most one coordinate inside an edge carry a node.  The
// element apply reads the compact Dp x Dp matrix of those DOFs (Dp = 60 or
// 96 instead of 81 or 192), formed from the full one after each refresh.
template <int K>
struct Ser {
  static constexpr int NP = K == 2 ? 20 : 32;
  static constexpr int DP = 3 * NP;
  static constexpr int TB = (DP + 31) / 32 * 32;
};

// Lattice-local position of the p-th serendipity node (in lattice order).
template <int K>
__device__ __forceinline__ int ser_pos(int p) {
  constexpr int NA = K + 1;
  int cnt = 0;
  for (int a = 0; a < NA * NA * NA; ++a) {
    const int ix = a % NA, iy = (a / NA) % NA, iz = a / (NA * NA);
    const int inner = (ix % K != 0) + (iy % K != 0) + (iz % K != 0);
    if (inner <= 1) {
      if (cnt == p) return a;
      ++cnt;
    }
  }
  return 0;
}

template <int K, typename T>
__global__ void k_ser_compact(long E, const double* __restrict__ Kf, T* __restrict__ Kc) {
  constexpr int D = Deg<K>::D, DP = Ser<K>::DP;
  __shared__ int pos[Ser<K>::NP];
  for (int t = threadIdx.x; t < Ser<K>::NP; t += blockDim.x) pos[t] = ser_pos<K>(t);
  __syncthreads();
  const long total = E * (long)DP * DP;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const long e = t / ((long)DP * DP);
    const int ent = (int)(t % ((long)DP * DP));
    const int r = ent / DP, c = ent % DP;
    const int R = 3 * pos[r / 3] + r % 3, C = 3 * pos[c / 3] + c % 3;
    Kc[t] = (T)Kf[e * (size_t)D * D + (size_t)R * D + C];
  }
}

template <int K, typename T>
__global__ void __launch_bounds__(Ser<K>::TB) k_ser_apply(int ex, int ey, long E, int Lx, int Ly,
                                                          const op_t<T>* __restrict__ Kc,
                                                          const uint8_t* __restrict__ mask,
                                                          const T* __restrict__ u, T* __restrict__ Y) {
  constexpr int D = Deg<K>::D, DP = Ser<K>::DP;
  __shared__ T ue[DP];
  __shared__ int pos[Ser<K>::NP];
  for (int t = threadIdx.x; t < Ser<K>::NP; t += blockDim.x) pos[t] = ser_pos<K>(t);
  __syncthreads();
  for (long e = blockIdx.x; e < E; e += gridDim.x) {
    const int exi = e % ex, eyi = (e / ex) % ey, ezi = e / ((long)ex * ey);
    bool free_dof = false;
    if (threadIdx.x < DP) {
      const int a = pos[threadIdx.x / 3], c = threadIdx.x % 3;
      const long d = 3 * elem_node_k<K>(exi, eyi, ezi, a, Lx, Ly) + c;
      free_dof = mask[d] == 0;
      ue[threadIdx.x] = free_dof ? u[d] : T(0);
    }
    if (!__syncthreads_or(free_dof)) continue;  // block-uniform
    if (threadIdx.x < DP) {
      const op_t<T>* Kcol = Kc + e * (size_t)DP * DP + threadIdx.x;  // symmetric: column = row
      Sum<T> acc;
#pragma unroll 4
      for (int b = 0; b < DP; ++b) acc.add(Kcol[(size_t)b * DP], ue[b]);
      Y[e * D + 3 * pos[threadIdx.x / 3] + threadIdx.x % 3] = acc.value();
    }
    __syncthreads();
  }
}

// y_n = sum of Y_e over the elements containing node n (fixed order), then
//   mode 0: out = b - y            (residual after the first smoothing)
//   mode 1: out = v + omega D^-1 (b - y)   (post-smoothing)
//   mode 2: out = y                (plain apply)
// Fixed DOFs are identity rows: y = v there.
template <int K, typename T>
__global__ void k_q2_gather(int Lx, int Ly, int Lz, int ex, int ey, int ez, const T* __restrict__ Y,
                            const T* __restrict__ b, const T* __restrict__ v,
                            const op_t<T>* __restrict__ dinv, const uint8_t* __restrict__ mask,
                            T omega, int mode, T* __restrict__ out, ChebStep cs) {
  constexpr int kD = Deg<K>::D, NA = K + 1;
  const long nn = (long)Lx * Ly * Lz;
  for (long node = blockIdx.x * (long)blockDim.x + threadIdx.x; node < nn;
       node += (long)gridDim.x * blockDim.x) {
    const int i = node % Lx, j = (node / Lx) % Ly, l = node / ((long)Lx * Ly);
    // elements along each axis containing this lattice coordinate
    int e0[3], e1[3];
    const int co[3] = {i, j, l}, ext[3] = {ex, ey, ez};
    for (int ax = 0; ax < 3; ++ax) elems_of<K>(co[ax], ext[ax], e0[ax], e1[ax]);
    // the output's vector inputs first, in flight together with the element loads
    constexpr bool kCheb = std::is_same<T, float>::value || std::is_same<T, double>::value;
    uint8_t mk[3];
    T vv[3], bb[3], dp[3];
    op_t<T> di[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const long d = 3 * node + c;
      mk[c] = mask[d];
      vv[c] = v[d];
      bb[c] = mode != 2 ? b[d] : T(0);
      di[c] = mode == 1 || mode == 3 ? dinv[d] : op_t<T>(0);
      dp[c] = vv[c];
      if constexpr (kCheb)
        if (mode == 3 && cs.dprev) dp[c] = static_cast<const T*>(cs.dprev)[d];
    }
    T y[3] = {T(0), T(0), T(0)};
    // the (at most) 2 x 2 x 2 elements, unrolled with predicates so that all
    // their loads are in flight together; summed in the order z, y, x
#pragma unroll
    for (int kz = 0; kz < 2; ++kz)
#pragma unroll
      for (int ky = 0; ky < 2; ++ky)
#pragma unroll
        for (int kx = 0; kx < 2; ++kx) {
          const int ex_ = e0[0] + kx, ey_ = e0[1] + ky, ez_ = e0[2] + kz;
          if (ex_ > e1[0] || ey_ > e1[1] || ez_ > e1[2]) continue;
          const long e = ex_ + (long)ex * (ey_ + (long)ey * ez_);
          const int a = (i - K * ex_) + NA * ((j - K * ey_) + NA * (l - K * ez_));
          const T* Ye = Y + e * kD + 3 * a;
          y[0] += Ye[0];
          y[1] += Ye[1];
          y[2] += Ye[2];
        }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const long d = 3 * node + c;
      const T yc = mk[c] ? vv[c] : y[c];
      if (mode == 0) {
        out[d] = bb[c] - yc;
      } else if (mode == 1) {
        out[d] = vv[c] + omega * di[c] * (bb[c] - yc);
      } else if (mode == 3) {
        if constexpr (kCheb) {
          const T* co = static_cast<const T*>(cs.coef);
          const T c1 = cs.ci < 0 ? T(0) : co[2 * cs.ci], c2 = cs.ci < 0 ? T(1) : co[2 * cs.ci + 1];
          const T o = vv[c] + c1 * dp[c] + c2 * di[c] * (bb[c] - yc);
          static_cast<T*>(cs.dout)[d] = o - vv[c];
          out[d] = o;
        }
      } else {
        out[d] = yc;
      }
    }
  }
}

// Inverse Jacobi diagonal: 1 / sum_e K^(e)_{3a+c, 3a+c}; fixed DOFs 1.
template <int K, typename T>
__global__ void k_q2_dinv(int Lx, int Ly, int Lz, int ex, int ey, int ez, const double* __restrict__ Ke,
                          const uint8_t* __restrict__ mask, T* __restrict__ dinv, int sym) {
  constexpr int kD = Deg<K>::D, kDD = Deg<K>::DD, NA = K + 1;
  const long nn = (long)Lx * Ly * Lz;
  for (long node = blockIdx.x * (long)blockDim.x + threadIdx.x; node < nn;
       node += (long)gridDim.x * blockDim.x) {
    const int i = node % Lx, j = (node / Lx) % Ly, l = node / ((long)Lx * Ly);
    int e0[3], e1[3];
    const int co[3] = {i, j, l}, ext[3] = {ex, ey, ez};
    for (int ax = 0; ax < 3; ++ax) elems_of<K>(co[ax], ext[ax], e0[ax], e1[ax]);
    double dg[3] = {0.0, 0.0, 0.0};
    for (int ez_ = e0[2]; ez_ <= e1[2]; ++ez_)
      for (int ey_ = e0[1]; ey_ <= e1[1]; ++ey_)
        for (int ex_ = e0[0]; ex_ <= e1[0]; ++ex_) {
          const long e = ex_ + (long)ex * (ey_ + (long)ey * ez_);
          const int a = (i - K * ex_) + NA * ((j - K * ey_) + NA * (l - K * ez_));
          for (int c = 0; c < 3; ++c)
            dg[c] += sym ? Ke[e * (size_t)kPS2 + sym2_idx(3 * a + c, 3 * a + c)]
                         : Ke[e * (size_t)kDD + (size_t)(3 * a + c) * kD + 3 * a + c];
        }
    for (int c = 0; c < 3; ++c) {
      const long d = 3 * node + c;
      dinv[d] = mask[d] ? T(1.0) : T(1.0 / dg[c]);
    }
  }
}

// Dense matrix of the coarsest level: elements of one parity class (no two
// share a node) add their matrices; fixed rows and columns are identity.
__global__ void k_q2_dense(int ex, int ey, int ez, int Lx, int Ly, int par, const double* __restrict__ Ke,
                           const uint8_t* __restrict__ mask, long n, double* __restrict__ A, int sym) {
  const int px = par & 1, py = (par >> 1) & 1, pz = par >> 2;
  const int cx = (ex - px + 1) / 2, cy = (ey - py + 1) / 2, cz = (ez - pz + 1) / 2;
  const long Ec = (long)cx * cy * cz;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < Ec * kDD;
       t += (long)gridDim.x * blockDim.x) {
    const long q = t / kDD;
    const int ent = (int)(t % kDD);
    const int exi = 2 * (int)(q % cx) + px, eyi = 2 * (int)((q / cx) % cy) + py,
              ezi = 2 * (int)(q / ((long)cx * cy)) + pz;
    const long e = exi + (long)ex * (eyi + (long)ey * ezi);
    const int R = ent / kD, C = ent % kD;
    const long dr = 3 * elem_node(exi, eyi, ezi, R / 3, Lx, Ly) + R % 3;
    const long dc = 3 * elem_node(exi, eyi, ezi, C / 3, Lx, Ly) + C % 3;
    if (mask[dr] || mask[dc]) continue;
    A[dr * n + dc] += sym ? Ke[e * (size_t)kPS2 + sym2_idx(R, C)] : Ke[e * (size_t)kDD + ent];
  }
}

__global__ void k_q2_dense_fixed(long n, const uint8_t* __restrict__ mask, double* __restrict__ A) {
  for (long d = blockIdx.x * (long)blockDim.x + threadIdx.x; d < n; d += (long)gridDim.x * blockDim.x)
    if (mask[d]) A[d * n + d] = 1.0;
}

// Sensitivities, Sec. 3.4: s_{e,i} = u_e^T K^(e_i) u_e for every (element,
// subcell), dc/drho_i = -p rho_i^(p-1) (E0 - Emin) s (accumulated over load
// cases unless first).  Block per element: u_e staged, warps over subcells,
// lanes over rows.
template <int K>
__global__ void k_q2_energy_grad(int ex, int ey, long E, int n, int Lx, int Ly,
                                 const double* __restrict__ u, const double* __restrict__ tab,
                                 const double* __restrict__ rho, double penal, double dE, int Dx,
                                 int Dy, int first, double* __restrict__ g) {
  constexpr int kD = Deg<K>::D, kDD = Deg<K>::DD;
  __shared__ double ue[kD];
  const int m = n * n * n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (long e = blockIdx.x; e < E; e += gridDim.x) {
    const int exi = e % ex, eyi = (e / ex) % ey, ezi = e / ((long)ex * ey);
    for (int t = threadIdx.x; t < kD; t += blockDim.x)
      ue[t] = u[3 * elem_node_k<K>(exi, eyi, ezi, t / 3, Lx, Ly) + t % 3];
    __syncthreads();
    for (int s = warp; s < m; s += nw) {
      const double* Ks = tab + (size_t)s * kDD;
      double acc = 0.0;
      for (int R = lane; R < kD; R += 32) {
        double y = 0.0;
        for (int C = 0; C < kD; ++C) y += Ks[(size_t)R * kD + C] * ue[C];
        acc += ue[R] * y;
      }
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) {
        const int a = s % n, b = (s / n) % n, c = s / (n * n);
        const long cell = (n * exi + a) + (long)Dx * ((n * eyi + b) + (long)Dy * (n * ezi + c));
        const double r = rho[cell];
        const double gv = -penal * pow(r, penal - 1.0) * dE * acc;
        g[cell] = first ? gv : g[cell] + gv;
      }
    }
    __syncthreads();
  }
}

// Sensitivities of Lagrange degree-2 elements (Sec. 3.4) from the strain
// energy: s_{e,i} = u_e^T K^(e_i) u_e = int over subcell i of
// lam (tr eps)^2 + 2 mu eps:eps (E = 1), integrated exactly by 3-point
// Gauss-Legendre per axis and subcell (the integrand has degree <= 4 per
// axis): the 3n points per axis form a tensor grid, on which the
// displacement gradients come by sum factorisation (contract the 27 nodal
// values over z, then y, then x with the 1D basis values and derivatives).
// The strain energy vanishes on rigid motions, so the element's
// least-squares rigid motion t + w x x (w = 1/36 sum_a x_a x u_a on the
// nodes x_a in {-1, 0, 1}^3, where sum x x^T = 18 I) is removed in FP64
// first; the remaining field is the strain part alone, and the passes and
// the energy densities run in FP32 (64 times FP64's issue rate on this
// part) with no cancellation of large terms.  The subcell sums are FP64.
// dc/drho_i = -p rho_i^(p-1) (E0 - Emin) s_{e,i}, accumulated over load
// cases unless first.  Block of 256 threads per element; each subcell's sum
// is taken in a fixed order by one thread.
// Coordinate d of local node a of the 27-node element, in {-1, 0, 1}.
__device__ __forceinline__ int node_x(int a, int d) {
  return d == 0 ? a % 3 - 1 : (d == 1 ? (a / 3) % 3 - 1 : a / 9 - 1);
}
constexpr int kEgMaxN = 4;
__host__ __device__ constexpr int eg_smem_doubles(int n) {
  // U 81 + rigid motion 8 (FP64) | then FP32: Uf 81 | Tz 3 x 2 x 9 x 3n | Tyz 3 x 3 x 3 x (3n)^2 |
  // energy (3n)^3 | tables 2 x 3n x 3 + 3n  (counted in doubles, rounded up)
  return 89 + (81 + 3 * 2 * 9 * 3 * n + 27 * 9 * n * n + 27 * n * n * n + 2 * 9 * n + 3 * n + 1) / 2;
}
__global__ void __launch_bounds__(256) k_q2_energy_sf(int ex, int ey, long E, int n, int Lx, int Ly, double h,
                                                     double nu, const double* __restrict__ u,
                                                     const double* __restrict__ rho, double penal, double dE,
                                                     int Dx, int Dy, int first, double* __restrict__ g) {
  extern __shared__ double egs[];
  const int Q = 3 * n;  // quadrature points per axis
  double* U = egs;                              // [c][az][ay][ax], FP64
  double* rig = U + 81;                         // t (3), w (3)
  float* Uf = reinterpret_cast<float*>(egs + 89);  // the deflated field, FP32
  float* Tz = Uf + 81;                          // [c][mz][ax + 3 ay][qz]
  float* Tyz = Tz + 3 * 2 * 9 * Q;              // [c][combo][ax][qy * Q + qz], combo: (my,mz) 00 10 01
  float* En = Tyz + 27 * Q * Q;                 // energy density x weight per point
  float* B = En + Q * Q * Q;                    // [m][q][alpha]
  float* Wq = B + 2 * Q * 3;                    // 1D weight per point
  const int tid = threadIdx.x, nt = blockDim.x;
  const double gp[3] = {-sqrt(0.6), 0.0, sqrt(0.6)};
  const double gw[3] = {5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0};
  for (int t = tid; t < Q * 3; t += nt) {
    const int q = t / 3, al = t % 3;
    const double xi = -1.0 + (2 * (q / 3) + 1) / (double)n + gp[q % 3] / n;
    B[q * 3 + al] = (float)lag(al, xi);
    B[Q * 3 + q * 3 + al] = (float)dlag(al, xi);
    if (al == 0) Wq[q] = (float)(gw[q % 3] / n);
  }
  const float lam = (float)(nu / ((1.0 + nu) * (1.0 - 2.0 * nu)));
  const float mu = (float)(1.0 / (2.0 * (1.0 + nu)));
  const float s2h = (float)(2.0 / h);         // d/dx = (2/h) d/dxi
  const double jac = 0.125 * h * h * h;       // dx = (h/2)^3 dxi
  __syncthreads();
  for (long e = blockIdx.x; e < E; e += gridDim.x) {
    const int exi = (int)(e % ex), eyi = (int)((e / ex) % ey), ezi = (int)(e / ((long)ex * ey));
    for (int t = tid; t < 81; t += nt) {
      const int c = t % 3, a = t / 3;
      U[c * 27 + a] = u[3 * elem_node_k<2>(exi, eyi, ezi, a, Lx, Ly) + c];
    }
    __syncthreads();
    if (tid < 6) {  // t_c = mean of component c; w = (1/36) sum_a x_a x u_a (sum x_a = 0)
      double acc = 0.0;
      if (tid < 3) {
        for (int a = 0; a < 27; ++a) acc += U[tid * 27 + a];
        acc *= 1.0 / 27.0;
      } else {
        const int k = tid - 3, k1 = (k + 1) % 3, k2 = (k + 2) % 3;  // (x x u)_k = x_k1 u_k2 - x_k2 u_k1
        for (int a = 0; a < 27; ++a) acc += node_x(a, k1) * U[k2 * 27 + a] - node_x(a, k2) * U[k1 * 27 + a];
        acc *= 1.0 / 36.0;
      }
      rig[tid] = acc;
    }
    __syncthreads();
    for (int t = tid; t < 81; t += nt) {  // u - t - w x x, rounded to FP32
      const int c = t / 27, a = t % 27;
      const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
      const double wx = rig[3 + c1] * node_x(a, c2) - rig[3 + c2] * node_x(a, c1);  // (w x x)_c
      Uf[t] = (float)(U[t] - rig[c] - wx);
    }
    __syncthreads();
    for (int t = tid; t < 3 * 2 * 9 * Q; t += nt) {  // over az
      const int qz = t % Q, xy = (t / Q) % 9, mz = (t / (Q * 9)) % 2, c = t / (Q * 18);
      const float* bz = B + mz * Q * 3 + qz * 3;
      const float* uc = Uf + c * 27 + xy;
      Tz[t] = bz[0] * uc[0] + bz[1] * uc[9] + bz[2] * uc[18];
    }
    __syncthreads();
    for (int t = tid; t < 27 * Q * Q; t += nt) {  // over ay
      const int yz = t % (Q * Q), ax = (t / (Q * Q)) % 3, cb = (t / (Q * Q * 3)) % 3, c = t / (Q * Q * 9);
      const int my = cb == 1, mz = cb == 2;
      const int qy = yz / Q, qz = yz % Q;
      const float* by = B + my * Q * 3 + qy * 3;
      const float* tz = Tz + ((c * 2 + mz) * 9 + ax) * Q + qz;
      Tyz[t] = by[0] * tz[0] + by[1] * tz[3 * Q] + by[2] * tz[6 * Q];
    }
    __syncthreads();
    for (int t = tid; t < Q * Q * Q; t += nt) {  // over ax, then the energy density at the point
      const int qx = t % Q, yz = t / Q, qy = yz / Q, qz = yz % Q;
      const float* b0 = B + qx * 3;
      const float* b1 = B + Q * 3 + qx * 3;
      float gr[3][3];  // gr[c][s] = d u_c / d x_s
#pragma unroll
      for (int c = 0; c < 3; ++c) {
#pragma unroll
        for (int sd = 0; sd < 3; ++sd) {
          const int cb = sd == 0 ? 0 : sd;  // x: (0,0) with B1 in x; y: combo 1; z: combo 2
          const float* bx = sd == 0 ? b1 : b0;
          const float* ty = Tyz + ((c * 3 + cb) * 3) * Q * Q + yz;
          gr[c][sd] = s2h * (bx[0] * ty[0] + bx[1] * ty[Q * Q] + bx[2] * ty[2 * Q * Q]);
        }
      }
      const float tr = gr[0][0] + gr[1][1] + gr[2][2];
      const float e01 = 0.5f * (gr[0][1] + gr[1][0]), e02 = 0.5f * (gr[0][2] + gr[2][0]),
                  e12 = 0.5f * (gr[1][2] + gr[2][1]);
      const float ee = gr[0][0] * gr[0][0] + gr[1][1] * gr[1][1] + gr[2][2] * gr[2][2] +
                       2.0f * (e01 * e01 + e02 * e02 + e12 * e12);
      En[t] = (lam * tr * tr + 2.0f * mu * ee) * Wq[qx] * Wq[qy] * Wq[qz];
    }
    __syncthreads();
    for (int sc = tid; sc < n * n * n; sc += nt) {  // subcell sums, fixed order, FP64
      const int a = sc % n, b = (sc / n) % n, c = sc / (n * n);
      double acc = 0.0;
      for (int k = 0; k < 27; ++k) {
        const int qx = 3 * a + k % 3, qy = 3 * b + (k / 3) % 3, qz = 3 * c + k / 9;
        acc += (double)En[(qy * Q + qz) * Q + qx];  // the layout of the point loop: x fastest, then z, then y
      }
      acc *= jac;
      const long cell = (n * exi + a) + (long)Dx * ((n * eyi + b) + (long)Dy * (n * ezi + c));
      const double gv = -penal * simp_pow(rho[cell], penal - 1.0) * dE * acc;
      g[cell] = first ? gv : g[cell] + gv;
    }
    __syncthreads();
  }
}

// Mixed trilinear / triquadratic meshes (the coupling rule of the mixed
// reading): a non-vertex lattice node touching a trilinear element is slaved
// to the linear interpolation of the 2^q vertices of its edge, face or cell
// (q = number of its odd lattice coordinates, weight 2^-q each).  The slaved
// values of an element come from its own corners, so the constraint is local,
// K^(e) <- T_e^T K^(e) T_e: the triquadratic elements apply it inside their
// sum-factorised set-up (k_q2_elem_sf), the trilinear ones carry their own
// 24 x 24 matrix on the vertices (k_q1v_elem).

// Trilinear elements of a mixed level 0: K1^(e) = sum_i w_{e,i} K1_i over the
// n^3 subcells (the trilinear subcell table at this element size), written
// into the vertex DOFs of the element's 81 x 81 slot; the rest of the slot
// is zero from create and never written (the slot is read by the apply's
// vertex block, the Jacobi diagonal and a one-level dense coarse operator).
// kEB elements per block: the 300 entries of the symmetric 24 x 24 block
// share each table read and are staged in shared memory.
__device__ __forceinline__ int q1v_vertex_node(int v) {  // vertex 0..7 -> its 27-node local index
  return 2 * (v & 1) + 3 * (2 * ((v >> 1) & 1)) + 9 * (2 * (v >> 2));
}
__global__ void __launch_bounds__(256) k_q1v_elem(int ex, int ey, long E1, const int* __restrict__ list, int n,
                                                  const double* __restrict__ w, int Dx, int Dy,
                                                  const double* __restrict__ tab1, int sym,
                                                  double* __restrict__ Ke) {
  extern __shared__ double q1sm[];  // wq[kEB * m], then Kq[kEB][576]
  const int m = n * n * n;
  double* wq = q1sm;
  double* Kq = q1sm + kEB * m;
  for (long e0 = blockIdx.x * (long)kEB; e0 < E1; e0 += (long)gridDim.x * kEB) {
    const int ne = (int)min((long)kEB, E1 - e0);
    __syncthreads();
    for (int t = threadIdx.x; t < kEB * m; t += blockDim.x) {
      const int q = t / m, s = t % m;
      double v = 0.0;
      if (q < ne) {
        const long e = list[e0 + q];
        const int exi = e % ex, eyi = (e / ex) % ey, ezi = e / ((long)ex * ey);
        const int a = s % n, b = (s / n) % n, c = s / (n * n);
        v = w[(n * exi + a) + (long)Dx * ((n * eyi + b) + (long)Dy * (n * ezi + c))];
      }
      wq[t] = v;
    }
    __syncthreads();
    for (int u = threadIdx.x; u < 300; u += blockDim.x) {  // upper triangle of the 24 x 24 block
      int r = 0, off = 0;
      while (off + (24 - r) <= u) { off += 24 - r; ++r; }
      const int c = r + u - off;
      double acc[kEB];
#pragma unroll
      for (int q = 0; q < kEB; ++q) acc[q] = 0.0;
      for (int s = 0; s < m; ++s) {
        const double tv = tab1[(size_t)s * 576 + r * 24 + c];
#pragma unroll
        for (int q = 0; q < kEB; ++q) acc[q] += wq[q * m + s] * tv;
      }
#pragma unroll
      for (int q = 0; q < kEB; ++q) {
        Kq[q * 576 + r * 24 + c] = acc[q];
        Kq[q * 576 + c * 24 + r] = acc[q];
      }
    }
    __syncthreads();
    for (int q = 0; q < ne; ++q) {  // the vertex block only: the rest of the slot stays 0 from create
      double* out = Ke + (size_t)list[e0 + q] * (sym ? kPS2 : kDD);
      for (int t = threadIdx.x; t < 576; t += blockDim.x) {
        const int r = t / 24, c = t % 24;
        const int R = 3 * q1v_vertex_node(r / 3) + r % 3, Cc = 3 * q1v_vertex_node(c / 3) + c % 3;
        if (sym && R > Cc) continue;
        out[sym ? sym2_idx(R, Cc) : R * kD + Cc] = Kq[q * 576 + t];
      }
    }
  }
}

// f <- T^T f: every vertex node collects 2^-q of the value of each slaved
// neighbour (q = number of nonzero offsets); fixed order.
__global__ void k_q2_fold(int Lx, int Ly, int Lz, const uint8_t* __restrict__ slv, double* __restrict__ f) {
  const long nn = (long)Lx * Ly * Lz;
  for (long node = blockIdx.x * (long)blockDim.x + threadIdx.x; node < nn;
       node += (long)gridDim.x * blockDim.x) {
    const int i = node % Lx, j = (node / Lx) % Ly, l = node / ((long)Lx * Ly);
    if ((i | j | l) & 1) continue;  // vertices only
    double acc[3] = {0.0, 0.0, 0.0};
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int q = (dx != 0) + (dy != 0) + (dz != 0);
          if (q == 0) continue;
          const int ii = i + dx, jj = j + dy, ll = l + dz;
          if (ii < 0 || ii >= Lx || jj < 0 || jj >= Ly || ll < 0 || ll >= Lz) continue;
          const long s = ii + (long)Lx * (jj + (long)Ly * ll);
          if (!slv[s]) continue;
          const double w = 1.0 / (1 << q);
          for (int c = 0; c < 3; ++c) acc[c] += w * f[3 * s + c];
        }
    for (int c = 0; c < 3; ++c) f[3 * node + c] += acc[c];
  }
}

// u <- T u on the slaved nodes (their parents are vertices, never slaved).
__global__ void k_q2_expand(int Lx, int Ly, int Lz, const uint8_t* __restrict__ slv, double* __restrict__ u) {
  const long nn = (long)Lx * Ly * Lz;
  for (long node = blockIdx.x * (long)blockDim.x + threadIdx.x; node < nn;
       node += (long)gridDim.x * blockDim.x) {
    if (!slv[node]) continue;
    const int i = node % Lx, j = (node / Lx) % Ly, l = node / ((long)Lx * Ly);
    const int xs[2] = {i & 1 ? i - 1 : i, i & 1 ? i + 1 : i};
    const int ys[2] = {j & 1 ? j - 1 : j, j & 1 ? j + 1 : j};
    const int zs[2] = {l & 1 ? l - 1 : l, l & 1 ? l + 1 : l};
    const int nx = (i & 1) + 1, ny = (j & 1) + 1, nz = (l & 1) + 1;
    const double w = 1.0 / (nx * ny * nz);
    double acc[3] = {0.0, 0.0, 0.0};
    for (int c2 = 0; c2 < nz; ++c2)
      for (int b = 0; b < ny; ++b)
        for (int a = 0; a < nx; ++a) {
          const long p = xs[a] + (long)Lx * (ys[b] + (long)Ly * zs[c2]);
          for (int c = 0; c < 3; ++c) acc[c] += w * u[3 * p + c];
        }
    for (int c = 0; c < 3; ++c) u[3 * node + c] = acc[c];
  }
}

inline int grid_for2(long work, int cap = 65536) {
  long g = (work + 255) / 256;
  if (g < 1) g = 1;
  return (int)(g < cap ? g : cap);
}

}  // namespace

// ---- launchers -------------------------------------------------------------

void launch_q2_subcell_table(int n, double nu, double h, int family, double* tab, cudaStream_t st) {
  k_q2_subcell_table<<<n * n * n, 256, 0, st>>>(n, nu, h, family, tab);
}

void launch_q2_moment_basis(double nu, int family, double* cmom, cudaStream_t st) {
  if (family == 1)
    k_s2_moment_basis<<<(int)(((long)kNM * kDD + 255) / 256), 256, 0, st>>>(nu, cmom);
  else
    k_q2_moment_basis<<<(int)(((long)kNM * kDD + 255) / 256), 256, 0, st>>>(nu, cmom);
}

void launch_s2_restrict(int vt, const Level& F, const Level& C, const float* W, const void* dinvc, double omega,
                        void* vc, cudaStream_t st) {
  const long Ec = (long)C.ex * C.ey * C.ez;
  long ge = (long)F.sms * 8;
  if (ge > Ec) ge = Ec;
  const int g = grid_for2(C.nn);
  const bool pdeg = F.k == 3;  // degree 3 -> 2 on the same elements
  auto run = [&](auto tag) {
    using T = decltype(tag);
    if (C.lag && !pdeg) {  // products of 1D Lagrange transfers, one pass
      if constexpr (std::is_same<T, float>::value || std::is_same<T, double>::value) {
        long g5 = (C.nn + 35) / 36;  // 192 threads: 6 warps of 6 nodes
        if (g5 > 65536) g5 = 65536;
        k_l2_restrict5<T><<<(int)g5, 192, 0, st>>>(F.Lx, F.Ly, F.Lz, C.Lx, C.Ly, C.Lz, (const T*)F.r, C.mask,
                                                   (T*)C.b, (const op_t<T>*)dinvc, (T)omega, (T*)vc);
      } else {
        k_l2_restrict<T><<<g, 256, 0, st>>>(F.Lx, F.Ly, F.Lz, C.Lx, C.Ly, C.Lz, (const T*)F.r, C.mask, (T*)C.b,
                                            (const op_t<T>*)dinvc, (T)omega, (T*)vc);
      }
      return;
    }
    if (pdeg)
      k_s2_restrict_elem<3, T><<<(int)ge, 96, 0, st>>>(F.Lx, F.Ly, C.ex, C.ey, Ec, W, (const T*)F.r, (T*)C.Y);
    else
      k_s2_restrict_elem<4, T><<<(int)ge, 96, 0, st>>>(F.Lx, F.Ly, C.ex, C.ey, Ec, W, (const T*)F.r, (T*)C.Y);
    k_s2_restrict_gather<T><<<g, 256, 0, st>>>(C.Lx, C.Ly, C.Lz, C.ex, C.ey, C.ez, (const T*)C.Y, C.mask,
                                               (T*)C.b, (const op_t<T>*)dinvc, (T)omega, (T*)vc);
  };
  if (vt == kVtF64) run(double());
  else if (vt == kVtF32) run(float());
  else run(dfloat(0.f, 0.f));
}

void launch_s2_prolong(int vt, const Level& F, const Level& C, const float* W, cudaStream_t st) {
  const int g = grid_for2(F.nn);
  auto run = [&](auto tag) {
    using T = decltype(tag);
    if (C.lag && F.k == 2) {
      k_l2_prolong<T><<<g, 256, 0, st>>>(F.Lx, F.Ly, F.Lz, C.Lx, C.Ly, C.ex, C.ey, C.ez, F.mask, (const T*)C.z,
                                         (T*)F.v);
      return;
    }
    if (F.k == 3)
      k_s2_prolong<3, T><<<g, 256, 0, st>>>(F.Lx, F.Ly, F.Lz, C.Lx, C.Ly, C.ex, C.ey, C.ez, W, F.mask,
                                            (const T*)C.z, (T*)F.v);
    else
      k_s2_prolong<4, T><<<g, 256, 0, st>>>(F.Lx, F.Ly, F.Lz, C.Lx, C.Ly, C.ex, C.ey, C.ez, W, F.mask,
                                            (const T*)C.z, (T*)F.v);
  };
  if (vt == kVtF64) run(double());
  else if (vt == kVtF32) run(float());
  else run(dfloat(0.f, 0.f));
}

void launch_q2_elem(const Level& L, int n, const double* w, int Dx, int Dy, const double* tab,
                    double* Ke, cudaStream_t st) {
  const long E = (long)L.ex * L.ey * L.ez;
  const size_t sm = (size_t)kEB * n * n * n * sizeof(double);
  if (L.k == 3)
    k_q2_elem<3><<<(int)((E + kEB - 1) / kEB), 256, sm, st>>>(L.ex, L.ey, E, n, w, Dx, Dy, tab, Ke);
  else
    k_q2_elem<2><<<(int)((E + kEB - 1) / kEB), 256, sm, st>>>(L.ex, L.ey, E, n, w, Dx, Dy, tab, Ke);
}

void launch_ser_compact(const Level& L, cudaStream_t st) {
  const long E = (long)L.ex * L.ey * L.ez;
  const int DP = L.k == 3 ? Ser<3>::DP : Ser<2>::DP;
  const int g = grid_for2(E * DP * DP);
  if (L.Kc64) {
    if (L.k == 3) k_ser_compact<3, double><<<g, 256, 0, st>>>(E, L.K64, L.Kc64);
    else k_ser_compact<2, double><<<g, 256, 0, st>>>(E, L.K64, L.Kc64);
  }
  if (L.Kc32) {  // from the FP64 matrix, rounded once
    if (L.k == 3) k_ser_compact<3, float><<<g, 256, 0, st>>>(E, L.K64, L.Kc32);
    else k_ser_compact<2, float><<<g, 256, 0, st>>>(E, L.K64, L.Kc32);
  }
}

void launch_q3_subcell_table(int n, double nu, double h, int family, double* grad_scratch, double* tab,
                             cudaStream_t st) {
  const long ng = (long)n * n * n * 64 * 64;
  k_q3_grads<<<grid_for2(ng), 256, 0, st>>>(n, h, family, grad_scratch);
  const long nt = (long)n * n * n * Deg<3>::DD;
  k_q3_subcell_table<<<grid_for2(nt), 256, 0, st>>>(n, nu, h, grad_scratch, tab);
}

bool q2_elem_sf_supported(int N) { return N >= 1 && N <= kSfMaxN; }

void launch_q2_elem_sf(const Level& L, const double* w, int Dx, int Dy, double nu, const int* list, long count,
                       const uint8_t* slv, double* Ke, cudaStream_t st) {
  const long E = list ? count : (long)L.ex * L.ey * L.ez;
  if (E <= 0) return;
  const size_t sm = sizeof(SfSmem);
  static std::once_flag attr;  // handles may be created from several threads
  std::call_once(attr, [sm] {
    cudaFuncSetAttribute(k_q2_elem_sf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  });
  long g = (long)L.sms * 3;  // three 70 KB blocks of 512 threads per SM
  if (g > E) g = E;
  if (g < 1) g = 1;
  k_q2_elem_sf<<<(int)g, 512, sm, st>>>(L.ex, L.ey, E, L.nsub, L.h, nu, w, Dx, Dy, list, slv, L.Lx, L.Ly,
                                        L.sym ? 1 : 0, Ke);
}

void launch_q2_coarse_elem(const Level& L, const double* w, int Dx, int Dy, const double* cmom,
                           double* Mscr, double* Ke, cudaStream_t st) {
  const long E = (long)L.ex * L.ey * L.ez;
  const int N = L.nsub;
  k_q2_moments<<<(int)E, N * N >= 128 ? 128 : 32, 0, st>>>(L.ex, L.ey, N, w, Dx, Dy, Mscr);
  k_q2_moments_to_ke<double><<<(int)((E + kEB - 1) / kEB), 256, 0, st>>>(E, L.h, Mscr, cmom, Ke);
}

void launch_q2_dinv(bool fp64, const Level& L, const double* Ke, void* dinv, cudaStream_t st) {
  const int g = grid_for2(L.nn);
  if (L.k == 3) {
    if (fp64)
      k_q2_dinv<3, double><<<g, 256, 0, st>>>(L.Lx, L.Ly, L.Lz, L.ex, L.ey, L.ez, Ke, L.mask, (double*)dinv, 0);
    else
      k_q2_dinv<3, float><<<g, 256, 0, st>>>(L.Lx, L.Ly, L.Lz, L.ex, L.ey, L.ez, Ke, L.mask, (float*)dinv, 0);
  } else {
    if (fp64)
      k_q2_dinv<2, double><<<g, 256, 0, st>>>(L.Lx, L.Ly, L.Lz, L.ex, L.ey, L.ez, Ke, L.mask, (double*)dinv,
                                              L.sym ? 1 : 0);
    else
      k_q2_dinv<2, float><<<g, 256, 0, st>>>(L.Lx, L.Ly, L.Lz, L.ex, L.ey, L.ez, Ke, L.mask, (float*)dinv,
                                             L.sym ? 1 : 0);
  }
}

void launch_q2_dense(const Level& L, const double* Ke, double* A, cudaStream_t st) {
  const long n = L.ndof;
  for (int par = 0; par < 8; ++par)
    k_q2_dense<<<grid_for2((long)L.ex * L.ey * L.ez * kDD / 8 + 1), 256, 0, st>>>(
        L.ex, L.ey, L.ez, L.Lx, L.Ly, par, Ke, L.mask, n, A, L.sym ? 1 : 0);
  k_q2_dense_fixed<<<grid_for2(n), 256, 0, st>>>(n, L.mask, A);
}

// y = A_l v (element apply + gather) with the given mode; T is the vector
// type (double, float, dfloat), the element matrices are op_t<T>.
void launch_q2_op(int vt, const Level& L, const void* Ke, void* Y, const void* b, const void* v,
                  const void* dinv, double omega, int mode, void* out, int sms, cudaStream_t st,
                  const ChebStep* cs) {
  const ChebStep chs = cs ? *cs : ChebStep{};
  // packed symmetric storage: the FP64 operator and its FP32 copy
  const bool symK = L.sym && (Ke == (const void*)L.K64 || Ke == (const void*)L.K32);
  static std::once_flag sym_attr;  // the FP64 ring needs more than the default 48 KB
  std::call_once(sym_attr, [] {
    cudaFuncSetAttribute(k_q2_apply_sym<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * kPS2 * 8);
  });
  const long E = (long)L.ex * L.ey * L.ez;
  long ga = (long)sms * 16;
  if (ga > E) ga = E;
  if (ga < 1) ga = 1;
  const int gg = grid_for2(L.nn);
  // serendipity levels apply their compact matrices
  const void* Kc = Ke == (const void*)L.K64 ? (const void*)L.Kc64
                   : (Ke == (const void*)L.K32 ? (const void*)L.Kc32 : nullptr);
  auto run = [&](auto tag) {
    using T = decltype(tag);
    if (Kc != nullptr) {
      if (L.k == 3)
        k_ser_apply<3, T><<<(int)ga, Ser<3>::TB, 0, st>>>(L.ex, L.ey, E, L.Lx, L.Ly, (const op_t<T>*)Kc, L.mask,
                                                           (const T*)v, (T*)Y);
      else
        k_ser_apply<2, T><<<(int)ga, Ser<2>::TB, 0, st>>>(L.ex, L.ey, E, L.Lx, L.Ly, (const op_t<T>*)Kc, L.mask,
                                                           (const T*)v, (T*)Y);
      if (L.k == 3)
        k_q2_gather<3, T><<<gg, 256, 0, st>>>(L.Lx, L.Ly, L.Lz, L.ex, L.ey, L.ez, (const T*)Y, (const T*)b,
                                              (const T*)v, (const op_t<T>*)dinv, L.mask, (T)omega, mode,
                                              (T*)out, chs);
      else
        k_q2_gather<2, T><<<gg, 256, 0, st>>>(L.Lx, L.Ly, L.Lz, L.ex, L.ey, L.ez, (const T*)Y, (const T*)b,
                                              (const T*)v, (const op_t<T>*)dinv, L.mask, (T)omega, mode,
                                              (T*)out, chs);
      return;
    }
    if (L.el2 != nullptr) {  // mixed level 0: triquadratic list, then the trilinear vertex blocks
      long g2 = (long)sms * 16;
      if (g2 > L.ne2) g2 = L.ne2;
      if (g2 >= 1 && symK && std::is_same<T, float>::value)
        k_q2_apply_sym32<<<(int)(g2 < 8L * sms ? g2 : 8L * sms), 96, 0, st>>>(L.ex, L.ey, L.ne2, L.Lx, L.Ly, (const float*)Ke, L.mask,
                                                 (const float*)v, (float*)Y, L.el2, L.err);
      else if (g2 >= 1 && symK)
        k_q2_apply_sym<T><<<(int)g2, 96, 2 * kPS2 * sizeof(op_t<T>), st>>>(
            L.ex, L.ey, L.ne2, L.Lx, L.Ly, (const op_t<T>*)Ke, L.mask, (const T*)v, (T*)Y, L.el2, L.err);
      else if (g2 >= 1)
        k_q2_apply<2, T><<<(int)g2, Deg<2>::TB, 0, st>>>(L.ex, L.ey, L.ne2, L.Lx, L.Ly, (const op_t<T>*)Ke,
                                                          L.mask, (const T*)v, (T*)Y, L.el2);
      long g1 = (long)sms * 8;
      if (g1 > (L.ne1 + 3) / 4) g1 = (L.ne1 + 3) / 4;
      if (g1 >= 1)
        k_q1v_apply<T><<<(int)g1, 128, 0, st>>>(L.ex, L.ey, L.ne1, L.Lx, L.Ly, (const op_t<T>*)Ke, L.mask,
                                                (const T*)v, (T*)Y, L.el1, symK ? 1 : 0);
      k_q2_gather<2, T><<<gg, 256, 0, st>>>(L.Lx, L.Ly, L.Lz, L.ex, L.ey, L.ez, (const T*)Y, (const T*)b,
                                            (const T*)v, (const op_t<T>*)dinv, L.mask, (T)omega, mode,
                                            (T*)out, chs);
      return;
    }
    if (L.k == 3) {
      k_q2_apply<3, T><<<(int)ga, Deg<3>::TB, 0, st>>>(L.ex, L.ey, E, L.Lx, L.Ly, (const op_t<T>*)Ke, L.mask,
                                                        (const T*)v, (T*)Y, nullptr);
      k_q2_gather<3, T><<<gg, 256, 0, st>>>(L.Lx, L.Ly, L.Lz, L.ex, L.ey, L.ez, (const T*)Y, (const T*)b,
                                            (const T*)v, (const op_t<T>*)dinv, L.mask, (T)omega, mode,
                                            (T*)out, chs);
    } else {
      if (symK && std::is_same<T, float>::value)  // 8 blocks of 27 KB per SM
        k_q2_apply_sym32<<<(int)(ga < 8L * sms ? ga : 8L * sms), 96, 0, st>>>(L.ex, L.ey, E, L.Lx, L.Ly, (const float*)Ke, L.mask,
                                                 (const float*)v, (float*)Y, nullptr, L.err);
      else if (symK)
        k_q2_apply_sym<T><<<(int)ga, 96, 2 * kPS2 * sizeof(op_t<T>), st>>>(
            L.ex, L.ey, E, L.Lx, L.Ly, (const op_t<T>*)Ke, L.mask, (const T*)v, (T*)Y, nullptr, L.err);
      else
        k_q2_apply<2, T><<<(int)ga, Deg<2>::TB, 0, st>>>(L.ex, L.ey, E, L.Lx, L.Ly, (const op_t<T>*)Ke, L.mask,
                                                          (const T*)v, (T*)Y, nullptr);
      k_q2_gather<2, T><<<gg, 256, 0, st>>>(L.Lx, L.Ly, L.Lz, L.ex, L.ey, L.ez, (const T*)Y, (const T*)b,
                                            (const T*)v, (const op_t<T>*)dinv, L.mask, (T)omega, mode,
                                            (T*)out, chs);
    }
  };
  if (vt == kVtF64) run(double());
  else if (vt == kVtF32) run(float());
  else run(dfloat(0.f, 0.f));
}

void launch_elem_fp32(const Level& L, const double* K64, float* K32, cudaStream_t st) {
  launch_to_fp32((size_t)L.ex * L.ey * L.ez * elem_stride(L), K64, K32, st);
}

void launch_q1v_elem(const Level& L, int n, const double* w, int Dx, int Dy, const double* tab1, double* Ke,
                     cudaStream_t st) {
  if (L.ne1 <= 0) return;
  const int m = n * n * n;
  long g = (L.ne1 + kEB - 1) / kEB;
  if (g > (long)L.sms * 8) g = (long)L.sms * 8;
  k_q1v_elem<<<(int)g, 256, (size_t)kEB * (m + 576) * sizeof(double), st>>>(L.ex, L.ey, L.ne1, L.el1, n, w, Dx,
                                                                             Dy, tab1, L.sym ? 1 : 0, Ke);
}

void launch_q2_fold(const Level& L, const uint8_t* slv, double* f, cudaStream_t st) {
  k_q2_fold<<<grid_for2(L.nn), 256, 0, st>>>(L.Lx, L.Ly, L.Lz, slv, f);
}

void launch_q2_expand(const Level& L, const uint8_t* slv, double* u, cudaStream_t st) {
  k_q2_expand<<<grid_for2(L.nn), 256, 0, st>>>(L.Lx, L.Ly, L.Lz, slv, u);
}

bool q2_energy_sf_supported(int n) { return n >= 1 && n <= kEgMaxN; }

void launch_q2_energy_sf(const Level& L0, int n, double nu, const double* u, const double* rho, double penal,
                         double dE, int Dx, int Dy, bool first, double* g, int sms, cudaStream_t st) {
  const long E = (long)L0.ex * L0.ey * L0.ez;
  const size_t sm = (size_t)eg_smem_doubles(n) * sizeof(double);
  static std::once_flag attr;  // handles may be created from several threads
  std::call_once(attr, [] {
    cudaFuncSetAttribute(k_q2_energy_sf, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(eg_smem_doubles(kEgMaxN) * sizeof(double)));
  });
  long gr = (long)sms * 4;
  if (gr > E) gr = E;
  k_q2_energy_sf<<<(int)gr, 256, sm, st>>>(L0.ex, L0.ey, E, n, L0.Lx, L0.Ly, L0.h, nu, u, rho, penal, dE, Dx,
                                           Dy, first ? 1 : 0, g);
}

void launch_q2_energy_grad(const Level& L0, int n, const double* u, const double* tab,
                           const double* rho, double penal, double dE, int Dx, int Dy, bool first,
                           double* g, int sms, cudaStream_t st) {
  const long E = (long)L0.ex * L0.ey * L0.ez;
  long gr = (long)sms * 8;
  if (gr > E) gr = E;
  if (L0.k == 3)
    k_q2_energy_grad<3><<<(int)gr, 256, 0, st>>>(L0.ex, L0.ey, E, n, L0.Lx, L0.Ly, u, tab, rho, penal, dE,
                                                 Dx, Dy, first ? 1 : 0, g);
  else
    k_q2_energy_grad<2><<<(int)gr, 256, 0, st>>>(L0.ex, L0.ey, E, n, L0.Lx, L0.Ly, u, tab, rho, penal, dE,
                                                 Dx, Dy, first ? 1 : 0, g);
}

}  // namespace tos
