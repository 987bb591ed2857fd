// Fixing design variables and suppressing displacement DOFs (Sec. 6.1).
//
// A displacement element is void when all its densities are <= rho_lo and
// all its design-gradient components are >= -eps, solid when all densities
// are >= rho_hi and all gradient components are <= eps.  An element is
// fixed when every element sharing a node with it (inside the domain) is of
// its own kind.  A lattice node whose every element is a fixed void element
// is suppressed: its three DOFs join the supports of level 0 (u = 0, rows
// and columns out of K, loads ignored).  Integer work only: every decision
// is a comparison of stored FP64 values.
#include "internal.cuh"

namespace tos {
namespace {

inline int grid_for(long n, int cap = 4096) {
  long g = (n + kBS - 1) / kBS;
  if (g < 1) g = 1;
  return (int)(g < cap ? g : cap);
}

// cls[e] = 1 void, 2 solid, 0 neither.  rho on the density grid (n cells per
// element edge), g (may be null) on the design grid (d per edge).
__global__ void k_fix_classify(int ex, int ey, int ez, int n, int d, const double* __restrict__ rho,
                               const double* __restrict__ g, double lo, double hi, double eps,
                               int8_t* __restrict__ cls) {
  const long E = (long)ex * ey * ez;
  const long Dx = (long)n * ex, Dy = (long)n * ey, Gx = (long)d * ex, Gy = (long)d * ey;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < E; e += (long)gridDim.x * blockDim.x) {
    const long i = e % ex, j = (e / ex) % ey, k = e / ((long)ex * ey);
    bool vd = true, sd = true;
    for (int c = 0; c < n; ++c)
      for (int b = 0; b < n; ++b)
        for (int a = 0; a < n; ++a) {
          const double r = rho[(n * i + a) + Dx * ((n * j + b) + Dy * (n * k + c))];
          vd = vd && r <= lo;
          sd = sd && r >= hi;
        }
    if (g != nullptr)
      for (int c = 0; c < d; ++c)
        for (int b = 0; b < d; ++b)
          for (int a = 0; a < d; ++a) {
            const double v = g[(d * i + a) + Gx * ((d * j + b) + Gy * (d * k + c))];
            vd = vd && v >= -eps;
            sd = sd && v <= eps;
          }
    cls[e] = vd ? 1 : (sd ? 2 : 0);
  }
}

// fixed[e] = cls[e] when all in-domain elements sharing a node with e have
// the same class, else 0.
__global__ void k_fix_surround(int ex, int ey, int ez, const int8_t* __restrict__ cls,
                               int8_t* __restrict__ fixed) {
  const long E = (long)ex * ey * ez;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < E; e += (long)gridDim.x * blockDim.x) {
    const int i = e % ex, j = (e / ex) % ey, k = e / ((long)ex * ey);
    const int8_t c0 = cls[e];
    bool same = c0 != 0;
    for (int c = max(k - 1, 0); same && c <= min(k + 1, ez - 1); ++c)
      for (int b = max(j - 1, 0); same && b <= min(j + 1, ey - 1); ++b)
        for (int a = max(i - 1, 0); a <= min(i + 1, ex - 1); ++a)
          same = same && cls[a + (long)ex * (b + (long)ey * c)] == c0;
    fixed[e] = same ? c0 : 0;
  }
}

// Per design variable: the class of its fixed element.
__global__ void k_fix_design(int ex, int ey, int ez, int d, const int8_t* __restrict__ fixed,
                             uint8_t* __restrict__ out) {
  const long Gx = (long)d * ex, Gy = (long)d * ey, G = Gx * Gy * ((long)d * ez);
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < G; t += (long)gridDim.x * blockDim.x) {
    const long cx = t % Gx, cy = (t / Gx) % Gy, cz = t / (Gx * Gy);
    out[t] = (uint8_t)fixed[cx / d + (long)ex * (cy / d + (long)ey * (cz / d))];
  }
}

// Elements of a degree-k lattice containing node coordinate c along one
// axis of e elements: [lo, hi].
__device__ __forceinline__ void elem_range(int c, int k, int e, int& lo, int& hi) {
  lo = (c % k == 0) ? (c - 1) / k : c / k;
  if (c == 0) lo = 0;
  hi = c / k;
  if (hi > e - 1) hi = e - 1;
}

// Level-0 mask: base (supports, slaved nodes) plus the suppressed nodes.
__global__ void k_fix_mask(int k, int ex, int ey, int ez, int Lx, int Ly, int Lz,
                           const int8_t* __restrict__ fixed, const uint8_t* __restrict__ base,
                           uint8_t* __restrict__ mask) {
  const long nn = (long)Lx * Ly * Lz;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < nn; t += (long)gridDim.x * blockDim.x) {
    const int i = t % Lx, j = (t / Lx) % Ly, l = t / ((long)Lx * Ly);
    int x0, x1, y0, y1, z0, z1;
    elem_range(i, k, ex, x0, x1);
    elem_range(j, k, ey, y0, y1);
    elem_range(l, k, ez, z0, z1);
    bool sup = true;
    for (int c = z0; sup && c <= z1; ++c)
      for (int b = y0; sup && b <= y1; ++b)
        for (int a = x0; a <= x1; ++a) sup = sup && fixed[a + (long)ex * (b + (long)ey * c)] == 1;
    for (int q = 0; q < 3; ++q) mask[3 * t + q] = (uint8_t)(base[3 * t + q] | (sup ? 1 : 0));
  }
}

__global__ void k_zero_fixed_void(long n, const uint8_t* __restrict__ xfix, double* __restrict__ g) {
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
    if (xfix[t] == 1) g[t] = 0.0;
}

}  // namespace

void launch_fix_classify(const Level& L0, int n, int d, const double* rho, const double* g, double lo,
                         double hi, double eps, int8_t* cls, cudaStream_t st) {
  const long E = (long)L0.ex * L0.ey * L0.ez;
  k_fix_classify<<<grid_for(E), kBS, 0, st>>>(L0.ex, L0.ey, L0.ez, n, d, rho, g, lo, hi, eps, cls);
}

void launch_fix_surround(const Level& L0, const int8_t* cls, int8_t* fixed, cudaStream_t st) {
  const long E = (long)L0.ex * L0.ey * L0.ez;
  k_fix_surround<<<grid_for(E), kBS, 0, st>>>(L0.ex, L0.ey, L0.ez, cls, fixed);
}

void launch_fix_design(const Level& L0, int d, const int8_t* fixed, uint8_t* out, cudaStream_t st) {
  const long G = (long)L0.ex * L0.ey * L0.ez * d * d * d;
  k_fix_design<<<grid_for(G), kBS, 0, st>>>(L0.ex, L0.ey, L0.ez, d, fixed, out);
}

void launch_fix_mask(const Level& L0, const int8_t* fixed, const uint8_t* base, cudaStream_t st) {
  k_fix_mask<<<grid_for(L0.nn), kBS, 0, st>>>(L0.k, L0.ex, L0.ey, L0.ez, L0.Lx, L0.Ly, L0.Lz, fixed, base,
                                              L0.mask);
}

void launch_zero_fixed_void(long n, const uint8_t* xfix, double* g, cudaStream_t st) {
  k_zero_fixed_void<<<grid_for(n), kBS, 0, st>>>(n, xfix, g);
}

}  // namespace tos
