// Density projection (thresholding) and the Heaviside projection (Sec. 5).
//
//  * tosolve_heaviside: eta with sum h(rho_i, beta, eta) = sum rho_i by
//    Newton's method (start 1/2, each step's sums are deterministic block
//    reductions; a step that would leave (0, 1) is halved), then
//    out = h(rho, beta, eta).
//  * tosolve_threshold_density: round densities >= hi to 1 and <= lo to 0,
//    make the floor(vfrac n) largest 1 and the rest 0 (a stable sort in
//    descending order: among equal densities the lower index wins), then
//    test the angle condition (Eq. angle) between d = out - rho_rounded and
//    -grad L.
//  * tosolve_threshold_gradient: the same rounding; alpha_i is the step at
//    which rho_i - alpha grad_i reaches 0 (grad_i > 0) or 1 (grad_i < 0).
//    The steps are sorted (ties by index); at candidate j the components
//    0..j sit at their bound and the others have moved by -alpha_j grad, so
//    grad^T d = S1_j - alpha_j G_j and ||d||^2 = S2_j + alpha_j^2 G_j with
//    prefix sums S1 (grad (t - rho)), S2 ((t - rho)^2) over the reached
//    components and G the sum of grad^2 over the others; a prefix count of
//    safeguard violations (reaching 1 from below v_min^u, 0 from above
//    v_max^l) bars every later candidate.  alpha~ is the last candidate that
//    passes (0 if none), out = clip(rho - alpha~ grad, 0, 1).
//
// The sort is a least-significant-digit radix sort of 64-bit keys with the
// element index as payload, 8 bits per pass; each pass is a per-tile digit
// histogram, one scan of the histograms (digit-major, so equal digits keep
// tile order) and a stable scatter that ranks each tile's elements in order
// (warp match + per-warp counts).  Every sum is a fixed-order reduction.
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace tos {
namespace {

constexpr int kTB = 256;                  // threads per block
constexpr int kPer = 8;                   // elements per thread and tile
constexpr int kTileN = kTB * kPer;        // elements per tile
constexpr int kDigits = 256;

inline int tiles_of(long n) { return (int)((n + kTileN - 1) / kTileN); }

__global__ void k_round(long n, const double* __restrict__ rho, double lo, double hi, double* __restrict__ r) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const double v = rho[i];
    r[i] = v >= hi ? 1.0 : (v <= lo ? 0.0 : v);
  }
}

// keys for a descending sort of densities in [0, 1]: larger density, smaller
// key (the bit pattern of a non-negative double orders like its value).
__global__ void k_keys_desc(long n, const double* __restrict__ r, uint64_t* __restrict__ k, int* __restrict__ idx) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    k[i] = ~(uint64_t)__double_as_longlong(r[i]);
    idx[i] = (int)i;
  }
}

// keys for an ascending sort of the steps alpha_i >= 0 (+inf where grad = 0)
__global__ void k_keys_alpha(long n, const double* __restrict__ r, const double* __restrict__ g,
                             uint64_t* __restrict__ k, int* __restrict__ idx) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const double gi = g[i];
    double a = __longlong_as_double(0x7ff0000000000000LL);  // +inf
    if (gi > 0.0) a = r[i] / gi;
    else if (gi < 0.0) a = (r[i] - 1.0) / gi;
    if (a == 0.0) a = 0.0;  // -0.0 (rho = 1, grad < 0) sorts as +0.0: reached at once
    k[i] = (uint64_t)__double_as_longlong(a);
    idx[i] = (int)i;
  }
}

__global__ void __launch_bounds__(kTB) k_sort_hist(long n, const uint64_t* __restrict__ keys, int shift,
                                                   int ntiles, unsigned* __restrict__ hist) {
  __shared__ unsigned h[kDigits];
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    h[threadIdx.x] = 0;
    __syncthreads();
    const long base = (long)t * kTileN;
    for (int q = 0; q < kPer; ++q) {
      const long e = base + q * kTB + threadIdx.x;
      if (e < n) atomicAdd(&h[(keys[e] >> shift) & 0xff], 1u);
    }
    __syncthreads();
    hist[(long)threadIdx.x * ntiles + t] = h[threadIdx.x];
    __syncthreads();
  }
}

// Exclusive scan of m unsigned counts in place, one block of 1024 threads
// (each a contiguous chunk).
__global__ void __launch_bounds__(1024) k_scan_u32(long m, unsigned* __restrict__ a) {
  __shared__ unsigned s[1024];
  const long chunk = (m + 1023) / 1024;
  const long b = threadIdx.x * chunk, e = min(b + chunk, m);
  unsigned tot = 0;
  for (long i = b; i < e; ++i) tot += a[i];
  s[threadIdx.x] = tot;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const unsigned v = threadIdx.x >= o ? s[threadIdx.x - o] : 0u;
    __syncthreads();
    s[threadIdx.x] += v;
    __syncthreads();
  }
  unsigned run = s[threadIdx.x] - tot;
  for (long i = b; i < e; ++i) {
    const unsigned v = a[i];
    a[i] = run;
    run += v;
  }
}

__global__ void __launch_bounds__(kTB) k_sort_scatter(long n, const uint64_t* __restrict__ kin,
                                                      const int* __restrict__ vin, int shift, int ntiles,
                                                      const unsigned* __restrict__ off,
                                                      uint64_t* __restrict__ kout, int* __restrict__ vout) {
  __shared__ unsigned run[kDigits];
  __shared__ unsigned wc[kTB / 32][kDigits];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    run[threadIdx.x] = off[(long)threadIdx.x * ntiles + t];
    const long base = (long)t * kTileN;
    for (int q = 0; q < kPer; ++q) {
      for (int w = 0; w < kTB / 32; ++w) wc[w][threadIdx.x] = 0;
      __syncthreads();
      const long e = base + q * kTB + threadIdx.x;
      const bool valid = e < n;
      uint64_t key = 0;
      int val = 0;
      int dg = kDigits;  // invalid lanes share a digit no valid lane has
      if (valid) {
        key = kin[e];
        val = vin[e];
        dg = (int)((key >> shift) & 0xff);
      }
      const unsigned same = __match_any_sync(0xffffffffu, dg);
      const int rank = __popc(same & lt);
      if (valid && rank == 0) wc[warp][dg] = __popc(same);
      __syncthreads();
      if (valid) {
        unsigned pos = run[dg] + rank;
        for (int w = 0; w < warp; ++w) pos += wc[w][dg];
        kout[pos] = key;
        vout[pos] = val;
      }
      __syncthreads();
      unsigned add = 0;
      for (int w = 0; w < kTB / 32; ++w) add += wc[w][threadIdx.x];
      run[threadIdx.x] += add;
      __syncthreads();
    }
  }
}

// ---- reductions -------------------------------------------------------------

template <int K>
struct Vec {
  double v[K];
};

template <int K>
__device__ __forceinline__ Vec<K> block_sum_k(Vec<K> x) {
  __shared__ double red[K][kTB / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k)
    for (int o = 16; o > 0; o >>= 1) x.v[k] += __shfl_xor_sync(0xffffffffu, x.v[k], o);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) red[k][warp] = x.v[k];
  __syncthreads();
  Vec<K> s;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    s.v[k] = 0.0;
    if (threadIdx.x == 0)
      for (int w = 0; w < kTB / 32; ++w) s.v[k] += red[k][w];
  }
  return s;
}

template <int K>
__global__ void __launch_bounds__(kTB) k_sum_parts(int np, const double* __restrict__ part, double* __restrict__ out) {
  Vec<K> x;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    x.v[k] = 0.0;
    for (int t = threadIdx.x; t < np; t += kTB) x.v[k] += part[(long)k * np + t];
  }
  x = block_sum_k<K>(x);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = x.v[k];
}

// Heaviside sums at eta: sum h - rho and sum dh/deta (partials per block).
__global__ void __launch_bounds__(kTB) k_heav_sums(long n, const double* __restrict__ r, double beta, double eta,
                                                   int np, double* __restrict__ part) {
  const double tn = tanh(beta * eta), t1 = tanh(beta * (1.0 - eta));
  const double den = tn + t1;
  const double dden = beta * (1.0 - tn * tn) - beta * (1.0 - t1 * t1);
  Vec<2> x{{0.0, 0.0}};
  for (long i = blockIdx.x * (long)kTB + threadIdx.x; i < n; i += (long)np * kTB) {
    const double tr = tanh(beta * (r[i] - eta));
    const double num = tn + tr;
    const double dnum = beta * (1.0 - tn * tn) - beta * (1.0 - tr * tr);
    x.v[0] += num / den - r[i];
    x.v[1] += (dnum * den - num * dden) / (den * den);
  }
  x = block_sum_k<2>(x);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = x.v[0];
    part[np + blockIdx.x] = x.v[1];
  }
}

__global__ void k_heav_apply(long n, const double* __restrict__ r, double beta, double eta, double* __restrict__ out) {
  const double tn = tanh(beta * eta), den = tn + tanh(beta * (1.0 - eta));
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    out[i] = (tn + tanh(beta * (r[i] - eta))) / den;
}

// out[idx[j]] = j < k ? 1 : 0
__global__ void k_top_k(long n, long k, const int* __restrict__ idx, double* __restrict__ out) {
  for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < n; j += (long)gridDim.x * blockDim.x)
    out[idx[j]] = j < k ? 1.0 : 0.0;
}

// angle sums: grad^T d, ||grad||^2, ||d||^2 with d = out - r
__global__ void __launch_bounds__(kTB) k_angle_sums(long n, const double* __restrict__ g, const double* __restrict__ out,
                                                    const double* __restrict__ r, int np, double* __restrict__ part) {
  Vec<3> x{{0.0, 0.0, 0.0}};
  for (long i = blockIdx.x * (long)kTB + threadIdx.x; i < n; i += (long)np * kTB) {
    const double d = out[i] - r[i];
    x.v[0] += g[i] * d;
    x.v[1] += g[i] * g[i];
    x.v[2] += d * d;
  }
  x = block_sum_k<3>(x);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < 3; ++k) part[(long)k * np + blockIdx.x] = x.v[k];
}

// ---- gradient strategy ---------------------------------------------------------

// Per sorted position j: (S1, S2, P, B) terms, P = grad^2, B = 1 for a
// safeguard violation.  Tile-local inclusive scans; tile totals to tot.
__global__ void __launch_bounds__(kTB) k_grad_scan(long n, const int* __restrict__ idx, const double* __restrict__ r,
                                                   const double* __restrict__ g, double vu, double vl,
                                                   double* __restrict__ S, double* __restrict__ tot) {
  __shared__ double sh[4][kTB];
  const long base = (long)blockIdx.x * kTileN + (long)threadIdx.x * kPer;
  double loc[kPer][4];
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int q = 0; q < kPer; ++q) {
    const long j = base + q;
    double t4[4] = {0.0, 0.0, 0.0, 0.0};
    if (j < n) {
      const int i = idx[j];
      const double gi = g[i], ri = r[i];
      if (gi != 0.0) {
        const double t = gi > 0.0 ? 0.0 : 1.0;
        t4[0] = gi * (t - ri);
        t4[1] = (t - ri) * (t - ri);
        t4[3] = ((gi < 0.0 && ri < vu) || (gi > 0.0 && ri > vl)) ? 1.0 : 0.0;
      }
      t4[2] = gi * gi;
    }
    for (int c = 0; c < 4; ++c) {
      acc[c] += t4[c];
      loc[q][c] = acc[c];
    }
  }
  for (int c = 0; c < 4; ++c) sh[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int o = 1; o < kTB; o <<= 1) {  // inclusive scan of the thread totals
    double v[4];
    for (int c = 0; c < 4; ++c) v[c] = threadIdx.x >= o ? sh[c][threadIdx.x - o] : 0.0;
    __syncthreads();
    for (int c = 0; c < 4; ++c) sh[c][threadIdx.x] += v[c];
    __syncthreads();
  }
  double pre[4];
  for (int c = 0; c < 4; ++c) pre[c] = sh[c][threadIdx.x] - acc[c];
  for (int q = 0; q < kPer; ++q) {
    const long j = base + q;
    if (j < n)
      for (int c = 0; c < 4; ++c) S[(long)c * n + j] = pre[c] + loc[q][c];
  }
  if (threadIdx.x == kTB - 1)
    for (int c = 0; c < 4; ++c) tot[(long)c * gridDim.x + blockIdx.x] = sh[c][kTB - 1];
}

// Exclusive scan of the tile totals (4 quantities), one block.
__global__ void __launch_bounds__(1024) k_scan_tot(int nt, double* __restrict__ tot) {
  __shared__ double s[1024];
  const int chunk = (nt + 1023) / 1024;
  const int b = threadIdx.x * chunk, e = min(b + chunk, nt);
  for (int c = 0; c < 4; ++c) {
    double sum = 0.0;
    for (int i = b; i < e; ++i) sum += tot[(long)c * nt + i];
    s[threadIdx.x] = sum;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      const double v = threadIdx.x >= o ? s[threadIdx.x - o] : 0.0;
      __syncthreads();
      s[threadIdx.x] += v;
      __syncthreads();
    }
    double run = s[threadIdx.x] - sum;
    for (int i = b; i < e; ++i) {
      const double v = tot[(long)c * nt + i];
      tot[(long)c * nt + i] = run;
      run += v;
    }
    __syncthreads();
  }
}

// Candidate j passes: finite step, no violation up to j, angle condition.
// Largest passing j per block (or -1).
__global__ void __launch_bounds__(kTB) k_grad_pick(long n, const uint64_t* __restrict__ keys,
                                                   const double* __restrict__ S, const double* __restrict__ tot,
                                                   int nt, double gsum2, double cmax, long long* __restrict__ best) {
  __shared__ long long bm[kTB / 32];
  long long mine = -1;
  const double ng = sqrt(gsum2);
  for (long j = blockIdx.x * (long)kTB + threadIdx.x; j < n; j += (long)gridDim.x * kTB) {
    const double a = __longlong_as_double((long long)keys[j]);
    if (!(a < __longlong_as_double(0x7ff0000000000000LL))) continue;
    const int t = (int)(j / kTileN);
    const double s1 = S[j] + tot[t], s2 = S[n + j] + tot[nt + t];
    const double p = S[2 * n + j] + tot[2 * nt + t], bad = S[3 * n + j] + tot[3 * nt + t];
    if (bad > 0.0) continue;
    const double G = gsum2 - p;
    const double gd = s1 - a * G;
    const double dd = sqrt(fmax(s2 + a * a * G, 0.0));
    if (dd > 0.0 && ng > 0.0 && -gd / (ng * dd) > cmax) mine = j > mine ? j : mine;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const long long v = __shfl_xor_sync(0xffffffffu, mine, o);
    mine = v > mine ? v : mine;
  }
  if ((threadIdx.x & 31) == 0) bm[threadIdx.x >> 5] = mine;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long m = -1;
    for (int w = 0; w < kTB / 32; ++w) m = bm[w] > m ? bm[w] : m;
    best[blockIdx.x] = m;
  }
}

__global__ void k_proj_step(long n, const double* __restrict__ r, const double* __restrict__ g, double alpha,
                            double* __restrict__ out) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    out[i] = fmin(fmax(r[i] - alpha * g[i], 0.0), 1.0);
}

inline int grid_of(long n, int cap = 2048) {
  long g = (n + kTB - 1) / kTB;
  if (g < 1) g = 1;
  return (int)(g < cap ? g : cap);
}

// Scratch layout (bytes, each part 256-aligned).
struct Scratch {
  double* r;
  uint64_t* k0;
  uint64_t* k1;
  int* i0;
  int* i1;
  unsigned* hist;
  double* S;
  double* tot;
  double* part;
  double* sums;
  long long* best;
};

inline size_t al(size_t b) { return (b + 255) & ~size_t(255); }

size_t scratch_layout(long n, Scratch* s, char* base) {
  const int nt = tiles_of(n);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + o : nullptr;
    o += al(bytes);
    return p;
  };
  s->r = (double*)take(n * 8);
  s->k0 = (uint64_t*)take(n * 8);
  s->k1 = (uint64_t*)take(n * 8);
  s->i0 = (int*)take(n * 4);
  s->i1 = (int*)take(n * 4);
  s->hist = (unsigned*)take((size_t)kDigits * nt * 4);
  s->S = (double*)take((size_t)4 * n * 8);
  s->tot = (double*)take((size_t)4 * nt * 8);
  s->part = (double*)take((size_t)3 * 2048 * 8);
  s->sums = (double*)take(4 * 8);
  s->best = (long long*)take(2048 * 8);
  return o;
}

// Stable ascending sort of keys (k0) with payload (i0); the result ends in
// k0 / i0 (eight passes: an even number of swaps).
cudaError_t radix_sort(long n, Scratch& s, cudaStream_t st) {
  const int nt = tiles_of(n);
  const long m = (long)kDigits * nt;
  const int g = nt < 4096 ? nt : 4096;
  uint64_t *ka = s.k0, *kb = s.k1;
  int *ia = s.i0, *ib = s.i1;
  for (int shift = 0; shift < 64; shift += 8) {
    k_sort_hist<<<g, kTB, 0, st>>>(n, ka, shift, nt, s.hist);
    k_scan_u32<<<1, 1024, 0, st>>>(m, s.hist);
    k_sort_scatter<<<g, kTB, 0, st>>>(n, ka, ia, shift, nt, s.hist, kb, ib);
    uint64_t* tk = ka; ka = kb; kb = tk;
    int* ti = ia; ia = ib; ib = ti;
  }
  return cudaGetLastError();
}

}  // namespace

size_t threshold_scratch_bytes(long n) {
  Scratch s;
  return scratch_layout(n, &s, nullptr);
}

tosolve_status heaviside(const double* rho, long n, double beta, double* out, double* eta_out, int* its_out,
                         void* scratch, size_t bytes, cudaStream_t st, std::string* why) {
  Scratch s;
  if (scratch_layout(n, &s, (char*)scratch) > bytes) { *why = "scratch too small"; return TOSOLVE_EINVAL; }
  const int np = grid_of(n);
  double h[2];
  double eta = 0.5;
  int it = 0;
  const double scale = (double)n;
  for (; it < 100; ++it) {
    k_heav_sums<<<np, kTB, 0, st>>>(n, rho, beta, eta, np, s.part);
    k_sum_parts<2><<<1, kTB, 0, st>>>(np, s.part, s.sums);
    if (cudaMemcpyAsync(h, s.sums, 2 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      *why = "Newton step failed";
      return TOSOLVE_ECUDA;
    }
    if (std::fabs(h[0]) <= 1e-12 * scale) break;
    double step = h[0] / h[1];
    int halvings = 0;
    while (!(eta - step > 0.0 && eta - step < 1.0) && halvings < 200) {
      step *= 0.5;
      ++halvings;
    }
    eta -= step;
    if (std::fabs(step) < 1e-14) { ++it; break; }
  }
  k_heav_apply<<<grid_of(n), kTB, 0, st>>>(n, rho, beta, eta, out);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
    *why = "Heaviside apply failed";
    return TOSOLVE_ECUDA;
  }
  if (eta_out) *eta_out = eta;
  if (its_out) *its_out = it;
  return TOSOLVE_OK;
}

static bool angle_ok(const double* g, const double* out, const Scratch& s, long n, double cmax, cudaStream_t st,
                     bool* ok) {
  const int np = grid_of(n);
  k_angle_sums<<<np, kTB, 0, st>>>(n, g, out, s.r, np, s.part);
  k_sum_parts<3><<<1, kTB, 0, st>>>(np, s.part, s.sums);
  double a[3];
  if (cudaMemcpyAsync(a, s.sums, sizeof(a), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return false;
  const double ng = std::sqrt(a[1]), nd = std::sqrt(a[2]);
  *ok = ng > 0.0 && nd > 0.0 && -a[0] / (ng * nd) > cmax;
  return true;
}

tosolve_status threshold_density(const double* rho, long n, double vfrac, double lo, double hi, const double* grad,
                                 double theta_deg, double* out, int* accepted, void* scratch, size_t bytes,
                                 cudaStream_t st, std::string* why) {
  Scratch s;
  if (scratch_layout(n, &s, (char*)scratch) > bytes) { *why = "scratch too small"; return TOSOLVE_EINVAL; }
  const long k = (long)std::floor(vfrac * (double)n);
  k_round<<<grid_of(n), kTB, 0, st>>>(n, rho, lo, hi, s.r);
  k_keys_desc<<<grid_of(n), kTB, 0, st>>>(n, s.r, s.k0, s.i0);
  if (radix_sort(n, s, st) != cudaSuccess) { *why = "sort failed"; return TOSOLVE_ECUDA; }
  k_top_k<<<grid_of(n), kTB, 0, st>>>(n, k, s.i0, out);
  bool ok = false;
  if (!angle_ok(grad, out, s, n, std::cos(theta_deg * M_PI / 180.0), st, &ok)) {
    *why = "angle test failed";
    return TOSOLVE_ECUDA;
  }
  if (accepted) *accepted = ok ? 1 : 0;
  return TOSOLVE_OK;
}

tosolve_status threshold_gradient(const double* rho, long n, double lo, double hi, const double* grad, double vu,
                                  double vl, double theta_deg, double* out, double* alpha_out, void* scratch,
                                  size_t bytes, cudaStream_t st, std::string* why) {
  Scratch s;
  if (scratch_layout(n, &s, (char*)scratch) > bytes) { *why = "scratch too small"; return TOSOLVE_EINVAL; }
  const int nt = tiles_of(n);
  k_round<<<grid_of(n), kTB, 0, st>>>(n, rho, lo, hi, s.r);
  k_keys_alpha<<<grid_of(n), kTB, 0, st>>>(n, s.r, grad, s.k0, s.i0);
  if (radix_sort(n, s, st) != cudaSuccess) { *why = "sort failed"; return TOSOLVE_ECUDA; }
  k_grad_scan<<<nt, kTB, 0, st>>>(n, s.i0, s.r, grad, vu, vl, s.S, s.tot);
  k_scan_tot<<<1, 1024, 0, st>>>(nt, s.tot);
  // sum of grad^2 over all components: the last prefix of P
  double gl[2] = {0.0, 0.0};
  if (cudaMemcpyAsync(&gl[0], s.S + 2 * n + (n - 1), 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(&gl[1], s.tot + 2 * nt + (nt - 1), 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    *why = "gradient sums failed";
    return TOSOLVE_ECUDA;
  }
  const double gsum2 = gl[0] + gl[1];
  const int np = grid_of(n);
  k_grad_pick<<<np, kTB, 0, st>>>(n, s.k0, s.S, s.tot, nt, gsum2, std::cos(theta_deg * M_PI / 180.0), s.best);
  std::vector<long long> best(np);
  if (cudaMemcpyAsync(best.data(), s.best, np * sizeof(long long), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    *why = "candidate search failed";
    return TOSOLVE_ECUDA;
  }
  long long jb = -1;
  for (long long b : best) jb = b > jb ? b : jb;
  double alpha = 0.0;
  if (jb >= 0) {
    uint64_t key = 0;
    if (cudaMemcpyAsync(&key, s.k0 + jb, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      *why = "candidate read failed";
      return TOSOLVE_ECUDA;
    }
    std::memcpy(&alpha, &key, 8);
  }
  k_proj_step<<<grid_of(n), kTB, 0, st>>>(n, s.r, grad, alpha, out);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
    *why = "projection failed";
    return TOSOLVE_ECUDA;
  }
  if (alpha_out) *alpha_out = alpha;
  return TOSOLVE_OK;
}

}  // namespace tos
