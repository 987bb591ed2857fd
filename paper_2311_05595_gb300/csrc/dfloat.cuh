// Unevaluated pair of floats (hi + lo, |lo| <= ulp(hi)/2): about 48
// significant bits computed on the FP32 pipes, for the multigrid vectors of
// the FP32X2 preconditioner.  FP64 issues at 1/64 of the FP32 rate on this
// GPU, while the V-cycle on high-contrast densities needs more than FP32's
// 24 bits in its vector arithmetic (the FP32 operators themselves are
// enough).  Built from the classical error-free transformations:
//   TwoSum      Knuth, TAOCP vol. 2 (s + e = a + b exactly),
//   FastTwoSum  Dekker 1971 (the same for |a| >= |b|),
//   TwoProduct  with a fused multiply-add (p + e = a * b exactly),
// and the compensated dot product Dot2 of Ogita, Rump and Oishi (SIAM J.
// Sci. Comput. 26, 2005), whose result is as accurate as if computed in
// twice the working precision.  Relies on IEEE float semantics without
// reassociation (nvcc's default; fused multiply-adds are written out).
#pragma once

#include <cuda_runtime.h>

namespace tos {

struct __align__(8) dfloat {
  float hi, lo;
  dfloat() = default;
  __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr dfloat(int v) : hi((float)v), lo(0.f) {}
  __host__ __device__ constexpr dfloat(float v) : hi(v), lo(0.f) {}
  __host__ __device__ explicit dfloat(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ dfloat two_sum(float a, float b) {
  const float s = a + b;
  const float bp = s - a;
  const float ap = s - bp;
  return dfloat(s, (a - ap) + (b - bp));
}

__device__ __forceinline__ dfloat fast_two_sum(float a, float b) {
  const float s = a + b;
  return dfloat(s, b - (s - a));
}

__device__ __forceinline__ dfloat two_prod(float a, float b) {
  const float p = a * b;
  return dfloat(p, __fmaf_rn(a, b, -p));
}

__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
  dfloat s = two_sum(a.hi, b.hi);
  const dfloat t = two_sum(a.lo, b.lo);
  s = fast_two_sum(s.hi, s.lo + t.hi);
  return fast_two_sum(s.hi, s.lo + t.lo);
}

__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }

__device__ __forceinline__ dfloat operator*(float a, dfloat b) {
  const dfloat p = two_prod(a, b.hi);
  return fast_two_sum(p.hi, __fmaf_rn(a, b.lo, p.lo));
}
__device__ __forceinline__ dfloat operator*(dfloat b, float a) { return a * b; }

__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
  const dfloat p = two_prod(a.hi, b.hi);
  return fast_two_sum(p.hi, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo)));
}

__device__ __forceinline__ dfloat& operator+=(dfloat& a, dfloat b) { return a = a + b; }

// Dot2 accumulator: sum of a_k * x_k (a_k float, x_k dfloat).  The running
// sum p carries the leading part; every rounding error (of the products and
// of the additions to p) is collected in s, added once at the end.
struct Dot2 {
  float p = 0.f, s = 0.f;
  __device__ __forceinline__ void add(float a, dfloat x) {
    const dfloat h = two_prod(a, x.hi);
    const dfloat q = two_sum(p, h.hi);
    p = q.hi;
    s += q.lo + __fmaf_rn(a, x.lo, h.lo);
  }
  __device__ __forceinline__ void add(const Dot2& o) {
    const dfloat q = two_sum(p, o.p);
    p = q.hi;
    s += q.lo + o.s;
  }
  __device__ __forceinline__ dfloat value() const { return two_sum(p, s); }
};

}  // namespace tos
