// Autotuning for the batching pattern: which descriptor variant (the
// preconditioner's precision and operator kernels, its levels) solves an
// instance class fastest.  tosolve_tune times candidates on a
// representative instance through the public entry points; tosolve_tune_pick
// turns timings into a choice with a median over repeats and a minimum gain
// over the default, so that timing noise does not flip a class to a
// variant that is not really faster.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <limits>
#include <string>
#include <vector>

#include "../../include/tosolve.h"

namespace tos {
void set_last_error(const char* msg);  // the message of tosolve_last_error(NULL)
}

namespace {

constexpr double kInf = std::numeric_limits<double>::infinity();

// Median of the finite entries of v[0..n), or +inf when fewer than half are
// finite (the lower middle element for an even count of finite entries).
double median_finite(const double* v, int n) {
  std::vector<double> f;
  for (int i = 0; i < n; ++i)
    if (std::isfinite(v[i])) f.push_back(v[i]);
  if (f.empty() || 2 * (int)f.size() < n) return kInf;
  std::sort(f.begin(), f.end());
  return f[(f.size() - 1) / 2];
}

}  // namespace

extern "C" tosolve_status tosolve_tune_pick(const double* ms, int nclass, int ncand, int reps, double min_gain,
                                            int* choice) {
  if (ms == nullptr || choice == nullptr || nclass < 1 || nclass > 4096 || ncand < 1 || ncand > 64 || reps < 1 ||
      reps > 64 || !(min_gain >= 0.0 && min_gain < 1.0)) {
    tos::set_last_error("tosolve_tune_pick: NULL pointer or size / min_gain out of range");
    return TOSOLVE_EINVAL;
  }
  for (int k = 0; k < nclass; ++k) {
    std::vector<double> med(ncand);
    int best = -1;
    for (int c = 0; c < ncand; ++c) {
      med[c] = median_finite(ms + ((size_t)k * ncand + c) * reps, reps);
      if (std::isfinite(med[c]) && (best < 0 || med[c] < med[best])) best = c;
    }
    if (best > 0 && std::isfinite(med[0]) && !(med[best] < (1.0 - min_gain) * med[0])) best = 0;
    choice[k] = best;
  }
  return TOSOLVE_OK;
}

extern "C" tosolve_status tosolve_tune(const tosolve_desc* cand, int ncand, const uint8_t* mask_host,
                                       const uint8_t* elem_q1_host, const double* x_dev, const double* f_dev,
                                       int nrhs, double rtol, int maxit, int reps, void* cuda_stream,
                                       double* ms_out) {
  if (cand == nullptr || mask_host == nullptr || x_dev == nullptr || f_dev == nullptr || ms_out == nullptr ||
      ncand < 1 || ncand > 64 || reps < 1 || reps > 64 || nrhs < 1) {
    tos::set_last_error("tosolve_tune: NULL pointer, or ncand / reps outside 1..64, or nrhs < 1");
    return TOSOLVE_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  for (int i = 0; i < ncand * reps; ++i) ms_out[i] = kInf;
  for (int c = 0; c < ncand; ++c) {
    tosolve_t h = nullptr;
    const tosolve_status s = elem_q1_host ? tosolve_create_mixed(&cand[c], mask_host, elem_q1_host, st, &h)
                                          : tosolve_create(&cand[c], mask_host, st, &h);
    if (s != TOSOLVE_OK) continue;  // not offered for this instance: stays +inf
    int lv[3] = {0, 0, 0};
    if (tosolve_level_dims(h, 0, lv) != TOSOLVE_OK) {
      tosolve_destroy(h);
      continue;
    }
    const size_t ndof = 3 * (size_t)lv[0] * lv[1] * lv[2];
    double* u = nullptr;
    if (cudaMalloc(&u, ndof * nrhs * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      tosolve_destroy(h);
      tos::set_last_error("tosolve_tune: cudaMalloc of the solution buffer failed");
      return TOSOLVE_ECUDA;
    }
    bool ok = tosolve_set_densities(h, x_dev) == TOSOLVE_OK;
    for (int r = -1; ok && r < reps; ++r) {  // r = -1: the untimed warm-up solve
      ok = cudaMemsetAsync(u, 0, ndof * nrhs * sizeof(double), st) == cudaSuccess;
      tosolve_info info{};
      if (ok) ok = tosolve_solve(h, f_dev, nrhs, u, rtol, maxit, &info) == TOSOLVE_OK;
      if (ok && r >= 0) ms_out[(size_t)c * reps + r] = info.ms;
    }
    cudaStreamSynchronize(st);
    cudaFree(u);
    tosolve_destroy(h);
    cudaGetLastError();
  }
  return TOSOLVE_OK;
}
