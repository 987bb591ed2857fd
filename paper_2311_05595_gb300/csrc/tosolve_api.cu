// C ABI of the solver (declared in include/tosolve.h): validation, memory
// plan, the per-design refresh, the graph-captured PCG loop and the
// gradient.  Every device step is one of the kernels in k_*.cu.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "internal.cuh"
#include "pool.h"

using namespace tos;

struct tosolve_batch_s {
  std::vector<tosolve_t> hs;
  std::vector<int> nrhs;
  std::vector<const double*> f;
  std::vector<double*> u;
  cudaStream_t st = nullptr;
  cudaStream_t bs = nullptr;
  std::vector<cudaStream_t> branch;
  std::vector<cudaEvent_t> ev;  // per instance: ordering with the handle's stream
  cudaEvent_t evf = nullptr, evd = nullptr, t0 = nullptr, t1 = nullptr;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  double* hparams = nullptr;  // pinned {rtol^2, maxit}
  double* dparams = nullptr;
  tos::DevState* hst = nullptr;  // pinned, one per (instance, load case)
  int total = 0;
  std::string err;
};

namespace {

thread_local std::string g_err;

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      h->err = std::string(#call) + " failed: " + cudaGetErrorString(e_);            \
      return TOSOLVE_ECUDA;                                                           \
    }                                                                                 \
  } while (0)

struct Plan {
  int L = 1;
  int n = 1, m = 1;
  int Dx = 0, Dy = 0, Dz = 0;
  long ncell = 0;
  int dm = 1;     // design cells per element edge
  long ndes = 0;  // design variables
  struct Lv {
    int ex, ey, ez, Lx, Ly, Lz;
    long nn, ndof;
    int nsub;
    bool s64, s32;
  } lv[kMaxLevels];
  long nc = 0;
  int noff = 0;
  size_t bytes = 0;
};

// Degree 3: level 0 is the cubic mesh, level 1 the quadratic mesh of the
// same elements (the degree is coarsened first), and each further level
// halves the mesh.  Otherwise every level halves the mesh of the one above.
int level_degree(const tosolve_desc& d, int l) { return d.degree == 3 ? (l == 0 ? 3 : 2) : d.degree; }
int level_shift(const tosolve_desc& d, int l) { return d.degree == 3 ? (l == 0 ? 0 : l - 1) : l; }

bool divisible(const tosolve_desc& d, int levels) {
  const int s = 1 << level_shift(d, levels - 1);
  return d.nx % s == 0 && d.ny % s == 0 && d.nz % s == 0;
}

long coarse_dofs(const tosolve_desc& d, int levels) {
  const int s = 1 << level_shift(d, levels - 1);
  const long k = level_degree(d, levels - 1);
  return 3L * (k * (d.nx / s) + 1) * (k * (d.ny / s) + 1) * (k * (d.nz / s) + 1);
}

int count_offsets(int n, double rmin) {
  if (rmin <= 0.0) return 1;
  const double rc2 = (rmin * n) * (rmin * n);
  const int R = (int)std::floor(rmin * n + 1e-9);
  int cnt = 0;
  for (int k = -R; k <= R; ++k)
    for (int j = -R; j <= R; ++j)
      for (int i = -R; i <= R; ++i)
        if (i * i + j * j + k * k <= rc2 * (1.0 + 1e-12)) ++cnt;
  return cnt;
}

// Validates the descriptor and computes the level structure and the bytes
// tosolve_create allocates.  No CUDA calls.
tosolve_status plan_for(const tosolve_desc* dp, Plan* P, std::string* why) {
  if (dp == nullptr) { *why = "descriptor is NULL"; return TOSOLVE_EINVAL; }
  tosolve_desc d = *dp;
  if (d.nx < 1 || d.ny < 1 || d.nz < 1) { *why = "nx, ny, nz must be >= 1"; return TOSOLVE_EINVAL; }
  if ((long)d.nx * d.ny * d.nz > (1L << 28)) { *why = "mesh too large"; return TOSOLVE_EINVAL; }
  if (d.degree < 1 || d.degree > 3) { *why = "degree must be 1, 2 or 3"; return TOSOLVE_EINVAL; }
  if (d.family != 0 && d.family != 1) { *why = "family must be 0 (Lagrange) or 1 (serendipity)"; return TOSOLVE_EINVAL; }
  if (d.family == 1 && d.degree == 1) { *why = "the serendipity element is built for degree 2 and 3"; return TOSOLVE_EINVAL; }
  if (d.degree == 3 && d.mg_levels == 1) { *why = "degree 3 needs mg_levels >= 2 (its next level is degree 2)"; return TOSOLVE_EINVAL; }
  if (d.prolongation != 0 && d.prolongation != 1) { *why = "prolongation must be 0 or 1"; return TOSOLVE_EINVAL; }
  if (d.prolongation == 1 && d.family == 1) {
    *why = "the serendipity element takes shape-function transfers (prolongation = 0)";
    return TOSOLVE_EINVAL;
  }
  if (d.n_mr < 1 || d.n_mr > 8) { *why = "n_mr must be in 1..8"; return TOSOLVE_EINVAL; }
  if (d.d_mr != 0 && (d.d_mr < 1 || d.d_mr > d.n_mr)) { *why = "d_mr must be in 1..n_mr"; return TOSOLVE_EINVAL; }
  if (d.d_mr != 0 && d.d_mr != d.n_mr && !(d.rmin > 0.0)) {
    *why = "a coarser design grid (d_mr < n_mr) needs a projection radius rmin > 0";
    return TOSOLVE_EINVAL;
  }
  if (!(d.E0 > 0.0) || !(d.Emin > 0.0) || d.Emin > d.E0) { *why = "need 0 < Emin <= E0"; return TOSOLVE_EINVAL; }
  if (!(d.nu > -1.0 && d.nu < 0.5)) { *why = "nu must be in (-1, 0.5)"; return TOSOLVE_EINVAL; }
  if (!(d.penal >= 1.0)) { *why = "penal must be >= 1"; return TOSOLVE_EINVAL; }
  if (!(d.rmin >= 0.0) || d.rmin * d.n_mr > 16.0) { *why = "rmin*n_mr must be in [0, 16]"; return TOSOLVE_EINVAL; }
  if (d.precision != TOSOLVE_PREC_FP64 && d.precision != TOSOLVE_PREC_FP32 &&
      d.precision != TOSOLVE_PREC_TF32 && d.precision != TOSOLVE_PREC_FP32X2 &&
      d.precision != TOSOLVE_PREC_BF16 && d.precision != TOSOLVE_PREC_BF16X3 &&
      d.precision != TOSOLVE_PREC_F16X3) {
    *why = "unknown precision";
    return TOSOLVE_EINVAL;
  }
  const bool tcp = d.precision == TOSOLVE_PREC_TF32 || d.precision == TOSOLVE_PREC_BF16 ||
                   d.precision == TOSOLVE_PREC_BF16X3 || d.precision == TOSOLVE_PREC_F16X3;
  if (tcp && d.degree == 3) {
    *why = "the tensor-core preconditioners are built for degree 1 (TF32) and degree 2";
    return TOSOLVE_EINVAL;
  }
  if (tcp && d.precision != TOSOLVE_PREC_TF32 && d.degree != 2) {
    *why = "the BF16, BF16X3 and F16X3 tensor-core preconditioners are built for degree 2";
    return TOSOLVE_EINVAL;
  }
  if (d.precision == TOSOLVE_PREC_TF32 && d.degree == 1 && !tc_supported(d.n_mr)) {
    *why = "TF32 tensor-core preconditioner needs n_mr <= 2 (24 n^3 stacked rows <= 256)";
    return TOSOLVE_EINVAL;
  }
  if (tcp && d.degree == 2 && (d.family != 0 || !tc2_supported(d.n_mr))) {
    *why = "the degree-2 tensor-core preconditioner needs Lagrange elements and n_mr <= 3";
    return TOSOLVE_EINVAL;
  }
  if (d.omega != 0.0 && !(d.omega > 0.0 && d.omega < 2.0)) { *why = "omega must be in (0, 2)"; return TOSOLVE_EINVAL; }
  if (d.cycle_gamma != 0 && d.cycle_gamma != 1) { *why = "only the V-cycle (gamma = 1) is built"; return TOSOLVE_EINVAL; }
  if (d.max_rhs < 0 || d.max_rhs > 64) { *why = "max_rhs must be in 0..64"; return TOSOLVE_EINVAL; }
  if (d.inner_its < 0 || d.inner_its > 64) { *why = "inner_its must be in 0..64"; return TOSOLVE_EINVAL; }
  if (d.inner_its > 0 && (d.degree != 2 || d.precision == TOSOLVE_PREC_FP64 || d.precision == TOSOLVE_PREC_FP32X2 ||
                          d.mg_levels == 1)) {
    *why = "inner FP32 iterations need degree 2, an FP32-vector precision and a V-cycle (mg_levels != 1)";
    return TOSOLVE_EINVAL;
  }
  if (d.smoother != 0 && d.smoother != 1) { *why = "smoother is 0 (Jacobi) or 1 (Chebyshev)"; return TOSOLVE_EINVAL; }
  if (d.smoother == 1 && (d.degree < 2 || d.precision == TOSOLVE_PREC_FP32X2)) {
    *why = "Chebyshev smoothing needs degree 2 or 3 and a precision other than FP32X2";
    return TOSOLVE_EINVAL;
  }
  if (d.cheb_degree < 0 || d.cheb_degree > 4) { *why = "cheb_degree must be in 0..4"; return TOSOLVE_EINVAL; }
  int L = d.mg_levels;
  if (L == 0) {
    L = d.degree == 3 ? 2 : 1;
    while (L < kMaxLevels && divisible(d, L + 1) && coarse_dofs(d, L) > 1500) ++L;
  }
  if (L < 1 || L > kMaxLevels) { *why = "mg_levels must be in 1..8"; return TOSOLVE_EINVAL; }
  if (!divisible(d, L)) { *why = "nx, ny, nz must be divisible by 2^(mg_levels-1)"; return TOSOLVE_EINVAL; }
  if (d.n_mr * (1 << level_shift(d, L - 1)) > 1024) { *why = "too many levels for n_mr"; return TOSOLVE_EINVAL; }
  P->L = L;
  P->n = d.n_mr;
  P->m = d.n_mr * d.n_mr * d.n_mr;
  P->Dx = d.n_mr * d.nx;
  P->Dy = d.n_mr * d.ny;
  P->Dz = d.n_mr * d.nz;
  P->ncell = (long)P->Dx * P->Dy * P->Dz;
  P->dm = d.d_mr != 0 ? d.d_mr : d.n_mr;
  P->ndes = (long)P->dm * P->dm * P->dm * d.nx * d.ny * d.nz;
  P->noff = count_offsets(d.n_mr, d.rmin);
  const bool fp32 = d.precision != TOSOLVE_PREC_FP64;
  const bool tf32 = d.precision == TOSOLVE_PREC_TF32 && L > 1 && d.degree == 1;
  const bool tc2 = tcp && L > 1 && d.degree == 2;
  const bool x2 = d.precision == TOSOLVE_PREC_FP32X2;
  const int maxrhs = d.max_rhs > 0 ? d.max_rhs : 1;
  size_t B = 0;
  size_t keB = 0;
  for (int l = 0; l < L; ++l) {
    Plan::Lv& v = P->lv[l];
    const int sh = level_shift(d, l), kl = level_degree(d, l);
    v.ex = d.nx >> sh; v.ey = d.ny >> sh; v.ez = d.nz >> sh;
    v.Lx = kl * v.ex + 1; v.Ly = kl * v.ey + 1; v.Lz = kl * v.ez + 1;
    v.nn = (long)v.Lx * v.Ly * v.Lz;
    v.ndof = 3 * v.nn;
    v.nsub = d.n_mr << sh;
    const bool coarsest = l == L - 1;
    if (d.degree >= 2) {  // element matrices instead of stencils
      const size_t E = (size_t)v.ex * v.ey * v.ez;
      const size_t dd = kl == 3 ? (size_t)kDD3 : (elem_sym(d.family, kl, v.nsub) ? (size_t)kPS2 : (size_t)kDD2);
      const size_t tsz = (fp32 && !x2) ? 4 : 8;
      v.s64 = v.s32 = false;
      B += v.ndof + v.ndof * 8 + 4 * v.ndof * tsz;  // mask, dinv64, b v r z
      if (fp32) B += v.ndof * 4;
      B += coarsest ? E * dd * 8 : E * dd * (8 + (fp32 && !(tc2 && l == 0) ? 4 : 0));
      if (d.family == 1 && (!coarsest || l == 0)) {  // compact copies of the serendipity levels
        const size_t dp = kl == 3 ? 96 : 60;
        B += E * dp * dp * (8 + (fp32 && !coarsest ? 4 : 0));
      }
      if (l > 0) B += E * kNM2 * 8;
      continue;
    }
    v.s64 = (l == 0) || !fp32 || coarsest || x2;  // FP32X2: every level formed in FP64
    v.s32 = fp32 && !coarsest && !(tf32 && l == 0);  // TF32: level 0 runs on tensor cores
    const size_t tsz = (fp32 && !x2) ? 4 : 8;
    B += v.ndof;  // mask
    if (v.s64) B += op_len(v.nn) * 8 + v.ndof * 8;
    if (v.s32) B += op_len(v.nn) * 4 + v.ndof * 4;
    B += 4 * v.ndof * tsz;  // b, v, r, z
  }
  {
    int ex[kMaxLevels], ey[kMaxLevels], ez[kMaxLevels];
    for (int l = 0; l < L; ++l) { ex[l] = P->lv[l].ex; ey[l] = P->lv[l].ey; ez[l] = P->lv[l].ez; }
    keB = slab_scratch_bytes(ex, ey, ez, L - 1 > 0 ? L - 1 : 1);
    keB += keB / (kSym * 8) * 27 * 8;  // moments of a slab
    const Plan::Lv& c = P->lv[L - 1];
    keB += (size_t)c.ex * c.ey * c.ez * (kSym + 27) * 8;  // coarsest level's own
    if (d.degree == 2)  // apply results + tables instead of the slab scratch
      keB = (size_t)ex[0] * ey[0] * ez[0] * kD2 * 8 + ((size_t)P->m + kNM2) * kDD2 * 8;
    if (d.degree == 3)  // and the gradients the cubic tables are built from
      keB = (size_t)ex[0] * ey[0] * ez[0] * kD3 * 8 + ((size_t)P->m * kDD3 + (size_t)kNM2 * kDD2) * 8 +
            (size_t)P->m * 64 * 64 * 3 * 8;
  }
  P->nc = P->lv[L - 1].ndof;
  if (P->nc > kMaxCoarse) { *why = "coarsest level too large for the dense solve: add levels"; return TOSOLVE_EINVAL; }
  const long ndof0 = P->lv[0].ndof;
  B += keB;
  B += (size_t)P->ncell * 8 * 5;                      // rho, w, invom, gtmp, staging x
  B += (size_t)P->noff * (sizeof(int4) + 8);
  B += (size_t)P->m * (576 + kSym) * 8 + 27 * kSym * 8;  // tables
  const long nc = P->nc;
  B += (size_t)(2 * nc * nc + 2 * nc * kNB + kNB * kNB) * 8;  // coarse operator, inverse, sweeps
  B += (size_t)ndof0 * 8 * 7;                         // u r p q f tmpa tmpb
  B += (size_t)ndof0 * 8 * 2 * maxrhs;                // host-step staging f, u
  B += 4 * kMaxPart * 8 + sizeof(DevState) + (size_t)P->ndes * 8 * 2;
  B += (size_t)ndof0 + 2 * (size_t)d.nx * d.ny * d.nz + (size_t)P->ndes;  // fixing (Sec. 6.1)
  B += ((size_t)(P->lv[0].nn + kTN - 1) / kTN + 1) * sizeof(int);  // level-0 tile order
  if (tf32) {
    const size_t E0 = (size_t)d.nx * d.ny * d.nz;
    B += E0 * (P->m + 24) * 4 + (size_t)P->m * 576 * 4 + P->lv[0].ndof * 4;
  }
  if (d.inner_its > 0) B += 4 * (size_t)P->lv[0].ndof * 4;  // inner PCG vectors
  if (d.smoother == 1)  // step difference vectors, coefficients, Lanczos scratch
    for (int l = 0; l + 1 < L; ++l) B += (size_t)P->lv[l].ndof * 8 + 16 * 12 + 64 * 8;
  if (tc2) {  // weights, element results and the table image of the tensor-core level
    const size_t E0 = (size_t)d.nx * d.ny * d.nz;
    B += E0 * (P->m + tc2_result_stride() + 1) * 4 + tc2_pack_bytes(tc2_mode_of(d.precision), (long)E0) +
         tc2_image_bytes(tc2_mode_of(d.precision), P->m) + (size_t)P->m * 576 * 8 +
         (size_t)P->lv[0].ndof * 4 + (size_t)P->lv[0].nn / 2 +  // the mixed fold's raw assembly, vertex masks
         (E0 * kQ1Sym + 4) * 4;  // FP32 trilinear vertex blocks (at most every element trilinear)
  }
  P->bytes = B;
  return TOSOLVE_OK;
}

// Device memory from the library's pool, ordered on the handle's stream and
// complete before it is returned (so any stream may use it).
template <typename T>
cudaError_t dalloc(tosolve_s* h, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  void* q = nullptr;
  cudaError_t e = pool_alloc(&q, count * sizeof(T), h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (e == cudaSuccess) {
    *p = static_cast<T*>(q);
    h->bytes += count * sizeof(T);
  }
  return e;
}

void free_all(tosolve_s* h) {
  cudaStream_t fs = h->st;
  auto F = [fs](void* p) { if (p) pool_free(p, fs); };
  for (int l = 0; l < kMaxLevels; ++l) {
    Level& L = h->lv[l];
    F(L.mask); F(L.S64); F(L.S32); F(L.dinv64); F(L.dinv32); F(L.b); F(L.v); F(L.r); F(L.z);
    F(L.K64); F(L.K32); F(L.Kc64); F(L.Kc32); F(L.tl_buf); F(L.tcnt_buf);
  }
  F(h->rho); F(h->w); F(h->invom); F(h->foff); F(h->fwgt); F(h->gtmp);
  F(h->Yq); F(h->Mq); F(h->Mqc); F(h->slv0); F(h->fix0);
  F(h->base0); F(h->ecls); F(h->efix); F(h->xfix); F(h->ptab); F(h->ptab3);
  F(h->tab64); F(h->tabsym64); F(h->cmom64); F(h->KT32); F(h->w32); F(h->Ye); F(h->tcimg); F(h->Y2); F(h->Ke); F(h->Kec); F(h->Mom); F(h->Momc);
  F(h->inner.e); F(h->inner.ri); F(h->inner.pi); F(h->inner.qi);
  F(h->el2); F(h->sl2); F(h->el1); F(h->tab64q1); F(h->tcyraw); F(h->tck1v); F(h->tcvnb); F(h->tcpack); F(h->tcscale);
  F(h->lz); F(h->lmax);
  F(h->Ad); F(h->Wp); F(h->Vp); F(h->Pg); F(h->Ainv);
  F(h->u); F(h->r); F(h->p); F(h->q); F(h->f); F(h->tmpa); F(h->tmpb); F(h->part); F(h->ds);
  F(h->cnt);
  F(h->hx); F(h->hf); F(h->hu); F(h->hg);
  if (fs) cudaStreamSynchronize(fs);
  if (h->hs) cudaFreeHost(h->hs);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->graph) cudaGraphDestroy(h->graph);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  if (h->evf) cudaEventDestroy(h->evf);
  if (h->evj) cudaEventDestroy(h->evj);
  if (h->st2) cudaStreamDestroy(h->st2);
  if (h->own_stream && h->st) cudaStreamDestroy(h->st);
}

// Arithmetic of the multigrid vectors for the handle's precision.
int vt_of(const tosolve_s* h) {
  switch (h->d.precision) {
    case TOSOLVE_PREC_FP64: return kVtF64;
    case TOSOLVE_PREC_FP32X2: return kVtDF;
    default: return kVtF32;
  }
}

// Appends the PCG loop of one right-hand side to the stream capture active
// on cs: prep, r0 = f - K u0 and the convergence test; a device-side while
// node whose body (captured on bs) is z = B r (multigrid cycle), direction,
// q = K p, update and test; then the FP64 true residual.  The loop runs
// without host round trips.
cudaError_t append_solve(tosolve_s* h, cudaStream_t cs, cudaStream_t bs) {
  const int vt = vt_of(h);
  Level& L0 = h->lv[0];
  const int np = h->np;
  double* part0 = h->part;
  double* part1 = h->part + kMaxPart;
  double* part2 = h->part + 2 * kMaxPart;
  double* part3 = h->part + 3 * kMaxPart;
  if (h->mixed) launch_q2_fold(L0, h->slv0, h->f, cs);  // f <- T^T f
  launch_cg_prep(L0, h->f, h->u, part0, np, cs);
  cudaStreamCaptureStatus cst;
  cudaGraph_t cgraph = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cgraph, &deps, nullptr, &ndeps);
  cudaGraphConditionalHandle hc = 0;
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hc, cgraph, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) {
    launch_cg_residual(vt, L0, h->d.omega, h->f, h->u, h->r, 1, part1, part0, np, h->ds, h->cnt, hc,
                       1, cs);
    e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cgraph, &deps, nullptr, &ndeps);
  }
  cudaGraphNode_t cnode = nullptr;
  cudaGraph_t body = nullptr;
  if (e == cudaSuccess) {
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = hc;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    e = cudaGraphAddNode(&cnode, cgraph, deps, nullptr, ndeps, &cp);
    if (e == cudaSuccess) body = cp.conditional.phGraph_out[0];
  }
  if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(cs, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies);
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    const CgDots cd{h->r, h->q, part2, part3, h->ds, h->cnt + 1};
    if (h->inner.its > 0) {
      launch_inner_pcg(h->lv, h->L, h->d.omega, h->Ainv, h->tc, h->inner, part2, part3, h->ds, h->cnt + 1, bs);
      launch_cg_dots_rz(vt, L0, h->r, h->q, part2, part3, np, h->ds, h->cnt + 1, bs);
    } else if (!launch_vcycle(vt, h->lv, h->L, h->d.omega, 1, h->Ainv, h->tc, bs, &cd)) {
      launch_cg_dots_rz(vt, L0, h->r, h->q, part2, part3, np, h->ds, h->cnt + 1, bs);
    }
    launch_cg_dir(vt, L0, h->p, np, h->ds, bs);
    launch_cg_apply(L0, h->p, h->q, part0, np, h->ds, h->cnt + 2, bs);
    launch_cg_update(vt, L0, h->d.omega, h->u, h->r, h->p, h->q, part1, np, h->ds, h->cnt + 3, hc, 1,
                     bs);
    cudaGraph_t bo = nullptr;
    e = cudaStreamEndCapture(bs, &bo);
  }
  if (e == cudaSuccess) {
    launch_cg_residual(vt, L0, h->d.omega, h->f, h->u, h->tmpa, 2, part1, part0, np, h->ds, h->cnt,
                       hc, 0, cs);
    if (h->mixed) launch_q2_expand(L0, h->slv0, h->u, cs);  // u <- T u
  }
  return e;
}

// The handle's own graph: one right-hand side, launched by tosolve_solve.
tosolve_status build_graph(tosolve_s* h) {
  cudaStream_t cs = h->st;
  cudaStream_t bs = nullptr;
  CK(cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaStreamDestroy(bs);
    h->err = std::string("begin capture: ") + cudaGetErrorString(e);
    return TOSOLVE_ECUDA;
  }
  e = append_solve(h, cs, bs);
  cudaError_t e2 = cudaStreamEndCapture(cs, &g);
  cudaStreamDestroy(bs);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    h->err = std::string("graph capture failed: ") + cudaGetErrorString(e != cudaSuccess ? e : e2);
    cudaGetLastError();
    return TOSOLVE_ECUDA;
  }
  h->graph = g;
  CK(cudaGraphInstantiate(&h->gexec, g, 0));
  h->graph_ready = true;
  return TOSOLVE_OK;
}

constexpr int kChebLanczos = 8;  // Lanczos steps of the lambda_max estimate

tosolve_status set_err(tosolve_t h, tosolve_status s, const char* msg) {
  if (h) h->err = msg;
  g_err = msg;
  return s;
}

}  // namespace

extern "C" {

tosolve_status tosolve_footprint(const tosolve_desc* desc, size_t* bytes) {
  Plan P;
  std::string why;
  const tosolve_status s = plan_for(desc, &P, &why);
  if (s != TOSOLVE_OK) { g_err = why; return s; }
  if (bytes == nullptr) { g_err = "bytes is NULL"; return TOSOLVE_EINVAL; }
  *bytes = P.bytes;
  return TOSOLVE_OK;
}

// Degree-2 shape function a (lattice position a % 3, a / 3 % 3, a / 9) at
// reference point x: the tensor-product Lagrange basis (family 0) or the
// 20-node serendipity basis (family 1; zero at face and element centres).
static double quad_shape(int family, int a, const double x[3]) {
  const int c[3] = {a % 3 - 1, (a / 3) % 3 - 1, a / 9 - 1};
  if (family == 0) {
    double v = 1.0;
    for (int q = 0; q < 3; ++q)
      v *= c[q] == -1 ? 0.5 * x[q] * (x[q] - 1.0) : (c[q] == 0 ? 1.0 - x[q] * x[q] : 0.5 * x[q] * (x[q] + 1.0));
    return v;
  }
  const int nmid = (c[0] == 0) + (c[1] == 0) + (c[2] == 0);
  if (nmid >= 2) return 0.0;
  if (nmid == 0)
    return (1.0 + x[0] * c[0]) * (1.0 + x[1] * c[1]) * (1.0 + x[2] * c[2]) *
           (x[0] * c[0] + x[1] * c[1] + x[2] * c[2] - 2.0) / 8.0;
  double v = 0.25;
  for (int q = 0; q < 3; ++q) v *= c[q] == 0 ? 1.0 - x[q] * x[q] : 1.0 + x[q] * c[q];
  return v;
}

static tosolve_status create_impl(const tosolve_desc* desc, const uint8_t* mask_host,
                                  const uint8_t* elem_q1, void* cuda_stream, tosolve_t* out) {
  if (out == nullptr) { g_err = "out is NULL"; return TOSOLVE_EINVAL; }
  *out = nullptr;
  Plan P;
  std::string why;
  tosolve_status s = plan_for(desc, &P, &why);
  if (s != TOSOLVE_OK) { g_err = why; return s; }
  if (mask_host == nullptr) { g_err = "mask is NULL"; return TOSOLVE_EINVAL; }
  tosolve_s* h = new (std::nothrow) tosolve_s();
  if (h == nullptr) { g_err = "host allocation failed"; return TOSOLVE_ENOMEM; }
  h->d = *desc;
  // damped Jacobi: 0.5 (Sec. 7 intro), which needs lambda_max(D^-1 A) < 4.
  // Measured on these elements: Lagrange degree 2 3.2, degree 3 4.0,
  // serendipity degree 2 5.3, degree 3 5.0; so 0.4 for cubic Lagrange and
  // 0.3 for serendipity (about 1.6 / lambda_max)
  if (h->d.omega == 0.0) h->d.omega = h->d.family == 1 ? 0.3 : (h->d.degree >= 2 ? 0.4 : 0.5);
  // Chebyshev: each level's D^-1 is divided by theta at set-up, so the first
  // step of every smoothing sweep is D^-1 r with weight 1
  if (h->d.smoother == 1) {
    h->d.omega = 1.0;
    if (h->d.cheb_degree == 0) h->d.cheb_degree = 2;
  }
  if (h->d.cycle_gamma == 0) h->d.cycle_gamma = 1;
  if (h->d.max_rhs == 0) h->d.max_rhs = 1;
  h->d.d_mr = P.dm;
  h->ndes = P.ndes;
  h->d.mg_levels = P.L;
  h->L = P.L;
  h->m = P.m;
  h->Dx = P.Dx; h->Dy = P.Dy; h->Dz = P.Dz;
  h->ncell = (int)P.ncell;
  h->noff = P.noff;
  h->nc = (int)P.nc;
  const bool fp32 = h->d.precision != TOSOLVE_PREC_FP64;
  const bool tf32 = h->d.precision == TOSOLVE_PREC_TF32 && P.L > 1 && h->d.degree == 1;
  const bool tc2 = (h->d.precision == TOSOLVE_PREC_TF32 || h->d.precision == TOSOLVE_PREC_BF16 ||
                    h->d.precision == TOSOLVE_PREC_BF16X3 || h->d.precision == TOSOLVE_PREC_F16X3) &&
                   P.L > 1 && h->d.degree == 2;
  auto fail = [&](tosolve_status st) {
    free_all(h);
    g_err = h->err;
    delete h;
    return st;
  };
#define CKC(call)                                                                     \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      h->err = std::string(#call) + " failed: " + cudaGetErrorString(e_);             \
      cudaGetLastError();                                                             \
      return fail(e_ == cudaErrorMemoryAllocation ? TOSOLVE_ENOMEM : TOSOLVE_ECUDA);  \
    }                                                                                 \
  } while (0)
  CKC(cudaGetDevice(&h->dev));
  if (cuda_stream == nullptr) {
    // a blocking stream: ordered with the legacy default stream
    CKC(cudaStreamCreate(&h->st));
    h->own_stream = true;
  } else {
    h->st = (cudaStream_t)cuda_stream;
  }
  cudaStream_t st = h->st;
  // levels and masks
  std::vector<uint8_t> mask(mask_host, mask_host + P.lv[0].ndof);
  std::vector<uint8_t> slv;
  if (elem_q1 != nullptr) {  // nodes slaved to their vertices; level 0 treats them as fixed
    const Plan::Lv& v = P.lv[0];
    slv.assign(v.nn, 0);
    for (int ez = 0; ez < v.ez; ++ez)
      for (int ey = 0; ey < v.ey; ++ey)
        for (int ex = 0; ex < v.ex; ++ex) {
          if (!elem_q1[ex + (long)v.ex * (ey + (long)v.ey * ez)]) continue;
          for (int c = 0; c < 3; ++c)
            for (int b = 0; b < 3; ++b)
              for (int a = 0; a < 3; ++a)
                if ((a | b | c) & 1)
                  slv[(2 * ex + a) + (long)v.Lx * ((2 * ey + b) + (long)v.Ly * (2 * ez + c))] = 1;
        }
    h->mixed = true;
    CKC(dalloc(h, &h->slv0, v.nn));
    CKC(cudaMemcpyAsync(h->slv0, slv.data(), v.nn, cudaMemcpyHostToDevice, st));
    // element lists: triquadratic ones (with the masks of their slaved local
    // nodes) and trilinear ones, each ascending
    std::vector<int> l2, l1;
    std::vector<uint32_t> m2;
    for (int ez = 0; ez < v.ez; ++ez)
      for (int ey = 0; ey < v.ey; ++ey)
        for (int ex = 0; ex < v.ex; ++ex) {
          const long e = ex + (long)v.ex * (ey + (long)v.ey * ez);
          if (elem_q1[e]) {
            l1.push_back((int)e);
            continue;
          }
          uint32_t msk = 0;
          for (int a = 0; a < 27; ++a)
            if (slv[(2 * ex + a % 3) + (long)v.Lx * ((2 * ey + (a / 3) % 3) + (long)v.Ly * (2 * ez + a / 9))])
              msk |= 1u << a;
          l2.push_back((int)e);
          m2.push_back(msk);
        }
    h->ne2 = (long)l2.size();
    h->ne1 = (long)l1.size();
    CKC(dalloc(h, &h->el2, l2.size() + 1));
    CKC(dalloc(h, &h->sl2, m2.size() + 1));
    CKC(dalloc(h, &h->el1, l1.size() + 1));
    if (!l2.empty()) {
      CKC(cudaMemcpyAsync(h->el2, l2.data(), l2.size() * sizeof(int), cudaMemcpyHostToDevice, st));
      CKC(cudaMemcpyAsync(h->sl2, m2.data(), m2.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
    }
    if (!l1.empty())
      CKC(cudaMemcpyAsync(h->el1, l1.data(), l1.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    CKC(cudaStreamSynchronize(st));  // the host vectors go out of scope
    CKC(dalloc(h, &h->fix0, v.ndof));
    CKC(cudaMemcpyAsync(h->fix0, mask.data(), v.ndof, cudaMemcpyHostToDevice, st));
    for (long nd = 0; nd < v.nn; ++nd)
      if (slv[nd]) mask[3 * nd] = mask[3 * nd + 1] = mask[3 * nd + 2] = 1;
  }
  // serendipity: no node at face and element centres, held at 0 on every level
  // (degree k lattice: two or three coordinates inside an element edge)
  auto hold_absent = [&](const Plan::Lv& v, int k, std::vector<uint8_t>& m) {
    if (h->d.family != 1) return;
    for (long nd = 0; nd < v.nn; ++nd) {
      const long i = nd % v.Lx, j = (nd / v.Lx) % v.Ly, l = nd / ((long)v.Lx * v.Ly);
      if ((i % k != 0) + (j % k != 0) + (l % k != 0) >= 2) m[3 * nd] = m[3 * nd + 1] = m[3 * nd + 2] = 1;
    }
  };
  hold_absent(P.lv[0], level_degree(h->d, 0), mask);
  h->free_dofs = 0;
  for (uint8_t m : mask) h->free_dofs += m == 0;
  h->free_base = h->free_dofs;
  {  // level-0 mask before any suppression, and the fixing workspace
    const size_t E0 = (size_t)P.lv[0].ex * P.lv[0].ey * P.lv[0].ez;
    CKC(dalloc(h, &h->base0, P.lv[0].ndof));
    CKC(cudaMemcpyAsync(h->base0, mask.data(), P.lv[0].ndof, cudaMemcpyHostToDevice, st));
    CKC(dalloc(h, &h->ecls, E0));
    CKC(dalloc(h, &h->efix, E0));
    CKC(dalloc(h, &h->xfix, P.ndes));
    CKC(cudaMemsetAsync(h->xfix, 0, P.ndes, st));
  }
  for (int l = 0; l < P.L; ++l) {
    const Plan::Lv& v = P.lv[l];
    Level& L = h->lv[l];
    L.ex = v.ex; L.ey = v.ey; L.ez = v.ez;
    L.Lx = v.Lx; L.Ly = v.Ly; L.Lz = v.Lz;
    L.nn = (int)v.nn; L.ndof = (int)v.ndof;
    L.nsub = v.nsub;
    L.h = (double)(1 << level_shift(h->d, l));
    L.op64 = !fp32 || l == P.L - 1;
    CKC(dalloc(h, &L.mask, v.ndof));
    CKC(cudaMemcpyAsync(L.mask, mask.data(), v.ndof, cudaMemcpyHostToDevice, st));
    if (l == 0) {  // storage of the tile order used after a suppression
      CKC(dalloc(h, &L.tl_buf, (v.nn + kTN - 1) / kTN));
      CKC(dalloc(h, &L.tcnt_buf, 1));
    }
    if (v.s64) {  // padding coefficients of the last tile stay zero
      CKC(dalloc(h, &L.S64, op_len(v.nn)));
      CKC(cudaMemsetAsync(L.S64, 0, op_len(v.nn) * sizeof(double), st));
      CKC(dalloc(h, &L.dinv64, v.ndof));
    }
    if (v.s32) {
      CKC(dalloc(h, &L.S32, op_len(v.nn)));
      CKC(cudaMemsetAsync(L.S32, 0, op_len(v.nn) * sizeof(float), st));
      CKC(dalloc(h, &L.dinv32, v.ndof));
    }
    if (tf32 && l == 0) CKC(dalloc(h, &L.dinv32, v.ndof));
    L.k = level_degree(h->d, l);
    if (L.k >= 2) {  // element matrices; the coarsest level's go to Kec
      const size_t E = (size_t)v.ex * v.ey * v.ez;
      L.sym = elem_sym(h->d.family, L.k, v.nsub);
      const size_t dd = elem_stride(L);
      CKC(dalloc(h, &L.dinv64, v.ndof));
      if (fp32) CKC(dalloc(h, &L.dinv32, v.ndof));
      if (l + 1 < P.L || l == 0) CKC(dalloc(h, &L.K64, E * dd));  // level 0: the CG's K
      if (l == 0 && elem_q1 != nullptr)  // trilinear slots: only their vertex blocks are ever written
        CKC(cudaMemsetAsync(L.K64, 0, E * dd * sizeof(double), st));
      if (l + 1 < P.L && fp32 && !(tc2 && l == 0)) CKC(dalloc(h, &L.K32, E * dd));  // tensor cores: no level-0 copy
      if (h->d.family == 1) {  // compact copies for the apply
        const size_t dp = L.k == 3 ? 96 : 60;
        if (L.K64) CKC(dalloc(h, &L.Kc64, E * dp * dp));
        if (L.K32) CKC(dalloc(h, &L.Kc32, E * dp * dp));
      }
    }
    const size_t tsz = vt_of(h) == kVtF32 ? 4 : 8;
    void** vecs[5] = {&L.b, &L.v, &L.r, &L.z, &L.d};
    const int nv = (h->d.smoother == 1 && l + 1 < P.L) ? 5 : 4;
    for (int q = 0; q < nv; ++q) {
      char* p = nullptr;
      CKC(dalloc(h, &p, v.ndof * tsz));
      CKC(cudaMemsetAsync(p, 0, v.ndof * tsz, st));
      *vecs[q] = p;
    }
    if (nv == 5) {  // Chebyshev coefficients of steps 2..4
      L.cheb = h->d.cheb_degree;
      CKC(dalloc(h, &L.cheb64, 8));
      CKC(dalloc(h, &L.cheb32, 8));
    }
    if (l + 1 < P.L && L.k == 3) {
      // degree 3 -> 2 on the same elements: a quadratic DOF is fixed iff
      // every cubic DOF of that component at its place is fixed (per axis a
      // vertex coordinate 2I meets 3I, a midpoint 2I + 1 meets 3I + 1 and
      // 3I + 2 inside the same edge)
      const Plan::Lv& c = P.lv[l + 1];
      std::vector<uint8_t> cm(c.ndof);
      auto span = [](int I, int& a, int& b) {
        if (I % 2 == 0) { a = b = 3 * I / 2; } else { a = 3 * (I - 1) / 2 + 1; b = a + 1; }
      };
      for (int K = 0; K < c.Lz; ++K)
        for (int J = 0; J < c.Ly; ++J)
          for (int I = 0; I < c.Lx; ++I) {
            int i0, i1, j0, j1, k0, k1;
            span(I, i0, i1);
            span(J, j0, j1);
            span(K, k0, k1);
            const long cn = I + (long)c.Lx * (J + (long)c.Ly * K);
            for (int q = 0; q < 3; ++q) {
              bool all = true;
              for (int kk = k0; kk <= k1; ++kk)
                for (int jj = j0; jj <= j1; ++jj)
                  for (int ii = i0; ii <= i1; ++ii)
                    all = all && mask[3 * (ii + (long)v.Lx * (jj + (long)v.Ly * kk)) + q] != 0;
              cm[3 * cn + q] = all ? 1 : 0;
            }
          }
      hold_absent(c, 2, cm);
      mask.swap(cm);
    } else if (l + 1 < P.L) {  // coarse DOF fixed iff the coincident fine DOF is fixed
      const Plan::Lv& c = P.lv[l + 1];
      std::vector<uint8_t> cm(c.ndof);
      for (int K = 0; K < c.Lz; ++K)
        for (int J = 0; J < c.Ly; ++J)
          for (int I = 0; I < c.Lx; ++I) {
            const long cn = I + (long)c.Lx * (J + (long)c.Ly * K);
            const long fn = 2 * I + (long)v.Lx * (2 * J + (long)v.Ly * 2 * K);
            for (int q = 0; q < 3; ++q) cm[3 * cn + q] = mask[3 * fn + q];
          }
      hold_absent(c, 2, cm);
      mask.swap(cm);
    }
  }
  if (h->mixed) {
    Level& L0 = h->lv[0];
    L0.el2 = h->el2;
    L0.ne2 = h->ne2;
    L0.sl2 = h->sl2;
    L0.el1 = h->el1;
    L0.ne1 = h->ne1;
    // the trilinear elements' subcell table (Sec. 3.3) at the level-0 size
    CKC(dalloc(h, &h->tab64q1, (size_t)P.m * 576));
    launch_subcell_table(P.n, h->d.nu, L0.h, h->tab64q1, st);
  }
  // tables (Sec. 3.3: the subcell matrices are computed once)
  if (h->d.degree >= 2) {
    if (h->d.degree == 3) {
      double* gscr = nullptr;
      CKC(dalloc(h, &h->tab64, (size_t)P.m * kDD3));
      CKC(dalloc(h, &gscr, (size_t)P.m * 64 * 64 * 3));
      launch_q3_subcell_table(P.n, h->d.nu, 1.0, h->d.family, gscr, h->tab64, st);
      CKC(cudaStreamSynchronize(st));
      pool_free(gscr, st);
      // degree 3 -> 2 transfer: the 27 quadratic shape functions (Lagrange or
      // serendipity) at the 64 cubic nodes of an element
      std::vector<float> W(27 * 64, 0.f);
      for (int a = 0; a < 27; ++a) {
        const int c[3] = {a % 3 - 1, (a / 3) % 3 - 1, a / 9 - 1};
        const int nmid = (c[0] == 0) + (c[1] == 0) + (c[2] == 0);
        if (h->d.family == 1 && nmid >= 2) continue;
        for (int f = 0; f < 64; ++f) {
          const double x[3] = {-1.0 + 2.0 * (f % 4) / 3.0, -1.0 + 2.0 * ((f / 4) % 4) / 3.0,
                               -1.0 + 2.0 * (f / 16) / 3.0};
          W[a * 64 + f] = (float)quad_shape(h->d.family, a, x);
        }
      }
      CKC(dalloc(h, &h->ptab3, W.size()));
      CKC(cudaMemcpyAsync(h->ptab3, W.data(), W.size() * sizeof(float), cudaMemcpyHostToDevice, st));
      h->lv[1].ptab = h->ptab3;
    } else {
      CKC(dalloc(h, &h->tab64, (size_t)P.m * kDD2));
      launch_q2_subcell_table(P.n, h->d.nu, 1.0, h->d.family, h->tab64, st);
    }
    CKC(dalloc(h, &h->cmom64, (size_t)kNM2 * kDD2));
    launch_q2_moment_basis(h->d.nu, h->d.family, h->cmom64, st);
    if (h->d.family == 1 || h->d.prolongation == 0) {
      // shape-function transfers: the 27 coarse shape functions at the 125
      // quarter points of a coarse element (always for the serendipity
      // element; for degree-2 Lagrange unless linear lattice interpolation is
      // asked for)
      std::vector<float> W(27 * 125, 0.f);
      auto lag1 = [](int j, double x) {  // quadratic Lagrange basis on -1, 0, 1
        return j == 0 ? 0.5 * x * (x - 1.0) : (j == 1 ? 1.0 - x * x : 0.5 * x * (x + 1.0));
      };
      for (int a = 0; a < 27; ++a) {
        const int c[3] = {a % 3 - 1, (a / 3) % 3 - 1, a / 9 - 1};
        const int nmid = (c[0] == 0) + (c[1] == 0) + (c[2] == 0);
        if (h->d.family == 1 && nmid >= 2) continue;
        for (int f = 0; f < 125; ++f) {
          const double x[3] = {-1.0 + 0.5 * (f % 5), -1.0 + 0.5 * ((f / 5) % 5), -1.0 + 0.5 * (f / 25)};
          double v;
          if (h->d.family == 0) {
            v = lag1(a % 3, x[0]) * lag1((a / 3) % 3, x[1]) * lag1(a / 9, x[2]);
          } else if (nmid == 0) {
            v = (1.0 + x[0] * c[0]) * (1.0 + x[1] * c[1]) * (1.0 + x[2] * c[2]) *
                (x[0] * c[0] + x[1] * c[1] + x[2] * c[2] - 2.0) / 8.0;
          } else {
            v = 0.25;
            for (int q = 0; q < 3; ++q) v *= c[q] == 0 ? 1.0 - x[q] * x[q] : 1.0 + x[q] * c[q];
          }
          W[a * 125 + f] = (float)v;
        }
      }
      CKC(dalloc(h, &h->ptab, W.size()));
      CKC(cudaMemcpyAsync(h->ptab, W.data(), W.size() * sizeof(float), cudaMemcpyHostToDevice, st));
      // into every degree-2 level that halves the mesh of the level above
      for (int l = (h->d.degree == 3 ? 2 : 1); l < P.L; ++l) {
        h->lv[l].ptab = h->ptab;
        h->lv[l].lag = h->d.family == 0;
      }
    }
    const Plan::Lv& v0 = P.lv[0];
    CKC(dalloc(h, &h->Yq, (size_t)v0.ex * v0.ey * v0.ez * (h->d.degree == 3 ? kD3 : kD2)));
    for (int l = 0; l < P.L; ++l) h->lv[l].Y = h->Yq;
  } else {
    CKC(dalloc(h, &h->tab64, (size_t)P.m * 576));
    CKC(dalloc(h, &h->tabsym64, (size_t)P.m * kSym));
    CKC(dalloc(h, &h->cmom64, 27 * kSym));
    launch_subcell_table(P.n, h->d.nu, 1.0, h->tab64, st);
    launch_symmetrize(P.m, h->tab64, h->tabsym64, st);
    launch_moment_basis(h->d.nu, h->cmom64, st);
  }
  if (tc2) {  // degree 2: weights, results and the stacked table's image
    const size_t E0 = (size_t)P.lv[0].ex * P.lv[0].ey * P.lv[0].ez;
    const int mode = tc2_mode_of(h->d.precision);
    CKC(dalloc(h, &h->tcimg, tc2_image_bytes(mode, P.m)));
    CKC(dalloc(h, &h->w32, E0 * P.m));
    CKC(dalloc(h, &h->Y2, E0 * tc2_result_stride()));
    // positions no product writes (the non-vertex rows of trilinear elements
    // of a mixed mesh) stay 0: the mixed fold assembles every node raw
    CKC(cudaMemsetAsync(h->Y2, 0, E0 * tc2_result_stride() * sizeof(float), st));
    CKC(dalloc(h, &h->tcpack, tc2_pack_bytes(mode, (long)E0)));
    CKC(dalloc(h, &h->tcscale, E0 + 256));
    h->tc.apack = h->tcpack;
    h->tc.escale = h->tcscale;
    std::vector<double> tab((size_t)P.m * kDD2);
    CKC(cudaMemcpyAsync(tab.data(), h->tab64, tab.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    CKC(cudaStreamSynchronize(st));
    const float tscale = tc2_table_scale(mode, tab.data(), tab.size());
    launch_tc2_image(mode, P.m, h->tab64, tscale, h->tcimg, st);
    if (h->mixed) {
      // trilinear elements: FP32 copies of their vertex blocks (k_q1v_apply32)
      CKC(dalloc(h, &h->tck1v, (size_t)h->ne1 * kQ1Sym + 4));
      h->tc.K1v = h->tck1v;
      // the node lattice's fold of the slaved nodes after assembly
      CKC(dalloc(h, &h->tcyraw, (size_t)h->lv[0].ndof));
      {
        const Level& L0 = h->lv[0];
        std::vector<uint8_t> sv(L0.nn);
        CKC(cudaMemcpyAsync(sv.data(), h->slv0, L0.nn, cudaMemcpyDeviceToHost, st));
        CKC(cudaStreamSynchronize(st));
        const int Vx = (L0.Lx + 1) / 2, Vy = (L0.Ly + 1) / 2, Vz = (L0.Lz + 1) / 2;
        std::vector<uint32_t> nb((size_t)Vx * Vy * Vz, 0u);
        for (int c = 0; c < Vz; ++c)
          for (int b = 0; b < Vy; ++b)
            for (int a = 0; a < Vx; ++a)
              for (int k = 0; k < 27; ++k) {
                const int ii = 2 * a + k % 3 - 1, jj = 2 * b + (k / 3) % 3 - 1, ll = 2 * c + k / 9 - 1;
                if (k == 13 || ii < 0 || ii >= L0.Lx || jj < 0 || jj >= L0.Ly || ll < 0 || ll >= L0.Lz) continue;
                if (sv[ii + (size_t)L0.Lx * (jj + (size_t)L0.Ly * ll)])
                  nb[a + (size_t)Vx * (b + (size_t)Vy * c)] |= 1u << k;
              }
        CKC(dalloc(h, &h->tcvnb, nb.size()));
        CKC(cudaMemcpyAsync(h->tcvnb, nb.data(), nb.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
        CKC(cudaStreamSynchronize(st));
      }
      h->lv[0].slv = h->slv0;
      h->lv[0].yraw = h->tcyraw;
      h->lv[0].vnb = h->tcvnb;
    }
    int sms = 1;
    CKC(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->dev));
    h->tc.on = true;
    h->tc.deg = 2;
    h->tc.mode = mode;
    h->tc.prec = h->d.precision;
    h->tc.tscale = tscale;
    h->tc.m = P.m;
    h->tc.w32 = h->w32;
    h->tc.img = h->tcimg;
    h->tc.Y2 = h->Y2;
    h->tc.sms = sms;
  }
  if (tf32) {  // tensor-core operands of the finest level
    const size_t E0 = (size_t)P.lv[0].ex * P.lv[0].ey * P.lv[0].ez;
    CKC(dalloc(h, &h->KT32, (size_t)P.m * 576));
    CKC(dalloc(h, &h->w32, E0 * P.m));
    CKC(dalloc(h, &h->Ye, E0 * 24));
    launch_to_fp32((size_t)P.m * 576, h->tab64, h->KT32, st);
    int sms = 1;
    CKC(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->dev));
    h->tc.on = true;
    h->tc.m = P.m;
    h->tc.w32 = h->w32;
    h->tc.KT = h->KT32;
    h->tc.Ye = h->Ye;
    h->tc.sms = sms;
  }
  // filter stencil: integer offsets with di^2+dj^2+dk^2 <= (r n)^2 (ties in)
  {
    std::vector<int4> off;
    std::vector<double> wgt;
    if (h->d.rmin <= 0.0) {
      off.push_back(make_int4(0, 0, 0, 0));
      wgt.push_back(1.0);
    } else {
      const int n = P.n;
      const double r = h->d.rmin, rc2 = (r * n) * (r * n), sig = r / 3.0;
      const int R = (int)std::floor(r * n + 1e-9);
      for (int k = -R; k <= R; ++k)
        for (int j = -R; j <= R; ++j)
          for (int i = -R; i <= R; ++i) {
            const int q = i * i + j * j + k * k;
            if (q <= rc2 * (1.0 + 1e-12)) {
              off.push_back(make_int4(i, j, k, 0));
              wgt.push_back(std::exp(-(q / (double)(n * n)) / (2.0 * sig * sig)));
            }
          }
    }
    h->noff = (int)off.size();
    CKC(dalloc(h, &h->foff, off.size()));
    CKC(dalloc(h, &h->fwgt, wgt.size()));
    CKC(cudaMemcpyAsync(h->foff, off.data(), off.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
    CKC(cudaMemcpyAsync(h->fwgt, wgt.data(), wgt.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  }
  CKC(dalloc(h, &h->rho, P.ncell));
  CKC(dalloc(h, &h->w, P.ncell));
  CKC(dalloc(h, &h->invom, P.ncell));
  CKC(dalloc(h, &h->gtmp, 2 * P.ncell));
  if (P.dm != P.n) {  // Eq. projdsgn from the coarser design grid
    h->proj = true;
    h->pg = ProjGrid{P.Dx, P.Dy, P.Dz, P.dm * h->d.nx, P.dm * h->d.ny, P.dm * h->d.nz, P.n, P.dm,
                     (int)std::ceil(h->d.rmin * P.dm) + 1, h->d.rmin};
    launch_proj_init(h->pg, h->invom, st);
  } else {
    launch_filter_init(P.Dx, P.Dy, P.Dz, h->noff, h->foff, h->fwgt, h->invom, st);
  }
  {
    // levels refreshed on the main stream (all but the coarsest, or the one
    // level) share one slab scratch; the coarsest level has its own
    int ex[kMaxLevels], ey[kMaxLevels], ez[kMaxLevels];
    for (int l = 0; l < P.L; ++l) { ex[l] = P.lv[l].ex; ey[l] = P.lv[l].ey; ez[l] = P.lv[l].ez; }
    const Plan::Lv& c = P.lv[P.L - 1];
    const size_t Ec = (size_t)c.ex * c.ey * c.ez;
    if (h->d.degree >= 2) {
      size_t em = 1;
      for (int l = 1; l + 1 < P.L; ++l) em = std::max(em, (size_t)ex[l] * ey[l] * ez[l]);
      CKC(dalloc(h, &h->Mq, em * kNM2));
      CKC(dalloc(h, &h->Mqc, Ec * kNM2));
      CKC(dalloc(h, &h->Kec, Ec * (elem_sym(h->d.family, level_degree(h->d, P.L - 1), c.nsub) ? kPS2 : kDD2)));
    } else {
      h->ke_bytes = slab_scratch_bytes(ex, ey, ez, P.L > 1 ? P.L - 1 : 1);
      CKC(dalloc(h, (char**)&h->Ke, h->ke_bytes));
      CKC(dalloc(h, &h->Mom, h->ke_bytes / (kSym * 8) * 27));
      CKC(dalloc(h, &h->Kec, Ec * kSym));
      CKC(dalloc(h, &h->Momc, Ec * 27));
    }
  }
  CKC(cudaStreamCreateWithFlags(&h->st2, cudaStreamNonBlocking));
  CKC(cudaEventCreateWithFlags(&h->evf, cudaEventDisableTiming));
  CKC(cudaEventCreateWithFlags(&h->evj, cudaEventDisableTiming));
  // coarse dense solve
  {
    const long nc = P.nc;
    CKC(dalloc(h, &h->Ad, nc * nc));
    CKC(dalloc(h, &h->Wp, nc * kNB));
    CKC(dalloc(h, &h->Vp, nc * kNB));
    CKC(dalloc(h, &h->Pg, kNB * kNB));
    CKC(dalloc(h, &h->Ainv, nc * nc));
    h->cgrid = coarse_sweep_grid();
    if (h->cgrid < 1) { h->err = "coarse sweep kernel cannot be made co-resident"; return fail(TOSOLVE_ECUDA); }
  }
  // PCG
  const long nd = P.lv[0].ndof;
  double** vec64[7] = {&h->u, &h->r, &h->p, &h->q, &h->f, &h->tmpa, &h->tmpb};
  for (double** pv : vec64) {
    CKC(dalloc(h, pv, nd));
    CKC(cudaMemsetAsync(*pv, 0, nd * 8, st));
  }
  if (h->d.inner_its > 0) {
    float** iv[4] = {&h->inner.e, &h->inner.ri, &h->inner.pi, &h->inner.qi};
    for (float** pv : iv) {
      CKC(dalloc(h, pv, nd));
      CKC(cudaMemsetAsync(*pv, 0, nd * sizeof(float), st));
    }
    h->inner.its = h->d.inner_its;
  }
  CKC(dalloc(h, &h->part, 4 * kMaxPart));
  CKC(cudaMemsetAsync(h->part, 0, 4 * kMaxPart * 8, st));
  CKC(dalloc(h, &h->cnt, 4));
  CKC(cudaMemsetAsync(h->cnt, 0, 4 * sizeof(unsigned), st));
  CKC(dalloc(h, &h->ds, 1));
  CKC(cudaMemsetAsync(h->ds, 0, sizeof(DevState), st));
  if (h->tc.on) h->tc.err = &h->ds->tc_status;
  {
    int sms = 1;
    CKC(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->dev));
    for (int l = 0; l < P.L; ++l) {
      h->lv[l].err = &h->ds->tile_status;
      h->lv[l].sms = sms;
    }
    CKC(configure_tile_kernels());
  }
  CKC(cudaMallocHost((void**)&h->hs, sizeof(DevState)));
  std::memset(h->hs, 0, sizeof(DevState));
  h->np = parts_for(h->lv[0].nn);
  // host-step staging
  h->hrhs = h->d.max_rhs;
  CKC(dalloc(h, &h->hx, P.ndes));
  CKC(dalloc(h, &h->hf, nd * h->hrhs));
  CKC(dalloc(h, &h->hu, nd * h->hrhs));
  CKC(dalloc(h, &h->hg, P.ndes));
  if (h->d.smoother == 1) {
    CKC(dalloc(h, &h->lz, 64));
    CKC(dalloc(h, &h->lmax, P.L));
    CKC(cudaMemsetAsync(h->lmax, 0, P.L * sizeof(double), st));
  }
  CKC(cudaEventCreate(&h->ev0));
  CKC(cudaEventCreate(&h->ev1));
  CKC(cudaStreamSynchronize(st));
  CKC(cudaGetLastError());
  if (std::getenv("TOSOLVE_NO_GRAPH") == nullptr) {
    s = build_graph(h);
    if (s != TOSOLVE_OK) return fail(s);
  }
  *out = h;
  return TOSOLVE_OK;
#undef CKC
}

tosolve_status tosolve_create(const tosolve_desc* desc, const uint8_t* mask_host, void* cuda_stream,
                              tosolve_t* out) {
  return create_impl(desc, mask_host, nullptr, cuda_stream, out);
}

tosolve_status tosolve_create_mixed(const tosolve_desc* desc, const uint8_t* mask_host,
                                    const uint8_t* elem_q1_host, void* cuda_stream, tosolve_t* out) {
  if (desc == nullptr || elem_q1_host == nullptr) { g_err = "NULL argument"; return TOSOLVE_EINVAL; }
  if (desc->degree != 2) { g_err = "a mixed mesh lives on the degree-2 lattice (degree = 2)"; return TOSOLVE_EINVAL; }
  if (desc->family != 0) { g_err = "a mixed mesh couples Lagrange elements (family = 0)"; return TOSOLVE_EINVAL; }
  return create_impl(desc, mask_host, elem_q1_host, cuda_stream, out);
}

tosolve_status tosolve_free_dofs(tosolve_t h, long long* n) {
  if (h == nullptr || n == nullptr) return set_err(h, TOSOLVE_EINVAL, "NULL argument");
  *n = h->free_dofs;
  return TOSOLVE_OK;
}

void tosolve_destroy(tosolve_t h) {
  if (h == nullptr) return;
  cudaStreamSynchronize(h->st);
  free_all(h);
  delete h;
}

const char* tosolve_last_error(tosolve_t h) {
  if (h == nullptr) return g_err.c_str();
  return h->err.c_str();
}

// The multigrid setup for the current weights w and level masks (Sec. 7.2:
// every level's operator, Jacobi diagonal and the coarse factorisation).
static tosolve_status refresh(tosolve_t h) {
  cudaStream_t st = h->st;
  const tosolve_desc& d = h->d;
  const int n = d.n_mr;
  const int L = h->L;
  const bool fp32 = d.precision != TOSOLVE_PREC_FP64;
  // The coarsest level (FP64 operator, dense matrix and its inverse)
  // only needs the weights: with more than one level it runs on a second
  // stream, overlapped with the FP64-bound assembly of the finer levels.
  cudaStream_t cst = st;
  if (L > 1) {
    CK(cudaEventRecord(h->evf, st));
    CK(cudaStreamWaitEvent(h->st2, h->evf, 0));
    cst = h->st2;
  }
  Level& C = h->lv[L - 1];
  if (d.degree >= 2) {
    // Lagrange degree-2 levels by sum factorisation; the serendipity element
    // and the cubic finest level by their subcell tables / moment bases
    auto form = [&](Level& Lv, int l, double* Kdst, double* Mscr, cudaStream_t s) {
      if (l == 0 && h->mixed) {  // triquadratic elements constrained, trilinear ones on their vertices
        launch_q2_elem_sf(Lv, h->w, h->Dx, h->Dy, d.nu, Lv.el2, Lv.ne2, h->slv0, Kdst, s);
        launch_q1v_elem(Lv, n, h->w, h->Dx, h->Dy, h->tab64q1, Kdst, s);
      } else if (d.family == 0 && Lv.k == 2 && q2_elem_sf_supported(Lv.nsub))
        launch_q2_elem_sf(Lv, h->w, h->Dx, h->Dy, d.nu, nullptr, 0, nullptr, Kdst, s);
      else if (l == 0)
        launch_q2_elem(Lv, n, h->w, h->Dx, h->Dy, h->tab64, Kdst, s);
      else
        launch_q2_coarse_elem(Lv, h->w, h->Dx, h->Dy, h->cmom64, Mscr, Kdst, s);
    };
    const double* Kc = h->Kec;
    if (L > 1) {
      form(C, L - 1, h->Kec, h->Mqc, cst);
    } else {
      form(C, 0, C.K64, nullptr, cst);
      Kc = C.K64;
    }
    CK(cudaMemsetAsync(h->Ad, 0, (size_t)h->nc * h->nc * sizeof(double), cst));
    launch_q2_dense(C, Kc, h->Ad, cst);
    CK(cudaMemsetAsync(&h->ds->coarse_status, 0, sizeof(int), cst));
    CK(launch_coarse_invert(h->nc, h->Ad, h->Wp, h->Vp, h->Pg, h->Ainv, &h->ds->coarse_status,
                            h->cgrid, cst));
    for (int l = 0; l + 1 < L; ++l) {
      Level& Lv = h->lv[l];
      form(Lv, l, Lv.K64, h->Mq, st);
      launch_q2_dinv(true, Lv, Lv.K64, Lv.dinv64, st);
      if (Lv.K32) launch_elem_fp32(Lv, Lv.K64, Lv.K32, st);
      if (Lv.dinv32) launch_q2_dinv(false, Lv, Lv.K64, Lv.dinv32, st);
      if (l == 0 && h->tc.on) launch_weights_elem(Lv, n, h->w, h->Dx, h->Dy, h->w32, st);
      if (Lv.Kc64 || Lv.Kc32) launch_ser_compact(Lv, st);
    }
    if (L > 1) {
      CK(cudaEventRecord(h->evj, h->st2));
      CK(cudaStreamWaitEvent(st, h->evj, 0));
    }
    if (h->tck1v) launch_q1v_compact32(h->lv[0], h->lv[0].K64, h->tck1v, st);
    if (d.smoother == 1)  // lambda_max of every smoothing operator, then the Chebyshev coefficients
      launch_cheb_setup(vt_of(h), h->lv, L, h->tc, kChebLanczos, h->part, h->cnt, h->lz, h->lmax, st);
    CK(cudaGetLastError());
    return TOSOLVE_OK;
  }
  if (L > 1) {
    launch_elem_moments(true, C, 0, C.ez, h->w, h->Dx, h->Dy, h->cmom64, h->Momc, h->Kec, cst);
    launch_assemble(true, C, 0, C.Lz, 0, h->Kec, C.S64, C.dinv64, cst);
  } else {
    for_each_slab(C, h->ke_bytes, kSym * 8, [&](int l0, int l1, int ze0, int ze1) {
      launch_elem_direct(true, C, ze0, ze1, n, h->w, h->Dx, h->Dy, h->tabsym64, h->Ke, cst);
      launch_assemble(true, C, l0, l1, ze0, h->Ke, C.S64, C.dinv64, cst);
    });
    if (C.S32) {
      launch_to_fp32(op_len(C.nn), C.S64, C.S32, cst);
      launch_to_fp32((size_t)C.ndof, C.dinv64, C.dinv32, cst);
    }
  }
  CK(cudaMemsetAsync(h->Ad, 0, (size_t)h->nc * h->nc * sizeof(double), cst));
  launch_coarse_dense(C, h->Ad, cst);
  CK(cudaMemsetAsync(&h->ds->coarse_status, 0, sizeof(int), cst));
  CK(launch_coarse_invert(h->nc, h->Ad, h->Wp, h->Vp, h->Pg, h->Ainv, &h->ds->coarse_status,
                          h->cgrid, cst));
  for (int l = 0; l + 1 < L; ++l) {
    Level& Lv = h->lv[l];
    if (l == 0) {
      for_each_slab(Lv, h->ke_bytes, kSym * 8, [&](int l0, int l1, int ze0, int ze1) {
        launch_elem_direct(true, Lv, ze0, ze1, n, h->w, h->Dx, h->Dy, h->tabsym64, h->Ke, st);
        launch_assemble(true, Lv, l0, l1, ze0, h->Ke, Lv.S64, Lv.dinv64, st);
      });
      if (Lv.S32) launch_to_fp32(op_len(Lv.nn), Lv.S64, Lv.S32, st);
      if (Lv.dinv32) launch_to_fp32((size_t)Lv.ndof, Lv.dinv64, Lv.dinv32, st);
      if (h->tc.on) launch_weights_elem(Lv, n, h->w, h->Dx, h->Dy, h->w32, st);
    } else {
      const bool op64 = !fp32 || d.precision == TOSOLVE_PREC_FP32X2;
      for_each_slab(Lv, h->ke_bytes, kSym * (op64 ? 8 : 4), [&](int l0, int l1, int ze0, int ze1) {
        launch_elem_moments(op64, Lv, ze0, ze1, h->w, h->Dx, h->Dy, h->cmom64, h->Mom, h->Ke, st);
        if (op64)
          launch_assemble(true, Lv, l0, l1, ze0, h->Ke, Lv.S64, Lv.dinv64, st);
        else
          launch_assemble(false, Lv, l0, l1, ze0, h->Ke, Lv.S32, Lv.dinv32, st);
      });
      if (op64 && Lv.S32) {  // FP32X2: FP32 copy of the FP64-formed operator
        launch_to_fp32(op_len(Lv.nn), Lv.S64, Lv.S32, st);
        launch_to_fp32((size_t)Lv.ndof, Lv.dinv64, Lv.dinv32, st);
      }
    }
  }
  if (L > 1) {
    CK(cudaEventRecord(h->evj, h->st2));
    CK(cudaStreamWaitEvent(st, h->evj, 0));
  }
  CK(cudaGetLastError());
  return TOSOLVE_OK;
}

tosolve_status tosolve_set_densities(tosolve_t h, const double* x_dev) {
  if (h == nullptr) return set_err(h, TOSOLVE_EINVAL, "handle is NULL");
  if (x_dev == nullptr) return set_err(h, TOSOLVE_EINVAL, "x is NULL");
  cudaStream_t st = h->st;
  const tosolve_desc& d = h->d;
  if (h->proj)
    launch_proj_fwd(h->pg, h->invom, x_dev, d.Emin, d.E0 - d.Emin, d.penal, h->rho, h->w, st);
  else
    launch_filter_fwd(h->Dx, h->Dy, h->Dz, h->noff, h->foff, h->fwgt, h->invom, x_dev, d.Emin,
                      d.E0 - d.Emin, d.penal, h->rho, h->w, st);
  const tosolve_status s = refresh(h);
  if (s != TOSOLVE_OK) return s;
  h->have_rho = true;
  return TOSOLVE_OK;
}

// After the level-0 mask changed: the free count of level 0 is read back and
// its tile order puts the tiles with a free DOF first (the stencil kernels
// pass the others through as identity rows).  The coarse levels keep the
// supports alone: a coarse node that coincides with a suppressed node can
// still carry a correction for the free nodes near it (the transfers mask
// the fine side), whereas fixing it would clamp the coarse elements that
// reach from the void into the structure.
static tosolve_status remask(tosolve_t h) {
  cudaStream_t st = h->st;
  Level& L0 = h->lv[0];
  const int nt = (L0.nn + kTN - 1) / kTN;
  std::vector<uint8_t> m(L0.ndof);
  CK(cudaMemcpyAsync(m.data(), L0.mask, L0.ndof, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  std::vector<int> order;
  order.reserve(nt);
  int nact = 0;
  for (int pass = 0; pass < 2; ++pass) {
    for (int t = 0; t < nt; ++t) {
      const long d0 = 3L * kTN * t, d1 = std::min<long>(d0 + 3L * kTN, L0.ndof);
      bool all = true;
      for (long q = d0; q < d1 && all; ++q) all = m[q] != 0;
      if (all == (pass == 1)) order.push_back(t);
    }
    if (pass == 0) nact = (int)order.size();
  }
  long long nfree = 0;
  for (uint8_t v : m) nfree += v == 0;
  h->free_dofs = nfree;
  // The stored order always matches the current mask (a batch graph recorded
  // while an order was in force keeps reading it); the kernels of the
  // handle's own graph follow it only while some tile is all fixed.
  CK(cudaMemcpyAsync(L0.tcnt_buf, &nact, sizeof(int), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(L0.tl_buf, order.data(), nt * sizeof(int), cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  int* want = nact < nt ? L0.tl_buf : nullptr;
  if (want != L0.tl) {  // the kernel arguments change: record the graph again
    L0.tl = want;
    L0.tcnt = want ? L0.tcnt_buf : nullptr;
    if (h->graph_ready) {
      cudaGraphExecDestroy(h->gexec);
      cudaGraphDestroy(h->graph);
      h->gexec = nullptr;
      h->graph = nullptr;
      h->graph_ready = false;
      return build_graph(h);
    }
  }
  return TOSOLVE_OK;
}

tosolve_status tosolve_fix_variables(tosolve_t h, const double* dcdx_dev, double rho_lo, double rho_hi,
                                     double eps_grad, uint8_t* fixed_dev, long long* suppressed_dofs) {
  if (h == nullptr) return set_err(h, TOSOLVE_EINVAL, "handle is NULL");
  if (!h->have_rho) return set_err(h, TOSOLVE_EINVAL, "call tosolve_set_densities first");
  if (!(rho_lo >= 0.0) || !(rho_hi <= 1.0) || !(rho_lo < rho_hi) || !(eps_grad >= 0.0))
    return set_err(h, TOSOLVE_EINVAL, "need 0 <= rho_lo < rho_hi <= 1 and eps_grad >= 0");
  cudaStream_t st = h->st;
  const Level& L0 = h->lv[0];
  const int dm = h->proj ? h->pg.d : h->d.n_mr;
  launch_fix_classify(L0, h->d.n_mr, dm, h->rho, dcdx_dev, rho_lo, rho_hi, eps_grad, h->ecls, st);
  launch_fix_surround(L0, h->ecls, h->efix, st);
  launch_fix_design(L0, dm, h->efix, h->xfix, st);
  launch_fix_mask(L0, h->efix, h->base0, st);
  if (fixed_dev) CK(cudaMemcpyAsync(fixed_dev, h->xfix, (size_t)h->ndes, cudaMemcpyDeviceToDevice, st));
  tosolve_status s = remask(h);
  if (s != TOSOLVE_OK) return s;
  h->fixing = true;
  if (suppressed_dofs) *suppressed_dofs = h->free_base - h->free_dofs;
  s = refresh(h);
  if (s != TOSOLVE_OK) return s;
  CK(cudaStreamSynchronize(st));
  return TOSOLVE_OK;
}

// ---- thresholding and the Heaviside projection (Sec. 5) ----------------------

size_t tosolve_threshold_scratch_bytes(long long n) {
  if (n < 0 || n > INT_MAX) return 0;
  return threshold_scratch_bytes((long)n);
}

static tosolve_status thresh_args(const double* a, const double* b, long long n, const void* scratch,
                                  double theta) {
  if (n < 0 || n > INT_MAX) { g_err = "n must be in 0..2^31-1"; return TOSOLVE_EINVAL; }
  if (n > 0 && (a == nullptr || b == nullptr)) { g_err = "NULL argument"; return TOSOLVE_EINVAL; }
  if (n > 0 && scratch == nullptr) { g_err = "scratch is NULL"; return TOSOLVE_EINVAL; }
  if (!(theta > 0.0 && theta < 180.0)) { g_err = "theta_max must be in (0, 180) degrees"; return TOSOLVE_EINVAL; }
  return TOSOLVE_OK;
}

tosolve_status tosolve_heaviside(const double* rho_dev, long long n, double beta, double* out_dev, double* eta,
                                 int* newton_its, void* scratch_dev, size_t scratch_bytes, void* cuda_stream) {
  tosolve_status s = thresh_args(rho_dev, out_dev, n, scratch_dev, 90.0);
  if (s != TOSOLVE_OK) return s;
  if (!(beta > 0.0)) { g_err = "beta must be > 0"; return TOSOLVE_EINVAL; }
  if (n == 0) {
    if (eta) *eta = 0.5;
    if (newton_its) *newton_its = 0;
    return TOSOLVE_OK;
  }
  return heaviside(rho_dev, (long)n, beta, out_dev, eta, newton_its, scratch_dev, scratch_bytes,
                   (cudaStream_t)cuda_stream, &g_err);
}

tosolve_status tosolve_threshold_density(const double* rho_dev, long long n, double vfrac, double round_lo,
                                         double round_hi, const double* gradL_dev, double theta_max_deg,
                                         double* out_dev, int* accepted, void* scratch_dev, size_t scratch_bytes,
                                         void* cuda_stream) {
  tosolve_status s = thresh_args(rho_dev, out_dev, n, scratch_dev, theta_max_deg);
  if (s != TOSOLVE_OK) return s;
  if (n > 0 && gradL_dev == nullptr) { g_err = "gradL is NULL"; return TOSOLVE_EINVAL; }
  if (!(vfrac >= 0.0 && vfrac <= 1.0)) { g_err = "vfrac must be in [0, 1]"; return TOSOLVE_EINVAL; }
  if (!(round_lo >= 0.0 && round_lo < round_hi && round_hi <= 1.0)) {
    g_err = "need 0 <= round_lo < round_hi <= 1";
    return TOSOLVE_EINVAL;
  }
  if (n == 0) {
    if (accepted) *accepted = 0;
    return TOSOLVE_OK;
  }
  return threshold_density(rho_dev, (long)n, vfrac, round_lo, round_hi, gradL_dev, theta_max_deg, out_dev, accepted,
                           scratch_dev, scratch_bytes, (cudaStream_t)cuda_stream, &g_err);
}

tosolve_status tosolve_threshold_gradient(const double* rho_dev, const double* gradL_dev, long long n,
                                          double round_lo, double round_hi, double vu_min, double vl_max,
                                          double theta_max_deg, double* out_dev, double* alpha, void* scratch_dev,
                                          size_t scratch_bytes, void* cuda_stream) {
  tosolve_status s = thresh_args(rho_dev, out_dev, n, scratch_dev, theta_max_deg);
  if (s != TOSOLVE_OK) return s;
  if (n > 0 && gradL_dev == nullptr) { g_err = "gradL is NULL"; return TOSOLVE_EINVAL; }
  if (!(round_lo >= 0.0 && round_lo < round_hi && round_hi <= 1.0)) {
    g_err = "need 0 <= round_lo < round_hi <= 1";
    return TOSOLVE_EINVAL;
  }
  if (n == 0) {
    if (alpha) *alpha = 0.0;
    return TOSOLVE_OK;
  }
  return threshold_gradient(rho_dev, (long)n, round_lo, round_hi, gradL_dev, vu_min, vl_max, theta_max_deg, out_dev,
                            alpha, scratch_dev, scratch_bytes, (cudaStream_t)cuda_stream, &g_err);
}

tosolve_status tosolve_release_variables(tosolve_t h) {
  if (h == nullptr) return set_err(h, TOSOLVE_EINVAL, "handle is NULL");
  cudaStream_t st = h->st;
  CK(cudaMemcpyAsync(h->lv[0].mask, h->base0, (size_t)h->lv[0].ndof, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemsetAsync(h->xfix, 0, (size_t)h->ndes, st));
  tosolve_status s = remask(h);
  if (s != TOSOLVE_OK) return s;
  h->fixing = false;
  if (h->have_rho) {
    s = refresh(h);
    if (s != TOSOLVE_OK) return s;
  }
  CK(cudaStreamSynchronize(st));
  return TOSOLVE_OK;
}

static tosolve_status run_loop_nograph(tosolve_t h) {
  // Same kernels as the graph, driven from the host (profiling path: ncu
  // cannot profile kernels of a graph that holds a conditional node).
  const int vt = vt_of(h);
  Level& L0 = h->lv[0];
  const int np = h->np;
  double *part0 = h->part, *part1 = h->part + kMaxPart, *part2 = h->part + 2 * kMaxPart,
         *part3 = h->part + 3 * kMaxPart;
  cudaStream_t st = h->st;
  if (h->mixed) launch_q2_fold(L0, h->slv0, h->f, st);
  launch_cg_prep(L0, h->f, h->u, part0, np, st);
  launch_cg_residual(vt, L0, h->d.omega, h->f, h->u, h->r, 1, part1, part0, np, h->ds, h->cnt, 0, 0,
                     st);
  CK(cudaMemcpyAsync(h->hs, h->ds, sizeof(DevState), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  while (!h->hs->converged && h->hs->status == 0 && h->hs->iter < h->hs->maxit) {
    const CgDots cd{h->r, h->q, part2, part3, h->ds, h->cnt + 1};
    if (h->inner.its > 0) {
      launch_inner_pcg(h->lv, h->L, h->d.omega, h->Ainv, h->tc, h->inner, part2, part3, h->ds, h->cnt + 1, st);
      launch_cg_dots_rz(vt, L0, h->r, h->q, part2, part3, np, h->ds, h->cnt + 1, st);
    } else if (!launch_vcycle(vt, h->lv, h->L, h->d.omega, 1, h->Ainv, h->tc, st, &cd)) {
      launch_cg_dots_rz(vt, L0, h->r, h->q, part2, part3, np, h->ds, h->cnt + 1, st);
    }
    launch_cg_dir(vt, L0, h->p, np, h->ds, st);
    launch_cg_apply(L0, h->p, h->q, part0, np, h->ds, h->cnt + 2, st);
    launch_cg_update(vt, L0, h->d.omega, h->u, h->r, h->p, h->q, part1, np, h->ds, h->cnt + 3, 0, 0,
                     st);
    CK(cudaMemcpyAsync(h->hs, h->ds, sizeof(DevState), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  launch_cg_residual(vt, L0, h->d.omega, h->f, h->u, h->tmpa, 2, part1, part0, np, h->ds, h->cnt, 0,
                     0, st);
  if (h->mixed) launch_q2_expand(L0, h->slv0, h->u, st);
  return TOSOLVE_OK;
}

tosolve_status tosolve_solve(tosolve_t h, const double* f_dev, int nrhs, double* u_dev, double rtol,
                             int maxit, tosolve_info* info) {
  if (info) std::memset(info, 0, sizeof(*info));
  auto finish = [&](tosolve_status s) {
    if (info) info->status = (int)s;
    return s;
  };
  if (h == nullptr) return finish(set_err(h, TOSOLVE_EINVAL, "handle is NULL"));
  if (f_dev == nullptr || u_dev == nullptr) return finish(set_err(h, TOSOLVE_EINVAL, "f or u is NULL"));
  if (nrhs < 1 || nrhs > h->d.max_rhs) return finish(set_err(h, TOSOLVE_EINVAL, "nrhs must be in 1..max_rhs"));
  if (!(rtol > 0.0) || maxit < 1 || maxit > 100000)
    return finish(set_err(h, TOSOLVE_EINVAL, "need rtol > 0 and 1 <= maxit <= 100000"));
  if (!h->have_rho) return finish(set_err(h, TOSOLVE_EINVAL, "call tosolve_set_densities first"));
  cudaStream_t st = h->st;
  const size_t nd = h->lv[0].ndof;
  tosolve_status result = TOSOLVE_OK;
  int total = 0, last = 0;
  double worst = 0.0;
  auto worse = [](double a, double b) { return (a == a && b == b) ? std::fmax(a, b) : NAN; };  // NaN stays
  if (cudaEventRecord(h->ev0, st) != cudaSuccess) return finish(set_err(h, TOSOLVE_ECUDA, "event record failed"));
  for (int r = 0; r < nrhs && result == TOSOLVE_OK; ++r) {
    const double* fr = f_dev + r * nd;
    double* ur = u_dev + r * nd;
    int used = 0;
    for (int attempt = 0; attempt < 4; ++attempt) {
      h->hs->tol2 = rtol * rtol;
      h->hs->maxit = maxit - used;
      if (cudaMemcpyAsync(&h->ds->tol2, &h->hs->tol2, sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
          cudaMemcpyAsync(&h->ds->maxit, &h->hs->maxit, sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess ||
          cudaMemcpyAsync(h->f, fr, nd * 8, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
          cudaMemcpyAsync(h->u, ur, nd * 8, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return finish(set_err(h, TOSOLVE_ECUDA, "copy into the solver failed"));
      if (h->graph_ready) {
        if (cudaGraphLaunch(h->gexec, st) != cudaSuccess)
          return finish(set_err(h, TOSOLVE_ECUDA, "graph launch failed"));
      } else {
        const tosolve_status s2 = run_loop_nograph(h);
        if (s2 != TOSOLVE_OK) return finish(s2);
      }
      CK(cudaMemcpyAsync(ur, h->u, nd * 8, cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(h->hs, h->ds, sizeof(DevState), cudaMemcpyDeviceToHost, st));
      const cudaError_t e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) {
        h->err = std::string("solve: ") + cudaGetErrorString(e);
        return finish(TOSOLVE_ECUDA);
      }
      const DevState& S = *h->hs;
      used += S.iter;
      if (S.tc_status || S.tile_status) {  // sticky: the handle stays unusable
        h->err = S.tc_status ? "a tensor-core tile did not complete within its bounded wait"
                             : "an operator tile copy did not complete within its bounded wait";
        return finish(TOSOLVE_ECUDA);
      }
      if (S.ff == 0.0) {  // f = 0: the solution is u = 0
        CK(cudaMemsetAsync(ur, 0, nd * 8, st));
        last = 0;
        break;
      }
      const double rel = std::sqrt(S.rr_true / S.ff);
      last = used;
      if (S.status != 0) {
        result = TOSOLVE_EBREAKDOWN;
        h->err = S.coarse_status ? "coarse sweep met a non-positive pivot (coarsest operator not SPD)" : "PCG breakdown (p^T K p <= 0 or NaN)";
        worst = worse(worst, rel);
        break;
      }
      if (rel <= rtol) { worst = worse(worst, rel); break; }
      if (used >= maxit || attempt == 3) {
        worst = worse(worst, rel);
        result = TOSOLVE_ENOTCONV;
        h->err = used >= maxit ? "maxit reached before the tolerance"
                               : "the true residual stayed above the tolerance after 3 restarts";
        break;
      }
      // recursive residual met the tolerance but the true one did not:
      // restart from the current iterate with a freshly computed residual
    }
    total += used;
  }
  CK(cudaEventRecord(h->ev1, st));
  CK(cudaEventSynchronize(h->ev1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, h->ev0, h->ev1);
  if (info) {
    info->iterations = last;
    info->total_iterations = total;
    info->rel_residual = worst;
    info->ms = ms;
  }
  return finish(result);
}

tosolve_status tosolve_compliance_grad(tosolve_t h, const double* u_dev, const double* f_dev, int nrhs,
                                       double* c_host, double* dcdx_dev, double* dcdrho_dev) {
  if (h == nullptr) return set_err(h, TOSOLVE_EINVAL, "handle is NULL");
  if (u_dev == nullptr || f_dev == nullptr || c_host == nullptr) return set_err(h, TOSOLVE_EINVAL, "u, f or c is NULL");
  if (nrhs < 1 || nrhs > h->d.max_rhs) return set_err(h, TOSOLVE_EINVAL, "nrhs must be in 1..max_rhs");
  if (!h->have_rho) return set_err(h, TOSOLVE_EINVAL, "call tosolve_set_densities first");
  cudaStream_t st = h->st;
  const tosolve_desc& d = h->d;
  const size_t nd = h->lv[0].ndof;
  double* g = h->gtmp;
  double* gt = h->gtmp + h->ncell;
  const bool want_grad = dcdx_dev != nullptr || dcdrho_dev != nullptr;
  for (int r = 0; r < nrhs; ++r) {
    launch_compliance(h->lv[0], h->mixed ? h->fix0 : h->lv[0].mask, f_dev + r * nd, u_dev + r * nd,
                      h->part, h->np, h->ds, st);
    CK(cudaMemcpyAsync(&h->hs->c, &h->ds->c, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    c_host[r] = h->hs->c;
    if (want_grad && d.degree == 2 && d.family == 0 && q2_energy_sf_supported(d.n_mr))
      launch_q2_energy_sf(h->lv[0], d.n_mr, d.nu, u_dev + r * nd, h->rho, d.penal, d.E0 - d.Emin, h->Dx, h->Dy,
                          r == 0, g, h->lv[0].sms, st);
    else if (want_grad && d.degree >= 2)
      launch_q2_energy_grad(h->lv[0], d.n_mr, u_dev + r * nd, h->tab64, h->rho, d.penal, d.E0 - d.Emin,
                            h->Dx, h->Dy, r == 0, g, h->lv[0].sms, st);
    else if (want_grad)
      launch_energy_grad(h->lv[0], d.n_mr, u_dev + r * nd, h->tabsym64, h->rho, d.penal,
                         d.E0 - d.Emin, h->Dx, h->Dy, r == 0, g, st);
  }
  if (dcdrho_dev) CK(cudaMemcpyAsync(dcdrho_dev, g, (size_t)h->ncell * 8, cudaMemcpyDeviceToDevice, st));
  if (dcdx_dev) {
    launch_scale((size_t)h->ncell, g, h->invom, gt, st);
    if (h->proj)
      launch_proj_T(h->pg, gt, dcdx_dev, st);
    else
      launch_filter_T(h->Dx, h->Dy, h->Dz, h->noff, h->foff, h->fwgt, gt, dcdx_dev, st);
    if (h->fixing) launch_zero_fixed_void(h->ndes, h->xfix, dcdx_dev, st);
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  return TOSOLVE_OK;
}

tosolve_status tosolve_step_host(tosolve_t h, const double* x_host, const double* f_host, int nrhs,
                                 double rtol, int maxit, int warm, double* u_host, double* c_host,
                                 double* dcdx_host, tosolve_info* info) {
  if (h == nullptr) return set_err(h, TOSOLVE_EINVAL, "handle is NULL");
  if (x_host == nullptr || f_host == nullptr || c_host == nullptr) return set_err(h, TOSOLVE_EINVAL, "x, f or c is NULL");
  if (nrhs < 1 || nrhs > h->hrhs) return set_err(h, TOSOLVE_EINVAL, "nrhs must be in 1..max_rhs");
  cudaStream_t st = h->st;
  const size_t nd = h->lv[0].ndof;
  CK(cudaMemcpyAsync(h->hx, x_host, (size_t)h->ndes * 8, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(h->hf, f_host, nd * nrhs * 8, cudaMemcpyHostToDevice, st));
  if (!h->have_u || !warm) {
    CK(cudaMemsetAsync(h->hu, 0, nd * h->hrhs * 8, st));
    h->have_u = true;
  }
  tosolve_status s = tosolve_set_densities(h, h->hx);
  if (s != TOSOLVE_OK) return s;
  s = tosolve_solve(h, h->hf, nrhs, h->hu, rtol, maxit, info);
  if (s != TOSOLVE_OK && s != TOSOLVE_ENOTCONV) return s;
  const tosolve_status s2 = tosolve_compliance_grad(h, h->hu, h->hf, nrhs, c_host,
                                                    dcdx_host ? h->hg : nullptr, nullptr);
  if (s2 != TOSOLVE_OK) return s2;
  if (u_host) CK(cudaMemcpyAsync(u_host, h->hu, nd * nrhs * 8, cudaMemcpyDeviceToHost, st));
  if (dcdx_host) CK(cudaMemcpyAsync(dcdx_host, h->hg, (size_t)h->ndes * 8, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return s;
}

tosolve_status tosolve_level_dims(tosolve_t h, int level, int* dims) {
  if (h == nullptr || dims == nullptr) return set_err(h, TOSOLVE_EINVAL, "NULL argument");
  if (level < 0 || level >= h->L) return set_err(h, TOSOLVE_EINVAL, "level out of range");
  dims[0] = h->lv[level].Lx;
  dims[1] = h->lv[level].Ly;
  dims[2] = h->lv[level].Lz;
  return TOSOLVE_OK;
}

tosolve_status tosolve_subcell_table(tosolve_t h, double* table_dev) {
  if (h == nullptr || table_dev == nullptr) return set_err(h, TOSOLVE_EINVAL, "NULL argument");
  const size_t dd = h->d.degree == 3 ? (size_t)kDD3 : (h->d.degree == 2 ? (size_t)kDD2 : 576);
  CK(cudaMemcpyAsync(table_dev, h->tab64, (size_t)h->m * dd * 8, cudaMemcpyDeviceToDevice, h->st));
  return TOSOLVE_OK;
}

tosolve_status tosolve_densities(tosolve_t h, double* rho_dev, double* w_dev) {
  if (h == nullptr) return set_err(h, TOSOLVE_EINVAL, "handle is NULL");
  if (!h->have_rho) return set_err(h, TOSOLVE_EINVAL, "call tosolve_set_densities first");
  if (rho_dev) CK(cudaMemcpyAsync(rho_dev, h->rho, (size_t)h->ncell * 8, cudaMemcpyDeviceToDevice, h->st));
  if (w_dev) CK(cudaMemcpyAsync(w_dev, h->w, (size_t)h->ncell * 8, cudaMemcpyDeviceToDevice, h->st));
  return TOSOLVE_OK;
}

tosolve_status tosolve_apply(tosolve_t h, int level, int precision, const double* x_dev, double* y_dev) {
  if (h == nullptr || x_dev == nullptr || y_dev == nullptr) return set_err(h, TOSOLVE_EINVAL, "NULL argument");
  if (level < 0 || level >= h->L) return set_err(h, TOSOLVE_EINVAL, "level out of range");
  if (!h->have_rho) return set_err(h, TOSOLVE_EINVAL, "call tosolve_set_densities first");
  const Level& L = h->lv[level];
  if (L.k >= 2 && (precision == 0 || precision == 1 || precision == 3)) {
    const bool ok = precision == 0 ? L.K64 != nullptr : L.K32 != nullptr;
    const bool vt_ok = precision == 0 || (precision == 1) == (vt_of(h) == kVtF32);
    if (!ok || !vt_ok) return set_err(h, TOSOLVE_EINVAL, "this level has no operator in that precision");
    launch_apply_diag(precision == 0 ? kVtF64 : (precision == 1 ? kVtF32 : kVtDF), L, x_dev, y_dev, h->st);
  } else if (precision == 0) {
    if (!L.S64) return set_err(h, TOSOLVE_EINVAL, "this level has no FP64 operator");
    launch_apply_diag(kVtF64, L, x_dev, y_dev, h->st);
  } else if (precision == 1 || precision == 3) {
    if (!L.S32) return set_err(h, TOSOLVE_EINVAL, "this level has no FP32 operator");
    launch_apply_diag(precision == 1 ? kVtF32 : kVtDF, L, x_dev, y_dev, h->st);
  } else if (precision == 2 || precision >= 4) {
    if (level != 0 || !h->tc.on || precision != (h->tc.deg == 2 ? h->tc.prec : 2))
      return set_err(h, TOSOLVE_EINVAL, "no tensor-core operator of that precision on this level");
    Level& L0 = h->lv[0];
    if (h->tc.deg == 2) {  // the kernel zeroes fixed DOFs itself; the gather keeps them as identity rows
      launch_cast(false, (size_t)L0.ndof, x_dev, L0.v, true, h->st);
      CK(launch_tc2_apply(h->tc, L0, (const float*)L0.v, h->st));
      launch_tc2_gather(L0, h->Y2, (const float*)L0.v, (const float*)L0.v, L0.dinv32, 0.f, 2, (float*)L0.r,
                        h->st);
      launch_cast(true, (size_t)L0.ndof, L0.r, y_dev, false, h->st);
      CK(cudaGetLastError());
      return TOSOLVE_OK;
    }
    // masked copy feeds the elements; the unmasked copy gives the identity rows
    launch_cast(false, (size_t)L0.ndof, x_dev, L0.b, true, h->st);
    launch_cast(false, (size_t)L0.ndof, x_dev, L0.v, true, h->st);
    launch_mask_fp32(L0, (float*)L0.v, h->st);
    CK(launch_tc_apply(L0, h->tc.m, (const float*)L0.v, h->w32, h->KT32, h->Ye, h->tc.err, h->tc.sms, h->st));
    launch_tc_gather(L0, h->Ye, (const float*)L0.b, (const float*)L0.b, L0.dinv32, 0.f, 2, (float*)L0.r, h->st);
    launch_cast(true, (size_t)L0.ndof, L0.r, y_dev, false, h->st);
  } else {
    return set_err(h, TOSOLVE_EINVAL, "precision must be 0 .. 6");
  }
  CK(cudaGetLastError());
  return TOSOLVE_OK;
}

tosolve_status tosolve_tc_stage(tosolve_t h, int part, int stages, const double* x_dev) {
  if (h == nullptr) return set_err(h, TOSOLVE_EINVAL, "NULL argument");
  if (!h->have_rho) return set_err(h, TOSOLVE_EINVAL, "call tosolve_set_densities first");
  if (!h->tc.on || h->tc.deg != 2) return set_err(h, TOSOLVE_EINVAL, "the handle has no degree-2 tensor-core operator");
  if (part < 0 || part > 1 || stages < 1 || stages > 3) return set_err(h, TOSOLVE_EINVAL, "part must be 0 or 1, stages 1 .. 3");
  if (part == 1 && !h->mixed) return set_err(h, TOSOLVE_EINVAL, "part 1 needs a mixed mesh");
  Level& L0 = h->lv[0];
  if (stages & 1) {
    if (x_dev == nullptr) return set_err(h, TOSOLVE_EINVAL, "NULL argument");
    launch_cast(false, (size_t)L0.ndof, x_dev, L0.v, true, h->st);
  }
  CK(launch_tc2_apply(h->tc, L0, (const float*)L0.v, h->st, part, stages));
  return TOSOLVE_OK;
}

tosolve_status tosolve_smoother_lmax(tosolve_t h, int level, double* lmax_host) {
  if (h == nullptr || lmax_host == nullptr) return set_err(h, TOSOLVE_EINVAL, "NULL argument");
  if (h->d.smoother != 1) return set_err(h, TOSOLVE_EINVAL, "the handle smooths with damped Jacobi");
  if (level < 0 || level + 1 >= h->L) return set_err(h, TOSOLVE_EINVAL, "level must be below the coarsest");
  CK(cudaMemcpyAsync(lmax_host, h->lmax + level, sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  return TOSOLVE_OK;
}

tosolve_status tosolve_precondition(tosolve_t h, const double* b_dev, double* z_dev) {
  if (h == nullptr || b_dev == nullptr || z_dev == nullptr) return set_err(h, TOSOLVE_EINVAL, "NULL argument");
  if (!h->have_rho) return set_err(h, TOSOLVE_EINVAL, "call tosolve_set_densities first");
  const int vt = vt_of(h);
  Level& L0 = h->lv[0];
  launch_vec_in(vt, (size_t)L0.ndof, b_dev, L0.b, h->st);
  if (h->L > 1) launch_smooth0(vt, L0, h->d.omega, h->st);
  launch_vcycle(vt, h->lv, h->L, h->d.omega, 1, h->Ainv, h->tc, h->st);
  launch_vec_out(vt, (size_t)L0.ndof, L0.z, z_dev, h->st);
  CK(cudaGetLastError());
  return TOSOLVE_OK;
}

}  // extern "C"

void tos::set_last_error(const char* msg) { g_err = msg; }

extern "C" {

static void batch_free(tosolve_batch_t b) {
  if (b->ge) cudaGraphExecDestroy(b->ge);
  if (b->g) cudaGraphDestroy(b->g);
  for (cudaStream_t x : b->branch) if (x) cudaStreamDestroy(x);
  for (cudaEvent_t x : b->ev) if (x) cudaEventDestroy(x);
  if (b->evf) cudaEventDestroy(b->evf);
  if (b->evd) cudaEventDestroy(b->evd);
  if (b->t0) cudaEventDestroy(b->t0);
  if (b->t1) cudaEventDestroy(b->t1);
  if (b->bs) cudaStreamDestroy(b->bs);
  if (b->st) cudaStreamDestroy(b->st);
  if (b->hparams) cudaFreeHost(b->hparams);
  if (b->hst) cudaFreeHost(b->hst);
  if (b->dparams) cudaFree(b->dparams);
}

tosolve_status tosolve_batch_create(const tosolve_t* handles, int count, const int* nrhs,
                                    const double* const* f_dev, double* const* u_dev,
                                    tosolve_batch_t* out) {
  if (out == nullptr) { g_err = "out is NULL"; return TOSOLVE_EINVAL; }
  *out = nullptr;
  if (handles == nullptr || nrhs == nullptr || f_dev == nullptr || u_dev == nullptr || count < 1 ||
      count > 4096) {
    g_err = "need 1 <= count <= 4096 and non-NULL arrays";
    return TOSOLVE_EINVAL;
  }
  for (int i = 0; i < count; ++i) {
    if (handles[i] == nullptr || f_dev[i] == nullptr || u_dev[i] == nullptr) { g_err = "NULL handle or buffer"; return TOSOLVE_EINVAL; }
    if (nrhs[i] < 1 || nrhs[i] > handles[i]->d.max_rhs) { g_err = "nrhs out of range for a handle"; return TOSOLVE_EINVAL; }
    if (!handles[i]->graph_ready) { g_err = "handle built without graphs"; return TOSOLVE_EINVAL; }
    for (int j = 0; j < i; ++j)
      if (handles[j] == handles[i]) { g_err = "a handle appears twice in the batch"; return TOSOLVE_EINVAL; }
  }
  tosolve_batch_s* b = new (std::nothrow) tosolve_batch_s();
  if (b == nullptr) { g_err = "host allocation failed"; return TOSOLVE_ENOMEM; }
  b->hs.assign(handles, handles + count);
  b->nrhs.assign(nrhs, nrhs + count);
  b->f.assign(f_dev, f_dev + count);
  b->u.assign(u_dev, u_dev + count);
  for (int i = 0; i < count; ++i) b->total += nrhs[i];
  auto fail = [&](cudaError_t e, const char* what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();
    batch_free(b);
    delete b;
    return e == cudaErrorMemoryAllocation ? TOSOLVE_ENOMEM : TOSOLVE_ECUDA;
  };
#define CKB(call)                                  \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return fail(e_, #call); \
  } while (0)
  CKB(cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking));
  CKB(cudaStreamCreateWithFlags(&b->bs, cudaStreamNonBlocking));
  CKB(cudaEventCreateWithFlags(&b->evf, cudaEventDisableTiming));
  CKB(cudaEventCreateWithFlags(&b->evd, cudaEventDisableTiming));
  CKB(cudaEventCreate(&b->t0));
  CKB(cudaEventCreate(&b->t1));
  CKB(cudaMallocHost((void**)&b->hparams, 2 * sizeof(double)));
  CKB(cudaMallocHost((void**)&b->hst, (size_t)b->total * sizeof(DevState)));
  CKB(cudaMalloc((void**)&b->dparams, 2 * sizeof(double)));
  b->branch.resize(count, nullptr);
  b->ev.resize(count, nullptr);
  for (int i = 0; i < count; ++i) {
    CKB(cudaStreamCreateWithFlags(&b->branch[i], cudaStreamNonBlocking));
    CKB(cudaEventCreateWithFlags(&b->ev[i], cudaEventDisableTiming));
  }
  // record: fork one branch per instance, its load cases in sequence
  CKB(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaEventRecord(b->evf, b->st);
  int k = 0;
  for (int i = 0; i < count && e == cudaSuccess; ++i) {
    tosolve_s* h = b->hs[i];
    cudaStream_t si = b->branch[i];
    const size_t nd = h->lv[0].ndof;
    e = cudaStreamWaitEvent(si, b->evf, 0);
    if (e == cudaSuccess) launch_set_params(h->ds, b->dparams, si);
    for (int r = 0; r < b->nrhs[i] && e == cudaSuccess; ++r, ++k) {
      e = cudaMemcpyAsync(h->f, b->f[i] + r * nd, nd * 8, cudaMemcpyDeviceToDevice, si);
      if (e == cudaSuccess) e = cudaMemcpyAsync(h->u, b->u[i] + r * nd, nd * 8, cudaMemcpyDeviceToDevice, si);
      if (e == cudaSuccess) e = append_solve(h, si, b->bs);
      if (e == cudaSuccess) e = cudaMemcpyAsync(b->u[i] + r * nd, h->u, nd * 8, cudaMemcpyDeviceToDevice, si);
      if (e == cudaSuccess) e = cudaMemcpyAsync(&b->hst[k], h->ds, sizeof(DevState), cudaMemcpyDeviceToHost, si);
    }
    if (e == cudaSuccess) e = cudaEventRecord(b->ev[i], si);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->st, b->ev[i], 0);
  }
  cudaError_t e2 = cudaStreamEndCapture(b->st, &b->g);
  if (e != cudaSuccess) return fail(e, "batch capture");
  if (e2 != cudaSuccess) return fail(e2, "batch capture end");
  CKB(cudaGraphInstantiate(&b->ge, b->g, 0));
#undef CKB
  *out = b;
  return TOSOLVE_OK;
}

tosolve_status tosolve_batch_solve(tosolve_batch_t b, double rtol, int maxit, tosolve_info* infos) {
  if (b == nullptr) { g_err = "batch is NULL"; return TOSOLVE_EINVAL; }
  const int count = (int)b->hs.size();
  if (infos) std::memset(infos, 0, count * sizeof(tosolve_info));
  if (!(rtol > 0.0) || maxit < 1 || maxit > 100000) { g_err = "need rtol > 0 and 1 <= maxit <= 100000"; return TOSOLVE_EINVAL; }
  for (int i = 0; i < count; ++i)
    if (!b->hs[i]->have_rho) { g_err = "call tosolve_set_densities on every handle first"; return TOSOLVE_EINVAL; }
  auto cuda_fail = [&](cudaError_t e) {
    g_err = std::string("batch solve: ") + cudaGetErrorString(e);
    return TOSOLVE_ECUDA;
  };
  b->hparams[0] = rtol * rtol;
  b->hparams[1] = (double)maxit;
  cudaError_t e = cudaMemcpyAsync(b->dparams, b->hparams, 2 * sizeof(double), cudaMemcpyHostToDevice, b->st);
  for (int i = 0; i < count && e == cudaSuccess; ++i) {  // after everything issued on the handles
    e = cudaEventRecord(b->ev[i], b->hs[i]->st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->st, b->ev[i], 0);
  }
  if (e == cudaSuccess) e = cudaEventRecord(b->t0, b->st);
  if (e == cudaSuccess) e = cudaGraphLaunch(b->ge, b->st);
  if (e == cudaSuccess) e = cudaEventRecord(b->t1, b->st);
  if (e == cudaSuccess) e = cudaEventRecord(b->evd, b->st);
  for (int i = 0; i < count && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(b->hs[i]->st, b->evd, 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
  if (e != cudaSuccess) return cuda_fail(e);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, b->t0, b->t1);
  tosolve_status result = TOSOLVE_OK;
  int k = 0;
  for (int i = 0; i < count; ++i) {
    tosolve_s* h = b->hs[i];
    tosolve_info inf;
    std::memset(&inf, 0, sizeof(inf));
    inf.ms = ms;
    const size_t nd = h->lv[0].ndof;
    for (int r = 0; r < b->nrhs[i]; ++r, ++k) {
      const DevState& S = b->hst[k];
      double* ur = b->u[i] + r * nd;
      int used = S.iter;
      double rel = 0.0;
      tosolve_status st = TOSOLVE_OK;
      if (S.tc_status || S.tile_status) {
        st = TOSOLVE_ECUDA;
        h->err = "a tensor-core or operator tile copy did not complete within its bounded wait";
      } else if (S.ff == 0.0) {  // f = 0: the solution is u = 0
        e = cudaMemsetAsync(ur, 0, nd * 8, b->st);
        if (e != cudaSuccess) return cuda_fail(e);
        used = 0;
      } else {
        rel = std::sqrt(S.rr_true / S.ff);
        if (S.status != 0) {
          st = TOSOLVE_EBREAKDOWN;
        } else if (rel > rtol && used < maxit) {
          // the recursive residual met the tolerance, the true one did not:
          // finish this load case alone, warm-started from the batch result
          tosolve_info more;
          st = tosolve_solve(h, b->f[i] + r * nd, 1, ur, rtol, maxit - used, &more);
          used += more.total_iterations;
          rel = more.rel_residual;
        } else if (rel > rtol) {
          st = TOSOLVE_ENOTCONV;
        }
      }
      inf.iterations = used;
      inf.total_iterations += used;
      inf.rel_residual = std::fmax(inf.rel_residual, rel);
      if (st != TOSOLVE_OK && inf.status == TOSOLVE_OK) inf.status = st;
      if (st != TOSOLVE_OK && (result == TOSOLVE_OK || result == TOSOLVE_ENOTCONV)) result = st;
    }
    if (infos) infos[i] = inf;
  }
  e = cudaStreamSynchronize(b->st);
  if (e != cudaSuccess) return cuda_fail(e);
  if (result == TOSOLVE_ENOTCONV) g_err = "a load case reached maxit before the tolerance";
  else if (result == TOSOLVE_EBREAKDOWN) g_err = "breakdown in a load case (PCG, or a non-positive coarse pivot)";
  else if (result == TOSOLVE_ECUDA) g_err = "a tensor-core or operator tile copy did not complete within its bounded wait";
  return result;
}

void tosolve_batch_destroy(tosolve_batch_t b) {
  if (b == nullptr) return;
  if (b->st) cudaStreamSynchronize(b->st);
  batch_free(b);
  delete b;
}

}  // extern "C"
