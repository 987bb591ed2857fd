// Internal declarations of the tosolve library (not part of the C ABI).
//
// Data layout in HBM (all arrays owned by the handle, allocated once in
// tosolve_create):
//   * DOF vectors: 3 values per lattice node, node id i + Lx*(j + Ly*l);
//   * level operators: a 27-point stencil of 3x3 blocks per node, in tiles
//     of 32 consecutive nodes: S[((node/32)*243 + e)*32 + node%32] with
//     e = o*9 + 3r + c and neighbour offset o = (dx+1) + 3*((dy+1) +
//     3*(dz+1)).  A tile (243 x 32 coefficients) is one contiguous block
//     that a single bulk copy moves into shared memory, and within it one
//     warp reads the 32 nodes' coefficient e in one transaction.  The node
//     count is padded to whole tiles (padding coefficients are zero);
//   * element matrices: upper triangle (300 of 24x24) per element;
//   * density / design grid: one FP64 per cell, x fastest.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <functional>
#include <string>

#include "../../include/tosolve.h"
#include "dfloat.cuh"

namespace tos {

constexpr int kBS = 256;       // threads per block of the vector / stencil kernels
constexpr int kMaxPart = 608;  // partial sums per reduction (4 blocks per SM)
constexpr int kMaxLevels = 8;
constexpr int kEdofQ1 = 24;    // DOFs of a trilinear hexahedron
constexpr int kSym = 300;      // entries of a 24x24 symmetric upper triangle
constexpr int kNB = 32;        // largest pivot block of the coarse sweeps
constexpr int kTile = 32;      // output tile of the coarse inverse product
constexpr int kMaxCoarse = 4096;  // largest coarse system (DOFs)
constexpr int kTN = 32;        // nodes per operator tile
constexpr size_t kSlabBytes = size_t(1) << 30;  // element-matrix scratch of the refresh

// Scratch for the element matrices of the levels refreshed slab by slab
// (ex x ey x ez elements per level, up to kSym doubles each): whole levels
// when they fit in kSlabBytes, else slabs of at least two element layers.
inline size_t slab_scratch_bytes(const int* ex, const int* ey, const int* ez, int nlev) {
  size_t b = 0;
  for (int l = 0; l < nlev; ++l) {
    const size_t layer = (size_t)ex[l] * ey[l] * kSym * 8;
    const size_t full = layer * ez[l];
    size_t need = kSlabBytes > 2 * layer ? kSlabBytes : 2 * layer;
    if (need > full) need = full;
    if (need > b) b = need;
  }
  return b;
}

// Position of coefficient e (= o*9 + 3r + c) of node in a level operator.
__host__ __device__ inline size_t op_idx(long node, int e) {
  return ((size_t)(node / kTN) * 243 + e) * kTN + (size_t)(node % kTN);
}
// Coefficients stored for a level of nn nodes (whole tiles).
inline size_t op_len(long nn) { return (size_t)((nn + kTN - 1) / kTN) * 243 * kTN; }

// Scalars of the PCG loop, kept on the device so the loop runs as a CUDA
// graph with a device-side while condition.
struct DevState {
  double ff;       // ||f||^2
  double rr;       // ||r||^2 (recursive residual)
  double rz;       // r^T z of the current direction
  double rz_next;  // r^T z of the next direction (written by cg_dir)
  double alpha;    // step of the last update
  double beta;
  double tol2;     // rtol^2
  double rr_true;  // ||f - K u||^2 after the loop
  double c;        // compliance f^T u
  int iter;
  int maxit;
  int status;      // 0 ok, TOSOLVE_EBREAKDOWN on breakdown
  int converged;
  int coarse_status;  // non-zero if the coarse sweeps met a non-positive pivot
  int tc_status;      // non-zero if a tensor-core tile wait timed out
  int tile_status;    // non-zero if an operator tile copy wait timed out
  int pad;
  // inner FP32 PCG (the preconditioner of the outer flexible CG)
  double in_rho;      // ri^T z of the current inner direction
  double in_rho_next; // ri^T z of the next inner direction
  double in_alpha;    // inner step
  double in_beta;     // inner flexible coefficient
};

// One Chebyshev smoothing step fused into an operator gather (mode 3):
//   out = v + c1 dprev + c2 D^-1 (b - A v),  dout = out - v,
// with c1 = coef[2 ci], c2 = coef[2 ci + 1] for ci >= 0, and c1 = 0, c2 = 1
// for ci < 0 (the first step from a nonzero iterate: the level's D^-1 is
// already divided by theta).  dprev null: the previous iterate was 0, so
// dprev = v.  out may alias v and dout dprev (element-wise updates).
struct ChebStep {
  const void* dprev = nullptr;
  void* dout = nullptr;
  const void* coef = nullptr;  // the level's coefficients in the vector type
  int ci = -1;
};

struct Level {
  int ex, ey, ez;   // elements per axis
  int Lx, Ly, Lz;   // node lattice
  int nn, ndof;
  int nsub;         // density cells per element edge at this level
  double h;         // element edge length
  bool op64;        // operator stored in FP64 for the V-cycle
  int sms = 1;      // SMs of the device (grid of the tile kernels)
  int* err = nullptr;  // set when an operator tile copy times out
  int k = 1;        // Lagrange degree of the level's elements
  const float* ptab = nullptr;  // shape-function transfers into this level: the table W (else null)
  bool lag = false;             // ... products of 1D quadratic Lagrange transfers (degree 2 -> 2)
  // degree 2: the operator as element matrices (81 x 81 each, full, or
  // packed symmetric when sym: kPS2 entries per element)
  bool sym = false;
  double* K64 = nullptr;
  float* K32 = nullptr;
  // serendipity levels: the compact matrices of the element's own DOFs
  // (60 x 60 for degree 2, 96 x 96 for degree 3), read by the apply
  double* Kc64 = nullptr;
  float* Kc32 = nullptr;
  void* Y = nullptr;  // per-element results of an apply (shared scratch)
  // mixed trilinear / triquadratic level 0: the triquadratic elements (el2,
  // ne2; sl2 the 27-bit masks of their slaved local nodes) and the
  // trilinear ones (el1, ne1), ascending; null elsewhere
  const int* el2 = nullptr;
  long ne2 = 0;
  const uint32_t* sl2 = nullptr;
  const int* el1 = nullptr;
  long ne1 = 0;
  const uint8_t* slv = nullptr;  // per lattice node, 1 = slaved (mixed level 0 on tensor cores)
  float* yraw = nullptr;         // its raw assembled products before the fold (ndof)
  const uint32_t* vnb = nullptr; // per vertex of the lattice, its slaved neighbours (27-bit)
  uint8_t* mask = nullptr;
  int* tl = nullptr;    // tile order in force (LevelView::tl), or null: index order
  int* tcnt = nullptr;  // number of tiles with a free DOF (device), with tl
  int* tl_buf = nullptr;    // level 0: storage of the order used after a suppression
  int* tcnt_buf = nullptr;
  double* S64 = nullptr;   // FP64 stencil (level 0 always; others when op64)
  float* S32 = nullptr;    // FP32 stencil (FP32 preconditioner levels)
  double* dinv64 = nullptr;
  float* dinv32 = nullptr;
  // Chebyshev smoothing (degree >= 2 hierarchies): steps before and after
  // the coarse correction (0: damped Jacobi), the step difference vector,
  // and the coefficients (c1, c2 theta) of steps 2.. in FP64 and FP32
  int cheb = 0;
  void* d = nullptr;
  double* cheb64 = nullptr;
  float* cheb32 = nullptr;
  void* b = nullptr;  // V-cycle vectors in the preconditioner precision
  void* v = nullptr;
  void* r = nullptr;
  void* z = nullptr;
};

// Arithmetic of the multigrid vectors: FP64, FP32, or float pairs (FP32X2,
// on FP32 operators).
enum Vt : int { kVtF64 = 0, kVtF32 = 1, kVtDF = 2 };

// Storage type of the operator and Jacobi diagonal used with vectors of T.
template <typename T>
struct OpOf { using type = T; };
template <>
struct OpOf<dfloat> { using type = float; };
template <typename T>
using op_t = typename OpOf<T>::type;

// Density grid (Dx, Dy, Dz; n cells per element edge) and a coarser design
// grid (Gx, Gy, Gz; d per edge) of the projection, radius r in element
// units; R bounds the design-cell offsets a density cell can reach.
struct ProjGrid {
  int Dx, Dy, Dz, Gx, Gy, Gz, n, d, R;
  double r;
};

// Read-only view of a level's operator for the kernels.
template <typename T>
struct LevelView {
  int Lx, Ly, Lz, nn;
  const op_t<T>* S;
  const op_t<T>* dinv;
  const uint8_t* mask;
  int* err;
  int sms;
  // Operator tiles in processing order, or null for index order: the
  // tcnt[0] tiles that hold a free DOF first, then the tiles whose 32 nodes
  // are all fixed (identity rows: y = x there, no coefficients read).
  const int* tl;
  const int* tcnt;
};

// ---- launchers (k_setup.cu) ----------------------------------------------
void launch_proj_init(const ProjGrid& P, double* invom, cudaStream_t st);
void launch_proj_fwd(const ProjGrid& P, const double* invom, const double* x, double Emin, double dE,
                     double penal, double* rho, double* w, cudaStream_t st);
void launch_proj_T(const ProjGrid& P, const double* gt, double* gx, cudaStream_t st);
void launch_subcell_table(int n, double nu, double h, double* tab, cudaStream_t st);
void launch_symmetrize(int m, const double* tab, double* tabsym, cudaStream_t st);
void launch_moment_basis(double nu, double* cmom, cudaStream_t st);
void launch_filter_init(int Dx, int Dy, int Dz, int noff, const int4* off, const double* wgt,
                        double* invom, cudaStream_t st);
void launch_filter_fwd(int Dx, int Dy, int Dz, int noff, const int4* off, const double* wgt,
                       const double* invom, const double* x, double Emin, double dE,
                       double penal, double* rho, double* w, cudaStream_t st);
// Element matrices of the element z-layers [ze0, ze1), written from the
// start of Ke (a slab of the level).
void launch_elem_direct(bool fp64, const Level& L, int ze0, int ze1, int n, const double* w, int Dx,
                        int Dy, const double* tabsym, void* Ke, cudaStream_t st);
void launch_elem_moments(bool fp64, const Level& L, int ze0, int ze1, const double* w, int Dx, int Dy,
                         const double* cmom, void* Mscr, void* Ke, cudaStream_t st);
// Stencil rows of the node z-layers [l0, l1) from a slab of element matrices
// that starts at element layer ze0.
void launch_assemble(bool fp64, const Level& L, int l0, int l1, int ze0, const void* Ke, void* S,
                     void* dinv, cudaStream_t st);
// Splits a level into z-slabs whose element matrices (elem_bytes each) fit
// in scratch_bytes: fn(l0, l1, ze0, ze1) for node layers [l0, l1) and the
// element layers [ze0, ze1) they touch (consecutive slabs share one layer).
void for_each_slab(const Level& L, size_t scratch_bytes, size_t elem_bytes,
                   const std::function<void(int, int, int, int)>& fn);
void launch_to_fp32(size_t n, const double* a, float* b, cudaStream_t st);
void launch_coarse_dense(const Level& L, double* A, cudaStream_t st);
cudaError_t launch_coarse_invert(int n, double* A, double* W, double* V, double* Pg, double* Ainv,
                                 int* status, int grid, cudaStream_t st);
int coarse_sweep_grid();

// ---- launchers (k_tc.cu) -------------------------------------------------
// Finest-level operator of the TF32 preconditioner on tcgen05.
struct TcOp {
  bool on = false;
  int deg = 1;              // Lagrange degree of the finest level
  int mode = 0;             // degree 2: operands (tc2_mode_of: TF32, BF16, BF16X3, F16X3)
  int prec = 0;             // degree 2: the tosolve_precision this mode serves
  float tscale = 1.f;       // degree 2, F16X3: power-of-two scale of the table image
  unsigned char* apack = nullptr;  // degree 2: the packed A tiles (tc2_pack_bytes)
  float* escale = nullptr;         // degree 2, F16X3: per listed element, its row scale
  int m = 1;                // subcells per element
  const float* w32 = nullptr;  // E x m element-major weights
  const float* KT = nullptr;   // degree 1: m x 24 x 24 FP32 table
  float* Ye = nullptr;         // degree 1: E x 24 element results
  const unsigned char* img = nullptr;  // degree 2: stacked table in the shared-memory image
  float* Y2 = nullptr;         // degree 2: E x tc2_result_stride() element results
  const float* K1v = nullptr;  // mixed meshes: ne1 x kQ1Sym FP32 trilinear vertex blocks (packed)
  int* err = nullptr;
  int sms = 1;
};
// Message returned by tosolve_last_error(NULL) for calls that have no handle.
void set_last_error(const char* msg);
bool tc_supported(int n);
cudaError_t launch_tc_apply(const Level& L0, int m, const float* v, const float* w32, const float* KT,
                            float* Ye, int* err, int sms, cudaStream_t st);
void launch_tc_gather(const Level& L0, const float* Ye, const float* b, const float* v, const float* dinv,
                      float omega, int mode, float* out, cudaStream_t st);
void launch_weights_elem(const Level& L0, int n, const double* w, int Dx, int Dy, float* w32,
                         cudaStream_t st);
void launch_mask_fp32(const Level& L, float* x, cudaStream_t st);

// ---- launchers (k_tc2.cu): degree-2 finest level on tcgen05 ---------------
// n_mr with a tensor-core kernel for degree 2 (m = n^3 subcells: 1, 8, 27).
bool tc2_supported(int n);
// Packed upper triangle of a trilinear element's 24 x 24 vertex block.
constexpr int kQ1Sym = 24 * 25 / 2;
// FP32 packed vertex blocks of the trilinear elements of a mixed level 0
// (L0.el1 order) from the level's FP64 element matrices K64.
void launch_q1v_compact32(const Level& L0, const double* K64, float* K1v, cudaStream_t st);
// Operand mode of a tensor-core precision: TF32 0, BF16 1, BF16X3 2, F16X3 3.
inline int tc2_mode_of(int precision) {
  return precision == TOSOLVE_PREC_TF32 ? 0 : precision == TOSOLVE_PREC_BF16 ? 1
                                         : precision == TOSOLVE_PREC_BF16X3 ? 2 : 3;
}
// Bytes of the stacked triquadratic table's shared-memory image for an
// operand mode.
size_t tc2_image_bytes(int mode, int m);
// Floats per element in the result buffer (81 rounded up to 16 bytes).
size_t tc2_result_stride();
// Bytes of the packed A tiles for E elements (whole work units).
size_t tc2_pack_bytes(int mode, long E);
// Power-of-two scale of the table image (F16X3: largest entry into
// [0.5, 1) after dividing by it; else 1), from the host copy of the table.
float tc2_table_scale(int mode, const double* tab_host, size_t count);
void launch_tc2_image(int mode, int m, const double* tab, float tscale, unsigned char* img, cudaStream_t st);
// tc.Y2 = per-element stacked contraction of the level-0 vector v (fixed
// DOFs as zero), weights tc.w32 (E x m); on a mixed level 0 the triquadratic
// elements with their slaved nodes (T_e^T K T_e), and the trilinear ones on
// their vertices by FP32 products with tc.K1v on the CUDA cores.  part: -1
// every element, 0 the triquadratic (all on a single-degree mesh), 1 the
// trilinear ones of a mixed mesh; stages: bit 0 packs the operand rows,
// bit 1 runs the contraction on the packed rows (and, with part 1 or with
// part -1 without bit 0, the trilinear products; part -1 with both bits
// runs them beside the row packing).
cudaError_t launch_tc2_apply(const TcOp& tc, const Level& L0, const float* v, cudaStream_t st, int part = -1,
                             int stages = 3);
// Node gather of Y fused with the V-cycle step: mode 0 b - y, 1 v + omega
// D^-1 (b - y), 2 y; identity rows at fixed DOFs.
void launch_tc2_gather(const Level& L0, const float* Y, const float* b, const float* v, const float* dinv,
                       float omega, int mode, float* out, cudaStream_t st, const ChebStep* cs = nullptr);

// ---- launchers (k_solve.cu) ----------------------------------------------
template <typename T>
LevelView<T> view(const Level& L);
// Operands of the PCG step that follows the V-cycle (r^T z, z^T q and beta,
// as launch_cg_dots_rz): when the finest level's last smoothing step is a
// stencil kernel, launch_vcycle folds this reduction into it and returns
// true; otherwise the caller launches launch_cg_dots_rz.
struct CgDots {
  const double* r;
  const double* q;
  double* part_rz;  // kMaxPart partials each
  double* part_zq;
  DevState* ds;
  unsigned* cnt;
};
bool launch_vcycle(int vt, Level* lv, int L, double omega, int gamma, const double* Ainv,
                   const TcOp& tc, cudaStream_t st, const CgDots* dots = nullptr);
// Vectors of the inner FP32 PCG on level 0 (ndof floats each).
struct InnerPcg {
  int its = 0;           // inner iterations per outer iteration (0: the V-cycle alone)
  float* e = nullptr;    // inner solution
  float* ri = nullptr;   // inner residual
  float* pi = nullptr;   // inner direction
  float* qi = nullptr;   // A pi
};
// z0 = approximation of A0^-1 b0 by `its` iterations of FP32 PCG on the
// level-0 preconditioner operator (tensor cores when tc.on, else the FP32
// element matrices), each preconditioned by one V-cycle; b0 and v0 = omega
// D^-1 b0 are set by the outer kernels.  Reductions in FP64, fixed order.
// Chebyshev smoothing set-up: for every level with lv[l].cheb > 0, `steps`
// Lanczos steps estimate lambda_max(D^-1 A) of its smoothing operator, the
// step coefficients go to lv[l].cheb64 / cheb32 and the level's D^-1 (of the
// vector type vt, FP64 or FP32) is divided by theta.  part: kMaxPart
// doubles, cnt a zeroed counter, lz 64 doubles of scratch; lmax_out (device,
// optional) receives each level's estimate.
void launch_cheb_setup(int vt, Level* lv, int L, const TcOp& tc, int steps, double* part, unsigned* cnt,
                       double* lz, double* lmax_out, cudaStream_t st);
void launch_inner_pcg(Level* lv, int L, double omega, const double* Ainv, const TcOp& tc, const InnerPcg& in,
                      double* part_a, double* part_b, DevState* ds, unsigned* cnt, cudaStream_t st);
void launch_smooth0(int vt, const Level& L0, double omega, cudaStream_t st);
void launch_set_params(DevState* ds, const double* params, cudaStream_t st);
void launch_cg_prep(const Level& L0, double* f, double* u, double* part, int np, cudaStream_t st);
void launch_cg_residual(int vt, const Level& L0, double omega, const double* f, const double* u,
                        double* r, int mode, double* part, const double* part_ff, int np,
                        DevState* ds, unsigned* cnt, cudaGraphConditionalHandle hc, int use_cond,
                        cudaStream_t st);
void launch_cg_dots_rz(int vt, const Level& L0, const double* r, const double* q, double* part_rz,
                       double* part_zq, int np, DevState* ds, unsigned* cnt, cudaStream_t st);
void launch_cg_dir(int vt, const Level& L0, double* p, int np, const DevState* ds,
                   cudaStream_t st);
void launch_cg_apply(const Level& L0, const double* p, double* q, double* part, int np, DevState* ds,
                     unsigned* cnt, cudaStream_t st);
void launch_cg_update(int vt, const Level& L0, double omega, double* u, double* r, const double* p,
                      const double* q, double* part_rr, int np, DevState* ds, unsigned* cnt,
                      cudaGraphConditionalHandle hc, int use_cond, cudaStream_t st);
void launch_apply_diag(int vt, const Level& L, const double* x, double* y, cudaStream_t st);
// Lets the stencil tile kernels use their shared-memory ring (once per
// process and device, before the first launch).
cudaError_t configure_tile_kernels();

// ---- launchers (k_q2.cu): Lagrange degree 2 in element form ---------------
constexpr int kD2 = 81;       // DOFs of a triquadratic element
constexpr int kDD2 = 81 * 81;
constexpr int kNM2 = 125;     // moments of a degree-2 element matrix
constexpr int kD3 = 192;      // DOFs of a tricubic element
constexpr int kDD3 = 192 * 192;
// Lagrange degree-2 levels formed by sum factorisation keep each element
// matrix as its packed upper triangle, row by row (kSym2 entries, stride
// kPS2 so that every element starts on a 16-byte boundary); the others keep
// the full kD x kD matrix.
constexpr int kSym2 = 81 * 82 / 2;
constexpr int kPS2 = 3324;
__host__ __device__ inline int sym2_idx(int R, int C) {
  if (R > C) {
    const int t = R;
    R = C;
    C = t;
  }
  return R * 81 - R * (R - 1) / 2 + C - R;
}
void launch_q2_subcell_table(int n, double nu, double h, int family, double* tab, cudaStream_t st);
void launch_q2_moment_basis(double nu, int family, double* cmom, cudaStream_t st);
// Degree-3 subcell tables (family 0 Lagrange, 1 the 32-node serendipity
// element): grad_scratch holds n^3 * 64 * 64 * 3 doubles.
void launch_q3_subcell_table(int n, double nu, double h, int family, double* grad_scratch, double* tab,
                             cudaStream_t st);
// Serendipity levels: Kc64 / Kc32 from K64 (after every refresh of K64).
void launch_ser_compact(const Level& L, cudaStream_t st);
// Degree-2 levels with shape-function transfers (always for the serendipity
// element): W = the 27 x 125 table of coarse shape values at the fine
// lattice points of a coarse element (device, FP32).
void launch_s2_restrict(int vt, const Level& F, const Level& C, const float* W, const void* dinvc, double omega,
                        void* vc, cudaStream_t st);
void launch_s2_prolong(int vt, const Level& F, const Level& C, const float* W, cudaStream_t st);
void launch_q2_elem(const Level& L, int n, const double* w, int Dx, int Dy, const double* tab,
                    double* Ke, cudaStream_t st);
// Lagrange degree 2: element matrices of any level by sum factorisation over
// the moments of its N^3 density cells per element (N = L.nsub <= 64); with
// a list only the listed elements; with slv (per lattice node, 1 = slaved)
// each element's matrix is constrained, T_e^T K T_e.
bool q2_elem_sf_supported(int N);
inline bool elem_sym(int family, int k, int nsub) { return family == 0 && k == 2 && q2_elem_sf_supported(nsub); }
void launch_q2_elem_sf(const Level& L, const double* w, int Dx, int Dy, double nu, const int* list, long count,
                       const uint8_t* slv, double* Ke, cudaStream_t st);
// Trilinear elements of a mixed level 0 (L.el1): sum of the n^3 weighted
// trilinear subcell matrices tab1 (m x 24 x 24), on the vertex DOFs of each
// element's 81 x 81 slot, zero elsewhere.
void launch_q1v_elem(const Level& L, int n, const double* w, int Dx, int Dy, const double* tab1, double* Ke,
                     cudaStream_t st);
void launch_q2_coarse_elem(const Level& L, const double* w, int Dx, int Dy, const double* cmom,
                           double* Mscr, double* Ke, cudaStream_t st);
void launch_q2_dinv(bool fp64, const Level& L, const double* Ke, void* dinv, cudaStream_t st);
void launch_q2_dense(const Level& L, const double* Ke, double* A, cudaStream_t st);
// The FP32 copy of a level's element matrices (in the FP64 ones' layout).
void launch_elem_fp32(const Level& L, const double* K64, float* K32, cudaStream_t st);
// Entries per element matrix of a degree >= 2 level.
inline size_t elem_stride(const Level& L) {
  return L.sym ? (size_t)kPS2 : (L.k == 3 ? (size_t)kDD3 : (size_t)kDD2);
}
// out = f(A_l v) in vector type vt: mode 0 b - Av, 1 v + omega D^-1 (b - Av),
// 2 Av (identity rows at fixed DOFs).  Ke is FP64 for kVtF64, else FP32.
void launch_q2_op(int vt, const Level& L, const void* Ke, void* Y, const void* b, const void* v,
                  const void* dinv, double omega, int mode, void* out, int sms, cudaStream_t st,
                  const ChebStep* cs = nullptr);
// Mixed degree: f <- T^T f; u <- T u (slv: per lattice node, 1 = slaved).
void launch_q2_fold(const Level& L, const uint8_t* slv, double* f, cudaStream_t st);
void launch_q2_expand(const Level& L, const uint8_t* slv, double* u, cudaStream_t st);
// Lagrange degree 2: the same sensitivities from the strain energy at the
// tensor Gauss points, by sum factorisation (n <= 4).
bool q2_energy_sf_supported(int n);
void launch_q2_energy_sf(const Level& L0, int n, double nu, const double* u, const double* rho, double penal,
                         double dE, int Dx, int Dy, bool first, double* g, int sms, cudaStream_t st);
void launch_q2_energy_grad(const Level& L0, int n, const double* u, const double* tab,
                           const double* rho, double penal, double dE, int Dx, int Dy, bool first,
                           double* g, int sms, cudaStream_t st);
// FP64 vector <-> multigrid vector of arithmetic vt.
void launch_vec_in(int vt, size_t n, const double* a, void* b, cudaStream_t st);
void launch_vec_out(int vt, size_t n, const void* a, double* b, cudaStream_t st);
void launch_cast(bool to_fp64, size_t n, const void* a, void* b, bool src_fp64,
                 cudaStream_t st);

// ---- launchers (k_fix.cu): fixing variables, Sec. 6.1 ----------------------
void launch_fix_classify(const Level& L0, int n, int d, const double* rho, const double* g, double lo,
                         double hi, double eps, int8_t* cls, cudaStream_t st);
void launch_fix_surround(const Level& L0, const int8_t* cls, int8_t* fixed, cudaStream_t st);
void launch_fix_design(const Level& L0, int d, const int8_t* fixed, uint8_t* out, cudaStream_t st);
void launch_fix_mask(const Level& L0, const int8_t* fixed, const uint8_t* base, cudaStream_t st);
void launch_zero_fixed_void(long n, const uint8_t* xfix, double* g, cudaStream_t st);

// ---- thresholding and the Heaviside projection (k_thresh.cu), Sec. 5 -------
size_t threshold_scratch_bytes(long n);
tosolve_status heaviside(const double* rho, long n, double beta, double* out, double* eta_out, int* its_out,
                         void* scratch, size_t bytes, cudaStream_t st, std::string* why);
tosolve_status threshold_density(const double* rho, long n, double vfrac, double lo, double hi, const double* grad,
                                 double theta_deg, double* out, int* accepted, void* scratch, size_t bytes,
                                 cudaStream_t st, std::string* why);
tosolve_status threshold_gradient(const double* rho, long n, double lo, double hi, const double* grad, double vu,
                                  double vl, double theta_deg, double* out, double* alpha_out, void* scratch,
                                  size_t bytes, cudaStream_t st, std::string* why);

// ---- launchers (k_grad.cu) -----------------------------------------------
void launch_energy_grad(const Level& L0, int n, const double* u, const double* tabsym,
                        const double* rho, double penal, double dE, int Dx, int Dy,
                        bool first, double* g_rho, cudaStream_t st);
void launch_scale(size_t n, const double* a, const double* s, double* out, cudaStream_t st);
void launch_filter_T(int Dx, int Dy, int Dz, int noff, const int4* off, const double* wgt,
                     const double* gt, double* gx, cudaStream_t st);
// c = f^T u over the DOFs that fixed marks 0 (the supports only: slaved DOFs
// of a mixed mesh carry load and displacement).
void launch_compliance(const Level& L0, const uint8_t* fixed, const double* f, const double* u,
                       double* part, int np, DevState* ds, cudaStream_t st);

// Blocks of the node-parallel solve kernels (64 nodes per block); also the
// number of partial sums their reductions produce.
inline int parts_for(long nn) {
  long g = (nn + 63) / 64;
  return (int)(g < kMaxPart ? (g < 1 ? 1 : g) : kMaxPart);
}

__host__ __device__ inline int sym_index(int r, int c) {
  // r <= c < 24: row-major upper triangle
  return r * kEdofQ1 - (r * (r - 1)) / 2 + (c - r);
}

// x^p of the SIMP law (Eq. matrixK): repeated products when p is a small
// non-negative integer (the paper's p = 3), else pow.  FP64 is scarce on
// this part and pow costs dozens of FP64 instructions.
__device__ __forceinline__ double simp_pow(double x, double p) {
  if (p >= 0.0 && p <= 8.0 && (double)(int)p == p) {
    double r = 1.0;
    for (int q = 0; q < (int)p; ++q) r *= x;
    return r;
  }
  return pow(x, p);
}

}  // namespace tos

// The opaque handle of the C ABI.
struct tosolve_s {
  tosolve_desc d;
  cudaStream_t st = nullptr;
  cudaStream_t st2 = nullptr;  // coarse-level chain of the refresh
  cudaEvent_t evf = nullptr, evj = nullptr;
  bool own_stream = false;
  int dev = 0;
  int L = 1;
  tos::Level lv[tos::kMaxLevels];
  int Dx = 0, Dy = 0, Dz = 0, ncell = 0;
  int m = 1;  // subcells per fine element
  // density side
  double* rho = nullptr;
  double* w = nullptr;
  double* invom = nullptr;
  int noff = 0;
  int4* foff = nullptr;
  double* fwgt = nullptr;
  double* gtmp = nullptr;
  // element tables
  double* tab64 = nullptr;     // m x 24 x 24 (degree 2: m x 81 x 81)
  double* tabsym64 = nullptr;  // m x 300
  double* cmom64 = nullptr;    // 27 x 300 (degree 2: 125 x 81 x 81)
  double* Yq = nullptr;        // degree 2: per-element apply results (E0 x 81)
  double* Mq = nullptr;        // degree 2: moments of the finer coarse levels
  double* Mqc = nullptr;       // degree 2: moments of the coarsest level
  // mixed trilinear / triquadratic mesh (degree-2 lattice)
  bool proj = false;           // design grid coarser than the density grid
  tos::ProjGrid pg = {};
  long ndes = 0;               // design variables
  bool mixed = false;
  long long free_dofs = 0;     // unknowns: DOFs neither supported nor slaved
  uint8_t* slv0 = nullptr;     // per lattice node: 1 = slaved to its vertices
  int* el2 = nullptr;          // triquadratic elements (ascending)
  uint32_t* sl2 = nullptr;     // their slaved local nodes (bit a = local node a)
  int* el1 = nullptr;          // trilinear elements (ascending)
  long ne2 = 0, ne1 = 0;
  double* tab64q1 = nullptr;   // trilinear subcell table of a mixed mesh
  float* tcyraw = nullptr;          // raw assembled products before the slaved fold
  float* tck1v = nullptr;           // FP32 packed vertex blocks of the trilinear elements
  uint32_t* tcvnb = nullptr;        // per lattice vertex, its slaved neighbours (bit (dx+1)+3(dy+1)+9(dz+1))
  // Chebyshev smoothing: Lanczos scratch (64) and each level's estimate of
  // lambda_max(D^-1 A) (mg_levels)
  double* lz = nullptr;
  double* lmax = nullptr;
  uint8_t* fix0 = nullptr;     // per DOF: the supports alone (level 0 mask adds slaved)
  // fixing variables (Sec. 6.1)
  float* ptab = nullptr;         // shape-function transfer table (27 x 125)
  float* ptab3 = nullptr;        // degree 3 -> 2 transfer table (27 x 64)
  uint8_t* base0 = nullptr;    // level-0 mask before suppression (supports, slaved)
  int8_t* ecls = nullptr;      // per element: 1 void, 2 solid, 0 neither
  int8_t* efix = nullptr;      // per element: the class if fixed, else 0
  uint8_t* xfix = nullptr;     // per design variable: the class of its fixed element
  bool fixing = false;
  long long free_base = 0;     // unknowns without suppression
  float* KT32 = nullptr;       // m x 24 x 24 FP32 (tensor-core operand)
  float* w32 = nullptr;        // E x m element-major FP32 weights
  float* Ye = nullptr;         // E x 24 element results of the tensor-core apply
  unsigned char* tcimg = nullptr;  // degree 2: the stacked table as shared-memory chunk images
  unsigned char* tcpack = nullptr; // degree 2: packed A tiles of the tensor-core apply
  float* tcscale = nullptr;        // degree 2: their per-element scales
  float* Y2 = nullptr;         // degree 2: element results of the tensor-core apply
  tos::TcOp tc;
  tos::InnerPcg inner;
  void* Ke = nullptr;
  size_t ke_bytes = 0;     // size of Ke (slab_scratch_bytes)
  double* Kec = nullptr;  // element matrices of the coarsest level (second stream)
  double* Mom = nullptr;   // 27 moments per element, finer coarse levels
  double* Momc = nullptr;  // 27 moments per element, coarsest level
  // coarse level
  int nc = 0;
  double* Ad = nullptr;
  double* Wp = nullptr;    // block-row scratch of the sweeps, nc x kNB
  double* Vp = nullptr;    // the same rows before the sweep, nc x kNB
  double* Pg = nullptr;    // the next pivot block's -P^{-1}, kNB x kNB
  double* Ainv = nullptr;
  int cgrid = 1;
  // PCG
  double *u = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *f = nullptr;
  double *tmpa = nullptr, *tmpb = nullptr;
  double* part = nullptr;  // 4 x kMaxPart
  unsigned* cnt = nullptr; // last-block counters of the fused reductions (4)
  int np = 1;
  tos::DevState* ds = nullptr;
  tos::DevState* hs = nullptr;  // pinned mirror
  bool graph_ready = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaGraphConditionalHandle hcond = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // host-step staging
  double *hx = nullptr, *hf = nullptr, *hu = nullptr, *hg = nullptr;
  int hrhs = 0;
  bool have_u = false;
  bool have_rho = false;
  std::string err;
  size_t bytes = 0;
};
