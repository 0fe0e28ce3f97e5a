// Internal declarations shared by the host code (hg_host.cpp, hg_gmg.cpp) and
// the CUDA kernels (*.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/hytet.h"

#if defined(__CUDACC__)
#define HG_HD __host__ __device__ __forceinline__
#else
#define HG_HD inline
#endif

namespace hg {

// ---------------------------------------------------------------- indexing
// Tetrahedral / triangular numbers and the linearisation t_w (Sec. 4).
HG_HD int64_t ntet(int64_t w) { return w > 0 ? w * (w + 1) * (w + 2) / 6 : 0; }
HG_HD int64_t ntri(int64_t w) { return w > 0 ? w * (w + 1) / 2 : 0; }
HG_HD int64_t tw(int64_t w, int64_t i, int64_t j, int64_t k) {
  return ntet(w) - ntet(w - k) + ntri(w - k) - ntri(w - k - j) + i;
}
// 32-bit variants for device loops (valid for w <= 1025).
HG_HD int ntet32(int w) { return w > 0 ? w * (w + 1) * (w + 2) / 6 : 0; }
HG_HD int ntri32(int w) { return w > 0 ? w * (w + 1) / 2 : 0; }
HG_HD int tw32(int w, int i, int j, int k) {
  return ntet32(w) - ntet32(w - k) + ntri32(w - k) - ntri32(w - k - j) + i;
}
// Start of row (j,k) of I_tet(w) and the offset of plane k.
HG_HD int row_start(int w, int j, int k) { return tw32(w, 0, j, k); }

// 15-point neighbourhood of a micro-vertex: centre + 7 lattice edge
// directions and their negatives.  Order fixed here and used everywhere.
//   0:(0,0,0)
//   1:(+1,0,0)  2:(-1,0,0)  3:(0,+1,0)  4:(0,-1,0)  5:(0,0,+1)  6:(0,0,-1)
//   7:(-1,+1,0) 8:(+1,-1,0) 9:(-1,0,+1) 10:(+1,0,-1)
//  11:(0,-1,+1) 12:(0,+1,-1) 13:(+1,-1,+1) 14:(-1,+1,-1)
constexpr int kNDir = 15;
#if defined(__CUDACC__)
__host__ __device__
#endif
inline void dir_offset(int d, int& di, int& dj, int& dk) {
  const signed char t[15][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                                {0, 0, 1},  {0, 0, -1}, {-1, 1, 0}, {1, -1, 0}, {-1, 0, 1},
                                {1, 0, -1}, {0, -1, 1}, {0, 1, -1}, {1, -1, 1}, {-1, 1, -1}};
  di = t[d][0];
  dj = t[d][1];
  dk = t[d][2];
}

// Boundary class of a cell-local point: bit0 on face opposite v0
// (i+j+k = n), bit1 on i = 0 (opposite v1), bit2 on j = 0, bit3 on k = 0.
// Row item r -> (cell, j, k) of a lattice with w points per macro edge
// (cells of ntri(w) rows each; plane k has w-k rows).
HG_HD void row_item(int w, int r, int& cell, int& j, int& k) {
  const int per = (int)ntri(w);
  cell = r / per;
  const int rr = r - cell * per;
  const float q = 2.0f * w + 1.0f;
  const float disc = q * q - 8.0f * rr;
  int kk = (int)floorf((q - sqrtf(disc > 0.0f ? disc : 0.0f)) * 0.5f);
  if (kk < 0) kk = 0;
  while ((kk + 1) * (2 * w - kk) / 2 <= rr) ++kk;
  while (kk * (2 * w - kk + 1) / 2 > rr) --kk;
  k = kk;
  j = rr - kk * (2 * w - kk + 1) / 2;
}

HG_HD int point_class(int n, int i, int j, int k) {
  return (i + j + k == n ? 1 : 0) | (i == 0 ? 2 : 0) | (j == 0 ? 4 : 0) | (k == 0 ? 8 : 0);
}

// Per-(cell, class) flags.
// CF_MULTI: the point lies on a macro primitive contained in two or more
// cells, so its value is a sum over copies (the interface items form it).
enum : uint8_t { CF_DIRICHLET = 1, CF_OWNER = 2, CF_MULTI = 4 };

// Point of a macro primitive, seen from one of the cells that contain it.
struct IfaceCopy {
  int32_t cell;
  int8_t loc[4];  // cell-local vertex index (0..3) of the primitive's vertex m; -1 unused
};
// A macro primitive (vertex, edge or face) shared by >= 1 cells.
struct IfacePrim {
  int32_t dim;         // 0 vertex, 1 edge, 2 face
  int32_t ncopies;     // cells containing it (sorted ascending cell id)
  int32_t first_copy;  // index into the copy array
  int32_t dirichlet;   // 1 if on the domain boundary
};

// Number of interior points of a primitive at n intervals per macro edge.
HG_HD int prim_points(int dim, int n) {
  return dim == 0 ? 1 : dim == 1 ? (n - 1 > 0 ? n - 1 : 0) : (int)ntri(n - 2);
}
// Barycentric weights (over the primitive's vertices, sorted by global id)
// of point p of a primitive.  Faces: rows b = 1..n-2, a = 1..n-1-b.
HG_HD void prim_point_weights(int dim, int n, int p, int wts[3]) {
  if (dim == 0) {
    wts[0] = n; wts[1] = 0; wts[2] = 0;
  } else if (dim == 1) {
    int t = p + 1;
    wts[0] = n - t; wts[1] = t; wts[2] = 0;
  } else {
    // row b has n-1-b points (a = 1..n-1-b); rows b = 1..n-2
    int b = 1, rem = p;
    while (rem >= n - 1 - b) { rem -= n - 1 - b; ++b; }
    int a = rem + 1;
    wts[0] = n - a - b; wts[1] = a; wts[2] = b;
  }
}
// Cell-local (i,j,k) of a primitive point given the copy's local vertex ids.
// (select-based so that no register array is indexed dynamically)
HG_HD void copy_local_ijk(const IfaceCopy& c, int dim, const int wts[3], int& i, int& j, int& k) {
  i = j = k = 0;
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    const int wm = m <= dim ? wts[m] : 0;
    i += c.loc[m] == 1 ? wm : 0;
    j += c.loc[m] == 2 ? wm : 0;
    k += c.loc[m] == 3 ? wm : 0;
  }
}

// Streaming constant-stencil kernel (hg_p1stream.cu).  One CTA per SM copies
// a contiguous stretch of the (cell, band, plane) sequence into a ring of
// kStreamSlots shared-memory slots, kStreamSlotBytes each, by 1-D bulk
// copies, and forms the band's points of every plane from the staged rows of
// planes k-1, k, k+1.  A band is the rows j0 .. j0+rows-1 of a plane; when a
// whole plane fits a slot the band is the whole plane and consecutive planes
// (contiguous in t_w order) share one copy.  The plan, built
// on the host per level and element size, lists per CTA:
//  * copies {cell, ga, nelem, 0}: [ga, ga+nelem) of the cell's stored array
//    (16-byte aligned), copy c of the CTA into slot c mod kStreamSlots;
//  * items, 3 int4 each: {cell, k, ja | jb << 16, arrivals},
//    {c0, cm, cp, 0}, {ga0, gam, gap, 0}: the rows [ja, jb) of plane k, the
//    CTA-local copies holding planes k, k-1, k+1 (-1: none) and their ga;
//    arrivals packs the counts (10 bits each) with which the item arrives on
//    the distinct copies c0, cm, cp after reading them: every slot phase
//    expects kStreamArrive arrivals, the first reader of a copy adds the
//    readers that do not exist.
constexpr int kStreamSlotBytes = 40 * 1024;
constexpr int kStreamSlots = 4;
constexpr int kStreamArrive = 256;
constexpr int kStreamPiece = 512;
struct StreamPlanDev {
  int4* copies;
  int4* items;
  int32_t* cta_copies;  // [nctas + 1]
  int32_t* cta_items;   // [nctas + 1]
  int nctas;
  int band_rows;
};
struct StreamPlanHost {
  std::vector<int4> copies, items;
  std::vector<int32_t> cta_copies, cta_items;
  int nctas = 0, band_rows = 0;
};
// CTAs of the streaming kernel for a level (at most one per SM).
int stream_ctas(int n, int ncells, int n_items, int sms);
// Rows per band at n intervals per edge and element size esize (w = n+1: whole planes).
int stream_band_rows(int n, int esize);
int stream_plan(int n, int ncells, int nctas, int esize, StreamPlanHost& P);

// Device-resident description of one level of one hierarchy (P1 vertex lattice).
struct LevelDev {
  int level, n, w;           // w = n + 1 vertices per macro edge
  int ncells;
  int64_t cell_stride;       // stored elements per cell (padded)
  int64_t n_stored, n_unique, n_inner;
  // device arrays
  uint8_t* cls_flags;        // [ncells*16]
  int32_t* canon;            // [n_stored] stored -> canonical, -1 padding
  int64_t* canon_rep;        // [n_unique] a stored index of each unique DoF
  IfacePrim* prims;          // [n_prims], non-Dirichlet first
  IfaceCopy* copies;
  int n_prims, n_prims_inner, max_copies;
  int32_t* prim_point_base;  // [n_prims+1] prefix sums of prim_points
  // work items of the fused kernels
  int* err;                  // device error word shared by the hierarchy's kernels
  int4* items;               // interface items (first_copy, p0, dim|ncopies<<4|dirichlet<<12, 0),
  int32_t* item_prim;        //   32 consecutive points of one primitive; item -> primitive
  int n_items, n_items_inner;
  // operator-application work items
  int4* citems;              // interface items of the apply: (first_copy, p0, meta as above,
  int n_citems;              //   points); points = floor(32 / ncopies), one lane per copy
  uint2* clane;              // [n_citems * 32]: what each lane of an apply item works on
                             //   (lane = c * P + pt: copy c of point pt, P = 32 / C points),
                             //   x = i | j << 10 | k << 20 | dirichlet << 30 (the copy's
                             //   cell-local point), y = cell | C << 24 | active << 30 (C: the
                             //   primitive's copies; lanes past the item's points: point 0,
                             //   copy 0, not active; C = 63: more than 32 copies, serial path)
  int4* mitems;              // apply items of the primitives with >= 2 copies only
  int n_mitems, n_mitems_inner;  //   (non-Dirichlet first): the streaming kernel's exchange
  int2* mlanes;              // [n_mitems * 32]: per lane (copy-major: lane = copy * (32 / C)
                             //   + point) the copy's stored index and
                             //   cell * 16 + class ({-1, 0}: none; not for > 32 copies)
  StreamPlanDev splan[2];    // the streaming kernel's plans for HG_F32 and HG_F64
  int4* ptiles;              // plane-window tiles of ONE cell (the same for every cell):
  int n_ptiles_cell;         //   (k | windows << 16, lane-0 offset z, j0 << 16 | i0, 0)
  int2* march;               // column-march items of ONE cell: (k | i0 << 16, j0 | j1 << 16),
  int n_march_cell;          //   columns i0..i0+31 of plane k, rows j0..j1-1
  uint8_t* colour;           // Gauss-Seidel colour (0..3) per stored point, or null
};

// Windows of 30 consecutive lattice offsets per plane-window tile of the
// constant-stencil kernels.
#ifndef HG_PLANE_STEPS
#define HG_PLANE_STEPS 16
#endif
constexpr int kPlaneSteps = HG_PLANE_STEPS;
// Rows marched by one column-march item of the constant-stencil kernels.
#ifndef HG_MARCH_ROWS
#define HG_MARCH_ROWS 16
#endif
constexpr int kMarchRows = HG_MARCH_ROWS;

// Dense FP64 coarse-grid solver data.
struct CoarseDev {
  int n;                 // interior unknowns
  double* ainv;          // [n*n] row-major inverse of the coarse matrix
  int64_t* stored_rep;   // [n] stored index of one copy of each unknown
  int32_t* int_of_canon; // [n_unique] interior index of a canonical DoF, -1 if Dirichlet
  double* xint;          // [n] solution workspace
};

// ------------------------------------------------------------ errors
void set_error(const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
#define HG_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return ::hg::cuda_fail(e_, #call); \
  } while (0)

// ------------------------------------------------------------ launchers
// Operation of the cell kernel + interface kernel pair.
// OP_GS: one colour sub-sweep of Gauss-Seidel, out of place (points of other
// colours copied)
// OP_CHEB: one step of the Chebyshev semi-iteration for D^-1 A (Sec. 5.2.1,
// Chebyshev-accelerated Jacobi): d' = cheb_a d + omega D^-1 (b - A x),
// out = x + d', d <- d' in place (cheb_a == 0: d is not read).  Dirichlet
// DoFs: out = x, d untouched.
enum CellOp : int { OP_APPLY = 0, OP_RESID = 1, OP_JACOBI = 2, OP_DIAG = 3, OP_GS = 6, OP_CHEB = 7 };

// Interior-stencil pattern of a constant-coefficient level: the directions
// (indices of dir_offset) that may be nonzero under kPat7.
constexpr int kPat7 = 1;
constexpr unsigned kPat7Mask = (1u << 0) | (1u << 1) | (1u << 2) | (1u << 7) | (1u << 8) |
                               (1u << 11) | (1u << 12);

// True for the operations that scale the residual by the inverse diagonal.
HG_HD constexpr bool op_scaled(int op) { return op == OP_JACOBI || op == OP_GS || op == OP_CHEB; }

struct StencilArgs {
  const void* x;        // input
  const void* b;        // rhs (RESID/JACOBI)
  void* out;            // output
  const void* sten;     // [ncells][16][16] T (class, direction)
  const void* sst;      // or stored stencils [n_stored][16] T: the partial stencil of every
                        // stored point (its cell's micro-cells), 15 weights + 1/centre
  double omega;         // JACOBI: weight; CHEB: beta of the residual term
  int op, mode, mask;
  int colour;           // OP_GS: the colour updated
  int pattern;          // constant stencils: 0, or kPat7 when every cell's interior stencil is
                        // zero outside centre, +-(1,0,0), +-(1,-1,0), +-(0,-1,1)
  void* dvec;           // OP_CHEB: Chebyshev direction d (read if cheb_a != 0, written)
  double cheb_a;        // OP_CHEB: weight of the previous direction
};

int launch_p1_const(const LevelDev& L, int dtype, const StencilArgs& a, cudaStream_t s);
// The streaming form of the constant-stencil operator (a.sten, a.pattern), for
// levels whose slot ring fits in shared memory (p1_stream_fits).
bool p1_stream_fits(int w, int dtype);
// The kernel choice of hg_set_p1_kernel (HG_P1_KERNEL_*).
int set_p1_kernel(int mode);
int launch_p1_stream(const LevelDev& L, int dtype, const StencilArgs& a, cudaStream_t s);

// ------------------------------------------------------------------- P2
// A P2 function on level l (vertex and edge DoFs of the level-l micro-cells)
// is stored on the vertex lattice of level l+1: the micro-vertices are the
// even points of the doubled lattice and every other point is the midpoint
// of exactly one level-l micro-edge.  The level-(l+1) P1 tables (copies,
// interface items, canonical keys, Dirichlet flags) therefore serve P2.
//
// Element data of one macro cell on one P2 level for the element-wise
// kernels: the element matrix of a micro-cell of type t is
//   K = sum_q kq C_q H_t C_q^T,  kq = w_q |T| k(x_q),
// with C_q the P2 gradient coefficients at quadrature point q (functions of
// its barycentric coordinates only) and H_t = G G^T of the type's
// barycentric gradients.  k(x) = a + b sin(2 pi x) sin(2 pi y) sin(2 pi z)
// is evaluated separably: x_q = x_p + d_{t,q} (anchor position x_p), so
// sin(2 pi x_q) = sin(2 pi x_p) cos(2 pi d) + cos(2 pi x_p) sin(2 pi d).
template <typename T>
struct P2Cell {
  T H[6][10];        // G G^T per type: 00 01 02 03 11 12 13 22 23 33
  T kA[14], kB[14];  // w_q |T| a, w_q |T| b
  T sc[6][14][6];    // per type and point: sin, cos of 2 pi d per axis
  T x0[3];           // anchor (i,j,k) sits at x0 + i e[0] + j e[1] + k e[2]
  T e[3][3];
  T vol;             // micro-cell volume (mass element matrix = vol * M_ref)
  T pad;
};
enum { P2_STIFF = 0, P2_MASS = 1, P2_DIAG = 2, P2_N1 = 3, P2_N1DIAG = 4 };
// Lowest-order Nedelec (N1) operator alpha curl curl + beta I of one macro
// cell and level: the DoFs are the micro-edges, stored at the edge-midpoint
// points of the same level+1 lattice as the P2 edge DoFs (the vertex points
// stay zero).  Per micro-cell type the 6x6 element matrix (local edges
// (0,1),(0,2),(0,3),(1,2),(1,3),(2,3)) with the orientation signs of the
// cell folded in; affine cells make it the same for every micro-cell of a
// type.
template <typename T>
struct N1Cell {
  T K[6][36];
};
// Apply of one P2 level: 8 colour phases accumulate the element products
// into acc (zeroed first), a finish pass sums interface copies and forms the
// operation (apply / residual / Jacobi with invdiag / 1 / diagonal).
struct P2Args {
  int n;                     // micro-intervals per macro edge on the P2 level
  int ncells;
  const void* cells;         // P2Cell<T>[ncells]
  const uint32_t* anchors;   // device: packed (i | j << 10 | k << 20) per colour, concatenated
  int anchor_off[9];         // host: colour offsets into anchors
  int mode;                  // P2_STIFF / P2_MASS
  void* acc;                 // work vector of the level (stored layout)
  const void* invdiag;
};
constexpr int OP_INVDIAG = 4;  // finish pass writing 1 / (assembled diagonal)
int p2_upload_constants(const double qbary[14][4], const double qw[14], const double mass[10][10]);
int launch_p2(const LevelDev& L, int dtype, const StencilArgs& a, const P2Args& P, cudaStream_t s);
int launch_p2_diag(const LevelDev& L, int dtype, const P2Args& P, void* invdiag, cudaStream_t s);
// P2 transfers between P2 levels l-1 and l, given the lattices F (level l+1)
// and C (level l) that store them: x_f += P e_c (quadratic interpolation) and
// r_c = P^T r_f.
int launch_prolong_p2(const LevelDev& F, const LevelDev& C, int dtype, const void* ec, void* xf,
                      cudaStream_t s);
int launch_restrict_p2(const LevelDev& F, const LevelDev& C, int dtype, const void* rf, void* rc,
                       cudaStream_t s);


// Variable-coefficient P1 operator data of one level and dtype.
struct VarCoef {
  const void* k;        // coefficient at stored vertices
  const void* K;        // [ncells][24][4] element-matrix rows of the incidences
  const void* invdiag;  // stored 1/diag(A) (non-Dirichlet DoFs)
};
int launch_p1_divkgrad(const LevelDev& L, int dtype, const StencilArgs& a, const VarCoef& vc,
                       cudaStream_t s);
// Polynomial surrogate of the div-k-grad operator: degree, coefficients
// [ncells][15][nterm] (terms ordered by the power of i, then of j, then of
// k, in the shifted coordinates i/n - 1/4, j/n - 1/4, k/n - 1/4) and the
// bands of interior rows of one cell (j0 | k << 10 | j1 << 20: rows
// j0..j1-1 of plane k, at most kSurRows of them).
struct SurCoef {
  int degree;
  const void* coef;
  const int* segs;
  int n_segs_cell;
  int pattern;  // kPat7: every cell's fitted weights vanish outside the seven-point subset
};
constexpr int kSurMaxDegree = 4;
constexpr int kSurRows = 8;
__host__ __device__ constexpr int sur_nterm(int q) { return (q + 1) * (q + 2) * (q + 3) / 6; }
int launch_p1_surrogate(const LevelDev& L, int dtype, const StencilArgs& a, const VarCoef& vc,
                        const SurCoef& sc, cudaStream_t s);
// Projections M[cell][d][t] = sum over the P interior points p of one cell of
// Q[p][t] * S[16 * (cell * stride + pidx[p]) + d] (FP64, t < T; S: the exact
// stored stencils), for the least-squares fit of the surrogate.
int launch_surrogate_moments(const LevelDev& L, const double* S, const int* pidx, int P,
                             const double* Q, int T, double* M, cudaStream_t s);
// Stored stencils of the div-k-grad operator: S[16 q + d] = the weight of
// direction d in the partial stencil of stored point q (zero outside the
// lattice); S[16 q + 15] = 1 / S[16 q] for points inside a cell, else 0.
int launch_divkgrad_stencil(const LevelDev& L, int dtype, const VarCoef& vc, void* S,
                            cudaStream_t s);
int launch_index_enumerate(int w, int64_t* out, cudaStream_t s);
int launch_interface_dump(const LevelDev& L, int64_t* out, cudaStream_t s);
// Stored <-> canonical order; can_dtype: element type of the canonical side
// (-1 = dtype, else HG_F32/HG_F64, converted by rounding to nearest).
int launch_to_canonical(const LevelDev& L, int dtype, const void* st, void* can, cudaStream_t s,
                        int can_dtype = -1);
int launch_from_canonical(const LevelDev& L, int dtype, const void* can, void* st, cudaStream_t s,
                          int can_dtype = -1);
int launch_restrict_p1(const LevelDev& F, const LevelDev& C, int dtype, const void* rf, void* rc,
                       cudaStream_t s);
int launch_prolong_p1(const LevelDev& F, const LevelDev& C, int dtype, const void* ec, void* xf,
                      cudaStream_t s);
// FP64 dot over owned points; partial sums go to `scratch` (>= dot_scratch_len(L) doubles),
// the final value to `result_dev` (device double).
int64_t dot_scratch_len(const LevelDev& L);
int launch_dot(const LevelDev& L, int dtype, const void* x, const void* y, int mask,
               double* scratch, double* result_dev, cudaStream_t s);
int launch_coarse_solve(const LevelDev& L, const CoarseDev& C, int dtype, const void* b, void* x,
                        cudaStream_t s);
int launch_demote_scaled(int64_t n, const double* r, double scale, float* out, cudaStream_t s);
// Learned smoother network (params: W1 32x16 | W2 32x32 | w3 32, FP32 master).
constexpr int kMlpParams = 512 + 1024 + 32;
int launch_mlp_forward(const float* X, int64_t N, const float* W1, const float* W2,
                       const float* w3, float* out, cudaStream_t s);
int mlp_grad_blocks(int64_t count);
int launch_mlp_grad(const void* Xs, const float* ts, int64_t N, int64_t first, int64_t count,
                    const float* W1, const float* W2, const float* w3, float* partial,
                    double* lpart, float* grad, double* loss, cudaStream_t s);
int launch_mlp_adam(float* p, const float* grad, float* m, float* v, float lr, int step,
                    cudaStream_t s);
int launch_learned_step(const LevelDev& L, const float* x, const float* r, const float* inv,
                        float omega, const float* params, float* xo, cudaStream_t s);
int64_t learned_sample_count(const LevelDev& L, int sstride, int soff);
int launch_learned_sample(const LevelDev& L, const float* r, const float* inv, const float* xstar,
                          const float* x, float omega, int sstride, int soff, void* X, float* t,
                          cudaStream_t s);
int launch_promote_axpy(int64_t n, double alpha, const float* d, double* x, cudaStream_t s);

// ------------------------------------------------------------ batched stages
// Many independent problems in one persistent launch: each problem
// contributes `units` blocks; base[p] = sum of the units of problems < p.
enum BatchEw : int { EW_ZERO = 0, EW_COPY = 1, EW_DEMOTE = 2, EW_PROMOTE = 3 };
struct EwDesc {         // element-wise stage on one problem's stored vector
  int64_t n;
  void* a;              // ZERO a=0 | COPY a=b | DEMOTE a(f32)=b(f64)/|r| | PROMOTE a(f64)+=|r| b(f32)
  const void* b;
  const double* rr;     // |r|^2 of the problem (DEMOTE/PROMOTE)
  int dtype;            // ZERO/COPY element type
};
struct DotDesc {        // FP64 dot over owned non-Dirichlet DoFs of one problem
  int n;
  int64_t stride;
  const uint8_t* flags;
  int n_rows;
  const void* x;
  const void* y;
};
struct CoarseBDesc {    // dense coarse solve of one problem
  int nint;
  const double* ainv;
  const int64_t* rep;
  const void* b;
  double* xint;
  int64_t n_stored;
  const int32_t* canon;
  const int32_t* ioc;
  void* x;
};
constexpr int kDotRowsPerUnit = 128;  // lattice rows per unit of the batched dot
int64_t dot_units(int n_rows);
int64_t ew_units(int64_t n);
int launch_batched_ew(int op, const EwDesc* d, const int* base, int nprob, int grid, cudaStream_t s);
int launch_batched_dot(int dtype, const DotDesc* d, const int* base, int nprob, int grid,
                       double* partial, double* rr, cudaStream_t s);
int launch_batched_coarse(int dtype, const CoarseBDesc* d, const int* base_mv, const int* base_sc,
                          int nprob, int grid, cudaStream_t s);
int64_t coarse_units_mv(int nint);
int64_t coarse_units_sc(int64_t n_stored);
// descriptors of the cell/transfer stages (built on the host, raw bytes)
size_t p1_desc_bytes(int dtype);
int p1_make_desc(const LevelDev& L, int dtype, const StencilArgs& a, void* dst, int* units);
size_t restrict_desc_bytes(int dtype);
int restrict_make_desc(const LevelDev& F, const LevelDev& C, int dtype, const void* rf, void* rc,
                       void* dst, int* units);
size_t prolong_desc_bytes(int dtype);
int prolong_make_desc(const LevelDev& F, const LevelDev& C, int dtype, const void* ec, void* xf,
                      void* dst, int* units);
int launch_p1_batched(int dtype, int op, int rows, const void* descs, const int* base, int nprob,
                      int grid, cudaStream_t s);
int launch_restrict_batched(int dtype, const void* descs, const int* base, int nprob, int grid,
                            cudaStream_t s);
int launch_prolong_batched(int dtype, const void* descs, const int* base, int nprob, int grid,
                           cudaStream_t s);

}  // namespace hg
