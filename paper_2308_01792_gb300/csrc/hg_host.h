// Host-side data structures: macro mesh with its primitive graph, the level
// hierarchy and operators.  Internal to the library.
#pragma once

#include <array>
#include <vector>

#include "hg_internal.h"

namespace hg {

extern const int kTypeOff[6][4][3];
extern const int kTypeDelta[6];
extern const int kEdgeVerts[6][2];

// A macro primitive (vertex, edge or face) with the macro cells containing it
// (ascending id).  vid: its macro vertex ids, ascending (unused = -1).
struct Prim {
  std::array<int64_t, 3> vid;
  std::vector<int> cells;
  bool dirichlet = false;
};

// Macro mesh and its primitive graph (Sec. 2: one data structure per coarse
// vertex/edge/face/cell with links to the neighbours).
struct Mesh {
  int64_t nv = 0, nc = 0;
  std::vector<double> xyz;
  std::vector<std::array<int64_t, 4>> cells;
  std::vector<Prim> faces, edges, verts;
  std::vector<std::array<int, 4>> cell_face;  // face opposite local vertex f
  std::vector<std::array<int, 6>> cell_edge;  // local edge e = kEdgeVerts[e]
  int64_t n_boundary_faces = 0;
  int grid_denom = 0;                         // D with integer xyz*D, 0 if none
  std::vector<int64_t> ixyz;
  // 4-colouring of every level's lattice: colour = (a X + b Y + c Z) mod 4 of
  // the exact lattice point, with (a, b, c) such that no micro-edge joins two
  // points of one colour; gs_abc[0] < 0 if no such triple exists
  int gs_abc[3] = {-1, 0, 0};
  void find_colouring();

  int build(const double* xyz, int64_t nv, const int64_t* cells, int64_t nc);
  void cell_jacobian(int64_t c, double J[9]) const;
  const Prim* class_prim(int64_t c, int cls) const;
  uint8_t class_flags(int64_t c, int cls) const;
};

struct LevelHost {
  LevelDev dev{};
  std::vector<uint8_t> cls_flags;
  std::vector<IfacePrim> prims;
  std::vector<IfaceCopy> copies;
  std::vector<int32_t> prim_point_base;
  std::vector<int32_t> canon;
  std::vector<int64_t> canon_rep;
  std::vector<uint8_t> dirichlet;
  std::vector<double> canon_xyz;
  std::vector<int64_t> canon_keys;  // packed (z,y,x) lattice keys, ascending
  std::vector<uint8_t> colour;      // 4-colouring per stored point (empty if none)
};

struct Hier {
  const Mesh* mesh = nullptr;
  int lmin = 0, lmax = 0;
  std::vector<LevelHost> lv;
  double* dot_scratch = nullptr;
  double* dot_result = nullptr;
  double* dot_host = nullptr;
  int* err_dev = nullptr;   // device error word of all kernels of this hierarchy
  int* err_host = nullptr;  // pinned mirror

  int build(const Mesh* m, int lmin, int lmax);
  int check_limits() const;
  int build_level(int l);
  // Enqueue a read of the error word on s (no sync); check_error() after a sync.
  int fetch_error(cudaStream_t s) const;
  int check_error() const;
  ~Hier();
};

// Index into Hier::lv of the lattice that stores `space` on `level` (P2 on
// level l uses the lattice of level l+1), or -1 if the hierarchy lacks it.
int lattice_index(const Hier* h, int space, int level);
// Plane-window tiles of one cell lattice with n intervals (the same for every cell).
std::vector<int4> plane_tiles(int n);
// Column-march items of one cell lattice with n intervals (the same for every cell).
std::vector<int2> march_items(int n);
// Anchors of the P2/N1 colour phases (n intervals), off[9] colour offsets.
std::vector<uint32_t> p2_anchors(int n, int off[9]);

struct Op {
  const Hier* hier = nullptr;
  int kind = 0;
  int space = HG_SPACE_P1;
  int lmin = 0, lmax = 0;       // levels of the operator's space
  // P2 (per P2 level): element data per cell (P2Cell<T>), anchors by colour,
  // accumulation vector and inverse assembled diagonal per dtype
  std::vector<void*> p2cells[2], p2acc[2], p2inv[2];
  std::vector<uint32_t*> p2anchors;
  std::vector<std::vector<int>> p2off;
  int p2mode = 0;
  const LevelHost& host(int l) const { return hier->lv[lattice_index(hier, space, l)]; }
  const LevelDev& dev(int l) const { return host(l).dev; }
  int build_p2(const double* coeff);
  int build_n1(const double* coeff);
  int8_t* n1sign = nullptr;      // N1: orientation sign per (cell, lattice direction), [nc][8]
  double n1alpha = 0.0, n1beta = 0.0;  // N1: alpha curl curl + beta I
  std::vector<double*> sten64;  // per level [ncells][16][16] (constant-coefficient kinds)
  std::vector<float*> sten32;
  std::vector<int> pattern;     // per level: kPat7 when the interior stencils allow it
  // variable-coefficient P1 (per level): k at stored vertices, element rows, 1/diag
  std::vector<void*> vk[2], vK[2], vinv[2];
  // stored-stencil P1 (per level): per stored point 16 values, point-major [n_stored][16]:
  // the 15 partial-stencil weights and the inverse centre weight
  std::vector<void*> sst[2];
  // surrogate P1 (per level): polynomial coefficients [ncells][15][nterm] per
  // dtype and the interior row segments of one cell (j | k << 10 | i0 << 20)
  int sdeg = -1;
  std::vector<void*> scoef[2];
  std::vector<int*> ssegs;
  std::vector<int> n_ssegs;
  std::vector<int> spat;        // per level: kPat7 when the fit vanishes outside it
  int build_surrogate(const double* coeff, int degree);

  int build(const Hier* h, int kind, const double* coeff);
  int build_divkgrad(const double* coeff);
  int build_stored();
  // One cell operation (apply / residual / Jacobi / diagonal) of this operator.
  int launch(int level, int dtype, StencilArgs a, cudaStream_t s) const;
  ~Op();
};

// Lowest-order Nedelec prolongation by fine-point class r = q mod 4 (q in
// the fine F lattice): up to 6 terms, coarse DoF at C-lattice offset `off`
// (x | y << 2 | z << 4) from 2 floor(q / 4), its lattice direction `dir`
// (index into kN1Dir) and the weight with the local orientation folded in;
// fine_dir: the direction of the fine edge at q (-1 for vertex points).
// The restriction r_C = P^T r_F by coarse parity class pc (1..7; the coarse
// DoF's direction is pc - 1): entries res_start[pc] .. res_start[pc+1]-1
// with the fine point at F-lattice offset res_d (dx+8 | dy+8 << 5 | dz+8 <<
// 10) from 2c, the weight and the fine point's direction.
constexpr int kN1MaxRes = 512;
struct N1ProlongTable {
  int n[64];
  int off[64][6];
  int dir[64][6];
  double w[64][6];
  int fine_dir[64];
  int res_start[9];
  int res_d[kN1MaxRes];
  double res_w[kN1MaxRes];
  int res_fdir[kN1MaxRes];
};
// The 7 lattice edge directions, index = parity class (x | y << 1 | z << 2)
// of the edge midpoints minus 1.
extern const int kN1Dir[7][3];
int n1_prolong_table(const N1ProlongTable** out);
// N1 transfers between lattices F (fine, level l+1) and C (level l) with the
// per-cell orientation signs (int8 [ncells][8]): N1_PROLONG xf += P ec,
// N1_RESTRICT rc = P^T rf (fine N1 level l, coarse l-1); N1_GRAD u = G phi
// (P1 level l on C to N1 level l on F), N1_GRADT rp = G^T r, N1_GRAD_ADD
// u += scale G phi.
enum { N1_PROLONG = 0, N1_RESTRICT = 1, N1_GRAD = 2, N1_GRADT = 3, N1_GRAD_ADD = 4 };
int launch_n1_transfer(int which, const LevelDev& F, const LevelDev& C, int dtype,
                       const int8_t* sign, const void* src, void* dst, cudaStream_t s,
                       double scale = 1.0);

// A function on a level range (Sec. 5.1): one stored vector per level of one
// space and element type, in caller-owned device memory bound level by level,
// plus the library's device staging buffers for copies from and to host
// memory in canonical order.
struct Func {
  const Hier* hier = nullptr;
  int space = HG_SPACE_P1;
  int dtype = HG_F64;
  std::vector<void*> ptr;        // per lattice index of the hierarchy (null = unbound)
  std::vector<void*> stage;      // per lattice index, n_unique * 8 bytes once used
  // The bound stored vector of `level`; sets the error message and returns
  // null if the level is outside the hierarchy or unbound.
  void* data(int level) const;
  ~Func();
};

// Parameters and optimiser state of the learned smoother network (device).
struct Mlp {
  float* params = nullptr;   // kMlpParams
  float* grad = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  float* partial = nullptr;  // [blocks][kMlpParams] gradient partials
  double* lpart = nullptr;
  double* loss = nullptr;
  double* loss_host = nullptr;
  int partial_blocks = 0;
  int step = 0;
  int build();
  ~Mlp();
};

void micro_cell_coords(const Mesh& m, int64_t c, int n, int type, double X[4][3]);
// Symmetric 14-point degree-5 rule on the tetrahedron (barycentric points,
// weights summing to 1), derived once from its moment equations.
int sym14_rule(double bary[14][4], double w[14]);
void bary_gradients(const double X[4][3], double G[4][3], double* vol);
void p1_cell_stencils(const Mesh& m, int64_t c, int n, int kind, double S[16][16]);

}  // namespace hg
