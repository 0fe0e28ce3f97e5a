// Element-wise P2 operators (Sec. 5.2, element-wise pattern with element
// matrices formed on the fly for variable coefficients; Sec. 5.1 P2 as vertex
// plus edge DoFs).
//
// A P2 function of level l lives on the vertex lattice of level l+1 (see
// hg_internal.h).  The micro-cells of level l are the six types anchored at
// the level-l points p (Sec. 3.2): all six lie in the unit cube [p, p+1]^3,
// whose doubled-lattice points (2p + {0,1,2}^3) hold their 10 DoFs each.
// Anchors of equal parity (i, j, k mod 2) have disjoint closed cubes, so the
// apply is 8 colour phases; in a phase one thread takes one anchor, loads the
// 27 cube points once, sums the products of its micro-cells' element
// matrices in registers and adds them into the accumulation vector with one
// plain read-modify-write per point (no two threads touch a DoF; the order of
// contributions to every DoF is fixed: colour, then type).
//
// Element matrices are never stored: for type t and quadrature point q the
// gradients of the 10 basis functions are C_q (barycentric gradients), with
//   vertex i:  (4 l_i - 1) grad l_i,   edge ij:  4 (l_i grad l_j + l_j grad l_i),
// so K x = sum_q kq C_q (H_t (C_q^T x)) costs ~50 FMA per point and needs
// only H_t = G G^T (10 numbers per type and cell) and the coefficient
// factor kq = w_q |T| k(x_q).
//
// The finish pass (one launch) sums the per-cell partials of interface DoFs
// over their copies in ascending cell order (the ghost-layer exchange,
// Sec. 2), writes the sum to every copy, and forms the requested operation.
#include <cuda_runtime.h>

#include "hg_internal.h"

namespace hg {

namespace {

constexpr int kP2Block = 128;
constexpr int kFinBlock = 256;
constexpr int kFinWarps = kFinBlock / 32;

__constant__ double c_qb64[14][4];
__constant__ float c_qb32[14][4];
__constant__ double c_mass64[10][10];
__constant__ float c_mass32[10][10];

template <typename T>
__device__ __forceinline__ T qbary(int q, int m);
template <>
__device__ __forceinline__ double qbary<double>(int q, int m) { return c_qb64[q][m]; }
template <>
__device__ __forceinline__ float qbary<float>(int q, int m) { return c_qb32[q][m]; }
template <typename T>
__device__ __forceinline__ T mass_ref(int a, int b);
template <>
__device__ __forceinline__ double mass_ref<double>(int a, int b) { return c_mass64[a][b]; }
template <>
__device__ __forceinline__ float mass_ref<float>(int a, int b) { return c_mass32[a][b]; }

__device__ __forceinline__ void sincos_2pi(float x, float* s, float* c) { sincospif(2.0f * x, s, c); }
__device__ __forceinline__ void sincos_2pi(double x, double* s, double* c) { sincospi(2.0 * x, s, c); }

// Vertex offsets (level-l units) of the six micro-cell types and the largest
// anchor sum they admit (n-1-delta): I-up, I-down, four octahedral cells
// around the inner edge p+e2 -- p+e1+e3.
__device__ constexpr int kToff[6][4][3] = {
    {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}},
    {{1, 1, 0}, {1, 0, 1}, {0, 1, 1}, {1, 1, 1}},
    {{0, 1, 0}, {1, 0, 1}, {1, 0, 0}, {0, 0, 1}},
    {{0, 1, 0}, {1, 0, 1}, {0, 0, 1}, {0, 1, 1}},
    {{0, 1, 0}, {1, 0, 1}, {0, 1, 1}, {1, 1, 0}},
    {{0, 1, 0}, {1, 0, 1}, {1, 1, 0}, {1, 0, 0}}};
__device__ constexpr int kDelta[6] = {0, 2, 1, 1, 1, 1};
__device__ constexpr int kEdge[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

// Element product y = K_t x (stiffness with the coefficient factors of the
// cell), y = vol M x (mass) or the diagonal of K_t (diag).
template <typename T, int MODE>
__device__ __forceinline__ void p2_element(const P2Cell<T>& C, int t, const T sxyz[6],
                                           const T xv[10], T yv[10]) {
#pragma unroll
  for (int a = 0; a < 10; ++a) yv[a] = T(0);
  if (MODE == P2_MASS) {
#pragma unroll
    for (int a = 0; a < 10; ++a) {
      T acc = T(0);
#pragma unroll
      for (int b = 0; b < 10; ++b) acc += mass_ref<T>(a, b) * xv[b];
      yv[a] = C.vol * acc;
    }
    return;
  }
  const T* H = C.H[t];
  const T h00 = H[0], h01 = H[1], h02 = H[2], h03 = H[3], h11 = H[4], h12 = H[5], h13 = H[6],
          h22 = H[7], h23 = H[8], h33 = H[9];
#pragma unroll 2
  for (int q = 0; q < 14; ++q) {
    const T l0 = qbary<T>(q, 0), l1 = qbary<T>(q, 1), l2 = qbary<T>(q, 2), l3 = qbary<T>(q, 3);
    const T* sc = C.sc[t][q];
    const T sx = sxyz[0] * sc[1] + sxyz[1] * sc[0];
    const T sy = sxyz[2] * sc[3] + sxyz[3] * sc[2];
    const T sz = sxyz[4] * sc[5] + sxyz[5] * sc[4];
    const T kq = C.kA[q] + C.kB[q] * (sx * sy * sz);
    const T f0 = T(4) * l0 - T(1), f1 = T(4) * l1 - T(1), f2 = T(4) * l2 - T(1), f3 = T(4) * l3 - T(1);
    const T g0 = T(4) * l0, g1 = T(4) * l1, g2 = T(4) * l2, g3 = T(4) * l3;
    if (MODE == P2_DIAG) {
      yv[0] += kq * f0 * f0 * h00;
      yv[1] += kq * f1 * f1 * h11;
      yv[2] += kq * f2 * f2 * h22;
      yv[3] += kq * f3 * f3 * h33;
      yv[4] += kq * (g0 * g0 * h11 + T(2) * g0 * g1 * h01 + g1 * g1 * h00);
      yv[5] += kq * (g0 * g0 * h22 + T(2) * g0 * g2 * h02 + g2 * g2 * h00);
      yv[6] += kq * (g0 * g0 * h33 + T(2) * g0 * g3 * h03 + g3 * g3 * h00);
      yv[7] += kq * (g1 * g1 * h22 + T(2) * g1 * g2 * h12 + g2 * g2 * h11);
      yv[8] += kq * (g1 * g1 * h33 + T(2) * g1 * g3 * h13 + g3 * g3 * h11);
      yv[9] += kq * (g2 * g2 * h33 + T(2) * g2 * g3 * h23 + g3 * g3 * h22);
      continue;
    }
    // u = C_q^T x
    const T u0 = f0 * xv[0] + g1 * xv[4] + g2 * xv[5] + g3 * xv[6];
    const T u1 = f1 * xv[1] + g0 * xv[4] + g2 * xv[7] + g3 * xv[8];
    const T u2 = f2 * xv[2] + g0 * xv[5] + g1 * xv[7] + g3 * xv[9];
    const T u3 = f3 * xv[3] + g0 * xv[6] + g1 * xv[8] + g2 * xv[9];
    // v = kq H u
    const T v0 = kq * (h00 * u0 + h01 * u1 + h02 * u2 + h03 * u3);
    const T v1 = kq * (h01 * u0 + h11 * u1 + h12 * u2 + h13 * u3);
    const T v2 = kq * (h02 * u0 + h12 * u1 + h22 * u2 + h23 * u3);
    const T v3 = kq * (h03 * u0 + h13 * u1 + h23 * u2 + h33 * u3);
    // y += C_q v
    yv[0] += f0 * v0;
    yv[1] += f1 * v1;
    yv[2] += f2 * v2;
    yv[3] += f3 * v3;
    yv[4] += g0 * v1 + g1 * v0;
    yv[5] += g0 * v2 + g2 * v0;
    yv[6] += g0 * v3 + g3 * v0;
    yv[7] += g1 * v2 + g2 * v1;
    yv[8] += g1 * v3 + g3 * v1;
    yv[9] += g2 * v3 + g3 * v2;
  }
}

// One colour phase: thread = anchor of colour `col` in cell blockIdx.y.
// Resident blocks per SM the register budget is sized for (FP32 / FP64;
// FP32 measured best at 5 against 4 and 6 on the 48-cell cube at P2 level 6).
template <typename T>
struct P2MinBlocks {
  static constexpr int value = sizeof(T) == 4 ? 5 : 1;
};

template <typename T, int MODE>
__global__ void __launch_bounds__(kP2Block, P2MinBlocks<T>::value) p2_phase_kernel(const P2Cell<T>* __restrict__ cells,
                                                            const uint32_t* __restrict__ anchors,
                                                            int n_anchors, int n, int64_t stride,
                                                            const T* __restrict__ x,
                                                            T* __restrict__ acc) {
  __shared__ P2Cell<T> C;
  const int cell = blockIdx.y;
  {
    const int* src = reinterpret_cast<const int*>(cells + cell);
    int* dst = reinterpret_cast<int*>(&C);
    for (int q = threadIdx.x; q < (int)(sizeof(P2Cell<T>) / 4); q += blockDim.x) dst[q] = src[q];
  }
  __syncthreads();
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n_anchors) return;
  const uint32_t pk = __ldg(anchors + a);
  const int i = pk & 1023, j = (pk >> 10) & 1023, k = pk >> 20;
  const int s = i + j + k;
  const int w2 = 2 * n + 1;
  const int64_t base = (int64_t)cell * stride;
  const T* __restrict__ xc = x + base;
  T* __restrict__ yc = acc + base;
  // row starts of the cube's doubled-lattice rows (J = 2j+b, K = 2k+c)
  int rs[3][3];
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int c = 0; c < 3; ++c) rs[b][c] = row_start(w2, 2 * j + b, 2 * k + c);
  T sxyz[6];
  if (MODE != P2_MASS) {
    const T px = C.x0[0] + T(i) * C.e[0][0] + T(j) * C.e[1][0] + T(k) * C.e[2][0];
    const T py = C.x0[1] + T(i) * C.e[0][1] + T(j) * C.e[1][1] + T(k) * C.e[2][1];
    const T pz = C.x0[2] + T(i) * C.e[0][2] + T(j) * C.e[1][2] + T(k) * C.e[2][2];
    sincos_2pi(px, &sxyz[0], &sxyz[1]);
    sincos_2pi(py, &sxyz[2], &sxyz[3]);
    sincos_2pi(pz, &sxyz[4], &sxyz[5]);
  }
  // the 27 doubled-lattice points 2p + (dx, dy, dz) of the anchor's cube are
  // loaded once (those inside the macro cell), the six micro-cells accumulate
  // into registers, every point is written back once
  T X[27], Y[27];
#pragma unroll
  for (int c = 0; c < 27; ++c) {
    const int dx = c % 3, dy = (c / 3) % 3, dz = c / 9;
    const bool in = 2 * s + dx + dy + dz <= 2 * n;
    X[c] = (MODE == P2_DIAG || !in) ? T(0) : xc[rs[dy][dz] + 2 * i + dx];
    Y[c] = T(0);
  }
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    if (s > n - 1 - kDelta[t]) continue;
    int cid[10];
#pragma unroll
    for (int v = 0; v < 4; ++v)
      cid[v] = 2 * kToff[t][v][0] + 6 * kToff[t][v][1] + 18 * kToff[t][v][2];
#pragma unroll
    for (int e = 0; e < 6; ++e) {
      const int va = kEdge[e][0], vb = kEdge[e][1];
      cid[4 + e] = (kToff[t][va][0] + kToff[t][vb][0]) + 3 * (kToff[t][va][1] + kToff[t][vb][1]) +
                   9 * (kToff[t][va][2] + kToff[t][vb][2]);
    }
    T xv[10], yv[10];
#pragma unroll
    for (int v = 0; v < 10; ++v) xv[v] = X[cid[v]];
    p2_element<T, MODE>(C, t, sxyz, xv, yv);
#pragma unroll
    for (int v = 0; v < 10; ++v) Y[cid[v]] += yv[v];
  }
#pragma unroll
  for (int c = 0; c < 27; ++c) {
    const int dx = c % 3, dy = (c / 3) % 3, dz = c / 9;
    if (2 * s + dx + dy + dz <= 2 * n) {
      const int q = rs[dy][dz] + 2 * i + dx;
      yc[q] += Y[c];
    }
  }
}

// N1 colour phase (lowest-order Nedelec, alpha curl curl + beta I): the same
// anchors and cubes as the P2 phases; the DoFs are the cube points with an
// odd doubled coordinate (edge midpoints), and every micro-cell applies its
// type's 6x6 matrix from the cell's table (DIAG: adds the diagonal only).
// Points of the cube that are no micro-edge of its cells receive 0.
template <typename T, bool DIAG>
__global__ void __launch_bounds__(kP2Block) n1_phase_kernel(const N1Cell<T>* __restrict__ cells,
                                                            const uint32_t* __restrict__ anchors,
                                                            int n_anchors, int n, int64_t stride,
                                                            const T* __restrict__ x,
                                                            T* __restrict__ acc) {
  __shared__ N1Cell<T> C;
  const int cell = blockIdx.y;
  {
    const int* src = reinterpret_cast<const int*>(cells + cell);
    int* dst = reinterpret_cast<int*>(&C);
    for (int q = threadIdx.x; q < (int)(sizeof(N1Cell<T>) / 4); q += blockDim.x) dst[q] = src[q];
  }
  __syncthreads();
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n_anchors) return;
  const uint32_t pk = __ldg(anchors + a);
  const int i = pk & 1023, j = (pk >> 10) & 1023, k = pk >> 20;
  const int s = i + j + k;
  const int w2 = 2 * n + 1;
  const int64_t base = (int64_t)cell * stride;
  const T* __restrict__ xc = x + base;
  T* __restrict__ yc = acc + base;
  int rs[3][3];
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int c = 0; c < 3; ++c) rs[b][c] = row_start(w2, 2 * j + b, 2 * k + c);
  T X[27], Y[27];
#pragma unroll
  for (int c = 0; c < 27; ++c) {
    const int dx = c % 3, dy = (c / 3) % 3, dz = c / 9;
    const bool dof = ((dx | dy | dz) & 1) && 2 * s + dx + dy + dz <= 2 * n;
    X[c] = (DIAG || !dof) ? T(0) : xc[rs[dy][dz] + 2 * i + dx];
    Y[c] = T(0);
  }
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    if (s > n - 1 - kDelta[t]) continue;
    int eid[6];
#pragma unroll
    for (int e = 0; e < 6; ++e) {
      const int va = kEdge[e][0], vb = kEdge[e][1];
      eid[e] = (kToff[t][va][0] + kToff[t][vb][0]) + 3 * (kToff[t][va][1] + kToff[t][vb][1]) +
               9 * (kToff[t][va][2] + kToff[t][vb][2]);
    }
    const T* K = C.K[t];
    if (DIAG) {
#pragma unroll
      for (int e = 0; e < 6; ++e) Y[eid[e]] += K[7 * e];
    } else {
      T xv[6];
#pragma unroll
      for (int e = 0; e < 6; ++e) xv[e] = X[eid[e]];
#pragma unroll
      for (int e = 0; e < 6; ++e) {
        T v = T(0);
#pragma unroll
        for (int f = 0; f < 6; ++f) v += K[6 * e + f] * xv[f];
        Y[eid[e]] += v;
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 27; ++c) {
    const int dx = c % 3, dy = (c / 3) % 3, dz = c / 9;
    if (((dx | dy | dz) & 1) && 2 * s + dx + dy + dz <= 2 * n) yc[rs[dy][dz] + 2 * i + dx] += Y[c];
  }
}

// Finish pass of one apply on the lattice L of the P2 level.
template <typename T>
struct P2Fin {
  int n, w;
  int64_t stride;
  const uint8_t* flags;
  const int4* items;
  int n_items, nb_items;
  const IfaceCopy* copies;
  int n_rows;
  const T* acc;
  const T* x;
  const T* b;
  T* y;
  const T* invdiag;
  T omega;
  int mode, mask;
  T* dvec;   // OP_CHEB: direction, updated in place
  T cheb_a;  // OP_CHEB: weight of the previous direction
};

// Result at stored position g from the summed product v; `own`: this thread
// is the one that writes position g (OP_CHEB also updates d there).
template <typename T, int OP>
__device__ __forceinline__ T p2_result(const P2Fin<T>& F, int64_t g, T v, bool own = true) {
  if (OP == OP_APPLY) return F.mode == HG_ADD ? F.y[g] + v : v;
  if (OP == OP_RESID) return F.b[g] - v;
  if (OP == OP_JACOBI) return F.x[g] + F.omega * F.invdiag[g] * (F.b[g] - v);
  if (OP == OP_CHEB) {
    T dn = F.omega * F.invdiag[g] * (F.b[g] - v);
    if (own) {
      if (F.cheb_a != T(0)) dn += F.cheb_a * F.dvec[g];
      F.dvec[g] = dn;
    }
    return F.x[g] + dn;
  }
  return v != T(0) ? T(1) / v : T(0);  // OP_INVDIAG
}

template <typename T, int OP>
__global__ void __launch_bounds__(kFinBlock) p2_finish_kernel(P2Fin<T> F) {
  const int lane = threadIdx.x & 31;
  const int wg = blockIdx.x * kFinWarps + (threadIdx.x >> 5);
  const int n = F.n, w = F.w;
  if ((int)blockIdx.x < F.nb_items) {
    if (wg >= F.n_items) return;
    // interface item: lane = pt * C + c takes copy c of point pt
    const int4 it = F.items[wg];
    const int dim = it.z & 15, C = (it.z >> 4) & 255, dirichlet = (it.z >> 12) & 1;
    if (C > 32) {
      // one lane per point, copies in turn
      if (lane >= it.w) return;
      int wts[3];
      prim_point_weights(dim, n, it.y + lane, wts);
      T sum = T(0);
      for (int q = 0; q < C; ++q) {
        int i, j, k;
        copy_local_ijk(F.copies[it.x + q], dim, wts, i, j, k);
        sum += F.acc[(int64_t)F.copies[it.x + q].cell * F.stride + tw32(w, i, j, k)];
      }
      for (int q = 0; q < C; ++q) {
        int i, j, k;
        copy_local_ijk(F.copies[it.x + q], dim, wts, i, j, k);
        const int64_t g = (int64_t)F.copies[it.x + q].cell * F.stride + tw32(w, i, j, k);
        T v;
        if (dirichlet && (OP != OP_APPLY || F.mask == HG_MASK_INNER))
          v = op_scaled(OP) ? F.x[g] : T(0);
        else
          v = p2_result<T, OP>(F, g, sum);
        F.y[g] = v;
      }
      return;
    }
    const int pt = lane / C, c = lane - pt * C;
    const bool act = pt < it.w;
    int wts[3];
    prim_point_weights(dim, n, it.y + (act ? pt : 0), wts);
    const IfaceCopy cpy = F.copies[it.x + (act ? c : 0)];
    int i, j, k;
    copy_local_ijk(cpy, dim, wts, i, j, k);
    const int64_t g = (int64_t)cpy.cell * F.stride + tw32(w, i, j, k);
    const T part = F.acc[g];
    T sum = T(0);
    const int g0 = pt * C;
    for (int q = 0; q < C; ++q) sum += __shfl_sync(0xffffffffu, part, (g0 + q) & 31);
    T v;
    if (dirichlet && (OP != OP_APPLY || F.mask == HG_MASK_INNER))
      v = op_scaled(OP) ? F.x[g] : T(0);
    else
      v = p2_result<T, OP>(F, g, sum, act);
    if (act) F.y[g] = v;
    return;
  }
  // interior points (class 0) of every cell, one warp per lattice row
  const int r = wg - F.nb_items * kFinWarps;
  if (r >= F.n_rows) return;
  int cell, j, k;
  row_item(w, r, cell, j, k);
  if (j == 0 || k == 0) return;
  const int64_t r0 = (int64_t)cell * F.stride + row_start(w, j, k);
  for (int i = 1 + lane; i + j + k < n; i += 32) {
    const int64_t g = r0 + i;
    F.y[g] = p2_result<T, OP>(F, g, F.acc[g]);
  }
}

template <typename T, int MODE>
int run_phases(const P2Args& P, int64_t stride, const void* x, void* acc, int64_t n_stored,
               cudaStream_t s) {
  HG_CUDA(cudaMemsetAsync(acc, 0, n_stored * sizeof(T), s));
  const int* off = P.anchor_off;
  for (int col = 0; col < 8; ++col) {
    const int na = off[col + 1] - off[col];
    if (na == 0) continue;
    const dim3 grid((na + kP2Block - 1) / kP2Block, P.ncells);
    p2_phase_kernel<T, MODE><<<grid, kP2Block, 0, s>>>(
        (const P2Cell<T>*)P.cells, P.anchors + off[col], na, P.n, stride, (const T*)x, (T*)acc);
    HG_CUDA(cudaGetLastError());
  }
  return HG_OK;
}

template <typename T>
P2Fin<T> fin_args(const LevelDev& L, const StencilArgs& a, const P2Args& P, int n_items) {
  P2Fin<T> F;
  F.n = L.n;
  F.w = L.w;
  F.stride = L.cell_stride;
  F.flags = L.cls_flags;
  F.items = L.citems;
  F.n_items = n_items;
  F.nb_items = (n_items + kFinWarps - 1) / kFinWarps;
  F.copies = L.copies;
  F.n_rows = L.ncells * ntri32(L.w);
  F.acc = (const T*)P.acc;
  F.x = (const T*)a.x;
  F.b = (const T*)a.b;
  F.y = (T*)a.out;
  F.invdiag = (const T*)P.invdiag;
  F.omega = (T)a.omega;
  F.mode = a.mode;
  F.mask = a.mask;
  F.dvec = (T*)a.dvec;
  F.cheb_a = (T)a.cheb_a;
  return F;
}

template <typename T, bool DIAG>
int run_phases_n1(const P2Args& P, int64_t stride, const void* x, void* acc, int64_t n_stored,
                  cudaStream_t s) {
  HG_CUDA(cudaMemsetAsync(acc, 0, n_stored * sizeof(T), s));
  const int* off = P.anchor_off;
  for (int col = 0; col < 8; ++col) {
    const int na = off[col + 1] - off[col];
    if (na == 0) continue;
    const dim3 grid((na + kP2Block - 1) / kP2Block, P.ncells);
    n1_phase_kernel<T, DIAG><<<grid, kP2Block, 0, s>>>(
        (const N1Cell<T>*)P.cells, P.anchors + off[col], na, P.n, stride, (const T*)x, (T*)acc);
    HG_CUDA(cudaGetLastError());
  }
  return HG_OK;
}

template <typename T, int OP>
int run_finish(const LevelDev& L, const StencilArgs& a, const P2Args& P, cudaStream_t s) {
  const int n_items = L.n_citems;
  const P2Fin<T> F = fin_args<T>(L, a, P, n_items);
  const int grid = F.nb_items + (F.n_rows + kFinWarps - 1) / kFinWarps;
  p2_finish_kernel<T, OP><<<grid, kFinBlock, 0, s>>>(F);
  HG_CUDA(cudaGetLastError());
  return HG_OK;
}

template <typename T>
int run_p2(const LevelDev& L, const StencilArgs& a, const P2Args& P, cudaStream_t s) {
  const void* x = a.x;
  int r = P.mode == P2_N1     ? run_phases_n1<T, false>(P, L.cell_stride, x, P.acc, L.n_stored, s)
          : P.mode == P2_MASS ? run_phases<T, P2_MASS>(P, L.cell_stride, x, P.acc, L.n_stored, s)
                              : run_phases<T, P2_STIFF>(P, L.cell_stride, x, P.acc, L.n_stored, s);
  if (r) return r;
  switch (a.op) {
    case OP_APPLY: return run_finish<T, OP_APPLY>(L, a, P, s);
    case OP_RESID: return run_finish<T, OP_RESID>(L, a, P, s);
    case OP_JACOBI: return run_finish<T, OP_JACOBI>(L, a, P, s);
    case OP_CHEB: return run_finish<T, OP_CHEB>(L, a, P, s);
  }
  set_error("P2 operator: operation %d not available", a.op);
  return HG_ERR_UNSUPPORTED;
}

}  // namespace

int p2_upload_constants(const double qbary[14][4], const double qw[14],
                        const double mass[10][10]) {
  (void)qw;
  float qb32[14][4], m32[10][10];
  for (int q = 0; q < 14; ++q)
    for (int m = 0; m < 4; ++m) qb32[q][m] = (float)qbary[q][m];
  for (int a = 0; a < 10; ++a)
    for (int b = 0; b < 10; ++b) m32[a][b] = (float)mass[a][b];
  HG_CUDA(cudaMemcpyToSymbol(c_qb64, qbary, sizeof(double) * 56));
  HG_CUDA(cudaMemcpyToSymbol(c_qb32, qb32, sizeof qb32));
  HG_CUDA(cudaMemcpyToSymbol(c_mass64, mass, sizeof(double) * 100));
  HG_CUDA(cudaMemcpyToSymbol(c_mass32, m32, sizeof m32));
  return HG_OK;
}

int launch_p2(const LevelDev& L, int dtype, const StencilArgs& a, const P2Args& P,
              cudaStream_t s) {
  return dtype == HG_F64 ? run_p2<double>(L, a, P, s) : run_p2<float>(L, a, P, s);
}

int launch_p2_diag(const LevelDev& L, int dtype, const P2Args& P, void* invdiag,
                   cudaStream_t s) {
  StencilArgs a{};
  a.out = invdiag;
  a.mode = HG_REPLACE;
  a.mask = HG_MASK_ALL;
  a.op = OP_INVDIAG;
  const bool n1 = P.mode == P2_N1;
  if (dtype == HG_F64) {
    if (int r = n1 ? run_phases_n1<double, true>(P, L.cell_stride, nullptr, P.acc, L.n_stored, s)
                   : run_phases<double, P2_DIAG>(P, L.cell_stride, nullptr, P.acc, L.n_stored, s))
      return r;
    return run_finish<double, OP_INVDIAG>(L, a, P, s);
  }
  if (int r = n1 ? run_phases_n1<float, true>(P, L.cell_stride, nullptr, P.acc, L.n_stored, s)
                 : run_phases<float, P2_DIAG>(P, L.cell_stride, nullptr, P.acc, L.n_stored, s))
    return r;
  return run_finish<float, OP_INVDIAG>(L, a, P, s);
}

}  // namespace hg
