/*
 * hytet.h - C ABI of the GB300 matrix-free P1/P2 library.
 *
 * The calls follow the paper's statement of the problem (Kohl, Bauer, Boehm,
 * Ruede, "Fundamental data structures for matrix-free finite elements on
 * hybrid tetrahedral grids"): build the macro mesh (Sec. 2, macro-primitive
 * graph), refine it to a range of levels (Sec. 3.1, Bey's rule; Sec. 5.1,
 * functions on level ranges), apply an operator (Sec. 5.2, apply()), and run
 * geometric multigrid on the refinement hierarchy (Sec. 1/5.1, multigrid by
 * design).
 *
 * Conventions
 * -----------
 * - Every function returns 0 (HG_OK) or a negative HG_ERR_* code; the
 *   message of the last error on the calling thread is hg_last_error().
 * - Handles are opaque and owned by the library; *_destroy frees them.
 *   Passing NULL to a destroy function is a no-op.
 * - Vectors are caller-owned device buffers (plain pointers), laid out as
 *   "stored" vectors: macro cell c occupies elements
 *   [c*cell_stride, (c+1)*cell_stride).  Inside a cell the micro-vertex
 *   (i,j,k), i+j+k <= n (n = 2^level), is at t_{n+1}(i,j,k) (Sec. 4,
 *   linearisation t_w).  A P2 function on level l (vertex and edge DoFs of
 *   the level-l micro-cells, Sec. 5.1) is stored as the vertex lattice of
 *   level l+1: micro-vertices are its even points and every other point is
 *   the midpoint of exactly one level-l micro-edge (the seven parity classes
 *   are the seven edge directions), so P2 on level l uses the layout, copies
 *   and canonical order of lattice level l+1; a hierarchy built to lmax
 *   serves P2 levels up to lmax-1.
 *   Tail padding of each cell block is never written by the library.
 *   Micro-vertices on macro faces/edges/vertices are stored once per macro
 *   cell that contains them; every library call leaves all copies equal.
 * - The library never frees caller memory.  It allocates its own device
 *   tables (maps, stencils, work vectors) when a handle is created.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Calls are asynchronous with respect to the host unless stated.
 * - Dirichlet DoFs are those on macro faces with one incident macro cell and
 *   on the edges/vertices of such faces.  HG_MASK_INNER computes the rows of
 *   the other DoFs (taking x as given at the Dirichlet DoFs) and sets the
 *   Dirichlet entries of the destination to 0 for an apply (HG_REPLACE and
 *   HG_ADD alike) and a residual, and to x's values for the smoothing steps
 *   (Jacobi, Gauss-Seidel, Chebyshev); HG_MASK_ALL computes the full Neumann
 *   rows.
 */
#ifndef HYTET_H
#define HYTET_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  HG_OK = 0,
  HG_ERR_INVALID_ARG = -1,
  HG_ERR_BAD_MESH = -2,
  HG_ERR_LEVEL_RANGE = -3,
  HG_ERR_CUDA = -4,
  HG_ERR_NOT_CONVERGED = -5,
  HG_ERR_TIMEOUT = -6,
  HG_ERR_UNSUPPORTED = -7
};

enum { HG_F32 = 0, HG_F64 = 1 };
enum { HG_SPACE_P1 = 1, HG_SPACE_P2 = 2 };
enum { HG_REPLACE = 0, HG_ADD = 1 };
enum { HG_MASK_INNER = 0, HG_MASK_ALL = 1 };

/* Operator kinds (Sec. 5.2, operator examples). */
enum {
  HG_OP_P1_LAPLACE = 0,  /* -div grad, constant-coefficient 15-point stencils     */
  HG_OP_P1_MASS = 1,     /* P1 mass, constant-coefficient stencils               */
  HG_OP_P1_DIVKGRAD = 2, /* -div(k grad), element-wise, k_T = mean of vertex k   */
  HG_OP_P2_LAPLACE = 3,  /* P2 -div grad, element-wise                           */
  HG_OP_P2_MASS = 4,     /* P2 mass, element-wise                                */
  HG_OP_P2_DIVKGRAD = 5, /* P2 -div(k grad), k(x) = a + b sin2pix sin2piy sin2piz
                            by quadrature on the fly                             */
  HG_OP_P1_DIVKGRAD_STORED = 6, /* HG_OP_P1_DIVKGRAD with grid-aware precomputation
                            (Sec. 5.2): the 15-point partial stencil of every
                            stored point kept in HBM (16 values per stored DoF
                            and level: 15 weights and the inverse centre weight;
                            FP64 and FP32 copies) and streamed by the apply     */
  HG_OP_N1_CURLCURL = 7, /* lowest-order Nedelec (first kind) alpha curl curl +
                            beta I, coeff = {alpha >= 0, beta > 0}: one DoF per
                            micro-edge (tangential line integral, oriented from
                            the lower to the higher canonical vertex key),
                            stored as HG_SPACE_P2 vectors at the edge-midpoint
                            points (vertex points stay 0); element-wise 6x6
                            matrices; apply, residual, Jacobi and Chebyshev
                            steps; multigrid with Hiptmair smoothing           */
  HG_OP_P1_DIVKGRAD_SURROGATE = 8 /* HG_OP_P1_DIVKGRAD with polynomial surrogate
                            stencils (Sec. 5.2): made by hg_op_create_surrogate */
};

typedef struct hg_mesh hg_mesh;
typedef struct hg_hier hg_hier;
typedef struct hg_op hg_op;
typedef struct hg_gmg hg_gmg;

/* Message of the last failed call on this thread ("" if none). */
const char* hg_last_error(void);

/* ---------------------------------------------------------------- mesh --
 * Macro mesh (Sec. 2: triangulation conditions; macro-primitive graph of
 * vertices/edges/faces/cells with neighbour links).
 *   xyz   : host, nv*3 doubles, vertex coordinates.
 *   cells : host, nc*4 int64 vertex ids; the order in each row is the local
 *           vertex order v0..v3 of the macro cell and fixes its refinement
 *           (inner edge v02-v13, Sec. 3.1).
 * Checks: ids in range, no repeated vertex in a cell, every vertex in some
 * cell, nonzero volume, every
 * face shared by at most two cells, which lie on opposite sides of it (a
 * cell listed twice, or two cells folded over a common face, overlap and are
 * rejected).  Errors: HG_ERR_INVALID_ARG,
 * HG_ERR_BAD_MESH.  Copies the input; caller keeps ownership. */
int hg_mesh_create(const double* xyz, int64_t nv, const int64_t* cells, int64_t nc,
                   hg_mesh** out);
void hg_mesh_destroy(hg_mesh* mesh);
/* counts[0..5] = macro vertices, edges, faces, cells, boundary faces,
 * interior faces. */
int hg_mesh_counts(const hg_mesh* mesh, int64_t counts[6]);

/* --------------------------------------------------------- hierarchy --
 * Refinement of every macro cell to levels lmin..lmax (Sec. 3.1, Bey's
 * rule applied recursively; Sec. 5.1, functions allocated on a level range).
 * 0 <= lmin <= lmax <= 9.  Uploads per-level maps to the current device.
 * Limits, checked before anything is allocated (HG_ERR_UNSUPPORTED): at most
 * 2^31 - 1 stored points on level lmax; on meshes with coordinates on a
 * lattice of spacing 1/D, |coordinate| x D x 2^lmax below 2^20; no macro
 * face, edge or vertex in more than 255 cells.
 * Errors: HG_ERR_LEVEL_RANGE, HG_ERR_UNSUPPORTED, HG_ERR_CUDA. */
int hg_hier_create(const hg_mesh* mesh, int lmin, int lmax, hg_hier** out);
void hg_hier_destroy(hg_hier* hier);

/* Sizes of a stored vector (n_stored, including per-cell copies and padding),
 * the number of unique DoFs (n_unique) and of non-Dirichlet unique DoFs
 * (n_inner), and the per-cell stride (a multiple of 32 elements with at least
 * 32 spare; the kernels may read, never write, the spare elements).  Any
 * output may be NULL.  space: HG_SPACE_P1 or HG_SPACE_P2. */
int hg_function_size(const hg_hier* hier, int space, int level, int64_t* n_stored,
                     int64_t* n_unique, int64_t* n_inner, int64_t* cell_stride);

/* Canonical order of unique DoFs: ascending (z, y, x) of the exact lattice
 * point (P2: of the doubled lattice, edge DoFs at midpoints).  Host outputs:
 *   stored_to_canon : n_stored int64, -1 for padding     (may be NULL)
 *   xyz             : n_unique*3 doubles, coordinates    (may be NULL)
 *   dirichlet       : n_unique uint8, 1 on the boundary  (may be NULL)
 * Requires vertex coordinates that are integers after scaling by some
 * D <= 64 (HG_ERR_UNSUPPORTED otherwise). */
int hg_canonical_info(const hg_hier* hier, int space, int level, int64_t* stored_to_canon,
                      double* xyz, uint8_t* dirichlet);

/* Device gather stored -> canonical (one value per unique DoF) and scatter
 * canonical -> every stored copy (padding untouched).  dtype HG_F32/HG_F64. */
int hg_to_canonical(const hg_hier* hier, int space, int level, int dtype, const void* stored,
                    void* canonical, void* stream);
int hg_from_canonical(const hg_hier* hier, int space, int level, int dtype,
                      const void* canonical, void* stored, void* stream);

/* ------------------------------------------------------------- functions --
 * A finite-element function on a level range (Sec. 5.1: one vector per level
 * of the hierarchy).  hg_function_create makes an empty function of `space`
 * and element type `dtype` (HG_F32/HG_F64) on the levels of `hier`; the
 * function keeps a pointer to the hierarchy, which must outlive it.
 * hg_function_bind attaches the caller's device buffer dev_ptr (a stored
 * vector of that level, at least n_stored elements of dtype, 16-byte
 * aligned; NULL unbinds) to `level`; the library never frees it.
 * hg_function_data returns the bound pointer (NULL if none).
 * Errors: HG_ERR_INVALID_ARG (null handle, short or unaligned buffer, bad
 * dtype), HG_ERR_LEVEL_RANGE, HG_ERR_UNSUPPORTED (space). */
typedef struct hg_func hg_func;
int hg_function_create(const hg_hier* hier, int space, int dtype, hg_func** out);
void hg_function_destroy(hg_func* f);
int hg_function_bind(hg_func* f, int level, void* dev_ptr, int64_t nbytes);
int hg_function_data(const hg_func* f, int level, void** dev_ptr);

/* Copy the function's vector on `level` to or from HOST memory in canonical
 * order (one value per unique DoF, the order of hg_canonical_info).
 *   host       : n values of host_dtype (HG_F32/HG_F64); pinned memory makes
 *                the call fully asynchronous, pageable memory is allowed
 *   n          : must equal the level's n_unique
 *   dir        : HG_COPY_FROM_HOST: host -> device, then every stored copy of
 *                a DoF set (padding untouched); HG_COPY_TO_HOST: one value
 *                per DoF gathered, then device -> host
 * A host dtype other than the function's is converted on the device
 * (rounding to nearest).  Stream-ordered on `stream`: a TO_HOST result is in
 * `host` once the stream has been synchronised.  The first copy on a level
 * allocates the function's staging buffer (n_unique * 8 bytes, so it must
 * not be the first inside a stream capture); copies of one function on one
 * level share that buffer, so the caller orders them (one stream, or events).
 * Errors: HG_ERR_INVALID_ARG (n, dtype, direction, unbound level),
 * HG_ERR_LEVEL_RANGE, HG_ERR_UNSUPPORTED (no exact lattice), HG_ERR_CUDA. */
enum { HG_COPY_TO_HOST = 0, HG_COPY_FROM_HOST = 1 };
int hg_function_copy_canonical(hg_func* f, int level, void* host, int host_dtype, int64_t n,
                               int dir, void* stream);

/* hg_apply on the functions' bound vectors of `level` (same hierarchy and
 * space as the operator, same element type; x and y distinct functions). */
int hg_apply_function(const hg_op* op, int level, const hg_func* x, hg_func* y, int mode, int mask,
                      void* stream);

/* ------------------------------------------------ distribution over ranks --
 * (Sec. 2: macro primitives distributed over processes, one ghost-layer
 * exchange per operator application.)  Host only; no device is touched.
 *
 * hg_partition_cells: part[c] in 0..nparts-1 for each macro cell c (nc int32,
 * caller-owned): recursive coordinate bisection of the cell centroids (cut
 * along the longest extent, cells ordered by that coordinate, then the
 * others, then id; set sizes in proportion to the parts on either side).
 * Deterministic.  HG_ERR_INVALID_ARG unless 1 <= nparts <= nc.
 *
 * hg_exchange_plan: what rank `rank` sends, receives and sums on `level`
 * when each rank stores only its own cells, in ascending global cell id,
 * with the single-device cell stride (local stored index = local cell *
 * stride + t_{n+1}(i,j,k)).  The points planned are the interface points
 * whose copies lie on two or more ranks, this rank's among them, in a fixed
 * global order (faces, edges, vertices in mesh order, points in primitive
 * order).  After a local application that leaves at those points the
 * partial sum of each copy's own cell, the rank
 *   - sends to rank r the partials at send_idx[off_r .. off_r+send_count[r])
 *     (off_r = sum of the counts of ranks below r): its copies of the points
 *     it shares with r, point by point, copies in ascending cell id;
 *   - receives recv_count[r] partials from r in r's matching order, the
 *     buffers of all ranks concatenated by ascending rank;
 *   - for point p, sums the terms point_start[p] .. point_start[p+1]-1 in
 *     that order (all copies in ascending global cell id): term_src >= 0 is a
 *     local stored index, term_src = -(1 + s) is slot s of the concatenated
 *     receive buffer; and writes the sum to the local stored indices
 *     target_idx[target_start[p] .. target_start[p+1]-1] (its own copies).
 * This is the summation order of the single-device kernels, so the result
 * is identical.  For norms and dots each point counts once, at the copy of
 * its lowest-id cell: a planned point is owned by this rank iff its first
 * term is local (term_src[point_start[p]] >= 0, that index being the owned
 * copy).  sizes (host int64[6]) receives: number of send entries,
 * receive entries, points, terms, targets and the cell stride; call with the
 * arrays NULL to size them (send_count, recv_count: nparts entries;
 * point_start, target_start: points + 1).  Errors: HG_ERR_INVALID_ARG,
 * HG_ERR_LEVEL_RANGE (level outside 0..9). */
int hg_partition_cells(const hg_mesh* mesh, int nparts, int32_t* part);
int hg_exchange_plan(const hg_mesh* mesh, int level, const int32_t* part, int nparts, int rank,
                     int64_t sizes[6], int64_t* send_count, int64_t* send_idx,
                     int64_t* recv_count, int64_t* point_start, int64_t* term_src,
                     int64_t* target_start, int64_t* target_idx);

/* Synchronise `stream` and report whether any kernel of this hierarchy gave
 * up a bounded wait (HG_ERR_TIMEOUT; the word is then cleared).  Kernels
 * never spin without a limit: a wait that runs out records the error and the
 * kernel finishes, so the context stays usable.  hg_dot and hg_solve check
 * the same word at their synchronisation points. */
int hg_device_status(const hg_hier* hier, void* stream);

/* The plane-window tiles the constant-stencil and stored-stencil apply
 * kernels use on one cell lattice of `level` (host, needs no GPU; the same
 * for every cell), 4 ints per tile: (k | windows << 16, lattice offset of
 * lane 0's first point, j0 << 16 | i0 of that point, 0).  *n_tiles gets the
 * count; out may be NULL to query it.  Exported so that tests can check the
 * kernels' lane walk against the lattice on the CPU. */
int hg_plane_tiles(int level, int* out, int* n_tiles);

/* The column-march items of the constant-stencil kernel (HG_P1_KERNEL_MARCH)
 * on one cell lattice of `level` (host, needs no GPU; the same for every
 * cell), 2 ints per item: (k | i0 << 16, j0 | j1 << 16): columns i0..i0+31 of
 * plane k, rows j0..j1-1.  *n_items gets the count; out may be NULL.  For the
 * CPU emulation of the kernel's loads in the tests. */
int hg_march_items(int level, int* out, int* n_items);

/* The plan of the streaming constant-stencil apply kernel for one level of a
 * mesh with `ncells` macro cells, split over `nctas` CTAs, for dtype
 * HG_F32/HG_F64 (host, needs no GPU).  copies: 4 ints per copy (cell, first
 * element, elements, 0); items: 12 ints per item (cell, plane k, ja | jb << 16,
 * arrival counts; the CTA-local copies holding planes k, k-1, k+1 or -1; the
 * first elements of those copies); cta_copies / cta_items: nctas + 1 offsets.
 * counts receives (copies, items, rows per band).  Any output pointer may be
 * NULL (counts only).  Exported so that tests can check on the CPU that the
 * items cover every lattice point once and read inside the staged copies. */
int hg_stream_plan(int level, int ncells, int nctas, int dtype, int* copies, int* items,
                   int* cta_copies, int* cta_items, int* counts);

/* Shared-memory layout of the streaming kernel on `level` for dtype
 * HG_F32/HG_F64 (host, needs no GPU): the number of ring slots (copy c of a
 * CTA goes to slot c mod ring_slots), the elements per slot and the guard
 * elements before the first and after the last slot.
 * Exported so that tests can check the kernel's index arithmetic on the CPU. */
int hg_stream_layout(int level, int dtype, int* ring_slots, int* slot_elems, int* guard_elems);

/* The anchors of the element-wise colour phases of a P2 or N1 level (host,
 * needs no GPU): packed i | j << 10 | k << 20 (anchor p of the unit cube
 * [p, p+1]^3 that holds the six micro-cells of p), grouped by parity colour
 * c = (i & 1) | (j & 1) << 1 | (k & 1) << 2 in [off[c], off[c+1]) (off: 9
 * ints).  *n_anchors gets the count; out and off may be NULL.  Exported so
 * that tests can check on the CPU that the threads of one phase touch
 * disjoint DoFs. */
int hg_p2_anchors(int level, uint32_t* out, int* off, int* n_anchors);

/* ----------------------------------------------------- index functions --
 * t_w(i,j,k) = N_tet(w) - N_tet(w-k) + N_tri(w-k) - N_tri(w-k-j) + i
 * (Sec. 4).  Host evaluation, 1 <= w <= 2^20 (N_tet(w) fits in int64);
 * HG_ERR_INVALID_ARG if w is out of that range, (i,j,k) is not in I_tet(w)
 * or out is NULL. */
int hg_index_tw(int64_t w, int64_t i, int64_t j, int64_t k, int64_t* out);

/* Device enumeration of I_tet(w) with the same traversal the operator
 * kernels use: out[t_w(i,j,k)] = i + (j << 20) + (k << 40) for every point.
 * out: device, N_tet(w) int64.  1 <= w <= 1025. */
int hg_index_enumerate(int64_t w, int64_t* out, void* stream);

/* Device dump of the interface ("ghost-layer") map of a level: for every
 * shared or boundary macro primitive (vertex/edge/face) point, the cells and
 * cell-local indices of all its copies, in the order the exchange kernel sums
 * them.  Output (device int64): rows of 2*max_copies+1 entries
 * [ncopies, cell_0, local_0, cell_1, local_1, ...], unused entries -1.
 * *n_rows receives the row count (host); call with out == NULL to query
 * n_rows and max_copies first. */
int hg_interface_dump(const hg_hier* hier, int space, int level, int64_t* out,
                      int64_t* n_rows, int64_t* max_copies, void* stream);

/* ---------------------------------------------------------- operators --
 * kind: HG_OP_*.  coeff: for HG_OP_P1_DIVKGRAD(_STORED), host array of k at the
 * unique vertices of level lmax in canonical order (injected to coarser
 * levels), every value positive and finite; for HG_OP_P2_DIVKGRAD, host
 * {a, b} with finite a > |b| (k stays positive); for HG_OP_N1_CURLCURL, host
 * {alpha >= 0, beta > 0}; otherwise NULL.  Other values: HG_ERR_INVALID_ARG.
 * P2 operators (levels max(0, lmin-1) .. lmax-1 of the hierarchy) are
 * element-wise: per micro-cell the 10x10 element matrix acts on the fly by
 * the 14-point rule of hg_quadrature_rule, with k evaluated exactly at every
 * quadrature point; Jacobi uses the assembled diagonal.  P2 applies use an
 * operator-owned accumulation vector per level and dtype: calls on the same
 * operator, level and dtype must not run concurrently on different streams.
 * Element matrices/stencils are computed per macro cell and level in FP64
 * (Sec. 5.2: constant-coefficient stencils precomputed per macro primitive,
 * element matrices on the fly for variable coefficients). */
int hg_op_create(const hg_hier* hier, int kind, const double* coeff, hg_op** out);

/* Surrogate operator of -div(k grad) (Sec. 5.2, surrogate operators: the
 * stencil weights of a variable-coefficient operator vary smoothly over a
 * macro cell and are replaced by low-degree polynomials of the position).
 * Per level, macro cell and stencil direction d (the 15 lattice directions),
 * the exact weights A[p, p+d] at the cell's interior points p = (i, j, k)
 * (i, j, k >= 1, i + j + k <= n - 1) are fitted by least squares with the
 * polynomials of total degree <= `degree` in (i/n, j/n, k/n); interior rows
 * use the fitted weights, every other row (points on macro faces, edges,
 * vertices) stays exact (element-wise, as HG_OP_P1_DIVKGRAD).  When a level
 * has too few interior points to fix every coefficient, the fit is the
 * least-squares projection onto the polynomials the points separate (the
 * fitted values are unique).  k as for HG_OP_P1_DIVKGRAD; degree 0..4, else
 * HG_ERR_INVALID_ARG.  The fit runs once per level in FP64 on the device
 * (a QR factorisation of the polynomial basis at the interior points on the
 * host, the projections of the weights on the device); the polynomials are
 * evaluated on the fly, per lattice row by Horner's rule in i.  Apply,
 * residual, Jacobi, Gauss-Seidel and Chebyshev steps and multigrid work as
 * for the other P1 kinds; the diagonal is the surrogate's own. */
int hg_op_create_surrogate(const hg_hier* hier, const double* k, int degree, hg_op** out);

/* Kernel of the P1 constant-stencil operators (apply, residual, Jacobi,
 * Gauss-Seidel and Chebyshev steps), process-wide, for calls made after it:
 *   HG_P1_KERNEL_AUTO (default): the streaming kernel (whole planes staged in
 *     shared memory by bulk copies, one CTA per SM, plus a light exchange
 *     launch) for FP32 levels of at least 8 Mi stored points; the
 *     plane-window kernel (one launch) otherwise, where launch latency or
 *     FP64 arithmetic dominates;
 *   HG_P1_KERNEL_WINDOWS / HG_P1_KERNEL_STREAM: always that kernel (the
 *     streaming one falls back to plane windows on levels whose staged
 *     planes do not fit in shared memory);
 *   HG_P1_KERNEL_MARCH: the column-march kernel (one launch: each warp holds
 *     32 interior columns of one plane and marches up to 16 rows, keeping the
 *     values of the rows it has read in registers; interface items as in the
 *     plane-window kernel).
 * Both give the same results up to rounding order.  Other values:
 * HG_ERR_INVALID_ARG.  Not synchronised with calls in flight. */
enum { HG_P1_KERNEL_AUTO = 0, HG_P1_KERNEL_WINDOWS = 1, HG_P1_KERNEL_STREAM = 2,
       HG_P1_KERNEL_MARCH = 3 };
int hg_set_p1_kernel(int mode);

/* Class table of the lowest-order Nedelec prolongation (host, needs no GPU).
 * A fine N1 DoF sits at an odd point q of the fine F lattice (the level+1
 * lattice of the fine N1 level); with q = 4p + r, r in {0..3}^3 and class
 * c = r_x + 4 r_y + 16 r_z, its value is
 *   s[fine_dir[c]] * sum_{t < n[c]} w[6c+t] * s[dir[6c+t]] * u_C(2p + off[6c+t])
 * where u_C are the coarse N1 DoFs on the C lattice, off packs (x | y << 2 |
 * z << 4), s[d] is the orientation sign of lattice direction d in the macro
 * cell (+1 when its physical vector has a positive first nonzero of z, y, x)
 * and the directions d = 0..6 are (1,0,0), (0,1,0), (-1,1,0), (0,0,1),
 * (-1,0,1), (0,-1,1), (1,-1,1) (the midpoints of direction d have parity
 * class d + 1).  Outputs (host, any may be NULL): n[64], off[384], dir[384],
 * w[384], fine_dir[64] (-1 for classes of vertex points). */
int hg_n1_prolong_table(int* n, int* off, int* dir, double* w, int* fine_dir);

/* The transpose of that table, per coarse parity class pc = 1..7 (the coarse
 * DoF c has direction pc - 1): entries start[pc] .. start[pc+1]-1 (start: 9
 * ints, start[8] = total, at most 512) give the fine points 2c + delta
 * (delta packed as dx+8 | (dy+8) << 5 | (dz+8) << 10, F-lattice units), so
 *   r_C(c) = s[pc-1] * sum_e w[e] * s[fine_dir[e]] * r_F(2c + delta[e])
 * over the fine points inside the cell.  Host, needs no GPU; any output may
 * be NULL (d, w, fine_dir: at least start[8] entries). */
int hg_n1_restrict_table(int* start, int* d, double* w, int* fine_dir);

/* Nedelec transfers and discrete gradient (op: an HG_OP_N1_CURLCURL operator;
 * N1 vectors are HG_SPACE_P2 vectors of the N1 level, P1 vectors of the P1
 * level; dtype HG_F32 or HG_F64; device pointers; stream-ordered).
 * - hg_n1_prolong_add: x_f += P e_c, fine N1 level `fine_level`, coarse
 *   fine_level - 1 (P = tangential line integrals of the coarse function);
 *   boundary (tangential Dirichlet) fine DoFs are left unchanged.
 * - hg_n1_restrict: r_c = P^T r_f on the non-boundary coarse DoFs, 0 on the
 *   boundary ones and at vertex points.
 * - hg_n1_gradient: u = G phi on N1 level `level` from the P1 function phi of
 *   the same level: (G phi)_e = phi(end) - phi(start) in the edge's
 *   orientation, 0 at boundary edges and vertex points.
 * - hg_n1_gradient_t: r_p = G^T r at the non-boundary vertices (0 on the
 *   boundary); r's boundary entries are expected to be 0.
 * Errors: HG_ERR_INVALID_ARG (not an N1 operator, bad pointers),
 * HG_ERR_LEVEL_RANGE. */
int hg_n1_prolong_add(const hg_op* op, int fine_level, int dtype, const void* ec, void* xf,
                      void* stream);
int hg_n1_restrict(const hg_op* op, int fine_level, int dtype, const void* rf, void* rc,
                   void* stream);
int hg_n1_gradient(const hg_op* op, int level, int dtype, const void* phi, void* u, void* stream);
int hg_n1_gradient_t(const hg_op* op, int level, int dtype, const void* r, void* rp,
                     void* stream);

/* The quadrature rule of the P2 element matrices: the symmetric 14-point,
 * degree-5, positive-weight rule (orbits 4+4+6), derived by the library from
 * its moment equations.  Host outputs: bary 14x4 barycentric coordinates,
 * weights 14 (sum 1), *npoints = 14; any may be NULL.  Needs no GPU. */
int hg_quadrature_rule(double* bary, double* weights, int* npoints);
void hg_op_destroy(hg_op* op);

/* y = A x (HG_REPLACE) or y += A x (HG_ADD) on one level; the ghost-layer
 * exchange between macro cells is part of the call (Sec. 5.2 apply()).
 * x and y are distinct stored vectors of the operator's space/level/dtype. */
int hg_apply(const hg_op* op, int level, int dtype, const void* x, void* y, int mode,
             int mask, void* stream);

/* r = b - A x on the non-Dirichlet DoFs, r = 0 on Dirichlet DoFs. */
int hg_residual(const hg_op* op, int level, int dtype, const void* x, const void* b, void* r,
                void* stream);

/* Weighted Jacobi step x_out = x + omega D^-1 (b - A x) on non-Dirichlet
 * DoFs; Dirichlet DoFs copied from x.  x and x_out must not alias. */
int hg_jacobi(const hg_op* op, int level, int dtype, double omega, const void* x,
              const void* b, void* x_out, void* stream);

/* One colour sub-sweep of 4-colour Gauss-Seidel, out of place: x_out = x
 * with the DoFs of `colour` (0..3) replaced by x + D^-1 (b - A x), every
 * other DoF copied.  Colours 0,1,2,3 in turn (ping-ponging x and x_out) are
 * one sweep.  The colour of a lattice point is (a X + b Y + c Z) mod 4 of its
 * exact integer coordinates, with (a, b, c) chosen by the hierarchy so that
 * no micro-edge joins two points of one colour.  P1 operators only; x and
 * x_out must not alias.  Errors: HG_ERR_UNSUPPORTED (P2 operator, or no
 * such colouring for this mesh), HG_ERR_INVALID_ARG. */
int hg_gauss_seidel(const hg_op* op, int level, int dtype, int colour, const void* x,
                    const void* b, void* x_out, void* stream);

/* The Gauss-Seidel colours of a P1 level in canonical DoF order (host,
 * n_unique bytes).  HG_ERR_UNSUPPORTED if the mesh admits no colouring. */
int hg_gs_colours(const hg_hier* hier, int level, uint8_t* colours);

/* Grid transfers between level and level-1 (nodal interpolation P and its
 * transpose): r_coarse = P^T r_fine (Dirichlet DoFs of r_coarse set to 0);
 * x_fine += P e_coarse (Dirichlet DoFs of x_fine untouched). */
int hg_restrict(const hg_hier* hier, int space, int fine_level, int dtype, const void* r_fine,
                void* r_coarse, void* stream);
int hg_prolong_add(const hg_hier* hier, int space, int fine_level, int dtype,
                   const void* e_coarse, void* x_fine, void* stream);

/* Deterministic FP64 dot product over unique DoFs (each counted once),
 * non-Dirichlet only (HG_MASK_INNER) or all (HG_MASK_ALL).  The result is
 * written to *result (host) after the call synchronises `stream`. */
int hg_dot(const hg_hier* hier, int space, int level, int dtype, const void* x, const void* y,
           int mask, double* result, void* stream);

/* Same dot product as hg_dot, for callers that cannot allocate device memory
 * (the paper has no counterpart: this is a deployment variant).  Such
 * callers are code running inside a memory pool or arena that owns the whole
 * device, code that must not trigger the implicit synchronisation of
 * cudaMalloc/cudaFree, or code on paths where allocation is not allowed.
 * hg_dot_noalloc allocates nothing: its per-block partial sums live in one
 * fixed 4 KB array in device global memory (512 doubles, kept by every GPU
 * that loads the library until the process exits), and the result goes to
 * the caller's device pointer `result` (one double) without synchronising.
 *   Limit: at most 512 x 256 = 131072 lattice rows per level (rows = cells x
 *   (n+1)(n+2)/2); larger levels are rejected with HG_ERR_INVALID_ARG.
 *   The first call on a device looks up the array's device address (with
 *   that device current); make that first call before any stream capture.
 *   All calls share the array: calls that overlap on the GPU (other streams
 *   or host threads) race and give wrong results.  Each call rewrites the
 *   partials it reads, so nothing has to be cleared between calls. */
int hg_dot_noalloc(const hg_hier* hier, int space, int level, int dtype, const void* x,
                   const void* y, int mask, double* result, void* stream);

/* ---------------------------------------------------------- multigrid --
 * Geometric multigrid on the refinement hierarchy (multigrid by design,
 * Sec. 5.1): V(nu1,nu2) cycles with weighted-Jacobi smoothing (Sec. 5.2.1:
 * smoothers that need only the matrix-vector product and the diagonal),
 * Chebyshev-accelerated Jacobi (Sec. 5.2.1; order 2 in the FMG solver of
 * Sec. 6) or 4-colour Gauss-Seidel (P1 operators),
 * restriction P^T and prolongation P (nodal interpolation), and an exact
 * FP64 solve on the coarsest level (dense Cholesky inverse, <= 2048
 * unknowns; built at creation by applying the operator to unit vectors).
 * Every P1 and P2 operator kind is accepted.  For HG_OP_N1_CURLCURL the
 * smoothing is Hiptmair's hybrid scheme (Sec. 6): a smoothing step on the
 * edge operator, the residual taken to the P1 potential space by G^T, a
 * smoothing step from zero with G^T A G = beta * (P1 Laplacian) and the
 * correction G e_p added; N1 transfers.  Smoothers: HG_SMOOTH_JACOBI
 * (weighted Jacobi in both spaces, omega in (0, 0.6]: lambda_max(D^-1 A)
 * exceeds 3 for the edge matrices; 1/2 is the tested choice; else
 * HG_ERR_INVALID_ARG) or HG_SMOOTH_CHEB (cheb_order Chebyshev steps in both
 * spaces on [cheb_lo, cheb_hi] times each space's lambda_max, the paper's
 * choice); HG_SMOOTH_GS: HG_ERR_UNSUPPORTED. */
enum { HG_PREC_F64 = 0,   /* plain FP64 V-cycles                                  */
       HG_PREC_MIXED = 1  /* FP32 V-cycles inside FP64 iterative refinement: the
                             outer residual, norms and coarse solve stay FP64   */
};

typedef struct {
  int nu1, nu2;        /* pre-/post-smoothing steps (default 3, 3)               */
  double omega;        /* Jacobi weight (default 2/3)                            */
  int lmin;            /* coarsest level; -1 = the hierarchy's lmin              */
  int inner_cycles;    /* FP32 V-cycles per refinement step (default 1)          */
  int smoother;        /* HG_SMOOTH_JACOBI (default); HG_SMOOTH_GS: one step =
                          one 4-colour Gauss-Seidel sweep (P1 operators);
                          HG_SMOOTH_CHEB: one step = cheb_order steps of the
                          Chebyshev semi-iteration for D^-1 A on the interval
                          [cheb_lo, cheb_hi] * lambda_max (any operator kind)    */
  int cheb_order;      /* Chebyshev: matrix-vector products per step (default 2) */
  int cheb_iters;      /* Chebyshev: power iterations per level for lambda_max at
                          creation (default 20)                                  */
  double cheb_lo, cheb_hi; /* Chebyshev interval in units of lambda_max
                          (default 0.1, 1.1)                                     */
} hg_gmg_params;
enum { HG_SMOOTH_JACOBI = 0, HG_SMOOTH_GS = 1, HG_SMOOTH_CHEB = 2 };

/* Fill *p with the defaults above. */
void hg_gmg_default_params(hg_gmg_params* p);

/* Allocates per-level work vectors (FP64; FP32 on first mixed use) and the
 * coarse inverse on the current device.  p == NULL selects the defaults.
 * Errors: HG_ERR_LEVEL_RANGE, HG_ERR_INVALID_ARG (bad parameters, coarse
 * level too large or not SPD), HG_ERR_UNSUPPORTED, HG_ERR_CUDA. */
int hg_gmg_create(const hg_op* op, const hg_gmg_params* p, hg_gmg** out);
void hg_gmg_destroy(hg_gmg* g);

/* One V-cycle on `level` (lmin < level <= lmax: smoothing, residual,
 * restriction, recursion, prolongation; level == lmin: coarse solve):
 * x is updated in place towards A^-1 b.  x, b: stored vectors of dtype. */
int hg_vcycle(hg_gmg* g, int level, int dtype, void* x, const void* b, void* stream);

/* Solve A x = b on lmax (FP64 stored vectors) from x = 0 until
 * ||b - A x||_2 <= rel_tol ||b||_2 over the non-Dirichlet DoFs, at most
 * max_iter V-cycles (HG_PREC_F64) or refinement steps (HG_PREC_MIXED).
 * Synchronises `stream` once per iteration to test convergence.  Outputs
 * iterations and the final relative residual (may be NULL).
 * HG_ERR_NOT_CONVERGED when the cap is reached (x holds the last iterate). */
int hg_solve(hg_gmg* g, int precision, double* x, const double* b, double rel_tol, int max_iter,
             int* iters, double* rel_res, void* stream);

/* hg_solve on the functions' bound vectors of the finest level lmax (FP64
 * functions of the operator's hierarchy and space). */
int hg_solve_function(hg_gmg* g, int precision, hg_func* x, const hg_func* b, double rel_tol,
                      int max_iter, int* iters, double* rel_res, void* stream);

/* Relative residuals of the last solve (entry 0 = 1 for x = 0); *n gets the
 * count, at most cap values are written to out (host). */
int hg_gmg_history(const hg_gmg* g, double* out, int cap, int* n);

/* Chebyshev smoothing needs lambda_max(D^-1 A) on every smoothed level
 * (lmin < level <= lmax).  hg_gmg_create estimates it with cheb_iters steps
 * of the power iteration from a fixed pseudo-random start vector (SplitMix64
 * of the canonical DoF index, in [-1, 1), 0 on Dirichlet DoFs).
 * hg_gmg_lambda reads the value in use, hg_gmg_set_lambda replaces it
 * (lam > 0, finite).  hg_gmg_power_lambda runs the power iteration from a
 * caller's start vector v0 (FP64 stored vector of the level, device; its
 * Dirichlet entries are ignored): v = v0 / ||v0||, then `iters` times
 * w = D^-1 A v, lambda = ||w||, v = w / ||w||, 2-norms over the unique
 * non-Dirichlet DoFs; *lam gets the last lambda (the value in use is not
 * changed).  It uses the level's FP64 work vectors and synchronises `stream`
 * once per step.  Errors: HG_ERR_LEVEL_RANGE, HG_ERR_INVALID_ARG (iters
 * outside 1..10000, v0 zero on the non-Dirichlet DoFs). */
int hg_gmg_lambda(const hg_gmg* g, int level, double* lam);
int hg_gmg_set_lambda(hg_gmg* g, int level, double lam);
int hg_gmg_power_lambda(hg_gmg* g, int level, const double* v0, int iters, double* lam,
                        void* stream);
/* Nedelec multigrid with Chebyshev smoothing: lambda_max(D^-1 K) of the
 * potential space (the P1 Laplacian K; D^-1 A is the same for beta K) per
 * smoothed level, estimated at creation like the edge space's (power
 * iteration from the SplitMix64 start vector of the P1 canonical DoFs);
 * read and replace it.  HG_ERR_INVALID_ARG for other operators. */
int hg_gmg_potential_lambda(const hg_gmg* g, int level, double* lam);
int hg_gmg_set_potential_lambda(hg_gmg* g, int level, double lam);

/* Full multigrid (nested iteration; the paper's solver in Sec. 6 runs five
 * V(1,1) cycles per level): b (stored vector of dtype on `level`) is
 * restricted to every coarser level (b_{l-1} = P^T b_l), the coarsest level
 * is solved exactly, and on each finer level l the prolongated solution of
 * level l-1 starts `cycles` V-cycles.  x (stored vector of dtype on `level`)
 * receives the result; its input is ignored.  Stream-ordered, no host
 * synchronisation.  Uses the work vectors of the levels below `level`. */
int hg_fmg(hg_gmg* g, int level, int dtype, void* x, const void* b, int cycles, void* stream);

/* New GMG for the same operator and parameters with its own work vectors
 * (the coarse inverse is copied, not rebuilt); for batches of problems that
 * share a hierarchy. */
int hg_gmg_clone(const hg_gmg* src, hg_gmg** out);

/* --------------------------------------------------------- batched solves --
 * A batch solves `count` independent problems A_p x_p = b_p (each a GMG over
 * its own hierarchy and constant-stencil operator; x_p, b_p FP64 stored
 * vectors of its finest level, device pointers fixed for the batch's life)
 * with FP32 V-cycles inside FP64 iterative refinement (Sec. 5.1 multigrid,
 * many problems at once).  Each V-cycle stage (a smoothing sweep, the
 * residual, a restriction, the coarse solves, a prolongation) and each
 * refinement step is ONE persistent launch over the work of all problems
 * taking part; problems with fewer levels are aligned by the distance from
 * their finest level.
 *   flags: HG_BATCH_GRAPH    capture the stage sequence as two CUDA graphs
 *                            (residual + norms; correction) and replay them,
 *          HG_BATCH_AUTOTUNE time the stage-kernel variants (plane-window
 *                            prefetch depth 0/1/2 x 1/2/4 x 4 blocks per SM)
 *                            at creation and keep the fastest.
 * Every problem needs its own hg_gmg (hg_gmg_clone) with the same
 * nu1/nu2/inner_cycles; a problem may not appear twice.  The batch holds
 * the problems' handles: destroy it before them. */
typedef struct hg_batch hg_batch;
enum { HG_BATCH_GRAPH = 1, HG_BATCH_AUTOTUNE = 2 };
int hg_batch_create(hg_gmg* const* problems, int count, double* const* x, const double* const* b,
                    int flags, hg_batch** out);
void hg_batch_destroy(hg_batch* batch);
/* Zero every x_p, then iterate until every problem has met rel_tol (or
 * max_iter).  iters[p]: the step at which problem p first met rel_tol;
 * rel_res[p]: its relative residual then (or at exit).  A converged problem
 * keeps its iterate unchanged while the others continue.  Ordered after
 * `stream`'s prior work, synchronises it.  Errors: HG_ERR_NOT_CONVERGED
 * (results still written), HG_ERR_INVALID_ARG. */
int hg_batch_solve(hg_batch* batch, double rel_tol, int max_iter, int* iters, double* rel_res,
                   void* stream);
/* The stage-kernel variant in use: plane-window prefetch depth, blocks per SM / 4,
 * and (after autotuning) the fastest finest-stage time in microseconds. */
int hg_batch_tuning(const hg_batch* batch, int* rows, int* grid_factor, double* stage_us);

/* ------------------------------------------------- learned local smoother --
 * A small network N (16 -> 32 -> 32 -> 1, ReLU, no biases, so N(a s) =
 * a N(s) for a > 0) maps the 15-point neighbourhood of s = D^-1 (b - A x) at
 * a DoF to a correction; the learned smoothing step is
 *   x <- x + omega s + N(s)  (macro-cell-interior DoFs),  x + omega s  (others).
 * The paper has no learned component; this extends its matvec+diagonal
 * smoothers.  Evaluated and trained with BF16 tensor-core kernels that
 * accumulate in FP32.  Parameters: 1568 floats = W1 (32x16, row = output) |
 * W2 (32x32) | w3 (32). */
typedef struct hg_mlp hg_mlp;

/* New network with zero weights (N = 0) on the current device. */
int hg_mlp_create(hg_mlp** out);
void hg_mlp_destroy(hg_mlp* mlp);
/* Host copies of the 1568 FP32 parameters; set also resets the optimiser. */
int hg_mlp_set_params(hg_mlp* mlp, const float* params);
int hg_mlp_get_params(const hg_mlp* mlp, float* params);
/* out[b] = N(X[b]) for n rows of 16 FP32 features (device, rounded to bf16). */
int hg_mlp_forward(const hg_mlp* mlp, const float* X, int64_t n, float* out, void* stream);
/* Gradient of L = mean_b (N(X_b) - t_b)^2 over n samples: X device bf16
 * [n][16] (16-byte aligned), t device FP32 [n].  grad (host, 1568 floats)
 * and loss (host) may be NULL.  Synchronises `stream`. */
int hg_mlp_grad(hg_mlp* mlp, const void* X, const float* t, int64_t n, float* grad,
                double* loss, void* stream);
/* `steps` Adam steps (lr, beta 0.9/0.999) on consecutive minibatches of
 * `batch` samples (wrapping); *final_loss (if not NULL) = L over all n. */
int hg_mlp_train(hg_mlp* mlp, const void* X, const float* t, int64_t n, int steps,
                 int64_t batch, double lr, double* final_loss, void* stream);
/* Training pairs from one residual/error state on `level` (FP32 stored
 * vectors r = b - A x, the converged solution xstar and the iterate x):
 * every stride-th macro-cell-interior DoF (interior rank % stride == offset)
 * gives the features s(15 neighbours) / |s-neighbourhood| (bf16 [16], last 0)
 * and the target (xstar - x - omega s) / |s-neighbourhood|.  With X == NULL
 * only *count is returned. */
int hg_learn_samples(const hg_op* op, int level, const float* r, const float* xstar,
                     const float* x, double omega, int stride, int offset, void* X, float* t,
                     int64_t* count, void* stream);
/* One learned smoothing step on `level` of a P1 operator with a stored
 * diagonal (HG_OP_P1_DIVKGRAD, or its stored-stencil form): with s = D^-1 r
 * (r = b - A x given, FP32 stored vectors; D the operator's diagonal),
 *   x_out = x + omega s + N(F)  at macro-cell-interior DoFs, where F holds s
 *           at the DoF and its 14 lattice neighbours in the cell's own
 *           directions, in the order (0,0,0), (+-1,0,0), (0,+-1,0),
 *           (0,0,+-1), +-(-1,1,0), +-(-1,0,1), +-(0,-1,1), +-(1,-1,1), then 0;
 *   x_out = x + omega s  at the other non-Dirichlet DoFs;  x_out = x  at
 *           Dirichlet DoFs.
 * The step V-cycles use with hg_gmg_set_learned, exposed for tests.  x, r,
 * x_out: device FP32, stored layout; x_out must not alias x or r.  Errors:
 * HG_ERR_INVALID_ARG, HG_ERR_LEVEL_RANGE, HG_ERR_UNSUPPORTED (no stored
 * diagonal). */
int hg_learned_step(const hg_op* op, const hg_mlp* mlp, int level, const float* x,
                    const float* r, double omega, float* x_out, void* stream);

/* Use `mlp` (NULL: none) for the smoothing steps on the finest level of
 * FP32 V-cycles (hg_vcycle with HG_F32, hg_solve with HG_PREC_MIXED).  In a
 * solve, a refinement step that increases the FP64 residual switches the
 * rest of the solve back to the plain smoother (counted). */
int hg_gmg_set_learned(hg_gmg* g, const hg_mlp* mlp);
int hg_gmg_learned_fallbacks(const hg_gmg* g, int* n);

#ifdef __cplusplus
}
#endif
#endif /* HYTET_H */
