// P1 constant-stencil operator application as a streaming kernel
// (Sec. 5.2 apply(), stencil-based pattern, one stencil per macro cell).
//
// A macro cell's lattice is stored plane by plane (k), row by row (j), with
// unit-stride x-lines (i) (the t_w order of Sec. 4), so any run of rows of one
// plane is one contiguous range, and consecutive whole planes are too.  The
// 15-point stencil of plane k reads planes k-1, k and k+1.
//
//  * One CTA per SM: a producer warp and 20 (FP32) or 12 (FP64) consumer
//    warps.  A plan built
//    on the host (stream_plan) gives the CTA a contiguous stretch of the
//    sequence (cell, band of rows, plane), as a list of copies and a list of
//    items (see hg_internal.h).
//  * The producer moves the copies into a ring of kStreamSlots slots of
//    kStreamSlotBytes with 1-D bulk copies (cp.async.bulk, the TMA engine),
//    completion counted in bytes on the slot's mbarrier.  A bulk copy costs
//    the TMA engine a fixed time of the order of 0.2 us, so copies are made
//    large: whole planes where a plane fits a slot, several consecutive planes
//    per copy when they are small.
//  * Consumer warp w takes items w, w + W, ... (W warps): it waits for the
//    copies holding planes k-1, k, k+1, forms the item's interior points from
//    shared memory (32 columns at a time, marching the item's rows with the
//    previous row's values kept in registers; 32-bit shared addresses), then
//    its boundary points, writes y to HBM directly, and arrives on the copies'
//    release barriers.  Every x value crosses HBM once.
//  * Points on the cell's boundary are formed in the pass from the
//    cell's partial stencil: the whole row where the point lies on a
//    primitive of this cell only, the cell's partial where several cells share
//    it.  A second, light launch (the ghost-layer exchange of Sec. 2) adds the
//    copies' partials of every shared point and writes the operation's output
//    to all of them.
//
// Every wait is bounded (about one second): on expiry the kernel records
// HG_ERR_TIMEOUT in the hierarchy's error word, the other warps stop at their
// next wait, and the producer waits (again bounded) for the copies it issued
// before the CTA exits.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "hg_internal.h"
#include "hg_p1dev.cuh"

namespace hg {
namespace {

// Consumer warps (plus one producer warp): as many as the register budget of
// the stencil allows, the consumers being latency-bound.
template <typename T>
__host__ __device__ constexpr int swarps() { return sizeof(T) == 4 ? 20 : 12; }
template <typename T>
__host__ __device__ constexpr int sthreads() { return (swarps<T>() + 1) * 32; }
constexpr unsigned long long kWaitNs = 1000000000ull;
// Longest suspension of one try_wait (the thread resumes as soon as the
// phase completes): waiting warps then take no issue slots.
constexpr int kSuspendNs = 100000;

template <typename T>
__host__ __device__ constexpr int slot_elems() { return kStreamSlotBytes / (int)sizeof(T); }
// Elements before the first and after the last slot: the shared-memory loads
// of lanes past a row's end or next to a copy's edge reach at most w + 2
// elements before a copy's data and 2 w + 33 after it.
inline int guard_elems(int w) { return (4 * w + 64 + 31) / 32 * 32; }
// Barriers (full, empty), the stop flag and one copy tag per slot.
__host__ __device__ constexpr int barrier_bytes() {
  return (2 * kStreamSlots * 8 + 16 + 4 * kStreamSlots + 127) / 128 * 128;
}

// HG_ADD applies get their own instantiation (y += A x) so that a replacing
// apply never reads the destination.
constexpr int kOpApplyAdd = 100;
__host__ __device__ constexpr bool is_apply(int op) { return op == OP_APPLY || op == kOpApplyAdd; }

template <typename T>
struct StreamArgs {
  FusedArgs<T> f;             // operands, stencils, flags and the interface items
  StreamPlanDev plan;
  int guard;                  // elements before / after the ring
};

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* b, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive_cnt(uint64_t* b, int count) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(count)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(b)), "r"(parity), "n"(kSuspendNs)
      : "memory");
  return ok != 0;
}
// 1-D bulk copy global -> shared (16-byte aligned addresses, size a multiple
// of 16), completion counted in bytes on barrier b.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(b))
      : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for the phase of parity `parity` of b; false after kWaitNs, or as
// soon as *stop is set (stop == nullptr: no early exit).
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* stop) {
  if (mbar_try_wait(b, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (long long it = 0; it < (1ll << 40); ++it) {
    if (mbar_try_wait(b, parity)) return true;
    if ((it & 63) == 63) {
      if (stop && *stop) return false;
      if (global_ns() - t0 > kWaitNs) return false;
    }
  }
  return false;
}

// Shared-memory load from a 32-bit shared address plus a constant byte offset.
// Not volatile, so that loads can be scheduled together; the addresses derive
// from a token produced after the barrier waits (wait_token), which keeps the
// loads after them.
template <int OFF>
__device__ __forceinline__ float lds(float*, uint32_t a) {
  float v;
  asm("ld.shared.f32 %0, [%1+%2];" : "=f"(v) : "r"(a), "n"(OFF));
  return v;
}
template <int OFF>
__device__ __forceinline__ double lds(double*, uint32_t a) {
  double v;
  asm("ld.shared.f64 %0, [%1+%2];" : "=d"(v) : "r"(a), "n"(OFF));
  return v;
}
// A zero the compiler cannot see through, produced in program order after
// the preceding waits.
__device__ __forceinline__ uint32_t wait_token() {
  uint32_t z;
  asm volatile("mov.u32 %0, 0;" : "=r"(z)::"memory");
  return z;
}
#define HG_LDS(T, OFF, a) lds<(OFF) * (int)sizeof(T)>((T*)nullptr, (a))

// The operation's output at stored index g from the stencil sum acc.
template <typename T, int OP>
__device__ __forceinline__ void stream_out(const FusedArgs<T>& A, int64_t g, T c, T acc, T wd) {
  if (OP == OP_APPLY) {
    A.y[g] = acc;
  } else if (OP == kOpApplyAdd) {
    A.y[g] += acc;
  } else if (OP == OP_RESID) {
    A.y[g] = A.b[g] - acc;
  } else if (OP == OP_GS) {
    A.y[g] = A.colour[g] == A.gs_colour ? c + (A.b[g] - acc) * wd : c;
  } else if (OP == OP_CHEB) {
    T dn = (A.b[g] - acc) * wd;
    if (A.cheb_a != T(0)) dn += A.cheb_a * A.dvec[g];
    A.dvec[g] = dn;
    A.y[g] = c + dn;
  } else {
    A.y[g] = c + (A.b[g] - acc) * wd;
  }
}

// A point of the cell's boundary (class cls != 0) that lies on a primitive of
// this cell only and is not a fixed Dirichlet value: the cell's partial
// stencil is the whole row of the operator.  The band row's plane-k,
// plane-(k+1) and plane-(k-1) rows j start at P0, Pp and Pm.
template <typename T, int OP>
__device__ __forceinline__ void stream_boundary_point(const FusedArgs<T>& A, int cell, int i,
                                                      int j, int k, int len, const T* P0,
                                                      const T* Pp, const T* Pm, int64_t g,
                                                      bool partial, bool owner) {
  const int n = A.n;
  const int cls = (i == len - 1 ? 1 : 0) | (i == 0 ? 2 : 0) | (j == 0 ? 4 : 0) | (k == 0 ? 8 : 0);
  const T c = P0[i];
  const T* S = A.sten + (int64_t)cell * 256 + cls * 16;
  T sv[kNDir], xv[kNDir];
#pragma unroll
  for (int d = 0; d < kNDir; ++d) {
    int di, dj, dk;
    dir_offset(d, di, dj, dk);
    sv[d] = __ldg(S + d);
    const int a = i + di, b = j + dj, cc = k + dk;
    const bool in = a >= 0 && b >= 0 && cc >= 0 && a + b + cc <= n;
    // row of the neighbour relative to row j of its plane
    const T* P = dk == 0 ? P0 : dk > 0 ? Pp : Pm;
    const int ro = dj == 0 ? 0 : dk == 0 ? (dj > 0 ? len : -(len + 1)) : dk > 0 ? -len : len + 1;
    xv[d] = in ? P[ro + a] : T(0);
  }
  const T acc = dot15<T>(sv, xv);
  if (partial) {
    // a point several cells share: this cell's partial sum, which the
    // interface pass (interface_sum_kernel) adds over the copies; an HG_ADD
    // apply keeps y in the owner's (first) copy
    A.y[g] = (OP == kOpApplyAdd && owner) ? A.y[g] + acc : acc;
    return;
  }
  const T wd = (OP == OP_JACOBI || OP == OP_CHEB) ? A.omega / sv[0] : OP == OP_GS ? T(1) / sv[0]
                                                                                  : T(0);
  stream_out<T, OP>(A, g, c, acc, wd);
}

// Wait until copy c of the CTA has landed in its slot: first until the
// producer has started copy c there (tag), then for the slot's barrier phase.
// The tag makes the phase parity unambiguous: warps work on different items,
// so one may want a slot a use or two ahead of the others.
__device__ __forceinline__ bool copy_wait(uint64_t* full, volatile int* tag, int c,
                                          volatile int* stop) {
  const int s = c % kStreamSlots;
  if (tag[s] != c) {
    const unsigned long long t0 = global_ns();
    for (long long it = 0; tag[s] != c; ++it) {
      if (it >= 8) __nanosleep(32);  // leave the issue slots to the computing warps
      if ((it & 63) == 63 && (*stop || global_ns() - t0 > kWaitNs)) return false;
      if (it > (1ll << 40)) return false;
    }
  }
  __threadfence_block();
  return mbar_wait(&full[s], (c / kStreamSlots) & 1, stop);
}

// One item in shared memory: the rows [ja, jb) of plane k; element g (cell
// offset) of plane k / k+1 / k-1 is at byte address vb0 / vbp / vbm + g * E.
// A plane that is not in the stream aliases plane k (only boundary points lie
// next to it, and they do not read it).
struct ItemView {
  int cell, k, ja, jb;
  uint32_t vb0, vbp, vbm;
};

// Interior points (j >= 1, k >= 1, 1 <= i <= len-2) of the item.  A warp
// takes 32 columns i at a time and marches the item's rows j: the values of
// row j (i-1, i, i+1) and of row j-1 (i, i+1) come from the previous step, so
// a step loads three values of row j+1 and two (seven-point) or six (15-point)
// of planes k+1 and k-1; row starts and shared addresses advance by warp-
// uniform amounts (row j+1 starts len elements after row j, len shrinks by 1).
// The boundary points are left to item_boundary.
template <typename T, int OP, int PAT>
__device__ __forceinline__ void item_interior(const FusedArgs<T>& A, const ItemView& V,
                                              const T s[kNDir], T wdc, int64_t base, int lane) {
  constexpr int E = (int)sizeof(T);
  const int w = A.w, k = V.k;
  if (k == 0) return;  // the plane k = 0 is a face of the cell
  const int Tk = ntri32(w - k), Tk1 = ntri32(w - k + 1);
  const int j1 = max(V.ja, 1);
  if (j1 >= V.jb) return;
  const int len1 = w - k - j1;
  const int rs1 = row_start(w, j1, k);
  for (int c0 = 1; c0 <= len1 - 2; c0 += 32) {
    const int i = c0 + lane;
    int len = len1, j = j1;
    uint32_t L = (uint32_t)(len * E);
    // element i of row j in planes k, k+1 (row j at offset T(w-k) - j from
    // plane k's row j) and k-1 (at -T(w-k+1) + j)
    uint32_t a0 = V.vb0 + (uint32_t)((rs1 + i) * E);
    uint32_t ap = V.vbp + (uint32_t)((rs1 + Tk - j1 + i) * E);
    uint32_t am = V.vbm + (uint32_t)((rs1 - Tk1 + j1 + i) * E);
    int64_t g = base + rs1 + i;
    // row j of plane k at i-1, i, i+1; row j-1 (starts len+1 earlier) at i, i+1
    T cm1 = HG_LDS(T, -1, a0), c0v = HG_LDS(T, 0, a0), cp1 = HG_LDS(T, 1, a0);
    T pm_i = HG_LDS(T, 0, a0 - L - E), pm_ip1 = HG_LDS(T, 1, a0 - L - E);
    // 15-point: plane k+1 row j-1 at i, i+1 (starts len before row j of k+1),
    // plane k-1 row j at i, i+1
    T up_i = T(0), up_ip1 = T(0), dn_i = T(0), dn_ip1 = T(0);
    if (PAT != kPat7) {
      up_i = HG_LDS(T, 0, ap - L);
      up_ip1 = HG_LDS(T, 1, ap - L);
      dn_i = HG_LDS(T, 0, am);
      dn_ip1 = HG_LDS(T, 1, am);
    }
#pragma unroll 4
    for (; j < V.jb && c0 <= len - 2; ++j) {
      // row j+1 of plane k (starts len after row j) at i-1, i, i+1
      const T nm1 = HG_LDS(T, -1, a0 + L), n0 = HG_LDS(T, 0, a0 + L), np1 = HG_LDS(T, 1, a0 + L);
      T acc;
      if (PAT == kPat7) {
        // (0,-1,+1): plane k+1 row j-1 at i; (0,+1,-1): plane k-1 row j+1 at i
        const T x11 = HG_LDS(T, 0, ap - L), x12 = HG_LDS(T, 1, am + L);
        acc = ((s[0] * c0v + s[1] * cp1) + (s[2] * cm1 + s[7] * nm1)) +
              ((s[8] * pm_ip1 + s[11] * x11) + s[12] * x12);
      } else {
        // plane k+1 row j at i-1, i, i+1; plane k-1 row j+1 at i-1, i, i+1
        const T q9 = HG_LDS(T, -1, ap), q5 = HG_LDS(T, 0, ap), qp = HG_LDS(T, 1, ap);
        const T r14 = HG_LDS(T, 0, am + L), r12 = HG_LDS(T, 1, am + L), rp = HG_LDS(T, 2, am + L);
        const T a0s = s[0] * c0v + s[1] * cp1 + s[2] * cm1 + s[3] * n0 + s[4] * pm_i +
                      s[7] * nm1 + s[8] * pm_ip1;
        const T a1 = s[5] * q5 + s[9] * q9 + s[11] * up_i + s[13] * up_ip1;
        const T a2 = s[6] * dn_i + s[10] * dn_ip1 + s[12] * r12 + s[14] * r14;
        acc = a0s + (a1 + a2);
        // next step: plane k+1 row j at i, i+1; plane k-1 row j+1 at i, i+1
        up_i = q5;
        up_ip1 = qp;
        dn_i = r12;
        dn_ip1 = rp;
      }
      if (i <= len - 2) stream_out<T, OP>(A, g, c0v, acc, wdc);
      // shift the rows: row j-1 <- row j, row j <- row j+1
      pm_i = c0v;
      pm_ip1 = cp1;
      cm1 = nm1;
      c0v = n0;
      cp1 = np1;
      g += len;
      a0 += L;
      ap += L - E;
      am += L + E;
      --len;
      L -= E;
    }
  }
}

// A boundary point (i, j) of the item's plane: a fixed Dirichlet value, or
// the cell's partial stencil sum: the whole row where the point has one copy,
// else a partial that the interface pass adds over the copies.
template <typename T, int OP>
__device__ __forceinline__ void item_boundary_point(const FusedArgs<T>& A, const ItemView& V,
                                                    ulonglong2 fw, int64_t base, int j, int rs,
                                                    int i) {
  constexpr int E = (int)sizeof(T);
  const int w = A.w, k = V.k, len = w - k - j;
  const int cls = (i == len - 1 ? 1 : 0) | (i == 0 ? 2 : 0) | (j == 0 ? 4 : 0) | (k == 0 ? 8 : 0);
  const unsigned f = (unsigned)((cls < 8 ? fw.x >> (8 * cls) : fw.y >> (8 * (cls - 8))) & 0xffu);
  const int64_t g = base + rs + i;
  if ((f & CF_DIRICHLET) && (!is_apply(OP) || A.mask == HG_MASK_INNER)) {
    A.y[g] = op_scaled(OP) ? HG_LDS(T, 0, V.vb0 + (uint32_t)((rs + i) * E)) : T(0);
  } else {
    const T* P0 = reinterpret_cast<const T*>(__cvta_shared_to_generic(V.vb0 + (uint32_t)(rs * E)));
    const T* Pp = reinterpret_cast<const T*>(
        __cvta_shared_to_generic(V.vbp + (uint32_t)((rs + ntri32(w - k) - j) * E)));
    const T* Pm = reinterpret_cast<const T*>(
        __cvta_shared_to_generic(V.vbm + (uint32_t)((rs - ntri32(w - k + 1) + j) * E)));
    stream_boundary_point<T, OP>(A, V.cell, i, j, k, len, P0, Pp, Pm, g, (f & CF_MULTI) != 0,
                                 (f & CF_OWNER) != 0);
  }
}

// The boundary points of the item: all of plane k = 0 and of row j = 0 (32
// points per step), and both ends of every other row (16 rows per step).
template <typename T, int OP>
__device__ __forceinline__ void item_boundary(const FusedArgs<T>& A, const ItemView& V,
                                              ulonglong2 fw, int64_t base, int lane) {
  const int w = A.w, k = V.k;
  int jfirst = V.ja;
  if (k == 0 || V.ja == 0) {
    const int jlast = k == 0 ? V.jb : V.ja + 1;  // whole rows: all of plane 0, else row 0
    int rs = row_start(w, V.ja, k);
    for (int j = V.ja; j < jlast; ++j) {
      const int len = w - k - j;
      for (int i = lane; i < len; i += 32) item_boundary_point<T, OP>(A, V, fw, base, j, rs, i);
      rs += len;
    }
    jfirst = jlast;
  }
  for (int j0 = jfirst; j0 < V.jb; j0 += 16) {
    // lane 2 m + e: end e of row j0 + m (a row of length 1 has one end)
    const int j = j0 + (lane >> 1), e = lane & 1;
    if (j < V.jb) {
      const int len = w - k - j;
      if (!(e && len == 1))
        item_boundary_point<T, OP>(A, V, fw, base, j, row_start(w, j, k), e ? len - 1 : 0);
    }
  }
}

template <typename T, int OP, int PAT>
__global__ void __launch_bounds__(sthreads<T>(), 1) p1_stream_kernel(
    const __grid_constant__ StreamArgs<T> S) {
  constexpr int kSWarps = swarps<T>();
  extern __shared__ __align__(128) unsigned char smem[];
  const FusedArgs<T>& A = S.f;
  constexpr int R = kStreamSlots;
  constexpr int SE = slot_elems<T>();
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + R;
  volatile int* stop = reinterpret_cast<volatile int*>(empty + R);
  volatile int* tag = stop + 4;  // tag[s]: the copy the producer last started in slot s
  T* ring = reinterpret_cast<T*>(smem + barrier_bytes()) + S.guard;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < R; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kStreamArrive);
      tag[s] = -1;
    }
    *stop = 0;
    mbar_init_fence();
  }
  __syncthreads();
  const int cb = S.plan.cta_copies[blockIdx.x], ce = S.plan.cta_copies[blockIdx.x + 1];
  const int ib = S.plan.cta_items[blockIdx.x], ie = S.plan.cta_items[blockIdx.x + 1];

  if (warp == kSWarps) {
    // ------------------------------------------------------------ producer
    if (lane != 0) return;
    int c = 0;
    bool ok = true;
    for (; c < ce - cb; ++c) {
      const int4 C = S.plan.copies[cb + c];
      const int s = c % R;
      if (c >= R && !mbar_wait(&empty[s], (c / R - 1) & 1, stop)) {
        ok = false;
        break;
      }
      const uint32_t bytes = (uint32_t)C.z * (uint32_t)sizeof(T);
      mbar_expect_tx(&full[s], bytes);
      bulk_g2s(ring + s * SE, A.x + (int64_t)C.x * A.stride + C.y, bytes, &full[s]);
      __threadfence_block();
      tag[s] = c;
    }
    if (!ok) {
      atomicCAS(A.err, 0, HG_ERR_TIMEOUT);
      *stop = 1;
    }
    // every copy issued must have landed before the CTA's memory is released
    for (int t = c > R ? c - R : 0; t < c; ++t) mbar_wait(&full[t % R], (t / R) & 1, nullptr);
    return;
  }

  // -------------------------------------------------------------- consumers
  // 1. the items of this CTA
  const uint32_t ring_addr = smem_addr(ring);
  int cur_cell = -1;
  T s[kNDir];
  T wdc = T(0);
  ulonglong2 fw = make_ulonglong2(0, 0);
  for (int t = ib + warp; t < ie; t += kSWarps) {
    const int4 I0 = S.plan.items[3 * t], I1 = S.plan.items[3 * t + 1], I2 = S.plan.items[3 * t + 2];
    ItemView V;
    V.cell = I0.x;
    V.k = I0.y;
    V.ja = I0.z & 0xffff;
    V.jb = I0.z >> 16;
    const int c0 = I1.x, cm = I1.y, cp = I1.z;
    bool ok = copy_wait(full, tag, c0, stop);
    if (cm >= 0 && cm != c0) ok = ok && copy_wait(full, tag, cm, stop);
    if (cp >= 0 && cp != c0 && cp != cm) ok = ok && copy_wait(full, tag, cp, stop);
    if (!ok) {
      if (lane == 0) {
        atomicCAS(A.err, 0, HG_ERR_TIMEOUT);
        *stop = 1;
      }
      return;
    }
    constexpr int E = (int)sizeof(T);
    const uint32_t tok = wait_token();
    // virtual bases (modulo 2^32: only base + g * E, inside the slot, is used)
    V.vb0 = ring_addr + tok + (uint32_t)((c0 % R) * SE * E) - (uint32_t)I2.x * (uint32_t)E;
    V.vbp = cp >= 0 ? ring_addr + tok + (uint32_t)((cp % R) * SE * E) - (uint32_t)I2.z * (uint32_t)E
                    : V.vb0;
    V.vbm = cm >= 0 ? ring_addr + tok + (uint32_t)((cm % R) * SE * E) - (uint32_t)I2.y * (uint32_t)E
                    : V.vb0;
    if (V.cell != cur_cell) {
      cur_cell = V.cell;
      const T* Sc = A.sten + (int64_t)cur_cell * 256;
#pragma unroll
      for (int d = 0; d < kNDir; ++d) s[d] = __ldg(Sc + d);
      wdc = (OP == OP_JACOBI || OP == OP_CHEB) ? A.omega / s[0] : OP == OP_GS ? T(1) / s[0] : T(0);
      fw = __ldg(reinterpret_cast<const ulonglong2*>(A.flags + cur_cell * 16));
    }
    const int64_t base = (int64_t)V.cell * A.stride;
    item_interior<T, OP, PAT>(A, V, s, wdc, base, lane);
    item_boundary<T, OP>(A, V, fw, base, lane);
    // release the copies this item read
    __syncwarp();
    if (lane == 0) {
      mbar_arrive_cnt(&empty[c0 % R], I0.w & 1023);
      if (cm >= 0 && cm != c0) mbar_arrive_cnt(&empty[cm % R], (I0.w >> 10) & 1023);
      if (cp >= 0 && cp != c0 && cp != cm) mbar_arrive_cnt(&empty[cp % R], (I0.w >> 20) & 1023);
    }
  }
}

// The operation's output at an interface point from the sum of the copies'
// partials (sum) and centre weights (diag), read at stored index g (every copy
// holds the same x, b and d).  OP_CHEB writes the new direction: to this copy,
// or (all == true) to every copy of the item's point with weights wts.
template <typename T, int OP>
__device__ __forceinline__ T interface_output(const FusedArgs<T>& A, int64_t g, T sum, T diag,
                                              bool all, int first_copy, int C, int dim,
                                              const int* wts) {
  if (OP == OP_APPLY || OP == kOpApplyAdd) return sum;
  if (OP == OP_RESID) return A.b[g] - sum;
  if (OP == OP_GS) return A.colour[g] == A.gs_colour ? A.x[g] + (A.b[g] - sum) / diag : A.x[g];
  if (OP == OP_CHEB) {
    T dn = A.omega * (A.b[g] - sum) / diag;
    if (A.cheb_a != T(0)) dn += A.cheb_a * A.dvec[g];
    if (all) {
      for (int q = 0; q < C; ++q) {
        const IfaceCopy cpy = A.copies[first_copy + q];
        int i, j, k;
        copy_local_ijk(cpy, dim, wts, i, j, k);
        A.dvec[(int64_t)cpy.cell * A.stride + tw32(A.w, i, j, k)] = dn;
      }
    } else {
      A.dvec[g] = dn;
    }
    return A.x[g] + dn;
  }
  return A.x[g] + A.omega * (A.b[g] - sum) / diag;
}

// The ghost-layer exchange (Sec. 2) after the streaming pass: every point of
// a macro face, edge or vertex shared by several cells holds, in each copy,
// that cell's partial sum; lane pt * C + c of an interface item reads copy c
// of point pt (its stored index precomputed per lane), the partials are added
// in ascending cell order (lane order), and every lane writes the operation's
// output to its copy, so copies stay bit-identical.  Primitives with more
// than 32 copies take one lane per point and derive the copies' indices.
template <typename T, int OP>
__global__ void __launch_bounds__(256) interface_sum_kernel(const __grid_constant__ FusedArgs<T> A,
                                                            const int2* __restrict__ lanes) {
  const int lane = threadIdx.x & 31;
  const int item = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (item >= A.n_items) return;
  const int4 it = A.items[item];
  const int dim = it.z & 15, C = (it.z >> 4) & 255;
  if (C > 32) {
    // one lane per point, the copies in turn
    if (lane >= it.w) return;
    const int n = A.n, w = A.w;
    int wts[3];
    prim_weights(dim, n, it.y + lane, wts);
    T sum = T(0), diag = T(0);
    int64_t g0 = 0;
    for (int q = 0; q < C; ++q) {
      const IfaceCopy cpy = A.copies[it.x + q];
      int i, j, k;
      copy_local_ijk(cpy, dim, wts, i, j, k);
      const int64_t g = (int64_t)cpy.cell * A.stride + tw32(w, i, j, k);
      if (q == 0) g0 = g;
      sum += A.y[g];
      if (op_scaled(OP)) diag += __ldg(A.sten + (int64_t)cpy.cell * 256 + point_class(n, i, j, k) * 16);
    }
    const T v = interface_output<T, OP>(A, g0, sum, diag, true, it.x, C, dim, wts);
    for (int q = 0; q < C; ++q) {
      const IfaceCopy cpy = A.copies[it.x + q];
      int i, j, k;
      copy_local_ijk(cpy, dim, wts, i, j, k);
      A.y[(int64_t)cpy.cell * A.stride + tw32(w, i, j, k)] = v;
    }
    return;
  }
  const int2 ln = __ldg(lanes + (int64_t)item * 32 + lane);
  const bool act = ln.x >= 0;
  const int64_t g = act ? ln.x : 0;
  const T mine = act ? A.y[g] : T(0);
  const T mdiag = op_scaled(OP) && act ? __ldg(A.sten + (int64_t)ln.y * 16) : T(0);
  // the point's C lanes (copy-major: lane = copy * P + point), ascending copy
  // (= cell) order
  const int P = 32 / C, pt = lane % P;
  T sum = T(0), diag = T(0);
  for (int q = 0; q < C; ++q) {
    sum += __shfl_sync(0xffffffffu, mine, (q * P + pt) & 31);
    if (op_scaled(OP)) diag += __shfl_sync(0xffffffffu, mdiag, (q * P + pt) & 31);
  }
  if (!act) return;
  A.y[g] = interface_output<T, OP>(A, g, sum, diag, false, 0, 0, 0, nullptr);
}

template <typename T, int OP, int PAT>
int run_stream(const LevelDev& L, const StencilArgs& a, cudaStream_t s) {
  StreamArgs<T> S;
  memset(&S, 0, sizeof S);
  FusedArgs<T>& A = S.f;
  A.n = L.n;
  A.w = L.w;
  A.stride = L.cell_stride;
  A.flags = L.cls_flags;
  A.items = L.mitems;
  A.n_items = (is_apply(OP) && a.mask == HG_MASK_ALL) ? L.n_mitems : L.n_mitems_inner;
  A.prims = L.prims;
  A.copies = L.copies;
  A.x = (const T*)a.x;
  A.b = (const T*)a.b;
  A.y = (T*)a.out;
  A.sten = (const T*)a.sten;
  A.omega = (T)a.omega;
  A.mode = a.mode;
  A.mask = a.mask;
  A.colour = L.colour;
  A.gs_colour = a.colour;
  A.dvec = (T*)a.dvec;
  A.cheb_a = (T)a.cheb_a;
  A.err = L.err;
  S.plan = L.splan[sizeof(T) == 8 ? HG_F64 : HG_F32];
  S.guard = guard_elems(L.w);
  const size_t smem =
      barrier_bytes() + (size_t)(2 * S.guard + kStreamSlots * slot_elems<T>()) * sizeof(T);
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [] {
    attr_err = cudaFuncSetAttribute(p1_stream_kernel<T, OP, PAT>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  });
  HG_CUDA(attr_err);
  if (smem > 227 * 1024) {
    set_error("streaming kernel: %zu bytes of shared memory at w = %d", smem, L.w);
    return HG_ERR_UNSUPPORTED;
  }
  p1_stream_kernel<T, OP, PAT><<<S.plan.nctas, sthreads<T>(), smem, s>>>(S);
  HG_CUDA(cudaGetLastError());
  if (A.n_items > 0) {
    interface_sum_kernel<T, OP><<<(A.n_items + 7) / 8, 256, 0, s>>>(A, L.mlanes);
    HG_CUDA(cudaGetLastError());
  }
  return HG_OK;
}

template <typename T, int PAT>
int run_stream_op(const LevelDev& L, const StencilArgs& a, cudaStream_t s) {
  switch (a.op) {
    case OP_APPLY:
      return a.mode == HG_ADD ? run_stream<T, kOpApplyAdd, PAT>(L, a, s)
                              : run_stream<T, OP_APPLY, PAT>(L, a, s);
    case OP_RESID: return run_stream<T, OP_RESID, PAT>(L, a, s);
    case OP_JACOBI: return run_stream<T, OP_JACOBI, PAT>(L, a, s);
    case OP_GS: return run_stream<T, OP_GS, PAT>(L, a, s);
    case OP_CHEB: return run_stream<T, OP_CHEB, PAT>(L, a, s);
  }
  set_error("unknown cell operation %d", a.op);
  return HG_ERR_INVALID_ARG;
}

}  // namespace

bool p1_stream_fits(int w, int dtype) {
  const size_t e = dtype == HG_F64 ? 8 : 4;
  return barrier_bytes() + (2 * guard_elems(w)) * e + (size_t)kStreamSlots * kStreamSlotBytes <=
         227 * 1024;
}

int launch_p1_stream(const LevelDev& L, int dtype, const StencilArgs& a, cudaStream_t s) {
  if (a.pattern == kPat7)
    return dtype == HG_F64 ? run_stream_op<double, kPat7>(L, a, s)
                           : run_stream_op<float, kPat7>(L, a, s);
  return dtype == HG_F64 ? run_stream_op<double, 0>(L, a, s) : run_stream_op<float, 0>(L, a, s);
}

}  // namespace hg

extern "C" int hg_stream_layout(int level, int dtype, int* ring_slots, int* slot_elems,
                                int* guard_elems) {
  if (level < 0 || level > 12 || (dtype != HG_F32 && dtype != HG_F64) || !ring_slots ||
      !slot_elems || !guard_elems) {
    hg::set_error("hg_stream_layout: bad argument");
    return HG_ERR_INVALID_ARG;
  }
  const int w = (1 << level) + 1;
  *ring_slots = hg::kStreamSlots;
  *slot_elems = dtype == HG_F64 ? hg::slot_elems<double>() : hg::slot_elems<float>();
  *guard_elems = hg::guard_elems(w);
  return HG_OK;
}
