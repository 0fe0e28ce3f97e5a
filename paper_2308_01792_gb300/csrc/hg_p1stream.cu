// P1 constant-stencil operator application as a streaming kernel
// (Sec. 5.2 apply(), stencil-based pattern, one stencil per macro cell).
//
// A macro cell's lattice is stored plane by plane (k), row by row (j), with
// unit-stride x-lines (i) (the t_w order of Sec. 4).  The rows j0 .. j0+7 of
// one plane ("a band") are one contiguous offset range, and so are the rows
// j0-1 .. j0+8 that the 15-point stencil of the band reads in planes k-1, k
// and k+1.  The kernel marches bands plane by plane:
//
//  * one CTA per SM, a producer warp and kSWarps consumer warps;
//  * the producer copies the staged rows of every plane of its runs into a
//    ring of shared-memory slots with 1-D bulk copies (cp.async.bulk, the
//    TMA engine), one copy per plane, completion counted on the slot's
//    mbarrier; it runs up to R slots ahead of the consumers, so tens of KB
//    per SM are in flight from HBM at any time;
//  * the consumers compute a plane of the band once the slots of planes k-1,
//    k, k+1 have landed, the 32-point chunks of the band's rows going
//    round-robin over the warps (all addressing warp-uniform per row; the
//    round-robin continues across planes, so short planes near the top of a
//    band spread over the warps too), write the results to HBM directly, and
//    release the slot of plane k-1; a slot is thus read for three
//    consecutive planes and every x value crosses HBM once;
//  * points of the cell's boundary that lie on a primitive of this cell only
//    (boundary faces, edges and vertices) are formed in the same pass from
//    the cell's partial stencil; points shared by several cells (the
//    ghost-layer exchange of Sec. 2) are formed by the interface items, a
//    contiguous share per CTA that its consumer warps take after their runs
//    (the producer prefetches the share's item records into L2 at the start).
//
// Every wait on an mbarrier is bounded (about one second): on expiry the
// kernel records HG_ERR_TIMEOUT in the hierarchy's error word, the other
// warps stop at their next wait, and the producer waits (again bounded) for
// the copies it issued before the CTA exits.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "hg_internal.h"
#include "hg_p1dev.cuh"

namespace hg {
namespace {

constexpr int kSWarps = 16;                    // consumer warps
constexpr int kSThreads = (kSWarps + 1) * 32;  // and one producer warp
constexpr int kRingBytes = 160 * 1024;         // shared memory for the slot ring
constexpr unsigned long long kWaitNs = 1000000000ull;

template <typename T>
__host__ __device__ constexpr int vec_elems() { return 16 / (int)sizeof(T); }

// HG_ADD applies get their own instantiation (y += A x) so that a replacing
// apply never reads the destination.
constexpr int kOpApplyAdd = 100;
__host__ __device__ constexpr bool is_apply(int op) { return op == OP_APPLY || op == kOpApplyAdd; }

// Elements of one slot: kStreamBand + 2 rows of at most w points plus the
// 16-byte rounding of both ends, in whole 128-byte lines.
inline int slot_elems(int w) { return ((kStreamBand + 2) * w + 8 + 31) / 32 * 32; }
// Elements before the first and after the last slot: the unconditional
// shared-memory loads of lanes past a row's end or next to a band's edge reach
// at most w + 2 elements before a slot's data and 2 w + 33 after it.
inline int guard_elems(int w) { return (4 * w + 64 + 31) / 32 * 32; }
template <typename T>
int ring_slots(int w) {
  const int r = kRingBytes / (slot_elems(w) * (int)sizeof(T));
  return r < 4 ? 4 : r > 32 ? 32 : r;
}
__host__ __device__ inline int barrier_bytes(int R) { return (2 * R * 8 + 16 + 127) / 128 * 128; }

template <typename T>
struct StreamArgs {
  FusedArgs<T> f;             // operands, stencils, flags and the interface items
  const int4* units;          // runs (cell, j0 | rows << 16, k0 | k1 << 16, 0)
  const int32_t* cta_begin;
  int R;                      // ring slots
  int slot;                   // elements per slot
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
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(b)), "r"(parity)
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
// Bulk prefetch of [p, p + bytes) into L2 (16-byte aligned, size a multiple of 16).
__device__ __forceinline__ void l2_prefetch(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
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

// Offsets [ga, ge) (16-byte aligned) of the rows staged for plane kk of the
// band j0 .. j0+rows-1: rows max(j0-1, 0) .. min(j0+rows, w-1-kk).
template <typename T>
__device__ __forceinline__ void staged_range(int w, int j0, int rows, int kk, int& ga, int& ge) {
  constexpr int V = vec_elems<T>();
  const int jlo = max(j0 - 1, 0), jhi = min(j0 + rows, w - 1 - kk);
  const int g0 = row_start(w, jlo, kk);
  const int g1 = row_start(w, jhi, kk) + (w - kk - jhi);
  ga = g0 & ~(V - 1);
  ge = (g1 + V - 1) & ~(V - 1);
}

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

// A point of the cell's boundary (class cls != 0) of the band row whose
// plane-k, plane-(k+1) and plane-(k-1) rows j start at P0, Pp and Pm.
template <typename T, int OP>
__device__ __noinline__ void stream_boundary_point(const FusedArgs<T>& A, int cell, int i, int j,
                                                   int k, int len, const T* P0, const T* Pp,
                                                   const T* Pm, int64_t g) {
  const int n = A.n;
  const int cls = (i == len - 1 ? 1 : 0) | (i == 0 ? 2 : 0) | (j == 0 ? 4 : 0) | (k == 0 ? 8 : 0);
  const uint8_t f = __ldg(A.flags + cell * 16 + cls);
  const T c = P0[i];
  if ((f & CF_DIRICHLET) && (!is_apply(OP) || A.mask == HG_MASK_INNER)) {
    A.y[g] = op_scaled(OP) ? c : T(0);
    return;
  }
  if (f & CF_MULTI) return;  // a sum over cells: the interface items form it
  // single copy: this cell's partial stencil is the whole row of the operator
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
  const T wd = (OP == OP_JACOBI || OP == OP_CHEB) ? A.omega / sv[0] : OP == OP_GS ? T(1) / sv[0]
                                                                                  : T(0);
  stream_out<T, OP>(A, g, c, acc, wd);
}

template <typename T, int OP, int PAT>
__global__ void __launch_bounds__(kSThreads, 1) p1_stream_kernel(const StreamArgs<T> S) {
  extern __shared__ __align__(128) unsigned char smem[];
  const FusedArgs<T>& A = S.f;
  const int R = S.R;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + R;
  volatile int* stop = reinterpret_cast<volatile int*>(empty + R);
  T* ring = reinterpret_cast<T*>(smem + barrier_bytes(R)) + S.guard;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < R; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kSWarps);
    }
    *stop = 0;
    mbar_init_fence();
  }
  __syncthreads();
  const int w = A.w;
  const int ub = S.cta_begin[blockIdx.x], ue = S.cta_begin[blockIdx.x + 1];

  if (warp == kSWarps) {
    // ------------------------------------------------------------ producer
    if (lane != 0) return;
    {
      // the interface items of this CTA (read after its runs) into L2
      const int ib = (int)((int64_t)A.n_items * blockIdx.x / gridDim.x);
      const int ie = (int)((int64_t)A.n_items * (blockIdx.x + 1) / gridDim.x);
      if (ie > ib) l2_prefetch(A.items + ib, (uint32_t)(ie - ib) * (uint32_t)sizeof(int4));
    }
    int q = 0;
    bool ok = true;
    for (int u = ub; u < ue && ok; ++u) {
      const int4 U = S.units[u];
      const int cell = U.x, j0 = U.y & 0xffff, rows = U.y >> 16;
      const int k0 = U.z & 0xffff, k1 = U.z >> 16;
      const int kf = max(k0 - 1, 0), kl = min(k1, w - 1);
      const T* xc = A.x + (int64_t)cell * A.stride;
      for (int kk = kf; kk <= kl; ++kk) {
        const int s = q % R, m = q / R;
        if (m > 0 && !mbar_wait(&empty[s], (m - 1) & 1, stop)) {
          ok = false;
          break;
        }
        int ga, ge;
        staged_range<T>(w, j0, rows, kk, ga, ge);
        const uint32_t bytes = (uint32_t)(ge - ga) * (uint32_t)sizeof(T);
        mbar_expect_tx(&full[s], bytes);
        bulk_g2s(ring + s * S.slot, xc + ga, bytes, &full[s]);
        ++q;
      }
    }
    if (!ok) {
      atomicCAS(A.err, 0, HG_ERR_TIMEOUT);
      *stop = 1;
    }
    // every copy issued must have landed before the CTA's memory is released
    for (int t = q > R ? q - R : 0; t < q; ++t) mbar_wait(&full[t % R], (t / R) & 1, nullptr);
    return;
  }

  // -------------------------------------------------------------- consumers
  // 1. the runs of this CTA; their chunks go round-robin over the warps
  int q = 0, cbase = 0;
  for (int u = ub; u < ue; ++u) {
    const int4 U = S.units[u];
    const int cell = U.x, j0 = U.y & 0xffff, rows = U.y >> 16;
    const int k0 = U.z & 0xffff, k1 = U.z >> 16;
    const int kf = max(k0 - 1, 0), kl = min(k1, w - 1);
    const int64_t base = (int64_t)cell * A.stride;
    T s[kNDir];
    {
      const T* Sc = A.sten + (int64_t)cell * 256;
#pragma unroll
      for (int d = 0; d < kNDir; ++d) s[d] = __ldg(Sc + d);
    }
    const T wdc = (OP == OP_JACOBI || OP == OP_CHEB) ? A.omega / s[0]
                  : OP == OP_GS                      ? T(1) / s[0]
                                                     : T(0);
    for (int k = k0; k < k1; ++k) {
      const int qk = q + (k - kf);
      bool ok = true;
      if (k == k0) {
        if (k > kf) ok = mbar_wait(&full[(qk - 1) % R], ((qk - 1) / R) & 1, stop);
        ok = ok && mbar_wait(&full[qk % R], (qk / R) & 1, stop);
      }
      if (k < kl) ok = ok && mbar_wait(&full[(qk + 1) % R], ((qk + 1) / R) & 1, stop);
      if (!ok) {
        if (lane == 0) {
          atomicCAS(A.err, 0, HG_ERR_TIMEOUT);
          *stop = 1;
        }
        return;
      }
      int ga0, gam, gap, ge;
      staged_range<T>(w, j0, rows, k, ga0, ge);
      const T* s0 = ring + (qk % R) * S.slot;
      const T* sm = s0;
      const T* sp = s0;
      if (k > kf) {
        staged_range<T>(w, j0, rows, k - 1, gam, ge);
        sm = ring + ((qk - 1) % R) * S.slot;
      }
      if (k < kl) {
        staged_range<T>(w, j0, rows, k + 1, gap, ge);
        sp = ring + ((qk + 1) % R) * S.slot;
      }
      // 32-point chunks of the band's rows in this plane, continuing the
      // round-robin over the warps from the previous plane
      const int jn = min(rows, w - k - j0);
      int it = (warp - cbase % kSWarps + kSWarps) % kSWarps, cb = 0;
      for (int r = 0; r < jn; ++r) {
        const int j = j0 + r, len = w - k - j;
        const int nch = (len + 31) >> 5;
        if (it < cb + nch) {
          const int rs0 = row_start(w, j, k);
          const T* P0 = s0 + (rs0 - ga0);
          const T* Pp = k < kl ? sp + (rs0 + ntri32(w - k) - j - gap) : P0;
          const T* Pm = k > kf ? sm + (rs0 - ntri32(w - k + 1) + j - gam) : P0;
          const bool jk_in = j >= 1 && k >= 1;
          do {
            const int i = (it - cb) * 32 + lane;
            // the 15 neighbours; rows j-1 / j+1 of plane k start at -(len+1) / +len,
            // row j-1 of plane k+1 at -len, row j+1 of plane k-1 at +len+1
            const T c = P0[i];
            const T x1 = P0[i + 1], x2 = P0[i - 1];
            const T x7 = P0[len + i - 1], x8 = P0[i - len];
            const T x11 = Pp[i - len], x12 = Pm[len + 1 + i];
            T acc;
            if (PAT == kPat7) {
              const T a0 = s[0] * c + s[1] * x1 + s[2] * x2 + s[7] * x7 + s[8] * x8;
              acc = a0 + (s[11] * x11 + s[12] * x12);
            } else {
              const T x3 = P0[len + i], x4 = P0[i - len - 1];
              const T x5 = Pp[i], x6 = Pm[i];
              const T x9 = Pp[i - 1], x10 = Pm[i + 1];
              const T x13 = Pp[i - len + 1], x14 = Pm[len + i];
              const T a0 = s[0] * c + s[1] * x1 + s[2] * x2 + s[3] * x3 + s[4] * x4 + s[7] * x7 +
                           s[8] * x8;
              const T a1 = s[5] * x5 + s[9] * x9 + s[11] * x11 + s[13] * x13;
              const T a2 = s[6] * x6 + s[10] * x10 + s[12] * x12 + s[14] * x14;
              acc = a0 + (a1 + a2);
            }
            if (jk_in && i >= 1 && i <= len - 2)
              stream_out<T, OP>(A, base + rs0 + i, c, acc, wdc);
            else if (i < len)
              stream_boundary_point<T, OP>(A, cell, i, j, k, len, P0, Pp, Pm, base + rs0 + i);
            it += kSWarps;
          } while (it < cb + nch);
        }
        cb += nch;
      }
      cbase += cb;
      // release the slots no later plane of this run reads
      __syncwarp();
      if (lane == 0) {
        if (k > kf) mbar_arrive(&empty[(qk - 1) % R]);
        if (k == k1 - 1) {
          mbar_arrive(&empty[qk % R]);
          if (k < kl) mbar_arrive(&empty[(qk + 1) % R]);
        }
      }
    }
    q += kl - kf + 1;
  }

  // 2. points shared by several cells (interface items): a contiguous share
  //    per CTA, after the runs, when most of x has passed through L2
  const int ib = (int)((int64_t)A.n_items * blockIdx.x / gridDim.x);
  const int ie = (int)((int64_t)A.n_items * (blockIdx.x + 1) / gridDim.x);
  for (int it = ib + warp; it < ie; it += kSWarps)
    interface_item<T, is_apply(OP) ? OP_APPLY : OP, false>(A, it, lane);
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
  S.units = L.sunits;
  S.cta_begin = L.scta;
  S.R = ring_slots<T>(L.w);
  S.slot = slot_elems(L.w);
  S.guard = guard_elems(L.w);
  const size_t smem = barrier_bytes(S.R) + (size_t)(2 * S.guard + S.R * S.slot) * sizeof(T);
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
  p1_stream_kernel<T, OP, PAT><<<L.n_scta, kSThreads, smem, s>>>(S);
  HG_CUDA(cudaGetLastError());
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
  *ring_slots = dtype == HG_F64 ? hg::ring_slots<double>(w) : hg::ring_slots<float>(w);
  *slot_elems = hg::slot_elems(w);
  *guard_elems = hg::guard_elems(w);
  return HG_OK;
}
