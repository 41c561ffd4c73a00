// rk4_tile.cuh -- temporal blocking of one tile (Sec. 2.3 of the paper, on the GPU).
//
// A thread block owns a tile of W = blockDim.x * V consecutive sites of one chain: the G
// interior sites it will write back plus a halo of H = 4k sites on each side.  Thread t holds
// sites t*V .. t*V+V-1 in registers.  Every RK stage needs the coupling coordinate of both
// neighbours: inside a thread it is a register, across threads an exchange through shared
// memory (one __syncthreads per stage; see tile_advance).  Sites at the tile's
// ends read a stand-in value, so after m stages only sites [m, W - m) are exact -- the
// paper's observation that the error from the missing coupling moves one site inward per
// stage -- and after 4k stages exactly the interior [4k, W - 4k) is.
//
// Fixed ends: sites of the tile outside the chain are ghosts whose coupling coordinate is
// forced to zero at every stage (r_0 = r_{N+1} = 0).  Periodic ends: the tile is a window of
// the periodically extended chain (indices taken mod N), so no special case is needed.
#pragma once
#include <type_traits>

#include "rk4_device.cuh"
#include "rk4_internal.h"

namespace rk4d {

constexpr unsigned kFull = 0xffffffffu;

// Index checks of a debug build (-DRK4_DEBUG_BOUNDS): a range that would leave its buffer
// latches ST_BOUNDS in the status word and the access is skipped.  In a release build the
// check is the constant true and costs nothing.
__device__ __forceinline__ bool bounds_ok(WsHeader *hdr, bool ok) {
#ifdef RK4_DEBUG_BOUNDS
  if (!ok && hdr) atomicOr(&hdr->status, ST_BOUNDS);
  return ok;
#else
  (void)hdr;
  (void)ok;
  return true;
#endif
}

// Whether [first, first + count) lies inside [0, size).
__device__ __forceinline__ bool in_range(int64_t first, int64_t count, int64_t size) {
  return first >= 0 && count >= 0 && first + count <= size;
}

// NaN or infinity, tested on the exponent bits with integer instructions: a floating-point
// compare would take issue slots of the FP64 pipe, which bounds the FP64 kernels.
__device__ __forceinline__ bool nonfinite(double x) {
  return (__double2hiint(x) & 0x7ff00000) == 0x7ff00000;
}
__device__ __forceinline__ bool nonfinite(float x) {
  return (__float_as_uint(x) & 0x7f800000u) == 0x7f800000u;
}

// Latch ST_NONFINITE when any value of a result about to be stored is NaN or infinite (one
// thread per block reports; `any` is the block-wide vote).
__device__ __forceinline__ void report_nonfinite(WsHeader *hdr, int any) {
  if (any && threadIdx.x == 0 && hdr) atomicOr(&hdr->status, ST_NONFINITE);
}

// Largest block the tile kernels are compiled for, by sites per thread: the register budget
// (about 9 values per site plus temporaries) must fit 65536 registers per block.
__host__ __device__ constexpr int max_threads_for(int v) { return v <= 1 ? 1024 : (v <= 4 ? 512 : 256); }

// Neighbour exchange of the tile kernels, by sites per thread: with 4 or more, every thread
// publishes its end values in shared memory (fewer MIO instructions, measured +4-8 % in FP32
// and +2 % in heterogeneous FP64); with fewer, warp shuffles plus warp-edge slots (the
// per-thread slots' four address registers cost 6-12 more registers there, which drops a
// resident block: -12 to -18 %).
__host__ __device__ constexpr bool thread_exchange(int v) { return v >= 4; }
// Shared-memory values the exchange takes at the front of a tile kernel's dynamic shared memory.
__host__ __device__ constexpr int edge_values(int v) { return thread_exchange(v) ? 4 * max_threads_for(v) : 128; }

// Store v to shared memory only when p holds, as a predicated instruction (no divergent
// branch around it).
__device__ __forceinline__ void st_shared_if(bool p, float *a, float v) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(a));
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\t@q st.shared.f32 [%0], %1;\n\t}" ::"r"(s), "f"(v),
               "r"(static_cast<int>(p))
               : "memory");
}
__device__ __forceinline__ void st_shared_if(bool p, double *a, double v) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(a));
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\t@q st.shared.f64 [%0], %1;\n\t}" ::"r"(s), "d"(v),
               "r"(static_cast<int>(p))
               : "memory");
}

// Shared-memory accesses through 32-bit shared-window addresses (four such registers per
// thread carry the neighbour exchange below; generic pointers would take twice as many).
__device__ __forceinline__ unsigned smem_addr(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void st_shared(unsigned a, float v) {
  asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}
__device__ __forceinline__ void st_shared(unsigned a, double v) {
  asm volatile("st.shared.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory");
}
__device__ __forceinline__ void ld_shared(unsigned a, float &v) {
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
}
__device__ __forceinline__ void ld_shared(unsigned a, double &v) {
  asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"(a) : "memory");
}

// Synchronise this warp with its two neighbouring warps only, for a neighbour exchange in
// which each thread reads the slots of the threads just before and after it: one named barrier
// per pair of adjacent warps (ids 1 .. 15, 64 threads each; id 0 is __syncthreads), so a warp
// waits for its neighbours rather than for the slowest warp of the block.  Warp w takes the
// barrier it shares with w - 1 and then the one it shares with w + 1; the chain starting at
// warp 0 (which has no left barrier) completes every pair, so no warp waits forever.  The
// barriers also order the shared-memory accesses of the threads of each warp.  Needs a block of
// at most 16 warps (512 threads), every thread of a warp taking part.
__device__ __forceinline__ void neighbour_warp_sync() {
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (nw > 16) {  // more pairs than named barriers: the whole block instead (block-uniform)
    __syncthreads();
    return;
  }
  if (nw == 1) {
    __syncwarp();
    return;
  }
  if (w > 0) asm volatile("bar.sync %0, 64;" ::"r"(w) : "memory");
  if (w < nw - 1) asm volatile("bar.sync %0, 64;" ::"r"(w + 1) : "memory");
}

// The barrier of a tile kernel's neighbour exchange, where each thread (warp) reads only the
// slots of its neighbours: FP64 waits for the neighbouring warps only (neighbour_warp_sync,
// measured 7 % faster: the warps of a block no longer enter each stage's FP64 stream in lock
// step); FP32 keeps the one block-wide barrier per stage (the two named barriers measured 16-28 %
// slower there).
template <typename R> __device__ __forceinline__ void stage_sync() {
  if constexpr (sizeof(R) == 8) neighbour_warp_sync(); else __syncthreads();
}

// Advance the registers of one tile by K steps.  `edge` is edge_values(V) values of shared
// memory, two alternating slots by stage parity.  Per-thread exchange (thread_exchange(V)): a
// slot is [first x of each thread | last x of each thread], strided by the compile-time
// largest block so that the per-stage offsets are immediates; every thread stores its two
// coupling coordinates and, after the stage's one barrier, loads its neighbours'
// (conflict-free: consecutive threads, consecutive addresses), four shared-memory
// instructions per warp and stage.  Warp exchange: a slot is [first x of each warp | last x
// of each warp]; shuffles carry the values inside a warp and lanes 0 and 31 publish theirs by
// predicated stores, read back as uniform (broadcast) loads and selects.  Either way the two
// tile ends read a stand-in (their own value), which only ever reaches halo sites.  Stage 0
// of every step reads y directly (it is the stage state), so no register copies are needed
// between steps.
template <typename R, int MODEL, int V, bool KAHAN, bool MASK, bool HET = false>
__device__ __forceinline__ void tile_advance(R (&y)[V][Dim<MODEL>::D], R (&cmp)[V][Dim<MODEL>::D],
                                             uint32_t ghost, int K, const Coef<R> &cf, R *edge,
                                             const Coef<R> *cs = nullptr) {
  constexpr int D = Dim<MODEL>::D;
  constexpr bool kThread = thread_exchange(V);
  constexpr int NT = max_threads_for(V);
  const int tid = threadIdx.x;
  // per-thread exchange: this thread's slots (parity 0) and its neighbours' (unused and
  // never computed by the warp exchange)
  unsigned my_first = 0, my_last = 0, left_last = 0, right_first = 0;
  if constexpr (kThread) {
    my_first = smem_addr(edge + tid);
    my_last = smem_addr(edge + NT + tid);
    left_last = my_last - (tid > 0 ? (unsigned)sizeof(R) : 0u);
    right_first = my_first + (tid < (int)blockDim.x - 1 ? (unsigned)sizeof(R) : 0u);
  }
  // warp exchange
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int nw = blockDim.x >> 5;
  const bool is_first = lane == 0, is_last = lane == 31;
  const int prev = (warp > 0) ? warp - 1 : warp;
  const int next = (warp < nw - 1) ? warp + 1 : warp;
  R u[V][D], acc[V][D];
  // FP32-Kahan tiles with an even number of sites per thread run on packed instructions
  constexpr bool kPacked = std::is_same<R, float>::value && KAHAN && (V % 2 == 0);

#pragma unroll 2  // halves the loop-carried register moves (measured +4 % in FP32)
  for (int s = 0; s < K; ++s) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      R xs[V];
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const R x = (j == 0) ? y[v][0] : u[v][0];
        xs[v] = (MASK && ((ghost >> v) & 1u)) ? R(0) : x;
      }
      R left, right;
      if constexpr (kThread) {
        const unsigned po = (j & 1) * 2 * NT * (unsigned)sizeof(R);  // the stage's parity slot
        st_shared(my_first + po, xs[0]);
        st_shared(my_last + po, xs[V - 1]);
        stage_sync<R>();
        ld_shared(left_last + po, left);
        ld_shared(right_first + po, right);
      } else {
        left = __shfl_up_sync(kFull, xs[V - 1], 1);
        right = __shfl_down_sync(kFull, xs[0], 1);
        R *eb = edge + (j & 1) * 64;  // [0,32): first x of each warp, [32,64): last x
        st_shared_if(is_first, eb + warp, xs[0]);
        st_shared_if(is_last, eb + 32 + warp, xs[V - 1]);
        stage_sync<R>();
        const R from_prev = eb[32 + prev];
        const R from_next = eb[next];
        left = is_first ? from_prev : left;
        right = is_last ? from_next : right;
      }
      if constexpr (kPacked) {
        // sites v and v + 1 in the two halves of packed FP32 instructions
#pragma unroll
        for (int v = 0; v < V; v += 2) {
          const float2 xl = make_float2((v == 0) ? left : xs[v - 1], xs[v]);
          const float2 xr = make_float2(xs[v + 1], (v + 2 == V) ? right : xs[v + 2]);
          float2 yy[D], uu[D], ac[D], cm[D], k[D];
#pragma unroll
          for (int d = 0; d < D; ++d) {
            yy[d] = make_float2(y[v][d], y[v + 1][d]);
            uu[d] = (j == 0) ? yy[d] : make_float2(u[v][d], u[v + 1][d]);
            ac[d] = make_float2(acc[v][d], acc[v + 1][d]);
            cm[d] = make_float2(cmp[v][d], cmp[v + 1][d]);
          }
          const Coef2 c2 = HET ? pair_coef(cs[v], cs[v + 1]) : pair_coef(cf, cf);
          slope2<MODEL>(uu, xl, xr, c2, k);
          stage_update2<D>(j, k, yy, uu, ac, cm, c2);
#pragma unroll
          for (int d = 0; d < D; ++d) {
            y[v][d] = yy[d].x;
            y[v + 1][d] = yy[d].y;
            u[v][d] = uu[d].x;
            u[v + 1][d] = uu[d].y;
            acc[v][d] = ac[d].x;
            acc[v + 1][d] = ac[d].y;
            cmp[v][d] = cm[d].x;
            cmp[v + 1][d] = cm[d].y;
          }
        }
      } else {
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const R xl = (v == 0) ? left : xs[v - 1];
          const R xr = (v == V - 1) ? right : xs[v + 1];
          R k[D];
          if constexpr (HET)
            slope<R, MODEL>((j == 0) ? y[v] : u[v], xl, xr, cs[v], k);  // site-dependent f_i, g_i (Eq. (1))
          else
            slope<R, MODEL>((j == 0) ? y[v] : u[v], xl, xr, cf, k);
          stage_update<R, D, KAHAN>(j, k, y[v], u[v], acc[v], cmp[v], cf);
        }
      }
    }
  }
}

// Global loads: the read-only path for one-shot launches; L2-coherent loads (bypassing L1)
// inside the persistent kernel, whose buffers are rewritten by other blocks between barriers.
template <bool COH, typename T> __device__ __forceinline__ T gld(const T *p) {
  if constexpr (COH) return __ldcg(p); else return __ldg(p);
}

// Block-cooperative copies of `count` values between global and shared memory, two forms.
//
// copy_in_vec / copy_out_vec access global memory by 16-byte vectors wherever whole vectors
// lie inside the range, whatever the range's alignment: when the shared-memory side sits at the
// same 16-byte offset it is accessed by vectors too, otherwise each vector's values move to or
// from shared memory singly.  A vector that would reach past either end of the range is
// replaced by single accesses, so nothing outside the range is read or written.  The persistent
// kernel uses this form: its blocks load tiles in lock step after every grid barrier, and batch
// chains start anywhere, so single loads of misaligned windows sat on its critical path
// (measured 8 % faster with vectors).
//
// copy_in / copy_out move whole 16-byte vectors when both sides are aligned and the size is a
// multiple of 16 bytes (every tile of a single chain), single values otherwise.  In the one-shot
// tile kernels, whose loads overlap other blocks' arithmetic, this shorter code measured faster
// for single chains (4 %) and for batches alike (4 %, against copy_in_vec on the same batch).
template <bool COH, typename R>
__device__ __forceinline__ void copy_in(R *dst, const R *__restrict__ src, int count) {
  if ((reinterpret_cast<uintptr_t>(src) & 15u) == 0 && (reinterpret_cast<uintptr_t>(dst) & 15u) == 0 &&
      ((count * (int)sizeof(R)) & 15) == 0) {
    const int nv = count * (int)sizeof(R) / 16;
    const int4 *s4 = reinterpret_cast<const int4 *>(src);
    int4 *d4 = reinterpret_cast<int4 *>(dst);
    for (int e = threadIdx.x; e < nv; e += blockDim.x) d4[e] = gld<COH>(s4 + e);
  } else {
    for (int e = threadIdx.x; e < count; e += blockDim.x) dst[e] = gld<COH>(src + e);
  }
}
template <typename R>
__device__ __forceinline__ void copy_out(R *__restrict__ dst, const R *src, int count) {
  if ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0 && (reinterpret_cast<uintptr_t>(src) & 15u) == 0 &&
      ((count * (int)sizeof(R)) & 15) == 0) {
    const int nv = count * (int)sizeof(R) / 16;
    int4 *d4 = reinterpret_cast<int4 *>(dst);
    const int4 *s4 = reinterpret_cast<const int4 *>(src);
    for (int e = threadIdx.x; e < nv; e += blockDim.x) d4[e] = s4[e];
  } else {
    for (int e = threadIdx.x; e < count; e += blockDim.x) dst[e] = src[e];
  }
}
// copy_out for a range whose shared-memory side sits at the same 16-byte offset as its global
// side (the interior of a batch tile whose window starts on a 16-byte boundary): the values
// before the first and after the last whole vector singly, the rest by 16-byte vectors on both
// sides.  Any other range is copied singly.
template <typename R>
__device__ __forceinline__ void copy_out_matched(R *__restrict__ dst, const R *src, int count) {
  constexpr int kPer = 16 / (int)sizeof(R);
  const unsigned md = (unsigned)(reinterpret_cast<uintptr_t>(dst) & 15u);
  if (md != (unsigned)(reinterpret_cast<uintptr_t>(src) & 15u)) {
    for (int e = threadIdx.x; e < count; e += blockDim.x) dst[e] = src[e];
    return;
  }
  int head = (int)(((16u - md) & 15u) / sizeof(R));
  if (head > count) head = count;
  const int nv = (count - head) / kPer;
  for (int e = threadIdx.x; e < head; e += blockDim.x) dst[e] = src[e];
  int4 *d4 = reinterpret_cast<int4 *>(dst + head);
  const int4 *s4 = reinterpret_cast<const int4 *>(src + head);
  for (int e = threadIdx.x; e < nv; e += blockDim.x) d4[e] = s4[e];
  for (int e = head + nv * kPer + threadIdx.x; e < count; e += blockDim.x) dst[e] = src[e];
}

template <bool COH, typename R>
__device__ __forceinline__ void copy_in_vec(R *dst, const R *__restrict__ src, int count) {
  constexpr int kPer = 16 / (int)sizeof(R);
  const unsigned ms = (unsigned)(reinterpret_cast<uintptr_t>(src) & 15u);
  int head = (int)(((16u - ms) & 15u) / sizeof(R));  // values before the first whole vector
  if (head > count) head = count;
  const int nv = (count - head) / kPer;
  for (int e = threadIdx.x; e < head; e += blockDim.x) dst[e] = gld<COH>(src + e);
  const int4 *s4 = reinterpret_cast<const int4 *>(src + head);
  if (ms == (unsigned)(reinterpret_cast<uintptr_t>(dst) & 15u)) {
    int4 *d4 = reinterpret_cast<int4 *>(dst + head);
    for (int e = threadIdx.x; e < nv; e += blockDim.x) d4[e] = gld<COH>(s4 + e);
  } else {
    for (int e = threadIdx.x; e < nv; e += blockDim.x) {
      const int4 w = gld<COH>(s4 + e);
      const R *p = reinterpret_cast<const R *>(&w);
      R *d = dst + head + e * kPer;
#pragma unroll
      for (int q = 0; q < kPer; ++q) d[q] = p[q];
    }
  }
  for (int e = head + nv * kPer + threadIdx.x; e < count; e += blockDim.x) dst[e] = gld<COH>(src + e);
}
template <typename R>
__device__ __forceinline__ void copy_out_vec(R *__restrict__ dst, const R *src, int count) {
  constexpr int kPer = 16 / (int)sizeof(R);
  const unsigned md = (unsigned)(reinterpret_cast<uintptr_t>(dst) & 15u);
  int head = (int)(((16u - md) & 15u) / sizeof(R));
  if (head > count) head = count;
  const int nv = (count - head) / kPer;
  for (int e = threadIdx.x; e < head; e += blockDim.x) dst[e] = src[e];
  int4 *d4 = reinterpret_cast<int4 *>(dst + head);
  if (md == (unsigned)(reinterpret_cast<uintptr_t>(src) & 15u)) {
    const int4 *s4 = reinterpret_cast<const int4 *>(src + head);
    for (int e = threadIdx.x; e < nv; e += blockDim.x) d4[e] = s4[e];
  } else {
    for (int e = threadIdx.x; e < nv; e += blockDim.x) {
      int4 w;
      R *p = reinterpret_cast<R *>(&w);
      const R *sp = src + head + e * kPer;
#pragma unroll
      for (int q = 0; q < kPer; ++q) p[q] = sp[q];
      d4[e] = w;
    }
  }
  for (int e = head + nv * kPer + threadIdx.x; e < count; e += blockDim.x) dst[e] = src[e];
}

// Asynchronous global-to-shared copies (cp.async): the data lands in shared memory while the
// issuing threads go on computing; cp_async_wait<N>() waits until at most the N most recently
// committed groups are still in flight (a hardware wait that always ends).
__device__ __forceinline__ void cp_async(void *smem, const void *g, int bytes) {
  const unsigned s = smem_addr(smem);
  const size_t ga = __cvta_generic_to_global(g);
  if (bytes == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(ga) : "memory");
  else if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(ga) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(ga) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// copy_in's asynchronous form: 16-byte copies where both sides share their offset within a
// 16-byte line, single values otherwise; nothing outside the range is read.
template <typename R>
__device__ __forceinline__ void copy_in_async(R *dst, const R *__restrict__ src, int count) {
  constexpr int kPer = 16 / (int)sizeof(R);
  const unsigned ms = (unsigned)(reinterpret_cast<uintptr_t>(src) & 15u);
  if (ms != (unsigned)(reinterpret_cast<uintptr_t>(dst) & 15u)) {
    for (int e = threadIdx.x; e < count; e += blockDim.x) cp_async(dst + e, src + e, (int)sizeof(R));
    return;
  }
  int head = (int)(((16u - ms) & 15u) / sizeof(R));
  if (head > count) head = count;
  const int nv = (count - head) / kPer;
  for (int e = threadIdx.x; e < head; e += blockDim.x) cp_async(dst + e, src + e, (int)sizeof(R));
  for (int e = threadIdx.x; e < nv; e += blockDim.x) cp_async(dst + head + e * kPer, src + head + e * kPer, 16);
  for (int e = head + nv * kPer + threadIdx.x; e < count; e += blockDim.x) cp_async(dst + e, src + e, (int)sizeof(R));
}

// Copy the W sites starting at chain index t0 (may be negative or run past the end) of the
// chain at `off` into shared memory, coalesced.  Periodic: wrapped; fixed: zero outside the
// chain.  A tile that crosses a chain end is copied as a few contiguous segments (one index
// wrap per segment, not per element): at most 2 for chains longer than the tile, N / W + 2
// for shorter periodic chains.
template <typename R, int D, bool COH>
__device__ __forceinline__ void tile_load(R *tile, const R *__restrict__ src, int64_t off, int64_t n, int bc,
                                          int64_t t0, int W, int64_t sites, WsHeader *hdr) {
  const int total = W * D;
  if (t0 >= 0 && t0 + W <= n) {
    if (!bounds_ok(hdr, in_range(off + t0, W, sites))) return;
    if constexpr (COH) copy_in_vec<COH>(tile, src + (off + t0) * D, total);  // the persistent kernel
    else copy_in<COH>(tile, src + (off + t0) * D, total);
    return;
  }
  int covered = 0;  // block-uniform loop over contiguous segments
  while (covered < W) {
    const int64_t g = t0 + covered;
    const int64_t rest = W - covered;
    int len;
    const R *seg = nullptr;  // NULL: a run of fixed-end ghosts (zeros)
    if (bc == PERIODIC) {
      const int64_t gw = wrap(g, n);
      len = (int)(rest < n - gw ? rest : n - gw);
      seg = src + (off + gw) * D;
    } else if (g < 0) {
      len = (int)(rest < -g ? rest : -g);
    } else if (g >= n) {
      len = (int)rest;
    } else {
      len = (int)(rest < n - g ? rest : n - g);
      seg = src + (off + g) * D;
    }
    R *dst = tile + covered * D;
    const int cnt = len * D;
    if (seg && !bounds_ok(hdr, in_range(seg - src, cnt, sites * D))) seg = nullptr;
    if (seg) {
      for (int e = threadIdx.x; e < cnt; e += blockDim.x) dst[e] = gld<COH>(seg + e);
    } else {
      for (int e = threadIdx.x; e < cnt; e += blockDim.x) dst[e] = R(0);
    }
    covered += len;
  }
}

// tile_load for a tile kernel that prefetches its next tile: a window inside the chain is
// copied asynchronously (the caller commits and later waits); a window that crosses a chain
// end (wrapped or zero-filled segments, a few tiles per chain) is copied synchronously.
template <typename R, int D>
__device__ __forceinline__ void tile_load_async(R *tile, const R *__restrict__ src, int64_t off, int64_t n, int bc,
                                                int64_t t0, int W, int64_t sites, WsHeader *hdr) {
  if (t0 >= 0 && t0 + W <= n) {
    if (!bounds_ok(hdr, in_range(off + t0, W, sites))) return;
    copy_in_async(tile, src + (off + t0) * D, W * D);
    return;
  }
  tile_load<R, D, false>(tile, src, off, n, bc, t0, W, sites, hdr);
}

// Store `cnt` sites of the tile starting at tile-local site `first` to chain index g0 (VEC:
// copy_out_vec, for the persistent kernel; MATCHED: copy_out_matched, for tiles whose window
// starts on a 16-byte boundary).
template <typename R, int D, bool VEC = false, bool MATCHED = false>
__device__ __forceinline__ void tile_store(R *__restrict__ dst, const R *tile, int64_t off, int first, int64_t g0,
                                           int cnt, int64_t sites, int W, WsHeader *hdr) {
  if (!bounds_ok(hdr, in_range(off + g0, cnt, sites) && in_range(first, cnt, W))) return;
  if constexpr (MATCHED) copy_out_matched(dst + (off + g0) * D, tile + first * D, cnt * D);
  else if constexpr (VEC) copy_out_vec(dst + (off + g0) * D, tile + first * D, cnt * D);
  else copy_out(dst + (off + g0) * D, tile + first * D, cnt * D);
}

// Sites per 16 bytes of a [sites][D] array of R, in whole sites (16 / gcd(16, D sizeof(R))).
template <typename R, int D> __host__ __device__ constexpr int align_sites() {
  int a = D * (int)sizeof(R), b = 16;
  while (b) {
    const int t = a % b;
    a = b;
    b = t;
  }
  return 16 / a;
}

// Process one (chain, tile) item end to end: load, advance K steps, store the interior.
// ALN (batch tiles): the window starts at the last multiple of align_sites() at or before
// tile G - H in the state array, so it moves by whole 16-byte vectors wherever the chain
// starts; the left halo is then H .. H + A - 1 sites, and the host shrinks G by A - 1 so that
// the right halo keeps at least H.
// Shared memory: edge[edge_values(V)] | tile[W*D] | ctile[W*D] (Kahan) | ptile[W*P]
// (heterogeneous).
// `sites` is the number of sites in the state buffers (for the debug bounds checks); hdr the
// status word, where a non-finite stored value is reported.
template <typename R, int MODEL, int V, bool KAHAN, bool COH, bool HET = false, bool ALN = false>
__device__ __forceinline__ void tile_item(const R *__restrict__ in, R *__restrict__ out, const R *__restrict__ cin,
                                          R *__restrict__ cout, const ChainDesc &ch, int64_t tile, int K, int G,
                                          const Coef<R> &cf, unsigned char *smem, int64_t sites, WsHeader *hdr,
                                          const R *__restrict__ sp = nullptr) {
  constexpr int D = Dim<MODEL>::D;
  constexpr int P = Dim<MODEL>::P;
  R *edge = reinterpret_cast<R *>(smem);
  const int W = blockDim.x * V;
  const int H = 4 * K;
  const int64_t g0 = tile * (int64_t)G;  // first interior site
  int64_t t0 = g0 - H;
  if constexpr (ALN) {
    constexpr int A = align_sites<R, D>();
    const int64_t a = ch.off + t0;  // rounded down (toward minus infinity) to a multiple of A
    t0 = (a >= 0 ? a / A : -((-a + A - 1) / A)) * A - ch.off;
  }
  const int hl = (int)(g0 - t0);  // left halo: H, or up to A - 1 sites more with ALN
  R *tl = edge + edge_values(V);
  R *ctl = tl + W * D;
  R *ptl = ctl + (KAHAN ? W * D : 0);

  tile_load<R, D, COH>(tl, in, ch.off, ch.n, ch.bc, t0, W, sites, hdr);
  if constexpr (KAHAN) tile_load<R, D, COH>(ctl, cin, ch.off, ch.n, ch.bc, t0, W, sites, hdr);
  if constexpr (HET) tile_load<R, P, COH>(ptl, sp, ch.off, ch.n, ch.bc, t0, W, sites, hdr);
  __syncthreads();

  R y[V][D], cmp[V][D];
  const int base = threadIdx.x * V;
#pragma unroll
  for (int v = 0; v < V; ++v)
#pragma unroll
    for (int d = 0; d < D; ++d) {
      y[v][d] = tl[(base + v) * D + d];
      if constexpr (KAHAN) cmp[v][d] = ctl[(base + v) * D + d]; else cmp[v][d] = R(0);
    }

  Coef<R> cs[HET ? V : 1];
  if constexpr (HET) {
#pragma unroll
    for (int v = 0; v < V; ++v) cs[v] = site_coef<R, MODEL>(cf, ptl + (base + v) * P);
  }

  const bool edge_tile = (ch.bc == FIXED) && (t0 < 0 || t0 + W > ch.n);
  if (edge_tile) {
    uint32_t ghost = 0;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int64_t g = t0 + base + v;
      if (g < 0 || g >= ch.n) ghost |= 1u << v;
    }
    tile_advance<R, MODEL, V, KAHAN, true, HET>(y, cmp, ghost, K, cf, edge, cs);
  } else {
    tile_advance<R, MODEL, V, KAHAN, false, HET>(y, cmp, 0u, K, cf, edge, cs);
  }

  const int64_t rem = ch.n - g0;
  const int cnt = (int)(rem < G ? rem : G);
  bool bad = false;  // a stored (interior) value is NaN or infinite
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const bool stored = base + v >= hl && base + v < hl + cnt;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      tl[(base + v) * D + d] = y[v][d];
      if constexpr (KAHAN) ctl[(base + v) * D + d] = cmp[v][d];
      bad |= stored && nonfinite(y[v][d]);
    }
  }
  report_nonfinite(hdr, __syncthreads_or(bad));
  if (cnt > 0) {
    tile_store<R, D, COH, ALN>(out, tl, ch.off, hl, g0, cnt, sites, W, hdr);
    if constexpr (KAHAN) tile_store<R, D, COH, ALN>(cout, ctl, ch.off, hl, g0, cnt, sites, W, hdr);
  }
  __syncthreads();  // shared memory is reused by the next item
}

// Process one packed tile: segments s0 .. s1 - 1 of `segs`, side by side in slot order, each a
// window [g0 - H, g0 + cnt + H + pad) of its own chain (wrapped or zero outside the chain like a
// plain tile).  The neighbour exchange runs across segment borders as if the tile were one
// chain: a wrong neighbour at a border, like a missing one at a tile end, spoils one more site
// per stage, so after K steps only each segment's H-site halos are spoilt and its cnt interior
// sites are exact.  Every thread's sites lie in one segment (o and L are multiples of V), so a
// thread takes its chain's coupling strength and, for fixed ends, its ghost mask; threads past
// the last segment advance zeros that are never stored.
template <typename R, int MODEL, int V, bool KAHAN, bool COH>
__device__ __forceinline__ void packed_tile_item(const R *__restrict__ in, R *__restrict__ out,
                                                 const R *__restrict__ cin, R *__restrict__ cout,
                                                 const ChainDesc *chains, const SegDesc *segs, int s0, int s1,
                                                 int K, const Coef<R> &cf, unsigned char *smem, int64_t sites,
                                                 WsHeader *hdr) {
  constexpr int D = Dim<MODEL>::D;
  R *edge = reinterpret_cast<R *>(smem);
  R *tl = edge + edge_values(V);
  const int W = blockDim.x * V;
  R *ctl = tl + W * D;
  const int H = 4 * K;

  int used = 0;  // slots covered by the segments (they are in slot order)
  for (int s = s0; s < s1; ++s) {
    const SegDesc sd = segs[s];
    if (!bounds_ok(hdr, sd.o >= used && sd.L >= 0 && sd.o + sd.L <= W)) continue;
    const ChainDesc ch = chains[sd.chain];
    tile_load<R, D, COH>(tl + sd.o * D, in, ch.off, ch.n, ch.bc, sd.g0 - H, sd.L, sites, hdr);
    if constexpr (KAHAN) tile_load<R, D, COH>(ctl + sd.o * D, cin, ch.off, ch.n, ch.bc, sd.g0 - H, sd.L, sites, hdr);
    used = sd.o + sd.L;
  }
  for (int e = used * D + threadIdx.x; e < W * D; e += blockDim.x) {
    tl[e] = R(0);
    if constexpr (KAHAN) ctl[e] = R(0);
  }
  __syncthreads();

  // this thread's segment: the last one starting at or before its first slot
  const int base = threadIdx.x * V;
  int my = -1;
  if (s1 > s0) {
    int lo = s0, hi = s1 - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (segs[mid].o <= base) lo = mid; else hi = mid - 1;
    }
    if (segs[lo].o <= base && base < segs[lo].o + segs[lo].L) my = lo;
  }
  Coef<R> c = cf;
  uint32_t ghost = 0;
  int rel = 0, cnt = 0;  // first site's position in the segment's window; the segment's interior sites
  if (my >= 0) {
    const SegDesc sd = segs[my];
    const ChainDesc ch = chains[sd.chain];
    c.kappa = (R)ch.kappa;
    rel = base - sd.o;
    cnt = sd.cnt;
    if (ch.bc == FIXED) {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int64_t g = sd.g0 - H + rel + v;
        if (g < 0 || g >= ch.n) ghost |= 1u << v;
      }
    }
  }

  R y[V][D], cmp[V][D];
#pragma unroll
  for (int v = 0; v < V; ++v)
#pragma unroll
    for (int d = 0; d < D; ++d) {
      y[v][d] = tl[(base + v) * D + d];
      if constexpr (KAHAN) cmp[v][d] = ctl[(base + v) * D + d]; else cmp[v][d] = R(0);
    }
  tile_advance<R, MODEL, V, KAHAN, true>(y, cmp, ghost, K, c, edge);

  bool bad = false;  // a stored (interior) value is NaN or infinite
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const bool stored = my >= 0 && rel + v >= H && rel + v < H + cnt;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      tl[(base + v) * D + d] = y[v][d];
      if constexpr (KAHAN) ctl[(base + v) * D + d] = cmp[v][d];
      bad |= stored && nonfinite(y[v][d]);
    }
  }
  report_nonfinite(hdr, __syncthreads_or(bad));
  for (int s = s0; s < s1; ++s) {
    const SegDesc sd = segs[s];
    if (sd.cnt <= 0 || !bounds_ok(hdr, sd.o >= 0 && sd.o + sd.L <= W && sd.cnt + 2 * H <= sd.L)) continue;
    const ChainDesc ch = chains[sd.chain];
    tile_store<R, D, COH>(out, tl, ch.off, sd.o + H, sd.g0, sd.cnt, sites, W, hdr);
    if constexpr (KAHAN) tile_store<R, D, COH>(cout, ctl, ch.off, sd.o + H, sd.g0, sd.cnt, sites, W, hdr);
  }
  __syncthreads();  // shared memory is reused by the next item
}

// Locate the chain of a tile index through the prefix array (first tile of each chain).
__device__ __forceinline__ int find_chain(const int32_t *prefix, int nchains, int64_t tile) {
  int lo = 0, hi = nchains - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// find_chain by one warp: each round the 32 lanes test 32 evenly spaced candidates at once and
// the range shrinks 32-fold, so 4096 chains take three rounds of loads instead of twelve
// dependent ones.  Call with all 32 lanes of a warp; every lane returns the answer.
__device__ __forceinline__ int find_chain_warp(const int32_t *prefix, int nchains, int64_t tile) {
  const int lane = threadIdx.x & 31;
  int lo = 0, hi = nchains - 1;  // the answer (largest c with prefix[c] <= tile) lies in [lo, hi]
  while (hi > lo) {
    const int step = (hi - lo + 32) / 32;  // ceil((hi - lo + 1) / 32)
    const int c = lo + lane * step;
    const unsigned ok = __ballot_sync(kFull, c <= hi && prefix[c] <= tile);
    const int last = 31 - __clz(ok);  // lane 0's candidate, lo, always qualifies
    lo += last * step;
    hi = min(hi, lo + step - 1);
  }
  return lo;
}

// The chain of a batch tile, found once per block: the first warp searches (find_chain_warp)
// and passes the answer to the others through the first word of the block's shared memory (the
// neighbour-exchange area, which the tile kernels first write after the barrier that ends
// their tile load, when every thread has read the answer).
__device__ __forceinline__ int find_chain_block(const int32_t *prefix, int nchains, int64_t tile,
                                                unsigned char *smem) {
  int *slot = reinterpret_cast<int *>(smem);
  if (threadIdx.x < 32) {
    const int c = find_chain_warp(prefix, nchains, tile);
    if (threadIdx.x == 0) *slot = c;
  }
  __syncthreads();
  return *slot;
}

// Chain and chain-local tile index of full tile f of a batch launch: one load from the tile
// table when the launch has one, else the block's search of the first-tile prefix.  Every
// thread of the block calls it and gets the same answer.
__device__ __forceinline__ int batch_chain(const BatchTiles &bt, int nchains, int64_t f, unsigned char *smem,
                                           int64_t &local) {
  if (bt.tile_chain) {
    const int2 tc = __ldg(&bt.tile_chain[f]);
    local = tc.y;
    return tc.x;
  }
  const int ci = find_chain_block(bt.full_prefix, nchains, f, smem);
  local = f - bt.full_prefix[ci];
  return ci;
}

// Item `item` of a batch launch laid out by bt: the packed tiles first (they then run among the
// full tiles instead of alone at the end), then the full tiles of the chains.
template <typename R, int MODEL, int V, bool KAHAN, bool COH>
__device__ __forceinline__ void batch_item(const R *__restrict__ in, R *__restrict__ out, const R *__restrict__ cin,
                                           R *__restrict__ cout, const ChainDesc *chains, int nchains,
                                           const BatchTiles &bt, int64_t item, int K, int G, const Coef<R> &cf,
                                           unsigned char *smem, int64_t sites, WsHeader *hdr) {
  if (item < bt.npacked) {
    packed_tile_item<R, MODEL, V, KAHAN, COH>(in, out, cin, cout, chains, bt.segs, bt.pack_prefix[item],
                                              bt.pack_prefix[item + 1], K, cf, smem, sites, hdr);
  } else {
    int64_t local;
    const int ci = batch_chain(bt, nchains, item - bt.npacked, smem, local);
    const ChainDesc ch = chains[ci];
    Coef<R> c = cf;
    c.kappa = (R)ch.kappa;
    tile_item<R, MODEL, V, KAHAN, COH, false, true>(in, out, cin, cout, ch, local, K, G, c, smem, sites, hdr);
  }
}

template <typename R> __host__ __device__ inline Coef<R> to_coef(const CoefD &c, double kappa) {
  Coef<R> r;
  r.a = (R)c.a; r.b = (R)c.b; r.c = (R)c.c; r.kappa = (R)kappa; r.w2 = (R)c.w2;
  r.h2 = (R)c.h2; r.h1 = (R)c.h1; r.dt6 = (R)c.dt6; r.dt3 = (R)c.dt3; r.one = R(1);
  return r;
}

}  // namespace rk4d
