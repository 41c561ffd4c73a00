// k_persistent.cu -- one persistent, cooperative launch that integrates a whole batch of
// chains: for every block of k steps each resident thread block walks its share of the
// (chain, tile) items, then all blocks meet at a grid barrier before the next time block
// reads what the previous one wrote.  The barrier's wait is bounded: a block that waits
// longer than timeout_ns latches ST_TIMEOUT in the status word and the kernel returns.
#include "rk4_tile.cuh"

namespace rk4d {

__device__ __forceinline__ long long global_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier over the co-resident blocks of a cooperative launch.  Returns false when
// this block gave up waiting (or another block already did).
__device__ __forceinline__ bool grid_barrier(WsHeader *hdr, long long timeout_ns, int extra) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned *gen = &hdr->bar_gen;
    volatile int *status = &hdr->status;
    const unsigned g = *gen;
    __threadfence();
    const unsigned expected = gridDim.x + (unsigned)extra;
    const unsigned arrived = atomicAdd(&hdr->bar_count, 1u) + 1u;
    if (arrived == expected) {
      atomicExch(&hdr->bar_count, 0u);
      __threadfence();
      atomicAdd(&hdr->bar_gen, 1u);
    } else {
      const long long t0 = global_ns();
      while (*gen == g) {
        if ((*status & ST_TIMEOUT) || global_ns() - t0 > timeout_ns) {
          atomicOr(&hdr->status, ST_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// A packed tile of a batch (the segments of item p).  Not inlined, as in the one-shot blocked
// kernel: the segment bookkeeping then takes registers only inside this call, and the full-tile
// path, which runs nearly every item, keeps its own allocation (inlined, the FP32 batch kernel
// spilled at the 64-register cap of four resident blocks per SM).
template <typename R, int MODEL, int V, bool KAHAN>
__device__ __noinline__ void persistent_packed_call(const R *in, R *out, const R *cin, R *cout,
                                                    const ChainDesc *chains, const SegDesc *segs,
                                                    const int32_t *pack_prefix, int64_t p, int K, Coef<R> cf,
                                                    unsigned char *smem, int64_t sites, WsHeader *hdr) {
  packed_tile_item<R, MODEL, V, KAHAN, true>(in, out, cin, cout, chains, segs, pack_prefix[p], pack_prefix[p + 1], K,
                                             cf, smem, sites, hdr);
}

// One full tile, of a single chain or (BATCH) of a batch, as a call of its own: the tile's
// arithmetic then gets the register budget it has in the one-shot blocked kernel, instead of
// sharing it with the persistent loop's state (time block, item, buffers), which the call saves
// once per tile.
template <typename R, int MODEL, int V, bool KAHAN, bool BATCH>
__device__ __noinline__ void persistent_tile_call(const PersistentJob &job, int ki, const R *in, R *out,
                                                  const R *cin, R *cout, int64_t item, int K, int G, Coef<R> cf,
                                                  unsigned char *smem) {
  if constexpr (!BATCH)
    tile_item<R, MODEL, V, KAHAN, true>(in, out, cin, cout, job.one, item, K, G, cf, smem, job.total, job.hdr);
  else
    batch_item<R, MODEL, V, KAHAN, true>(in, out, cin, cout, job.chains, job.nchains, job.bt[ki], item, K, G, cf,
                                         smem, job.total, job.hdr);
}

template <typename R, int MODEL, int V, bool KAHAN, bool BATCH>
__global__ void __launch_bounds__(max_threads_for(V), (V >= 2 && KAHAN) ? 2 : 1)  // FP32: two resident blocks
    k_persistent(PersistentJob job, Coef<R> cf) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int64_t nblocks_t = job.nmain + job.ntail;
  for (int64_t t = 0; t < nblocks_t; ++t) {
    const int ki = (t < job.nmain) ? 0 : job.tail[t - job.nmain];
    const int K = job.kval[ki];
    const int G = job.Gval[ki];
    const int64_t ntiles = job.ntiles[ki];
    const R *in = static_cast<const R *>((t & 1) ? job.bufB : job.bufA);
    R *out = static_cast<R *>((t & 1) ? job.bufA : job.bufB);
    const R *cin = static_cast<const R *>((t & 1) ? job.cB : job.cA);
    R *cout = static_cast<R *>((t & 1) ? job.cA : job.cB);
    // Items are handed out dynamically (an atomic counter per time-block parity), so blocks
    // that drew cheaper items take more and all reach the barrier together.  Block 0 clears
    // the other parity's counter for the next time block (the barrier orders it).
    unsigned long long *ctr = &job.hdr->work[t & 1];
    if (blockIdx.x == 0 && threadIdx.x == 0 && t > 0) job.hdr->work[(t + 1) & 1] = 0ull;
    __shared__ long long s_item;
    if (threadIdx.x == 0) s_item = (long long)atomicAdd(ctr, 1ull);
    __syncthreads();
    for (int64_t item = s_item; item < ntiles;) {
      if (BATCH && item < job.bt[ki].npacked)
        persistent_packed_call<R, MODEL, V, KAHAN>(in, out, cin, cout, job.chains, job.bt[ki].segs,
                                                   job.bt[ki].pack_prefix, item, K, cf, smem, job.total, job.hdr);
      else
        persistent_tile_call<R, MODEL, V, KAHAN, BATCH>(job, ki, in, out, cin, cout, item, K, G, cf, smem);
      // both end with a barrier, so every thread has read s_item before it is rewritten
      if (threadIdx.x == 0) s_item = (long long)atomicAdd(ctr, 1ull);
      __syncthreads();
      item = s_item;
    }
    if (t + 1 < nblocks_t || job.extra_arrivals > 0) {
      if (!grid_barrier(job.hdr, job.timeout_ns, job.extra_arrivals)) return;
    }
  }
}

template <typename R, int MODEL, int V, bool KAHAN>
static cudaError_t setup_attr() {
  static PerDevice attr, attr_b;
  const cudaError_t e = set_smem_limit_once(k_persistent<R, MODEL, V, KAHAN, false>, 200 * 1024, attr);
  if (e != cudaSuccess) return e;
  return set_smem_limit_once(k_persistent<R, MODEL, V, KAHAN, true>, 200 * 1024, attr_b);
}

template <typename R, int MODEL, int V, bool KAHAN>
static cudaError_t launch_one(int block, int grid, const PersistentJob &job, const CoefD &cfd, cudaStream_t st) {
  cudaError_t e = setup_attr<R, MODEL, V, KAHAN>();
  if (e != cudaSuccess) return e;
  const size_t smem = blocked_smem_bytes(MODEL, KAHAN, V, block);
  Coef<R> cf = to_coef<R>(cfd, cfd.kappa);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (job.nchains > 1) return cudaLaunchKernelEx(&cfg, k_persistent<R, MODEL, V, KAHAN, true>, job, cf);
  return cudaLaunchKernelEx(&cfg, k_persistent<R, MODEL, V, KAHAN, false>, job, cf);
}

template <typename R, int MODEL, int V, bool KAHAN>
static int max_grid_one(int block) {
  if (setup_attr<R, MODEL, V, KAHAN>() != cudaSuccess) return 0;
  int per_sm = 0;
  const size_t smem = blocked_smem_bytes(MODEL, KAHAN, V, block);
  int per_sm_b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persistent<R, MODEL, V, KAHAN, false>, block, smem) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_b, k_persistent<R, MODEL, V, KAHAN, true>, block, smem) !=
          cudaSuccess)
    return 0;
  return std::min(per_sm, per_sm_b) * sm_count();  // a grid that stays co-resident with either form
}

#define RK4_DISPATCH_V(FN, ...)                                                                   \
  switch (v) {                                                                                     \
    case 1: return fp32 ? FN<float, MODEL, 1, true>(__VA_ARGS__) : FN<double, MODEL, 1, false>(__VA_ARGS__); \
    case 2: return fp32 ? FN<float, MODEL, 2, true>(__VA_ARGS__) : FN<double, MODEL, 2, false>(__VA_ARGS__); \
    case 4: return fp32 ? FN<float, MODEL, 4, true>(__VA_ARGS__) : FN<double, MODEL, 4, false>(__VA_ARGS__); \
    case 8: return fp32 ? FN<float, MODEL, 8, true>(__VA_ARGS__) : FN<double, MODEL, 8, false>(__VA_ARGS__); \
    default: break;                                                                                \
  }

template <int MODEL>
static cudaError_t launch_m(bool fp32, int v, int block, int grid, const PersistentJob &job, const CoefD &cf,
                            cudaStream_t st) {
  RK4_DISPATCH_V(launch_one, block, grid, job, cf, st)
  return cudaErrorInvalidValue;
}

template <int MODEL>
static int max_grid_m(bool fp32, int v, int block) {
  RK4_DISPATCH_V(max_grid_one, block)
  return 0;
}

cudaError_t launch_persistent(int model, bool fp32, int v, int block, int grid, const PersistentJob &job,
                              const CoefD &cf, cudaStream_t st) {
  return model == ROESSLER ? launch_m<ROESSLER>(fp32, v, block, grid, job, cf, st)
                           : launch_m<HARMONIC>(fp32, v, block, grid, job, cf, st);
}

int persistent_max_grid(int model, bool fp32, int v, int block) {
  return model == ROESSLER ? max_grid_m<ROESSLER>(fp32, v, block) : max_grid_m<HARMONIC>(fp32, v, block);
}

}  // namespace rk4d
