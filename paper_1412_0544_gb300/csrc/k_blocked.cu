// k_blocked.cu -- temporally blocked RK4 kernel: one thread block per (chain, tile) item,
// k steps per launch (k = 1 is the fused single-step kernel).  HET: heterogeneous chains
// (Eq. (1) of the paper), whose per-site parameters travel with the tile.
#include "rk4_tile.cuh"

namespace rk4d {

// Largest block and resident blocks per SM the blocked kernel is compiled for.  FP32 with 4+
// sites per thread asks for two blocks of the largest size (64 registers); the heterogeneous
// FP32 Roessler chain with 4 sites per thread, whose four per-site coefficients need more, is
// capped at 256 threads and asks for three such blocks (79 registers instead of 96, which
// allowed two).  Elsewhere no minimum: an explicit minimum of one block lets ptxas take more
// registers.
template <int MODEL, int V, bool KAHAN, bool HET> struct BlockedBounds {
  static constexpr bool kHetWide = HET && KAHAN && V == 4 && MODEL == ROESSLER;
  static constexpr int threads = kHetWide ? 256 : max_threads_for(V);
  static constexpr int min_blocks = kHetWide ? 3 : ((V >= 4 && KAHAN && !HET) ? 2 : 0);
};

// A batch launch's packed tiles (item p of them).  Not inlined: the segment bookkeeping then
// takes registers only inside this call, and the tile loop of k_blocked, which runs nearly
// every tile, keeps its own allocation (with the packed path inlined the FP32 tile kernel
// spilled 120 bytes and ran 4 % slower; as a second kernel launched after each batch launch
// its few blocks ran alone at the end of every launch).
template <typename R, int MODEL, int V, bool KAHAN>
__device__ __noinline__ void packed_tile_call(const void *in, void *out, const void *cin, void *cout,
                                              const ChainDesc *chains, const SegDesc *segs, const int32_t *pack_prefix,
                                              int64_t p, int K, Coef<R> cf, unsigned char *smem, int64_t sites,
                                              WsHeader *hdr) {
  packed_tile_item<R, MODEL, V, KAHAN, false>(static_cast<const R *>(in), static_cast<R *>(out),
                                              static_cast<const R *>(cin), static_cast<R *>(cout), chains, segs,
                                              pack_prefix[p], pack_prefix[p + 1], K, cf, smem, sites, hdr);
}

// PACKED: a packed batch's launch (its own instantiation, so that single chains run the plain
// tile path alone): the packed tiles come first, so that they run in the first wave beside full
// tiles instead of alone after the last one, then the full tiles with 16-byte-aligned windows.
template <typename R, int MODEL, int V, bool KAHAN, bool HET, bool PACKED = false>
__global__ void __launch_bounds__(BlockedBounds<MODEL, V, KAHAN, HET>::threads,
                                  BlockedBounds<MODEL, V, KAHAN, HET>::min_blocks)
    k_blocked(BlockedJob job, Coef<R> cf) {
  extern __shared__ __align__(16) unsigned char smem[];
  int64_t item = blockIdx.x;
  if constexpr (PACKED) {
    if (item < job.bt.npacked) {
      packed_tile_call<R, MODEL, V, KAHAN>(job.in, job.out, job.cin, job.cout, job.chains, job.bt.segs,
                                           job.bt.pack_prefix, item, job.K, cf, smem, job.total, job.hdr);
      return;
    }
    item -= job.bt.npacked;
  }
  ChainDesc ch;
  int64_t tile = item;
  Coef<R> c = cf;
  if (job.nchains == 1) {
    ch = job.one;
  } else {
    const int ci = batch_chain(job.bt, job.nchains, item, smem, tile);
    ch = job.chains[ci];
    c.kappa = (R)ch.kappa;
  }
  tile_item<R, MODEL, V, KAHAN, false, HET, PACKED>(static_cast<const R *>(job.in), static_cast<R *>(job.out),
                                            static_cast<const R *>(job.cin), static_cast<R *>(job.cout), ch, tile,
                                            job.K, job.G, c, smem, job.total, job.hdr,
                                            static_cast<const R *>(job.sp));
}

// The tile table of a batch launch: tile t's chain (the largest c with prefix[c] <= t, so
// chains without tiles are skipped) and its index within the chain.
__global__ void k_tile_chains(const int32_t *__restrict__ prefix, int nchains, int64_t ntiles,
                              int2 *__restrict__ tile_chain) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ntiles; t += (int64_t)gridDim.x * blockDim.x) {
    const int c = find_chain(prefix, nchains, t);
    tile_chain[t] = make_int2(c, (int)(t - prefix[c]));
  }
}

cudaError_t launch_tile_chains(const int32_t *prefix, int nchains, int64_t ntiles, int2 *tile_chain, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((ntiles + 255) / 256, (int64_t)sm_count() * 8);
  k_tile_chains<<<(unsigned)blocks, 256, 0, st>>>(prefix, nchains, ntiles, tile_chain);
  return cudaGetLastError();
}

size_t blocked_smem_bytes(int model, bool fp32, int v, int block, bool het) {
  const int D = model == ROESSLER ? 3 : 2;
  const int P = model == ROESSLER ? 4 : 2;
  const size_t rs = fp32 ? 4 : 8;
  return (size_t)edge_values(v) * rs + (size_t)block * v * rs * (D * (fp32 ? 2 : 1) + (het ? P : 0));
}

template <typename R, int MODEL, int V, bool KAHAN, bool HET>
static cudaError_t launch_one(int block, const BlockedJob &job, const CoefD &cfd, cudaStream_t st) {
  static PerDevice attr, attr_p;
  const size_t smem = blocked_smem_bytes(MODEL, KAHAN, V, block, HET);
  Coef<R> cf = to_coef<R>(cfd, cfd.kappa);
  if constexpr (!HET) {
    if (job.nchains > 1 && job.packed) {  // one block per packed tile and one per full tile
      const cudaError_t e = set_smem_limit_once(k_blocked<R, MODEL, V, KAHAN, false, true>, 200 * 1024, attr_p);
      if (e != cudaSuccess) return e;
      const int64_t grid = job.ntiles + job.bt.npacked;
      if (grid > 0) k_blocked<R, MODEL, V, KAHAN, false, true><<<(unsigned)grid, block, smem, st>>>(job, cf);
      return cudaGetLastError();
    }
  }
  const cudaError_t e = set_smem_limit_once(k_blocked<R, MODEL, V, KAHAN, HET>, 200 * 1024, attr);
  if (e != cudaSuccess) return e;
  if (job.ntiles > 0) k_blocked<R, MODEL, V, KAHAN, HET><<<(unsigned)job.ntiles, block, smem, st>>>(job, cf);
  return cudaGetLastError();
}

template <int MODEL, int V, bool HET>
static cudaError_t launch_v(bool fp32, int block, const BlockedJob &job, const CoefD &cf, cudaStream_t st) {
  return fp32 ? launch_one<float, MODEL, V, true, HET>(block, job, cf, st)
              : launch_one<double, MODEL, V, false, HET>(block, job, cf, st);
}

template <int MODEL>
static cudaError_t launch_m(bool fp32, int v, int block, const BlockedJob &job, const CoefD &cf, cudaStream_t st) {
  if (job.sp) {  // heterogeneous chains: 2 or 4 sites per thread
    switch (v) {
      case 2: return launch_v<MODEL, 2, true>(fp32, block, job, cf, st);
      case 4: return launch_v<MODEL, 4, true>(fp32, block, job, cf, st);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (v) {
    case 1: return launch_v<MODEL, 1, false>(fp32, block, job, cf, st);
    case 2: return launch_v<MODEL, 2, false>(fp32, block, job, cf, st);
    case 4: return launch_v<MODEL, 4, false>(fp32, block, job, cf, st);
    case 8: return launch_v<MODEL, 8, false>(fp32, block, job, cf, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_blocked(int model, bool fp32, int v, int block, const BlockedJob &job, const CoefD &cf,
                           cudaStream_t st) {
  return model == ROESSLER ? launch_m<ROESSLER>(fp32, v, block, job, cf, st)
                           : launch_m<HARMONIC>(fp32, v, block, job, cf, st);
}

template <typename R, int MODEL, int V, bool KAHAN, bool HET>
static int max_threads_one() {
  cudaFuncAttributes a;
  if (cudaFuncGetAttributes(&a, k_blocked<R, MODEL, V, KAHAN, HET>) != cudaSuccess) return 0;
  return a.maxThreadsPerBlock;
}

template <int MODEL, int V, bool HET>
static int max_threads_v(bool fp32) {
  return fp32 ? max_threads_one<float, MODEL, V, true, HET>() : max_threads_one<double, MODEL, V, false, HET>();
}

template <int MODEL>
static int max_threads_m(bool fp32, int v, bool het) {
  if (het) {
    if (v == 2) return max_threads_v<MODEL, 2, true>(fp32);
    if (v == 4) return max_threads_v<MODEL, 4, true>(fp32);
    return 0;
  }
  switch (v) {
    case 1: return max_threads_v<MODEL, 1, false>(fp32);
    case 2: return max_threads_v<MODEL, 2, false>(fp32);
    case 4: return max_threads_v<MODEL, 4, false>(fp32);
    case 8: return max_threads_v<MODEL, 8, false>(fp32);
    default: return 0;
  }
}

int blocked_max_threads(int model, bool fp32, int v, bool het) {
  return model == ROESSLER ? max_threads_m<ROESSLER>(fp32, v, het) : max_threads_m<HARMONIC>(fp32, v, het);
}

}  // namespace rk4d
