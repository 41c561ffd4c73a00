// k_reduce.cu -- FP64 reductions of the state (energy of the harmonic chain, half squared
// norm of the Roessler chain, non-finite detection) and the counter-based initial state.
//
// Reductions run in double whatever the state precision; an FP32-Kahan state contributes
// y - c per component (c being the compensation).  The single-chain reduction uses a fixed
// grid and a fixed combination tree, so its result is deterministic for a given N.
#include "rk4_tile.cuh"

namespace rk4d {

template <int MODEL, typename R>
__device__ __forceinline__ double site_value(const R *y, const R *c, int64_t idx) {
  double v = (double)y[idx];
  if (c) v -= (double)c[idx];
  return v;
}

// Energy contribution of site i (chain-local) plus its bond to the right neighbour; the left
// ghost bond of a fixed chain is added at i == 0.
template <int MODEL, typename R>
__device__ __forceinline__ double site_energy(const R *y, const R *c, const ChainDesc &ch, double w2, double kappa2,
                                              int64_t i, bool &bad) {
  constexpr int D = Dim<MODEL>::D;
  const int64_t g = ch.off + i;
  if constexpr (MODEL == ROESSLER) {
    const double x = site_value<MODEL>(y, c, g * D), yy = site_value<MODEL>(y, c, g * D + 1),
                 z = site_value<MODEL>(y, c, g * D + 2);
    bad |= !(isfinite(x) && isfinite(yy) && isfinite(z));
    return 0.5 * (x * x + yy * yy + z * z);
  } else {
    const double q = site_value<MODEL>(y, c, g * D), p = site_value<MODEL>(y, c, g * D + 1);
    bad |= !(isfinite(q) && isfinite(p));
    double qr;
    if (i + 1 < ch.n) qr = site_value<MODEL>(y, c, (g + 1) * D);
    else qr = (ch.bc == PERIODIC) ? site_value<MODEL>(y, c, ch.off * D) : 0.0;
    const double dq = qr - q;
    double e = 0.5 * p * p + 0.5 * w2 * q * q + 0.5 * ch.kappa * dq * dq;
    if (i == 0 && ch.bc == FIXED) e += 0.5 * ch.kappa * q * q;
    if (kappa2 != 0.0) {  // second-neighbour bonds (i, i+2), and the ghost bonds ending at sites 0, 1
      double q2;
      if (i + 2 < ch.n) q2 = site_value<MODEL>(y, c, (g + 2) * D);
      else q2 = (ch.bc == PERIODIC) ? site_value<MODEL>(y, c, (ch.off + (i + 2) % ch.n) * D) : 0.0;
      const double d2 = q2 - q;
      e += 0.5 * kappa2 * d2 * d2;
      if (i < 2 && ch.bc == FIXED) e += 0.5 * kappa2 * q * q;
    }
    return e;
  }
}

__device__ __forceinline__ double block_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = (lane < nw) ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  }
  return v;  // valid in thread 0
}

// Sum over the chain-local sites [lo, hi) of one chain (the whole chain: lo = 0, hi = n).
template <int MODEL, typename R>
__global__ void __launch_bounds__(256) k_energy_chain(const R *y, const R *c, ChainDesc ch, int64_t lo, int64_t hi,
                                                      double w2, double kappa2, double *partials, WsHeader *hdr) {
  __shared__ double red[32];
  bool bad = false;
  double acc = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < hi; i += stride)
    acc += site_energy<MODEL>(y, c, ch, w2, kappa2, i, bad);
  if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) atomicOr(&hdr->status, ST_NONFINITE);
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(1024) k_energy_final(const double *partials, int np, double *out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) acc += partials[i];
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) out[0] = s;
}

// One block per chain of a batch.
template <int MODEL, typename R>
__global__ void __launch_bounds__(256) k_energy_batch(const R *y, const R *c, const ChainDesc *chains, double w2,
                                                      double kappa2, double *out, WsHeader *hdr) {
  __shared__ double red[32];
  const ChainDesc ch = chains[blockIdx.x];
  bool bad = false;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < ch.n; i += blockDim.x) acc += site_energy<MODEL>(y, c, ch, w2, kappa2, i, bad);
  if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) atomicOr(&hdr->status, ST_NONFINITE);
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

template <int MODEL, typename R>
static cudaError_t energy_t(const void *state, const void *cmp, int nchains, const ChainDesc &one,
                            const ChainDesc *chains, const CoefD &cf, double *partials, double *out, WsHeader *hdr,
                            cudaStream_t st) {
  const R *y = static_cast<const R *>(state);
  const R *c = static_cast<const R *>(cmp);
  if (nchains == 1) {
    k_energy_chain<MODEL, R><<<kEnergyBlocks, 256, 0, st>>>(y, c, one, 0, one.n, cf.w2, cf.kappa2, partials, hdr);
    k_energy_final<<<1, 1024, 0, st>>>(partials, kEnergyBlocks, out);
  } else {
    k_energy_batch<MODEL, R><<<nchains, 256, 0, st>>>(y, c, chains, cf.w2, cf.kappa2, out, hdr);
  }
  return cudaGetLastError();
}

cudaError_t launch_energy(int model, bool fp32, const void *state, const void *cmp, int nchains, const ChainDesc &one,
                          const ChainDesc *chains, const CoefD &cf, double *partials, double *out, WsHeader *hdr,
                          cudaStream_t st) {
  if (model == ROESSLER)
    return fp32 ? energy_t<ROESSLER, float>(state, cmp, nchains, one, chains, cf, partials, out, hdr, st)
                : energy_t<ROESSLER, double>(state, cmp, nchains, one, chains, cf, partials, out, hdr, st);
  return fp32 ? energy_t<HARMONIC, float>(state, cmp, nchains, one, chains, cf, partials, out, hdr, st)
              : energy_t<HARMONIC, double>(state, cmp, nchains, one, chains, cf, partials, out, hdr, st);
}

template <int MODEL, typename R>
static cudaError_t energy_range_t(const void *state, const void *cmp, const ChainDesc &ch, int64_t lo, int64_t hi,
                                  const CoefD &cf, double *partials, double *out, WsHeader *hdr, cudaStream_t st) {
  k_energy_chain<MODEL, R><<<kEnergyBlocks, 256, 0, st>>>(static_cast<const R *>(state), static_cast<const R *>(cmp),
                                                          ch, lo, hi, cf.w2, cf.kappa2, partials, hdr);
  k_energy_final<<<1, 1024, 0, st>>>(partials, kEnergyBlocks, out);
  return cudaGetLastError();
}

cudaError_t launch_energy_range(int model, bool fp32, const void *state, const void *cmp, const ChainDesc &ch,
                                int64_t lo, int64_t hi, const CoefD &cf, double *partials, double *out,
                                WsHeader *hdr, cudaStream_t st) {
  if (model == ROESSLER)
    return fp32 ? energy_range_t<ROESSLER, float>(state, cmp, ch, lo, hi, cf, partials, out, hdr, st)
                : energy_range_t<ROESSLER, double>(state, cmp, ch, lo, hi, cf, partials, out, hdr, st);
  return fp32 ? energy_range_t<HARMONIC, float>(state, cmp, ch, lo, hi, cf, partials, out, hdr, st)
              : energy_range_t<HARMONIC, double>(state, cmp, ch, lo, hi, cf, partials, out, hdr, st);
}

// SplitMix64 output function (Steele, Lea and Flood, OOPSLA 2014) applied to state x.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <typename R>
__global__ void __launch_bounds__(256) k_fill_uniform(R *dst, int64_t count, uint64_t seed, uint64_t start) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < count; j += stride) {
    const uint64_t z = splitmix64(seed ^ (start + (uint64_t)j));
    const double u = (double)(z >> 11) * 0x1.0p-53;
    const double v = 2.0 * u - 1.0;  // exact
    if constexpr (sizeof(R) == 4) dst[j] = __double2float_rn(v); else dst[j] = v;
  }
}

cudaError_t launch_fill_uniform(void *dst, int64_t count, uint64_t seed, uint64_t start, bool fp32,
                                cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  int64_t grid = (count + 255) / 256;
  if (grid > (int64_t)sm_count() * 32) grid = (int64_t)sm_count() * 32;
  if (fp32)
    k_fill_uniform<float><<<(unsigned)grid, 256, 0, st>>>(static_cast<float *>(dst), count, seed, start);
  else
    k_fill_uniform<double><<<(unsigned)grid, 256, 0, st>>>(static_cast<double *>(dst), count, seed, start);
  return cudaGetLastError();
}

}  // namespace rk4d
