// k_staged.cu -- the paper's "standard implementation" (Sec. 2.2) on the GPU: one launch per
// RK stage, each a full sweep over every site.  It is the bit-identity reference for the
// blocked and persistent kernels (all three call the same per-site functions).
#include "rk4_tile.cuh"

namespace rk4d {

template <typename R, int MODEL, bool KAHAN>
__global__ void __launch_bounds__(256) k_staged(StagedJob job, Coef<R> cf, int j) {
  constexpr int D = Dim<MODEL>::D;
  R *Y = static_cast<R *>(job.y);
  R *CMP = static_cast<R *>(job.cmp);
  const R *src = (j == 0) ? Y : static_cast<const R *>(job.uin);
  R *UOUT = static_cast<R *>(job.uout);
  R *ACC = static_cast<R *>(job.acc);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < job.total; i += stride) {
    ChainDesc ch;
    Coef<R> c = cf;
    if (job.nchains == 1) {
      ch = job.one;
    } else {
      int lo = 0, hi = job.nchains - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (job.chains[mid].off <= i) lo = mid; else hi = mid - 1;
      }
      ch = job.chains[lo];
      c.kappa = (R)ch.kappa;
    }
    if (job.sp) c = site_coef<R, MODEL>(c, static_cast<const R *>(job.sp) + i * Dim<MODEL>::P);  // Eq. (1)
    const int64_t li = i - ch.off;  // index within the chain
    R u[D], y[D], acc[D], cmp[D], k[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      u[d] = src[i * D + d];
      y[d] = Y[i * D + d];
      acc[d] = (j > 0) ? ACC[i * D + d] : R(0);
      cmp[d] = (KAHAN && j == 3) ? CMP[i * D + d] : R(0);
    }
    R xl, xr;
    if (ch.bc == PERIODIC) {
      const int64_t il = (li == 0) ? ch.n - 1 : li - 1;
      const int64_t ir = (li == ch.n - 1) ? 0 : li + 1;
      if (!bounds_ok(job.hdr, in_range(ch.off + il, 1, job.total) && in_range(ch.off + ir, 1, job.total))) continue;
      xl = src[(ch.off + il) * D];
      xr = src[(ch.off + ir) * D];
    } else {
      if (!bounds_ok(job.hdr, in_range(li, 1, ch.n))) continue;
      xl = (li == 0) ? R(0) : src[(i - 1) * D];
      xr = (li == ch.n - 1) ? R(0) : src[(i + 1) * D];
    }
    slope<R, MODEL>(u, xl, xr, c, k);
    stage_update<R, D, KAHAN>(j, k, y, u, acc, cmp, c);
    if (j < 3) {
#pragma unroll
      for (int d = 0; d < D; ++d) {
        UOUT[i * D + d] = u[d];
        ACC[i * D + d] = acc[d];
      }
    } else {
      bool bad = false;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        Y[i * D + d] = y[d];
        if constexpr (KAHAN) CMP[i * D + d] = cmp[d];
        bad |= nonfinite(y[d]);
      }
      if (bad && job.hdr) atomicOr(&job.hdr->status, ST_NONFINITE);
    }
  }
}

template <typename R, int MODEL, bool KAHAN>
static cudaError_t launch_one(int j, const StagedJob &job, const CoefD &cfd, cudaStream_t st) {
  if (job.total <= 0) return cudaSuccess;
  const int block = 256;
  int64_t grid = (job.total + block - 1) / block;
  if (grid > (int64_t)sm_count() * 64) grid = (int64_t)sm_count() * 64;
  k_staged<R, MODEL, KAHAN><<<(unsigned)grid, block, 0, st>>>(job, to_coef<R>(cfd, cfd.kappa), j);
  return cudaGetLastError();
}

cudaError_t launch_staged(int model, bool fp32, int j, const StagedJob &job, const CoefD &cf, cudaStream_t st) {
  if (model == ROESSLER)
    return fp32 ? launch_one<float, ROESSLER, true>(j, job, cf, st) : launch_one<double, ROESSLER, false>(j, job, cf, st);
  return fp32 ? launch_one<float, HARMONIC, true>(j, job, cf, st) : launch_one<double, HARMONIC, false>(j, job, cf, st);
}

}  // namespace rk4d
