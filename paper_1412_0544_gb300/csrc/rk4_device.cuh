// rk4_device.cuh -- the per-site arithmetic every GPU scheme shares.
//
// All kernels (staged, blocked, persistent) call these functions and nothing else for the
// integrator's floating-point work, so each site runs the same operations in the same order
// with the same rounding, whatever the tiling: the blocked and persistent kernels are
// bit-identical to the one-stage-per-launch kernel.  Every operation is an explicit
// round-to-nearest intrinsic, so the compiler cannot contract or reorder differently in
// different kernels.
//
// Operation order (fixed):
//   coupling   lap = fma(-2, x_i, x_{i-1} + x_{i+1})       (symmetric in the neighbours)
//   Roessler   kx = fma(kappa, lap, -(y + z)); ky = fma(a, y, x); kz = fma(z, x - c, b)
//              (Eqs. (6)-(7) of the paper, summed as in Eq. (2))
//   harmonic   kq = p;  kp = fma(kappa, lap, -(omega0^2 q))
//   stages     u2 = fma(dt/2, k1, y); u3 = fma(dt/2, k2, y); u4 = fma(dt, k3, y)   (Eq. (4))
//   sum        acc = k1; acc = fma(2, k2, acc); acc = fma(2, k3, acc); acc = acc + k4
//   update     FP64:      y = fma(dt/6, acc, y)                                        (Eq. (5))
//              FP32-Kahan: s = fma(dt/6, acc, -c); t = y + s; c = (t - y) - s; y = t
// The Roessler step costs 49 floating-point instructions per site (4 x 7 slope + 9 stage +
// 9 sum + 3 update), 61 with the Kahan update.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace rk4d {

enum { ROESSLER = 0, HARMONIC = 1 };
enum { PERIODIC = 0, FIXED = 1 };

template <int MODEL> struct Dim;
template <> struct Dim<ROESSLER> { static constexpr int D = 3; static constexpr int P = 4; };
template <> struct Dim<HARMONIC> { static constexpr int D = 2; static constexpr int P = 2; };
// P: parameters per site of a heterogeneous chain (Eq. (1) of the paper): Roessler a, b, c,
// kappa; harmonic omega^2, kappa.

__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// Coefficients of one chain in the working precision R.  h2 = dt/2, h1 = dt, dt6 = dt/6 are
// rounded once on the host, so every kernel sees identical constants.
template <typename R> struct Coef {
  R a, b, c, kappa, w2, h2, h1, dt6;
};

// Slope (Eq. (3)) of one site from its stage state u and its neighbours' coupling
// coordinates xl, xr (already resolved by the boundary condition).
template <typename R, int MODEL>
__device__ __forceinline__ void slope(const R *u, R xl, R xr, const Coef<R> &cf, R *k) {
  const R lap = fma(R(-2), u[0], add(xl, xr));
  if constexpr (MODEL == ROESSLER) {
    k[0] = fma(cf.kappa, lap, -add(u[1], u[2]));
    k[1] = fma(cf.a, u[1], u[0]);
    k[2] = fma(u[2], sub(u[0], cf.c), cf.b);
  } else {
    k[0] = u[1];
    k[1] = fma(cf.kappa, lap, -mul(cf.w2, u[0]));
  }
}

// Stage j (0..3) bookkeeping after the slope k_j of a site is known: accumulate into acc and
// form the next stage state u (Eq. (4)); stage 3 finishes the step (Eq. (5)) in y (u is then
// stale: the next step's stage 0 reads y).  cmp is the Kahan compensation (ignored unless KAHAN).
template <typename R, int D, bool KAHAN>
__device__ __forceinline__ void stage_update(int j, const R *k, R *y, R *u, R *acc, R *cmp, const Coef<R> &cf) {
#pragma unroll
  for (int d = 0; d < D; ++d) {
    if (j == 0) {
      acc[d] = k[d];
      u[d] = fma(cf.h2, k[d], y[d]);
    } else if (j == 1) {
      acc[d] = fma(R(2), k[d], acc[d]);
      u[d] = fma(cf.h2, k[d], y[d]);
    } else if (j == 2) {
      acc[d] = fma(R(2), k[d], acc[d]);
      u[d] = fma(cf.h1, k[d], y[d]);
    } else {
      const R s4 = add(acc[d], k[d]);
      if constexpr (KAHAN) {
        const R s = fma(cf.dt6, s4, -cmp[d]);
        const R t = add(y[d], s);
        cmp[d] = sub(sub(t, y[d]), s);
        y[d] = t;
      } else {
        y[d] = fma(cf.dt6, s4, y[d]);
      }
    }
  }
}

// Coefficients of one site of a heterogeneous chain: the chain's coefficients with the
// site's own parameters p[0..P-1] substituted.
template <typename R, int MODEL>
__device__ __forceinline__ Coef<R> site_coef(const Coef<R> &cf, const R *p) {
  Coef<R> c = cf;
  if constexpr (MODEL == ROESSLER) {
    c.a = p[0];
    c.b = p[1];
    c.c = p[2];
    c.kappa = p[3];
  } else {
    c.w2 = p[0];
    c.kappa = p[1];
  }
  return c;
}

// Positive modulus for periodic index wrapping.
__device__ __forceinline__ int64_t wrap(int64_t g, int64_t n) {
  int64_t r = g % n;
  return r < 0 ? r + n : r;
}

}  // namespace rk4d
