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
//   Roessler   kx = fma(kappa, lap, -(y + z)); ky = fma(a, y, x)
//              kz = fma(z, x, fma(-c, z, b))  FP64;  fma(z, x - c, b)  FP32
//              (Eqs. (6)-(7) of the paper, summed as in Eq. (2))
//   harmonic   kq = p;  kp = fma(kappa, lap, -(omega0^2 q))
//   stages     u2 = fma(dt/2, k1, y); u3 = fma(dt/2, k2, y); u4 = fma(dt, k3, y)   (Eq. (4))
//   update     FP64: the weighted slopes go straight into the new state (Eq. (5) term by
//              term): a = fma(dt/6, k1, y); a = fma(dt/3, k2, a); a = fma(dt/3, k3, a);
//              y = fma(dt/6, k4, a)
//              FP32-Kahan: acc = k1; acc = fma(2, k2, acc); acc = fma(2, k3, acc);
//              acc = acc + k4; s = fma(dt/6, acc, -c); t = y + s; c = (t - y) - s; y = t
// The Roessler step costs 49 floating-point instructions per site (4 x 7 slope + 9 stage +
// 12 update); FP32-Kahan 58 (4 x 7 slope + 9 stage + 9 sum + 12 update).  In FP64 only 8 of
// the 49 are additions (DADD), the rest DFMA: on GB300 a DADD takes the FP64 pipe longer than
// a DFMA, and the FP64 forms above run the step 4.7 % faster than the FP32 forms would (same
// instruction count).
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

// Coefficients of one chain in the working precision R.  h2 = dt/2, h1 = dt, dt6 = dt/6,
// dt3 = dt/3 are rounded once on the host, so every kernel sees identical constants.  one = 1,
// passed at run time: the FP64 slope issues its additions as a x one + b, the exact sum
// rounded once like a DADD, on the DFMA rate (a DADD issues at 0.84 of it; with a literal 1
// the compiler would turn the FMA back into an addition).
template <typename R> struct Coef {
  R a, b, c, kappa, w2, h2, h1, dt6, dt3, one;
};

// Slope (Eq. (3)) of one site from its stage state u and its neighbours' coupling
// coordinates xl, xr (already resolved by the boundary condition).
template <typename R, int MODEL>
__device__ __forceinline__ void slope(const R *u, R xl, R xr, const Coef<R> &cf, R *k) {
  constexpr bool kFmaAdd = sizeof(R) == 8;  // FP64: additions as DFMA (see Coef::one)
  const R lap = fma(R(-2), u[0], kFmaAdd ? fma(xl, cf.one, xr) : add(xl, xr));
  if constexpr (MODEL == ROESSLER) {
    k[0] = fma(cf.kappa, lap, -(kFmaAdd ? fma(u[1], cf.one, u[2]) : add(u[1], u[2])));
    k[1] = fma(cf.a, u[1], u[0]);
    if constexpr (sizeof(R) == 8)
      k[2] = fma(u[2], u[0], fma(-cf.c, u[2], cf.b));  // two DFMA, no DADD
    else
      k[2] = fma(u[2], sub(u[0], cf.c), cf.b);  // as slope2 (packed) computes it
  } else {
    k[0] = u[1];
    k[1] = fma(cf.kappa, lap, -mul(cf.w2, u[0]));
  }
}

// Stage j (0..3) bookkeeping after the slope k_j of a site is known: accumulate into acc and
// form the next stage state u (Eq. (4)); stage 3 finishes the step (Eq. (5)) in y (u is then
// stale: the next step's stage 0 reads y).  cmp is the Kahan compensation (ignored unless KAHAN).
// Without KAHAN, acc is the new state being accumulated (the weighted slopes added to y one by
// one); with KAHAN, the slope sum k1 + 2 k2 + 2 k3 + k4.
template <typename R, int D, bool KAHAN>
__device__ __forceinline__ void stage_update(int j, const R *k, R *y, R *u, R *acc, R *cmp, const Coef<R> &cf) {
  if constexpr (!KAHAN) {
#pragma unroll
    for (int d = 0; d < D; ++d) {
      if (j == 0) {
        acc[d] = fma(cf.dt6, k[d], y[d]);
        u[d] = fma(cf.h2, k[d], y[d]);
      } else if (j == 1) {
        acc[d] = fma(cf.dt3, k[d], acc[d]);
        u[d] = fma(cf.h2, k[d], y[d]);
      } else if (j == 2) {
        acc[d] = fma(cf.dt3, k[d], acc[d]);
        u[d] = fma(cf.h1, k[d], y[d]);
      } else {
        y[d] = fma(cf.dt6, k[d], acc[d]);
      }
    }
    return;
  }
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
      const R s = fma(cf.dt6, s4, -cmp[d]);
      const R t = add(y[d], s);
      cmp[d] = sub(sub(t, y[d]), s);
      y[d] = t;
    }
  }
}

// ---- Packed FP32: two sites per instruction --------------------------------------------
// GB300 issues FP32 add, multiply and FMA on register pairs (f32x2): one instruction performs
// the same round-to-nearest operation on both halves, at the FMA pipe's per-lane rate, with
// half the issue slots.  The FP32 kernels are issue-bound, so the tile kernels advance two
// adjacent sites (the .x and .y halves) with these forms.  Each half gets exactly the
// operation the scalar functions above perform, and negation flips the sign bits (exact,
// signed zeros included), so packed and scalar kernels stay bit-identical.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mov.b64 rc, {%6, %7};\n\tfma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 neg2(float2 a) {
  return make_float2(__uint_as_float(__float_as_uint(a.x) ^ 0x80000000u),
                     __uint_as_float(__float_as_uint(a.y) ^ 0x80000000u));
}
__device__ __forceinline__ float2 splat(float a) { return make_float2(a, a); }

// The coefficients as pairs: both halves from one chain, or from two sites (heterogeneous).
struct Coef2 {
  float2 a, b, c, kappa, w2, h2, h1, dt6;
};
__device__ __forceinline__ Coef2 pair_coef(const Coef<float> &p, const Coef<float> &q) {
  return {make_float2(p.a, q.a),         make_float2(p.b, q.b),   make_float2(p.c, q.c),
          make_float2(p.kappa, q.kappa), make_float2(p.w2, q.w2), make_float2(p.h2, q.h2),
          make_float2(p.h1, q.h1),       make_float2(p.dt6, q.dt6)};
}

// slope() on two sites.
template <int MODEL>
__device__ __forceinline__ void slope2(const float2 *u, float2 xl, float2 xr, const Coef2 &cf, float2 *k) {
  const float2 lap = fma2(splat(-2.f), u[0], add2(xl, xr));
  if constexpr (MODEL == ROESSLER) {
    k[0] = fma2(cf.kappa, lap, neg2(add2(u[1], u[2])));
    k[1] = fma2(cf.a, u[1], u[0]);
    k[2] = fma2(u[2], sub2(u[0], cf.c), cf.b);
  } else {
    k[0] = u[1];
    k[1] = fma2(cf.kappa, lap, neg2(mul2(cf.w2, u[0])));
  }
}

// stage_update() on two sites (FP32 with the Kahan update).
template <int D>
__device__ __forceinline__ void stage_update2(int j, const float2 *k, float2 *y, float2 *u, float2 *acc, float2 *cmp,
                                              const Coef2 &cf) {
#pragma unroll
  for (int d = 0; d < D; ++d) {
    if (j == 0) {
      acc[d] = k[d];
      u[d] = fma2(cf.h2, k[d], y[d]);
    } else if (j == 1) {
      acc[d] = fma2(splat(2.f), k[d], acc[d]);
      u[d] = fma2(cf.h2, k[d], y[d]);
    } else if (j == 2) {
      acc[d] = fma2(splat(2.f), k[d], acc[d]);
      u[d] = fma2(cf.h1, k[d], y[d]);
    } else {
      const float2 s4 = add2(acc[d], k[d]);
      const float2 s = fma2(cf.dt6, s4, neg2(cmp[d]));
      const float2 t = add2(y[d], s);
      cmp[d] = sub2(sub2(t, y[d]), s);
      y[d] = t;
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
