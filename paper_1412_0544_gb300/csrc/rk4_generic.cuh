// rk4_generic.cuh -- per-site arithmetic of the generic explicit Runge-Kutta scheme (any
// tableau of up to kMaxStages stages, coupling range 1 or 2).  Shared by the staged and the
// blocked generic kernels so that both perform the same operations in the same order.
#pragma once
#include "rk4_tile.cuh"

namespace rk4d {

// Largest block of the generic tile kernel (it keeps every stage slope of every site in
// registers, so the register budget of a block decides): 512 threads for FP32 with two sites
// per thread or a compiled tableau shape (at most 128 registers per thread), 256 otherwise.
template <typename R, int V, uint64_t SHAPE> struct GenBounds {
  static constexpr int threads = (sizeof(R) == 4 && (SHAPE != 0 || V == 2)) ? 512 : 256;
};
// Shared-memory values of the generic tile kernel's neighbour exchange: 2 parities x 2 pairs
// of coupling coordinates per thread of the largest block any instantiation allows.
constexpr int kGenEdgeThreads = 512;
__host__ __device__ constexpr int gen_edge_values(int v) { return (void)v, 2 * 4 * kGenEdgeThreads; }

// The tableau in the working precision: a_jm dt and b_m dt rounded once on the host, plus
// bit masks of the nonzero entries (zero entries are skipped, in every kernel alike).
template <typename R> struct Tableau {
  int s;
  R adt[kMaxStages][kMaxStages];
  R bdt[kMaxStages];
  uint32_t anz[kMaxStages];
  uint32_t bnz;
};

// The nonzero pattern of a tableau ("shape") packed into one word, for kernels compiled for a
// fixed tableau: the stage count in bits 0-2, a_jm (m < j) at bit 3 + j (j - 1) / 2 + m, b_m
// at bit 24 + m.  SHAPE = 0 reads the pattern from the tableau at run time.  Either way the
// same zero entries are skipped, so both forms perform the same operations.
__host__ __device__ constexpr uint64_t shape_a_bit(int j, int m) { return 1ull << (3 + j * (j - 1) / 2 + m); }
__host__ __device__ constexpr uint64_t shape_b_bit(int m) { return 1ull << (24 + m); }
// Stages of a compiled shape that the result needs (bit m set): nonzero weight, or used by a
// needed later stage.  The others are skipped outright, exchange included.
__host__ __device__ constexpr uint32_t shape_needed(uint64_t shape) {
  const int s = (int)(shape & 7u);
  uint32_t need = 0;
  for (int m = 0; m < s; ++m)
    if (shape & shape_b_bit(m)) need |= 1u << m;
  for (int j = s - 1; j >= 0; --j)
    if ((need >> j) & 1u)
      for (int m = 0; m < j; ++m)
        if (shape & shape_a_bit(j, m)) need |= 1u << m;
  return need;
}
template <uint64_t SHAPE> __device__ __forceinline__ constexpr bool gen_stage_needed(int j) {
  if constexpr (SHAPE != 0) return (shape_needed(SHAPE) >> j) & 1u; else return true;
}
template <uint64_t SHAPE, typename R> __device__ __forceinline__ int gen_stages(const Tableau<R> &tb) {
  if constexpr (SHAPE != 0) return (int)(SHAPE & 7u); else return tb.s;
}
template <uint64_t SHAPE, typename R> __device__ __forceinline__ bool gen_a_nonzero(const Tableau<R> &tb, int j, int m) {
  if constexpr (SHAPE != 0) return (SHAPE & shape_a_bit(j, m)) != 0; else return (tb.anz[j] >> m) & 1u;
}
template <uint64_t SHAPE, typename R> __device__ __forceinline__ bool gen_b_nonzero(const Tableau<R> &tb, int m) {
  if constexpr (SHAPE != 0) return (SHAPE & shape_b_bit(m)) != 0; else return (tb.bnz >> m) & 1u;
}

// Eq. (4): stage state of stage j from the step's start y and the earlier slopes.
template <typename R, int D, uint64_t SHAPE = 0>
__device__ __forceinline__ void gen_stage_state(int j, const Tableau<R> &tb, const R *y, const R (*k)[D], R *u) {
#pragma unroll
  for (int d = 0; d < D; ++d) u[d] = y[d];
#pragma unroll
  for (int m = 0; m < kMaxStages; ++m) {
    if (m < j && gen_a_nonzero<SHAPE>(tb, j, m)) {
#pragma unroll
      for (int d = 0; d < D; ++d) u[d] = fma(tb.adt[j][m], k[m][d], u[d]);
    }
  }
}

// Eq. (3) with coupling range 1 (the RK4 kernels' slope) or 2 (second neighbours added
// inside the coupling term).
template <typename R, int MODEL, int RANGE>
__device__ __forceinline__ void slope_gen(const R *u, R xl, R xr, R xl2, R xr2, const Coef<R> &cf, R kappa2,
                                          R *k) {
  if constexpr (RANGE == 1) {
    slope<R, MODEL>(u, xl, xr, cf, k);
  } else {
    constexpr bool kFmaAdd = sizeof(R) == 8;  // FP64: additions as DFMA (see Coef::one)
    const R lap = fma(R(-2), u[0], kFmaAdd ? fma(xl, cf.one, xr) : add(xl, xr));
    const R lap2 = fma(R(-2), u[0], kFmaAdd ? fma(xl2, cf.one, xr2) : add(xl2, xr2));
    if constexpr (MODEL == ROESSLER) {
      k[0] = fma(cf.kappa, lap, fma(kappa2, lap2, -(kFmaAdd ? fma(u[1], cf.one, u[2]) : add(u[1], u[2]))));
      k[1] = fma(cf.a, u[1], u[0]);
      if constexpr (sizeof(R) == 8)
        k[2] = fma(u[2], u[0], fma(-cf.c, u[2], cf.b));  // as slope(): two DFMA, no DADD
      else
        k[2] = fma(u[2], sub(u[0], cf.c), cf.b);
    } else {
      k[0] = u[1];
      k[1] = fma(cf.kappa, lap, fma(kappa2, lap2, -mul(cf.w2, u[0])));
    }
  }
}

// Eq. (5): y += sum_m b_m dt k_m, in FP64 or with a Kahan-compensated update in FP32.
template <typename R, int D, bool KAHAN, uint64_t SHAPE = 0>
__device__ __forceinline__ void gen_combine(const Tableau<R> &tb, const R (*k)[D], R *y, R *cmp) {
#pragma unroll
  for (int d = 0; d < D; ++d) {
    R inc = R(0);
#pragma unroll
    for (int m = 0; m < kMaxStages; ++m)
      if (m < gen_stages<SHAPE>(tb) && gen_b_nonzero<SHAPE>(tb, m)) inc = fma(tb.bdt[m], k[m][d], inc);
    if constexpr (KAHAN) {
      const R s = sub(inc, cmp[d]);
      const R t = add(y[d], s);
      cmp[d] = sub(sub(t, y[d]), s);
      y[d] = t;
    } else {
      y[d] = add(y[d], inc);
    }
  }
}

}  // namespace rk4d
