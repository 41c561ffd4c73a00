// pipe_probe.cu -- measures the arithmetic issue rates the integrator's rooflines are quoted
// against (FP64 DFMA / DADD / DMUL and a 2:1 mix, FP32 FMA issued as scalar and as packed
// f32x2 instructions), the device copy bandwidth and the rate of the integrator's own RK4
// arithmetic on register-resident sites (FP64, packed FP32-Kahan), and checks that a packed
// FMA rounds each half exactly like a scalar FMA.  Stand-alone program (not part of
// librk4chain.so); built and run by pipe_probe.py, it prints one JSON object.
//
// Method: every thread runs CH independent dependency chains for `iters` iterations (enough
// chains to cover the pipe latency), on a grid of `bps` blocks of 256 threads per SM; best of
// 5 runs timed with CUDA events.  The copy is a grid-stride 16-byte copy of 2 GiB.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <cuda_runtime.h>

#include "paper_1412_0544_gb300/csrc/rk4_device.cuh"

#define CK(x)                                                                      \
  do {                                                                             \
    cudaError_t e_ = (x);                                                          \
    if (e_ != cudaSuccess) {                                                       \
      fprintf(stderr, "%s failed: %s\n", #x, cudaGetErrorString(e_));              \
      exit(1);                                                                     \
    }                                                                              \
  } while (0)

__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mov.b64 rc, {%6, %7};\n\tfma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}

// MODE 0 DFMA, 1 DADD, 2 DMUL, 3 two DFMA + one DADD; results are consumed only through a
// comparison that never holds, so nothing is stored.
template <int MODE, int CH>
__global__ void fp64_chain(double *out, int iters, double a, double b) {
  double acc[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) acc[c] = threadIdx.x + c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      if (MODE == 0) acc[c] = __fma_rn(acc[c], a, b);
      else if (MODE == 1) acc[c] = __dadd_rn(acc[c], b);
      else if (MODE == 2) acc[c] = __dmul_rn(acc[c], a);
      else {
        acc[c] = __fma_rn(acc[c], a, b);
        acc[c] = __fma_rn(acc[c], a, b);
        acc[c] = __dadd_rn(acc[c], b);
      }
    }
  }
  double s = 0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += acc[c];
  if (s == -12345.0) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// DFMA whose three operands are all per-chain registers that change every iteration (the form
// of most DFMAs in the RK4 step), against the chains above, whose multiplier and addend are
// loop-invariant.  Three coupled chains per group: x = x*y + z, y = y*z + x, z = z*x + y.
template <int G>
__global__ void fp64_3reg(double *out, int iters, double a, double b) {
  double x[G], y[G], z[G];
#pragma unroll
  for (int g = 0; g < G; ++g) {
    x[g] = 1.0 + 1e-9 * (threadIdx.x + g);
    y[g] = a;
    z[g] = b;
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int g = 0; g < G; ++g) {
      x[g] = __fma_rn(x[g], y[g], z[g]);
      y[g] = __fma_rn(y[g], z[g], x[g]);
      z[g] = __fma_rn(z[g], x[g], y[g]);
    }
  }
  double s = 0;
#pragma unroll
  for (int g = 0; g < G; ++g) s += x[g] + y[g] + z[g];
  if (s == -12345.0) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int CH>
__global__ void fp32_chain(double *out, int iters, double a, double b) {
  const float fa = (float)a, fb = (float)b;
  float acc[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) acc[c] = (float)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CH; ++c) acc[c] = __fmaf_rn(acc[c], fa, fb);
  }
  float s = 0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += acc[c];
  if (s == -12345.0f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int CH>  // CH register pairs: 2 CH FMA lanes per thread and iteration
__global__ void fp32x2_chain(double *out, int iters, double a, double b) {
  const float2 fa = make_float2((float)a, (float)a), fb = make_float2((float)b, (float)b);
  float2 acc[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) acc[c] = make_float2((float)(threadIdx.x + 2 * c), (float)(threadIdx.x + 2 * c + 1));
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CH; ++c) acc[c] = fma2(acc[c], fa, fb);
  }
  float s = 0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += acc[c].x + acc[c].y;
  if (s == -12345.0f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Packed against scalar FMA on n (even) values per operand; counts halves that differ in any bit.
__global__ void packed_bit_check(const float *a, const float *b, const float *c, int n, int *bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (2 * i + 1 >= n) return;
  const float2 r = fma2(make_float2(a[2 * i], a[2 * i + 1]), make_float2(b[2 * i], b[2 * i + 1]),
                        make_float2(c[2 * i], c[2 * i + 1]));
  const float s0 = __fmaf_rn(a[2 * i], b[2 * i], c[2 * i]);
  const float s1 = __fmaf_rn(a[2 * i + 1], b[2 * i + 1], c[2 * i + 1]);
  if (__float_as_uint(r.x) != __float_as_uint(s0) || __float_as_uint(r.y) != __float_as_uint(s1)) atomicAdd(bad, 1);
}

// The integrator's own arithmetic stream without memory traffic: the RK4 step of the Roessler
// chain (the slope and stage functions every tile kernel calls) on 4 register-resident sites
// per thread, each site's neighbours taken from the thread's own registers -- no loads,
// no neighbour exchange, no barrier.  Its rate is the most the tile kernels' instruction mix
// can reach; the tile kernels' distance from it is the cost of everything else.  The
// coefficients derive from the run-time arguments, so nothing folds at compile time.
// ROUNDTRIP: every stage each thread also stores its two edge values to shared memory and,
// after a barrier, reads them back as its neighbours -- the same values and arithmetic, plus
// the shared-memory traffic and barrier a tile kernel's neighbour exchange has.
template <int V, bool ROUNDTRIP = false>
__global__ void rk4_regs_fp64(double *out, int iters, double a, double b) {
  constexpr int D = 3;
  __shared__ double slot[ROUNDTRIP ? 2 * 2 * 256 : 1];
  const int tid = threadIdx.x;
  // one = 1 at run time (a - a = 0 for the finite argument), as the library passes it
  const rk4d::Coef<double> cf{0.2 * a, 1.0 * a, 9.0 * a, a, 1.0, 0.005 * a, 0.01 * a, 0.01 * a / 6.0, 0.01 * a / 3.0,
                              1.0 + (a - a)};
  double y[V][D], u[V][D], acc[V][D], cmp[V][D];
#pragma unroll
  for (int v = 0; v < V; ++v)
#pragma unroll
    for (int d = 0; d < D; ++d) {
      y[v][d] = 0.1 * (d + 1) + 1e-3 * (threadIdx.x + v) + b;
      cmp[v][d] = 0.0;
    }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      double xs[V];
#pragma unroll
      for (int v = 0; v < V; ++v) xs[v] = (j == 0) ? y[v][0] : u[v][0];
      double left = xs[V - 1], right = xs[0];
      if constexpr (ROUNDTRIP) {
        double *eb = slot + (j & 1) * 2 * 256;
        eb[tid] = xs[0];
        eb[256 + tid] = xs[V - 1];
        __syncthreads();
        left = eb[256 + tid];
        right = eb[tid];
      }
#pragma unroll
      for (int v = 0; v < V; ++v) {
        double k[D];
        rk4d::slope<double, rk4d::ROESSLER>((j == 0) ? y[v] : u[v], v == 0 ? left : xs[v - 1],
                                            v == V - 1 ? right : xs[v + 1], cf, k);
        rk4d::stage_update<double, D, false>(j, k, y[v], u[v], acc[v], cmp[v], cf);
      }
    }
  }
  double s = 0;
#pragma unroll
  for (int v = 0; v < V; ++v) s += y[v][0] + y[v][1] + y[v][2];
  if (s == -12345.0) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// The same for the FP32-Kahan step on packed f32x2 instructions (two sites per instruction).
template <int V>
__global__ void rk4_regs_fp32k(double *out, int iters, double a, double b) {
  constexpr int D = 3;
  const float fa = (float)a;
  const rk4d::Coef<float> c1{0.2f * fa, 1.0f * fa, 9.0f * fa, fa, 1.0f, 0.005f * fa, 0.01f * fa, 0.01f * fa / 6.0f,
                             0.01f * fa / 3.0f, 1.0f};
  const rk4d::Coef2 cf = rk4d::pair_coef(c1, c1);
  float2 y[V / 2][D], u[V / 2][D], acc[V / 2][D], cmp[V / 2][D];
#pragma unroll
  for (int p = 0; p < V / 2; ++p)
#pragma unroll
    for (int d = 0; d < D; ++d) {
      y[p][d] = make_float2(0.1f * (d + 1) + 1e-3f * (threadIdx.x + 2 * p) + (float)b,
                            0.1f * (d + 1) + 1e-3f * (threadIdx.x + 2 * p + 1) + (float)b);
      cmp[p][d] = make_float2(0.f, 0.f);
    }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float xs[V];
#pragma unroll
      for (int p = 0; p < V / 2; ++p) {
        const float2 x = (j == 0) ? y[p][0] : u[p][0];
        xs[2 * p] = x.x;
        xs[2 * p + 1] = x.y;
      }
#pragma unroll
      for (int p = 0; p < V / 2; ++p) {
        const int v = 2 * p;
        const float2 xl = make_float2(xs[(v + V - 1) % V], xs[v]);
        const float2 xr = make_float2(xs[v + 1], xs[(v + 2) % V]);
        float2 k[D];
        rk4d::slope2<rk4d::ROESSLER>((j == 0) ? y[p] : u[p], xl, xr, cf, k);
        rk4d::stage_update2<D>(j, k, y[p], u[p], acc[p], cmp[p], cf);
      }
    }
  }
  float s = 0;
#pragma unroll
  for (int p = 0; p < V / 2; ++p) s += y[p][0].x + y[p][1].y + y[p][2].x + cmp[p][0].y;
  if (s == -12345.0f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void copy16(const int4 *__restrict__ a, int4 *__restrict__ b, size_t n) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride) b[i] = a[i];
}

typedef void (*ChainKernel)(double *, int, double, double);

// Best-of-5 rate in operations per second; ops = lanes x iterations x ops per iteration.
static double rate(ChainKernel k, int sms, int iters, double ops_per_thread_iter, double *out) {
  const int bps = 4, threads = 256;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  k<<<sms * bps, threads>>>(out, iters, 0.999999, 1e-7);
  CK(cudaGetLastError());
  CK(cudaDeviceSynchronize());
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    CK(cudaEventRecord(e0));
    k<<<sms * bps, threads>>>(out, iters, 0.999999, 1e-7);
    CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best) best = ms;
  }
  CK(cudaEventDestroy(e0));
  CK(cudaEventDestroy(e1));
  return (double)sms * bps * threads * iters * ops_per_thread_iter / (best * 1e-3);
}

int main() {
  int dev = 0, sms = 0, clk_khz = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
  double *out = nullptr;
  CK(cudaMalloc(&out, sizeof(double) * sms * 4 * 256));
  const double dfma = rate(fp64_chain<0, 8>, sms, 4096, 8, out);
  const double dadd = rate(fp64_chain<1, 8>, sms, 4096, 8, out);
  const double dmul = rate(fp64_chain<2, 8>, sms, 4096, 8, out);
  const double dmix = rate(fp64_chain<3, 8>, sms, 2048, 24, out);
  const double d3reg = rate(fp64_3reg<8>, sms, 2048, 24, out);
  const double ffma8 = rate(fp32_chain<8>, sms, 1 << 16, 8, out);
  const double ffma16 = rate(fp32_chain<16>, sms, 1 << 16, 16, out);
  const double ffma2_4 = rate(fp32x2_chain<4>, sms, 1 << 16, 8, out);
  const double ffma2_8 = rate(fp32x2_chain<8>, sms, 1 << 16, 16, out);
  // per thread and iteration: 4 sites x 49 FP64 instructions; 4 sites x 58 FP32 lane-ops
  const double rk4_fp64 = rate(rk4_regs_fp64<4>, sms, 512, 4 * 49, out);
  const double rk4_fp64_rt = rate(rk4_regs_fp64<4, true>, sms, 512, 4 * 49, out);
  const double rk4_fp32k = rate(rk4_regs_fp32k<4>, sms, 4096, 4 * 58, out);
  // twice the independent site pairs per thread: how much of the stream's gap to the FMA rate is
  // dependency latency rather than the operation mix
  const double rk4_fp32k_v8 = rate(rk4_regs_fp32k<8>, sms, 2048, 8 * 58, out);

  // bit check on 2^20 operands per input, spread over many binades and both signs
  const int n = 1 << 20;
  float *h = static_cast<float *>(malloc(sizeof(float) * 3 * n));
  unsigned s = 12345u;
  for (int i = 0; i < 3 * n; ++i) {
    s = s * 1664525u + 1013904223u;
    const unsigned e = 100u + (s >> 27), m = (s * 2654435761u) & 0x7fffffu;
    const unsigned u = ((s & 1u) << 31) | (e << 23) | m;
    memcpy(&h[i], &u, sizeof(u));
  }
  float *d = nullptr;
  int *bad = nullptr;
  CK(cudaMalloc(&d, sizeof(float) * 3 * n));
  CK(cudaMalloc(&bad, sizeof(int)));
  CK(cudaMemcpy(d, h, sizeof(float) * 3 * n, cudaMemcpyHostToDevice));
  CK(cudaMemset(bad, 0, sizeof(int)));
  packed_bit_check<<<(n / 2 + 255) / 256, 256>>>(d, d + n, d + 2 * n, n, bad);
  CK(cudaGetLastError());
  int mismatches = -1;
  CK(cudaMemcpy(&mismatches, bad, sizeof(int), cudaMemcpyDeviceToHost));

  // copy bandwidth: 2 GiB read + 2 GiB written
  const size_t bytes = (size_t)2 << 30, nv = bytes / 16;
  int4 *a = nullptr, *b = nullptr;
  CK(cudaMalloc(&a, bytes));
  CK(cudaMalloc(&b, bytes));
  CK(cudaMemset(a, 0, bytes));
  CK(cudaMemset(b, 0, bytes));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  double best_gbs = 0.0;
  const int grids[3] = {sms * 4, sms * 8, sms * 16};
  for (int g : grids) {
    copy16<<<g, 512>>>(a, b, nv);
    CK(cudaDeviceSynchronize());
    for (int r = 0; r < 5; ++r) {
      CK(cudaEventRecord(e0));
      copy16<<<g, 512>>>(a, b, nv);
      CK(cudaEventRecord(e1));
      CK(cudaEventSynchronize(e1));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      const double gbs = 2.0 * bytes / (ms * 1e-3) / 1e9;
      if (gbs > best_gbs) best_gbs = gbs;
    }
  }
  printf("{\"sms\": %d, \"max_sm_clock_mhz\": %.0f, \"dfma_per_s\": %.5g, \"dadd_per_s\": %.5g, "
         "\"dmul_per_s\": %.5g, \"dfma2_dadd1_mix_per_s\": %.5g, \"dfma_3reg_per_s\": %.5g, "
         "\"ffma_scalar_8chains_per_s\": %.5g, "
         "\"ffma_scalar_16chains_per_s\": %.5g, \"ffma_packed_8lanes_per_s\": %.5g, "
         "\"ffma_packed_16lanes_per_s\": %.5g, \"packed_vs_scalar_fma_mismatches\": %d, "
         "\"packed_bit_check_values\": %d, \"copy_gbs\": %.1f, \"rk4_fp64_regs_inst_per_s\": %.5g, "
         "\"rk4_fp32k_regs_lane_ops_per_s\": %.5g, \"rk4_fp32k_regs_v8_lane_ops_per_s\": %.5g, "
         "\"rk4_fp64_regs_smem_roundtrip_inst_per_s\": %.5g}\n",
         sms, clk_khz / 1e3, dfma, dadd, dmul, dmix, d3reg, ffma8, ffma16, ffma2_4, ffma2_8, mismatches, n, best_gbs,
         rk4_fp64, rk4_fp32k, rk4_fp32k_v8, rk4_fp64_rt);
  free(h);
  return mismatches == 0 ? 0 : 2;
}
