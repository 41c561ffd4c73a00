// pipe_probe.cu -- measures the arithmetic issue rates the integrator's rooflines are quoted
// against (FP64 DFMA / DADD / DMUL and a 2:1 mix, FP32 FMA issued as scalar and as packed
// f32x2 instructions) and the device copy bandwidth, and checks that a packed FMA rounds each
// half exactly like a scalar FMA.  Stand-alone program (not part of librk4chain.so); built and
// run by pipe_probe.py, it prints one JSON object.
//
// Method: every thread runs CH independent dependency chains for `iters` iterations (enough
// chains to cover the pipe latency), on a grid of `bps` blocks of 256 threads per SM; best of
// 5 runs timed with CUDA events.  The copy is a grid-stride 16-byte copy of 2 GiB.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <cuda_runtime.h>

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
         "\"packed_bit_check_values\": %d, \"copy_gbs\": %.1f}\n",
         sms, clk_khz / 1e3, dfma, dadd, dmul, dmix, d3reg, ffma8, ffma16, ffma2_4, ffma2_8, mismatches, n, best_gbs);
  free(h);
  return mismatches == 0 ? 0 : 2;
}
