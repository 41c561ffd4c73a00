// k_copy.cu -- host <-> device copies of rk4_chain_integrate_host carried out by the SMs.
//
// Page-locked host memory is mapped into the device's address space, so a kernel can read
// and write it directly (over the CPU-GPU link).  On GB300 this moves the 3.2 GB state of a
// 2^27-site chain at the link's rate in either direction, while a copy-engine transfer
// (cudaMemcpyAsync) issued right after a long compute phase was measured at 9-14 GB/s instead
// of its idle 190-210 GB/s.  The kernel copies 16-byte vectors (both pointers 16-byte aligned,
// which the ABI requires of state buffers) and the remaining bytes singly.
#include "rk4_internal.h"

namespace rk4d {

__global__ void __launch_bounds__(512) k_copy(int4 *__restrict__ dst, const int4 *__restrict__ src, int64_t n16,
                                              unsigned char *__restrict__ dtail, const unsigned char *__restrict__ stail,
                                              int tail) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) dst[i] = src[i];
  if (blockIdx.x == 0 && (int)threadIdx.x < tail) dtail[threadIdx.x] = stail[threadIdx.x];
}

cudaError_t launch_copy(void *dst, const void *src, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return cudaSuccess;
  if ((reinterpret_cast<uintptr_t>(dst) & 15u) || (reinterpret_cast<uintptr_t>(src) & 15u))
    return cudaErrorInvalidValue;
  const int64_t n16 = (int64_t)(bytes / 16);
  const int tail = (int)(bytes % 16);
  int64_t grid = (n16 + 511) / 512;
  if (grid > (int64_t)sm_count() * 8) grid = (int64_t)sm_count() * 8;
  if (grid < 1) grid = 1;
  k_copy<<<(unsigned)grid, 512, 0, st>>>(static_cast<int4 *>(dst), static_cast<const int4 *>(src), n16,
                                        static_cast<unsigned char *>(dst) + n16 * 16,
                                        static_cast<const unsigned char *>(src) + n16 * 16, tail);
  return cudaGetLastError();
}

}  // namespace rk4d
