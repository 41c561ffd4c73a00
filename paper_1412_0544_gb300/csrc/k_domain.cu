// k_domain.cu -- the ghost-zone exchange of the sub-domain decomposition as one gather kernel:
// every ghost zone of the domain state (and of the Kahan compensation) is copied from the
// neighbouring part's sites in a single launch, instead of one copy call per zone.
//
// A zone is `ghost` consecutive rows; rows are D x sizeof(real) bytes, a whole number of 32-bit
// words (8, 12, 16 or 24 bytes), so the kernel moves words and serves every precision and
// model.  Sources are part interiors and destinations ghost rows, which never overlap.
#include "rk4_internal.h"

namespace rk4d {

__global__ void __launch_bounds__(256) k_ghost_copy(uint32_t *a, uint32_t *b, const GhostPair *pairs, int npairs,
                                                    int64_t zone_words, int row_words) {
  const int64_t total = (int64_t)npairs * zone_words;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
    const int64_t z = e / zone_words, w = e - z * zone_words;
    const GhostPair p = pairs[z];
    const int64_t dst = p.dst_row * row_words + w, src = p.src_row * row_words + w;
    a[dst] = a[src];
    if (b) b[dst] = b[src];
  }
}

cudaError_t launch_ghost_copy(void *state, void *comp, const GhostPair *pairs, int npairs, int64_t ghost,
                              int row_bytes, cudaStream_t st) {
  if (npairs <= 0 || ghost <= 0) return cudaSuccess;
  const int row_words = row_bytes / 4;
  const int64_t zone_words = ghost * row_words;
  int64_t grid = ((int64_t)npairs * zone_words + 255) / 256;
  if (grid > (int64_t)sm_count() * 8) grid = (int64_t)sm_count() * 8;
  k_ghost_copy<<<(unsigned)grid, 256, 0, st>>>(static_cast<uint32_t *>(state), static_cast<uint32_t *>(comp), pairs,
                                               npairs, zone_words, row_words);
  return cudaGetLastError();
}

}  // namespace rk4d
