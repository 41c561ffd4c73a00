// rk4_internal.h -- structures shared by the host runtime and the kernels' launchers.
// Not part of the public ABI (see include/rk4chain.h).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <mutex>

namespace rk4d {

// One chain of a (possibly single-chain) job.  32 bytes, stored in the workspace for batches.
struct ChainDesc {
  int64_t off;   // first site of the chain in the concatenated state
  int64_t n;     // sites
  double kappa;  // coupling strength
  int32_t bc;    // PERIODIC or FIXED
  int32_t pad;
};

// Coefficients in double; converted to the working precision once per launch on the host.
// kappa2: second-neighbour coupling (generic scheme only; 0 for the paper's chain).
struct CoefD {
  double a, b, c, kappa, w2, h2, h1, dt6, kappa2, dt3;
};

// Generic explicit Runge-Kutta tableau (strictly lower a, weights b), up to kMaxStages stages.
constexpr int kMaxStages = 7;
struct TableauD {
  int s;
  double a[kMaxStages][kMaxStages];
  double b[kMaxStages];
};

// Device status word bits (in the workspace header).  ST_BOUNDS is only ever set by a library
// built with -DRK4_DEBUG_BOUNDS (index checks on every global access; see rk4_tile.cuh).
enum : int { ST_NONFINITE = 1, ST_TIMEOUT = 2, ST_BOUNDS = 4 };

// Workspace header: status word, grid-barrier counters.  256 bytes.
struct WsHeader {
  int status;
  unsigned bar_count;
  unsigned bar_gen;
  int timeout_where;
  unsigned long long work[2];  // persistent kernel: next item of the current time block, by parity
  unsigned char pad[224];
};

// A piece of one batch chain placed in a shared ("packed") tile: the chain's last partial piece
// of interior sites (or the whole chain when it is shorter than a tile's interior), with its own
// halo of H sites on each side.  Several segments lie side by side in one tile; each thread's
// sites belong to one segment because o and L are multiples of the sites per thread.
struct SegDesc {
  int64_t g0;     // first interior site (chain-local index)
  int32_t chain;  // index into the chain table
  int32_t o;      // first tile slot of the segment's window
  int32_t cnt;    // interior sites
  int32_t L;      // window length in slots: H + cnt + H rounded up to a multiple of the sites per thread
};

// The tiles of one launch over a batch: the full tiles (G interior sites each) of every chain,
// numbered chain by chain (full_prefix: first full tile of each chain, nchains + 1 entries),
// and the packed tiles (pack_prefix: first segment of each packed tile, npacked + 1 entries,
// into segs).  The kernels process the packed tiles first.  A chain of n sites has
// floor(n / G) full tiles and, when G does not divide n, one segment.
// tile_chain, when not null, holds for each full tile its chain and chain-local tile index
// (filled on the device from full_prefix before the launches), so that a tile finds its chain
// with one load instead of a search of full_prefix.
struct BatchTiles {
  const int32_t *full_prefix;
  const int32_t *pack_prefix;
  const SegDesc *segs;
  const int2 *tile_chain;
  int64_t nfull;
  int64_t npacked;
};

// Arguments of one blocked launch (one chain, or a batch through a chain table).
struct BlockedJob {
  const void *in;    // state read by this launch
  void *out;         // state written by this launch
  const void *cin;   // Kahan compensation read (FP32) or NULL
  void *cout;        // Kahan compensation written
  int nchains;       // 1: use `one`; >1: use `chains` / `bt`
  ChainDesc one;
  const ChainDesc *chains;      // device table (batches)
  BatchTiles bt;                // batches: the tiles of the launch (full_prefix counts every tile
                                // of a chain when the batch is not packed)
  int packed;                   // 1: packed tiles (bt.npacked of them) precede the full tiles
  int K;                        // steps in this launch
  int G;                        // interior sites per tile
  int64_t ntiles;               // tiles in the launch (a packed batch: its full tiles, beside bt.npacked)
  const void *sp;               // per-site parameters of a heterogeneous chain, or NULL
  WsHeader *hdr;                // status word (non-finite results, debug bounds checks)
  int64_t total;                // sites in the state buffers
};

struct StagedJob {
  void *y;            // state, updated in place at the last stage
  void *cmp;          // Kahan compensation (FP32) or NULL, updated in place
  const void *uin;    // stage state read (stages 1..3)
  void *uout;         // stage state written (stages 0..2)
  void *acc;          // slope sum
  int nchains;
  ChainDesc one;
  const ChainDesc *chains;   // device table for batches (site -> chain by binary search)
  int64_t total;             // total sites
  const void *sp;            // per-site parameters of a heterogeneous chain, or NULL
  WsHeader *hdr;             // status word
};

// One step of the generic standard scheme: stage states, slopes and the combination, each a
// full sweep.  k holds s slope arrays of total * D values; u one stage state.
struct GenStagedJob {
  void *y;
  void *cmp;
  void *u;
  void *k;
  int nchains;
  ChainDesc one;
  const ChainDesc *chains;
  int64_t total;
  WsHeader *hdr;  // status word
};

struct PersistentJob {
  void *bufA, *bufB;            // state ping-pong: time block t reads A when t is even
  void *cA, *cB;                // compensation ping-pong (FP32) or NULL
  int nchains;
  ChainDesc one;
  const ChainDesc *chains;
  BatchTiles bt[4];             // batches: the tiles of a time block for each k (full, then packed)
  int nk;                       // distinct k values (1..4)
  int kval[4];                  // steps per time block
  int Gval[4];                  // interior sites per tile for each k
  int64_t ntiles[4];            // tiles per time block for each k
  int64_t nmain;                // leading time blocks that use kval[0]
  int ntail;                    // trailing time blocks (0..3)
  int tail[3];                  // their indices into kval
  WsHeader *hdr;                // status word and barrier counters (zeroed before launch)
  long long timeout_ns;         // bound on any single barrier wait
  int extra_arrivals;           // test hook: barrier waits for this many blocks that never come
  int64_t total;                // sites in the state buffers
};

// Launchers (return a cudaError_t).  R is selected by `fp32` (FP32 + Kahan) or double.
cudaError_t launch_blocked(int model, bool fp32, int v, int block, const BlockedJob &job, const CoefD &cf,
                           cudaStream_t st);  // job.sp != NULL selects the heterogeneous kernel (v = 2 or 4)
cudaError_t launch_staged(int model, bool fp32, int stage, const StagedJob &job, const CoefD &cf,
                          cudaStream_t st);
cudaError_t launch_persistent(int model, bool fp32, int v, int block, int grid, const PersistentJob &job,
                              const CoefD &cf, cudaStream_t st);
int persistent_max_grid(int model, bool fp32, int v, int block);
cudaError_t launch_energy(int model, bool fp32, const void *state, const void *cmp, int nchains,
                          const ChainDesc &one, const ChainDesc *chains, const CoefD &cf, double *partials,
                          double *out, WsHeader *hdr, cudaStream_t st);
// Energy of the chain-local sites [lo, hi) of one chain; neighbours outside the range are read
// from the state like any other site (a sub-domain's ghost zones).  out: one device double.
cudaError_t launch_energy_range(int model, bool fp32, const void *state, const void *cmp, const ChainDesc &ch,
                                int64_t lo, int64_t hi, const CoefD &cf, double *partials, double *out,
                                WsHeader *hdr, cudaStream_t st);
// One ghost zone of a sub-domain state: `ghost` rows starting at dst_row are copied from the
// rows starting at src_row.
struct GhostPair {
  int64_t dst_row, src_row;
};
// Every zone of `pairs` (a device table) in one launch, for the state and, if not NULL, the
// compensation; rows are row_bytes (a multiple of 4) long.
cudaError_t launch_ghost_copy(void *state, void *comp, const GhostPair *pairs, int npairs, int64_t ghost,
                              int row_bytes, cudaStream_t st);
// Copy `bytes` between two 16-byte-aligned buffers with a kernel (either side may be mapped
// page-locked host memory, given by its device pointer).
cudaError_t launch_copy(void *dst, const void *src, size_t bytes, cudaStream_t st);
// Fill tile_chain[t] = (chain, t - prefix[chain]) for the ntiles tiles numbered by prefix
// (nchains + 1 entries, the first tile of each chain).
cudaError_t launch_tile_chains(const int32_t *prefix, int nchains, int64_t ntiles, int2 *tile_chain, cudaStream_t st);
cudaError_t launch_fill_uniform(void *dst, int64_t count, uint64_t seed, uint64_t start, bool fp32,
                                cudaStream_t st);
cudaError_t launch_gen_staged_step(int model, bool fp32, int range, const GenStagedJob &job, const CoefD &cf,
                                   const TableauD &tb, double dt, cudaStream_t st);
cudaError_t launch_gen_blocked(int model, bool fp32, int range, int v, int block, const BlockedJob &job,
                               const CoefD &cf, const TableauD &tb, double dt, int H, cudaStream_t st);
size_t gen_blocked_smem_bytes(int model, bool fp32, int v, int block, const TableauD &tb);
int gen_blocked_max_threads(int model, bool fp32, int range, int v, const TableauD &tb);
size_t blocked_smem_bytes(int model, bool fp32, int v, int block, bool het = false);
int blocked_max_threads(int model, bool fp32, int v, bool het = false);

constexpr int kEnergyBlocks = 1024;  // fixed grid of the single-chain reduction (deterministic)

// Per-device state of host-side set-up that CUDA scopes to the current device (a kernel's
// shared-memory limit, a device attribute): done once for each device a process uses.
constexpr int kMaxDevices = 64;
struct PerDevice {
  std::mutex m;
  bool done[kMaxDevices] = {};
  cudaError_t err[kMaxDevices] = {};
  int value[kMaxDevices] = {};
};

// Raise `kernel`'s dynamic shared-memory limit to `bytes` on the current device, once per
// device (the attribute applies only to the device that is current when it is set).
template <typename K> inline cudaError_t set_smem_limit_once(K *kernel, int bytes, PerDevice &pd) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  std::lock_guard<std::mutex> g(pd.m);
  if (!pd.done[dev]) {
    pd.err[dev] = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    pd.done[dev] = true;
  }
  return pd.err[dev];
}

// Streaming multiprocessors of the current device (cached per device); grid-stride kernels
// size their grids as a multiple of it.
inline int sm_count() {
  static PerDevice pd;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 152;
  if (dev < 0 || dev >= kMaxDevices) {
    int n = 0;
    return cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0 ? n : 152;
  }
  std::lock_guard<std::mutex> g(pd.m);
  if (!pd.done[dev]) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
    pd.value[dev] = n;
    pd.done[dev] = true;
  }
  return pd.value[dev];
}

}  // namespace rk4d

struct rk4_chain;
namespace rk4d {
// Read-only view of a handle (model, precision, chain table on the host, coefficients, stream).
int handle_info(const rk4_chain *h, int *model, bool *fp32, int *nchains, const ChainDesc **chains, CoefD *cf,
                cudaStream_t *stream, bool *het);
// Stages of the handle's tableau and its coupling range (1, or 2 with second neighbours): one
// step reaches stages x range sites along the chain.
int scheme_reach(const rk4_chain *h, int *stages, int *range);
// For callers that capture a handle's integrations into a larger CUDA graph: a counter bumped
// by every setter (a captured graph is stale once it changes); the stream the handle enqueues
// on and its own graph replay, swapped during a capture; and the pinned host tables and
// buffers an integration of nsteps needs, prepared beforehand (preparing them may synchronise
// the stream, which must not happen while capturing).
unsigned config_version(const rk4_chain *h);
cudaStream_t swap_stream(rk4_chain *h, cudaStream_t st);
bool swap_graphs(rk4_chain *h, bool on);
int prepare_integrate(rk4_chain *h, int64_t nsteps);

}  // namespace rk4d
