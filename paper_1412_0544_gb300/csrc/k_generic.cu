// k_generic.cu -- any explicit Runge-Kutta tableau (up to 7 stages) and coupling range 1 or 2
// (nearest or next-nearest neighbours), the generalisations the paper names in Sec. 2 ("any
// other explicit Runge-Kutta method") and Sec. 5 ("next-nearest-neighbour couplings need twice
// as long overlaps").  Temporal blocking then needs a halo of s * range sites per side per
// step (s stages, each reaching `range` sites further).
//
// Two schemes share one per-site operation sequence (so they agree bit for bit):
//   * k_gen_state / k_gen_slope / k_gen_combine: the standard implementation, one sweep per
//     stage-state evaluation, one per slope evaluation and one for the combination (2s+1 sweeps
//     per step, Sec. 2.2);
//   * k_gen_blocked: tiles of W = block * v sites advanced k steps per launch in registers.
//
// Per-site operation order (fixed):
//   stage state  u = y; for m < j with a_jm != 0:  u = fma(a_jm dt, k_m, u)        (Eq. (4))
//   slope        range 1: as the RK4 kernels; range 2 adds lap2 = fma(-2, x, x_{i-2} + x_{i+2})
//                inside the coupling: kx = fma(kappa, lap, fma(kappa2, lap2, -(y + z)))
//   combine      inc = 0; for m with b_m != 0: inc = fma(b_m dt, k_m, inc)          (Eq. (5))
//                FP64: y = y + inc;  FP32-Kahan: s = inc - c; t = y + s; c = (t - y) - s; y = t
#include <algorithm>

#include "rk4_generic.cuh"

namespace rk4d {

// ---- one-stage-per-launch reference ------------------------------------------------------

template <typename R, int D>
__global__ void __launch_bounds__(256) k_gen_state(GenStagedJob job, Tableau<R> tb, int j) {
  const R *Y = static_cast<const R *>(job.y);
  const R *K = static_cast<const R *>(job.k);
  R *U = static_cast<R *>(job.u);
  const size_t plane = (size_t)job.total * D;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < job.total; i += stride) {
    R y[D], k[kMaxStages][D], u[D];
#pragma unroll
    for (int d = 0; d < D; ++d) y[d] = Y[i * D + d];
#pragma unroll
    for (int m = 0; m < kMaxStages; ++m)
#pragma unroll
      for (int d = 0; d < D; ++d) k[m][d] = (m < j) ? K[m * plane + i * D + d] : R(0);
    gen_stage_state<R, D>(j, tb, y, k, u);
#pragma unroll
    for (int d = 0; d < D; ++d) U[i * D + d] = u[d];
  }
}

template <typename R, int MODEL, int RANGE>
__global__ void __launch_bounds__(256) k_gen_slope(GenStagedJob job, Coef<R> cf, R kappa2, int j) {
  constexpr int D = Dim<MODEL>::D;
  const R *src = static_cast<const R *>(j == 0 ? job.y : job.u);
  R *K = static_cast<R *>(job.k) + (size_t)j * job.total * D;
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
    const int64_t li = i - ch.off;
    auto xat = [&](int64_t q) -> R {  // coupling coordinate of chain site q (boundary-resolved)
      const int64_t g = (ch.bc == PERIODIC) ? ch.off + wrap(q, ch.n) : ((q < 0 || q >= ch.n) ? -1 : ch.off + q);
      if (g < 0 || !bounds_ok(job.hdr, in_range(g, 1, job.total))) return R(0);
      return src[g * D];
    };
    R u[D], k[D];
#pragma unroll
    for (int d = 0; d < D; ++d) u[d] = src[i * D + d];
    slope_gen<R, MODEL, RANGE>(u, xat(li - 1), xat(li + 1), RANGE == 2 ? xat(li - 2) : R(0),
                               RANGE == 2 ? xat(li + 2) : R(0), c, kappa2, k);
#pragma unroll
    for (int d = 0; d < D; ++d) K[i * D + d] = k[d];
  }
}

template <typename R, int D, bool KAHAN>
__global__ void __launch_bounds__(256) k_gen_combine(GenStagedJob job, Tableau<R> tb) {
  R *Y = static_cast<R *>(job.y);
  R *CMP = static_cast<R *>(job.cmp);
  const R *K = static_cast<const R *>(job.k);
  const size_t plane = (size_t)job.total * D;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < job.total; i += stride) {
    R y[D], k[kMaxStages][D], cmp[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      y[d] = Y[i * D + d];
      cmp[d] = KAHAN ? CMP[i * D + d] : R(0);
    }
#pragma unroll
    for (int m = 0; m < kMaxStages; ++m)
#pragma unroll
      for (int d = 0; d < D; ++d) k[m][d] = (m < tb.s) ? K[m * plane + i * D + d] : R(0);
    gen_combine<R, D, KAHAN>(tb, k, y, cmp);
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

// ---- temporally blocked generic kernel ----------------------------------------------------

// Two values of the working precision as one 8- or 16-byte shared-memory access.
template <typename R> struct Pair;
template <> struct Pair<float> { using T = float2; };
template <> struct Pair<double> { using T = double2; };

// Advance one tile's registers K steps of the generic scheme.  `edge`: gen_edge_values(V)
// values of shared memory, two parities of [(first, second) coupling coordinate of each thread
// | (second-last, last) of each thread].  Every stage each thread stores its two pairs (two
// vector stores) and, after the stage's one barrier, reads its left neighbour's last pair and
// its right neighbour's first pair (two vector loads, conflict-free): four shared-memory
// instructions for the range-2 coupling, where shuffles plus warp-edge slots took 12 (FP32) or
// 16 (FP64).  The two tile ends read a stand-in (their own pair), which only reaches halo sites.
template <typename R, int MODEL, int V, int RANGE, bool KAHAN, bool MASK, uint64_t SHAPE>
__device__ __forceinline__ void gen_tile_advance(R (&y)[V][Dim<MODEL>::D], R (&cmp)[V][Dim<MODEL>::D],
                                                 uint32_t ghost, int K, const Coef<R> &cf, R kappa2,
                                                 const Tableau<R> &tb, R *edge) {
  constexpr int D = Dim<MODEL>::D;
  static_assert(V >= 2, "the generic kernel holds at least two sites per thread");
  constexpr int NT = kGenEdgeThreads;
  using R2 = typename Pair<R>::T;
  const int tid = threadIdx.x;
  const int lt = tid > 0 ? tid - 1 : tid;                           // left neighbour thread
  const int rt = tid < (int)blockDim.x - 1 ? tid + 1 : tid;          // right neighbour thread
  R k[V][kMaxStages][D];

  int parity = 0;  // edge slots alternate strictly from stage to stage (s may be odd)
#pragma unroll 1
  for (int s = 0; s < K; ++s) {
#pragma unroll
    for (int j = 0; j < kMaxStages; ++j) {
      if (j >= gen_stages<SHAPE>(tb)) break;
      if (!gen_stage_needed<SHAPE>(j)) continue;  // a compiled shape's dead stage: nothing reads it
      R u[V][D];
      R ext[V + 4];  // ext[2 + v] = x of site v; two neighbours on each side
      R2 *head = reinterpret_cast<R2 *>(edge) + parity * 2 * NT;  // (first, second) per thread
      R2 *tail = head + NT;                                         // (second-last, last) per thread
      parity ^= 1;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        gen_stage_state<R, D, SHAPE>(j, tb, y[v], k[v], u[v]);
        ext[2 + v] = (MASK && ((ghost >> v) & 1u)) ? R(0) : u[v][0];
      }
      R2 hv, tv;
      hv.x = ext[2];
      hv.y = ext[3];
      tv.x = ext[V];
      tv.y = ext[V + 1];
      head[tid] = hv;
      tail[tid] = tv;
      // each thread reads only its neighbour threads' slots: in FP64 the streaming form waits
      // for the neighbouring warps only (measured +4.6 % for Dormand-Prince 5); in FP32 the two
      // named barriers per stage cost 22 %, so it keeps the block-wide one
      if constexpr (SHAPE != 0 && sizeof(R) == 8) neighbour_warp_sync(); else __syncthreads();
      {
        const R2 l = tail[lt];
        const R2 r = head[rt];
        ext[0] = l.x;
        ext[1] = l.y;
        ext[V + 2] = r.x;
        ext[V + 3] = r.y;
      }
#pragma unroll
      for (int v = 0; v < V; ++v) {
        R kv[D];
        slope_gen<R, MODEL, RANGE>(u[v], ext[1 + v], ext[3 + v], RANGE == 2 ? ext[v] : R(0),
                                   RANGE == 2 ? ext[4 + v] : R(0), cf, kappa2, kv);
#pragma unroll
        for (int d = 0; d < D; ++d) k[v][j][d] = kv[d];
      }
    }
#pragma unroll
    for (int v = 0; v < V; ++v) gen_combine<R, D, KAHAN, SHAPE>(tb, k[v], y[v], cmp[v]);
  }
}

// The generic tile kernel.  With a compiled tableau shape (STREAM) it runs as a streaming
// loop: a resident set of blocks (grid sized by the host to what fits on the GPU) walks the
// tiles, block b taking tiles b, b + gridDim.x, ...  While a block computes one tile, the next
// one's window is already on its way into the second of two shared-memory buffers (cp.async),
// so a tile's load latency is hidden behind the previous tile's arithmetic.  That lets short
// launches (small k, and so a small halo of redundant sites) run without exposed load time,
// which matters here: the generic scheme's halo is s' x range sites per side and step (12 for
// Dormand-Prince 5 with second neighbours).  The run-time-shape form (SHAPE = 0) processes one
// tile per block (a loop around it would keep the tableau's coefficients in registers).
// Shared memory: edge[gen_edge_values(V)] | buffer 0: tile[W*D] (+ ctile[W*D]) | buffer 1
// (streaming only).
template <typename R, int MODEL, int V, int RANGE, bool KAHAN, uint64_t SHAPE = 0>
__global__ void __launch_bounds__(GenBounds<R, V, SHAPE>::threads) k_gen_blocked(BlockedJob job, Coef<R> cf,
                                                                                 R kappa2, Tableau<R> tb, int H) {
  constexpr int D = Dim<MODEL>::D;
  constexpr bool STREAM = SHAPE != 0;
  extern __shared__ __align__(16) unsigned char smem[];
  R *edge = reinterpret_cast<R *>(smem);
  const int W = blockDim.x * V;
  const int G = job.G;
  const int tsize = W * D * (KAHAN ? 2 : 1);  // one buffer: tile and compensation tile
  R *const buf0 = edge + gen_edge_values(V);
  const R *in = static_cast<const R *>(job.in);
  const R *cin = static_cast<const R *>(job.cin);

  // chain, chain-local tile index and coupling of item `it`
  auto locate = [&](int64_t it, ChainDesc &ch, int64_t &tile, Coef<R> &c) {
    c = cf;
    if (job.nchains == 1) {
      ch = job.one;
      tile = it;
    } else {
      int ci;
      if (job.bt.tile_chain) {
        const int2 tc = __ldg(&job.bt.tile_chain[it]);
        ci = tc.x;
        tile = tc.y;
      } else {
        ci = find_chain_warp(job.bt.full_prefix, job.nchains, it);  // every warp, three rounds of loads
        tile = it - job.bt.full_prefix[ci];
      }
      ch = job.chains[ci];
      c.kappa = (R)ch.kappa;
    }
  };
  auto issue = [&](int64_t it, R *buf) {
    ChainDesc ch;
    int64_t tile;
    Coef<R> c;
    locate(it, ch, tile, c);
    const int64_t t0 = tile * (int64_t)G - H;
    tile_load_async<R, D>(buf, in, ch.off, ch.n, ch.bc, t0, W, job.total, job.hdr);
    if constexpr (KAHAN) tile_load_async<R, D>(buf + W * D, cin, ch.off, ch.n, ch.bc, t0, W, job.total, job.hdr);
    cp_async_commit();
  };

  int64_t item = blockIdx.x;
  if (item >= job.ntiles) return;
  issue(item, buf0);
  int cur = 0;
  for (;;) {
    const int64_t next = item + gridDim.x;
    if (STREAM && next < job.ntiles) {
      issue(next, buf0 + (cur ^ 1) * tsize);  // that buffer was released by the last iteration's barrier
      cp_async_wait<1>();                     // this tile's copies are complete, the next one's may run on
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    R *tl = buf0 + cur * tsize;
    R *ctl = tl + W * D;
    ChainDesc ch;
    int64_t tile;
    Coef<R> c;
    locate(item, ch, tile, c);
    const int64_t t0 = tile * (int64_t)G - H;
    R y[V][D], cmp[V][D];
    const int base = threadIdx.x * V;
#pragma unroll
    for (int v = 0; v < V; ++v)
#pragma unroll
      for (int d = 0; d < D; ++d) {
        y[v][d] = tl[(base + v) * D + d];
        if constexpr (KAHAN) cmp[v][d] = ctl[(base + v) * D + d]; else cmp[v][d] = R(0);
      }
    const bool edge_tile = (ch.bc == FIXED) && (t0 < 0 || t0 + W > ch.n);
    if (edge_tile) {
      uint32_t ghost = 0;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int64_t g = t0 + base + v;
        if (g < 0 || g >= ch.n) ghost |= 1u << v;
      }
      gen_tile_advance<R, MODEL, V, RANGE, KAHAN, true, SHAPE>(y, cmp, ghost, job.K, c, kappa2, tb, edge);
    } else {
      gen_tile_advance<R, MODEL, V, RANGE, KAHAN, false, SHAPE>(y, cmp, 0u, job.K, c, kappa2, tb, edge);
    }
    const int64_t g0 = t0 + H;
    const int64_t rem = ch.n - g0;
    const int cnt = (int)(rem < G ? rem : G);
    bool bad = false;  // a stored (interior) value is NaN or infinite
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const bool stored = base + v >= H && base + v < H + cnt;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        tl[(base + v) * D + d] = y[v][d];
        if constexpr (KAHAN) ctl[(base + v) * D + d] = cmp[v][d];
        bad |= stored && nonfinite(y[v][d]);
      }
    }
    report_nonfinite(job.hdr, __syncthreads_or(bad));
    if (cnt > 0) {
      tile_store<R, D>(static_cast<R *>(job.out), tl, ch.off, H, g0, cnt, job.total, W, job.hdr);
      if constexpr (KAHAN) tile_store<R, D>(static_cast<R *>(job.cout), ctl, ch.off, H, g0, cnt, job.total, W, job.hdr);
    }
    if constexpr (!STREAM) break;
    __syncthreads();  // the buffer is refilled two iterations on; nobody may still read it
    cur ^= 1;
    item = next;
    if (item >= job.ntiles) break;
  }
}

// The nonzero pattern of a tableau (see shape_a_bit): the key of the compiled shapes.
static uint64_t tableau_shape(const TableauD &t) {
  uint64_t sh = (uint64_t)t.s & 7u;
  for (int j = 1; j < t.s; ++j)
    for (int m = 0; m < j; ++m)
      if (t.a[j][m] != 0.0) sh |= shape_a_bit(j, m);
  for (int m = 0; m < t.s; ++m)
    if (t.b[m] != 0.0) sh |= shape_b_bit(m);
  return sh;
}

// Shapes with tile kernels compiled for them (4 sites per thread): the classical RK4 tableau
// (the generic kernel runs it with second-neighbour coupling) and Dormand-Prince 5 (7 stages,
// a_61 = 0, b_1 = b_6 = 0).  Other tableaux run the kernel that reads the pattern at run time.
constexpr uint64_t kShapeRK4 = 4u | shape_a_bit(1, 0) | shape_a_bit(2, 1) | shape_a_bit(3, 2) | shape_b_bit(0) |
                               shape_b_bit(1) | shape_b_bit(2) | shape_b_bit(3);
constexpr uint64_t kShapeDopri5 =
    7u | shape_a_bit(1, 0) | shape_a_bit(2, 0) | shape_a_bit(2, 1) | shape_a_bit(3, 0) | shape_a_bit(3, 1) |
    shape_a_bit(3, 2) | shape_a_bit(4, 0) | shape_a_bit(4, 1) | shape_a_bit(4, 2) | shape_a_bit(4, 3) |
    shape_a_bit(5, 0) | shape_a_bit(5, 1) | shape_a_bit(5, 2) | shape_a_bit(5, 3) | shape_a_bit(5, 4) |
    shape_a_bit(6, 0) | shape_a_bit(6, 2) | shape_a_bit(6, 3) | shape_a_bit(6, 4) | shape_a_bit(6, 5) |
    shape_b_bit(0) | shape_b_bit(2) | shape_b_bit(3) | shape_b_bit(4) | shape_b_bit(5);

// The compiled shape a tableau runs with at v sites per thread (0: the run-time-shape kernel).
static uint64_t compiled_shape(const TableauD &t, int v) {
  if (v != 4) return 0;
  const uint64_t sh = tableau_shape(t);
  return (sh == kShapeDopri5 || sh == kShapeRK4) ? sh : 0;
}

template <typename R, int MODEL, int V, int RANGE, bool KAHAN, uint64_t SHAPE>
static int gen_max_threads_s() {
  cudaFuncAttributes a;
  if (cudaFuncGetAttributes(&a, k_gen_blocked<R, MODEL, V, RANGE, KAHAN, SHAPE>) != cudaSuccess) return 0;
  return a.maxThreadsPerBlock;
}

template <typename R, int MODEL, int V, int RANGE, bool KAHAN>
static int gen_max_threads_one(uint64_t shape) {
  if constexpr (V == 4) {
    if (shape == kShapeDopri5) return gen_max_threads_s<R, MODEL, V, RANGE, KAHAN, kShapeDopri5>();
    if (shape == kShapeRK4) return gen_max_threads_s<R, MODEL, V, RANGE, KAHAN, kShapeRK4>();
  }
  return gen_max_threads_s<R, MODEL, V, RANGE, KAHAN, 0>();
}

template <int MODEL, int RANGE>
static int gen_max_threads_m(bool fp32, int v, uint64_t sh) {
  if (v == 2) return fp32 ? gen_max_threads_one<float, MODEL, 2, RANGE, true>(sh) : gen_max_threads_one<double, MODEL, 2, RANGE, false>(sh);
  if (v == 4) return fp32 ? gen_max_threads_one<float, MODEL, 4, RANGE, true>(sh) : gen_max_threads_one<double, MODEL, 4, RANGE, false>(sh);
  return 0;
}

int gen_blocked_max_threads(int model, bool fp32, int range, int v, const TableauD &tb) {
  const uint64_t sh = compiled_shape(tb, v);
  if (model == ROESSLER) return range == 1 ? gen_max_threads_m<ROESSLER, 1>(fp32, v, sh) : gen_max_threads_m<ROESSLER, 2>(fp32, v, sh);
  return range == 1 ? gen_max_threads_m<HARMONIC, 1>(fp32, v, sh) : gen_max_threads_m<HARMONIC, 2>(fp32, v, sh);
}

size_t gen_blocked_smem_bytes(int model, bool fp32, int v, int block, const TableauD &tb) {
  const int D = model == ROESSLER ? 3 : 2;
  const size_t rs = fp32 ? 4 : 8;
  const size_t buffers = compiled_shape(tb, v) != 0 ? 2 : 1;  // the streaming form double-buffers
  return (size_t)gen_edge_values(v) * rs + buffers * (size_t)block * v * D * rs * (fp32 ? 2 : 1);
}

// ---- launchers ------------------------------------------------------------------------------

template <typename R>
static Tableau<R> to_tableau(const TableauD &t, double dt) {
  Tableau<R> r{};
  r.s = t.s;
  for (int j = 0; j < kMaxStages; ++j) {
    r.anz[j] = 0;
    for (int m = 0; m < kMaxStages; ++m) {
      const double a = (j < t.s && m < j) ? t.a[j][m] : 0.0;
      r.adt[j][m] = (R)(a * dt);
      if (a != 0.0) r.anz[j] |= 1u << m;
    }
  }
  r.bnz = 0;
  for (int m = 0; m < kMaxStages; ++m) {
    const double b = m < t.s ? t.b[m] : 0.0;
    r.bdt[m] = (R)(b * dt);
    if (b != 0.0) r.bnz |= 1u << m;
  }
  return r;
}

static int64_t staged_grid(int64_t total) {
  int64_t g = (total + 255) / 256;
  const int64_t cap = (int64_t)sm_count() * 64;
  return g > cap ? cap : (g < 1 ? 1 : g);
}

template <typename R, int MODEL, int RANGE, bool KAHAN>
static cudaError_t gen_staged_t(const GenStagedJob &job, const CoefD &cfd, const TableauD &td, double dt,
                                cudaStream_t st) {
  constexpr int D = Dim<MODEL>::D;
  if (job.total <= 0) return cudaSuccess;
  const Tableau<R> tb = to_tableau<R>(td, dt);
  const Coef<R> cf = to_coef<R>(cfd, cfd.kappa);
  const unsigned grid = (unsigned)staged_grid(job.total);
  for (int j = 0; j < td.s; ++j) {
    if (j > 0) k_gen_state<R, D><<<grid, 256, 0, st>>>(job, tb, j);
    k_gen_slope<R, MODEL, RANGE><<<grid, 256, 0, st>>>(job, cf, (R)cfd.kappa2, j);
  }
  k_gen_combine<R, D, KAHAN><<<grid, 256, 0, st>>>(job, tb);
  return cudaGetLastError();
}

cudaError_t launch_gen_staged_step(int model, bool fp32, int range, const GenStagedJob &job, const CoefD &cf,
                                   const TableauD &tb, double dt, cudaStream_t st) {
#define RK4_GEN_STAGED(MODEL)                                                                            \
  if (range == 1)                                                                                        \
    return fp32 ? gen_staged_t<float, MODEL, 1, true>(job, cf, tb, dt, st)                              \
                : gen_staged_t<double, MODEL, 1, false>(job, cf, tb, dt, st);                            \
  return fp32 ? gen_staged_t<float, MODEL, 2, true>(job, cf, tb, dt, st)                                 \
              : gen_staged_t<double, MODEL, 2, false>(job, cf, tb, dt, st);
  if (model == ROESSLER) {
    RK4_GEN_STAGED(ROESSLER)
  }
  RK4_GEN_STAGED(HARMONIC)
#undef RK4_GEN_STAGED
}

template <typename R, int MODEL, int V, int RANGE, bool KAHAN, uint64_t SHAPE>
static cudaError_t gen_blocked_s(int block, const BlockedJob &job, const CoefD &cfd, const TableauD &td, double dt,
                                 int H, cudaStream_t st) {
  static PerDevice attr;
  const cudaError_t attr_err = set_smem_limit_once(k_gen_blocked<R, MODEL, V, RANGE, KAHAN, SHAPE>, 200 * 1024, attr);
  if (attr_err != cudaSuccess) return attr_err;
  if (job.ntiles <= 0) return cudaSuccess;
  const size_t smem = gen_blocked_smem_bytes(MODEL, KAHAN, V, block, td);
  int64_t grid = job.ntiles;  // one tile per block, or
  if constexpr (SHAPE != 0) {  // the streaming form: as many blocks as stay resident together
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, k_gen_blocked<R, MODEL, V, RANGE, KAHAN, SHAPE>, block, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    grid = std::min<int64_t>(job.ntiles, (int64_t)per_sm * sm_count());
  }
  k_gen_blocked<R, MODEL, V, RANGE, KAHAN, SHAPE><<<(unsigned)grid, block, smem, st>>>(
      job, to_coef<R>(cfd, cfd.kappa), (R)cfd.kappa2, to_tableau<R>(td, dt), H);
  return cudaGetLastError();
}

template <typename R, int MODEL, int V, int RANGE, bool KAHAN>
static cudaError_t gen_blocked_t(int block, const BlockedJob &job, const CoefD &cfd, const TableauD &td, double dt,
                                 int H, cudaStream_t st) {
  if constexpr (V == 4) {
    const uint64_t sh = compiled_shape(td, V);
    if (sh == kShapeDopri5) return gen_blocked_s<R, MODEL, V, RANGE, KAHAN, kShapeDopri5>(block, job, cfd, td, dt, H, st);
    if (sh == kShapeRK4) return gen_blocked_s<R, MODEL, V, RANGE, KAHAN, kShapeRK4>(block, job, cfd, td, dt, H, st);
  }
  return gen_blocked_s<R, MODEL, V, RANGE, KAHAN, 0>(block, job, cfd, td, dt, H, st);
}

template <int MODEL, int RANGE>
static cudaError_t gen_blocked_m(bool fp32, int v, int block, const BlockedJob &job, const CoefD &cf,
                                 const TableauD &tb, double dt, int H, cudaStream_t st) {
  switch (v) {
    case 2:
      return fp32 ? gen_blocked_t<float, MODEL, 2, RANGE, true>(block, job, cf, tb, dt, H, st)
                  : gen_blocked_t<double, MODEL, 2, RANGE, false>(block, job, cf, tb, dt, H, st);
    case 4:
      return fp32 ? gen_blocked_t<float, MODEL, 4, RANGE, true>(block, job, cf, tb, dt, H, st)
                  : gen_blocked_t<double, MODEL, 4, RANGE, false>(block, job, cf, tb, dt, H, st);
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_gen_blocked(int model, bool fp32, int range, int v, int block, const BlockedJob &job,
                               const CoefD &cf, const TableauD &tb, double dt, int H, cudaStream_t st) {
  if (model == ROESSLER)
    return range == 1 ? gen_blocked_m<ROESSLER, 1>(fp32, v, block, job, cf, tb, dt, H, st)
                      : gen_blocked_m<ROESSLER, 2>(fp32, v, block, job, cf, tb, dt, H, st);
  return range == 1 ? gen_blocked_m<HARMONIC, 1>(fp32, v, block, job, cf, tb, dt, H, st)
                    : gen_blocked_m<HARMONIC, 2>(fp32, v, block, job, cf, tb, dt, H, st);
}

}  // namespace rk4d
