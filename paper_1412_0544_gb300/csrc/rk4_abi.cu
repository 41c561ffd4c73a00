// rk4_abi.cu -- host runtime behind the C ABI of include/rk4chain.h: argument checking,
// workspace layout, launch plans (k steps per launch, ping-pong buffers), CUDA-graph replay,
// the tiling autotuner, reductions and the status word.  Only host code lives here; every
// floating-point operation of the integrator runs in the kernels.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/rk4chain.h"
#include "rk4_internal.h"

using namespace rk4d;

namespace {

constexpr size_t kAlign = 256;
constexpr int kMaxDistinctK = 4;
constexpr size_t kMaxSmem = 200 * 1024;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct GraphKey {
  int kernel = -1;
  const void *state = nullptr, *comp = nullptr, *ws = nullptr;
  int64_t nsteps = -1;
  int block = 0, v = 0, k = 0;
  long long timeout = 0;
  const void *sp = nullptr;
  int generic = 0;
  bool operator==(const GraphKey &o) const {
    return kernel == o.kernel && state == o.state && comp == o.comp && ws == o.ws && nsteps == o.nsteps &&
           block == o.block && v == o.v && k == o.k && timeout == o.timeout && sp == o.sp && generic == o.generic;
  }
};

struct WsLayout {
  size_t hdr, partials, result, chains, prefix, tiles, state, comp, u0, u1, acc, total;
};

// One launch plan: the k of every launch (or time block) and whether the result needs copying
// back from the workspace because the count of ping-pong swaps is odd.
struct Plan {
  int64_t nmain = 0;            // launches with kval[0]
  std::vector<int> tail;        // indices into kval
  std::vector<int> kval;        // distinct k values, kval[0] = the main k
  bool copy_back = false;
  int64_t count() const { return nmain + (int64_t)tail.size(); }
  int k_at(int64_t i) const { return kval[i < nmain ? 0 : tail[i - nmain]]; }
};

}  // namespace

struct rk4_chain {
  int model = 0, precision = 0, D = 3;
  bool fp32 = false;
  int nchains = 1;
  std::vector<ChainDesc> chains;
  int64_t total = 0;
  double dt = 0.01;
  rk4_params p{};
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  int kernel = RK4_KERNEL_AUTO;
  bool tiling_auto = true;
  rk4_tiling tiling{};
  double t0 = 0.0;
  int64_t nstep = 0;
  bool graphs = true;
  long long timeout_ns = 2000000000LL;
  // pinned host staging: chain table followed by kMaxDistinctK per-k tile tables (see
  // ktable_bytes), in the same relative layout as in the workspace
  void *h_tables = nullptr;
  size_t tables_bytes = 0;
  std::vector<int> tables_k;  // the k values the tile tables currently describe
  int tables_W = 0;           // and the tile width they were computed for
  int tables_v = 0;           // the sites per thread (packed segments are aligned to it)
  int tables_halo = 0;        // the halo per step
  int tables_packed = -1;     // and whether they are packed (see packed_batch)
  int64_t nfull[kMaxDistinctK] = {};    // packed batches: full tiles per k slot
  int64_t npacked[kMaxDistinctK] = {};  // and packed tiles
  double *h_out = nullptr;    // pinned: reduction results (nchains doubles)
  int *h_status = nullptr;    // pinned: status word read-back
  GraphKey gkey;
  cudaGraphExec_t gexec = nullptr;
  // generic explicit RK scheme (any tableau, coupling range 1 or 2)
  bool has_tableau = false;
  TableauD tab{};
  double kappa2 = 0.0;
  // heterogeneous chain (Eq. (1)): caller-owned device array of P parameters per site
  const void *site_params = nullptr;
  unsigned gen_version = 0;  // bumped when the tableau or kappa2 changes (graph cache key)
  int tuned_kernel = 0;  // scheme rk4_chain_autotune measured fastest for RK4_KERNEL_AUTO (0: not tuned)
  bool timeout_set = false;                 // RK4_OPT_TIMEOUT_NS given explicitly
  unsigned config_version = 0;              // bumped by every setter (graphs captured by callers)
};

namespace {

bool use_generic(const rk4_chain *h);

bool use_het(const rk4_chain *h);

int tile_interior(const rk4_chain *h, int W, int k);

int effective_kernel(const rk4_chain *h) {
  if (h->kernel != RK4_KERNEL_AUTO) return h->kernel;
  if (h->tuned_kernel != 0) return h->tuned_kernel;  // the autotuner's measured choice
  if (h->nchains == 1 || use_generic(h) || use_het(h)) return RK4_KERNEL_BLOCKED;
  return RK4_KERNEL_PERSISTENT;  // batches
}

size_t elem_bytes(const rk4_chain *h) { return h->fp32 ? 4 : 8; }

// The generic kernels run when a tableau was set or second-neighbour coupling is on.
bool use_generic(const rk4_chain *h) { return h->has_tableau || h->kappa2 != 0.0; }
bool use_het(const rk4_chain *h) { return h->site_params != nullptr; }
int coupling_range(const rk4_chain *h) { return h->kappa2 != 0.0 ? 2 : 1; }
int stages(const rk4_chain *h) { return use_generic(h) ? h->tab.s : 4; }
// Stages the step's result depends on: those with a nonzero weight b_m and, recursively, the
// earlier stages a needed stage uses.  A stage outside this set (Dormand-Prince 5's seventh,
// with b_7 = 0) cannot influence y, so the dependency cone of one step spans at most this
// many stages: the tile halo and the sub-domain reach are sized by it.
int needed_stages(const rk4_chain *h) {
  if (!use_generic(h)) return 4;
  const TableauD &t = h->tab;
  uint32_t need = 0;
  for (int m = 0; m < t.s; ++m)
    if (t.b[m] != 0.0) need |= 1u << m;
  for (int j = t.s - 1; j >= 0; --j)
    if ((need >> j) & 1u)
      for (int m = 0; m < j; ++m)
        if (t.a[j][m] != 0.0) need |= 1u << m;
  int n = 0;
  for (int m = 0; m < t.s; ++m) n += (need >> m) & 1u;
  return n;
}

// Halo per side of one launch of k steps: s stages, each reaching `range` sites further.
int halo(const rk4_chain *h, int k) { return needed_stages(h) * coupling_range(h) * k; }

TableauD classical_rk4() {
  TableauD t{};
  t.s = 4;
  t.a[1][0] = 0.5;
  t.a[2][1] = 0.5;
  t.a[3][2] = 1.0;
  t.b[0] = 1.0 / 6.0;
  t.b[1] = 1.0 / 3.0;
  t.b[2] = 1.0 / 3.0;
  t.b[3] = 1.0 / 6.0;
  return t;
}

// Bytes of one k slot of the batch tile tables: the first-tile prefix (nchains + 1 entries;
// full tiles when packed, all tiles otherwise), the packed tiles' first-segment prefix
// (nchains + 1) and the segments (at most one per chain).
size_t ktable_bytes(int nchains) {
  return align_up(sizeof(int32_t) * (size_t)(nchains + 1)) * 2 + align_up(sizeof(SegDesc) * (size_t)nchains);
}

// Entries of one k slot's tile table (the chain of each full tile): room for tiles of at least
// kTileTableMinG interior sites; a launch with more tiles than that searches the prefix instead.
constexpr int kTileTableMinG = 64;
int64_t tile_table_entries(const rk4_chain *h) { return h->total / kTileTableMinG + h->nchains; }

WsLayout layout(const rk4_chain *h, int kernel) {
  WsLayout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t r = o;
    o = align_up(o + bytes);
    return r;
  };
  L.hdr = take(sizeof(WsHeader));
  L.partials = take(sizeof(double) * kEnergyBlocks);
  L.result = take(sizeof(double) * (size_t)h->nchains);
  L.chains = take(h->nchains > 1 ? sizeof(ChainDesc) * (size_t)h->nchains : 0);
  L.prefix = take(h->nchains > 1 ? ktable_bytes(h->nchains) * kMaxDistinctK : 0);
  L.tiles = take(h->nchains > 1 && kernel != RK4_KERNEL_STAGED
                     ? sizeof(int2) * (size_t)tile_table_entries(h) * kMaxDistinctK : 0);
  const size_t sz = (size_t)h->total * (size_t)h->D * elem_bytes(h);
  L.state = L.comp = L.u0 = L.u1 = L.acc = 0;
  if (kernel == RK4_KERNEL_STAGED && use_generic(h)) {
    L.u0 = take(sz);                     // stage state
    L.acc = take(sz * (size_t)h->tab.s);  // the s stage slopes
  } else if (kernel == RK4_KERNEL_STAGED) {
    L.u0 = take(sz);
    L.u1 = take(sz);
    L.acc = take(sz);
  } else {
    L.state = take(sz);
    if (h->fp32) L.comp = take(sz);
  }
  L.total = o;
  return L;
}

CoefD coef(const rk4_chain *h) {
  CoefD c;
  c.a = h->p.a;
  c.b = h->p.b;
  c.c = h->p.c;
  c.kappa = h->p.kappa;
  c.w2 = h->p.omega0 * h->p.omega0;
  c.h2 = h->dt / 2.0;
  c.h1 = h->dt;
  c.dt6 = h->dt / 6.0;
  c.dt3 = h->dt / 3.0;
  c.kappa2 = h->kappa2;
  return c;
}

int tiling_valid(const rk4_chain *h, int block, int v, int k) {
  if (block < 64 || block > 1024 || (block % 32) != 0) return 0;
  if (k < 1 || k > 16) return 0;
  const int W = block * v;
  if (use_generic(h)) {
    if (v != 2 && v != 4) return 0;
    const int H = halo(h, k);
    if (W - 2 * H < H) return 0;
    if (gen_blocked_smem_bytes(h->model, h->fp32, v, block, h->tab) > kMaxSmem) return 0;
    return 1;
  }
  if (v != 1 && v != 2 && v != 4 && v != 8) return 0;
  if (use_het(h) && v != 2 && v != 4) return 0;
  if (W - 8 * k < 8 * k) return 0;
  if (blocked_smem_bytes(h->model, h->fp32, v, block, use_het(h)) > kMaxSmem) return 0;
  return 1;
}

int tiling_max_threads(const rk4_chain *h, int v) {
  return use_generic(h) ? gen_blocked_max_threads(h->model, h->fp32, coupling_range(h), v, h->tab)
                        : blocked_max_threads(h->model, h->fp32, v, use_het(h));
}

void default_tiling(rk4_chain *h) {
  // Seed choice from the register and shared-memory budget (the paper suggests sizing the
  // cluster from the cache; here a tile should fill a block's registers): FP64 is bound by
  // the FP64 pipe, so k = 1 keeps the redundant halo work minimal; FP32 is bandwidth-bound
  // at k = 1, so several steps per launch pay off.
  if (use_generic(h)) {
    h->tiling.block = 128;
    h->tiling.v = 2;
    h->tiling.k = 1;
  } else if (use_het(h)) {
    h->tiling.block = 256;
    h->tiling.v = 2;
    h->tiling.k = h->fp32 ? 4 : 1;
  } else {
    h->tiling.block = 256;
    h->tiling.v = 4;
    h->tiling.k = h->fp32 ? 4 : 1;
  }
  h->tiling.G = tile_interior(h, h->tiling.block * h->tiling.v, h->tiling.k);
}

int64_t tiles_for(const rk4_chain *h, int G) {
  int64_t t = 0;
  for (const ChainDesc &c : h->chains) t += (c.n + G - 1) / G;
  return t;
}

// Batches on the classical homogeneous kernels (blocked and persistent) pack the chains' last
// partial pieces into shared tiles; the generic and heterogeneous kernels give every chain
// whole tiles of its own.
bool packed_batch(const rk4_chain *h) { return h->nchains > 1 && !use_generic(h) && !use_het(h); }

// Sites per 16 bytes of state in whole sites: a packed batch's full tiles start their windows at
// multiples of it (so they move by 16-byte vectors wherever the chain starts), which the interior
// pays with up to that many sites less than W - 2 H.
int batch_align(const rk4_chain *h) {
  int a = h->D * (int)elem_bytes(h), b = 16;
  while (b) {
    const int t = a % b;
    a = b;
    b = t;
  }
  return 16 / a;
}

// Interior sites per tile for tiles of W sites and k steps.
int tile_interior(const rk4_chain *h, int W, int k) {
  return W - 2 * halo(h, k) - (packed_batch(h) ? batch_align(h) - 1 : 0);
}


Plan make_plan(int64_t nsteps, int K) {
  Plan P;
  P.kval.push_back(K);
  const int64_t q = nsteps / K;
  const int r = (int)(nsteps % K);
  auto kidx = [&](int k) {
    for (size_t i = 0; i < P.kval.size(); ++i)
      if (P.kval[i] == k) return (int)i;
    P.kval.push_back(k);
    return (int)P.kval.size() - 1;
  };
  P.nmain = q;
  if (r > 0) P.tail.push_back(kidx(r));
  if (P.count() % 2 == 1) {
    if (r >= 2) {
      P.tail.clear();
      P.tail.push_back(kidx(r / 2));
      P.tail.push_back(kidx(r - r / 2));
    } else if (K >= 2 && q >= 1) {
      P.nmain = q - 1;
      std::vector<int> t;
      t.push_back(kidx(K / 2));
      t.push_back(kidx(K - K / 2));
      for (int x : P.tail) t.push_back(x);
      P.tail = t;
    } else {
      P.copy_back = true;
    }
  }
  return P;
}

cudaError_t ensure_pinned(rk4_chain *h) {
  if (!h->h_out) {
    cudaError_t e = cudaMallocHost((void **)&h->h_out, sizeof(double) * (size_t)h->nchains + 64);
    if (e != cudaSuccess) return e;
  }
  if (!h->h_status) {
    cudaError_t e = cudaMallocHost((void **)&h->h_status, 64);
    if (e != cudaSuccess) return e;
  }
  if (h->nchains > 1 && !h->h_tables) {
    // same relative layout as the workspace: chain table, then the prefix arrays at the next
    // 256-byte boundary
    h->tables_bytes = align_up(sizeof(ChainDesc) * (size_t)h->nchains) + ktable_bytes(h->nchains) * kMaxDistinctK;
    cudaError_t e = cudaMallocHost(&h->h_tables, h->tables_bytes);
    if (e != cudaSuccess) return e;
    std::memcpy(h->h_tables, h->chains.data(), sizeof(ChainDesc) * (size_t)h->nchains);
  }
  return cudaSuccess;
}

// The batch tile tables of k slot `ki` (pinned host copy, same layout as the workspace).
struct KTables {
  int32_t *prefix, *pack_prefix;
  SegDesc *segs;
};
KTables host_ktables(rk4_chain *h, int ki) {
  char *p = static_cast<char *>(h->h_tables) + align_up(sizeof(ChainDesc) * (size_t)h->nchains) +
            ktable_bytes(h->nchains) * (size_t)ki;
  const size_t pre = align_up(sizeof(int32_t) * (size_t)(h->nchains + 1));
  return {reinterpret_cast<int32_t *>(p), reinterpret_cast<int32_t *>(p + pre), reinterpret_cast<SegDesc *>(p + 2 * pre)};
}
BatchTiles dev_ktables(const rk4_chain *h, const char *ws, const WsLayout &L, int ki) {
  const char *p = ws + L.prefix + ktable_bytes(h->nchains) * (size_t)ki;
  const size_t pre = align_up(sizeof(int32_t) * (size_t)(h->nchains + 1));
  BatchTiles bt{};
  bt.full_prefix = reinterpret_cast<const int32_t *>(p);
  bt.pack_prefix = reinterpret_cast<const int32_t *>(p + pre);
  bt.segs = reinterpret_cast<const SegDesc *>(p + 2 * pre);
  bt.nfull = h->nfull[ki];
  bt.npacked = h->npacked[ki];
  const int64_t entries = tile_table_entries(h);
  bt.tile_chain = L.tiles && bt.nfull <= entries
                      ? reinterpret_cast<const int2 *>(ws + L.tiles + sizeof(int2) * (size_t)entries * (size_t)ki)
                      : nullptr;
  return bt;
}

// Fill the tile tables of the first nslots k slots on the device (after upload_tables).
cudaError_t fill_tile_tables(const rk4_chain *h, char *ws, const WsLayout &L, int nslots, cudaStream_t st) {
  if (h->nchains == 1) return cudaSuccess;
  for (int i = 0; i < nslots; ++i) {
    const BatchTiles bt = dev_ktables(h, ws, L, i);
    if (!bt.tile_chain) continue;
    const cudaError_t e =
        launch_tile_chains(bt.full_prefix, h->nchains, bt.nfull, const_cast<int2 *>(bt.tile_chain), st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Pack the segments of one k slot into tiles of W slots: each chain's last partial piece of
// cnt = n mod G interior sites (the whole chain when n < G) needs a window of
// L = H + cnt + H slots, rounded up to a multiple of v.  Best fit in decreasing order of L (the
// fullest tile that still has room, ties to the earliest opened), which leaves little unused
// room.  Returns the number of packed tiles; fills pack_prefix and segs in tile order.
int64_t pack_segments(const rk4_chain *h, int G, int H, int W, int v, int32_t *pack_prefix, SegDesc *segs) {
  struct Piece {
    int chain, cnt, L;
  };
  std::vector<Piece> pieces;
  for (int c = 0; c < h->nchains; ++c) {
    const int cnt = (int)(h->chains[c].n % G);
    if (cnt == 0) continue;
    const int L = (cnt + 2 * H + v - 1) / v * v;
    pieces.push_back({c, cnt, L});
  }
  std::stable_sort(pieces.begin(), pieces.end(), [](const Piece &a, const Piece &b) { return a.L > b.L; });
  // open tiles by free room (in units of v slots): the tiles of each room size, earliest first
  const int units = W / v;
  std::vector<std::vector<int>> by_room(units + 1);
  std::vector<int> room;                       // free slots of each tile
  std::vector<std::vector<int>> members;       // pieces of each tile, in slot order
  for (int i = 0; i < (int)pieces.size(); ++i) {
    const int need = pieces[i].L / v;
    int t = -1;
    for (int r = need; r <= units && t < 0; ++r)
      if (!by_room[r].empty()) {
        // earliest-opened tile of this room size (tiles are only appended in opening order)
        auto &bucket = by_room[r];
        auto it = std::min_element(bucket.begin(), bucket.end());
        t = *it;
        bucket.erase(it);
      }
    if (t < 0) {
      t = (int)room.size();
      room.push_back(units);
      members.emplace_back();
    }
    members[t].push_back(i);
    room[t] -= need;
    by_room[room[t]].push_back(t);
  }
  int32_t next = 0;
  for (size_t t = 0; t < members.size(); ++t) {
    pack_prefix[t] = next;
    int o = 0;
    for (int i : members[t]) {
      const Piece &p = pieces[i];
      SegDesc &sd = segs[next++];
      sd.chain = p.chain;
      sd.cnt = p.cnt;
      sd.L = p.L;
      sd.o = o;
      sd.g0 = h->chains[p.chain].n - p.cnt;
      o += p.L;
    }
  }
  pack_prefix[members.size()] = next;
  return (int64_t)members.size();
}

// Fill the pinned batch tile tables for the plan's k values (waits for earlier uses first).
cudaError_t prepare_tables(rk4_chain *h, const std::vector<int> &kval, int W) {
  if (h->nchains == 1) return cudaSuccess;
  const int packed = packed_batch(h) ? 1 : 0;
  if (h->tables_k == kval && h->tables_W == W && h->tables_v == h->tiling.v && h->tables_halo == halo(h, 1) &&
      h->tables_packed == packed)
    return cudaSuccess;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return e;
  for (size_t i = 0; i < kval.size(); ++i) {
    const int H = halo(h, kval[i]);
    const int G = tile_interior(h, W, kval[i]);
    KTables t = host_ktables(h, (int)i);
    int64_t acc = 0;
    for (int c = 0; c < h->nchains; ++c) {
      t.prefix[c] = (int32_t)acc;
      acc += packed ? h->chains[c].n / G : (h->chains[c].n + G - 1) / G;
    }
    t.prefix[h->nchains] = (int32_t)acc;
    h->nfull[i] = acc;
    h->npacked[i] = packed ? pack_segments(h, G, H, W, h->tiling.v, t.pack_prefix, t.segs) : 0;
  }
  h->tables_k = kval;
  h->tables_W = W;
  h->tables_v = h->tiling.v;
  h->tables_halo = halo(h, 1);
  h->tables_packed = packed;
  return cudaSuccess;
}

cudaError_t upload_tables(rk4_chain *h, char *ws, const WsLayout &L, cudaStream_t st) {
  if (h->nchains == 1) return cudaSuccess;
  return cudaMemcpyAsync(ws + L.chains, h->h_tables, h->tables_bytes, cudaMemcpyHostToDevice, st);
}

const ChainDesc *dev_chains(const rk4_chain *h, char *ws, const WsLayout &L) {
  return h->nchains > 1 ? reinterpret_cast<const ChainDesc *>(ws + L.chains) : nullptr;
}

// Enqueue the whole launch sequence of an integration on stream st.
cudaError_t enqueue_integrate(rk4_chain *h, int kernel, void *state, void *comp, char *ws, const WsLayout &L,
                              const Plan &P, int64_t nsteps, cudaStream_t st) {
  const CoefD cf = coef(h);
  const int W = h->tiling.block * h->tiling.v;
  // a fresh status word (and barrier counters) for every integration
  cudaError_t e = cudaMemsetAsync(ws + L.hdr, 0, sizeof(WsHeader), st);
  if (e != cudaSuccess) return e;
  e = upload_tables(h, ws, L, st);
  if (e != cudaSuccess) return e;
  const size_t bytes = (size_t)h->total * h->D * elem_bytes(h);
  if (kernel == RK4_KERNEL_STAGED && use_generic(h)) {
    GenStagedJob j{};
    j.y = state;
    j.cmp = comp;
    j.u = ws + L.u0;
    j.k = ws + L.acc;
    j.nchains = h->nchains;
    j.one = h->chains[0];
    j.chains = dev_chains(h, ws, L);
    j.total = h->total;
    j.hdr = reinterpret_cast<WsHeader *>(ws + L.hdr);
    for (int64_t s = 0; s < nsteps; ++s) {
      e = launch_gen_staged_step(h->model, h->fp32, coupling_range(h), j, cf, h->tab, h->dt, st);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  if (kernel == RK4_KERNEL_STAGED) {
    StagedJob j{};
    j.y = state;
    j.cmp = comp;
    j.sp = h->site_params;
    j.nchains = h->nchains;
    j.one = h->chains[0];
    j.chains = dev_chains(h, ws, L);
    j.total = h->total;
    j.hdr = reinterpret_cast<WsHeader *>(ws + L.hdr);
    j.acc = ws + L.acc;
    void *u0 = ws + L.u0, *u1 = ws + L.u1;
    for (int64_t s = 0; s < nsteps; ++s) {
      // stage 0 reads y and writes u0; 1: u0 -> u1; 2: u1 -> u0; 3: u0 -> y
      for (int st4 = 0; st4 < 4; ++st4) {
        j.uin = (st4 == 2) ? u1 : u0;
        j.uout = (st4 == 1) ? u1 : u0;
        e = launch_staged(h->model, h->fp32, st4, j, cf, st);
        if (e != cudaSuccess) return e;
      }
    }
    return cudaSuccess;
  }
  void *wsS = ws + L.state;
  void *wsC = h->fp32 ? (void *)(ws + L.comp) : nullptr;
  e = fill_tile_tables(h, ws, L, (int)P.kval.size(), st);
  if (e != cudaSuccess) return e;
  if (kernel == RK4_KERNEL_BLOCKED) {
    BlockedJob j{};
    j.nchains = h->nchains;
    j.one = h->chains[0];
    j.chains = dev_chains(h, ws, L);
    j.sp = h->site_params;
    j.hdr = reinterpret_cast<WsHeader *>(ws + L.hdr);
    j.total = h->total;
    j.packed = packed_batch(h) ? 1 : 0;
    for (int64_t i = 0; i < P.count(); ++i) {
      const int k = P.k_at(i);
      int ki = 0;
      while (P.kval[ki] != k) ++ki;
      j.K = k;
      j.G = tile_interior(h, W, k);
      if (h->nchains > 1) {
        // ntiles counts the full tiles (or, unpacked, every tile); the packed tiles follow them
        // in the same launch
        j.bt = dev_ktables(h, ws, L, ki);
        j.ntiles = j.bt.nfull;
      } else {
        j.ntiles = tiles_for(h, j.G);
      }
      const bool even = (i % 2) == 0;
      j.in = even ? state : wsS;
      j.out = even ? wsS : state;
      j.cin = even ? comp : wsC;
      j.cout = even ? wsC : comp;
      if (use_generic(h))
        e = launch_gen_blocked(h->model, h->fp32, coupling_range(h), h->tiling.v, h->tiling.block, j, cf, h->tab,
                               h->dt, halo(h, k), st);
      else
        e = launch_blocked(h->model, h->fp32, h->tiling.v, h->tiling.block, j, cf, st);
      if (e != cudaSuccess) return e;
    }
  } else {  // persistent
    PersistentJob j{};
    j.bufA = state;
    j.bufB = wsS;
    j.cA = comp;
    j.cB = wsC;
    j.nchains = h->nchains;
    j.one = h->chains[0];
    j.chains = dev_chains(h, ws, L);
    j.nk = (int)P.kval.size();
    int64_t maxtiles = 0;
    for (int i = 0; i < j.nk; ++i) {
      j.kval[i] = P.kval[i];
      j.Gval[i] = tile_interior(h, W, P.kval[i]);
      if (h->nchains > 1) {
        j.bt[i] = dev_ktables(h, ws, L, i);
        j.ntiles[i] = j.bt[i].nfull + j.bt[i].npacked;
      } else {
        j.ntiles[i] = tiles_for(h, j.Gval[i]);
      }
      maxtiles = std::max(maxtiles, j.ntiles[i]);
    }
    j.nmain = P.nmain;
    j.ntail = (int)P.tail.size();
    for (int i = 0; i < j.ntail; ++i) j.tail[i] = P.tail[i];
    j.hdr = reinterpret_cast<WsHeader *>(ws + L.hdr);
    j.total = h->total;
    // A barrier waits at most one time block; unless the caller set the bound, allow 20x a
    // pessimistic estimate of one (1e9 site-steps/s) so that very large batches cannot time
    // out spuriously.
    {
      int kmax = 1;
      for (int kv : P.kval) kmax = std::max(kmax, kv);
      const double est_ns = (double)h->total * kmax;  // at 1e9 site-steps/s: 1 ns per site-step
      j.timeout_ns = h->timeout_set ? h->timeout_ns : std::max<long long>(h->timeout_ns, (long long)(20.0 * est_ns));
    }
    j.extra_arrivals = 0;
    int grid = persistent_max_grid(h->model, h->fp32, h->tiling.v, h->tiling.block);
    if (grid <= 0) return cudaErrorInvalidConfiguration;
    grid = (int)std::min<int64_t>(grid, std::max<int64_t>(1, maxtiles));
    e = launch_persistent(h->model, h->fp32, h->tiling.v, h->tiling.block, grid, j, cf, st);
    if (e != cudaSuccess) return e;
  }
  if (P.copy_back) {
    e = cudaMemcpyAsync(state, wsS, bytes, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    if (h->fp32) e = cudaMemcpyAsync(comp, wsC, bytes, cudaMemcpyDeviceToDevice, st);
  }
  return e;
}

int check_buffers(const rk4_chain *h, const void *state, const void *comp, const void *ws) {
  if (!state || !ws) return RK4_EINVAL;
  if (h->fp32 != (comp != nullptr)) return RK4_EINVAL;
  if ((reinterpret_cast<uintptr_t>(ws) % kAlign) != 0) return RK4_EINVAL;
  if ((reinterpret_cast<uintptr_t>(state) % 16) != 0) return RK4_EINVAL;
  if (comp && (reinterpret_cast<uintptr_t>(comp) % 16) != 0) return RK4_EINVAL;
  return RK4_OK;
}

int integrate_impl(rk4_chain *h, void *state, void *comp, void *ws, size_t ws_bytes, int64_t nsteps) {
  int rc = check_buffers(h, state, comp, ws);
  if (rc) return rc;
  if (nsteps < 0) return RK4_EINVAL;
  const int kernel = effective_kernel(h);
  if (kernel == RK4_KERNEL_PERSISTENT && (use_generic(h) || use_het(h))) return RK4_EUNSUPPORTED;
  if (use_generic(h) && use_het(h)) return RK4_EUNSUPPORTED;
  const WsLayout L = layout(h, kernel);
  if (ws_bytes < L.total) return RK4_ENOMEM_WS;
  if (nsteps == 0) return RK4_OK;
  if (ensure_pinned(h) != cudaSuccess) return RK4_ECUDA;
  const int K = (kernel == RK4_KERNEL_STAGED) ? 1 : h->tiling.k;
  const Plan P = make_plan(nsteps, kernel == RK4_KERNEL_STAGED ? 1 : K);
  if (kernel != RK4_KERNEL_STAGED) {
    // tile counts must fit a 1-D grid and the int32 prefix tables
    const int kmax = *std::max_element(P.kval.begin(), P.kval.end());
    if (tiles_for(h, tile_interior(h, h->tiling.block * h->tiling.v, kmax)) > 0x7fffffffLL) return RK4_EUNSUPPORTED;
  }
  if (prepare_tables(h, P.kval, h->tiling.block * h->tiling.v) != cudaSuccess) return RK4_ECUDA;
  char *w = static_cast<char *>(ws);

  const bool use_graph = h->graphs && (kernel != RK4_KERNEL_BLOCKED || P.count() > 1);
  if (!use_graph) {
    return enqueue_integrate(h, kernel, state, comp, w, L, P, nsteps, h->stream) == cudaSuccess ? RK4_OK
                                                                                                : RK4_ECUDA;
  }
  GraphKey key;
  key.kernel = kernel;
  key.state = state;
  key.comp = comp;
  key.ws = ws;
  key.nsteps = nsteps;
  key.block = h->tiling.block;
  key.v = h->tiling.v;
  key.k = h->tiling.k;
  key.timeout = h->timeout_ns;
  key.sp = h->site_params;
  key.generic = use_generic(h) ? 1 + (int)h->gen_version : 0;
  if (!(h->gexec && key == h->gkey)) {
    if (h->gexec) {
      cudaGraphExecDestroy(h->gexec);
      h->gexec = nullptr;
    }
    if (!h->cap_stream && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
      return RK4_ECUDA;
    if (cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) return RK4_ECUDA;
    cudaError_t e = enqueue_integrate(h, kernel, state, comp, w, L, P, nsteps, h->cap_stream);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      return RK4_ECUDA;
    }
    e = cudaGraphInstantiate(&h->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      h->gexec = nullptr;
      return RK4_ECUDA;
    }
    h->gkey = key;
  }
  return cudaGraphLaunch(h->gexec, h->stream) == cudaSuccess ? RK4_OK : RK4_ECUDA;
}

int validate_common(int model, int precision, double dt, const rk4_params *p) {
  if (model != RK4_ROESSLER && model != RK4_HARMONIC) return RK4_EINVAL;
  if (precision != RK4_FP64 && precision != RK4_FP32_KAHAN) return RK4_EINVAL;
  if (!(std::isfinite(dt) && dt > 0.0)) return RK4_EINVAL;
  if (p && !(std::isfinite(p->a) && std::isfinite(p->b) && std::isfinite(p->c) && std::isfinite(p->kappa) &&
             std::isfinite(p->omega0)))
    return RK4_EINVAL;
  return RK4_OK;
}

rk4_chain *new_handle(int model, int precision, double dt, const rk4_params *p, void *stream) {
  rk4_chain *h = new (std::nothrow) rk4_chain();
  if (!h) return nullptr;
  h->model = model;
  h->precision = precision;
  h->fp32 = precision == RK4_FP32_KAHAN;
  h->D = model == RK4_ROESSLER ? 3 : 2;
  h->dt = dt;
  if (p) h->p = *p; else rk4_params_default(&h->p);
  h->stream = static_cast<cudaStream_t>(stream);
  h->tab = classical_rk4();
  default_tiling(h);
  return h;
}

// Device address of page-locked host memory that the device can access, or NULL (pageable
// memory, or memory the runtime does not know).
void *mapped_host(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // clear the error of the query
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || a.devicePointer == nullptr) return nullptr;
  // the device address of this very byte (the query names the start of p's allocation)
  return static_cast<char *>(a.devicePointer) + (static_cast<const char *>(p) - static_cast<const char *>(a.hostPointer));
}

// One host <-> device transfer of integrate_host: by the SMs when the host buffer is mapped
// page-locked memory and both sides are 16-byte aligned (k_copy.cu), else by cudaMemcpyAsync.
cudaError_t host_transfer(void *dst, const void *src, size_t bytes, bool to_device, cudaStream_t st) {
  void *hd = mapped_host(to_device ? src : dst);
  if (hd && ((reinterpret_cast<uintptr_t>(hd) | reinterpret_cast<uintptr_t>(to_device ? dst : src)) & 15u) == 0)
    return to_device ? launch_copy(dst, hd, bytes, st) : launch_copy(hd, src, bytes, st);
  return cudaMemcpyAsync(dst, src, bytes, to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost, st);
}

}  // namespace

// Read-only view of a handle for the allocation-free reduction entry point.
int rk4d::handle_info(const rk4_chain *h, int *model, bool *fp32, int *nchains, const ChainDesc **chains, CoefD *cf,
                      cudaStream_t *stream, bool *het) {
  if (!h) return RK4_EINVAL;
  *het = use_het(h);
  *model = h->model;
  *fp32 = h->fp32;
  *nchains = h->nchains;
  *chains = h->chains.data();
  *cf = coef(h);
  *stream = h->stream;
  return RK4_OK;
}

unsigned rk4d::config_version(const rk4_chain *h) { return h->config_version; }

cudaStream_t rk4d::swap_stream(rk4_chain *h, cudaStream_t st) {
  cudaStream_t old = h->stream;
  h->stream = st;
  return old;
}

bool rk4d::swap_graphs(rk4_chain *h, bool on) {
  const bool old = h->graphs;
  h->graphs = on;
  return old;
}

int rk4d::prepare_integrate(rk4_chain *h, int64_t nsteps) {
  if (!h || nsteps < 1) return RK4_EINVAL;
  if (ensure_pinned(h) != cudaSuccess) return RK4_ECUDA;
  const int kernel = effective_kernel(h);
  const Plan P = make_plan(nsteps, kernel == RK4_KERNEL_STAGED ? 1 : h->tiling.k);
  return prepare_tables(h, P.kval, h->tiling.block * h->tiling.v) == cudaSuccess ? RK4_OK : RK4_ECUDA;
}

int rk4d::scheme_reach(const rk4_chain *h, int *s, int *range) {
  if (!h) return RK4_EINVAL;
  *s = needed_stages(h);
  *range = coupling_range(h);
  return RK4_OK;
}

extern "C" {

void rk4_params_default(rk4_params *p) {
  if (!p) return;
  p->a = 0.2;
  p->b = 1.0;
  p->c = 9.0;
  p->kappa = 1.0;
  p->omega0 = 1.0;
}

int rk4_chain_create(rk4_chain **out, int model, int precision, int64_t n, double dt, int bc, const rk4_params *p,
                     void *cuda_stream) {
  if (!out) return RK4_EINVAL;
  *out = nullptr;
  int rc = validate_common(model, precision, dt, p);
  if (rc) return rc;
  if (n < 1 || n > ((int64_t)1 << 40)) return RK4_EINVAL;
  if (bc != RK4_PERIODIC && bc != RK4_FIXED) return RK4_EINVAL;
  rk4_chain *h = new_handle(model, precision, dt, p, cuda_stream);
  if (!h) return RK4_EINVAL;
  ChainDesc c{};
  c.off = 0;
  c.n = n;
  c.kappa = h->p.kappa;
  c.bc = bc;
  h->chains.push_back(c);
  h->nchains = 1;
  h->total = n;
  *out = h;
  return RK4_OK;
}

int rk4_batch_create(rk4_chain **out, int model, int precision, int nchains, const int64_t *lengths,
                     const double *kappa, const int8_t *bc, double dt, const rk4_params *p, void *cuda_stream) {
  if (!out) return RK4_EINVAL;
  *out = nullptr;
  int rc = validate_common(model, precision, dt, p);
  if (rc) return rc;
  if (nchains < 1 || !lengths || !kappa || !bc) return RK4_EINVAL;
  int64_t total = 0;
  for (int c = 0; c < nchains; ++c) {
    if (lengths[c] < 1 || !std::isfinite(kappa[c]) || (bc[c] != RK4_PERIODIC && bc[c] != RK4_FIXED))
      return RK4_EINVAL;
    total += lengths[c];
    if (total > ((int64_t)1 << 40)) return RK4_EINVAL;
  }
  rk4_chain *h = new_handle(model, precision, dt, p, cuda_stream);
  if (!h) return RK4_EINVAL;
  int64_t off = 0;
  for (int c = 0; c < nchains; ++c) {
    ChainDesc d{};
    d.off = off;
    d.n = lengths[c];
    d.kappa = kappa[c];
    d.bc = bc[c];
    h->chains.push_back(d);
    off += lengths[c];
  }
  h->nchains = nchains;
  h->total = total;
  *out = h;
  return RK4_OK;
}

int rk4_chain_workspace_bytes(const rk4_chain *h, size_t *bytes) {
  if (!h || !bytes) return RK4_EINVAL;
  *bytes = layout(h, effective_kernel(h)).total;
  return RK4_OK;
}

int rk4_chain_shape(const rk4_chain *h, int64_t *total_sites, int *dim) {
  if (!h) return RK4_EINVAL;
  if (total_sites) *total_sites = h->total;
  if (dim) *dim = h->D;
  return RK4_OK;
}

int rk4_chain_set_kernel(rk4_chain *h, int kernel) {
  if (!h || kernel < RK4_KERNEL_AUTO || kernel > RK4_KERNEL_PERSISTENT) return RK4_EINVAL;
  h->config_version++;
  h->kernel = kernel;
  h->tuned_kernel = 0;
  return RK4_OK;
}

int rk4_chain_set_tiling(rk4_chain *h, int block, int v, int k) {
  if (!h) return RK4_EINVAL;
  h->config_version++;
  if (block == 0) {
    h->tiling_auto = true;
    default_tiling(h);
    return RK4_OK;
  }
  if (!tiling_valid(h, block, v, k)) return RK4_EINVAL;
  const int maxt = tiling_max_threads(h, v);
  if (maxt > 0 && block > maxt) return RK4_EINVAL;
  if (h->tuned_kernel == RK4_KERNEL_STAGED) h->tuned_kernel = 0;  // a tiling asks for a tiled scheme
  h->tiling_auto = false;
  h->tiling.block = block;
  h->tiling.v = v;
  h->tiling.k = k;
  h->tiling.G = tile_interior(h, block * v, k);
  return RK4_OK;
}

int rk4_chain_get_tiling(const rk4_chain *h, rk4_tiling *out) {
  if (!h || !out) return RK4_EINVAL;
  *out = h->tiling;
  return RK4_OK;
}

int rk4_chain_get_kernel(const rk4_chain *h, int *kernel) {
  if (!h || !kernel) return RK4_EINVAL;
  *kernel = effective_kernel(h);
  return RK4_OK;
}

// NVTX range around a host-side call (visible in Nsight timelines; no cost without a tool).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

int rk4_chain_integrate(rk4_chain *h, void *state, void *comp, void *ws, size_t ws_bytes, int64_t nsteps, double *t) {
  if (!h) return RK4_EINVAL;
  NvtxRange range("rk4_chain_integrate");
  int rc = integrate_impl(h, state, comp, ws, ws_bytes, nsteps);
  if (rc == RK4_OK) {
    h->nstep += nsteps;
    if (t) *t = h->t0 + (double)h->nstep * h->dt;
  }
  return rc;
}

int rk4_chain_step(rk4_chain *h, void *state, void *comp, void *ws, size_t ws_bytes, double *t) {
  return rk4_chain_integrate(h, state, comp, ws, ws_bytes, 1, t);
}

int rk4_chain_integrate_host(rk4_chain *h, void *host_state, void *host_comp, void *dev_state, void *dev_comp,
                             void *ws, size_t ws_bytes, int64_t nsteps, double *t) {
  if (!h || !host_state) return RK4_EINVAL;
  if (h->fp32 != (host_comp != nullptr)) return RK4_EINVAL;
  int rc = check_buffers(h, dev_state, dev_comp, ws);
  if (rc) return rc;
  if (ws_bytes < layout(h, effective_kernel(h)).total) return RK4_ENOMEM_WS;
  const size_t bytes = (size_t)h->total * h->D * elem_bytes(h);
  if (host_transfer(dev_state, host_state, bytes, true, h->stream) != cudaSuccess) return RK4_ECUDA;
  if (h->fp32 && host_transfer(dev_comp, host_comp, bytes, true, h->stream) != cudaSuccess) return RK4_ECUDA;
  rc = rk4_chain_integrate(h, dev_state, dev_comp, ws, ws_bytes, nsteps, t);
  if (rc) return rc;
  if (host_transfer(host_state, dev_state, bytes, false, h->stream) != cudaSuccess) return RK4_ECUDA;
  if (h->fp32 && host_transfer(host_comp, dev_comp, bytes, false, h->stream) != cudaSuccess) return RK4_ECUDA;
  return cudaStreamSynchronize(h->stream) == cudaSuccess ? RK4_OK : RK4_ECUDA;
}

int rk4_chain_energy(rk4_chain *h, const void *state, const void *comp, void *ws, size_t ws_bytes, double *out) {
  if (!h || !out) return RK4_EINVAL;
  NvtxRange range("rk4_chain_energy");
  if (use_het(h) && h->model == RK4_HARMONIC) return RK4_EUNSUPPORTED;
  int rc = check_buffers(h, state, comp, ws);
  if (rc) return rc;
  const WsLayout L = layout(h, effective_kernel(h));
  if (ws_bytes < L.total) return RK4_ENOMEM_WS;
  if (ensure_pinned(h) != cudaSuccess) return RK4_ECUDA;
  char *w = static_cast<char *>(ws);
  WsHeader *hdr = reinterpret_cast<WsHeader *>(w + L.hdr);
  if (cudaMemsetAsync(hdr, 0, sizeof(WsHeader), h->stream) != cudaSuccess) return RK4_ECUDA;
  if (upload_tables(h, w, L, h->stream) != cudaSuccess) return RK4_ECUDA;
  const CoefD cf = coef(h);
  double *res = reinterpret_cast<double *>(w + L.result);
  if (launch_energy(h->model, h->fp32, state, comp, h->nchains, h->chains[0], dev_chains(h, w, L), cf,
                    reinterpret_cast<double *>(w + L.partials), res, hdr, h->stream) != cudaSuccess)
    return RK4_ECUDA;
  if (cudaMemcpyAsync(h->h_out, res, sizeof(double) * h->nchains, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
    return RK4_ECUDA;
  if (cudaMemcpyAsync(h->h_status, &hdr->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
    return RK4_ECUDA;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return RK4_ECUDA;
  std::memcpy(out, h->h_out, sizeof(double) * h->nchains);
  if (*h->h_status & ST_NONFINITE) return RK4_ENONFINITE;
  return RK4_OK;
}

int rk4_chain_status(rk4_chain *h, void *ws) {
  if (!h || !ws) return RK4_EINVAL;
  if (ensure_pinned(h) != cudaSuccess) return RK4_ECUDA;
  const WsLayout L = layout(h, effective_kernel(h));
  WsHeader *hdr = reinterpret_cast<WsHeader *>(static_cast<char *>(ws) + L.hdr);
  if (cudaMemcpyAsync(h->h_status, &hdr->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
    return RK4_ECUDA;
  if (cudaMemsetAsync(&hdr->status, 0, sizeof(int), h->stream) != cudaSuccess) return RK4_ECUDA;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return RK4_ECUDA;
  const int s = *h->h_status;
  if (s & ST_TIMEOUT) return RK4_ETIMEOUT;
  if (s & ST_BOUNDS) return RK4_EBOUNDS;
  if (s & ST_NONFINITE) return RK4_ENONFINITE;
  return RK4_OK;
}

int rk4_chain_set_option(rk4_chain *h, int option, int64_t value) {
  if (!h) return RK4_EINVAL;
  h->config_version++;
  if (option == RK4_OPT_GRAPHS) {
    if (value != 0 && value != 1) return RK4_EINVAL;
    h->graphs = value != 0;
    return RK4_OK;
  }
  if (option == RK4_OPT_TIMEOUT_NS) {
    if (value < 1000 || value > (int64_t)600 * 1000000000LL) return RK4_EINVAL;
    h->timeout_ns = value;
    h->timeout_set = true;
    return RK4_OK;
  }
  return RK4_EINVAL;
}

int rk4_debug_barrier_timeout(rk4_chain *h, void *state, void *comp, void *ws, size_t ws_bytes, int64_t timeout_ns) {
  if (!h) return RK4_EINVAL;
  int rc = check_buffers(h, state, comp, ws);
  if (rc) return rc;
  if (timeout_ns < 1000 || timeout_ns > 10LL * 1000000000LL) return RK4_EINVAL;
  const WsLayout L = layout(h, RK4_KERNEL_PERSISTENT);
  if (ws_bytes < L.total) return RK4_ENOMEM_WS;
  if (ensure_pinned(h) != cudaSuccess) return RK4_ECUDA;
  const Plan P = make_plan(h->tiling.k, h->tiling.k);  // one time block
  const int W = h->tiling.block * h->tiling.v;
  if (prepare_tables(h, P.kval, W) != cudaSuccess) return RK4_ECUDA;
  char *w = static_cast<char *>(ws);
  if (upload_tables(h, w, L, h->stream) != cudaSuccess) return RK4_ECUDA;
  if (fill_tile_tables(h, w, L, 1, h->stream) != cudaSuccess) return RK4_ECUDA;
  PersistentJob j{};
  j.bufA = state;
  j.bufB = w + L.state;
  j.cA = comp;
  j.cB = h->fp32 ? (void *)(w + L.comp) : nullptr;
  j.nchains = h->nchains;
  j.one = h->chains[0];
  j.chains = dev_chains(h, w, L);
  j.nk = 1;
  j.kval[0] = h->tiling.k;
  if (use_generic(h)) return RK4_EUNSUPPORTED;
  j.Gval[0] = tile_interior(h, W, h->tiling.k);
  if (h->nchains > 1) {
    j.bt[0] = dev_ktables(h, w, L, 0);
    j.ntiles[0] = j.bt[0].nfull + j.bt[0].npacked;
  } else {
    j.ntiles[0] = tiles_for(h, j.Gval[0]);
  }
  j.nmain = 1;
  j.ntail = 0;
  j.hdr = reinterpret_cast<WsHeader *>(w + L.hdr);
  j.total = h->total;
  j.timeout_ns = timeout_ns;
  j.extra_arrivals = 1;
  int grid = persistent_max_grid(h->model, h->fp32, h->tiling.v, h->tiling.block);
  if (grid <= 0) return RK4_ECUDA;
  grid = (int)std::min<int64_t>(grid, std::max<int64_t>(1, j.ntiles[0]));
  if (cudaMemsetAsync(w + L.hdr, 0, sizeof(WsHeader), h->stream) != cudaSuccess) return RK4_ECUDA;
  if (launch_persistent(h->model, h->fp32, h->tiling.v, h->tiling.block, grid, j, coef(h), h->stream) !=
      cudaSuccess)
    return RK4_ECUDA;
  return RK4_OK;
}

int rk4_chain_autotune(rk4_chain *h, void *state, void *comp, void *ws, size_t ws_bytes, int probe_steps,
                       rk4_tiling *best) {
  if (!h || probe_steps < 1 || probe_steps > 100000) return RK4_EINVAL;
  NvtxRange range("rk4_chain_autotune");
  int rc = check_buffers(h, state, comp, ws);
  if (rc) return rc;
  if (h->kernel == RK4_KERNEL_STAGED) {  // the one-stage-per-launch scheme has nothing to tune
    if (best) *best = h->tiling;
    return RK4_OK;
  }
  // Candidate schemes.  An explicit choice is kept.  On RK4_KERNEL_AUTO: the blocked scheme, for
  // a batch also the persistent one, and the staged scheme whenever ws is large enough for it.
  const bool tiled_only = use_generic(h) || use_het(h);
  const bool on_auto = h->kernel == RK4_KERNEL_AUTO;
  std::vector<int> kernels;
  if (!on_auto) {
    kernels.push_back(h->kernel);
  } else {
    if (h->nchains > 1 && !tiled_only) kernels.push_back(RK4_KERNEL_PERSISTENT);
    kernels.push_back(RK4_KERNEL_BLOCKED);
  }
  for (size_t i = 0; i < kernels.size();)  // only the schemes the caller's workspace can hold
    if (ws_bytes < layout(h, kernels[i]).total) kernels.erase(kernels.begin() + (long)i); else ++i;
  const bool try_staged = on_auto && ws_bytes >= layout(h, RK4_KERNEL_STAGED).total;
  if (kernels.empty() && !try_staged) return RK4_ENOMEM_WS;
  const rk4_tiling saved = h->tiling;
  const int saved_tuned = h->tuned_kernel;
  int best_kernel = 0;
  const bool saved_graphs = h->graphs;
  h->graphs = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    h->graphs = saved_graphs;
    return RK4_ECUDA;
  }
  // Per-step time of an integration of `steps` after a warm-up of `warm`, or a negative value
  // when the configuration fails to run.
  auto time_steps = [&](int64_t warm, int64_t steps) -> float {
    if (integrate_impl(h, state, comp, ws, ws_bytes, warm) != RK4_OK) return -1.f;
    cudaEventRecord(e0, h->stream);
    if (integrate_impl(h, state, comp, ws, ws_bytes, steps) != RK4_OK) return -1.f;
    cudaEventRecord(e1, h->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      rc = RK4_ECUDA;
      return -1.f;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms / (float)steps;
  };
  static const int blocks[] = {64, 128, 256, 512, 1024};
  static const int vs[] = {1, 2, 4, 8};
  static const int ks[] = {1, 2, 4, 8, 16};
  float best_ms = 1e30f;
  rk4_tiling best_t = saved;
  bool have_tiling = false;
  rc = RK4_OK;
  for (int kern : kernels) {
    if (rc != RK4_OK) break;
    if (on_auto) h->tuned_kernel = kern;
    for (int b : blocks)
      for (int v : vs)
        for (int k : ks) {
          if (rc != RK4_OK) break;
          if (!tiling_valid(h, b, v, k)) continue;
          if (b == 64 && !use_generic(h)) continue;
          const int maxt = tiling_max_threads(h, v);
          if (maxt <= 0 || b > maxt) continue;
          if (kern == RK4_KERNEL_PERSISTENT && persistent_max_grid(h->model, h->fp32, v, b) <= 0) continue;
          h->tiling.block = b;
          h->tiling.v = v;
          h->tiling.k = k;
          h->tiling.G = tile_interior(h, b * v, k);
          const int64_t steps = ((probe_steps + 2 * k - 1) / (2 * k)) * 2 * k;  // whole, even launch count
          const float per_step = time_steps(2 * k, steps);
          if (per_step >= 0.f && per_step < best_ms) {
            best_ms = per_step;
            best_t = h->tiling;
            best_kernel = kern;
            have_tiling = true;
          }
        }
  }
  if (rc == RK4_OK && try_staged) {
    h->tuned_kernel = RK4_KERNEL_STAGED;
    const float per_step = time_steps(1, probe_steps);
    if (per_step >= 0.f && per_step < best_ms) {
      best_ms = per_step;
      best_kernel = RK4_KERNEL_STAGED;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->graphs = saved_graphs;
  if (rc != RK4_OK || best_ms >= 1e30f) {
    h->tiling = saved;
    h->tuned_kernel = saved_tuned;
    return rc != RK4_OK ? rc : RK4_ECUDA;
  }
  h->tuned_kernel = on_auto ? best_kernel : 0;
  h->config_version++;
  h->tiling = have_tiling ? best_t : saved;
  h->tiling_auto = !have_tiling && h->tiling_auto;
  if (best) *best = h->tiling;
  return RK4_OK;
}

int rk4_chain_set_tableau(rk4_chain *h, int s, const double *A, const double *b) {
  if (!h) return RK4_EINVAL;
  h->config_version++;
  h->tuned_kernel = 0;
  if (s == 0) {  // back to the classical RK4 kernels
    h->has_tableau = false;
    h->tab = classical_rk4();
    default_tiling(h);
    return RK4_OK;
  }
  if (s < 1 || s > kMaxStages || !A || !b) return RK4_EINVAL;
  TableauD t{};
  t.s = s;
  for (int j = 0; j < s; ++j) {
    if (!std::isfinite(b[j])) return RK4_EINVAL;
    t.b[j] = b[j];
    for (int m = 0; m < s; ++m) {
      const double a = A[j * s + m];
      if (!std::isfinite(a)) return RK4_EINVAL;
      if (m >= j && a != 0.0) return RK4_EINVAL;  // explicit schemes only
      if (m < j) t.a[j][m] = a;
    }
  }
  h->has_tableau = true;
  h->tab = t;
  h->gen_version++;
  default_tiling(h);
  return RK4_OK;
}

int rk4_chain_set_coupling2(rk4_chain *h, double kappa2) {
  if (!h || !std::isfinite(kappa2)) return RK4_EINVAL;
  h->config_version++;
  h->tuned_kernel = 0;
  h->kappa2 = kappa2;
  if (!h->has_tableau) h->tab = classical_rk4();
  h->gen_version++;
  default_tiling(h);
  return RK4_OK;
}

int rk4_chain_set_site_params(rk4_chain *h, const void *params) {
  if (!h) return RK4_EINVAL;
  if (params && (reinterpret_cast<uintptr_t>(params) % 16) != 0) return RK4_EINVAL;
  h->config_version++;
  h->tuned_kernel = 0;
  h->site_params = params;
  default_tiling(h);
  return RK4_OK;
}

int rk4_chain_get_clock(const rk4_chain *h, double *t0, int64_t *nstep) {
  if (!h) return RK4_EINVAL;
  if (t0) *t0 = h->t0;
  if (nstep) *nstep = h->nstep;
  return RK4_OK;
}

int rk4_chain_set_clock(rk4_chain *h, double t0, int64_t nstep) {
  if (!h || !std::isfinite(t0) || nstep < 0) return RK4_EINVAL;
  h->t0 = t0;
  h->nstep = nstep;
  return RK4_OK;
}

int rk4_chain_set_time(rk4_chain *h, double t0) {
  if (!h || !std::isfinite(t0)) return RK4_EINVAL;
  h->t0 = t0;
  h->nstep = 0;
  return RK4_OK;
}

int rk4_chain_destroy(rk4_chain *h) {
  if (!h) return RK4_OK;
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->h_tables) cudaFreeHost(h->h_tables);
  if (h->h_out) cudaFreeHost(h->h_out);
  if (h->h_status) cudaFreeHost(h->h_status);
  delete h;
  return RK4_OK;
}

const char *rk4_strerror(int code) {
  switch (code) {
    case RK4_OK: return "ok";
    case RK4_EINVAL: return "invalid argument";
    case RK4_ENOMEM_WS: return "workspace too small";
    case RK4_ECUDA: return "CUDA runtime error";
    case RK4_ENONFINITE: return "non-finite value in the state";
    case RK4_ETIMEOUT: return "device-side wait timed out";
    case RK4_EUNSUPPORTED: return "unsupported request";
    case RK4_EBOUNDS: return "an index check of the debug build caught an out-of-range access";
    default: return "unknown error";
  }
}

int rk4_fill_uniform(void *dst, int64_t count, uint64_t seed, uint64_t start, int precision, void *cuda_stream) {
  if (!dst || count < 0) return RK4_EINVAL;
  if (precision != RK4_FP64 && precision != RK4_FP32_KAHAN) return RK4_EINVAL;
  return launch_fill_uniform(dst, count, seed, start, precision == RK4_FP32_KAHAN,
                             static_cast<cudaStream_t>(cuda_stream)) == cudaSuccess
             ? RK4_OK
             : RK4_ECUDA;
}

}  // extern "C"
