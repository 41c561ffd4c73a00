// rk4_domain.cu -- host runtime of the sub-domain decomposition (include/rk4chain.h,
// rk4_domain_*): one chain split into contiguous parts, each stored with ghost zones and
// integrated as an independent fixed-end chain between ghost exchanges.
//
// Why the interiors come out exact: a fixed-end part sees zeros beyond its outer ghost site,
// so its outermost sites go wrong, and the error front moves one coupling range per stage:
// after m steps of an s-stage scheme with coupling range r it has reached s r m sites into the
// part.  With ghost zones of `ghost` sites, exchanging every floor(ghost / (s r)) steps keeps
// the front inside the ghosts, and every interior site performs exactly the operations it
// performs in the undivided chain (the kernels evaluate each site with the same per-site code
// whatever the tiling), so the interiors are bit-identical to the whole-chain run.  This is
// the paper's granularity with overlap (Sec. 2.3) applied to memory partitions instead of
// cache-sized clusters.
//
// Layout of the domain state: the parts' extended blocks back to back, part p holding rows
// [ghost_left | sites | ghost_right].  A part has a left (right) ghost zone unless it is the
// first (last) part of a fixed-end chain.  The parts form one batch handle of fixed-end
// chains, so one launch advances all of them.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/rk4chain.h"
#include "rk4_internal.h"

using namespace rk4d;

struct rk4_domain {
  rk4_chain *h = nullptr;  // batch of nparts fixed-end chains over the extended blocks
  int model = 0, D = 3, bc = 0, nparts = 1;
  bool fp32 = false;
  size_t es = 8;
  int64_t n = 0, ghost = 0, rows = 0;
  double dt = 0.01;
  std::vector<int64_t> site0, sites, row, gl, gr;  // per part
  cudaStream_t stream = nullptr;
  std::vector<GhostPair> pairs;  // every ghost zone and the rows it is copied from
  GhostPair *h_pairs = nullptr;   // pinned copy of `pairs`, uploaded to the workspace
  double *h_out = nullptr;        // pinned: per-part energies
  int *h_status = nullptr;        // pinned: status word read-back
  int64_t nstep = 0;              // steps taken (t = nstep dt)
  // one CUDA graph of whole exchange periods (exchange + the parts' launches), replayed
  cudaStream_t cap = nullptr;
  cudaGraphExec_t gexec = nullptr;
  const void *g_state = nullptr, *g_comp = nullptr, *g_ws = nullptr;
  int64_t g_period = 0, g_nper = 0;
  unsigned g_version = 0;
};

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

bool any_ghost(const rk4_domain *d) { return d->bc == RK4_PERIODIC || d->nparts > 1; }

size_t batch_ws_bytes(const rk4_domain *d) {
  size_t b = 0;
  rk4_chain_workspace_bytes(d->h, &b);
  return align_up(b);
}

// Domain workspace: the batch handle's workspace, then a status header, the reduction partials,
// one result per part and the ghost-zone table.
struct DomLayout {
  size_t batch, hdr, partials, result, pairs, total;
};

DomLayout dom_layout(const rk4_domain *d) {
  DomLayout L{};
  L.batch = batch_ws_bytes(d);
  L.hdr = L.batch;
  L.partials = L.hdr + align_up(sizeof(WsHeader));
  L.result = L.partials + align_up(sizeof(double) * kEnergyBlocks);
  L.pairs = L.result + align_up(sizeof(double) * (size_t)d->nparts);
  L.total = L.pairs + align_up(sizeof(GhostPair) * d->pairs.size());
  return L;
}

int check_pair(const rk4_domain *d, const void *state, const void *comp) {
  if (!state) return RK4_EINVAL;
  if (d->fp32 != (comp != nullptr)) return RK4_EINVAL;
  if ((reinterpret_cast<uintptr_t>(state) % 16) != 0) return RK4_EINVAL;
  if (comp && (reinterpret_cast<uintptr_t>(comp) % 16) != 0) return RK4_EINVAL;
  return RK4_OK;
}

cudaError_t copy_rows(const rk4_domain *d, void *dst, int64_t dst_row, const void *src, int64_t src_row,
                      int64_t nrows) {
  if (nrows <= 0) return cudaSuccess;
  const size_t rb = (size_t)d->D * d->es;
  return cudaMemcpyAsync(static_cast<char *>(dst) + (size_t)dst_row * rb,
                         static_cast<const char *>(src) + (size_t)src_row * rb, (size_t)nrows * rb,
                         cudaMemcpyDeviceToDevice, d->stream);
}

// Every ghost zone and its source: the left ghosts of part p are the last `ghost` sites of part
// p - 1, its right ghosts the first `ghost` sites of part p + 1 (cyclically for periodic ends;
// a single periodic part is its own neighbour).
void build_pairs(rk4_domain *d) {
  const int P = d->nparts;
  for (int p = 0; p < P; ++p) {
    if (d->gl[p]) {
      const int q = (p + P - 1) % P;
      d->pairs.push_back({d->row[p], d->row[q] + d->gl[q] + d->sites[q] - d->ghost});
    }
    if (d->gr[p]) {
      const int r = (p + 1) % P;
      d->pairs.push_back({d->row[p] + d->gl[p] + d->sites[p], d->row[r] + d->gl[r]});
    }
  }
}

// The exchange as plain device-to-device copies, one per zone and array (for the calls that
// have no workspace to hold the zone table).
cudaError_t exchange(const rk4_domain *d, void *state, void *comp) {
  for (const GhostPair &z : d->pairs) {
    cudaError_t e = copy_rows(d, state, z.dst_row, state, z.src_row, d->ghost);
    if (e == cudaSuccess && comp) e = copy_rows(d, comp, z.dst_row, comp, z.src_row, d->ghost);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// The zone table into the workspace (once per call); then every exchange is one launch.  The
// pinned staging copy is made on first use (creating a domain touches no CUDA API).
cudaError_t upload_pairs(rk4_domain *d, char *ws, const DomLayout &L) {
  if (d->pairs.empty()) return cudaSuccess;
  if (!d->h_pairs) {
    cudaError_t e = cudaMallocHost((void **)&d->h_pairs, sizeof(GhostPair) * d->pairs.size());
    if (e != cudaSuccess) return e;
    std::memcpy(d->h_pairs, d->pairs.data(), sizeof(GhostPair) * d->pairs.size());
  }
  return cudaMemcpyAsync(ws + L.pairs, d->h_pairs, sizeof(GhostPair) * d->pairs.size(), cudaMemcpyHostToDevice,
                         d->stream);
}

cudaError_t exchange_kernel(const rk4_domain *d, void *state, void *comp, char *ws, const DomLayout &L) {
  return launch_ghost_copy(state, comp, reinterpret_cast<const GhostPair *>(ws + L.pairs), (int)d->pairs.size(),
                           d->ghost, d->D * (int)d->es, d->stream);
}

}  // namespace

extern "C" {

int rk4_domain_create(rk4_domain **out, int model, int precision, int64_t n, double dt, int bc, const rk4_params *p,
                      int nparts, const int64_t *part_lengths, int64_t ghost, void *cuda_stream) {
  if (!out) return RK4_EINVAL;
  *out = nullptr;
  if (bc != RK4_PERIODIC && bc != RK4_FIXED) return RK4_EINVAL;
  if (n < 1 || n > ((int64_t)1 << 40) || nparts < 1 || nparts > 65536 || nparts > n) return RK4_EINVAL;
  if (ghost < 0 || ghost > ((int64_t)1 << 30)) return RK4_EINVAL;
  rk4_domain *d = new (std::nothrow) rk4_domain();
  if (!d) return RK4_EINVAL;
  d->model = model;
  d->bc = bc;
  d->nparts = nparts;
  d->n = n;
  d->ghost = ghost;
  d->dt = dt;
  d->D = model == RK4_ROESSLER ? 3 : 2;
  d->fp32 = precision == RK4_FP32_KAHAN;
  d->es = d->fp32 ? 4 : 8;
  d->stream = static_cast<cudaStream_t>(cuda_stream);
  const bool ghosts = any_ghost(d);
  if (ghosts && ghost < 1) {
    delete d;
    return RK4_EINVAL;
  }
  int64_t s0 = 0, r0 = 0;
  for (int q = 0; q < nparts; ++q) {
    const int64_t len = part_lengths ? part_lengths[q] : n / nparts + (q < n % nparts ? 1 : 0);
    // a neighbour's ghost zone is copied from one part's interior only
    if (len < 1 || (ghosts && len < ghost)) {
      delete d;
      return RK4_EINVAL;
    }
    const int64_t l = (bc == RK4_PERIODIC || q > 0) ? ghost : 0;
    const int64_t r = (bc == RK4_PERIODIC || q < nparts - 1) ? ghost : 0;
    d->site0.push_back(s0);
    d->sites.push_back(len);
    d->row.push_back(r0);
    d->gl.push_back(l);
    d->gr.push_back(r);
    s0 += len;
    r0 += l + len + r;
  }
  if (s0 != n) {
    delete d;
    return RK4_EINVAL;
  }
  d->rows = r0;
  build_pairs(d);
  std::vector<int64_t> ext(nparts);
  std::vector<double> kap(nparts);
  std::vector<int8_t> bcs(nparts, (int8_t)RK4_FIXED);
  rk4_params prm;
  if (p) prm = *p; else rk4_params_default(&prm);
  for (int q = 0; q < nparts; ++q) {
    ext[q] = d->gl[q] + d->sites[q] + d->gr[q];
    kap[q] = prm.kappa;
  }
  int rc = rk4_batch_create(&d->h, model, precision, nparts, ext.data(), kap.data(), bcs.data(), dt, &prm,
                            cuda_stream);
  if (rc != RK4_OK) {
    delete d;
    return rc;
  }
  // few long parts: one blocked launch over all of them is the natural scheme.  FP32 runs
  // several steps per launch (bandwidth-bound at k = 1): an exchange period of P steps runs as
  // two launches of P / 2 steps (an integration ends in the caller's buffer after an even
  // number of launches), so that is the default k
  rk4_chain_set_kernel(d->h, RK4_KERNEL_BLOCKED);
  if (d->fp32 && ghosts) {
    const int k = (int)std::min<int64_t>(16, std::max<int64_t>(1, ghost / 8));
    rk4_chain_set_tiling(d->h, 256, 4, k);  // keeps the default if this shape is not valid
  }
  *out = d;
  return RK4_OK;
}

int rk4_domain_part(const rk4_domain *d, int part, int64_t *first_site, int64_t *sites, int64_t *row,
                    int64_t *ghost_left, int64_t *ghost_right) {
  if (!d || part < 0 || part >= d->nparts) return RK4_EINVAL;
  if (first_site) *first_site = d->site0[part];
  if (sites) *sites = d->sites[part];
  if (row) *row = d->row[part];
  if (ghost_left) *ghost_left = d->gl[part];
  if (ghost_right) *ghost_right = d->gr[part];
  return RK4_OK;
}

int rk4_domain_shape(const rk4_domain *d, int64_t *rows, int *dim) {
  if (!d) return RK4_EINVAL;
  if (rows) *rows = d->rows;
  if (dim) *dim = d->D;
  return RK4_OK;
}

int rk4_domain_chain(rk4_domain *d, rk4_chain **parts) {
  if (!d || !parts) return RK4_EINVAL;
  *parts = d->h;
  return RK4_OK;
}

int rk4_domain_workspace_bytes(const rk4_domain *d, size_t *bytes) {
  if (!d || !bytes) return RK4_EINVAL;
  *bytes = dom_layout(d).total;
  return RK4_OK;
}

int rk4_domain_scatter(rk4_domain *d, const void *chain_state, const void *chain_comp, void *state, void *comp) {
  if (!d) return RK4_EINVAL;
  if (check_pair(d, chain_state, chain_comp) || check_pair(d, state, comp)) return RK4_EINVAL;
  for (int p = 0; p < d->nparts; ++p) {
    if (copy_rows(d, state, d->row[p] + d->gl[p], chain_state, d->site0[p], d->sites[p]) != cudaSuccess)
      return RK4_ECUDA;
    if (comp && copy_rows(d, comp, d->row[p] + d->gl[p], chain_comp, d->site0[p], d->sites[p]) != cudaSuccess)
      return RK4_ECUDA;
  }
  return exchange(d, state, comp) == cudaSuccess ? RK4_OK : RK4_ECUDA;
}

int rk4_domain_gather(rk4_domain *d, const void *state, const void *comp, void *chain_state, void *chain_comp) {
  if (!d) return RK4_EINVAL;
  if (check_pair(d, state, comp) || check_pair(d, chain_state, chain_comp)) return RK4_EINVAL;
  for (int p = 0; p < d->nparts; ++p) {
    if (copy_rows(d, chain_state, d->site0[p], state, d->row[p] + d->gl[p], d->sites[p]) != cudaSuccess)
      return RK4_ECUDA;
    if (comp && copy_rows(d, chain_comp, d->site0[p], comp, d->row[p] + d->gl[p], d->sites[p]) != cudaSuccess)
      return RK4_ECUDA;
  }
  return RK4_OK;
}

int rk4_domain_exchange(rk4_domain *d, void *state, void *comp) {
  if (!d) return RK4_EINVAL;
  if (check_pair(d, state, comp)) return RK4_EINVAL;
  return exchange(d, state, comp) == cudaSuccess ? RK4_OK : RK4_ECUDA;
}

}  // extern "C"

namespace {

constexpr int64_t kGraphPeriods = 8;  // exchange periods per captured graph

// A chunk of nper whole exchange periods as one CUDA graph, replayed `reps` times: captured on
// first use and reused while the buffers, the chunk and the parts' configuration stay the same
// (the chunk does not depend on a call's step count, so calls of any length share the graph).
int run_periods_graph(rk4_domain *d, void *state, void *comp, char *w, const DomLayout &L, int64_t period,
                      int64_t nper, int64_t reps) {
  // the parts' pinned tables must describe this period's launch plan when the graph runs
  // (another plan, e.g. a remainder of fewer steps, may have rewritten them since)
  int rc = prepare_integrate(d->h, period);
  if (rc != RK4_OK) return rc;
  const unsigned ver = config_version(d->h);
  const bool hit = d->gexec && d->g_state == state && d->g_comp == comp && d->g_ws == w && d->g_period == period &&
                   d->g_nper == nper && d->g_version == ver;
  if (!hit) {
    if (d->gexec) {
      cudaGraphExecDestroy(d->gexec);
      d->gexec = nullptr;
    }
    if (!d->cap && cudaStreamCreateWithFlags(&d->cap, cudaStreamNonBlocking) != cudaSuccess) return RK4_ECUDA;
    if (cudaStreamBeginCapture(d->cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) return RK4_ECUDA;
    const cudaStream_t old_stream = swap_stream(d->h, d->cap);
    const bool old_graphs = swap_graphs(d->h, false);
    double t0 = 0.0;
    int64_t n0 = 0;
    rk4_chain_get_clock(d->h, &t0, &n0);
    const GhostPair *pairs = reinterpret_cast<const GhostPair *>(w + L.pairs);
    for (int64_t p = 0; p < nper && rc == RK4_OK; ++p) {
      if (launch_ghost_copy(state, comp, pairs, (int)d->pairs.size(), d->ghost, d->D * (int)d->es, d->cap) !=
          cudaSuccess)
        rc = RK4_ECUDA;
      else
        rc = rk4_chain_integrate(d->h, state, comp, w, L.batch, period, nullptr);
    }
    swap_graphs(d->h, old_graphs);
    swap_stream(d->h, old_stream);
    rk4_chain_set_clock(d->h, t0, n0);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(d->cap, &g);
    if (rc != RK4_OK || e != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      return rc != RK4_OK ? rc : RK4_ECUDA;
    }
    const cudaError_t ei = cudaGraphInstantiate(&d->gexec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      d->gexec = nullptr;
      return RK4_ECUDA;
    }
    d->g_state = state;
    d->g_comp = comp;
    d->g_ws = w;
    d->g_period = period;
    d->g_nper = nper;
    d->g_version = ver;
  }
  for (int64_t r = 0; r < reps; ++r)
    if (cudaGraphLaunch(d->gexec, d->stream) != cudaSuccess) return RK4_ECUDA;
  return RK4_OK;
}

}  // namespace

extern "C" {

int rk4_domain_integrate(rk4_domain *d, void *state, void *comp, void *ws, size_t ws_bytes, int64_t nsteps,
                         double *t) {
  if (!d || nsteps < 0) return RK4_EINVAL;
  if (check_pair(d, state, comp) || !ws || (reinterpret_cast<uintptr_t>(ws) % kAlign) != 0) return RK4_EINVAL;
  int model = 0, nch = 0, s = 4, range = 1;
  bool fp32 = false, het = false;
  const ChainDesc *chains = nullptr;
  CoefD cf{};
  cudaStream_t st = nullptr;
  handle_info(d->h, &model, &fp32, &nch, &chains, &cf, &st, &het);
  scheme_reach(d->h, &s, &range);
  if (het) return RK4_EUNSUPPORTED;  // the parameters would need ghost zones too
  const DomLayout L = dom_layout(d);
  if (ws_bytes < L.total) return RK4_ENOMEM_WS;
  // steps between exchanges: the error front of the parts' fixed ends stays in the ghosts
  const int64_t period = any_ghost(d) ? d->ghost / ((int64_t)s * range) : std::max<int64_t>(nsteps, 1);
  if (period < 1) return RK4_EUNSUPPORTED;
  char *w = static_cast<char *>(ws);
  if (nsteps > 0 && upload_pairs(d, w, L) != cudaSuccess) return RK4_ECUDA;
  int64_t done = 0;
  const int64_t reps = any_ghost(d) ? nsteps / (period * kGraphPeriods) : 0;
  if (reps >= 1) {  // chunks of whole periods replayed from one graph
    const int rc = run_periods_graph(d, state, comp, w, L, period, kGraphPeriods, reps);
    if (rc != RK4_OK) return rc;
    done = reps * kGraphPeriods * period;
  }
  for (; done < nsteps;) {
    const int64_t m = std::min(period, nsteps - done);
    if (exchange_kernel(d, state, comp, w, L) != cudaSuccess) return RK4_ECUDA;
    const int rc = rk4_chain_integrate(d->h, state, comp, ws, L.batch, m, nullptr);
    if (rc != RK4_OK) return rc;
    done += m;
  }
  d->nstep += nsteps;
  if (t) *t = (double)d->nstep * d->dt;
  return RK4_OK;
}

int rk4_domain_energy(rk4_domain *d, void *state, void *comp, void *ws, size_t ws_bytes, double *out) {
  if (!d || !out) return RK4_EINVAL;
  if (check_pair(d, state, comp) || !ws || (reinterpret_cast<uintptr_t>(ws) % kAlign) != 0) return RK4_EINVAL;
  int model = 0, nch = 0, s = 4, range = 1;
  bool fp32 = false, het = false;
  const ChainDesc *chains = nullptr;
  CoefD cf{};
  cudaStream_t st = nullptr;
  handle_info(d->h, &model, &fp32, &nch, &chains, &cf, &st, &het);
  scheme_reach(d->h, &s, &range);
  if (het && model == RK4_HARMONIC) return RK4_EUNSUPPORTED;  // as rk4_chain_energy
  if (any_ghost(d) && d->ghost < range) return RK4_EUNSUPPORTED;  // bonds must end inside the ghosts
  const DomLayout L = dom_layout(d);
  if (ws_bytes < L.total) return RK4_ENOMEM_WS;
  if (!d->h_out && cudaMallocHost((void **)&d->h_out, sizeof(double) * (size_t)d->nparts) != cudaSuccess)
    return RK4_ECUDA;
  if (!d->h_status && cudaMallocHost((void **)&d->h_status, sizeof(int)) != cudaSuccess) return RK4_ECUDA;
  char *w = static_cast<char *>(ws);
  WsHeader *hdr = reinterpret_cast<WsHeader *>(w + L.hdr);
  double *partials = reinterpret_cast<double *>(w + L.partials);
  double *res = reinterpret_cast<double *>(w + L.result);
  // bonds that cross a part boundary read the neighbour's site from the ghost zone
  if (upload_pairs(d, w, L) != cudaSuccess || exchange_kernel(d, state, comp, w, L) != cudaSuccess)
    return RK4_ECUDA;
  if (cudaMemsetAsync(hdr, 0, sizeof(WsHeader), d->stream) != cudaSuccess) return RK4_ECUDA;
  for (int p = 0; p < d->nparts; ++p) {
    // part p as the fixed-end chain the kernels integrate; its interior is [gl, gl + sites)
    ChainDesc ch = nch > 1 ? chains[p] : chains[0];
    if (launch_energy_range(model, fp32, state, comp, ch, d->gl[p], d->gl[p] + d->sites[p], cf, partials, res + p,
                            hdr, d->stream) != cudaSuccess)
      return RK4_ECUDA;
  }
  if (cudaMemcpyAsync(d->h_out, res, sizeof(double) * (size_t)d->nparts, cudaMemcpyDeviceToHost, d->stream) !=
      cudaSuccess)
    return RK4_ECUDA;
  if (cudaMemcpyAsync(d->h_status, &hdr->status, sizeof(int), cudaMemcpyDeviceToHost, d->stream) != cudaSuccess)
    return RK4_ECUDA;
  if (cudaStreamSynchronize(d->stream) != cudaSuccess) return RK4_ECUDA;
  double e = 0.0;
  for (int p = 0; p < d->nparts; ++p) e += d->h_out[p];  // fixed order: deterministic
  *out = e;
  return (*d->h_status & ST_NONFINITE) ? RK4_ENONFINITE : RK4_OK;
}

int rk4_domain_status(rk4_domain *d, void *ws) {
  if (!d || !ws) return RK4_EINVAL;
  return rk4_chain_status(d->h, ws);
}

int rk4_domain_destroy(rk4_domain *d) {
  if (!d) return RK4_OK;
  if (d->gexec) cudaGraphExecDestroy(d->gexec);
  if (d->cap) cudaStreamDestroy(d->cap);
  rk4_chain_destroy(d->h);
  if (d->h_pairs) cudaFreeHost(d->h_pairs);
  if (d->h_out) cudaFreeHost(d->h_out);
  if (d->h_status) cudaFreeHost(d->h_status);
  delete d;
  return RK4_OK;
}

}  // extern "C"
