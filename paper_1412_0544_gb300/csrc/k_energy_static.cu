// k_energy_static.cu -- the FP64 energy / norm reduction for callers that cannot allocate
// device memory (for example code running where cudaMalloc is forbidden or unavailable: inside
// a host callback, a signal-safe monitoring hook, or an embedding that hands the library no
// workspace).  The reduction's scratch -- block partial sums, per-chain results, the batch
// chain table and the status word -- lives in one file-scope __device__ array instead of the
// caller's workspace.
//
// The array holds kStaticMaxChains chains' worth of scratch (about 330 KB) and stays resident
// on every GPU that loads this library until the process exits.  All calls share it: two
// calls whose work overlaps on the GPU (different streams, or different host threads on one
// device) race on it and must be serialised by the caller.  Each call clears the status word
// before use; everything else it reads is fully rewritten first.
#include <mutex>

#include "../../include/rk4chain.h"
#include "rk4_internal.h"

using namespace rk4d;

namespace {

constexpr int kStaticMaxChains = 8192;

struct StaticScratch {
  WsHeader hdr;
  double partials[kEnergyBlocks];
  double result[kStaticMaxChains];
  ChainDesc chains[kStaticMaxChains];
};

// Host code must not pass this symbol to a kernel: on the host it is only a stand-in whose
// device address comes from cudaGetSymbolAddress (see scratch_for_current_device).
static __device__ __align__(256) unsigned char g_energy_scratch[sizeof(StaticScratch)];

// The address of the array belongs to the device's current context: a cudaDeviceReset
// destroys that context, and the array lives at a new address in the next one.  So the cached
// address is keyed by the context's unique id (cuCtxGetId: ids are never reused within a
// process), read through the driver entry points the runtime exposes.
typedef int (*CtxGetCurrentFn)(void **ctx);
typedef int (*CtxGetIdFn)(void *ctx, unsigned long long *id);

struct Cached {
  bool valid;
  unsigned long long ctx_id;
  StaticScratch *ptr;
};

std::mutex g_mu;
Cached g_cache[kMaxDevices] = {};

// Unique id of the calling thread's current context; false when it cannot be read (no
// current context yet, or a driver without the entry points).
bool current_context_id(unsigned long long *id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    looked_up = true;
    cudaDriverEntryPointQueryResult q1, q2;
    void *f1 = nullptr, *f2 = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
      get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
      get_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
  }
  if (!get_current || !get_id) return false;
  void *ctx = nullptr;
  if (get_current(&ctx) != 0 || !ctx) return false;
  return get_id(ctx, id) == 0;
}

// Device address of the scratch array in the current device's context.  Looked up with
// cudaGetSymbolAddress on the first call on each device and again whenever that device's
// context has changed since (a cudaDeviceReset in between); every call when the context id
// cannot be read.
cudaError_t scratch_for_current_device(StaticScratch **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  unsigned long long id = 0;
  bool have_id = current_context_id(&id);
  Cached &c = g_cache[dev];
  if (!(c.valid && have_id && c.ctx_id == id)) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_energy_scratch);  // creates the primary context if needed
    if (e != cudaSuccess) return e;
    if (!have_id) have_id = current_context_id(&id);
    c.ptr = static_cast<StaticScratch *>(p);
    c.ctx_id = id;
    c.valid = have_id;
  }
  *out = c.ptr;
  return cudaSuccess;
}

}  // namespace

extern "C" int rk4_chain_energy_static(rk4_chain *h, const void *state, const void *comp, double *out) {
  int model = 0, nchains = 0;
  bool fp32 = false;
  const ChainDesc *chains = nullptr;
  CoefD cf{};
  cudaStream_t st = nullptr;
  bool het = false;
  if (!out || !state) return RK4_EINVAL;
  if (handle_info(h, &model, &fp32, &nchains, &chains, &cf, &st, &het) != RK4_OK) return RK4_EINVAL;
  if (het && model == RK4_HARMONIC) return RK4_EUNSUPPORTED;  // as rk4_chain_energy
  if (fp32 != (comp != nullptr)) return RK4_EINVAL;
  if (nchains < 1 || nchains > kStaticMaxChains) return RK4_EINVAL;
  StaticScratch *s = nullptr;
  if (scratch_for_current_device(&s) != cudaSuccess) return RK4_ECUDA;
  if (cudaMemsetAsync(&s->hdr, 0, sizeof(WsHeader), st) != cudaSuccess) return RK4_ECUDA;
  if (nchains > 1 &&
      cudaMemcpyAsync(s->chains, chains, sizeof(ChainDesc) * (size_t)nchains, cudaMemcpyHostToDevice, st) !=
          cudaSuccess)
    return RK4_ECUDA;
  if (launch_energy(model, fp32, state, comp, nchains, chains[0], s->chains, cf, s->partials, s->result, &s->hdr,
                    st) != cudaSuccess)
    return RK4_ECUDA;
  int status = 0;
  if (cudaMemcpyAsync(out, s->result, sizeof(double) * (size_t)nchains, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return RK4_ECUDA;
  if (cudaMemcpyAsync(&status, &s->hdr.status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return RK4_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return RK4_ECUDA;
  return (status & ST_NONFINITE) ? RK4_ENONFINITE : RK4_OK;
}
