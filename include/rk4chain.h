/*
 * rk4chain.h -- C ABI of librk4chain.so: classical fixed-step RK4 integration of long
 * one-dimensional chains with nearest-neighbour coupling on an NVIDIA GB300 (sm_103a).
 *
 * The problem is the one stated in Mulansky, "Optimizing Large-Scale ODE Simulations"
 * (arXiv:1412.0544):
 *   - Sec. 2.1, Eq. (2): a homogeneous chain r_i' = f(r_i) + g(r_i, r_{i-1}, r_{i+1}) of N
 *     sites, each a D-dimensional state, stored site after site (Fig. 1: x1 y1 z1 x2 ...);
 *   - Sec. 2.2, Eqs. (3)-(5): an explicit Runge-Kutta step; here the classical RK4 tableau
 *     c = (0, 1/2, 1/2, 1), a21 = a32 = 1/2, a43 = 1, b = (1/6, 1/3, 1/3, 1/6), combined as
 *     y <- y + dt/6 (k1 + 2 k2 + 2 k3 + k4);
 *   - Sec. 3.1, Eqs. (6)-(7): the coupled Roessler chain (D = 3) with a = 0.2, b = 1, c = 9,
 *     f = (-y - z, x + a y, b + z (x - c)), g = kappa (x_{i-1} - 2 x_i + x_{i+1}, 0, 0);
 *     kappa = 1 is the paper's chain;
 *   - a harmonic chain from the same class (D = 2): q' = p,
 *     p' = -omega0^2 q + kappa (q_{i-1} - 2 q_i + q_{i+1});
 *   - Sec. 3.1: periodic ends r_0 = r_N, r_{N+1} = r_1; or fixed ends r_0 = r_{N+1} = 0
 *     (a Dirichlet reading; the paper only uses periodic ends).
 * Sec. 2.3's granularity with overlap (a cluster of G sites plus s = 4 sites of halo per side
 * per step) is realised as temporal blocking: one thread block advances a tile of G sites,
 * plus 4k halo sites per side, by k steps per launch, redundantly recomputing the halo.
 *
 * Conventions for every call:
 *   - Return value: RK4_OK (0) or a negative RK4_E* code; rk4_strerror() names it.  No C++
 *     exception crosses this boundary.  A call that fails with RK4_EINVAL enqueues nothing.
 *   - Device buffers are plain device pointers owned by the caller.  The library never
 *     allocates device memory; it owns only host-side plan state inside the handle.
 *   - Work is enqueued on the CUDA stream given at creation (NULL = the legacy default
 *     stream) and is asynchronous unless the call says it synchronises.
 *   - Threads: a handle holds host-side plan state (tables, a cached CUDA graph) and must not
 *     be used by two host threads at once; distinct handles are independent.  A workspace
 *     must not be shared by integrations that can overlap on the GPU.
 *   - State layout: [N][D] site-major ("AoS", Fig. 1), contiguous, FP64 (double) for
 *     RK4_FP64 or FP32 (float) for RK4_FP32_KAHAN.  For a batch the chains lie back to
 *     back in the order given at creation.
 *   - comp: for RK4_FP32_KAHAN, the Kahan compensation of every state component, same
 *     shape and type as the state, zero before the first step and preserved by the caller
 *     between calls (it is part of the integrator's state).  NULL for RK4_FP64.
 *   - ws / ws_bytes: a device workspace of at least rk4_chain_workspace_bytes() bytes,
 *     256-byte aligned; contents need not be preserved between calls.  It holds the
 *     ping-pong copy of the state, reduction partials, the device status word and, for a
 *     batch, its chain and tile tables (8 bytes per tile of at least 64 interior sites).
 *   - Device-side errors (a NaN or infinity in a state that an integration stores or a
 *     reduction reads, a barrier wait that ran out of time, in a debug build an index out of
 *     range) are latched in the status word inside ws and reported by rk4_chain_status().
 *     Every integrate and energy call clears the status word when it starts, so the status
 *     describes the most recent such call on that workspace.
 *   - Debug build: librk4chain_debug.so (build.py --debug-bounds) checks every global memory
 *     range a kernel reads or writes against the buffer extents; an out-of-range access is
 *     skipped and latches RK4_EBOUNDS.  Same ABI and results; slower.
 */
#ifndef RK4CHAIN_H
#define RK4CHAIN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RK4_OK 0
#define RK4_EINVAL (-1)        /* bad argument (NULL, N < 1, dt not finite and > 0, ...) */
#define RK4_ENOMEM_WS (-2)     /* ws_bytes smaller than rk4_chain_workspace_bytes() */
#define RK4_ECUDA (-3)         /* a CUDA runtime call failed */
#define RK4_ENONFINITE (-4)    /* a NaN or infinity was found in the state */
#define RK4_ETIMEOUT (-5)      /* a bounded device-side wait gave up */
#define RK4_EUNSUPPORTED (-6)  /* valid request the library does not support */
#define RK4_EBOUNDS (-7)       /* debug build only: an index check caught an out-of-range access
                                  (the access was skipped); see the build notes below */

enum rk4_model { RK4_ROESSLER = 0, RK4_HARMONIC = 1 };
enum rk4_precision { RK4_FP64 = 0, RK4_FP32_KAHAN = 1 };
enum rk4_bc { RK4_PERIODIC = 0, RK4_FIXED = 1 };

/* Which GPU scheme advances the state.
 * RK4_KERNEL_STAGED: the paper's "standard implementation" (Sec. 2.2): one launch per RK
 *   stage, each a full sweep over the chain (4 launches per step).
 * RK4_KERNEL_BLOCKED: temporal blocking (Sec. 2.3 on the GPU): tiles of G sites plus a halo
 *   of 4k sites per side advance k steps per launch; k = 1 is the fused single-step kernel.
 * RK4_KERNEL_PERSISTENT: (batches) one persistent cooperative launch walks the tile list for
 *   every block of k steps, separated by a bounded-wait grid barrier.
 * Every scheme performs the same floating-point operations per site, so all give
 * bit-identical results. */
enum rk4_kernel { RK4_KERNEL_AUTO = 0, RK4_KERNEL_STAGED = 1, RK4_KERNEL_BLOCKED = 2, RK4_KERNEL_PERSISTENT = 3 };

/* Model parameters.  Defaults (rk4_params_default): a = 0.2, b = 1, c = 9 (Sec. 3.1),
 * kappa = 1 (Eq. (7) has no coefficient), omega0 = 1. */
typedef struct {
  double a, b, c;  /* Roessler f, Eq. (6) */
  double kappa;    /* coupling strength multiplying g, Eq. (7) */
  double omega0;   /* harmonic chain on-site frequency */
} rk4_params;

/* Tiling of the blocked kernels: a tile is block * v sites, of which G = block * v - 2 H are
 * written back, H = 4k (classical RK4) or s' * range * k (generic scheme) being the halo on each
 * side; s' counts the stages the step's result needs (those with a nonzero weight and the
 * stages they use), e.g. 6 of Dormand-Prince 5's 7. */
typedef struct {
  int block;  /* threads per block: 64 .. 1024, a multiple of 32 */
  int v;      /* consecutive sites per thread: 1, 2, 4 or 8 (generic kernels: 2 or 4) */
  int k;      /* RK4 steps per launch: 1 .. 16 */
  int G;      /* output: interior sites per tile */
} rk4_tiling;

typedef struct rk4_chain rk4_chain; /* opaque host-side handle */

/* Fills *p with the defaults listed above. */
void rk4_params_default(rk4_params *p);

/* Creates a handle for one chain of n >= 1 sites.  model: enum rk4_model; precision: enum
 * rk4_precision; bc: enum rk4_bc; dt > 0 and finite; p may be NULL for the defaults;
 * cuda_stream is a cudaStream_t (NULL = legacy default stream).  On success *out owns the
 * handle (free it with rk4_chain_destroy).  Errors: RK4_EINVAL. */
int rk4_chain_create(rk4_chain **out, int model, int precision, int64_t n, double dt, int bc,
                     const rk4_params *p, void *cuda_stream);

/* Creates a handle for nchains independent chains integrated together (host arrays of
 * nchains entries, copied): lengths[c] >= 1, kappa[c] replaces p->kappa for chain c,
 * bc[c] is its boundary.  The state is the chains' [N_c][D] blocks back to back.
 * Errors: RK4_EINVAL. */
int rk4_batch_create(rk4_chain **out, int model, int precision, int nchains, const int64_t *lengths,
                     const double *kappa, const int8_t *bc, double dt, const rk4_params *p,
                     void *cuda_stream);

/* Bytes of workspace the handle needs for its current kernel choice and tiling. */
int rk4_chain_workspace_bytes(const rk4_chain *h, size_t *bytes);

/* Total sites (sum over chains) and per-site dimension D of the handle's state. */
int rk4_chain_shape(const rk4_chain *h, int64_t *total_sites, int *dim);

/* Chooses the scheme (enum rk4_kernel).  AUTO runs the scheme rk4_chain_autotune measured
 * fastest; before any autotuning, BLOCKED for one chain (and for the generic and heterogeneous
 * schemes) and PERSISTENT for a batch.  Setting a scheme forgets the autotuner's choice.
 * Errors: RK4_EINVAL. */
int rk4_chain_set_kernel(rk4_chain *h, int kernel);

/* The scheme the handle will run (AUTO resolved).  Errors: RK4_EINVAL. */
int rk4_chain_get_kernel(const rk4_chain *h, int *kernel);

/* Sets the tiling (block, v, k; G is computed).  block = 0 restores the automatic choice.
 * The largest block depends on the kernel the handle runs (its register budget): 1024
 * threads for v = 1, 512 for v = 2 and 4, 256 for v = 8, the generic scheme and the
 * heterogeneous FP32 Roessler chain with v = 4.  Errors: RK4_EINVAL when block, v or k is out
 * of range for the kernel or G < 8k (for the generic scheme: G < its halo per side). */
int rk4_chain_set_tiling(rk4_chain *h, int block, int v, int k);
int rk4_chain_get_tiling(const rk4_chain *h, rk4_tiling *out);

/* Replaces the classical RK4 tableau with any explicit Runge-Kutta tableau of 1 <= s <= 7
 * stages (the paper notes the technique applies to any explicit RK method, Sec. 2): A is s x s
 * row-major and must be strictly lower triangular, b holds the s weights (Eqs. (4)-(5)); both
 * are copied.  s = 0 restores the classical RK4 kernels.  The generic kernels keep every stage
 * slope per site and need a halo of s' * range sites per side per step (s' <= s: the stages
 * the result needs; a stage with weight 0 that no such stage uses is not); tilings then use v = 2
 * or 4 sites per thread.  The persistent kernel does not support them (RK4_EUNSUPPORTED).
 * Resets the tiling to its default.  Errors: RK4_EINVAL. */
int rk4_chain_set_tableau(rk4_chain *h, int s, const double *A, const double *b);

/* Second-neighbour coupling strength kappa2: the coupling becomes
 * kappa (x_{i-1} - 2 x_i + x_{i+1}) + kappa2 (x_{i-2} - 2 x_i + x_{i+2}) (the longer coupling
 * range of Sec. 5, which needs twice the overlap).  kappa2 != 0 selects the generic kernels
 * (with the current tableau, classical RK4 by default); the harmonic energy then includes the
 * second-neighbour bonds.  0 restores nearest-neighbour coupling.  Resets the tiling to its
 * default.  Errors: RK4_EINVAL. */
int rk4_chain_set_coupling2(rk4_chain *h, double kappa2);

/* Heterogeneous chain (Eq. (1): site-dependent f_i and g_i).  params is a caller-owned device
 * array of total_sites x P values in the state's precision, 16-byte aligned, kept valid and
 * unchanged while the handle integrates: RK4_ROESSLER P = 4 (a_i, b_i, c_i, kappa_i),
 * RK4_HARMONIC P = 2 (omega_i^2, kappa_i); the coupling of site i is
 * kappa_i (x_{i-1} - 2 x_i + x_{i+1}).  The per-site values replace the handle's (and a
 * batch's per-chain kappa).  NULL returns to the homogeneous chain.  Supported by the staged
 * and blocked kernels with the classical tableau (v = 2 or 4 sites per thread); the
 * persistent and generic kernels return RK4_EUNSUPPORTED, and so does the energy of a
 * heterogeneous harmonic chain.  Resets the tiling.  Errors: RK4_EINVAL (misaligned). */
int rk4_chain_set_site_params(rk4_chain *h, const void *params);

/* Times the candidate tilings on the caller's buffers and keeps the fastest (the paper
 * picks G by a performance study, Sec. 3.2.1).  On RK4_KERNEL_AUTO it also chooses the scheme:
 * for a batch the persistent against the blocked scheme, and for any handle the staged scheme
 * (the paper's standard implementation, Sec. 2.2) when ws_bytes is at least the workspace that
 * scheme needs (rk4_chain_workspace_bytes after rk4_chain_set_kernel(h, RK4_KERNEL_STAGED)):
 * a caller that can afford the larger workspace lets the autotuner pick the unblocked scheme
 * where it measures faster.  After a call that chose STAGED, rk4_chain_workspace_bytes reports
 * its size, and rk4_chain_set_tiling returns the handle to the tiled schemes.  The call
 * integrates `state` (and comp) forward by an unspecified number of steps: pass scratch copies.
 * Synchronises the stream.  *best (may be NULL) receives the chosen tiling (the best tiled one
 * when STAGED wins).  Errors: RK4_EINVAL, RK4_ENOMEM_WS, RK4_ECUDA. */
int rk4_chain_autotune(rk4_chain *h, void *state, void *comp, void *ws, size_t ws_bytes,
                       int probe_steps, rk4_tiling *best);

/* Advances the state one RK4 step (Eqs. (3)-(5)); equivalent to integrate with nsteps = 1. */
int rk4_chain_step(rk4_chain *h, void *state, void *comp, void *ws, size_t ws_bytes, double *t);

/* Advances the device state nsteps >= 0 RK4 steps in place (stream-ordered).  If t is not
 * NULL it receives t0 + n dt, n being the steps taken through this handle so far (no
 * repeated addition).  Launch sequences of the same shape are replayed from a cached CUDA
 * graph.  The blocked scheme makes launches of k steps (the tiling's k) into a ping-pong copy
 * in ws and must end in `state` after an even number of launches: an odd count is evened by
 * splitting one launch in two (nsteps = k runs as two launches of k / 2), so calls of an
 * even multiple of k steps run at the tiling's full k.  Errors: RK4_EINVAL, RK4_ENOMEM_WS,
 * RK4_ECUDA. */
int rk4_chain_integrate(rk4_chain *h, void *state, void *comp, void *ws, size_t ws_bytes,
                        int64_t nsteps, double *t);

/* The same starting from and returning to HOST buffers: copies host_state (and host_comp)
 * into the device buffers dev_state (dev_comp), integrates, copies the result back and
 * synchronises the stream.  The host buffers hold the whole state ([N][D] values of the
 * handle's precision).  Page-locked (pinned) host memory that the device can address, 16-byte
 * aligned, is read and written by a copy kernel through its device address; any other host
 * memory goes through cudaMemcpyAsync. */
int rk4_chain_integrate_host(rk4_chain *h, void *host_state, void *host_comp, void *dev_state,
                             void *dev_comp, void *ws, size_t ws_bytes, int64_t nsteps, double *t);

/* FP64 reductions of the state (with the compensation subtracted for RK4_FP32_KAHAN):
 * RK4_HARMONIC: the energy sum_i (p_i^2/2 + omega0^2 q_i^2/2) + kappa/2 sum_bonds (dq)^2,
 * including the bonds to the zero ghosts for fixed ends; RK4_ROESSLER: (1/2) sum_i |r_i|^2,
 * a monitored norm (the Roessler chain is dissipative, not Hamiltonian).  out (host)
 * receives one value for a single chain, nchains values for a batch.  Synchronises the
 * stream.  Returns RK4_ENONFINITE if a NaN or infinity was seen. */
int rk4_chain_energy(rk4_chain *h, const void *state, const void *comp, void *ws, size_t ws_bytes,
                     double *out);

/* The same reduction without a workspace, for callers that cannot allocate device memory --
 * code that runs where cudaMalloc is not allowed or not reachable (a host callback or hook, a
 * plug-in whose host application owns all device allocations), so it cannot provide ws.  The
 * paper has no counterpart: this is a library convenience.  Scratch space (partial sums, one
 * result per chain, the batch chain table, a status word) is a fixed array compiled into the
 * library, about 330 KB on every GPU that loads it, held until the process exits; batches
 * of more than 8192 chains are rejected with RK4_EINVAL.  The call allocates nothing (no
 * cudaMalloc, cudaMallocHost or cudaFree).  The first call on each device looks up the
 * array's device address (and a call after that device's context was replaced, e.g. by
 * cudaDeviceReset, looks it up again), so make that first call before any stream capture.  All calls
 * share the array: calls whose work overlaps on the GPU race and must be serialised by the
 * caller.  out (host) receives one value per chain.  Synchronises the stream.  Returns
 * RK4_ENONFINITE if a NaN or infinity was seen, RK4_EINVAL for bad arguments. */
int rk4_chain_energy_static(rk4_chain *h, const void *state, const void *comp, double *out);

/* Synchronises the stream, reads and clears the device status word in ws, and returns the
 * latched error (RK4_ETIMEOUT, else RK4_EBOUNDS, else RK4_ENONFINITE) or RK4_OK.  An
 * integration that stored a NaN or infinity (an unstable dt, a blow-up) reports
 * RK4_ENONFINITE here. */
int rk4_chain_status(rk4_chain *h, void *ws);

/* Options (enum rk4_option): RK4_OPT_GRAPHS (1 = replay launch sequences from a cached CUDA
 * graph, the default; 0 = launch directly), RK4_OPT_TIMEOUT_NS (bound on any device-side
 * barrier wait of the persistent kernel; by default 2e9 ns or 20 ns per site-step of one time
 * block, whichever is larger).  Errors: RK4_EINVAL. */
enum rk4_option { RK4_OPT_GRAPHS = 0, RK4_OPT_TIMEOUT_NS = 1 };
int rk4_chain_set_option(rk4_chain *h, int option, int64_t value);

/* Test hook for failure detection: runs the persistent kernel for one time block and then
 * makes its grid barrier wait for one block that never arrives, so that the bounded wait
 * runs out after timeout_ns and latches RK4_ETIMEOUT in the status word (read it with
 * rk4_chain_status).  The state is advanced by an unspecified amount: pass scratch buffers.
 * Needs a batch handle or the persistent kernel.  No GPU fault is involved. */
int rk4_debug_barrier_timeout(rk4_chain *h, void *state, void *comp, void *ws, size_t ws_bytes,
                              int64_t timeout_ns);

/* The handle's clock: time origin t0 and steps taken n (t = t0 + n dt).  set_clock restores
 * both, e.g. when resuming from a checkpoint, so that t stays t0 + n dt with one rounding.
 * Errors: RK4_EINVAL. */
int rk4_chain_get_clock(const rk4_chain *h, double *t0, int64_t *nstep);
int rk4_chain_set_clock(rk4_chain *h, double t0, int64_t nstep);

/* Sets the time origin t0 and resets the step counter. */
int rk4_chain_set_time(rk4_chain *h, double t0);

/* Frees the handle (and its cached graphs).  NULL is accepted. */
int rk4_chain_destroy(rk4_chain *h);

/* Static description of an error code. */
const char *rk4_strerror(int code);

/* Counter-based initial state (SplitMix64, Steele-Lea-Flood 2014): dst[j] for
 * j = 0 .. count-1 is 2 u - 1 with u = (splitmix64(seed XOR (start + j)) >> 11) * 2^-53, as a
 * double (exact) or rounded to the nearest float (precision RK4_FP32_KAHAN).  The paper
 * starts from random initial conditions (Sec. 3.2).  Asynchronous on cuda_stream. */
int rk4_fill_uniform(void *dst, int64_t count, uint64_t seed, uint64_t start, int precision,
                     void *cuda_stream);

/* ---- Sub-domain decomposition of one chain --------------------------------------------------
 * One chain of n sites split into nparts contiguous parts, each stored with ghost zones of
 * `ghost` sites per side and integrated as an independent fixed-end chain between ghost
 * exchanges: Sec. 2.3's granularity with overlap (a cluster plus s sites of overlap per side
 * per step, recomputed redundantly) applied to memory partitions -- the form a chain takes
 * when it is spread over several memories, with one neighbour exchange every few steps.
 * A scheme whose result needs s stages, with coupling range r, moves information s r sites per
 * step, so the parts run floor(ghost / (s r)) steps between exchanges (ghost / 4 for classical RK4 with
 * nearest neighbours), and every interior site performs the same operations as in the
 * undivided chain: the gathered result is bit-identical to rk4_chain_integrate on the whole
 * chain with the same model, precision, parameters and tableau.
 *
 * Domain state layout: the parts' blocks back to back, part p occupying rows
 * [row_p, row_p + ghost_left_p + sites_p + ghost_right_p) of a [rows][D] array in the chain's
 * precision: its left ghost zone, its sites first_site_p .. first_site_p + sites_p - 1, its
 * right ghost zone.  Every part has both ghost zones except the first (no left) and the last
 * (no right) part of a fixed-end chain.  comp (RK4_FP32_KAHAN) has the same layout.  Buffers
 * are caller-owned device memory, 16-byte aligned; ws 256-byte aligned.  Calls are
 * stream-ordered on the domain's stream unless they say they synchronise.  Inside
 * rk4_domain_integrate and rk4_domain_energy an exchange is one gather-kernel launch over a
 * table of the ghost zones kept in ws; rk4_domain_scatter and rk4_domain_exchange, which have
 * no workspace, issue one device-to-device cudaMemcpyAsync per ghost zone and array. */
typedef struct rk4_domain rk4_domain; /* opaque host-side handle */

/* Creates a domain over one chain (model, precision, n, dt, bc, p, cuda_stream as for
 * rk4_chain_create).  nparts >= 1 parts; part_lengths (host, nparts entries summing to n,
 * copied) gives each part's sites, or NULL for an even split (the first n % nparts parts one
 * site longer).  ghost >= 1 sites per ghost zone (0 allowed only for one part of a fixed-end
 * chain, which has none), and every part at least `ghost` sites long when ghost zones exist.
 * The parts are integrated by one batch handle of fixed-end chains (RK4_KERNEL_BLOCKED unless
 * changed through rk4_domain_chain).  Errors: RK4_EINVAL. */
int rk4_domain_create(rk4_domain **out, int model, int precision, int64_t n, double dt, int bc,
                      const rk4_params *p, int nparts, const int64_t *part_lengths, int64_t ghost,
                      void *cuda_stream);

/* Where part `part` lives: its first chain site and site count, its first row in the domain
 * state, and its ghost zone widths (any pointer may be NULL).  Errors: RK4_EINVAL. */
int rk4_domain_part(const rk4_domain *d, int part, int64_t *first_site, int64_t *sites, int64_t *row,
                    int64_t *ghost_left, int64_t *ghost_right);

/* Rows of the domain state (sites plus ghost zones of all parts) and D. */
int rk4_domain_shape(const rk4_domain *d, int64_t *rows, int *dim);

/* The batch handle that integrates the parts, owned by the domain (do not destroy it, and do
 * not integrate it directly: that skips the exchanges).  Use it to choose the kernel and the
 * tiling, a tableau or second-neighbour coupling, and options; a tableau or coupling range
 * whose reach s r exceeds the ghost width makes rk4_domain_integrate return
 * RK4_EUNSUPPORTED.  Errors: RK4_EINVAL. */
int rk4_domain_chain(rk4_domain *d, rk4_chain **parts);

/* Bytes of workspace rk4_domain_integrate and rk4_domain_energy need (the batch handle's
 * workspace for its current kernel and tiling, plus reduction scratch). */
int rk4_domain_workspace_bytes(const rk4_domain *d, size_t *bytes);

/* Copies a whole-chain state [n][D] (and comp) into the domain layout, ghost zones included.
 * Errors: RK4_EINVAL, RK4_ECUDA. */
int rk4_domain_scatter(rk4_domain *d, const void *chain_state, const void *chain_comp, void *state,
                       void *comp);

/* Copies the parts' sites (not the ghosts) back into a whole-chain state [n][D] (and comp).
 * Errors: RK4_EINVAL, RK4_ECUDA. */
int rk4_domain_gather(rk4_domain *d, const void *state, const void *comp, void *chain_state,
                      void *chain_comp);

/* Refreshes every ghost zone from the neighbouring part's sites (cyclically for periodic
 * ends).  Errors: RK4_EINVAL, RK4_ECUDA. */
int rk4_domain_exchange(rk4_domain *d, void *state, void *comp);

/* Advances the domain nsteps >= 0 steps: exchange the ghosts, integrate every part
 * floor(ghost / (s r)) steps (fewer at the end), repeat.  Whole periods run in chunks of 8 from
 * one CUDA graph, captured on first use and replayed while the buffers and the parts'
 * configuration stay the same (calls of any length share it).  If t is not NULL it receives n dt, n the steps taken
 * through this domain so far.
 * Errors: RK4_EINVAL, RK4_ENOMEM_WS, RK4_ECUDA, RK4_EUNSUPPORTED (heterogeneous parameters
 * set on the batch handle, or a scheme whose reach per step exceeds the ghost width). */
int rk4_domain_integrate(rk4_domain *d, void *state, void *comp, void *ws, size_t ws_bytes,
                         int64_t nsteps, double *t);

/* The whole chain's FP64 energy or half squared norm (as rk4_chain_energy), summed part by
 * part over the parts' sites after a ghost exchange, so that bonds across part boundaries are
 * counted once.  Synchronises the stream.  Returns RK4_ENONFINITE if a NaN or infinity was
 * seen; RK4_EUNSUPPORTED if the coupling range exceeds the ghost width. */
int rk4_domain_energy(rk4_domain *d, void *state, void *comp, void *ws, size_t ws_bytes, double *out);

/* rk4_chain_status of the parts' batch handle on ws (the most recent integration period). */
int rk4_domain_status(rk4_domain *d, void *ws);

/* Frees the domain and its batch handle.  NULL is accepted. */
int rk4_domain_destroy(rk4_domain *d);

#ifdef __cplusplus
}
#endif

#endif /* RK4CHAIN_H */
