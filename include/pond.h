/*
 * pond.h -- C ABI of the GB300 Particles-on-Demand (PonD) step library.
 *
 * Method: Dorschner, Bosch, Karlin, "Particles-on-Demand for Kinetic
 * Theory" (arXiv 1806.05089).  One time step on a periodic D2Q16 lattice
 * (tensor product of the four roots of He4, T_L = 1; the default) or the
 * paper's own D2Q9 lattice (App. A: speeds -1, 0, 1, weights 1/6, 2/3, 1/6,
 * T_L = 1/3):
 *   - departure points x - (sqrt(theta) c_i + u) dt        (Eqs. advection, vi)
 *   - gauge transform of neighbour populations by moment
 *     matching, f' = M_target^-1 M_source f                 (Eqs. moments, match,
 *                                                           transform)
 *   - bicubic Lagrange reconstruction at the departure point (Eq. interpolation,
 *                                                           App. C)
 *   - predictor-corrector fixed point on rho, u, T          (Eqs. conservation_*,
 *                                                           density..precollision,
 *                                                           App. E Eq. convergence)
 *   - BGK relaxation toward rho W in the co-moving gauge     (Eqs. equilibrium,
 *                                                           postcollision)
 *
 * Conventions shared by every entry point:
 *   - n1 speeds per dimension (4 on D2Q16, 3 on D2Q9), Q = n1^2
 *     populations; population index q = n1 k + l, k the x-speed index and
 *     l the y-speed index of the ascending speeds c_0 < ... < c_{n1-1};
 *   - fields are row-major [ny][nx] (x fastest); populations are
 *     structure-of-arrays [Q][ny][nx];
 *   - every array crossing this boundary is FP64 (double), whatever the
 *     internal precision; gauges are (u_x, u_y, T) with theta = T / T_L;
 *   - lattice units: dx = 1, dt from the config (default 1).
 *
 * Ownership: the caller owns every buffer it passes (host memory, or device
 * memory of the context's device when on_device != 0).  The library copies
 * into its own device state, allocated by pond_create and freed by
 * pond_destroy.  All device work is enqueued on the stream given to
 * pond_create (or pond_set_stream); calls that return data to host memory
 * synchronise that stream before returning.
 *
 * Errors: every call returns a pond_status; nothing throws across the
 * boundary and no kernel traps.  pond_last_error() gives a message for the
 * most recent failing call on a context.
 */
#ifndef POND_H
#define POND_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pond_ctx pond_ctx; /* opaque; owned by the library */

typedef enum pond_status {
    POND_OK = 0,
    POND_ERR_ARG = 1,           /* invalid argument (NULL, size, grid index) */
    POND_ERR_OOM = 2,           /* device allocation failed */
    POND_ERR_CUDA = 3,          /* a CUDA runtime call or launch failed */
    POND_ERR_NONPHYSICAL = 4,   /* rho <= 0, T <= 0 or NaN met at some node */
    POND_ERR_NOT_CONVERGED = 5, /* strict mode: a node hit max_iter */
    POND_ERR_TIMEOUT = 6,       /* a bounded device wait gave up */
    POND_ERR_STATE = 7          /* call out of order (e.g. step before set_state) */
} pond_status;

enum { POND_FP64 = 0, POND_FP32_MIXED = 1 };

/* Lattices (pond_config.lattice). */
enum { POND_D2Q16 = 0, POND_D2Q9 = 1 };

/* Step kernels (pond_config.kernel). */
enum { POND_KERNEL_DEFAULT = 0, POND_KERNEL_STAGED = 1, POND_KERNEL_DIRECT = 2 };

/* Run configuration.  Fill with pond_config_default() and override. */
typedef struct pond_config {
    int32_t precision;  /* POND_FP64: all arithmetic and storage FP64.
                           POND_FP32_MIXED: populations and bulk arithmetic
                           FP32; gauges stored and accumulated in FP64; the
                           gauge differences of the transform formed from the
                           FP64 gauges (tile-relative offsets), the
                           transform's polynomials and contractions in FP32;
                           convergence test in FP64. */
    int32_t thermal;    /* 1: energy equation in the predictor-corrector
                           (compressible); 0: isothermal, T kept fixed
                           (main text after Eq. postcollision). */
    double nu;          /* kinematic viscosity; beta = 1/(2 nu/(T_ref dt) + 1)
                           from nu = T (1/(2 beta) - 1/2) dt (Eq. postcollision) */
    double T_ref;       /* temperature in that relation (default 1) */
    double dt;          /* time step (default 1) */
    double eps_abs;     /* Eq. convergence tolerances (App. E); defaults   */
    double eps_rel;     /* 1e-12 / 1e-10 (FP64), 1e-6 / 1e-6 (FP32_MIXED)  */
    int32_t max_iter;   /* predictor-corrector pass limit (default 20) */
    int32_t fixed_iter; /* > 0: exactly this many passes, no early exit */
    int32_t ckpt_every; /* adjoint checkpoint interval (used by bindings) */
    int32_t strict;     /* 1: pond_step returns POND_ERR_NOT_CONVERGED when a
                           node hit max_iter without converging */
    int32_t seed_mode;  /* 0: previous gauge at the node (Eq. seed_gauge);
                           1: {0, T_L}; 2: {-u, T} (seed-independence study) */
    int32_t use_graph;  /* 1: pond_step replays a CUDA graph of two steps
                           (captured on first use, re-captured after
                           set_state / set_stream) */
    int32_t autotune;   /* 1 (tile kernels): the first pond_step times the
                           kernel's tile shapes (see tile_rows) on the
                           current state, without advancing it, and keeps
                           the fastest.  Results are cached per
                           process by grid-set signature and, when the
                           environment variable POND_AUTOTUNE_CACHE names a
                           file, in that JSON file across processes. */
    int32_t tile_rows;  /* tile kernels (the mixed form, and the FP64 form's
                           staged kernel): 0 = default tile (32 x 8 nodes;
                           32 x 4 for the FP64 form on D2Q9) or the
                           autotuner's choice; 4, 8 or 16 force a
                           32-wide tile of that many rows (16: mixed only),
                           -16 the direct mixed kernel's 32 x 16 tile with
                           two stacked nodes per thread (D2Q16 only); a
                           forced shape disables autotune. */
    int32_t lattice;    /* POND_D2Q16 (default) or POND_D2Q9.  Fixes Q and
                           T_L (so the meaning of theta = T / T_L and of the
                           seed {0, T_L}). */
    int32_t nodes_per_warp; /* FP64 form: target nodes per warp of the step
                           kernel, 1 (16 lanes per node, each lane half the
                           stencil rows), 2 (each lane all rows), on D2Q9
                           only 3 (10 lanes per node), or 32 (one node per
                           thread, looping over the populations); 0 = the
                           library default.  Other values are rejected
                           (POND_ERR_ARG).  They agree to rounding (the
                           stencil rows and the moments are summed in other
                           orders). */
    int32_t kernel;     /* POND_KERNEL_STAGED (and POND_KERNEL_DEFAULT): the
                           reference-gauge staged tile kernel, both forms.
                           Eq. transform composes, M_t^-1 M_s =
                           (M_t^-1 M_r)(M_r^-1 M_s), and the reconstruction
                           of Eq. interpolation is linear, so each CTA
                           stages the sources its tile's stencils reach
                           once per step, re-expressed in a reference
                           gauge r (the tile's centre node), and each pass
                           reconstructs in r and applies one map r -> target
                           per population: the same f_q up to rounding, with
                           a quarter (mixed) to a fifth (FP64) of the
                           per-pass arithmetic.  Tile
                           shapes 32 x 4 and 32 x 8 nodes (FP64), 32 x 4,
                           32 x 8, 32 x 16 (mixed).
                           POND_KERNEL_DIRECT: the per-(population, source)
                           kernels, G(s -> t) for every stencil node of
                           every population (FP64 mappings by
                           nodes_per_warp; mixed tiles by tile_rows,
                           including the paired -16 shape).
                           Other values: POND_ERR_ARG. */
} pond_config;

/* Counters accumulated over the steps of one pond_step call. */
typedef struct pond_stats {
    int64_t node_updates;  /* nodes x steps */
    int64_t passes;        /* predictor-corrector passes over all node updates */
    int32_t max_passes;    /* largest pass count at any node */
    int32_t tile_rows;     /* rows of the tile shape in use (32 columns) of
                              the tile kernels (the staged kernel in either
                              form, the direct mixed kernel); negative when
                              each thread owns two vertically adjacent nodes;
                              0 for the direct FP64 kernels */
    int64_t nonconverged;  /* node updates that hit max_iter unconverged */
    int64_t nonphysical;   /* node updates that met rho <= 0, T <= 0 or NaN */
    int64_t halo_fallback; /* stencils read from global memory instead of the
                              shared-memory window (tile kernels) */
    int64_t index_faults;  /* debug builds of the library (compiled with
                              POND_DEBUG): accesses of the staged kernel that
                              failed their index check and were skipped; 0
                              in release builds, which have no checks */
    int64_t busy_ns;       /* batched contexts on the staged kernel (one
                              persistent launch per step): CTA busy time
                              summed over the launches' CTAs, in ns */
    int64_t slot_ns;       /* the same launches' CTA slots: resident CTAs x
                              launch span, in ns.  1 - busy_ns / slot_ns is
                              the share of those slots left idle by the start
                              skew and the tail; both 0 for other contexts */
} pond_stats;

/* Defaults for a precision (POND_FP64 or POND_FP32_MIXED). */
void pond_config_default(pond_config* cfg, int32_t precision);

/* Create a context for n_grids independent periodic grids of sizes
 * nx[g] x ny[g] (n_grids == 1: single grid; > 1: batched ensemble advanced
 * together by one launch per step).  cuda_stream is a cudaStream_t (NULL =
 * legacy default stream).  Allocates the device state; the only later
 * allocations are a staging area for host buffers (20 FP64 values per node,
 * made by the first call that passes host pointers and grown for a larger
 * grid) and the adjoint's scratch (pond_adjoint_step's first call).
 * Ensembles run on the staged kernel in either precision, and on the
 * direct mixed kernel; the direct FP64 kernels step one grid.
 * Errors: POND_ERR_ARG (NULL pointers, n_grids < 1, a side < 1, a config
 * field out of its range or a combination this header rules out, n_grids > 1
 * with the direct FP64 kernels), POND_ERR_OOM, POND_ERR_CUDA. */
pond_status pond_create(const pond_config* cfg, int32_t n_grids, const int32_t* nx,
                        const int32_t* ny, void* cuda_stream, pond_ctx** out);

/* Replace the stream all later work is enqueued on.  Work already queued on
 * the old stream is waited for first (the host blocks until it ends), and the
 * step graphs (use_graph) are captured again on next use.
 * Errors: POND_ERR_ARG (NULL ctx), POND_ERR_CUDA. */
pond_status pond_set_stream(pond_ctx* ctx, void* cuda_stream);

/* Set the state of grid `grid` from macroscopic fields, each [ny][nx] FP64:
 * density rho, velocity (ux, uy), temperature T.  If f is NULL the
 * populations are the equilibrium f = rho W in each node's own gauge
 * (Eq. equilibrium; rho is then required).  If f is given ([Q][ny][nx]),
 * it is taken as the populations in the gauge (ux, uy, T) and rho is
 * ignored (may be NULL).  on_device: pointers are device (1) or host (0).
 * Errors: POND_ERR_ARG, POND_ERR_NONPHYSICAL (T <= 0 or a non-finite
 * gauge at some node, host or device input, checked on the device; the grid
 * then counts as never set until a valid call), POND_ERR_OOM (the host
 * staging area, host input only), POND_ERR_CUDA. */
pond_status pond_set_state(pond_ctx* ctx, int32_t grid, const void* rho, const void* ux,
                           const void* uy, const void* T, const void* f, int32_t on_device);

/* Advance every grid by nsteps PonD time steps.  stats may be NULL; when
 * given, the stream is synchronised and the counters filled.
 * Errors: POND_ERR_STATE (a grid never set), POND_ERR_ARG (nsteps < 0),
 * POND_ERR_CUDA, and -- only when stats is given -- POND_ERR_NONPHYSICAL /
 * POND_ERR_NOT_CONVERGED (strict) from the counters. */
pond_status pond_step(pond_ctx* ctx, int32_t nsteps, pond_stats* stats);

/* Macroscopic fields of grid `grid`, each [ny][nx] FP64 (any may be NULL):
 * rho = sum_q f_q (Eq. conservation_rho) and the stored gauge (u, T), which
 * is the co-moving frame of the populations (remark after Eq. precollision).
 * Errors: POND_ERR_ARG (NULL ctx, grid index), POND_ERR_STATE (grid never
 * set), POND_ERR_OOM (the host staging area, host output only),
 * POND_ERR_CUDA. */
pond_status pond_moments(pond_ctx* ctx, int32_t grid, void* rho, void* ux, void* uy,
                         void* T, int32_t on_device);

/* Raw state of grid `grid`: populations f [Q][ny][nx] in the stored gauge
 * and the gauge (ux, uy, T) [ny][nx]; any pointer may be NULL.
 * Errors: as pond_moments. */
pond_status pond_get_state(pond_ctx* ctx, int32_t grid, void* f, void* ux, void* uy,
                           void* T, int32_t on_device);

/* Predictor-corrector pass counts of the last step at every node of grid
 * `grid`, int32 [ny][nx] (the map of App. E's iteration figure; zeros before
 * the first step).
 * Errors: POND_ERR_ARG (NULL ctx or iters, grid index), POND_ERR_CUDA. */
pond_status pond_iterations(pond_ctx* ctx, int32_t grid, void* iters, int32_t on_device);

/* Vector-Jacobian product of one step (single-grid contexts).  The context's
 * current state is the step's INPUT state s; given the cotangents of the
 * step's output, f_bar_in [Q][ny][nx] and gauge_bar_in [3][ny][nx]
 * (ux, uy, T), writes the cotangents of s to f_bar_out and gauge_bar_out
 * (same layouts) and adds d(loss)/d(nu) to *nu_bar_accum (a host double;
 * the call then waits for the step's kernels), or, when nu_bar_accum is NULL,
 * to an accumulator the context keeps on the device (the call then returns
 * without waiting; read it with pond_adjoint_nu_bar).  The fixed point
 * is differentiated implicitly (the limit gauge of Eqs. density..T is a
 * function of the input state only; the seed gets no gradient).  All array
 * pointers are device pointers.  The state is left unchanged.  FP64 and
 * mixed contexts (the latter with FP32 pair arithmetic and an FP32 per-node
 * 3 x 3 solve; the nu cotangent accumulates in FP64); single-grid, thermal
 * mode, either lattice (POND_ERR_ARG otherwise).
 * Errors: POND_ERR_ARG, POND_ERR_STATE, POND_ERR_OOM, POND_ERR_CUDA. */
pond_status pond_adjoint_step(pond_ctx* ctx, const void* f_bar_in, const void* gauge_bar_in,
                              void* f_bar_out, void* gauge_bar_out, double* nu_bar_accum);

/* pond_adjoint_step with the step's output gauge given: ux_out, uy_out,
 * T_out (device, [ny][nx]) are the gauge that pond_step stores when it
 * advances the context's current state by one step (for instance read back
 * with pond_get_state after the forward step, as a checkpointed rollout has
 * it).  The adjoint then does not recompute the forward step.  The result
 * equals pond_adjoint_step's when the gauge is that step's output; another
 * gauge gives the VJP at another linearisation point, which is not detected.
 * Errors: as pond_adjoint_step, and POND_ERR_ARG for a NULL output gauge. */
pond_status pond_adjoint_step_given(pond_ctx* ctx, const void* ux_out, const void* uy_out,
                                    const void* T_out, const void* f_bar_in,
                                    const void* gauge_bar_in, void* f_bar_out,
                                    void* gauge_bar_out, double* nu_bar_accum);

/* The nu cotangent accumulated on the device by the adjoint calls made
 * with nu_bar_accum == NULL since the last read: written to *nu_bar (host),
 * and the accumulator cleared.  Waits for the context's stream.  0 before
 * the first adjoint call.
 * Errors: POND_ERR_ARG (NULL pointer), POND_ERR_CUDA. */
pond_status pond_adjoint_nu_bar(pond_ctx* ctx, double* nu_bar);

/* VJP of the equilibrium initialisation of pond_set_state (f = rho W,
 * Eq. equilibrium): rho_bar[x] = sum_q W_q f_bar[q][x].  Single-grid
 * contexts; device pointers, f_bar [Q][ny][nx], rho_bar [ny][nx].  (The
 * gauge cotangents pass through unchanged: set_state stores u and T as given.)
 * Errors: POND_ERR_ARG, POND_ERR_CUDA. */
pond_status pond_adjoint_init(pond_ctx* ctx, const void* f_bar, void* rho_bar);

/* Domain decomposition (spatial split of one grid over several contexts,
 * typically one per GPU).  Eq. advection reads only the state at t - dt, so
 * a sub-domain whose grid carries a halo at least as wide as the largest
 * displacement plus the stencil reach (max(|u| + c_max sqrt(theta)) dt + 2
 * nodes) can advance its interior for one step independently, after the
 * halo has been refreshed from its neighbours.  These calls give a context
 * that interior, move halo strips in and out of its state, and bound the
 * displacement.
 *
 * pond_set_interior: from now on pond_step updates only the rectangle
 * [x0, x0 + w) x [y0, y0 + h) of grid `grid` (the nodes outside it are read
 * as sources but not written; after a step they hold stale values until
 * the caller refreshes them).  The staged kernel only (POND_ERR_ARG for the
 * direct kernels or a rectangle outside the grid).  pond_stats.node_updates
 * then counts interior nodes. */
pond_status pond_set_interior(pond_ctx* ctx, int32_t grid, int32_t x0, int32_t y0, int32_t w,
                              int32_t h);

/* Copy the rectangle [x0, x0 + w) x [y0, y0 + h) of grid `grid`'s current
 * state to (pack) or from (unpack) a device buffer of (Q + 3) * w * h FP64
 * values: the Q population planes [Q][h][w], then u_x, u_y and
 * sqrt(T / T_L), each [h][w].  This is the stored representation
 * (populations widened exactly from FP32 in the mixed form, the gauge as
 * stored), meant for another context of the same configuration: a state
 * split over sub-domains and reassembled this way is bit-identical.  Work is
 * enqueued on the context's stream; the call does not synchronise.
 * Errors: POND_ERR_ARG (NULL buffer, rectangle outside the grid), POND_ERR_CUDA. */
pond_status pond_pack_rect(pond_ctx* ctx, int32_t grid, int32_t x0, int32_t y0, int32_t w,
                           int32_t h, void* buf);
pond_status pond_unpack_rect(pond_ctx* ctx, int32_t grid, int32_t x0, int32_t y0, int32_t w,
                             int32_t h, const void* buf);

/* Bound of the displacement of any particle of grid `grid` in one step from
 * the current state: max over nodes of (|u_x| or |u_y|) + c_max sqrt(theta),
 * times dt, in nodes (computed in FP32 on the device; synchronises the
 * stream).  A decomposition's halo must exceed this plus the stencil reach.
 * Errors: POND_ERR_ARG, POND_ERR_STATE (grid never set), POND_ERR_CUDA. */
pond_status pond_max_displacement(pond_ctx* ctx, int32_t grid, double* out);

/* Largest grid (nx * ny) pond_step_fp64_noalloc accepts. */
#define POND_NOALLOC_MAX_NODES 262144

/* One FP64 step of a single periodic grid that allocates nothing and needs
 * no context.  The paper has no counterpart: this exists for callers that
 * must not allocate device memory (code running inside a host callback, a
 * custom allocator or memory pool, a framework that has reserved all device
 * memory, a real-time loop that may not enter the allocator).
 *
 * All array arguments are device pointers of the current device, FP64, in
 * the layouts above: f_in/f_out [Q][ny][nx] (Q of cfg->lattice),
 * ux/uy/T [ny][nx]; iters
 * (int32 [ny][nx]) and stats may be NULL.  Output arrays must not overlap
 * the inputs.  cfg must have precision POND_FP64; the other fields mean what
 * they mean for pond_create.  Work is enqueued on cuda_stream; the call
 * returns without synchronising unless stats is given.
 *
 * The only extra device memory -- sqrt(T/T_L) of the input and output
 * gauges and the step counters -- is a fixed array inside the library, held
 * by every GPU that loads the library until the process exits
 * (2 x 8 x POND_NOALLOC_MAX_NODES + 256 bytes).  Every call on a device
 * shares that array and the counters are cleared at the start of each call,
 * so calls whose work can overlap on the GPU (different streams, or
 * different host threads) race and must be serialised by the caller.  Every
 * call looks up the array's device address (a lookup, not an allocation).
 * The first call in each CUDA context also uploads the lattice constants (a
 * synchronous copy), so make it before any stream capture; after a device
 * reset the next call sees the new context and uploads them again.  With
 * lazy module loading (the CUDA default) the driver loads this library's
 * device code, and so places the array, at that first call: a caller that
 * later reserves all free device memory should make one call first (a 1 x 1
 * grid will do).  No cudaMalloc, cudaFree or allocating library call is
 * made.
 *
 * Errors: POND_ERR_ARG (NULL pointer, bad config, nx * ny above
 * POND_NOALLOC_MAX_NODES), POND_ERR_CUDA, and with stats given
 * POND_ERR_NONPHYSICAL / POND_ERR_NOT_CONVERGED (strict) as pond_step. */
pond_status pond_step_fp64_noalloc(const pond_config* cfg, int32_t nx, int32_t ny,
                                   const double* f_in, const double* ux_in, const double* uy_in,
                                   const double* T_in, double* f_out, double* ux_out,
                                   double* uy_out, double* T_out, int32_t* iters,
                                   pond_stats* stats, void* cuda_stream);

/* Arithmetic pipes pond_measure_peak can time. */
enum { POND_PIPE_FP64 = 0, POND_PIPE_FP32 = 1, POND_PIPE_FP32X2 = 2 };

/* Measurement utility; the paper has no counterpart.  The PonD step is
 * bound by plain FMA arithmetic (FP64 pipe for the FP64 form, FP32 pipe for
 * the mixed form), so its roofline denominators are FMA rates.  This times
 * one launch (after a warm-up launch) of a kernel in which every thread of
 * a grid of (SM count x resident CTAs per SM) CTAs of 256 threads runs eight
 * independent FMA chains for iters x 16 steps, on the current device and
 * cuda_stream, and returns the rate in *tflops (2 flops per FMA; the packed
 * POND_PIPE_FP32X2 form, fma.rn.f32x2, counts two FMAs per instruction) and
 * the launch time in *seconds (may be NULL).  sink is a device buffer of at
 * least 8 bytes that is never written in practice (it keeps the chains
 * alive).  Synchronises the stream.
 * Errors: POND_ERR_ARG (NULL tflops or sink, iters < 1, unknown pipe),
 * POND_ERR_CUDA. */
pond_status pond_measure_peak(int32_t pipe, int32_t iters, void* sink, void* cuda_stream,
                              double* tflops, double* seconds);

void pond_destroy(pond_ctx* ctx);

/* Message of the last failing call on ctx ("" if none; static text if ctx is
 * NULL). */
const char* pond_last_error(const pond_ctx* ctx);

/* Library version string. */
const char* pond_version(void);

#ifdef __cplusplus
}
#endif

#endif /* POND_H */
