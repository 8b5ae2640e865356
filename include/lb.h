/*
 * lb.h -- C ABI of the GB300 thread-safe regularized lattice Boltzmann library.
 *
 * Method: "Thread-safe lattice Boltzmann for high-performance computing on
 * GPUs" (arXiv 2304.06437).  One time step rebuilds every population from the
 * hydrodynamic moments of its upstream node,
 *     f_a(x, t+1) = f^eq_a(rho, u)(x - c_a) + (1 - omega) fhat^neq_a(Pi^neq)(x - c_a)
 * (section 3, the multline step equation; fhat^neq is the order-2 Hermite
 * projection of Eq. hermite; f^eq the He-Luo equilibrium of Eq. equil), with
 * halfway bounce-back walls and a moving lid (section 5.1) fused in.  The
 * state is ONE population array; no second array is allocated (section 4,
 * memory discussion).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Return value: LB_OK (0) or a negative LB_E_* code.  Nothing aborts, no
 *    C++ exception crosses the ABI.  lb_status_string() names a code.
 *  - Node index idx = x + nx*(y + ny*z) ("canonical"); in 2D (D2Q9) nz = 1.
 *  - Population arrays are [q][N] doubles in the canonical velocity order:
 *    rest first, then by |c|^2, then lexicographically on (cx, cy, cz) with
 *    -1 < 0 < 1.  Velocity fields are [d][N]; a symmetric tensor is [3][N]
 *    (xx, yy, xy) in 2D and [6][N] (xx, yy, zz, xy, xz, yz) in 3D.
 *  - Faces are ordered -x, +x, -y, +y, -z, +z.  Opposite faces are either both
 *    periodic or both non-periodic.  A wall sits half a link outside the
 *    outermost node, so dims counts fluid nodes.
 *  - "u" is the velocity the state reports, u = (sum_a f_a c_a + F/2) / rho0
 *    (incompressible He-Luo reading of section 2 with a body force F).
 *  - Pointers: arguments named *_host are host memory; with on_device != 0 a
 *    pointer is device memory of the context's device, readable/writable on
 *    the context's stream.  The library does not wait for other streams: work
 *    that produces a device input, or still uses a device output buffer, must
 *    be complete (or ordered before the context stream) when the call is
 *    made.  Caller-owned buffers are only accessed during the call; the
 *    library owns everything it allocates and frees it in lb_destroy().
 *  - Streams: work is enqueued on the context stream (lb_options.stream, or a
 *    non-blocking stream the library creates).  lb_step() returns once the
 *    work is enqueued; calls that return data synchronise the stream first.
 *  - Threads: a context is not internally locked; use one context per host
 *    thread (or serialise calls).
 */
#ifndef LB_H
#define LB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LB_ABI_VERSION 1

#if defined(__GNUC__)
#define LB_API __attribute__((visibility("default")))
#else
#define LB_API
#endif

/* status codes */
#define LB_OK 0
#define LB_E_INVAL (-1)       /* bad argument, unsupported combination of sizes or kinds */
#define LB_E_NOMEM (-2)       /* device or host allocation failed */
#define LB_E_CUDA (-3)        /* a CUDA runtime call failed (no device, launch error, ...) */
#define LB_E_DIVERGED (-4)    /* a reduction found a non-finite value */
#define LB_E_TIMEOUT (-5)     /* a kernel gave up waiting for an asynchronous copy */
#define LB_E_UNSUPPORTED (-6) /* valid request this build does not implement */
#define LB_E_TOO_LARGE (-7)   /* grid exceeds the fixed scratch of lb_step_noalloc */
#define LB_E_ABANDONED (-8)   /* a kernel timed out and could not confirm that its copies ended */

typedef enum { LB_D2Q9 = 0, LB_D3Q19 = 1, LB_D3Q27 = 2 } lb_lattice;
/* LB_LINK: the face borders the slab of another context (a rank boundary of
 * the slab decomposition below); only the two faces of the slowest axis (z in
 * 3D, y in 2D) and only with the fused scheme. */
typedef enum { LB_PERIODIC = 0, LB_WALL = 1, LB_MOVING_WALL = 2, LB_LINK = 3 } lb_face_kind;

/* Storage precision of the population array.  Every mode stores the shifted
 * population f_a - t_a rho0 (exact in FP64; the accurate representation in the
 * narrower formats); arithmetic is FP64 for LB_F64 and FP32 otherwise. */
typedef enum { LB_F64 = 0, LB_F32 = 1, LB_F16S = 2, LB_BF16S = 3 } lb_storage;

/* Kernel schedule.
 *  LB_SCHEME_FUSED    one fused pull-stream + regularized-collision launch per
 *                     step over brick columns; neighbouring bricks exchange
 *                     post-collision boundary populations through a small
 *                     double-buffered shell (the default, the fast path).
 *  LB_SCHEME_TWO_PASS the paper's own schedule (section 4): a moments kernel
 *                     writes rho, u, Pi^neq to full-size arrays, then a rebuild
 *                     kernel pulls them and writes the populations. */
typedef enum { LB_SCHEME_FUSED = 0, LB_SCHEME_TWO_PASS = 1 } lb_scheme;

typedef struct {
  int32_t kind[6];      /* lb_face_kind per face */
  double wall_u[6][3];  /* wall velocity per face, read for LB_MOVING_WALL */
} lb_boundary;

typedef struct {
  int32_t storage;      /* lb_storage; default LB_F32 */
  int32_t scheme;       /* lb_scheme; default LB_SCHEME_FUSED */
  double rho0;          /* reference density; default 1 */
  double force[3];      /* body force per unit volume, lattice units; default 0 */
  void* stream;         /* cudaStream_t to enqueue on; NULL = library-owned stream */
  int32_t tile[3];      /* fused scheme: brick cross-section (bx, by) and sweep
                           length bz; 0 = library choice */
  int32_t device;       /* CUDA device ordinal; -1 = the current device */
} lb_options;

typedef struct lb_ctx lb_ctx;

typedef struct {
  int32_t lattice, q, d, storage, scheme;
  int64_t dims[3];
  int64_t steps_done;
  int32_t tile[3];          /* brick (bx, by, bz) used by the fused scheme */
  uint64_t population_bytes; /* the one population array */
  uint64_t aux_bytes;        /* shells (fused) or moment arrays (two-pass) */
  uint64_t algorithmic_bytes_per_update; /* 2 q s: one read + one write per population */
  int32_t nodes_per_thread;  /* fused scheme: 1 scalar kernel, 2 paired FP32x2 kernel */
  int32_t tma_slots;         /* fused scheme: TMA ring depth */
} lb_info_t;

/* Fills *opt with the defaults listed above. */
LB_API void lb_default_options(lb_options* opt);

/* Creates a context: allocates the population array (and the shell or moment
 * buffers of the chosen scheme) on the device and zeroes the state (rest at
 * rho0).  dims[2] must be 1 for D2Q9.  tau > 1/2 (nu = (tau - 1/2)/3, section
 * 2).  bnd may be NULL (all periodic); opt may be NULL (defaults).
 * Errors: LB_E_INVAL for bad sizes/kinds, LB_E_NOMEM, LB_E_CUDA. */
LB_API int lb_create(int32_t lattice, const int64_t dims[3], double tau, const lb_boundary* bnd,
              const lb_options* opt, lb_ctx** out);

/* Sets the state to f = f^eq(rho, u) + fhat^neq(pineq) - t_a c_a.F/(2 cs2):
 * Eq. equil plus the order-2 Hermite non-equilibrium part, shifted so that
 * the state reports u.  rho [N], u [d][N], pineq [3 or 6][N] or NULL (= 0).
 * All three are host (on_device = 0) or device (on_device = 1) FP64 arrays;
 * the stored (shifted) populations are computed in the kernels' arithmetic
 * (FP64 for LB_F64 storage, FP32 otherwise).  Host arrays cross a chunk of
 * nodes at a time through one device buffer of at most 512 MB, the copies
 * overlapping the conversion. */
LB_API int lb_init_moments(lb_ctx* ctx, const double* rho, const double* u, const double* pineq,
                    int32_t on_device);

/* Uniform equilibrium state (rho, u[0..d-1]); no caller buffers. */
LB_API int lb_init_uniform(lb_ctx* ctx, double rho, const double u[3]);

/* Copies populations in/out, [q][N] FP64, canonical order.  Setting rounds to
 * the storage precision. */
LB_API int lb_set_populations(lb_ctx* ctx, const double* f, int32_t on_device);
LB_API int lb_get_populations(lb_ctx* ctx, double* f, int32_t on_device);

/* Reads the populations of the box [lo, lo+size) into host memory f_host,
 * laid out [q][size_z][size_y][size_x].  For sampled checks on large grids. */
LB_API int lb_get_region(lb_ctx* ctx, const int64_t lo[3], const int64_t size[3], double* f_host);

/* Enqueues n time steps on the context stream (asynchronous).  Each step is
 * one application of the step of section 3 (Eq. LBexp with fhat^neq, the
 * multline step equation) with the walls of section 5.1.  For n >= 4 the
 * fused scheme launches a pair of steps captured once as a CUDA graph (held
 * by the context until it is re-planned or destroyed); if the caller is
 * capturing the context stream, the steps are launched one by one and land
 * in the caller's graph.  Errors: LB_E_INVAL (n < 0, or n > 1 on a slab with
 * a link face), LB_E_CUDA (a launch failed). */
LB_API int lb_step(lb_ctx* ctx, int64_t n);

/* Density rho [N] and velocity u [d][N] of the stored state, FP64 results.
 * FP64 storage sums in FP64; the other storages sum each node's populations
 * in FP32 carrying the rounding error of every addition in a second FP32 term
 * (about twice FP32's precision, ~1e-14 of the populations' magnitude), and
 * convert the two terms to FP64 (GB300 converts and adds FP64 at a small
 * fraction of its FP32 rate).
 * Either may be NULL.  Host outputs (on_device = 0) are filled a chunk of
 * nodes at a time through one device buffer of at most 512 MB. */
LB_API int lb_moments(lb_ctx* ctx, double* rho, double* u, int32_t on_device);

/* FP64 on-device reductions over all nodes (each node's sums formed as in
 * lb_moments, accumulated over nodes in FP64): total mass sum rho, total momentum
 * sum_a f_a c_a (without the F/2 shift), and -- if residual is not NULL -- the
 * relative velocity change ||u - u_prev||_2 / ||u||_2 since the previous call
 * that asked for it (1.0 on the first such call, and on the first after the
 * state was set by lb_init_moments / lb_init_uniform / lb_set_populations).
 * u_prev is kept as an FP32 snapshot (12 bytes per node, allocated on the
 * first such call), so the residual is that of the exact u_prev within
 * 2^-24 ||u_prev|| / ||u||.  Deterministic (fixed reduction order).  Returns
 * LB_E_DIVERGED if a value is not finite. */
LB_API int lb_reduce(lb_ctx* ctx, double* mass, double mom[3], double* residual);

/* Waits for the context stream; reports the context's sticky kernel status:
 * LB_E_TIMEOUT (a kernel gave up waiting for one of its copies: the
 * populations and the shell are undefined), LB_E_ABANDONED (the same, and
 * the kernel's bounded wait for its own copies still in flight ran out too:
 * destroy the context, its device memory may still be written), LB_E_INVAL
 * (lb_halo_unpack refused a message).  Setting the state from outside
 * (lb_init_moments, lb_init_uniform, lb_set_populations) clears LB_E_TIMEOUT
 * and LB_E_INVAL; LB_E_ABANDONED stays. */
LB_API int lb_sync(lb_ctx* ctx);

/* Frees everything the context owns.  NULL is allowed. */
LB_API void lb_destroy(lb_ctx* ctx);

/* Describes a context (sizes, scheme, bytes). */
LB_API int lb_info(const lb_ctx* ctx, lb_info_t* info);

/* Host-only: the velocity table of a lattice in canonical order, c [q][3]
 * (cz = 0 in 2D), weights w [q], opposite index opp [q].  Returns q or
 * LB_E_INVAL.  Needs no GPU. */
LB_API int lb_lattice_table(int32_t lattice, int32_t* c, double* w, int32_t* opp);

/* Host-only memory accounting (section 4 of the paper): the number of
 * full-size arrays and bytes per node each schedule keeps for a lattice --
 * the paper's moment scheme (q + m arrays), a two-array "flip-flop" scheme
 * (2q + d + 1 arrays) and this library's fused single-array scheme (q arrays
 * plus the shell, reported separately by lb_info).  s = bytes per value.
 * Needs no GPU. */
typedef struct {
  int32_t q, m;                 /* populations, stored moments 1 + d + d(d+1)/2 */
  int32_t arrays_moment_scheme; /* q + m      (15 for D2Q9, 29 for D3Q19) */
  int32_t arrays_flip_flop;     /* 2q + d + 1 (21 for D2Q9, 42 for D3Q19) */
  int32_t arrays_single;        /* q */
  double bytes_per_node_moment_scheme, bytes_per_node_flip_flop, bytes_per_node_single;
} lb_memory_plan_t;
LB_API int lb_memory_plan(int32_t lattice, int32_t bytes_per_value, lb_memory_plan_t* out);

/* The brick decomposition that lb_create() would choose for the fused scheme
 * (no device is touched): brick bx x by x bz columns and their counts, the
 * TMA pipeline depth, nodes per thread, dedicated export warps, dynamic
 * shared memory per CTA and the shell size (elements of one parity: every
 * brick face keeps the outgoing populations of its boundary nodes).  tile as
 * lb_options.tile (NULL = default); sms > 0 plans the sweep length for that
 * many SMs (0 = the current device's count, 152 if none is visible).  dims
 * in user axes as for lb_create().  Errors: LB_E_INVAL, LB_E_UNSUPPORTED (no
 * compiled brick shape matches the request). */
typedef struct {
  int32_t bx, by, bz, nbx, nby, nbz;
  int64_t bricks;
  int32_t tma_slots, nodes_per_thread, export_warps;
  int64_t shared_bytes;
  int64_t shell_elems_per_parity;
} lb_plan_t;
LB_API int lb_plan_fused(int32_t lattice, int32_t storage, const int64_t dims[3], const int32_t tile[3],
                         int32_t sms, lb_plan_t* out);

/* Allocation-free step for callers that cannot let a library call
 * cudaMalloc (device memory owned by another allocator or a fixed budget, or
 * loops that must not enter the driver's allocator).  The paper has no
 * counterpart: this is an interface variant of LB_SCHEME_TWO_PASS.
 *
 * Advances f by n steps in place, on `stream` (cudaStream_t, NULL = the
 * default stream); returns once the work is enqueued.  f is the caller's
 * device array of populations, [q][N] FP64 in the canonical order and layout
 * of lb_set_populations(); the result equals lb_set_populations() +
 * lb_step(n) + lb_get_populations() of an LB_F64 / LB_SCHEME_TWO_PASS
 * context with the same arguments.  lattice, dims, tau, bnd (NULL = all
 * periodic), rho0 and force (NULL = 0) mean what they mean for lb_create().
 *
 * Nothing is allocated: the moment arrays live in a file-scope device array
 * of LB_NOALLOC_SCRATCH_BYTES, shared by every call on a device and kept
 * until the process exits.  Hence (1 + d + d(d+1)/2) * N * 8 bytes must fit:
 * N <= 1,398,101 nodes for D2Q9 and N <= 838,860 for D3Q19 / D3Q27; larger
 * grids return LB_E_TOO_LARGE before any GPU work.  The first call in a
 * CUDA context (normally the device's primary context) looks up the array's
 * device address in that context and caches it under the context's unique id
 * (make that call before any stream capture); a new context, for instance
 * after cudaDeviceReset(), gets its own look-up.  Calls that overlap on the
 * GPU race on the shared array: order them on one stream.  Errors:
 * LB_E_INVAL, LB_E_TOO_LARGE, LB_E_UNSUPPORTED (internal y or z extent above
 * 65535): f untouched.  LB_E_CUDA: if a step's launch failed, f is shifted
 * back and holds the populations after an unspecified number of completed
 * steps; after a sticky device error its contents are undefined. */
#define LB_NOALLOC_SCRATCH_BYTES (64ull << 20)
LB_API int lb_step_noalloc(int32_t lattice, const int64_t dims[3], double tau, const lb_boundary* bnd,
                           double rho0, const double force[3], double* f, int64_t n, void* stream);

/* ---------------------------------------------------------------- autotuner
 * Picks the fused step's brick shape for a context by measurement (the paper
 * tunes nothing; its thread blocks are fixed, elongated along x).  Every
 * compiled shape of the context's lattice and storage -- brick bx x by, TMA
 * pipeline depth, one or two nodes per thread -- is timed for `steps` steps
 * on a proxy domain with the same cross-section, boundaries, tau and force and
 * at most ~4 GB of populations (the sweep axis shortened; the proxy is
 * allocated and freed inside the call, on the context's device).  The fastest
 * per node update is applied to the context: new shell buffers and TMA
 * descriptor, the shell rebuilt from the current populations, which are not
 * changed (every shape computes the same bits).  The choice is cached per
 * (lattice, storage, cross-section, sweep length rounded up to a power of two,
 * face kinds, forcing); a cached kind is applied without timing and reports
 * *n_entries = 0.  table (may be NULL) receives up to cap entries, one per
 * shape timed.  Synchronises the context stream.  Errors: LB_E_INVAL,
 * LB_E_UNSUPPORTED (two-pass scheme), LB_E_NOMEM, LB_E_CUDA. */
typedef struct {
  int32_t bx, by, bz;          /* brick and the sweep length the planner gave the proxy */
  int32_t slots;               /* TMA ring depth */
  int32_t nodes_per_thread;    /* 1 scalar, 2 paired FP32x2 kernel */
  int32_t export_warps;        /* dedicated shell-export warps (0: shared; n > 0 decoupled;
                                  -n: n warps inside the per-plane barrier) */
  int32_t status;              /* LB_OK, or why this shape could not be timed */
  double ns_per_update;        /* measured time per node update; -1 if not timed */
} lb_tune_entry;
LB_API int lb_autotune(lb_ctx* ctx, int32_t steps, lb_tune_entry* table, int32_t cap, int32_t* n_entries);

/* ------------------------------------------------------------------ batches
 * Many independent domains stepped together (the paper steps one domain; a
 * batch serves many small ones, which alone cannot fill the GPU).
 *
 * lb_batch_create groups n existing contexts of the fused scheme on one device
 * (any lattices, sizes, tau, boundaries and forces).  Contexts that share a
 * compiled brick shape and the forcing switch form a class; per time step each
 * class runs ONE persistent launch whose CTAs sweep a static, cost-balanced
 * list of the brick columns of all its domains, and the launches of two
 * consecutive steps are captured once in a CUDA graph and replayed.  The
 * populations of every domain are bit for bit those of stepping it alone.
 * Every storage is batched; two-pass contexts give LB_E_UNSUPPORTED.  The
 * batch keeps
 * pointers to the contexts, which must outlive it and must not be re-planned
 * while it exists; stepping a member alone between batch steps is allowed.
 * lb_batch_create re-plans members for batched throughput (kept after the
 * batch is destroyed; results are unchanged, every plan gives the same bits):
 * the preferred compiled brick shape that pads the domain's cross-section by
 * at most 25 % (else the least padded one), and one brick per column for
 * sweeps of up to 256 planes; where a class would then have fewer than two
 * bricks per persistent CTA, its members' sweeps are halved (down to 64
 * planes) until it has.  Classes run on parallel branches of the graph.
 * stream: cudaStream_t for the batch's work, NULL = a library-owned stream.
 * Errors: LB_E_INVAL (NULL, duplicates, mixed devices), LB_E_UNSUPPORTED,
 * LB_E_NOMEM, LB_E_CUDA. */
typedef struct lb_batch lb_batch;
typedef struct {
  int32_t n_domains, n_classes;
  int32_t launches_per_step;  /* one per class */
  int32_t ctas;               /* persistent CTAs over all classes */
  int64_t work_items;         /* brick columns over all domains */
  int64_t total_nodes;
  int64_t steps_done;
} lb_batch_info_t;
LB_API int lb_batch_create(lb_ctx* const* ctxs, int32_t n, void* stream, lb_batch** out);

/* Enqueues n time steps of every member (asynchronous).  The batch stream
 * first waits for work already queued on the members' own streams, and
 * afterwards each member's stream waits for the batch, so lb_moments() and
 * friends on a member see the batch's steps. */
LB_API int lb_batch_step(lb_batch* b, int64_t n);

/* lb_reduce for every member in one pass: the FP64 sums of all members are
 * enqueued on the batch stream (after the batch's steps and the work queued
 * on the members' own streams) and read back with one copy.  out[6 i + 0] =
 * mass, [6 i + 1 .. 3] = momentum (user axes), [6 i + 4] = residual (with
 * want_residual != 0; lb_reduce's definition and history, else 0), [6 i + 5]
 * = 0 or LB_E_DIVERGED for member i (in the order given to
 * lb_batch_create).  Synchronises the batch stream.  The first call allocates
 * the batch's sum buffers (7 doubles per member, device and pinned host).
 * Errors: LB_E_INVAL, LB_E_NOMEM, LB_E_CUDA. */
LB_API int lb_batch_reduce(lb_batch* b, int32_t want_residual, double* out);

/* Waits for the batch stream; returns LB_E_TIMEOUT if a kernel of the batch
 * gave up waiting for a copy. */
LB_API int lb_batch_sync(lb_batch* b);
LB_API int lb_batch_info(const lb_batch* b, lb_batch_info_t* info);

/* Frees the batch (not its contexts).  NULL is allowed. */
LB_API void lb_batch_destroy(lb_batch* b);

/* --------------------------------------------------- two-component model
 * The paper's colour-gradient (CG) model for two immiscible fluids, red and
 * blue (section 2.1), in the thread-safe form of section 4: per step one
 * launch takes the moments of each node (the regularized relaxation
 * coefficients of the total set g = f_R + f_B, the concentrations and the
 * phase field phi = (rho_R - rho_B)/rho), one takes grad phi by the isotropic
 * stencil (1/cs2) sum_a t_a c_a phi(x + c_a), and one rebuilds both colours
 * at every node from the upstream node's fields:
 *   g*_a = [Eq. LBexp with fhat^neq]_a + (9/4) sigma omega |grad phi|
 *          [t_a (c_a.n)^2 - B_a]                          (perturbation)
 *   f_R,a = (rho_R/rho) g*_a + beta (rho_R rho_B/rho) t_a (c_a.n)/|c_a|,
 *   f_B,a = g*_a - f_R,a                                  (recolouring)
 * with n = grad phi / |grad phi| and B_a = -4/27, 2/27, 5/108 (D2Q9) or
 * -2/9, 1/54, 1/27 (D3Q19) by |c|^2 shell.  Each colour is one population
 * array.  Periodic box, D2Q9 or D3Q19, LB_F64 or LB_F32 (storage and
 * arithmetic); rho0 = 1; u = sum_a (f_R + f_B) c_a / rho0.
 * Arrays are FP64 in the conventions above ([q][N] populations, [d][N]
 * velocity); host (on_device = 0) or device (1) pointers.
 * lb_cg_create: tau > 1/2, sigma >= 0 (surface tension), 0 <= beta <= 1
 *   (interface width); starts as an even mixture at rest.  stream as for
 *   lb_options.stream.  Errors: LB_E_INVAL, LB_E_UNSUPPORTED (other lattice
 *   or storage), LB_E_NOMEM, LB_E_CUDA.
 * lb_cg_init: f_k = (rho_k/rho) f^eq(rho, u) (Eq. equil); u may be NULL.
 * lb_cg_step enqueues n steps; the others synchronise the stream. */
typedef struct lb_cg lb_cg;
LB_API int lb_cg_create(int32_t lattice, const int64_t dims[3], double tau, double sigma, double beta,
                        int32_t storage, void* stream, lb_cg** out);
LB_API int lb_cg_init(lb_cg* c, const double* rho_r, const double* rho_b, const double* u, int32_t on_device);
LB_API int lb_cg_set_populations(lb_cg* c, const double* f_r, const double* f_b, int32_t on_device);
LB_API int lb_cg_get_populations(lb_cg* c, double* f_r, double* f_b, int32_t on_device);
LB_API int lb_cg_step(lb_cg* c, int64_t n);
LB_API int lb_cg_fields(lb_cg* c, double* rho_r, double* rho_b, double* u, int32_t on_device);
LB_API int lb_cg_sync(lb_cg* c);
LB_API void lb_cg_destroy(lb_cg* c);

/* Near-contact interactions (section 2.2): a short-range repulsion that keeps
 * approaching interfaces from coalescing.  Before each collision a node y is
 * flagged if, for some direction a, the node y - h c_a is bulk continuous
 * (blue) phase, phi < -1 + eps, while y and y - 2h c_a are not (the paper's
 * test from the bulk node, evaluated at the flagged node); a flagged node
 * collides with the body force F = amplitude * rho_R * grad phi / |grad phi|
 * (towards the dispersed, red phase; the forcing of the single-component
 * step), so the force grows as the films between interfaces thin.  The paper
 * gives no values for eps, h or the amplitude.  amplitude = 0 (the state after
 * lb_cg_create) switches the interactions off; amplitude >= 0 and finite,
 * 0 < eps < 2, h >= 1 with 2h <= every periodic extent, else LB_E_INVAL.
 * Takes effect from the next lb_cg_step. */
LB_API int lb_cg_set_nci(lb_cg* c, double amplitude, double eps, int32_t h);

/* Self-test of the bounded wait that every kernel applies to its mbarrier
 * waits (the paper has no counterpart: failure detection of this library).
 * Launches one tiny kernel that waits on a barrier nothing completes, for at
 * most limit_ns nanoseconds (0 .. 5e9), and returns the status the kernel
 * recorded -- LB_E_TIMEOUT when the wait ran out as designed -- with the time
 * it waited in *waited_ns (may be NULL).  Uses the current device and the
 * default stream; synchronises the device.  Errors: LB_E_INVAL, LB_E_NOMEM,
 * LB_E_CUDA. */
LB_API int lb_selftest_timeout(int64_t limit_ns, int64_t* waited_ns);

/* ------------------------------------------------------------------ slabs
 * Domain decomposition along the slowest axis (z in 3D, y in 2D), the
 * multi-GPU form of the method (the paper names multi-GPU scaling as its
 * future work, section 7).  Each rank owns a slab -- a context whose faces on
 * that axis are LB_LINK where it borders another slab -- and a rank boundary
 * is just another brick face of the fused scheme: the post-collision
 * populations that leave a slab through it are the shell records the
 * neighbouring slab's boundary bricks read in the next launch.  They travel
 * as one message per link face and step:
 *   sender:   lb_halo_pack(ctx, side, buf)      side 0 = low face, 1 = high face
 *   transport (a device copy on one GPU, NCCL send/recv between GPUs)
 *   receiver: lb_halo_unpack(ctx, 1 - side, buf)
 * after which the receiver takes one step, lb_step(ctx, 1) (a linked context
 * rejects n > 1: its halo is stale after one launch).  The message holds, for
 * the sender's outermost plane, its x- and y-face shell records (the lateral
 * populations of the neighbouring bricks, which the receiver needs for its
 * diagonal links) and the z-face records of its outermost brick row; the
 * receiver stores them in ghost slots of its shell, so no slab ever writes
 * another's memory.  Every slab computes the same bits as the single domain
 * (the shell records are the neighbour's rounded state collided once more).
 *
 * lb_halo_bytes: size of one message of ctx, a multiple of 16 (equal on both
 *   sides of a boundary when the slabs share lattice, storage, the extents of
 *   the two other axes and the brick cross-section).
 * lb_halo_pack: enqueues on the context stream the copy of the records that
 *   leave through face `side` of the current state into buf (device memory
 *   of the context's device, lb_halo_bytes, 16-byte aligned), preceded by a
 *   64-byte header naming the layout.
 * lb_halo_unpack: enqueues the copy of a neighbour's message into the ghost
 *   slots of face `side`.  If the header does not match this context (other
 *   lattice, precision, extents, brick cross-section, or a message packed for
 *   the same side), nothing is copied and the kernel records LB_E_INVAL,
 *   which the next lb_sync() returns.
 * Errors: LB_E_INVAL (NULL, side not 0/1, face `side` not LB_LINK), LB_E_CUDA. */
LB_API int lb_halo_bytes(const lb_ctx* ctx, int64_t* bytes);
LB_API int lb_halo_pack(lb_ctx* ctx, int32_t side, void* buf);
LB_API int lb_halo_unpack(lb_ctx* ctx, int32_t side, const void* buf);

/* A slab group: the decomposition run in one process on one device, one
 * context and one stream per rank -- the stand-in for one rank per GPU, with
 * the message copies on the device in place of NCCL.  lb_group_create cuts
 * the domain (arguments as for lb_create) into nranks slabs along the slowest
 * axis, counts[r] planes each (NULL: as even as possible; every count >= 1,
 * summing to the extent); faces between slabs become LB_LINK, and a periodic
 * slowest axis links the last slab to the first (a single rank then links to
 * itself).  Every rank uses the brick cross-section of rank 0; opt->stream is
 * ignored (each rank gets a library-owned stream).  Errors as for lb_create,
 * plus LB_E_INVAL for bad counts.
 * lb_group_rank: rank r's context (owned by the group: initialise and read it
 *   with the calls above; its node range is the global one from *offset
 *   planes on, in the canonical layout a contiguous range of nodes).
 * lb_group_step: n steps; per step every rank packs its link faces, waits
 *   (by events) for its neighbours' messages, unpacks them and launches its
 *   step, and a rank packs again only after its neighbours unpacked.
 * lb_group_sync: waits for every rank; returns the first non-OK status. */
typedef struct lb_group lb_group;
LB_API int lb_group_create(int32_t lattice, const int64_t dims[3], double tau, const lb_boundary* bnd,
                           const lb_options* opt, int32_t nranks, const int64_t* counts, lb_group** out);
LB_API int lb_group_rank(lb_group* grp, int32_t rank, lb_ctx** ctx, int64_t* offset);
LB_API int lb_group_step(lb_group* grp, int64_t n);
LB_API int lb_group_sync(lb_group* grp);
LB_API void lb_group_destroy(lb_group* grp);

/* Human-readable name of a status code. */
LB_API const char* lb_status_string(int code);

/* ABI version of the loaded library (LB_ABI_VERSION it was built with). */
LB_API int lb_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LB_H */
