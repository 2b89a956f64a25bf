/*
 * cmlbm.h -- C ABI of the GB300 (sm_103a) D3Q27 central-moment lattice Boltzmann solver with
 * external forcing of De Rosis, Huang & Coreixas, "Three-dimensional central-moments-based
 * lattice Boltzmann method with external forcing" (arXiv 1905.10182).
 *
 * What one step computes (Sec. II, the five-step time iteration at its end):
 *   1. rho = sum_i f_i, rho u = sum_i f_i c_i + F/2                       (Eq. macroscopic)
 *   2. the pre-collision central moments k4..k8                           (Eq. pre_collision)
 *   3. the 19 nonzero post-collision central moments, second-order moments relaxed at
 *      omega = 1/(3 nu + 1/2), every other moment at rate 1               (Eq. eq:relaxationMatrix,
 *                                                           Eq. post_collision_central_moments_forcing)
 *   4. f* = (T^T)^-1 k*                                                   (Eq. system)
 *   5. f_i(x + c_i, t + 1) = f*_i(x, t)                                   (Eq. streaming)
 * on the D3Q27 lattice of Sec. II, in lattice units (c_s^2 = 1/3).
 *
 * Conventions shared by every call
 *   - Grid: nx * ny * nz nodes; node n = x + nx*(y + ny*z) (x fastest).  Fields are arrays of
 *     N = nx*ny*nz floats in that order; populations are 27*N floats, population i of node n
 *     at [i*N + n], directions ordered as in Sec. II.
 *   - Boundaries: periodic in x and z; periodic in y unless walls_y, which places halfway
 *     bounce-back walls at y = -1/2 and y = ny - 1/2.  A mask marks solid nodes; links into
 *     a solid node bounce back halfway: f_opp(i)(x, t+1) = f*_i(x, t).  Solid nodes are never
 *     collided and are excluded from every diagnostic.
 *   - Force F is a force density (the forcing term carries no rho prefactor).
 *   - Pointers: arrays passed in may live in host or device memory (detected per call).  The
 *     caller owns them; the library copies what it keeps and never frees them.
 *   - Streams: every call enqueues its work on desc.stream (NULL = the legacy default stream).
 *     lbm_step only enqueues; lbm_macroscopic, lbm_get_populations, lbm_stats and
 *     lbm_synchronize wait for the stream.
 *   - Errors: no call throws or aborts.  Each returns an lbm_status; lbm_last_error() gives a
 *     message for the context (or, with NULL, for the last failed lbm_create on this thread).
 *     A context whose call returned LBM_ERR_CUDA should be destroyed.
 *   - Storage: populations are stored as deviations g_i = f_i - w_i rho0 in FP32, FP16 or
 *     BF16 (round to nearest even); all collision arithmetic is FP32.
 */
#ifndef CMLBM_H
#define CMLBM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LBM_API __attribute__((visibility("default")))
#else
#define LBM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = 1,         /* invalid argument (sizes, pointers, kinds)                        */
    LBM_ERR_CUDA = 2,        /* a CUDA call failed; the message names it                         */
    LBM_ERR_OOM = 3,         /* device allocation failed                                         */
    LBM_ERR_DIVERGED = 4,    /* some node reached rho <= 0, |u| >= 1 or NaN since the last check */
    LBM_ERR_TIMEOUT = 5,     /* a bounded device wait gave up                                    */
    LBM_ERR_STATE = 6,       /* call not valid in the context's current state                    */
    LBM_ERR_UNSUPPORTED = 7  /* combination not supported (e.g. Shan-Chen with walls or masks)    */
} lbm_status;

typedef enum {
    LBM_FP32 = 0,     /* 4 B per population */
    LBM_FP16_DEV = 1, /* 2 B per population, IEEE half deviation */
    LBM_BF16_DEV = 2  /* 2 B per population, bfloat16 deviation  */
} lbm_storage;

typedef enum {
    LBM_FORCE_NONE = 0,       /* F = 0                                                            */
    LBM_FORCE_UNIFORM = 1,    /* F = (params[0], params[1], params[2]) on every node              */
    LBM_FORCE_KOLMOGOROV = 2, /* F_x = params[0] * sin(2 pi y / ny), F_y = F_z = 0               */
    LBM_FORCE_FIELD = 3,      /* F from the fx, fy, fz arrays (N floats each, copied)             */
    LBM_FORCE_SHAN_CHEN = 4   /* F = -G psi(x) sum_i w_i c_i psi(x + c_i), psi = 1 - exp(-rho),
                                 G = params[0]; rho is the density at the current time step
                                 (Sec. III, static droplet).  Periodic domains only.             */
} lbm_force_kind;

typedef struct {
    int nx, ny, nz;        /* grid size, each >= 1; N = nx*ny*nz < 2^31                          */
    double nu;             /* kinematic viscosity > 0; omega = 1/(3 nu + 1/2) (Sec. II)          */
    double rho0;           /* reference density (> 0); initial state rho = rho0, u = 0 (Sec. III) */
    int walls_y;           /* 1: halfway bounce-back walls at y = -1/2 and y = ny - 1/2           */
    const uint8_t* mask;   /* NULL, or N bytes (host or device), nonzero = solid node             */
    int storage;           /* lbm_storage                                                         */
    void* stream;          /* cudaStream_t to run on; NULL = legacy default stream                */
    void* store;           /* NULL: the library allocates the population store.  Otherwise a
                              device buffer of lbm_store_bytes(desc) bytes, 256-byte aligned,
                              owned by the caller and kept alive until lbm_destroy.               */
    int slab_z;            /* 1: this context is one z slab (nz planes) of a larger domain that is
                              periodic in z across slabs; the store gets one ghost plane below and
                              one above, filled by lbm_halo_unpack (see there).  No masks and no
                              Shan-Chen or field forces with slabs.                               */
} lbm_desc;

/* Bytes of the population store for desc (27 * N * element size); 0 on invalid sizes. */
LBM_API size_t lbm_store_bytes(const lbm_desc* desc);

/* Creates a solver on the current CUDA device, initialised to rho = rho0, u = 0, F = 0
 * (Sec. III: the density starts at rho0 with the fluid at rest).  On failure *out = NULL. */
LBM_API lbm_status lbm_create(const lbm_desc* desc, lbm_ctx** out);

/* Selects the force source (lbm_force_kind).  params: see the kind; may be NULL for NONE and
 * FIELD.  fx, fy, fz: used by FIELD only (host or device, N floats each, copied). */
LBM_API lbm_status lbm_set_force(lbm_ctx* ctx, int kind, const double* params, const float* fx, const float* fy,
                         const float* fz);

/* Hermite truncation orders of the equilibrium (Eq. eq:truncation) and of the forcing term
 * (Eq. generalForcing) used by the collision, among the models compared in Sec. III:
 *   (6, 6)  complete expansions, the present method M1 (the default);
 *   (6, 2)  complete equilibrium, second-order (Guo) forcing term: M4;
 *   (2, 2)  classical second-order equilibrium and forcing term: M5;
 *   (2, 6)  second-order equilibrium with the complete forcing term.
 * With either order at 2 the central moments of order >= 3 (relaxed at rate 1) take the
 * velocity-dependent values of the truncated expansions; k0..k9 are unchanged.  Takes effect at
 * the next step; lbm_set_state keeps using the complete equilibrium (all truncations agree at
 * u = 0).  Orders other than 2 and 6: LBM_ERR_UNSUPPORTED. */
LBM_API lbm_status lbm_set_hermite_orders(lbm_ctx* ctx, int eq_order, int force_order);

/* Magnetic field (App. C): turns on a second LBM for the magnetic field b on D3Q7 (vector
 * populations h_l, l = rest, +-x, +-y, +-z; BGK with omega_m, eta = (1/omega_m - 1/2) / 4;
 * h_la^eq = w_l [b_a + 4 xi_lb (u_b b_a - b_b u_a)], w = 1/4, 1/8; b = sum_l h_l), coupled to the
 * fluid through the Lorentz force j x b added to the force density (Sec. III, Hartmann flow and
 * Orszag-Tang vortex).  The current is read from the populations: j = -(4 omega_m)(E - 2 u x b),
 * E_g = eps_gba sum_l xi_lb h_la (pre-collision), with u and j solved together from
 * rho u = sum f c + (F + j x b)/2 (linear in u).  At y walls the field b_wall (3 doubles, NULL:
 * zero) is held by anti-bounce-back.  Initial state h = h^eq(b, u) with u of the current fluid
 * state; bx, by, bz: N floats each (host or device; NULL: zero).  Every later lbm_step advances
 * both; lbm_macroscopic and lbm_stats include j x b / 2 in u.  Needs FP32 storage, no solid mask,
 * no z slab, force NONE or UNIFORM, even parity (after lbm_set_state or an even number of
 * steps), fewer than 2^32 / 27 (159 M) nodes: else LBM_ERR_UNSUPPORTED / LBM_ERR_STATE.  eta > 0.
 * Adds 84 B per node. */
LBM_API lbm_status lbm_set_magnetic(lbm_ctx* ctx, double eta, const double b_wall[3], const float* bx,
                                    const float* by, const float* bz);

/* Magnetic populations at the current time, natural order h[(3 l + a) N + n] (21 N floats, host
 * or device).  Set: only at even parity; get: any time.  LBM_ERR_STATE without a magnetic field. */
LBM_API lbm_status lbm_get_magnetic_populations(lbm_ctx* ctx, float* h);
LBM_API lbm_status lbm_set_magnetic_populations(lbm_ctx* ctx, const float* h);

/* b and j = curl b at the current time (N floats each, host or device, NULL to skip); syncs. */
LBM_API lbm_status lbm_magnetic(lbm_ctx* ctx, float* bx, float* by, float* bz, float* jx, float* jy, float* jz);

/* Colour-gradient two-phase model (App. D): red and blue fluids with D3Q27 populations f^r, f^b;
 * the total f = f^r + f^b takes the central-moment collision of Sec. II with the enhanced
 * equilibrium of App. D (phi_i(alpha), the sixth-order Hermite terms, the density-gradient terms
 * Phi_i), then the perturbation operator (interfacial tension, amplitude A) and the recolouring
 * (parameter beta) split it again.  Per node: phi = (rho_r/rho_r0 - rho_b/rho_b0) /
 * (rho_r/rho_r0 + rho_b/rho_b0); alpha_b = 8/27, alpha_r = 1 - (1 - alpha_b) rho_b0/rho_r0;
 * 1/nu = (1+phi)/(2 nu_r) + (1-phi)/(2 nu_b), omega = 1/(3 nu + 1/2) on k4..k8; gradients by the
 * isotropic central stencil (a neighbour behind a y wall takes the node's value); body force
 * F = (rho - (rho_r0 + rho_b0)/2) g (Sec. III, Rayleigh-Taylor instability).  Readings: the
 * perturbation uses (c_i . grad phi)^2 (it then conserves mass); recolouring uses rho phi_i(alpha)
 * as f^eq(rho, 0).  Initial state at rest: f^k_i = rho_k phi_i(alpha(phi)) from rho_r, rho_b
 * (N floats each, host or device).  Afterwards the context's store holds the red populations
 * (full, not deviations) and lbm_set_state / lbm_set_populations / lbm_get_populations answer
 * LBM_ERR_UNSUPPORTED; lbm_step, lbm_macroscopic (rho = rho_r + rho_b, u with F/2) and lbm_stats
 * work on the total.  Needs FP32 storage, no mask, no z slab, no magnetic field, force NONE,
 * fewer than 2^32 / 27 (159 M) nodes; rho_b0 / rho_r0 <= 27/19.  Adds 116 B per node. */
typedef struct {
    double rho_r0, rho_b0; /* densities of the pure red and blue fluids */
    double nu_r, nu_b;     /* their kinematic viscosities */
    double A;              /* perturbation amplitude (interfacial tension) */
    double beta;           /* recolouring parameter, 0..1 */
    double g[3];           /* gravity vector of the body force */
} lbm_cg_params;
LBM_API lbm_status lbm_set_colour_gradient(lbm_ctx* ctx, const lbm_cg_params* params, const float* rho_r,
                                           const float* rho_b);
/* Colour densities at the current time (N floats each, host or device, NULL to skip); syncs. */
LBM_API lbm_status lbm_colour_densities(lbm_ctx* ctx, float* rho_r, float* rho_b);
/* Red and blue populations at the current time, natural order, full populations (27 N floats
 * each, host or device).  Set: only at even parity. */
LBM_API lbm_status lbm_get_colour_populations(lbm_ctx* ctx, float* fr, float* fb);
LBM_API lbm_status lbm_set_colour_populations(lbm_ctx* ctx, const float* fr, const float* fb);

/* Sets f = f^eq(rho, u), the complete (sixth-order Hermite) equilibrium of Eq. eq:truncation,
 * on every fluid node (rest state on solid nodes).  Arrays: N floats each, host or device.
 * Resets the step counter to 0. */
LBM_API lbm_status lbm_set_state(lbm_ctx* ctx, const float* rho, const float* ux, const float* uy, const float* uz);

/* Sets the populations from g (27*N floats, deviations f_i - w_i rho0, host or device) and
 * resets the step counter to 0. */
LBM_API lbm_status lbm_set_populations(lbm_ctx* ctx, const float* g);

/* Copies the populations at the current time into g (27*N floats, deviations
 * f_i - w_i rho0, host or device), decoded from the stored precision.  Waits for the stream. */
LBM_API lbm_status lbm_get_populations(lbm_ctx* ctx, float* g);

/* Enqueues nsteps >= 0 time steps.  Returns LBM_ERR_DIVERGED if an earlier step (seen at the
 * last synchronising call) left the physical range. */
LBM_API lbm_status lbm_step(lbm_ctx* ctx, int nsteps);

/* Enqueues nsteps steps of free streaming: the collision is replaced by f* = f while the AA
 * addressing, periodic wrap and halfway bounce-back are those of lbm_step.  FP32 storage only
 * (LBM_ERR_UNSUPPORTED otherwise).  Populations move bit for bit, so a labelled state checks
 * the streaming indices exactly. */
LBM_API lbm_status lbm_stream_only(lbm_ctx* ctx, int nsteps);

/* ------------------------------------------------------------------------------------------
 * z-slab decomposition.  Even steps of the AA update touch only a node's own slots, so slabs
 * exchange nothing; an odd step reads and writes the slots of the neighbour nodes, so across each
 * slab face it needs the 9 populations with c_z pointing into the slab (before the step) and
 * returns the 9 it pushed out (after it).  Per odd step, with B = lbm_halo_bytes(ctx) bytes per
 * device buffer:
 *   before:  pack(face 0, stage 0) -> rank below;  pack(face 1, stage 0) -> rank above;
 *            unpack(face 1, stage 0) <- rank above; unpack(face 0, stage 0) <- rank below;
 *   lbm_step(ctx, 1);
 *   after:   pack(face 0, stage 1) -> rank below;  pack(face 1, stage 1) -> rank above;
 *            unpack(face 1, stage 1) <- rank above; unpack(face 0, stage 1) <- rank below.
 * Face 0 is the bottom (z = 0) side, face 1 the top.  One slab exchanging with itself is the
 * periodic domain.  The stage-1 unpack keeps every slot whose source lies behind a y wall (it
 * holds the node's own bounce-back, which nothing across the face pushed).  Read fields
 * (lbm_macroscopic, lbm_get_populations) at even parity.
 * ------------------------------------------------------------------------------------------ */
LBM_API size_t lbm_halo_bytes(const lbm_ctx* ctx);
LBM_API lbm_status lbm_halo_pack(lbm_ctx* ctx, int face, int stage, void* buf);
LBM_API lbm_status lbm_halo_unpack(lbm_ctx* ctx, int face, int stage, const void* buf);
/* Checkpoint / resume.  lbm_save writes a header (grid, storage, boundaries, nu, rho0, force
 * kind and parameters, Hermite orders, step counter, AA parity) and the raw population store to
 * path.  lbm_load reads it back into a context created and configured like the saved one: the
 * same grid, storage and boundaries, nu and rho0, force kind and parameters (lbm_set_force) and
 * Hermite orders (lbm_set_hermite_orders), else LBM_ERR_STATE and the context is unchanged.  It
 * restores the step counter and parity, so that a resumed run continues bit for bit.  Force
 * fields and masks are not saved: set them again on the new context.  Both wait for the stream.
 * A context with a magnetic field (lbm_set_magnetic) or a colour-gradient two-phase model
 * (lbm_set_colour_gradient): LBM_ERR_UNSUPPORTED. */
LBM_API lbm_status lbm_save(lbm_ctx* ctx, const char* path);
LBM_API lbm_status lbm_load(lbm_ctx* ctx, const char* path);

/* Storage parity: 0 after an odd step or a set call (natural order), 1 after an even step. */
LBM_API int lbm_parity(const lbm_ctx* ctx);

/* Writes rho and u (u includes F/2, Eq. macroscopic) at the current time.  Any output may be
 * NULL; each is N floats, host or device.  Solid nodes get rho0 and 0.  Waits for the stream;
 * returns LBM_ERR_DIVERGED when a step since the last check flagged a node. */
LBM_API lbm_status lbm_macroscopic(lbm_ctx* ctx, float* rho, float* ux, float* uy, float* uz);

#define LBM_STATS_LEN 10
/* FP64 diagnostics over fluid nodes at the current time (host array of LBM_STATS_LEN):
 *   [0] mass sum rho   [1..3] momentum sum rho u   [4] residual |u - u_prev|_2 / |u|_2, u_prev
 *   being u at the previous lbm_stats call (1.0 on the first call; NaN when the fields hold a
 *   non-finite value)   [5] kinetic energy,
 *   mean of |u|^2/2   [6] enstrophy, mean of |curl u|^2/2 (second-order central differences,
 *   u = 0 behind walls and on solid nodes)   [7] max |u|   [8] fluid node count   [9] step.
 * Deterministic: fixed reduction order.  Waits for the stream. */
LBM_API lbm_status lbm_stats(lbm_ctx* ctx, double* out);

/* Waits for the stream; LBM_ERR_DIVERGED if a step since the last check flagged a node. */
LBM_API lbm_status lbm_synchronize(lbm_ctx* ctx);

/* Kernel timing hook for benchmarks: with every >= 1, lbm_step records a CUDA event pair on the
 * context's stream around the stream-collide launch and the psi launch of the steps t with
 * t mod every in {0, 1} -- a pair of consecutive steps, so both AA parities (whose kernels differ)
 * are sampled equally; every = 1 times all steps, every = 0 turns it off.  It changes no result;
 * the cost is two event records per timed launch. */
LBM_API lbm_status lbm_profile(lbm_ctx* ctx, int every);

#define LBM_PROFILE_LEN 4
/* Waits for the stream, then returns and clears the totals gathered since the last read
 * (host array of LBM_PROFILE_LEN): [0] stream-collide kernel time in ms, [1] its launches,
 * [2] psi kernel time in ms, [3] its launches. */
LBM_API lbm_status lbm_profile_read(lbm_ctx* ctx, double* out);

/* Time steps taken since creation or the last lbm_set_state / lbm_set_populations. */
LBM_API long long lbm_time(const lbm_ctx* ctx);

/* Message of the last error of ctx (NULL ctx: of the last lbm_create on this thread). */
LBM_API const char* lbm_last_error(const lbm_ctx* ctx);
LBM_API const char* lbm_status_string(int status);

/* ------------------------------------------------------------------------------------------
 * Batched solver: many independent domains, each with its own grid, nu, constant force, walls
 * and solid mask, advanced together by one persistent kernel launch per time step over a
 * device-resident tile list, replayed from a captured CUDA graph.  The per-node step is the one
 * of lbm_step (Sec. II, FP32 storage), so each domain evolves exactly as a single domain would.
 * A domain whose FP64 residual r = |u^n - u^(n-D)|_2 / (D |u^n|_2) -- the mean relative velocity
 * change per step over the window D = check_every, norms over fluid nodes -- falls to tol is
 * retired: its state is frozen and it leaves the tile list.
 * ------------------------------------------------------------------------------------------ */
typedef struct lbm_batch lbm_batch;

typedef struct {
    int nx, ny, nz;        /* grid, N = nx*ny*nz < 2^31                                           */
    double nu;             /* viscosity > 0                                                        */
    double force[3];       /* constant force density                                               */
    int walls_y;           /* halfway bounce-back walls at y = -1/2 and ny - 1/2                   */
    const uint8_t* mask;   /* NULL or N bytes (host or device), nonzero = solid; copied            */
} lbm_domain;

/* Creates the batch (all domains at rest: rho = rho0, u = 0) on the current device and stream.
 * Population memory: 108 B per node in one pool, plus 16 B per node (links, previous u).  Each
 * domain holds fewer than 2^32 / 27 (159 M) nodes, else LBM_ERR_ARG. */
LBM_API lbm_status lbm_batch_create(const lbm_domain* domains, int count, double rho0, void* stream, lbm_batch** out);

/* Times trial_steps (rounded to even, >= 2) graph-replayed steps for each candidate launch shape
 * and keeps the fastest.  Candidates: 64, 128, 256 nodes per tile; schedule 0, strided (block b
 * takes tiles b, b + grid, ...), at 1/2x, 1x, 4x the resident blocks per SM or one block per tile;
 * schedule 1, contiguous (each block one run of consecutive tiles) and schedule 2, strided, both
 * prefetching the block's next tile into L2, at 1/2x, 1x, 4x.  out (optional, 4 doubles): best
 * MLUPS, nodes per tile, blocks per SM (0: one block per tile), schedule.  The trials advance
 * the state, so afterwards every domain is reset to rest: call it before lbm_batch_set_state. */
LBM_API lbm_status lbm_batch_autotune(lbm_batch* b, int trial_steps, double* out);

/* Sets the launch shape directly (a shape lbm_batch_autotune reported, for instance):
 * nodes_per_tile in {64, 128, 256}, 0 <= blocks_per_sm <= 64 (0: one block per tile), schedule 0
 * (strided), 1 (contiguous, prefetching) or 2 (strided, prefetching).  The state is not touched;
 * results do not depend on the shape. */
LBM_API lbm_status lbm_batch_set_shape(lbm_batch* b, int nodes_per_tile, int blocks_per_sm, int schedule);

/* Enqueues nsteps steps of every active domain. */
LBM_API lbm_status lbm_batch_step(lbm_batch* b, int nsteps);

/* Steps the active domains in graph-replayed chunks of check_every (even, >= 2) steps until each
 * reaches residual <= tol (after at least two checks), diverges, or max_steps elapse.  Per domain
 * (arrays of count, optional): steps[k] = steps taken at retirement (or at the end), residual[k]
 * = last residual, status[k] = 0 steady, 1 not steady after max_steps, 2 diverged (a NaN or
 * infinite residual: a domain whose fields hold a non-finite value is never reported steady). */
LBM_API lbm_status lbm_batch_run(lbm_batch* b, double tol, long long max_steps, int check_every, long long* steps,
                                 double* residual, int* status);

/* f = f^eq(rho, u) for domain k (arrays of N floats, host or device); needs even batch parity. */
LBM_API lbm_status lbm_batch_set_state(lbm_batch* b, int k, const float* rho, const float* ux, const float* uy,
                                       const float* uz);
/* rho, u (with F/2) of domain k; any output may be NULL; host or device; waits for the stream. */
LBM_API lbm_status lbm_batch_macroscopic(lbm_batch* b, int k, float* rho, float* ux, float* uy, float* uz);
/* Populations of domain k as FP32 deviations in natural order (27 * N floats, host or device). */
LBM_API lbm_status lbm_batch_get_populations(lbm_batch* b, int k, float* g);
LBM_API long long lbm_batch_nodes(const lbm_batch* b);
LBM_API long long lbm_batch_time(const lbm_batch* b);
LBM_API int lbm_batch_active(const lbm_batch* b);
LBM_API const char* lbm_batch_last_error(const lbm_batch* b);
LBM_API void lbm_batch_destroy(lbm_batch* b);

/* ------------------------------------------------------------------------------------------
 * Neural-operator warm start (no counterpart in the paper: a learned initial condition for the
 * steady solves of the batched solver; the plain CM-LBM run to the same residual judges it).
 * ------------------------------------------------------------------------------------------ */

/* BF16 tensor-core GEMM (tcgen05, FP32 accumulation), the contraction every layer of the neural
 * operator runs on:  C[b] = alpha * A[b] x B[b]  (beta != 0: C[b] += ...),  b < batch.
 * Element (m, k) of A[b] is at A + b*sab + m*sam + k*sak (BF16 elements), (k, n) of B at
 * B + b*sbb + k*sbk + n*sbn, (m, n) of C at C + b*scb + m*scm + n*scn (FP32, or BF16 with
 * out_bf16).  All pointers are device memory.  When A and B are 16-byte aligned with one unit
 * stride and the other strides multiples of 8 elements (K- or M/N-contiguous), the operands are
 * streamed by the tensor memory accelerator (persistent warp-specialised kernel; C written through
 * shared memory by the copy engine where C is row- or column-contiguous and aligned); any other
 * layout goes through a register-staged kernel.  Both give the same products up to FP32
 * summation order.  err is a device flag set to 1 if an internal bounded wait timed out, after
 * which C is undefined (MMAs committed before the timeout may still be writing it).  Enqueued on
 * stream; LBM_ERR_ARG on bad sizes. */
LBM_API lbm_status lbm_gemm_bf16(int M, int N, int K, int batch, const void* A, long long sam, long long sak,
                                 long long sab, const void* B, long long sbk, long long sbn, long long sbb, void* C,
                                 long long scm, long long scn, long long scb, int out_bf16, float alpha, int beta,
                                 unsigned int* err, void* stream);

/* 3D Fourier neural operator (FNO), predicting steady fields from inputs on a D^3 grid:
 *   h0 = P a + p;  h_{l+1} = act(K_l h_l + W_l h_l + b_l), act = GELU (identity on the last layer);
 *   out = Q h_L + q,
 * where K_l is the truncated spectral convolution: forward DFT over (z, y, x) without scaling,
 * modes |kz|, |ky| < m (both signs) and 0 <= kx < m, a learned complex width x width matrix per
 * mode, inverse DFT scaled by 1/D^3 taking the real part with kx > 0 counted twice (the inverse
 * of a real-to-complex transform).  Transforms and 1x1 maps run on lbm_gemm_bf16 (BF16 operands,
 * FP32 accumulation); parameters, gradients and Adam state are FP32.
 * Parameter vector (FP32): P[W][Ci], p[W], then per layer Wm[m][2m][2m][W][W][2] (kx, ky, kz,
 * out channel, in channel, re/im; ky and kz index the kept modes 0..m-1 then D-m..D-1),
 * Wc[W][W] (out, in), b[W]; then Q[Co][W], q[Co].  Tensors are [batch][channel][z][y][x] FP32. */
typedef struct lbm_no lbm_no;
/* D >= 4, 2 m <= D, W, L, Ci, Co, max_batch >= 1; parameters drawn from seed. */
LBM_API lbm_status lbm_no_create(int D, int width, int modes, int layers, int in_ch, int out_ch, int max_batch,
                                 unsigned long long seed, void* stream, lbm_no** out);
LBM_API long long lbm_no_param_count(const lbm_no* n);
/* Copies the parameter vector out of (set = 0) or into (set = 1) the model; host or device. */
LBM_API lbm_status lbm_no_params(lbm_no* n, float* params, int set);
/* Copies the gradient vector of the last lbm_no_backward / lbm_no_train_step; host or device. */
LBM_API lbm_status lbm_no_grads(lbm_no* n, float* grads);
/* out = model(in) for batch samples (device or host pointers); keeps the activations. */
LBM_API lbm_status lbm_no_forward(lbm_no* n, int batch, const float* in, float* out);
/* Gradient of sum(dout * out) of the last forward with respect to every parameter. */
LBM_API lbm_status lbm_no_backward(lbm_no* n, const float* dout);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the mean squared error over all outputs;
 * loss (optional, host) receives the loss before the step.  in, target: device or host pointers,
 * copied into the operator's buffers on its stream. */
LBM_API lbm_status lbm_no_train_step(lbm_no* n, int batch, const float* in, const float* target, float lr, double* loss);
/* enable != 0 (the default): from the second lbm_no_train_step on, the step (forward, loss,
 * backward, Adam) is captured once per batch size as a CUDA graph on a private stream and replayed,
 * ordered after the operator's stream by events; the inputs are first copied into the operator's
 * buffers.  The replayed kernels are the eager ones in the same order, so results are identical.
 * If a capture fails the operator trains eagerly from then on.  enable = 0: always eager. */
LBM_API lbm_status lbm_no_use_graphs(lbm_no* n, int enable);
/* A call that returns LBM_ERR_TIMEOUT (a tensor-core wait gave up) leaves the operator's outputs,
 * gradients, parameters and Adam state undefined: destroy it and create a new one. */
LBM_API const char* lbm_no_last_error(const lbm_no* n);
LBM_API void lbm_no_destroy(lbm_no* n);

/* Allocation-free FP64 diagnostics (the paper has no counterpart; this is a library service).
 * For callers that must not allocate device memory on their hot path -- a framework whose
 * caching allocator owns the device's memory budget, or a loop that cannot afford the implicit
 * device synchronisation of cudaMalloc/cudaFree.  It computes what lbm_stats computes, but over
 * fields the caller passes in, and it allocates nothing: its scratch is a fixed device array
 * inside the library (room for the partial sums of 1216 reduction blocks, about 88 KB, held by
 * every device that loads the library until the process exits).
 *   nx, ny, nz, walls_y: grid as in lbm_desc; N = nx*ny*nz must be < 2^31 (else LBM_ERR_ARG).
 *   mask: NULL or N device bytes, nonzero = solid (excluded).
 *   rho, ux, uy, uz: N device floats each (e.g. filled by lbm_macroscopic).
 *   uprev: NULL (residual = 1) or 3N device floats (ux, uy, uz blocks) of an earlier state.
 *   out: LBM_STATS_LEN - 1 doubles, host or device: entries [0..8] of the lbm_stats layout.
 *   stream: cudaStream_t (NULL = legacy default); the call waits for it before returning.
 * The first call on each device looks up the scratch array's device address (with that device
 * current); make that first call before any stream capture.  All calls on a device share the
 * one scratch array, so calls whose kernels overlap on the GPU (other streams, other threads)
 * race and must be serialised by the caller.  Every value it reads back is rewritten by the same
 * call, so nothing needs clearing between calls. */
LBM_API lbm_status lbm_reduce_fields_noalloc(int nx, int ny, int nz, int walls_y, const uint8_t* mask,
                                             const float* rho, const float* ux, const float* uy, const float* uz,
                                             const float* uprev, double* out, void* stream);

/* Frees everything the library allocated for ctx.  NULL is ignored.  Waits for the stream. */
LBM_API void lbm_destroy(lbm_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* CMLBM_H */
