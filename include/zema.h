/*
 * zema.h -- C ABI of the B300-native soft-rigid coupled IPC time step.
 *
 * The library advances a scene of tetrahedral soft bodies and 12-DOF affine
 * bodies by minimising, per time step, the barrier-augmented incremental
 * potential with lagged friction (paper section III: Eq. 1-11) with projected
 * Newton.  Every step of the Newton iteration runs in the library's CUDA
 * kernels on one GPU (sm_103a).
 *
 * Conventions for every entry point:
 *  - Return value: a zema_status; ZEMA_OK on success.  No C++ exception ever
 *    crosses this boundary.  zema_last_error() gives a message for the last
 *    failure on a scene.
 *  - Host arrays passed in are owned by the caller, read during the call and
 *    never retained.  Host arrays passed out are caller-allocated.
 *  - Arrays of 3-vectors are row-major (n x 3) doubles; index arrays int32.
 *  - A scene must not be used from two host threads at once.
 *  - Units are SI (m, kg, s).  Gravity comes from the scene parameters.
 *  - Affine state q = (p, a1, a2, a3), A = (a1, a2, a3)^T stored by rows; a
 *    rest vertex x0 maps to x = A x0 + p (Eq. 2).  The library works
 *    internally in a centre-of-mass frame and converts at the boundary.
 *  - Bodies in different environments (env) never interact; env ids are
 *    0 .. n_envs-1.
 *  - On a non-OK status from zema_step the state is left at the last
 *    completed time step.
 */
#ifndef ZEMA_H
#define ZEMA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ZEMA_OK = 0,
    ZEMA_ERR_INVALID_ARG = 1,
    ZEMA_ERR_OOM = 2,
    ZEMA_ERR_CUDA = 3,
    ZEMA_ERR_INTERSECTING_INPUT = 4,
    ZEMA_ERR_INVERTED_INPUT = 5,
    ZEMA_ERR_NEWTON_MAXITER = 6,
    ZEMA_ERR_LINESEARCH = 7,
    ZEMA_ERR_PCG_MAXITER = 8,    /* a linear solve reached max_pcg iterations without meeting
                                    pcg_rel_tol */
    ZEMA_ERR_NONFINITE = 9,
    ZEMA_ERR_FAULT_INJECTED = 10, /* a failure armed by zema_inject_fault */
    ZEMA_ERR_STATE = 11           /* call not allowed in the scene's current state */
} zema_status;

typedef struct zema_scene zema_scene; /* opaque; owns all of its device memory */

/* Device allocator hooks (optional).  alloc(bytes, stream, ctx) returns device
 * memory or NULL; free(ptr, stream, ctx) releases it.  When alloc is NULL the
 * library uses cudaMalloc / cudaFree. */
typedef void* (*zema_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*zema_free_fn)(void* ptr, void* stream, void* ctx);

typedef struct {
    double dt;             /* time step h (s) */
    double dhat;           /* barrier activation distance (m), Eq. 5 */
    double kappa;          /* barrier stiffness; <= 0 selects the adaptive rule */
    double eps_v;          /* friction velocity threshold (m/s), Eq. 10 */
    double newton_tol_rel; /* Newton stop: max |step| <= newton_tol_rel * bbox diagonal * dt */
    double gravity[3];     /* m/s^2 */
    double pcg_rel_tol;    /* PCG stop: |r| <= pcg_rel_tol * |b| */
    int32_t max_newton;    /* Newton iteration cap per solve */
    int32_t max_pcg;       /* PCG iteration cap per solve */
    int32_t max_al_rounds; /* kinematic augmented-Lagrangian rounds per env and step (each round
                              restarts the env's max_newton count) */
    int32_t precision;     /* 0: FP64 throughout; 1: mixed (FP32 Hessians, stored matrices,
                              preconditioner and PCG with FP64 residual refinement; FP64
                              gradients, energies, distances, ACCD and convergence test) */
    int32_t n_envs;        /* number of independent environments */
    int32_t warm_start;    /* 0: constant-velocity proposal; 1: learned proposal (needs weights) */
    int32_t pcg_kind;      /* 0: auto (one thread-block cluster per env when the env's vector fits
                              in shared memory, else the grid-wide solve); 1: grid-wide
                              cooperative solve; 2: cluster solve (zema_step returns
                              ZEMA_ERR_INVALID_ARG when the scene or device cannot run it) */
    void* stream;          /* cudaStream_t used for all work; NULL = legacy default stream */
    zema_alloc_fn alloc;   /* optional device allocator */
    zema_free_fn free;
    void* alloc_ctx;
    /* Schedule pins (0: chosen by the library).  Neither changes the method,
     * only the order of sums: with both pinned, an env's results depend on
     * that env alone, so a batch split into env ranges steps each env bit for
     * bit as the whole batch does. */
    double cell_size;      /* spatial-hash cell edge (m); <= 0: the mean surface edge length, at
                              least dhat */
    int32_t pcg_cluster_size; /* cluster schedule of the solve: CTAs per env (1, 2, 4, 8 or 16), plus 100
                                 for the two-CTAs-per-SM variant, or a size-binned code 1001, 1002, 1004,
                                 1101, 1102, 1104 (see zema_get_tuning); 0: about one CTA per 128 nodes
                                 or the autotuner's choice.  Any other value makes zema_create_scene
                                 return ZEMA_ERR_INVALID_ARG; a schedule the scene or device cannot run
                                 makes zema_step return it */
    int32_t al_extrapolate; /* 1 (default): each step starts the kinematic multipliers lambda_A of
                               Eq. 13 at 2 lambda^t - lambda^(t-1), the linear extrapolation of the
                               last two steps' converged values (the paper does not say how the
                               augmented-Lagrangian iteration starts; the rounds still run until
                               max |q - q~| <= tol, so the constraint met is the same); 0: each
                               step starts at lambda^t */
} zema_scene_params;

/* Per-step statistics (summed over the steps of one zema_step call, over all
 * environments; max for dmin-like fields as noted). */
typedef struct {
    int64_t steps;
    int64_t newton_iters;   /* applied Newton steps */
    int64_t pcg_iters;      /* PCG iterations over all solves */
    int64_t ls_halvings;    /* line-search halvings */
    int64_t al_rounds;      /* kinematic AL rounds: per step the largest count of any env */
    int64_t warm_accepted;  /* accepted warm-start proposals (per env step) */
    int64_t max_candidates; /* largest candidate-pair count seen in one broad phase */
    int64_t max_active;     /* largest active (d < dhat) pair count */
    double dmin;            /* smallest primitive distance after the last step (inf if none < dhat) */
    double kappa;           /* barrier stiffness of env 0 after the last step */
    double energy;          /* incremental potential of env 0 at the last converged iterate */
    double ms_phase[6];     /* host-timed phases: DCD, energy, Hessian, linear, CCD, other (ms) */
    int64_t pcg_refines;    /* FP64 residual-refinement correction solves of FP32 solves (mixed
                               precision), summed over envs */
    int64_t warm_learned;   /* accepted learned warm-start corrections (per env step) */
    int64_t warm_fallback;  /* steps redone from the constant-velocity start after Newton failed from the learned one */
} zema_step_stats;

/* Fills *p with defaults: dt 0.01, dhat 1e-3, adaptive kappa, eps_v 1e-3,
 * tol 1e-3, g = (0, -9.81, 0), pcg tol 1e-4, caps 100 / 10000 / 10, FP64,
 * one env, constant-velocity warm start, default stream and allocator. */
void zema_default_params(zema_scene_params* p);

/* Creates an empty scene.  Bodies are added next; the first zema_step (or
 * zema_finalize) builds the device data (scene precompute: surface
 * extraction, rest shapes, lumped and affine masses; Eq. 1, Eq. 2). */
zema_status zema_create_scene(const zema_scene_params* params, zema_scene** out);

/* Adds a tetrahedral soft body (Eq. 1, Neo-Hookean material).
 * X_rest: nv x 3 rest positions; tets: nt x 4 vertex indices, each tet
 * positively oriented (det[x1-x0, x2-x0, x3-x0] > 0, else
 * ZEMA_ERR_INVERTED_INPUT); x0, v0: nv x 3 initial positions / velocities,
 * NULL means X_rest / zero.  E (Pa), nu, rho (kg/m^3), mu_friction.  The
 * body id (shared numbering with affine bodies, in order of addition) is
 * written to *body_id. */
zema_status zema_add_tet_body(zema_scene* s, int32_t env, const double* X_rest, int64_t nv,
                              const int32_t* tets, int64_t nt, const double* x0, const double* v0,
                              double E, double nu, double rho, double mu_friction, int32_t* body_id);

/* Adds an affine body (Eq. 2): closed, outward-oriented triangle mesh
 * V_rest (nv x 3, caller's rest frame) / F (nf x 3); q0 and qdot0 (12 each,
 * qdot0 NULL = 0); density rho; stiffness = lambda of the orthogonality
 * energy; mode 0 dynamic, 1 fixed, 2 kinematic (driven to the target of
 * zema_set_kinematic_target by the augmented-Lagrangian term of Eq. 13).
 * ZEMA_ERR_INVALID_ARG when a face index is out of range, a face is
 * degenerate, the surface is not closed and consistently oriented (every
 * edge shared by two faces that traverse it in opposite directions), or its
 * signed volume is not positive (faces pointing inward); ZEMA_ERR_STATE after
 * the first step. */
zema_status zema_add_affine_body(zema_scene* s, int32_t env, const double* V_rest, int64_t nv,
                                 const int32_t* F, int64_t nf, const double q0[12], const double qdot0[12],
                                 double rho, double stiffness, double mu_friction, int32_t mode,
                                 int32_t* body_id);

/* Builds the device data now (optional; zema_step does it on first use).
 * Fails with ZEMA_ERR_INTERSECTING_INPUT when two primitives of the initial
 * state are at distance 0. */
zema_status zema_finalize(zema_scene* s);

/* Target q~ (12, caller's frame) of a kinematic affine body for the next
 * step (Eq. 13). */
zema_status zema_set_kinematic_target(zema_scene* s, int32_t body, const double q_target[12]);

/* The same for n kinematic bodies in one call (Eq. 13; the batched form of
 * the scripted grasps of the paper's parallel grasp generation): bodies (n
 * ids of affine bodies, each at most once) and q_targets (n x 12, caller's
 * frame, row k for bodies[k]), both host memory, read before the call
 * returns.  One host-to-device copy and one scatter on the scene's stream,
 * ordered before the next step; the call does not wait for them.
 * ZEMA_ERR_INVALID_ARG (nothing set) for a negative n, a NULL array with
 * n > 0, an id that is not an affine body, or a repeated id. */
zema_status zema_set_kinematic_targets(zema_scene* s, int64_t n, const int32_t* bodies, const double* q_targets);

/* Advances n_steps time steps (Eq. 11).  stats may be NULL.  Errors:
 * ZEMA_ERR_NEWTON_MAXITER (no convergence within max_newton iterations),
 * ZEMA_ERR_LINESEARCH (no energy decrease after 60 halvings),
 * ZEMA_ERR_PCG_MAXITER (a linear solve reached max_pcg iterations),
 * ZEMA_ERR_NONFINITE (a non-finite value in the linear solve),
 * ZEMA_ERR_FAULT_INJECTED (see zema_inject_fault),
 * ZEMA_ERR_INTERSECTING_INPUT (at the first step, as zema_finalize),
 * ZEMA_ERR_OOM, ZEMA_ERR_CUDA.  The state then stays at the last completed
 * step. */
zema_status zema_step(zema_scene* s, int32_t n_steps, zema_step_stats* stats);

/* State of one body into a caller-owned host buffer of cap doubles: the
 * quantities Eq. 11 advances, positions x^t and velocities v^t of a soft body
 * (Eq. 1), q^t and qdot^t of an affine body (Eq. 2).  Tet body: x then v
 * (nv x 3 each); affine body: q then qdot (12 each, the caller's frame, A by
 * rows).  *written (nullable) receives the number of doubles.  Before the
 * first step it returns the initial state given at add time.  A body id out
 * of range or cap too small: ZEMA_ERR_INVALID_ARG, buffer untouched.
 * Synchronises the scene's stream. */
zema_status zema_get_state(const zema_scene* s, int32_t body, double* out, int64_t cap, int64_t* written);

/* Sets the state (x^t, v^t or q^t, qdot^t of Eq. 11) of one body, same
 * layout as zema_get_state; n must equal the body's count exactly, else
 * ZEMA_ERR_INVALID_ARG with the state unchanged.  Before the first step it
 * replaces the initial state; afterwards the next step starts from it (the
 * caller is responsible for not creating intersections: nothing re-checks
 * them).  A fixed body's velocity is forced to zero.  Synchronises the
 * scene's stream. */
zema_status zema_set_state(zema_scene* s, int32_t body, const double* in, int64_t n);

/* The state of every body at once (Eq. 11's x^t, v^t, q^t, qdot^t): the
 * layouts of zema_get_state, bodies back to back in order of addition, n
 * doubles in all (zema_scene_state_size).  One copy each way through a
 * device buffer the scene owns; pinned host memory makes it a direct DMA.
 * Get: cap < n is ZEMA_ERR_INVALID_ARG (buffer untouched); set: n must equal
 * the size exactly, else ZEMA_ERR_INVALID_ARG with the state unchanged; a
 * fixed body's velocity is forced to zero, as with zema_set_state.  Both
 * synchronise the scene's stream; ZEMA_ERR_STATE before zema_finalize. */
zema_status zema_scene_state_size(const zema_scene* s, int64_t* n);
zema_status zema_get_scene_state(const zema_scene* s, double* out, int64_t cap, int64_t* written);
zema_status zema_set_scene_state(zema_scene* s, const double* in, int64_t n);

/* All positions/velocities at once, device-to-device: x_dev and v_dev are
 * device arrays of 3 * (total soft vertices) doubles in order of body
 * addition (either may be NULL). */
zema_status zema_copy_soft_state_device(const zema_scene* s, double* x_dev, double* v_dev);

/* Counts: [0] soft vertices, [1] tets, [2] affine bodies, [3] surface
 * vertices, [4] surface edges, [5] surface triangles, [6] nodes, [7] envs. */
zema_status zema_scene_counts(const zema_scene* s, int64_t out[8]);

/* Barrier stiffness kappa of an environment (after finalize). */
zema_status zema_get_kappa(const zema_scene* s, int32_t env, double* kappa);
/* Overrides kappa and kappa_min of an environment (disables the initial
 * gradient-balance rule for it). */
zema_status zema_set_kappa(zema_scene* s, int32_t env, double kappa, double kappa_min);

/* Whole-scene checkpoint (the time-stepping state of Eq. 11 with everything
 * else that carries over from one step to the next): node positions and
 * velocities x^t, v^t; the kinematic targets q~ and multipliers lambda_A of
 * Eq. 13 and the prismatic joints' multipliers; per env the barrier stiffness
 * kappa and kappa_min and the d_min of its doubling rule.  The scene's
 * definition (bodies, materials, springs, joints) is not part of it: load a
 * checkpoint only into a scene built by the same calls in the same order,
 * in either precision.  Stepping both scenes on then gives bit-identical
 * results (up to the autotuner's measured choice, see zema_autotune).
 * zema_checkpoint_size: bytes of a checkpoint of this scene (after
 * finalize; else ZEMA_ERR_STATE).  zema_save_checkpoint copies it into the
 * caller's host buffer of cap bytes (*written = its size; a smaller cap is
 * ZEMA_ERR_INVALID_ARG).  zema_load_checkpoint restores it; a header that does
 * not match the scene's node, affine-body, joint and env counts, a wrong
 * size or non-finite state is ZEMA_ERR_INVALID_ARG and leaves the scene
 * unchanged.  The buffer is the caller's; neither call retains it. */
zema_status zema_checkpoint_size(const zema_scene* s, int64_t* bytes);
zema_status zema_save_checkpoint(const zema_scene* s, void* buf, int64_t cap, int64_t* written);
zema_status zema_load_checkpoint(zema_scene* s, const void* buf, int64_t bytes);

/* Host-side fault injection for testing a caller's failure handling (the
 * paper has no counterpart).  Arms one failure at Newton iteration
 * newton_iter (0-based, counted over all Newton iterations of the next
 * zema_step call); it fires once and then disarms:
 *  ZEMA_FAULT_STATUS        a kernel reads the armed device flag and writes
 *                           ZEMA_ERR_FAULT_INJECTED into a device status word
 *                           that the host reads with the step-norm test;
 *  ZEMA_FAULT_SOLVE_NONFINITE a kernel reads the flag and marks the linear
 *                           solves of that iteration as having met a
 *                           non-finite value: ZEMA_ERR_NONFINITE;
 *  ZEMA_FAULT_NO_DECREASE   the line search of that iteration sees no trial
 *                           point lower the energy: ZEMA_ERR_LINESEARCH after
 *                           its 60 halvings.
 * zema_step then returns that status with the state at the last completed
 * step, as for a real failure.  ZEMA_FAULT_NONE disarms.  Nothing faults,
 * traps or hangs the GPU.  With the learned warm start, a no-decrease fault
 * in a step that started from the learned proposal is absorbed by its
 * fallback to the constant-velocity start. */
enum { ZEMA_FAULT_NONE = 0, ZEMA_FAULT_STATUS = 1, ZEMA_FAULT_SOLVE_NONFINITE = 2, ZEMA_FAULT_NO_DECREASE = 3 };
zema_status zema_inject_fault(zema_scene* s, int32_t kind, int32_t newton_iter);

/* Number of CUDA kernels the library has launched in this process (all
 * scenes and entry points); a benchmark reads it before and after a timed
 * region. */
long long zema_launch_count(void);

/* Live timing of one kernel for roofline reports: zema_profile_kernel(name)
 * selects the library kernel (by its function name, e.g. "k_pcg_cluster"; NULL
 * stops timing) and clears the totals; afterwards every launch of it is
 * bracketed by CUDA events on the stream it runs on.  zema_profile_read
 * returns the summed event time (ms), the number of timed launches and the
 * algorithmic bytes those launches declared (matrix, index and vector traffic
 * each launch must move at least once).  Synchronises the timed events. */
int zema_profile_kernel(const char* name);
int zema_profile_read(double* ms_total, long long* launches, double* alg_bytes);

/* Message of the last failed call on s (library-owned, valid until the next
 * call on s; "" if none; "null scene" for s == NULL).  It names the failing
 * step of the method, e.g. the Newton cap of the convergence test (config
 * Newton tolerance) or the line search of the minimisation of Eq. 11. */
const char* zema_last_error(const zema_scene* s);
/* Releases the scene and all device memory it owns (through the scene's
 * allocator hooks when given) after its stream's work completes.  NULL is a
 * no-op; s must not be used afterwards. */
void zema_destroy_scene(zema_scene* s);

/* ------------------------------------------------------------------------
 * Evaluation entry points used by parity tests and tools.  They run the same
 * device code as zema_step.
 * ------------------------------------------------------------------------ */

/* Prepares env state as at the start of a step (predictor, Eq. 1-3; lagged
 * friction, Eq. 9-10; kappa) without advancing, then evaluates the total
 * incremental potential B_t + D (Eq. 4, Eq. 11) at the current state.
 * energy: n_envs doubles.  grad (nullable): gradient in the caller's frame,
 * per body in order of addition: tet body 3 * nv, affine body 12 (dynamic and
 * kinematic bodies; fixed bodies contribute 12 zeros). */
zema_status zema_eval_energy_grad(zema_scene* s, int32_t apply_predictor, double* energy, double* grad);

/* Candidate pairs of a raw surface (spatial-hash broad phase, Table I "DCD"):
 * all PT (point, triangle) and EE (edge, edge) pairs whose axis-aligned boxes,
 * inflated by `inflate` per side, overlap -- swept over pos0 -> pos1 when pos1
 * is not NULL -- excluding pairs that share a vertex, pairs within one affine
 * body, pairs whose bodies are both fixed or kinematic, and cross-env pairs.
 * pos0/pos1: nsv x 3 host; sv_body: nsv; b_class (0 soft, 1 affine dynamic,
 * 2 fixed, 3 kinematic) and b_env: nb; edges ne x 2; tris nt x 3.  Outputs
 * (host, cap pairs each): pt_out (sv, tri) pairs, ee_out (edge, edge) with
 * first < second; n_out[0..1] = counts (may exceed cap: then outputs are
 * truncated).  cell_size <= 0 picks max(mean edge length, 2 * inflate). */
zema_status zema_candidates_raw(int64_t nsv, const double* pos0, const double* pos1, const int32_t* sv_body,
                                int64_t nb, const int32_t* b_class, const int32_t* b_env, int64_t ne,
                                const int32_t* edges, int64_t nt, const int32_t* tris, double inflate,
                                double cell_size, int64_t cap, int32_t* pt_out, int32_t* ee_out, int64_t* n_out,
                                void* stream);

/* zema_candidates_raw for callers that cannot allocate device memory (the
 * paper has no counterpart: it is a deployment variant of the broad phase).
 * Callers that draw all device memory from a pool fixed in advance, or must
 * not call an allocator inside a real-time loop, cannot use
 * zema_candidates_raw, which allocates scratch.  This entry point allocates
 * nothing: every scratch buffer lives in one file-scope device array of
 * 64 MiB that each GPU loading the library holds until the process exits.
 * It is not usable inside a CUDA stream capture: partway through, it
 * synchronises `stream` and reads counts back to the host to size the
 * following launches.
 *  - Inputs (pos0, pos1 nullable, sv_body, b_class, b_env, edges, tris) and
 *    outputs (pt_out, ee_out: cap pairs of int32 each) are DEVICE pointers;
 *    n_out (2 counts, may exceed cap: outputs then truncated) is host memory.
 *    Results equal zema_candidates_raw's, in the same order.
 *  - cell_size must be > 0 (no default: the default needs a reduction over
 *    host data).
 *  - Limits: nsv + ne + nt <= 65536, else ZEMA_ERR_INVALID_ARG; a scene whose
 *    grid entries and pair lists do not fit the 64 MiB array returns
 *    ZEMA_ERR_OOM.  Neither case writes the outputs or n_out.
 *  - The device index arrays are checked by a kernel before any other kernel
 *    indexes with them: a body id outside [0, nb), a body class outside
 *    [0, 3], a negative env or an edge or triangle vertex outside [0, nsv)
 *    returns ZEMA_ERR_INVALID_ARG with the outputs untouched.
 *  - The first call on a device resolves the array's device address
 *    (cudaGetSymbolAddress).
 *  - All calls share the one array and leave their contents in it; calls
 *    that overlap on the GPU (other streams or threads) race.  The call
 *    synchronises `stream` before returning, on every path. */
zema_status zema_candidates_raw_noalloc(int64_t nsv, const double* pos0, const double* pos1, const int32_t* sv_body,
                                        int64_t nb, const int32_t* b_class, const int32_t* b_env, int64_t ne,
                                        const int32_t* edges, int64_t nt, const int32_t* tris, double inflate,
                                        double cell_size, int64_t cap, int32_t* pt_out, int32_t* ee_out,
                                        int64_t* n_out, void* stream);

/* Batched local kernels on host arrays (n stencils):
 * barrier of PT (is_ee 0) or EE stencils x12 (n x 12): energy b (n), gradient
 * (n x 12) and PSD-projected Hessian (n x 144) of kappa * e * b(d) with
 * kappa = 1 (Eq. 5, Eq. 8); eps_x per stencil (EE mollifier). */
zema_status zema_local_barrier(int64_t n, const double* x12, const int32_t* is_ee, const double* eps_x,
                               double dhat, double* e_out, double* g_out, double* H_out, void* stream);
/* Squared distances and closest-point weights (n x 4) of stencils. */
zema_status zema_local_distance(int64_t n, const double* x12, const int32_t* is_ee, double* d2_out,
                                double* w_out, void* stream);
/* Neo-Hookean density Psi(F), F-space gradient (9) and PSD-projected Hessian
 * (81) of n deformation gradients F (row-major). */
zema_status zema_local_neo_hookean(int64_t n, const double* F9, double mu, double lam, double* psi_out,
                                   double* g_out, double* H_out, void* stream);
/* The same for any material: model 0 Neo-Hookean, 1 St. Venant-Kirchhoff,
 * 2 fixed corotated (zema_set_material); psi = +inf (and g, H untouched)
 * where the model is undefined (J <= 0 for 0 and 2). */
zema_status zema_local_elastic(int64_t n, const double* F9, double mu, double lam, int32_t model, double* psi_out,
                               double* g_out, double* H_out, void* stream);
/* Additive CCD step bound t in (0, 1] of n stencils moving by p12 (s = 0.1). */
zema_status zema_local_accd(int64_t n, const double* x12, const double* p12, const int32_t* is_ee,
                            double* t_out, void* stream);

/* Autotuner of the linear solve's launch schedule (the paper has no
 * counterpart).  The next solve of the scene times the cluster solve of that
 * step's system with every valid number of CTAs per environment (1, 2, 4, 8,
 * 16), in both residency variants (see zema_get_tuning; best of two runs
 * each, results discarded) and keeps the fastest for
 * the rest of the scene's life; that solve and every later one use it.  A
 * scene that is never tuned uses about one CTA per 128 nodes (at most 16)
 * and is bit-reproducible run to run; tuning picks by measured time, so two
 * tuned scenes may differ in rounding. */
zema_status zema_autotune(zema_scene* s);
/* The cluster schedule in use (0: not chosen yet, -1: grid-wide solve) for
 * precision 0 (FP64) or 1 (mixed), and the autotuner's measurements:
 * candidate schedules and solve times in ms (up to cap entries; *n =
 * count).  A schedule is the number of CTAs per env (1, 2, 4, 8, 16), plus
 * 100 for the variant that keeps two CTAs resident per SM (half the
 * registers per thread, matrix read through L1/L2).  Codes from 1000 are
 * size-binned: every env runs with m times the smallest cluster whose CTAs
 * hold its rows (at most 16; m = code % 100, 1, 2 or 4; plus 100 again for
 * two CTAs per SM), one launch per cluster size, each on a stream of its own
 * so that the sizes run at once.  The autotuner tries them all,
 * since with many envs of uneven sizes the solve is bound by how many
 * clusters run at once. */
zema_status zema_get_tuning(const zema_scene* s, int32_t precision, int32_t* cluster_size, int32_t* cand, float* ms,
                            int32_t cap, int32_t* n);

/* Learned Newton warm start (an addition to the method).  The network maps
 * 13 features of a soft vertex at the step's start to its predicted
 * displacement over the step, both scaled by s = h^2 |g| (the features:
 * position relative to the body centroid over the body's rest
 * half-diagonal; h v / s; (xhat - x) / s; nearest active pair distance over
 * dhat, capped at 1; that pair's unit normal pointing away from the other
 * primitive, or 0), and it predicts the displacement beyond the
 * constant-velocity one h v.  With params.warm_start = 1 the step first takes
 * the constant-velocity proposal x^t + alpha h v (CCD-bounded, kept only if
 * the energy does not rise), then the predicted correction of the soft
 * vertices the same way, kept only if it lowers the energy further; Newton
 * then runs to the same tolerance.  If Newton or its line search fails from
 * that start, the step is redone from x^t with the constant-velocity start
 * only, so the plain method decides every step the learned start cannot.
 *
 * A second network, per dynamic affine body, maps 40 features of the body
 * (the columns of A; the centre of mass relative to the env's initial
 * bounding-box centre over its diagonal; h qdot / s and (qhat - q) / s, the A
 * parts times the body's rest half-diagonal R; the nearest active pair
 * touching the body over dhat, capped at 1, and its normal pointing away from
 * the other primitive) to the change of q beyond h qdot in the same units
 * (12).  Its correction joins the soft vertices' in the same CCD-bounded,
 * energy-checked proposal.
 *
 * zema_load_warmstart: blob = uint32 magic 0x5357455A, uint32 n_layers,
 * uint32 dims[n_layers + 1], then the float32 parameters in the zema_mlp
 * layout.  dims[0] = 13 and dims[n_layers] = 3 load the per-vertex network;
 * dims[0] = 40 and dims[n_layers] = 12 the per-body network; any other shape
 * is ZEMA_ERR_INVALID_ARG.  The scene copies the blob. */
zema_status zema_load_warmstart(zema_scene* s, const void* blob, int64_t bytes);
/* Material of a tet body (paper Sec. "Constitutive Models"), before the
 * scene is finalized: 0 Neo-Hookean (the default; Psi = mu/2 (tr F^T F - 3) -
 * mu ln J + lam/2 (ln J)^2, +inf for J <= 0), 1 St. Venant-Kirchhoff
 * (Psi = mu E:E + lam/2 tr(E)^2 with E = (F^T F - I)/2, finite for every F),
 * 2 fixed corotated (Psi = mu |F - R|^2 + lam/2 (J - 1)^2, R the polar
 * rotation of F; +inf for J <= 0 so that R is a proper rotation).  The
 * F-space Hessians of 1 and 2 are PSD-projected by Jacobi rotations.  Other
 * models or a non-tet body: ZEMA_ERR_INVALID_ARG. */
zema_status zema_set_material(zema_scene* s, int32_t body, int32_t model);

/* Spring constraints (paper Sec. "Spring Constraints") on vertices of a tet
 * body: the term h^2 k |x_v - target_v|^2 per listed vertex (a potential
 * energy, scaled by h^2 like the elastic term, so k is in N/m and the spring
 * force is 2 k (x - target)).  verts: n body-local vertex indices; targets:
 * n x 3 positions; both copied.  Replaces the body's springs (n = 0 removes
 * them).  Allowed before or after finalize and between steps.  A non-tet
 * body, an index out of range, k < 0 or a non-finite value:
 * ZEMA_ERR_INVALID_ARG. */
zema_status zema_set_springs(zema_scene* s, int32_t body, const int32_t* verts, int64_t n, const double* targets,
                             double k);

/* Prismatic joint (paper Sec. "Joint Constraints") between two affine bodies
 * of one env, at least one of them dynamic, before the scene is finalized.
 * The joint keeps the bodies' relative orientation at its initial value and
 * lets body 2's copy of body 1's initial centre of mass move only along the
 * axis, a unit vector fixed in body 1 (`axis` in world coordinates at the
 * initial state).  It adds kappa |c|^2 - lambda . c to the incremental
 * potential with the 12-vector
 *   c = ( A1 B1 - A2 B2 ,  r x (A1 d1) ),
 * B_b the inverse of body b's initial A, d1 the axis in body 1's frame and r
 * the difference of the two bodies' images of the joint point; with both
 * initial A = I this is the paper's |A1 - A2|^2 + |((A1 c + p1) - (A2 c +
 * p2)) x (A1 d)|^2.  kappa <= 0 picks 1e3 x the mean of the two masses.
 * lambda starts at 0 and follows the augmented-Lagrangian rounds of the
 * kinematic bodies (lambda <- lambda - 2 kappa c while the rotation part
 * exceeds newton_tol_rel x dt or the slide part the Newton step
 * tolerance).  Its Hessian enters Newton as 2 kappa J^T J (Gauss-Newton,
 * PSD).  joint_id (nullable) receives the joint's index. */
zema_status zema_add_prismatic_joint(zema_scene* s, int32_t body1, int32_t body2, const double axis[3],
                                     double kappa, int32_t* joint_id);

/* Contact force sensing (paper Sec. "Contact Force Sensing"): for every body
 * (caller ids 0..n_bodies-1) the resultant barrier contact force at the
 * current state, forces[3 b .. 3 b + 2] = (1 / h^2) sum over the body's
 * surface vertices v of dB/dx_v, in newtons.  B is the barrier term of the
 * incremental potential (kappa e b(d) over the pairs with d < dhat, found by
 * a fresh broad phase at the current positions); the force the contacts
 * exert on the body is the negative of this vector.  Friction is not
 * included.  cap (doubles) below 3 n_bodies is ZEMA_ERR_INVALID_ARG. */
zema_status zema_contact_forces(zema_scene* s, double* forces, int64_t cap);

/* While recording, every following step writes the features of its soft
 * vertices (rows x 13) and their scaled displacement over the step (rows x 3)
 * into the caller's device buffers (rows = soft vertex count; the library's
 * node order: environments in order, bodies in the order they were added).
 * NULL / NULL stops.  cap_rows below the soft vertex count is an error. */
zema_status zema_record_warmstart(zema_scene* s, float* features, float* targets, int64_t cap_rows);
/* The same for the dynamic affine bodies: features (rows x 40) and the
 * scaled change of q beyond h qdot (rows x 12), rows = dynamic affine body
 * count in the library's order (environments in order, bodies in the order
 * they were added).  NULL / NULL stops; cap_rows below the count is an
 * error. */
zema_status zema_record_warmstart_affine(zema_scene* s, float* features, float* targets, int64_t cap_rows);

/* ------------------------------------------------------------------------
 * Small MLPs for the learned Newton warm start (the paper has no learned
 * component; this is an addition to the method).  A network maps
 * dims[0] -> dims[1] -> ... -> dims[n_layers] with ReLU after every layer but
 * the last.  Parameters are FP32 master copies, laid out layer by layer as
 * W_l (dims[l] x dims[l+1], row-major) followed by b_l (dims[l+1]); products
 * run on the tensor cores with BF16 operands and FP32 accumulation.  All
 * x / y / t pointers are device pointers (row-major, n rows); the network
 * owns its device memory.  Every call is stream-ordered on `stream` and
 * returns after its work completed.  Training is bit-reproducible (all
 * reductions in a fixed order).
 * ------------------------------------------------------------------------ */
typedef struct zema_mlp zema_mlp;
/* dims: n_layers + 1 widths (1..4096), n_layers 1..16 (else
 * ZEMA_ERR_INVALID_ARG); weights He-uniform from a SplitMix64 stream seeded
 * with `seed`, biases zero.  ZEMA_ERR_OOM when device memory runs out,
 * ZEMA_ERR_CUDA on any other CUDA failure (no device included); *out is
 * written only on success. */
zema_status zema_mlp_create(const int32_t* dims, int32_t n_layers, uint64_t seed, void* stream, zema_mlp** out);
void zema_mlp_destroy(zema_mlp* m);
zema_status zema_mlp_n_params(const zema_mlp* m, int64_t* n);
/* copies the FP32 parameters to / from host memory (cap / n = n_params) */
zema_status zema_mlp_get_params(const zema_mlp* m, float* host_out, int64_t cap);
zema_status zema_mlp_set_params(zema_mlp* m, const float* host_in, int64_t n);
/* Tensor-core path of the forward products: 0 (default) the fifth-generation
 * tensor cores (tcgen05.mma, accumulators in tensor memory) for layers with
 * dims[l] <= 128 and dims[l+1] <= 256, 1 the warp-level mma.sync kernel.
 * Backward products always use the warp-level kernel.  A tcgen05 product
 * whose completion wait times out makes the call return ZEMA_ERR_CUDA. */
zema_status zema_mlp_set_kernel(zema_mlp* m, int32_t kind);
/* y = net(x) */
zema_status zema_mlp_forward(zema_mlp* m, const float* x, int64_t n, float* y);
/* mean squared error of net(x) against t (mean over all n x dims[L]
 * entries) and its gradient with respect to the parameters (to host) */
zema_status zema_mlp_gradient(zema_mlp* m, const float* x, const float* t, int64_t n, float* grad_host, int64_t cap,
                              double* loss);
/* one AdamW step (decoupled weight decay) on the mean squared error of one batch */
zema_status zema_mlp_train_step(zema_mlp* m, const float* x, const float* t, int64_t n, float lr, float beta1,
                                float beta2, float eps, float weight_decay, double* loss);

#ifdef __cplusplus
}
#endif

#endif /* ZEMA_H */
