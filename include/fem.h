/*
 * fem.h -- C ABI of the B300 quasi-static tet-FEM indentation solver.
 *
 * The operation (Sec. III-A of Narang et al., "Sim-to-Real for Robotic Tactile
 * Sensing via Physics-Based Simulation and Learned Latent Projections"): a
 * volumetric tetrahedral mesh of a soft body with a per-element hyperelastic
 * law, fixed boundary conditions on some nodes, and a rigid indenter driven
 * into it; the simulator returns nodal displacements (positions) and nodal
 * contact forces, from which resultant forces are formed. Here the problem is
 * solved quasi-statically over prescribed load steps: at step k the indenter
 * sits at origin + d_k * a and the displacement is a minimiser of
 *
 *   Pi(u) = sum_e V_e Psi(F_e) + sum_i k_i/2 min(0, phi(X_i + u_i))^2,
 *   Psi(F) = mu/2 (tr F^T F - 3) - mu ln J + lam/2 (ln J)^2   (neo-Hookean),
 *   k_i = c_kappa * E_max,i * A_i / h_bar  (boundary node i, not fully fixed),
 *
 * with u = prescribed values on fixed DOFs. Convergence of a load step:
 * ||R_free||_2 <= tol * max(||f_c||_2, E_max * h_bar^2 * 1e-3), where R is the
 * FP64 gradient of Pi and f_c the nodal contact forces.
 *
 * Conventions for every entry point:
 *   - Return 0 (FEM_OK) on success, a negative FEM_ERR_* code on failure;
 *     fem_last_error() then holds a thread-local message.
 *   - The caller owns every array it passes. Inputs are copied; outputs are
 *     written into caller-allocated arrays. Output pointers may point to host
 *     memory (pageable or pinned) or to device memory of the current device;
 *     the library copies with cudaMemcpyDefault.
 *   - Units are the caller's (the library is unit-agnostic); the workloads use
 *     mm, N, MPa.
 *   - Node and tet indices are 0-based int32. Arrays are row-major.
 *   - Nothing here falls back to the CPU: without a CUDA device every entry
 *     point that touches the device returns FEM_ERR_CUDA.
 */
#ifndef FEM_B300_FEM_H
#define FEM_B300_FEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define FEM_OK                  0
#define FEM_ERR_ARG            -1   /* bad pointer, size, index or option */
#define FEM_ERR_DEGENERATE_TET -2   /* tet volume <= 1e-12 * (longest edge)^3, or inverted */
#define FEM_ERR_NONFINITE      -3   /* NaN/Inf in an input or in the FP64 residual */
#define FEM_ERR_OOM            -4   /* device or host allocation failed */
#define FEM_ERR_NOT_CONVERGED  -5   /* a load step hit max_newton or the line search failed;
                                       outputs hold the last iterate, stats are filled */
#define FEM_ERR_TIMEOUT        -6   /* a bounded device wait (grid barrier) expired */
#define FEM_ERR_CUDA           -7   /* a CUDA runtime call failed / no device */
#define FEM_ERR_BUSY           -9   /* request server: not running, or its admission queue is full */
#define FEM_PENDING             1   /* request server: the request has not finished yet */
#define FEM_ERR_TOO_LARGE      -8   /* mesh does not fit the single-solve kernel */
#define FEM_ERR_CHECK         -10   /* checked build (FEM_CHECKED) only: a kernel found an index
                                       of the mesh's device arrays out of range, or a NaN/Inf
                                       element force or stored tangent; the access was skipped,
                                       outputs are not to be trusted, the message names the check */

/* ---------------------------------------------------------------- shapes */
#define FEM_SPHERE   0   /* params[0] = radius; centre = pose origin                  */
#define FEM_CYLINDER 1   /* params[0] = radius; infinite, axis = third pose column    */
#define FEM_BOX      2   /* params[0..2] = half extents in the pose's local frame      */
#define FEM_PLANE    3   /* solid half-space behind the face through the origin whose  */
                         /* outward normal is the third pose column; no params         */

#define FEM_MAX_STEPS 256

/* tangent used inside the PCG */
#define FEM_TANGENT_PROJECTED 0  /* per-tet dP/dF eigenvalues clamped at 0               */
#define FEM_TANGENT_EXACT     1  /* exact dP/dF; PCG stops at negative curvature        */
#define FEM_TANGENT_ADAPTIVE  2  /* projected until the step's residual fell 100x, then */
                                 /* exact; back to projected on negative curvature or a */
                                 /* shortened line-search step (default)                */
#define FEM_TANGENT_ABS       3  /* negative eigenvalues replaced by their magnitude    */
/* The block-Jacobi preconditioner always uses the projected (PSD) blocks. */

typedef struct fem_mesh fem_mesh;           /* opaque; owns its device memory */

/* element laws (Sec. III-A: the paper's skin model is co-rotational linear elastic;
   its target data come from a Neo-Hookean model) */
#define FEM_MODEL_NEO_HOOKEAN 0  /* Psi = mu/2 (I1 - 3) - mu ln J + lam/2 (ln J)^2            */
#define FEM_MODEL_COROTATED   1  /* Psi = mu |F - R|^2 + lam/2 (tr(R^T F) - 3)^2, F = R S     */

typedef struct {
    double  E, nu;       /* Young's modulus, Poisson's ratio (Lame parameters mu, lam) */
    int32_t model;       /* FEM_MODEL_*                                               */
    int32_t reserved;    /* set to 0                                                  */
} fem_material;

typedef struct {
    double  c_kappa;          /* penalty factor (default 100)                         */
    int32_t max_newton;       /* Newton iterations per load step and friction pass (default 60) */
    int32_t max_cg;           /* PCG iterations per Newton iteration (default 2000)   */
    double  cg_rtol_max;      /* forcing term eta upper bound (default 0.2)           */
    double  cg_rtol_min;      /* forcing term eta lower bound (default 1e-2); Newton  */
                              /* stops on the FP64 residual whatever eta is            */
    int32_t max_backtracks;   /* Armijo halvings per Newton iteration (default 30)    */
    int32_t tangent;          /* FEM_TANGENT_* (default ADAPTIVE)                     */
    double  barrier_timeout_s;/* bound on every device-side wait (default 5 s)        */
    int32_t batch_engine;     /* fem_solve_batch: FEM_BATCH_AUTO (default),           */
                              /* FEM_BATCH_GROUPS or FEM_BATCH_CLUSTERS                */
    int32_t batch_parts;      /* CTAs per solve in fem_solve_batch, the same for all  */
                              /* solves (clusters: 1, 2, 4, 8 or 16); 0 = automatic:  */
                              /* groups get CTAs per solve from each mesh's size       */
                              /* (size classes), clusters from the largest mesh        */
    int32_t batch_tets_per_cta;/* automatic groups: target tets per CTA (default 1300) */
    int32_t precond_degree;   /* PCG preconditioner: 1 = block-Jacobi; d = 2..8:      */
                              /* Chebyshev polynomial of degree d in the block-Jacobi */
                              /* preconditioned tangent (d tangent products and one  */
                              /* reduction per PCG iteration; default 5)              */
    double  precond_ratio;    /* Chebyshev interval [4/ratio, 4] (default 120)         */
    double  dt;               /* load-step time step: 0 = quasi-static (default); > 0 */
                              /* = dynamic implicit stepping (backward Euler, lumped  */
                              /* mass): each load step of fem_solve, fem_solve_batch, */
                              /* fem_batch_run and the server is one time step of     */
                              /* length dt, starting from rest                         */
    double  density;          /* mass density for dt > 0, in the mesh's mass unit per */
                              /* unit volume (default 1.1e-9: 1100 kg/m^3 in t/mm^3   */
                              /* for coordinates in mm and moduli in MPa)             */
    double  mu_f;             /* Coulomb friction coefficient (default 0: frictionless)*/
                              /* Lagged and smoothed: at each load step the nodes'    */
                              /* normal forces and contact normals are frozen at the  */
                              /* step's start; the slip relative to the indenter's    */
                              /* translation carries the dissipation mu_f fn f0(|s|)  */
    double  friction_eps;     /* smoothing slip of f0, relative to the mesh's mean    */
                              /* edge length (default 0.01): below it a node sticks   */
                              /* elastically, above it it slides with force mu_f fn   */
    int32_t friction_passes;  /* solves per load step with friction, 1..64          */
                              /* (default 1). After each converged solve the normal   */
                              /* forces and normals are frozen again at the current   */
                              /* state, with the indenter at the step's own pose (the */
                              /* slip still counts from the step's start). The passes */
                              /* converge to friction that uses the step's own normal */
                              /* forces; newton_iters counts the iterations of all    */
                              /* passes                                                */
    int32_t tangent_fp16;     /* stored element tangent of the batched engines and the*/
                              /* request server: 0 = FP32, 30 floats per tet, as the  */
                              /* single-solve path (default 0); 1 = FP16, each value  */
                              /* over the tet's largest magnitude, with that scale in */
                              /* FP32 (64 bytes per tet instead of 128: half the bytes */
                              /* each tangent product streams; the tangent then      */
                              /* carries ~5e-4 relative rounding, which changes the   */
                              /* PCG path, not the FP64-residual stop). fem_solve and */
                              /* the single-pass diagnostics always use FP32          */
} fem_options;

/* engines of fem_solve_batch */
#define FEM_BATCH_AUTO     0
#define FEM_BATCH_GROUPS   1  /* cooperative launch of CTA groups, one solve per group;  */
                              /* parts sync through global memory (bounded waits)       */
#define FEM_BATCH_CLUSTERS 2  /* one thread-block cluster per solve; parts sync through */
                              /* distributed shared memory and cluster barriers         */

typedef struct {
    int32_t status;                         /* FEM_OK or the FEM_ERR_* of fem_solve    */
    int32_t steps_done;                     /* load steps that converged               */
    int32_t newton_iters;                   /* total Newton iterations                 */
    int32_t cg_iters;                       /* total PCG iterations                    */
    int32_t backtracks;                     /* total line-search halvings              */
    int32_t active_contacts;                /* nodes with phi < 0 at the last step     */
    double  residual;                       /* final ||R_free||_2                      */
    double  scale;                          /* final convergence scale                 */
    double  energy;                         /* final total energy Pi                   */
    double  kernel_ms;                      /* device time of the solve kernel          */
    int32_t exact_newton_iters;             /* Newton iterations on the exact tangent   */
    double  phase_ms[10];                   /* kernel time split (CTA 0 clock shares):
                                               eval (FP64 residual and energy passes),
                                               tangent (build + block-Jacobi), pcg init,
                                               pcg dot reductions, tangent products'
                                               element part (PCG and preconditioner),
                                               pcg and preconditioner vector updates,
                                               halo exchange waits, total, pcg scalars,
                                               tangent products' node gathers.
                                               fem_solve_batch: fractions of that
                                               solve's own time instead                */
    double  phase_max_ms[10];               /* the same phases, largest over CTAs       */
    double  phase_min_ms[10];               /* the same phases, smallest over CTAs      */
                                            /* (both 0 in fem_solve_batch)              */
    int32_t newton_per_step[FEM_MAX_STEPS];
    int32_t cg_per_step[FEM_MAX_STEPS];
    double  residual_per_step[FEM_MAX_STEPS];
    int64_t tangent_products;               /* element-tangent products (PCG and     */
                                            /* preconditioner) of the whole solve    */
    double  step_end_ms[FEM_MAX_STEPS];     /* device time from the solve's start to */
                                            /* the end of each load step (global     */
                                            /* timer of the solve's first CTA): the  */
                                            /* per-step timeline inside the one      */
                                            /* persistent launch                     */
} fem_stats;

typedef struct {
    int64_t n_nodes, n_tets;
    int32_t n_parts;            /* mesh partitions = CTAs of the solve kernel             */
    int64_t part_tets;          /* tets over all partitions (halo tets counted per part)  */
    int32_t max_owned_nodes, max_local_nodes, max_part_tets;
    int32_t smem_bytes;         /* dynamic shared memory per CTA                          */
    int32_t resident;           /* 1: part tangent and connectivity kept in shared memory */
    double  h_bar;              /* mean unique-edge length                                 */
    double  scale_floor;        /* E_max * h_bar^2 * 1e-3                                  */
    int64_t n_candidates;       /* contact candidate nodes                                 */
    int64_t device_bytes;       /* device memory owned by the mesh                         */
} fem_mesh_info;

/* Fill *opt with the defaults listed above. */
void fem_default_options(fem_options* opt);

/*
 * Upload a mesh (Sec. III-A: volumetric tet mesh, materials, fixed BCs).
 *   nodes        [n_nodes*3] reference coordinates.
 *   tets         [n_tets*4] node indices, positively oriented (V > 0).
 *   tet_material [n_tets] index into materials (NULL: all 0).
 *   materials    [n_materials] (E > 0, -1 < nu < 0.5).
 *   fixed_nodes  [n_fixed] nodes with prescribed displacement (default 0).
 *   fixed_mask   [n_fixed] bit0=x bit1=y bit2=z prescribed, or NULL for xyz.
 *   cuda_stream  cudaStream_t for every copy and launch on this mesh (NULL =
 *                the legacy default stream).
 *   out          receives the handle; destroy it with fem_destroy_mesh.
 * Errors: FEM_ERR_ARG (bad sizes/indices), FEM_ERR_NONFINITE (coordinates or
 * material), FEM_ERR_DEGENERATE_TET, FEM_ERR_TOO_LARGE, FEM_ERR_OOM, FEM_ERR_CUDA.
 * Validation happens on the host before any CUDA call.
 */
int fem_create_mesh(const double* nodes, int64_t n_nodes,
                    const int32_t* tets, int64_t n_tets,
                    const int32_t* tet_material, const fem_material* materials,
                    int32_t n_materials,
                    const int32_t* fixed_nodes, int64_t n_fixed,
                    const uint8_t* fixed_mask,
                    void* cuda_stream, fem_mesh** out);

/*
 * Set the rigid indenter (Sec. III-A: rigid objects driven into the sensor).
 *   shape          FEM_SPHERE / FEM_CYLINDER / FEM_BOX / FEM_PLANE.
 *   pose           [12] origin(3) followed by a 3x3 rotation, row-major, whose
 *                  columns are the indenter's local axes (orthonormal, det +1).
 *   params         [3] shape parameters (see FEM_* above); may be NULL for PLANE.
 *   dir            [3] unit approach direction a.
 *   depth_schedule [n_steps] depths d_k along a, measured from the pose (the
 *                  pose is the position of initial contact); 1 <= n_steps <=
 *                  FEM_MAX_STEPS.
 * Errors: FEM_ERR_ARG, FEM_ERR_NONFINITE.
 */
int fem_set_indenter(fem_mesh* mesh, int shape, const double pose[12],
                     const double* params, const double dir[3],
                     const double* depth_schedule, int32_t n_steps);

/*
 * Prescribed displacements on the fixed DOFs (default: zero). values has
 * [n_fixed*3] entries in fixed_nodes order; components not flagged by the
 * node's fixed_mask are ignored. The values are ramped over the load steps:
 * at step k the fixed DOFs hold values * k / K. NULL resets to zero.
 */
int fem_set_dirichlet_values(fem_mesh* mesh, const double* values);

/*
 * Solve the load steps (the hot path: FP64 residual and energy, FP32
 * PSD-projected element tangent, block-Jacobi pipelined PCG with FP64
 * reductions, Armijo line search with a J > 0 guard, FP64 displacement update),
 * all inside one cooperative persistent kernel launched on the mesh's stream.
 *   load_steps         must equal the schedule length, or 0 for all of it.
 *   tol                relative residual tolerance (e.g. 1e-6).
 *   opt                NULL for defaults.
 *   out_disp           [n_nodes*3] displacement after the last solved step.
 *   out_contact_force  [load_steps*3] resultant contact force on the body per
 *                      step, or NULL.
 *   out_nodal_contact  [n_nodes*3] nodal contact forces at the last step, or NULL.
 *   stats              filled when non-NULL.
 * Synchronises the mesh's stream before returning.
 * Errors: FEM_ERR_ARG, FEM_ERR_NOT_CONVERGED (outputs = last iterate),
 * FEM_ERR_NONFINITE, FEM_ERR_TIMEOUT, FEM_ERR_CUDA.
 */
int fem_solve(fem_mesh* mesh, int32_t load_steps, double tol, const fem_options* opt,
              double* out_disp, double* out_contact_force, double* out_nodal_contact,
              fem_stats* stats);

/*
 * Checkpoint and resume: solve load steps first_step..last_step (1-based,
 * inclusive) of the schedule set by fem_set_indenter, starting from a saved
 * state. The state of a solve after load step k is the pair of converged
 * displacements (u_k, u_{k-1}): the secant predictor of step k+1 and, for
 * dt > 0, the velocity (u_k - u_{k-1}) / dt come from it, and friction is
 * frozen from u_k. A solve split into ranges, each resumed from the state the
 * previous one returned, gives bitwise the results of one fem_solve.
 *   u0, u0_prev    [n_nodes*3] u_{first_step-1} and u_{first_step-2} (caller
 *                  node order, host or device). Both NULL for first_step = 1
 *                  (from rest); u0_prev NULL means u0_prev = u0.
 *   out_disp       [n_nodes*3] u of the last solved step (as fem_solve).
 *   out_prev_disp  [n_nodes*3] u of the step before it, or NULL: with out_disp
 *                  the state to resume the next range from.
 *   out_contact_force [n_steps*3] of the whole schedule; rows of steps outside
 *                  the range are zero. out_nodal_contact and stats as fem_solve
 *                  (steps_done is the last converged step of the schedule; the
 *                  per-step arrays are filled for the range's steps).
 * The saved state is the caller's; nothing persists in the mesh between calls
 * but the mesh itself. Errors: FEM_ERR_ARG (range outside the schedule, a range
 * after step 1 without u0) and those of fem_solve.
 */
int fem_solve_range(fem_mesh* mesh, int32_t first_step, int32_t last_step, const double* u0,
                    const double* u0_prev, double tol, const fem_options* opt, double* out_disp,
                    double* out_prev_disp, double* out_contact_force, double* out_nodal_contact,
                    fem_stats* stats);

/* One indenter of a batched solve (same meaning as fem_set_indenter's arguments). */
typedef struct {
    int32_t       shape;            /* FEM_SPHERE / FEM_CYLINDER / FEM_BOX / FEM_PLANE      */
    double        pose[12];         /* origin(3) + rotation (row-major, columns = axes)     */
    double        params[3];        /* radius | radius | half extents | unused              */
    double        dir[3];           /* unit approach direction                              */
    const double* depth_schedule;   /* [n_steps] host or device, depths from the pose       */
    int32_t       n_steps;          /* 1..FEM_MAX_STEPS                                     */
} fem_indenter;

/*
 * Solve n independent indentations in one launch (batched form of fem_solve;
 * Sec. III-A's indentations of one sensor, or of several meshes). Solve i uses
 * meshes[i] (the same handle may appear any number of times; all meshes must be
 * on the current device) and indenters[i]; prescribed values set with
 * fem_set_dirichlet_values are not used here (fixed DOFs are held at 0).
 * A slot of opt->batch_parts CTAs runs one solve (each mesh is cut into that
 * many parts, once per part count) and takes the next job from a queue when
 * done, so uneven meshes share the launch; the slots are CTA groups of one
 * cooperative launch (FEM_BATCH_GROUPS, the default) or thread-block clusters
 * (FEM_BATCH_CLUSTERS). A solve's result is bitwise independent of the other
 * jobs and of which slot ran it. The launch goes to meshes[0]'s stream; the
 * call synchronises it. The workspace (per solve ~56 B per node; per slot
 * ~110 B per node and 128 B per part tet of the largest mesh) is allocated
 * stream-ordered for the call and released before it returns.
 *   out_disp[i]           [n_nodes(i)*3] displacement after the last step.
 *   out_contact_force[i]  [n_steps(i)*3] resultant contact force per step (or
 *                         out_contact_force == NULL).
 *   stats[i]              per-solve statistics (or stats == NULL); kernel_ms is
 *                         the whole launch.
 * Returns FEM_OK if every solve converged, else the first solve's error code
 * (each stats[i].status holds its own; FEM_ERR_TIMEOUT for a solve whose
 * group abandoned a bounded wait, or that never started because of it).
 * FEM_ERR_TOO_LARGE if a part of the largest mesh does not fit one CTA or no
 * slot of that size fits the GPU.
 */
int fem_solve_batch(fem_mesh* const* meshes, const fem_indenter* indenters, int32_t n, double tol,
                    const fem_options* opt, double* const* out_disp, double* const* out_contact_force,
                    fem_stats* stats);

/*
 * Reusable batch plan: the batched solve of fem_solve_batch split into a
 * planning call and repeatable runs. fem_batch_create fixes the meshes, the
 * load-step count of each solve and the options (engine, part count, solver
 * settings); it builds the partitions, allocates the device workspace and
 * pinned staging, and captures the whole batch (workspace reset, upload of the
 * job table and schedules, the persistent launch, reordering of the outputs)
 * as a CUDA graph. Errors: as fem_solve_batch's planning (FEM_ERR_ARG,
 * FEM_ERR_TOO_LARGE, FEM_ERR_OOM, FEM_ERR_CUDA).
 */
typedef struct fem_batch fem_batch;
int fem_batch_create(fem_mesh* const* meshes, const int32_t* n_steps, int32_t n, const fem_options* opt,
                     fem_batch** out);

/*
 * One run of the plan: indenters[i] (n_steps must match the plan) at residual
 * tolerance tol; outputs and return value as fem_solve_batch (kernel_ms: the
 * replayed graph). Runs of one plan must not overlap (each run waits for the
 * GPU before it returns). Work queued earlier on meshes[0]'s stream completes
 * before the run starts.
 */
int fem_batch_run(fem_batch* batch, const fem_indenter* indenters, double tol, double* const* out_disp,
                  double* const* out_contact_force, fem_stats* stats);

typedef struct {
    int32_t engine;                 /* FEM_BATCH_GROUPS or FEM_BATCH_CLUSTERS        */
    int32_t parts;                  /* CTAs per solve                                */
    int32_t slots;                  /* solves in flight at once                      */
    int32_t graph;                  /* 1: runs replay a captured CUDA graph          */
    int32_t smem_bytes;             /* dynamic shared memory per CTA                 */
    int32_t global_bytes_per_cta;   /* per-CTA arrays that did not fit on chip        */
    int32_t resident_tangent;       /* 1: part tangents live in shared memory        */
    int64_t workspace_bytes;        /* device workspace of the plan                  */
} fem_batch_info;
int fem_batch_info_get(const fem_batch* batch, fem_batch_info* info);

/*
 * Autotuner of fem_solve_batch's slot shape: times candidate (engine, CTAs per
 * solve) pairs on the given jobs truncated to their first proxy_steps load
 * steps (one planned run each) and writes opt (NULL = defaults) with the
 * fastest batch_engine / batch_parts / batch_tets_per_cta to out_opt.
 * Candidates: CTA groups in size classes of 700, 1000, 1300, 1800, 2600 or
 * 3600 tets per CTA; uniform CTA groups with 1, 2, 4 or 8 groups sharing the SMs;
 * clusters of 8 or 16 CTAs. report (may be NULL) lists every candidate's proxy
 * rate (solves/s; 0 = did not fit or did not run) and the index of the best. Errors:
 * FEM_ERR_ARG, FEM_ERR_TOO_LARGE (no candidate runs), FEM_ERR_CUDA.
 */
typedef struct {
    int32_t n_candidates;
    int32_t engine[16];
    int32_t parts[16];              /* 0: size classes                               */
    int32_t tets_per_cta[16];       /* size classes: target tets per CTA             */
    double  rate[16];
    int32_t best;
} fem_tune_report;
int fem_batch_tune(fem_mesh* const* meshes, const fem_indenter* indenters, int32_t n, double tol,
                   const fem_options* opt, int32_t proxy_steps, fem_options* out_opt, fem_tune_report* report);

/* ------------------------------------------------------- request server
 * Continuous batching of indentation solves on a resident pool of meshes.
 * One persistent launch holds CTA groups in size classes (a mesh's class is
 * the smallest power of two up to opt->batch_parts, or 64, CTAs that keeps its
 * parts near opt->batch_tets_per_cta tets; one group per class, the remaining
 * SMs going one group at a time to the class with the most work per CTA when
 * requests are spread evenly over the pool). A host thread admits submitted
 * requests while result memory is free, publishes them to the GPU through
 * pinned host memory and collects the results; a request that arrives while
 * others run starts as soon as a group of its class is idle. Meshes with more
 * than 64 x batch_tets_per_cta tets are served by other launch shapes of the
 * persistent kernel. Shape 1 keeps as many groups of the largest size class as
 * leave at least half of the SMs and makes one group of the other SMs for the
 * "large" meshes, those whose parts at that count stay within
 * batch_tets_per_cta tets; shape 2 is one group of every SM for the larger
 * ("huge") meshes; each such mesh is always cut into its group's number of
 * parts. The host changes the shape first come, first served: when the oldest
 * unfinished request the live shape does not serve is older than every
 * unfinished request that only the live shape (of the two) serves, the running
 * solves leave at their next load-step boundary, the kernel is relaunched in
 * the shape that serves the waiting request, and the suspended solves resume
 * from their own state (the converged displacements of their last two steps,
 * kept in their result slot); it returns to shape 0 once nothing needs the
 * other shape. A request's result is bitwise independent of the others, of
 * the shape it ran in and of any suspension (its partition depends only on its
 * mesh; a resumed solve continues bitwise as if it had not been interrupted).
 */
typedef struct fem_server fem_server;

/* meshes: the resident pool (handles stay owned by the caller and must outlive
 * the server); max_steps: most load steps of any request; result_bytes: device
 * memory for results in flight (one result slot ~ 72 B per node of the largest
 * mesh + 32 B per step; at least one slot per group). Errors: FEM_ERR_ARG,
 * FEM_ERR_TOO_LARGE, FEM_ERR_OOM, FEM_ERR_CUDA. */
int fem_server_create(fem_mesh* const* meshes, int32_t n_meshes, int32_t max_steps, const fem_options* opt,
                      int64_t result_bytes, fem_server** out);

/* Launch the persistent kernel; it serves until fem_server_stop or for at most
 * max_seconds (groups leave once idle after that). */
int fem_server_start(fem_server* server, double max_seconds);

/* Queue one request (mesh = index into the pool); never blocks. *request_id
 * identifies it. FEM_ERR_BUSY if the server is not running or 4 x result-slot
 * requests already wait for admission (the request is rejected). */
int fem_server_submit(fem_server* server, int32_t mesh, const fem_indenter* indenter, double tol,
                      int64_t* request_id);

/* Wait up to wait_ms for a request. FEM_PENDING if it has not finished yet;
 * otherwise the request's status (as fem_solve) with out_disp [n_nodes*3]
 * (caller order), out_contact_force [n_steps*3], stats (kernel_ms: time from
 * admission to completion) and times [3] = (submitted, admitted, done) in
 * seconds of a monotonic host clock filled (each may be NULL); the request is
 * then forgotten. */
int fem_server_result(fem_server* server, int64_t request_id, int32_t wait_ms, double* out_disp,
                      double* out_contact_force, fem_stats* stats, double* times);

/* Stop serving: idle groups leave at once, busy ones after their solve;
 * requests not run finish with FEM_ERR_TIMEOUT. */
int fem_server_stop(fem_server* server);

typedef struct {
    int32_t n_classes;
    int32_t class_parts[8];         /* CTAs per solve of each size class */
    int32_t class_groups[8];        /* groups serving each class         */
    int32_t n_ctas;                 /* CTAs of the persistent launch      */
    int32_t result_slots;           /* requests in flight at most         */
    int64_t admitted, completed, rejected;
    int64_t workspace_bytes;
    int64_t suspended;              /* times a running solve left between load */
                                    /* steps for a change of launch shape and   */
                                    /* resumed after it                         */
    int64_t launches;               /* persistent launches: the first of each  */
                                    /* session and one per change of shape      */
    int32_t large_class;            /* class of the large meshes, -1 if none    */
    int32_t huge_class;             /* class of the huge meshes, -1 if none     */
    int32_t n_shapes;               /* launch shapes (1-3)                      */
    int32_t shape_ctas[3];          /* CTAs of each shape's launch              */
    int32_t shape_groups[3][8];     /* groups per class in each shape           */
} fem_server_info;
int fem_server_info_get(const fem_server* server, fem_server_info* info);

/* Stop (if running) and release the server (NULL is ignored). */
void fem_server_destroy(fem_server* server);

/* Release the plan (NULL is ignored). */
void fem_batch_destroy(fem_batch* batch);

/* Release the mesh and its device memory (NULL is ignored). */
void fem_destroy_mesh(fem_mesh* mesh);

/* Message of the last failing call on this thread ("" if none). */
const char* fem_last_error(void);

/*
 * 1 if this library was built with FEM_CHECKED, else 0. The checked build
 * (libfem_b300_checked.so; the Python binding loads it when the environment
 * sets FEM_B300_CHECKED=1) bounds every index its kernels read from the mesh's
 * device arrays and checks element forces and stored tangents for NaN/Inf; a
 * failed check skips the access and the entry point that ran the kernel
 * returns FEM_ERR_CHECK (fem_solve, the diagnostics, fem_batch_run,
 * fem_solve_batch; the request server reports it from fem_server_stop). It
 * stands in for a memory checker: the production build contains none of it.
 */
int fem_build_checked(void);

/* Sizes and derived constants of a mesh (partitioning, shared memory, h_bar). */
int fem_mesh_info_get(const fem_mesh* mesh, fem_mesh_info* info);

/*
 * Re-cut the mesh into n_parts partitions (one CTA of the solve kernel each;
 * the default is min(#SMs, n_nodes/48)). Used by the tile autotuner. Errors:
 * FEM_ERR_ARG, FEM_ERR_TOO_LARGE (more parts than co-resident CTAs, or a part
 * that does not fit in shared memory), FEM_ERR_OOM, FEM_ERR_CUDA.
 */
int fem_repartition(fem_mesh* mesh, int32_t n_parts);

/*
 * Element stress output (the paper's simulator reports element stress
 * tensors, Sec. III-A): Cauchy stress and von Mises equivalent stress of every
 * tet at displacement u [n_nodes*3] (caller node order, host or device), FP64.
 *   out_cauchy     [n_tets*6] per tet (xx, yy, zz, yz, xz, xy), caller tet order.
 *   out_von_mises  [n_tets] sqrt(3/2 s:s) of the deviator, or NULL.
 * Errors: FEM_ERR_ARG, FEM_ERR_OOM, FEM_ERR_CUDA.
 */
int fem_element_stress(fem_mesh* mesh, const double* u, double* out_cauchy, double* out_von_mises);

/* ------------------------------------------------------- diagnostics
 * Single passes of the hot-path kernels, for parity tests. They run the same
 * device code as fem_solve (same kernel, one phase) on a caller-supplied
 * displacement. */

/*
 * FP64 residual at displacement u and load step `step` (1-based; 0 = the pose
 * itself): out_R [n_nodes*3] = dPi/du (fixed DOFs included, not zeroed),
 * out_fc [n_nodes*3] nodal contact forces on the body (may be NULL),
 * out_energy [2] = (elastic energy, contact energy) (may be NULL).
 * c_kappa from opt (NULL = default). Host or device pointers.
 */
int fem_eval_residual(fem_mesh* mesh, const double* u, int32_t step, const fem_options* opt,
                      double* out_R, double* out_fc, double* out_energy);

/*
 * Allocation-free variant of fem_eval_residual (the paper has no counterpart:
 * this is a service of the library). Same arguments, outputs and errors; the
 * evaluation runs the same kernel, but every device buffer it needs apart from
 * the mesh itself comes from a fixed 8 MiB block of device memory that the
 * library keeps in its own module (present on each GPU that loads the library,
 * until the process exits), so the call itself never calls cudaMalloc,
 * cudaFree or any allocating routine. It is meant for callers that may not
 * allocate device memory once they are running: a real-time control loop with
 * a no-allocation rule after start-up, a host application that hands out all
 * device memory from its own pool, or a process already at its memory budget.
 *   - Limit: the block must hold 4 x 3 doubles per node, the per-part
 *     reduction slots and, for meshes whose parts do not fit in shared memory,
 *     the per-CTA arrays placed in global memory; about 87,000 nodes is the
 *     upper bound (reached when the parts fit on chip), and the real limit
 *     depends on the mesh's partition layout. Larger meshes return
 *     FEM_ERR_TOO_LARGE with the sizes and the node limit for that layout in
 *     the message.
 *   - The call runs on the mesh's device (made current for the call, the
 *     caller's current device restored afterwards). The first call on each
 *     device looks up the block's device address (with that device current)
 *     and caches it; make that first call before any stream capture.
 *   - All calls share the one block and each call overwrites it (the words that
 *     must start at zero are cleared at the start of every call). Calls that can
 *     overlap on the GPU (other streams, other host threads) race: serialise them.
 *   - The call also reuses the mesh's own per-tet force scratch, the one that
 *     fem_solve, fem_eval_residual and fem_apply_tangent use: it must not
 *     overlap any of those on the same mesh from another host thread (calls on
 *     the mesh's stream from one thread are ordered and safe).
 */
int fem_eval_residual_noalloc(fem_mesh* mesh, const double* u, int32_t step, const fem_options* opt,
                              double* out_R, double* out_fc, double* out_energy);

/*
 * FP32 tangent product y = K(u) p at displacement u and step `step`: element
 * part from the stored per-tet tangent (projected or exact per opt->tangent)
 * plus the Gauss-Newton contact term, rows and columns of fixed DOFs zeroed.
 * p and out_y are [n_nodes*3] FP64 (p is rounded to FP32 on the device).
 */
int fem_apply_tangent(fem_mesh* mesh, const double* u, int32_t step, const fem_options* opt,
                      const double* p, double* out_y);

/*
 * Self-check of the PCG's dot products (Sec. III-A's Newton solver needs the
 * inner linear solves; these are their reductions): (r,u), (w,u) and (r,r)
 * over the free DOFs of the mesh, with r, u, w [n_nodes*3] (host or device,
 * caller node order) rounded to FP32 as the PCG holds its vectors, summed by
 * the same device code as every PCG iteration of fem_solve: error-free FP32
 * products, compensated FP32-pair sums per CTA and over the CTAs in a fixed
 * order. out[3] receives the three sums (each pair's hi + lo as a double). The
 * mesh's evaluation buffers are overwritten. Errors: FEM_ERR_ARG, FEM_ERR_CUDA,
 * FEM_ERR_TIMEOUT.
 */
int fem_debug_pcg_dots(fem_mesh* mesh, const double* r, const double* u, const double* w, double out[3]);

/*
 * Failure-detection check: launch the solve kernel's grid barrier with one CTA
 * that never arrives, bounded by timeout_s (e.g. 0.05). The waiting CTAs give
 * up, set the device error word and return; the call returns FEM_ERR_TIMEOUT
 * and the CUDA context stays usable. Returns FEM_OK only if the barrier
 * (wrongly) completed.
 */
int fem_debug_barrier_timeout(double timeout_s);

/*
 * Self-check of the FP64 reciprocal and reciprocal square root that the element
 * kernels use instead of FP64 division and square root (FP32 hardware value
 * refined by one Newton-Raphson step): out_rcp[i] = 1/x[i], out_rsqrt[i] =
 * 1/sqrt(x[i]) as the kernels compute them, for n host values x with x and 1/x
 * in FP32's normal range (positive where out_rsqrt is asked for). out_rsqrt may
 * be NULL.
 * FEM_ERR_ARG on NULL x/out_rcp or n < 1; FEM_ERR_CUDA without a device.
 */
int fem_debug_reciprocals(const double* x, int64_t n, double* out_rcp, double* out_rsqrt);

/*
 * Host-only self-check of mesh preparation and partitioning (no CUDA call, so
 * it runs without a GPU): validates and prepares the mesh as fem_create_mesh
 * does, plans an n_parts partition for CTAs of the solve kernel, once on 8 host
 * threads (whatever the mesh size) and once on one thread, and fills out[8]:
 *   out[0] 1 if the two plans are identical, out[1] 1 if the evaluation owner
 *   lists are valid (every tet listed exactly once, by a part holding it, with
 *   its owner flag set), out[2]/out[3] the largest/smallest owned tet count of
 *   a part, out[4] the largest part tet count (owned plus halo), out[5] the
 *   host threads of the first plan (8), out[6] the largest owned node count, out[7] 1 if every
 *   part's local node->tet lists are ascending in local tet index within a
 *   node (the order the chunked gathers need).
 * Arguments as fem_create_mesh (fixed_mask may be NULL). Errors: those of
 * fem_create_mesh's host validation; FEM_ERR_ARG if n_parts is out of range.
 */
int fem_debug_plan_check(const double* nodes, int64_t n_nodes, const int32_t* tets, int64_t n_tets,
                         const int32_t* tet_material, const fem_material* materials, int32_t n_materials,
                         const int32_t* fixed_nodes, int64_t n_fixed, int32_t n_parts, int64_t out[8]);

/*
 * Host-only check of the request server's choice of launch shape (no CUDA
 * call; the paper has no counterpart: it is the server's scheduling rule).
 * shape_groups [n_shapes * n_classes]: groups of class c in shape s at
 * [s * n_classes + c] (> 0: the shape serves the class); cur: the live shape;
 * request_ids / request_classes [n_requests]: the unfinished requests (ids
 * grow with submission). Writes the shape the server would run next to
 * *out_shape: with o the oldest request the live shape does not serve and t
 * the first shape serving o's class, t when o is older than every request of
 * the classes cur serves and t does not (or there is none); with no such o,
 * shape 0 when cur != 0 and every unfinished request's class is served by
 * shape 0, else cur. Errors: FEM_ERR_ARG (1-3 shapes, 1-8 classes, every class
 * served by some shape, classes in range, cur in range).
 */
int fem_debug_pick_shape(int32_t n_shapes, int32_t n_classes, const int32_t* shape_groups, int32_t cur,
                         const int64_t* request_ids, const int32_t* request_classes, int32_t n_requests,
                         int32_t* out_shape);

#ifdef __cplusplus
}
#endif
#endif /* FEM_B300_FEM_H */
