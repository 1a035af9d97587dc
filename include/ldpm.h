/*
 * ldpm.h -- C ABI of libldpm.so: the explicit central-difference time step of the Lattice Discrete
 * Particle Model (LDPM) on one NVIDIA GB300 GPU (sm_103a).
 *
 * Method (arXiv 2603.13190, "LDPM: comparison of various time integration solvers and
 * implementations"):
 *   - facet strain from the rigid-body jump of the two particles, Sec. 2, Eq. (1);
 *   - facet constitutive law t = T(e, s, p), Sec. 2 and Appendix A (fracture A.1, compression A.2,
 *     friction A.3);
 *   - particle force and moment balance, Sec. 2, Eq. (2a)-(2b), with the projected area A = A0 n.n0;
 *   - M q'' + f_int(q) = f_ext with a lumped mass, integrated by the central-difference scheme of
 *     the explicit solvers (Sec. 3, Sec. 3.2, the lumped-mass rule of Sec. 3.2.5);
 *   - energy balance 100 |W_ext - W_int - W_kin| / W_ext, Sec. 4.
 *
 * Conventions shared by every entry point:
 *   - Units are consistent; the library does not convert.  mm-N-MPa-tonne-s is recommended.
 *   - Every function returns LDPM_OK (0) or a negative LDPM_E_* code; ldpm_last_error() then holds
 *     a message for the calling thread.  No C++ exception crosses this boundary.
 *   - Arrays passed in are host memory owned by the caller, read during the call and never kept.
 *     Arrays passed out are host memory owned by the caller and written before the call returns.
 *   - Device memory, streams and CUDA graphs are owned by the ldpm_t handle and released by
 *     ldpm_destroy().
 *   - Particle arrays use the caller's particle order; facet arrays use the caller's facet order
 *     and orientation (force "on I" means on facet_pi[k]).  The library reorders internally.
 *   - DOF order per particle: u_x, u_y, u_z, theta_x, theta_y, theta_z.
 */
#ifndef LDPM_H
#define LDPM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LDPM_OK 0
#define LDPM_E_INVALID_ARG (-1)   /* a pointer, size or option is invalid */
#define LDPM_E_BAD_GEOMETRY (-2)  /* geometry violates the mesh rules listed at ldpm_geometry */
#define LDPM_E_CUDA (-3)          /* a CUDA call failed (message names it) */
#define LDPM_E_OOM (-4)           /* device or host allocation failed */
#define LDPM_E_UNSTABLE (-5)      /* a velocity or displacement became NaN/Inf (step too large?) */
#define LDPM_E_TIMEOUT (-6)       /* a grid barrier of the persistent step kernel waited longer than its
                                     limit (ldpm_set_barrier_wait); the state is undefined until
                                     ldpm_set_state or ldpm_load_checkpoint */
#define LDPM_E_UNSUPPORTED (-7)   /* the persistent launch cannot be made co-resident on the device */

typedef struct ldpm_ctx *ldpm_t; /* opaque handle, owned by the library */

typedef enum {
    LDPM_FP64 = 0,  /* every stage in FP64 */
    LDPM_MIXED = 1  /* facet kinematics, constitutive law and facet forces in FP32 (subnormal FP32
                       values flushed to zero), as is the sum of each tetrahedron's 6 facet terms at
                       one of its vertices; the particle sums of those shares (Eq. (2a)-(2b)) and
                       the energy increments (products with the half-step velocity and their 6-DOF
                       sums, Sec. 4) in compensated float-float arithmetic (48-bit significand, on
                       the FP32 pipe); particle state, velocity update, the increments' factor dt/2
                       and the energy accumulators in FP64 */
} ldpm_precision;

/* Raw specimen geometry (paper Sec. 3.1: particles, Delaunay tetrahedra, 12 facets per
 * tetrahedron).  Mesh rules checked by ldpm_create (LDPM_E_BAD_GEOMETRY otherwise):
 *   - n_facets == 12 * n_tets, every tetrahedron has 4 distinct particles and nonzero volume;
 *   - every facet belongs to facet_tet[k], its particles facet_pi[k] != facet_pj[k] are two
 *     vertices of that tetrahedron, and each of the 6 tetrahedron edges carries exactly 2 facets;
 *   - facet triangles have nonzero area; particle distances are nonzero and below l_t. */
typedef struct {
    int32_t n_particles, n_tets, n_facets;
    const double *x;          /* [N][3] particle centres */
    const double *diameter;   /* [N] particle diameters (0 allowed for surface nodes); may be NULL
                                 only if `inertia` is given */
    const int32_t *tet;       /* [T][4] particle indices of each tetrahedron */
    const int32_t *facet_pi;  /* [F] particle I of facet k */
    const int32_t *facet_pj;  /* [F] particle J of facet k; n_k points from I to J */
    const int32_t *facet_tet; /* [F] tetrahedron owning facet k */
    const double *facet_vtx;  /* [F][9] the three vertices of the facet triangle: its centroid is the
                                 point the arms c_I, c_J reach; its area A0 and normal n0 give the
                                 projected area A = A0 |n . n0| (Sec. 2) */
    const double *mass;       /* [N] translational mass or NULL: tetrahedron mass rho V split
                                 equally over its 4 nodes (Sec. 3.2.5) */
    const double *inertia;    /* [N][3] diagonal rotary inertia or NULL: m d^2 / 10 (Sec. 3.2.5),
                                 nodes with d = 0 take the smallest positive diameter */
} ldpm_geometry;

/* Material parameters, Appendix A table (names follow the paper's symbols).  ldpm_create checks
 * (LDPM_E_INVALID_ARG otherwise): every value finite; rho, E0, alpha, sigma_t, l_t, r_st, sigma_c0,
 * kc3, sigma_N0, Ed_E0 > 0; n_t, k_t, r_s >= 0; kc0 >= 1; reserved == 0. */
typedef struct {
    double rho;      /* density */
    double E0;       /* effective normal modulus */
    double alpha;    /* shear-normal coupling */
    double sigma_t;  /* tensile strength */
    double l_t;      /* tensile characteristic length, l_t = 2 E0 G_t / sigma_t^2 */
    double r_st;     /* shear-to-tensile strength ratio sigma_s / sigma_t */
    double n_t;      /* softening exponent */
    double sigma_c0; /* compressive yielding strength */
    double Hc0_E0;   /* initial hardening modulus ratio */
    double Hc1_E0;   /* final hardening modulus ratio */
    double kc0, kc1, kc2, kc3; /* kappa_c0..kappa_c3 */
    double mu0, mu_inf;        /* initial and asymptotic friction */
    double sigma_N0;           /* transitional stress */
    double Ed_E0;              /* E_d / E0: normal stiffness while -t_N exceeds sigma_c0 (App. A.2) */
    double beta;               /* volumetric-deviatoric coupling */
    double k_t;                /* tensile reload: from zero traction, reloading starts at
                                  e_tr = k_t (e_max - sigma_bt / E0) (App. A.1); 0 = at once */
    double r_s;                /* shear softening modulus ratio, H_s = r_s E0 (App. A.1) */
    int32_t elastic;           /* 1: linear elastic facets t = E e (Sec. 2) */
    int32_t reserved;          /* must be 0 */
} ldpm_material;

/* Boundary-condition codes per DOF (ldpm_options.bc_mask, ldpm_set_bc). */
#define LDPM_BC_FREE 0
#define LDPM_BC_FIXED 1      /* velocity 0 */
#define LDPM_BC_VELOCITY 2   /* velocity bc_vel * ramp(t), ramp(t) = clamp(t / ramp_time, 0, 1),
                                ramp = 1 when ramp_time <= 0 */

typedef struct {
    int32_t precision;   /* ldpm_precision */
    int32_t graph_chunk; /* steps per captured CUDA graph in ldpm_step; 0 = 32; < 0: no graphs */
    double dt;           /* time step; <= 0: dt_factor * 2 / sqrt(lambda_max(M^-1 K)), the largest
                            eigenvalue found by power iteration on the elastic operator */
    double dt_factor;    /* <= 0 means 0.9 (the paper runs at about 90 % of the critical step) */
    void *cuda_stream;   /* cudaStream_t all work is enqueued on; NULL = a library-owned stream */
    const int32_t *bc_mask; /* [N][6] LDPM_BC_* or NULL (all free) */
    const double *bc_vel;   /* [N][6] prescribed velocities or NULL */
    double ramp_time;       /* ramp duration of prescribed velocities */
    const double *v0;       /* [N][6] initial velocity or NULL */
    const double *f_ext;    /* [N][6] constant external nodal forces or NULL */
    int32_t device;         /* CUDA device ordinal; < 0 = the current device */
    int32_t autotune;       /* 1: at create, time the launch shapes (tetrahedra per facet-pass block,
                               lanes per particle) on this model and keep the fastest; 0: defaults.
                               Results are deterministic for a given shape; the lanes per particle
                               set the order of a particle's force sums (rounding-level effect) */
} ldpm_options;

/* Create a specimen from raw geometry (copied).  Validates the mesh rules, derives facet frames,
 * arms and projected areas, the lumped mass, the particle-to-facet CSR list and the Morton-ordered
 * device layout, uploads, and estimates dt if not given.  Initial state: q = 0, v = v0 (fixed DOFs
 * 0, prescribed DOFs at their prescribed velocity), zero facet history.  On success *out owns all
 * device memory.  Errors: INVALID_ARG (options, material checks), BAD_GEOMETRY, OOM, CUDA. */
int ldpm_create(const ldpm_geometry *geom, const ldpm_material *mat, const ldpm_options *opt, ldpm_t *out);

/* Enqueue nsteps central-difference steps (Sec. 3) on the handle's stream and return without
 * waiting.  Each step: half kick and drift of every particle (prescribed DOFs follow their
 * velocity), then per facet the strain of Eq. (1), the Appendix A law and the force A P t, then the
 * per-particle sums of Eq. (2) in a fixed order, the second half kick and the energy increments.
 * nsteps == 0 is a no-op.  Errors: INVALID_ARG (nsteps < 0), CUDA. */
int ldpm_step(ldpm_t h, int64_t nsteps);

/* Wait for all work enqueued on the handle's stream.  Returns TIMEOUT if a grid barrier of the
 * persistent step kernel gave up, UNSTABLE if a step produced a non-finite velocity or displacement. */
int ldpm_sync(ldpm_t h);

/* Launch modes of ldpm_step (a library service; both run the steps of Sec. 3 with the same device
 * functions in the same order; each is deterministic, and the two agree to rounding, since the
 * compiler may schedule and contract multiply-adds differently in the two kernels):
 *   LDPM_LAUNCH_PAIRS       per step a facet-pass launch and a particle-pass launch, replayed from
 *                           captured CUDA graphs (chunks of options.graph_chunk steps);
 *   LDPM_LAUNCH_PERSISTENT  one cooperative launch per ldpm_step call (chunks of up to 4096 steps)
 *                           running every step: facet pass, grid barrier, particle pass, grid
 *                           barrier, with as many blocks as the device holds at once.  Each barrier
 *                           wait is bounded; a wait that runs out ends the launch and the handle
 *                           reports LDPM_E_TIMEOUT (see ldpm_set_barrier_wait).
 * ldpm_create starts in LDPM_LAUNCH_PAIRS; with options.autotune = 1 it times both modes on the model
 * and keeps the faster.  ldpm_set_launch_mode applies to steps enqueued afterwards.  Errors:
 * INVALID_ARG, UNSUPPORTED (the persistent grid cannot be co-resident on this device). */
#define LDPM_LAUNCH_PAIRS 1
#define LDPM_LAUNCH_PERSISTENT 2
int ldpm_set_launch_mode(ldpm_t h, int32_t mode);
/* The handle's launch mode (LDPM_LAUNCH_*), or a negative error code. */
int32_t ldpm_launch_mode(ldpm_t h);

/* Bound of one grid-barrier wait of the persistent step kernel: `seconds` of the GPU's global timer
 * (<= 0: 2 s, the default); a wait also gives up after 2^24 polls.  skip_block >= 0 is a
 * fault-injection hook for tests of that bound: block `skip_block` of the next persistent launches
 * does not arrive at the launch's first barrier, so every block's wait runs out and the call
 * reports LDPM_E_TIMEOUT; -1 (the default) disables it.  No counterpart in the paper.  Errors:
 * INVALID_ARG (seconds not finite or above 3600, skip_block < -1). */
int ldpm_set_barrier_wait(ldpm_t h, double seconds, int32_t skip_block);

/* Copy the state out (synchronises).  q, v: [N][6]; hist5: [F][5] per facet t_N, the tangential
 * traction t_M m + t_L l as a global 3-vector, e_max (the traction acting on facet_pi[k]); step: the
 * step counter.  Any pointer may be NULL.  Returns UNSTABLE after a non-finite state (data still
 * copied).  The history is put in the caller's facet order on the device and copied straight into
 * hist5; the first call allocates a device scratch buffer of 12 N + 5 F doubles that the handle keeps
 * until ldpm_destroy (OOM if it cannot). */
int ldpm_get_state(ldpm_t h, double *q, double *v, double *hist5, int64_t *step);

/* The state of ldpm_get_state (Sec. 2: particle displacements and rotations q, velocities v, facet
 * tractions and e_max; Sec. 3: whole-step values q_n, v_n), written into caller-owned DEVICE buffers
 * on the handle's device: q, v [N][6] FP64 in caller particle order, hist5 [F][5] FP64 in caller facet
 * order (the layout of ldpm_get_state), step one int64.  Any pointer may be NULL.  A batch handle
 * writes all specimens concatenated in index order.  The conversion runs in kernels enqueued on the
 * handle's stream; the call returns without waiting and without any host copy, so a caller on
 * another stream orders its use of the buffers after the handle's stream (a torch caller passes its
 * stream at create, or waits on an event).  Allocates nothing.  It does not report a non-finite
 * state (ldpm_sync does).  Errors: INVALID_ARG (bad handle), CUDA (a launch failed, e.g. a buffer on
 * another device). */
int ldpm_get_state_device(ldpm_t h, double *q, double *v, double *hist5, int64_t *step);

/* Replace the state (synchronises).  Same layouts as ldpm_get_state; hist5 may be NULL (zero
 * history).  The internal forces of the new state are rebuilt from the given tractions; energy
 * accumulators restart (W_ext = W_int = 0, W_kin0 = kinetic energy of v). */
int ldpm_set_state(ldpm_t h, const double *q, const double *v, const double *hist5, int64_t step);

/* Energies and reactions of the current state (synchronises).  out = {W_ext, W_int, W_kin, err%}
 * with err% = 100 |W_ext + W_kin0 - W_int - W_kin| / (|W_ext| + W_kin0) (Sec. 4; W_kin0 = 0 in the
 * loaded tests makes it the paper's formula).  reaction[12] (may be NULL): sums over fixed DOFs of
 * the force the supports apply, per DOF component (6), then the same over velocity-prescribed DOFs
 * (6). */
int ldpm_energy(ldpm_t h, double out[4], double reaction[12]);

/* Forces of the current state (synchronises): F3 [F][3] facet force A P t acting on facet_pi[k];
 * f6 [N][6] per-particle sums of facet forces and moments.  Either pointer may be NULL. */
int ldpm_facet_forces(ldpm_t h, double *F3, double *f6);

/* Post-processing fields of the current state (synchronises).  crack_opening [F] (caller facet
 * order): w = sqrt(w_N^2 + w_M^2 + w_L^2) per facet, the comparison field of Sec. 4, with only
 * positive inelastic normal strain opening the crack; the paper gives no formula for w_alpha, the
 * library takes the inelastic part of the jump, w_N = l <e_N - t_N/E0>, w_M,L = l (e_M,L - t_M,L /
 * (alpha E0)).  tet_volumetric_strain [T] (caller tetrahedron order): e_V of App. A.2, the field
 * compared for the uniaxial-strain test (Sec. 4.2).  Either pointer may be NULL. */
int ldpm_metrics(ldpm_t h, double *crack_opening, double *tet_volumetric_strain);

/* Replace the boundary conditions (takes effect for steps enqueued afterwards).  mask [N][6],
 * vel [N][6] (NULL = zeros), ramp measured from t = 0. */
int ldpm_set_bc(ldpm_t h, const int32_t *mask, const double *vel, double ramp_time);

/* Sizes and step: info[0..4] = N, T, F, precision, step counter (synchronises); *dt = time step. */
int ldpm_info(ldpm_t h, int64_t info[5], double *dt);

/* Per-kernel CUDA-event timing of ldpm_step on the handle's stream.  enable = 1 starts (and
 * clears) recording, 0 stops.  While recording, ldpm_step launches each step's two kernels directly
 * (no graph) with an event before the facet pass, one between the passes and one after the particle
 * pass, so the two kernel times of a step add up to its duration.  ldpm_profile_read fills ms[k]
 * (summed milliseconds) and count[k] (launches) for k = 0 kick, 1 facet pass, 2 gather+update,
 * 3 reverse facet pass, 4 reverse particle pass (ldpm_adjoint) and 5 persistent step launch (whole
 * launches: the persistent kernel has no per-pass split); n = entries the caller provides (at most 6
 * are written). */
int ldpm_profile(ldpm_t h, int32_t enable);
int ldpm_profile_read(ldpm_t h, double *ms, int64_t *count, int32_t n);

/* Checkpoint of the complete mutable state in the library's internal layout (bitwise resume).
 * ldpm_checkpoint_size gives the byte count; save/load copy through caller host memory and
 * synchronise. */
int64_t ldpm_checkpoint_size(ldpm_t h);
int ldpm_save_checkpoint(ldpm_t h, void *buf);
int ldpm_load_checkpoint(ldpm_t h, const void *buf);

/* Kinetic energy W_kin = sum_i 1/2 mass[i] v[i]^2 of caller-provided DEVICE arrays, written to the
 * caller's DEVICE double *out, enqueued on `stream` (cudaStream_t; NULL = the legacy default stream)
 * and returned without waiting.  The paper has no counterpart: this is a library service for callers
 * that may not allocate device memory, such as code running inside another component's CUDA graph
 * capture (where cudaMalloc is not permitted), processes whose device memory is owned by a fixed
 * pool or caching allocator, and monitoring hooks that must not add the implicit synchronisation of
 * an allocation to a running simulation.  It allocates nothing: its scratch (one partial sum per
 * block of 1024 DOFs) is a 32 KiB static device array that every GPU loading the library holds until
 * exit, so n_dof is limited to 4,194,304 (LDPM_E_INVALID_ARG beyond it, nothing launched).  The first
 * call on a device looks up that array's device address (cudaGetSymbolAddress) with the device
 * current; make that first call before any stream capture.  The address is kept per device ordinal
 * for the life of the process and belongs to the device's primary context: after cudaDeviceReset of
 * that device, or when the caller makes a non-primary (driver API) context current, it is no longer
 * valid, so call this function only from the primary context and not after a reset.  All calls share the one array: every
 * call overwrites the partials it reads, so nothing needs clearing, but calls that overlap on the GPU
 * (on different streams, or from different threads) race on it and must be serialised by the
 * caller.  The result equals the W_kin of ldpm_energy for the same velocities and masses up to
 * summation order.  Errors: INVALID_ARG (NULL pointer, n_dof < 0, n_dof over the limit), CUDA. */
int ldpm_kinetic_energy_noalloc(const double *v, const double *mass, int64_t n_dof, double *out, void *stream);

/* ---- Batches: many specimens (e.g. random realizations of uneven size) stepped together, one
 * facet-pass launch and one particle-pass launch per step for all of them.  Each specimen keeps its
 * own geometry, material, time step, boundary conditions and energies; all share the precision, the
 * stream and the step counter.  opts[0] supplies precision, stream, graph chunk, device and
 * autotune.  ldpm_step / ldpm_get_state / ldpm_metrics / checkpoints act on the whole batch (arrays
 * of all specimens concatenated in index order); ldpm_set_state, ldpm_set_bc and ldpm_energy need a
 * single-specimen handle (LDPM_E_INVALID_ARG otherwise).  The paper runs one specimen per solver
 * run; batching is a library service. */
int ldpm_batch_create(int32_t n, const ldpm_geometry *geoms, const ldpm_material *mats, const ldpm_options *opts,
                      ldpm_t *out);
int ldpm_batch_step(ldpm_t h, int64_t nsteps);  /* same as ldpm_step */
int32_t ldpm_batch_size(ldpm_t h);              /* number of specimens (or a negative error) */
/* State, energies (as ldpm_energy), metrics (as ldpm_metrics) and sizes/time step (as ldpm_info) of
 * specimen idx, in that specimen's own particle and facet order. */
int ldpm_batch_get_state(ldpm_t h, int32_t idx, double *q, double *v, double *hist5, int64_t *step);
int ldpm_batch_energy(ldpm_t h, int32_t idx, double out[4], double reaction[12]);
int ldpm_batch_metrics(ldpm_t h, int32_t idx, double *crack_opening, double *tet_volumetric_strain);
int ldpm_batch_info(ldpm_t h, int32_t idx, int64_t info[5], double *dt);

/* Launch shape in use: shape[0] tetrahedra per facet-pass block, shape[1] lanes per particle in the
 * particle pass (set by defaults, the LDPM_TETS_PER_BLOCK / LDPM_GATHER_LANES environment variables
 * at create, or the autotuner).  Library service; no counterpart in the paper. */
int ldpm_launch_shape(ldpm_t h, int32_t shape[2]);

/* Add dq [6*N] (caller particle order) to the displacements and rotations of the free DOFs of the
 * current state; constrained DOFs are left alone.  Velocities, tractions and e_max are kept, and the
 * next step's strain increment is measured from the perturbed state (as after ldpm_set_state).  For
 * perturbation studies like the paper's Sec. 5 (random vectors uniform in [-eta/2, eta/2] added to
 * all free displacements and rotations at intervals); the caller draws dq.  Synchronous.  Errors:
 * INVALID_ARG (NULL, non-finite entries), OOM, CUDA. */
int ldpm_perturb(ldpm_t h, const double *dq);

/* ---- Per-facet parameters and the adjoint.  The paper uses one material for all facets and has no
 * derivatives; these serve sensitivity and calibration studies of its explicit step (Sec. 3,
 * App. A).  Single-specimen handles only (LDPM_E_INVALID_ARG for batches). */

/* Give facet k its own E0[k], alpha[k], sigma_t[k] (caller facet order, [F] each, finite and > 0)
 * in place of the material's; a NULL array keeps the material's value for that parameter, all three
 * NULL restore the material everywhere.  The constants derived from them (App. A: sigma_s = r_st
 * sigma_t, H_c0 = (H_c0/E0) E0, e_c0 = sigma_c0 / E0, ...) follow per facet.  Acts from the next step;
 * the stored tractions are kept and dt is not re-estimated.  Synchronises the stream.  Errors:
 * INVALID_ARG, OOM, CUDA. */
int ldpm_set_facet_params(ldpm_t h, const double *E0, const double *alpha, const double *sigma_t);

/* Run `nsteps` steps from the current state (as ldpm_step would; the handle ends in the same state)
 * and return the objective
 *     J = (1 / nsteps) sum_{n=1..nsteps} sum_{constrained DOF i} seed[i] R_i(t_n),
 * the time mean of the seeded reactions R = m a - f of the fixed and prescribed DOFs (seed [6*N],
 * caller particle order, entries of free DOFs ignored; e.g. 1 on the u_z DOFs of the loaded face
 * gives its mean reaction force), with its gradient with respect to every facet's E0, alpha and
 * sigma_t (gE0, galpha, gsigma_t: [F] each in caller facet order; any may be NULL).  The reverse
 * pass needs the states of the forward run in reverse order: the state is checkpointed on the device
 * every `ckpt_every` steps, and each segment but the last is recomputed once, keeping its steps'
 * inputs (the last segment's are kept during the forward run; with ckpt_every >= nsteps nothing is
 * recomputed).  Device memory: (nsteps / ckpt_every + 1) states plus ckpt_every step inputs (mixed
 * mode: 96 B per particle and 16 B per facet each).  Arithmetic in the model's precision (mixed: FP32 facet terms, FP64
 * particle adjoints and gradient totals).  Derivatives at points where the law is not differentiable
 * (a switch of branch, sqrt at 0) are those of the branch the forward value takes.  With gE0, galpha
 * and gsigma_t all NULL only the forward run and J are computed.  Synchronous.
 * Errors: INVALID_ARG, OOM (checkpoint memory), UNSTABLE (non-finite state or gradient), CUDA. */
int ldpm_adjoint(ldpm_t h, int64_t nsteps, int32_t ckpt_every, const double *seed, double *J, double *gE0,
                 double *galpha, double *gsigma_t);

/* The constitutive update (App. A) and its vector-Jacobian product on the device, for n independent
 * facet states (a test and analysis hook; no counterpart in the paper).  in [n][16] = l, e_N, e_M,
 * e_L, de_N, de_M, de_L, e_V, t_N, t_M, t_L (previous tractions), e_max (previous), E0, alpha,
 * sigma_t, 0 (the remaining parameters from *mat).  adj_out [n][4] = adjoints of the new t_N, t_M,
 * t_L, e_max.  Writes out [n][4] = new t_N, t_M, t_L, e_max and adj_in [n][16] = the adjoints of the
 * inputs in the layout of `in` (slots 0 and 15 zero).  precision: LDPM_FP64 or LDPM_MIXED (FP32
 * law).  Synchronous; uses the current CUDA device.  Errors: INVALID_ARG, OOM, CUDA. */
int ldpm_facet_law_vjp(int32_t precision, const ldpm_material *mat, int64_t n, const double *in, const double *adj_out,
                       double *out, double *adj_in);

/* Release everything the handle owns (synchronises first).  NULL is a no-op. */
void ldpm_destroy(ldpm_t h);

/* Message of the last failing call on this thread ("" if none).  Valid until the next call. */
const char *ldpm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LDPM_H */
