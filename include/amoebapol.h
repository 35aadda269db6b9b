/*
 * amoebapol.h - C ABI of the GB300 (sm_103a) AMOEBA induced-dipole solver.
 *
 * The computation is the polarization step that dominates the AMOEBA runs of
 * the Tinker-HP performance study (arXiv:1906.01211), Section "Hotspots":
 *   - the right-hand side of the polarization equation, the permanent
 *     multipole field E0 (routine efld0_direct2);
 *   - the matrix-vector product T*mu applied at each iteration of the
 *     polarization solver (routine tmatxb_pme2), about nine calls per step
 *     (Section "Sequential performance");
 *   - the dipole polarization energy (routine epolar1).
 * The solver is preconditioned conjugate gradients on
 *     (diag(1/alpha) - T) mu = E0,
 * T = real-space Ewald (erfc-screened, Thole-damped) dipole field over cell
 * neighbour lists + smooth-PME reciprocal part + Ewald self term.
 *
 * Conventions for every call below.
 *   Pointers: all array arguments are DEVICE pointers owned by the caller,
 *     row-major, float64, indexed by the caller's atom order:
 *       positions, dipoles, fields, induced dipoles: [N][3];
 *       quadrupoles: [N][6] as xx, yy, zz, xy, xz, yz (traceless, Buckingham:
 *       potential r.Theta.r / r^5);  charges, alpha, thole: [N];  mol: int32 [N].
 *     Scalars returned through pointers (iters, rms, U, counts) are HOST pointers.
 *   Units: Angstrom, e, e*Angstrom, e*Angstrom^2, Angstrom^3; fields e/Angstrom^2;
 *     energy kcal/mol (Coulomb constant 332.0637133); residual RMS in Debye
 *     (4.8032047 D per e*Angstrom).
 *   Stream: work is enqueued on the stream given to amp_create; device
 *     outputs are valid once that stream has reached the call's end. Calls that
 *     return host scalars synchronise the stream.
 *   Errors: every int-returning call returns AMP_OK (0) or a negative code;
 *     amp_last_error() gives a message. After AMP_ERR_CUDA the context should
 *     be destroyed.
 *   Memory: the context owns its device buffers (cell lists, neighbour lists,
 *     pair tensors, PME grids, cuFFT plans, solver vectors); they are sized by
 *     amp_set_system and reused by every later call. No call allocates inside
 *     the solver loop.
 */
#ifndef AMOEBAPOL_H
#define AMOEBAPOL_H

#ifdef __cplusplus
extern "C" {
#endif

#define AMP_OK 0
#define AMP_ERR_ARG (-1)           /* invalid argument or configuration */
#define AMP_ERR_CUDA (-2)          /* CUDA or cuFFT failure */
#define AMP_ERR_OOM (-3)           /* device allocation failed */
#define AMP_ERR_NOT_CONVERGED (-4) /* PCG reached max_iter above tolerance */
#define AMP_ERR_GEOMETRY (-5)      /* cutoff >= box/2, list overflow, bad cell */
#define AMP_ERR_STATE (-6)         /* call order: no system set */
#define AMP_ERR_STALE (-8)         /* amp_update_positions: an atom moved more than skin/2 */

#define AMP_FP64 0   /* float64-accurate results. The permanent field E0
                        is float64 arithmetic (its reciprocal part, and the
                        excluded intramolecular real-space terms that cancel
                        against it); the per-pair terms, T*mu and its PME
                        spreading, FFTs and gather run in double-float (a
                        value is the unevaluated sum of two floats, ~48
                        significant bits, on the float32 units, because
                        float64 is 1/64 of the float32 rate on GB300); the
                        PCG vectors, dot products and scalars are float64 */
#define AMP_MIXED 1  /* float32 pair geometry/damping and a float32
                        operator input (PME as in AMP_FP64), float64
                        accumulation, scalars, self terms and a final float64
                        residual check (lower precision, paper Section
                        "Conclusion") */

typedef struct amp_ctx amp_ctx;

typedef struct {
  double box;        /* cubic box edge (Angstrom); must be > 2 * cutoff.
                        0 = isolated cluster: every pair, no cutoff, no Ewald
                        (cutoff, ewald_beta, pme_grid, pme_order ignored) */
  double cutoff;     /* real-space cutoff (Angstrom) */
  double ewald_beta; /* Ewald splitting parameter (1/Angstrom), > 0, with ewald_beta * cutoff <= 8 */
  int pme_grid;      /* PME points per axis, >= 8 */
  int pme_order;     /* B-spline order; must be 5 */
  double tol_debye;  /* PCG stop: RMS of alpha*residual in Debye < tol */
  int max_iter;      /* PCG iteration cap (>= 1) */
  int precision;     /* AMP_FP64 or AMP_MIXED */
} amp_config;

/* Create a context bound to a CUDA stream (cudaStream_t passed as void*;
 * NULL = legacy default stream). Validates cfg. Returns AMP_ERR_ARG on a bad
 * configuration (then *out is NULL). */
int amp_create(amp_ctx** out, const amp_config* cfg, void* cuda_stream);

/* Change box, cutoff, beta, tolerance and iteration cap of a context while
 * keeping its buffers and cuFFT plans: the PME grid size, B-spline order,
 * precision and cluster/periodic mode must stay those given to amp_create
 * (else AMP_ERR_ARG). Recomputes the influence function on the device when
 * box or beta change; the next call must be amp_set_system. */
int amp_reconfigure(amp_ctx* ctx, const amp_config* cfg);

/* Free every device buffer and plan of the context. NULL is ignored. */
void amp_destroy(amp_ctx* ctx);

/* Message of the last error on this context (static storage inside ctx). */
const char* amp_last_error(const amp_ctx* ctx);

/* Load a system of n_atoms sites and build the geometry-dependent state:
 * cell list (atoms re-ordered by cell), neighbour lists within the cutoff
 * (paper, Section "Hotspots": cell-based list builder mlistcell), per-pair
 * damped interaction tensors and permanent-field terms, and PME B-spline
 * weights. Inputs as described above; alpha must be > 0. Re-allocates only
 * when the system grows. Synchronises the stream once (list sizes). */
int amp_set_system(amp_ctx* ctx, int n_atoms, const double* xyz, const double* q,
                   const double* dip, const double* quad, const double* alpha,
                   const double* thole, const int* mol);

/* Neighbour-list skin (Angstrom, >= 0; periodic contexts; cutoff + skin <
 * box/2), used from the next amp_set_system on: that call then also keeps the
 * candidate pairs within cutoff + skin and the positions it saw, so that
 * amp_update_positions can rebuild the lists from them (Verlet-style list
 * reuse; the paper, Section "Hotspots", names the cell list builder among the
 * hotspots). 0, the default, keeps no candidates. */
int amp_set_list_skin(amp_ctx* ctx, double skin);

/* New positions xyz [N][3] (device, caller order) for the atoms of the last
 * amp_set_system, whose other inputs are kept. If a skin was set for that
 * call and no atom has moved more than skin/2 (minimum image) since it, the
 * neighbour lists are filtered out of its candidates (the same pairs, by the
 * same float64 decision, as a new cell search), the pair terms and PME
 * weights are rebuilt, and *reused = 1. Otherwise nothing changes and the call
 * returns AMP_ERR_STALE: call amp_set_system. Synchronises the stream once
 * (twice when it returns AMP_ERR_STALE). */
int amp_update_positions(amp_ctx* ctx, const double* xyz, int* reused);

/* Warm start along a trajectory: order k (0 .. 6) keeps the last k + 2
 * converged solutions of amp_solve_induced (cleared by amp_set_system, kept
 * by amp_update_positions), and use_guess = 2 starts the next solve from
 * their always-stable predictor-corrector extrapolation (Kolafa, J. Comput.
 * Chem. 25, 335 (2004): mu_0 = sum_j B_j mu_{-j}, B_j = (-1)^(j+1) j
 * C(2k+4, k+2-j) / C(2k+2, k+1)); the solve then converges to the same
 * tolerance from there. -1 (the default) keeps no history. */
int amp_set_predictor(amp_ctx* ctx, int order);

/* The predictor's coefficients B_1 .. B_{order+2} into b (host memory; no
 * context, no GPU). AMP_ERR_ARG for an order outside 0 .. 6. */
int amp_predictor_coefficients(int order, double* b);

/* Permanent-multipole field at every site, E0 [N][3] (real space with the
 * intramolecular exclusion + PME + self). The right-hand side of the
 * polarization equation (routine efld0_direct2). */
int amp_permanent_field(amp_ctx* ctx, double* E0);

/* General AMOEBA's second right-hand side (paper Section "Polarizable AMOEBA
 * force field" names the model; the two exclusion rules are Ren & Ponder's):
 * the permanent field with scale s_intra (0 <= s <= 1) for two sites of one
 * molecule instead of 0, E [N][3] (device, caller order):
 *   E = E0 + sum over intramolecular pairs of s * (Thole-damped bare field),
 * the "polarization" field E_p beside amp_permanent_field's "direct" E_d.
 * With mu_d = A^-1 E_d and mu_p = A^-1 E_p (amp_solve_induced on each), the
 * two-field energy is U = -1/2 C mu_d . E_p (amp_polarization_energy(mu_d,
 * E_p)). Periodic contexts. */
int amp_permanent_field_scaled(amp_ctx* ctx, double s_intra, double* E);

/* Gradients of that U at the two solutions (A is symmetric, so no re-solve):
 *   F = -dU/dr = 1/2 C [ d(mu_p . E_d) + d(mu_d . E_p) + d(mu_p . T mu_d) ],
 *   dU/dq, dU/dd, dU/dTheta = -1/2 C d(mu_p . E_d + mu_d . E_p)/d(moment)
 * (moment gradients as in amp_forces, unprojected). mu_d, mu_p [N][3]
 * (device, caller order); F required, gq, gdip, gquad may be NULL. Periodic
 * contexts. */
int amp_two_rhs_forces(amp_ctx* ctx, double s_intra, const double* mu_d, const double* mu_p, double* F, double* gq,
                       double* gdip, double* gquad);

/* Tmu = T * mu for any mu [N][3] (real + reciprocal + self), the operator
 * applied at each solver iteration (routine tmatxb_pme2). */
int amp_apply_T(amp_ctx* ctx, const double* mu, double* Tmu);

/* Solve (1/alpha - T) mu = E0 by diagonal-preconditioned CG.
 * use_guess = 0: start from mu = alpha*E0 (mu is output only);
 * use_guess = 1: start from the mu passed in;
 * use_guess = 2: start from the predictor of amp_set_predictor over the
 *   solutions this context has converged to since its last amp_set_system
 *   (alpha*E0 while there are fewer than order + 2 of them).
 * On return mu holds the solution; *iters the number of iterations and
 * *rms_debye the final preconditioned-residual RMS (Debye). In AMP_MIXED the
 * final check is a float64 residual; if it is above tol, iterations continue.
 * Returns AMP_ERR_NOT_CONVERGED (mu still written) if max_iter is reached. */
int amp_solve_induced(amp_ctx* ctx, const double* E0, double* mu, int use_guess,
                      int* iters, double* rms_debye);

/* Polarization energy U = -1/2 C sum_i mu_i . E0_i (kcal/mol) into *U (host). */
int amp_polarization_energy(amp_ctx* ctx, const double* mu, const double* E0, double* U);

/* Gradients of the polarization energy at the solution mu (paper, Section
 * "Hotspots": routine epolar1 computes the polarization energy and forces).
 * U is stationary in mu, so no re-solve: the adjoint is mu itself.
 *   mu    [N][3] the converged induced dipoles (caller order);
 *   F     [N][3] forces -dU/dr (kcal/mol/Angstrom), required;
 *   gq    [N]    dU/dq, gdip [N][3] dU/dd, gquad [N][6] dU/dTheta for the six
 *         stored components (xx, yy, zz, xy, xz, yz; each off-diagonal stands
 *         for two matrix entries); each may be NULL to skip it.
 * Multipoles are global-frame, so there are no torque terms. Uses the
 * geometry of the current system; allocates its buffers on the first call. */
int amp_forces(amp_ctx* ctx, const double* mu, double* F, double* gq, double* gdip, double* gquad);

/* Truncated conjugate gradient of order one (TCG-1), the non-iterative
 * solver the paper's outlook names (Section "Perspectives on Tinker-HP 1.2
 * performance"): one diagonal-preconditioned CG step from the direct guess,
 *   u = alpha E0, r = T u, z = alpha r, gamma = (r.z)/(z.A z), mu_1 = u + gamma z,
 *   U_1 = -1/2 C mu_1 . E0,
 * and the exact gradients of U_1 (mu_1 is not the minimiser, so they run
 * through gamma, r and z: three operator applications, no solve).
 *   E0    [N][3] the permanent field (device, caller order), required;
 *   mu    [N][3] mu_1 (may be NULL);  U: kcal/mol into *U (host; may be NULL);
 *   F     [N][3] -dU_1/dr, gq [N], gdip [N][3], gquad [N][6] the moment
 *         gradients as in amp_forces (unprojected); F may be NULL (energy
 *         only; then the moment gradients must be NULL too); periodic
 *         contexts only for the gradients.
 * Operator applications in the context's precision; scalars and sums in
 * float64. AMP_ERR_NOT_CONVERGED if z.A z <= 0. Synchronises the stream. */
int amp_tcg1(amp_ctx* ctx, const double* E0, double* mu, double* U, double* F, double* gq, double* gdip,
             double* gquad);

/* Divide-and-conquer Jacobi iterations (DC-JI), the polarization solver the
 * paper's outlook names for the outer level of its multi-timestep integrator
 * (Section "Perspectives on Tinker-HP 1.2 performance"; Nocito & Beran 2018).
 * The sites are split into blocks (whole molecules, as the caller chooses);
 * every iteration solves each block's own equations exactly with the other
 * blocks' dipoles from the previous iteration:
 *   mu <- mu + D^-1 (E0 - A mu),  mu^(0) = alpha E0,
 * D the block diagonal of A = diag(1/alpha) - T (real space, reciprocal space
 * and self term), until 4.8032047 sqrt(sum |alpha (E0 - A mu)_i|^2 / N) < tol
 * or max_iter iterations (the solver's criterion).
 *   E0       [N][3] the permanent field (device, caller order);
 *   block_of [N] block index of each site in [0, n_blocks) (host, caller
 *            order); every block must have a site, else AMP_ERR_ARG;
 *   mu       [N][3] the dipoles on return (device, caller order);
 *   iters, rms_debye: iterations done and the final RMS (host, may be NULL).
 * D is assembled from the context's operator one column at a time (3N
 * operator applications), then each block is symmetrised and factorised by
 * Cholesky in float64 (AMP_ERR_NOT_CONVERGED if one is not positive
 * definite); for small systems. Float64 contexts only; allocates and frees
 * its buffers and synchronises the stream. */
int amp_dcji(amp_ctx* ctx, const double* E0, const int* block_of, int n_blocks, double tol_debye, int max_iter,
             double* mu, int* iters, double* rms_debye);

/* Energy of the permanent multipoles with each other and its gradients (paper,
 * Section "Hotspots": routine empole1 computes this energy and its forces).
 * Ewald sum with tin-foil boundary:
 *   U = C [ sum over unique pairs within the cutoff of U_ij  (minimum image)
 *         + 1/2 sum_g Q(g) phi(g)                            (smooth PME)
 *         - beta/sqrt(pi) sum_i (q_i^2 + 2 beta^2/3 |d_i|^2 + 8 beta^4/45 Theta_i:Theta_i)
 *         - pi Q_tot^2 / (2 V beta^2) ],
 * U_ij = (q_i + d_i.grad + Theta_i:grad grad/3)(q_j - d_j.grad + Theta_j:grad grad/3) B_0
 * at r = x_i - x_j with the Ewald-screened kernels, minus the bare ones for two
 * sites of one molecule (excluded pair); no Thole damping.
 *   U     kcal/mol into *U (host); may be NULL;
 *   F     [N][3] -dU/dr (kcal/mol/Angstrom); gq [N] dU/dq; gdip [N][3] dU/dd;
 *   gquad [N][6] dU/dTheta for the six stored components, each off-diagonal
 *         standing for two entries, with the mean of the three diagonal ones
 *         removed (quadrupoles are traceless, so only traceless changes
 *         exist); each may be NULL to skip it (at least one output).
 * An isolated cluster (box = 0) has only the pair sum, over all pairs, with the
 * bare kernels. Caller order, device pointers except U. Float64 results in
 * both precision modes. Uses the geometry and lists of the current system;
 * allocates its buffers on the first call. */
int amp_multipole_energy(amp_ctx* ctx, double* U, double* F, double* gq, double* gdip, double* gquad);

/* Number of unique atom pairs within the cutoff of the current system. */
int amp_pair_count(const amp_ctx* ctx, long long* n_pairs);

/* Phase timers (CUDA events recorded on the context's stream around each
 * phase's launches; no effect on results). Phases: */
#define AMP_PHASE_LIST 0        /* cell sort + neighbour lists (kernel a) */
#define AMP_PHASE_PAIR 1        /* per-pair tensors and permanent-field terms */
#define AMP_PHASE_E0_REAL 2     /* real-space permanent field row sums */
#define AMP_PHASE_E0_RECIP 3    /* PME of the permanent multipoles */
#define AMP_PHASE_T_REAL 4      /* real-space T*v, one launch per application */
#define AMP_PHASE_T_RECIP 5     /* PME of dipoles: spread, FFTs, gather */
#define AMP_PHASE_PCG 6         /* fused PCG vector updates and reductions */
#define AMP_PHASE_FP64_CHECK 7  /* mixed path: float64 residual check */
#define AMP_PHASE_ENERGY 8      /* energy reduction */
#define AMP_PHASE_FORCES 9      /* forces and moment gradients (polarization, multipoles) */
#define AMP_PHASE_T_SPREAD 10   /* within AMP_PHASE_T_RECIP: the dipole spreading */
#define AMP_PHASE_T_FFT 11      /* within AMP_PHASE_T_RECIP: the 3D FFT convolution */
#define AMP_PHASE_T_GATHER 12   /* within AMP_PHASE_T_RECIP: the field gather */
#define AMP_PHASE_LIST_SEARCH 13  /* within AMP_PHASE_LIST: the cell search (k_neighbours) */
#define AMP_NPHASE 14

/* enable != 0: start recording (clears totals); 0: stop. */
int amp_profile(amp_ctx* ctx, int enable);

/* Synchronise the stream and return, per phase, the summed milliseconds and
 * the number of timed intervals since amp_profile(ctx, 1). Arrays of
 * AMP_NPHASE entries (host). */
int amp_profile_read(amp_ctx* ctx, double* ms, long long* count);

/* Number of kernels of this library launched on the context so far (library
 * kernels only; cuFFT's own kernels are not included). */
int amp_launch_count(const amp_ctx* ctx, long long* n);

/* Iterations and float64 residual checks of the last solve (host pointers,
 * either may be NULL). */
int amp_last_solve_stats(const amp_ctx* ctx, int* iters, int* fp64_checks);

/* ---- Local-frame multipoles (AMOEBA, paper Section "Polarizable AMOEBA
 * force field"; frame conventions of Ren & Ponder). Site i's dipole and
 * quadrupole are given in a frame fixed by its axis atoms zatom[i],
 * xatom[i]: v1 = x_z - x_i, v2 = x_x - x_i; kind 0 (Z-then-X): e_z = v1/|v1|;
 * kind 1 (bisector): e_z = a/|a|, a = v1/|v1| + v2/|v2|; then e_x = the unit
 * part of v2 normal to e_z, e_y = e_z x e_x, R = [e_x e_y e_z];
 * d = R d_loc, Theta = R Theta_loc R^T. Any other kind, or axis atoms that are
 * not two other atoms of the system, leaves the site's moments as given.
 * Both calls are context-free, enqueue one kernel on cuda_stream
 * (cudaStream_t as void*; NULL = legacy default stream), take device arrays
 * in caller order (xyz, dip [N][3], quad [N][6] as in amp_set_system; kind,
 * zatom, xatom int32 [N]) and allocate nothing. AMP_ERR_ARG for a null
 * pointer or n_atoms < 1; AMP_ERR_CUDA for a launch error (an error pending
 * on the thread from an earlier call is left pending). */

/* Global moments dip, quad from the local ones (for amp_set_system). */
int amp_frames_to_global(int n_atoms, const double* xyz, const double* dip_local, const double* quad_local,
                         const int* kind, const int* zatom, const int* xatom, double* dip, double* quad,
                         void* cuda_stream);

/* Frame terms of the forces: F_k -= sum_i dU/dd_i . dd_i/dx_k +
 * dU/dTheta_i . dTheta_i/dx_k over the sites i whose frames atom k fixes,
 * from the moment gradients gdip [N][3], gquad [N][6] (unprojected, each
 * off-diagonal standing for two entries, as amp_forces and amp_tcg1 return
 * them) of an energy at fixed frames. Adds to F [N][3] (float64 atomics). */
int amp_frame_forces(int n_atoms, const double* xyz, const double* dip_local, const double* quad_local,
                     const int* kind, const int* zatom, const int* xatom, const double* gdip, const double* gquad,
                     double* F, void* cuda_stream);

/* ---- Serving: continuous batching of many independent solves.
 *
 * The paper has no serving counterpart (its throughput runs are many MPI
 * ranks on one system, Section "Parallel performance"); the solves
 * themselves are the calls above. A server owns one GPU (the device given to
 * amp_server_create) and accepts requests at any time from any thread: an
 * isolated cluster (box = 0: every pair, no Ewald) or a periodic cubic box,
 * each with its own atoms. Requests run as soon as memory and a place free
 * up, beside those already running:
 *   - clusters of at most batch_max_atoms atoms (without a key) join the
 *     batched engine: one device arena, one PCG state per request, and every
 *     iteration of all of them is one pair of launches of persistent kernels
 *     that take (request, 64-row tile) work items from a device queue;
 *   - the other requests go to n_workers workers, each with its own CUDA
 *     stream, running the single-system calls above on contexts taken from
 *     a pool keyed by PME grid size (created on first need, kept for later
 *     requests of that size, destroyed to make room for another size when the
 *     memory budget is reached).
 * Admission: a request starts when its memory (an upper estimate for a new
 * context, the exact bytes of a pooled one; arena space in the batched
 * engine) fits in mem_budget_bytes beside what is in use. Dipoles of keyed
 * requests stay on the device (LRU, resident_bytes) and start the next solve
 * of the same key. Every request's inputs are copied at submission (host
 * arrays, caller's order, layouts as above); results are host copies. Each
 * request's arithmetic is that of a solve alone: the result does not depend
 * on what else runs. Failures are per request (invalid input, a request
 * larger than the whole budget); the server and the other requests go on. */
#define AMP_PENDING 1  /* amp_server_poll: the request has not finished */

typedef struct amp_server amp_server;

typedef struct {
  int n_workers;               /* context workers (>= 1) */
  long long mem_budget_bytes;  /* device memory for contexts, arena and resident dipoles */
  int precision;               /* AMP_MIXED or AMP_FP64, for every request */
  double tol_debye;            /* PCG stop, every request */
  int max_iter;                /* PCG iteration cap, every request */
  int batch_max_atoms;         /* clusters up to this size use the batched engine (0: no engine) */
  int batch_arena_atoms;       /* atoms the batched engine holds at once (>= batch_max_atoms) */
  int batch_max_requests;      /* requests the batched engine holds at once */
  long long resident_bytes;    /* budget of the resident dipoles of keyed requests */
} amp_server_config;

typedef struct {
  int status;        /* AMP_OK, or the request's error code */
  int iters;         /* PCG iterations */
  double rms_debye;  /* final preconditioned residual RMS (Debye) */
  double energy;     /* polarization energy U = -1/2 C mu.E0 (kcal/mol) */
  double t_submit, t_start, t_done;  /* seconds on the server's steady clock */
  int path;          /* 0 batched engine, 1 context worker */
  int warm_start;    /* 1 if started from a keyed request's resident dipoles */
  char error[160];   /* message when status != AMP_OK */
} amp_server_result;

typedef struct {
  long long submitted, done, failed;
  int queued, running_batch, running_workers, contexts;
  long long bytes_in_use, budget;
  long long batch_launches;  /* pair + vector launches of the batched engine */
} amp_server_counters;

/* Start a server on CUDA device `device` (threads and streams of its own).
 * AMP_ERR_ARG for a bad configuration, AMP_ERR_CUDA / AMP_ERR_OOM when the
 * device or the arena cannot be had. */
int amp_server_create(amp_server** out, const amp_server_config* cfg, int device);

/* Queue one request; *ticket identifies it. Host arrays in the layouts of
 * amp_set_system (copied before the call returns). box = 0: isolated
 * cluster; box > 0: periodic cubic box whose cutoff, Ewald beta and PME grid
 * are taken from cutoff, beta, grid when given (> 0), else cutoff =
 * min(7, box/2 - 1e-6), beta = 3.8122/cutoff (erfc(beta cutoff) = 7e-8) and
 * grid = the smallest 2,3,5-smooth size >= box beta/0.5446 (at least 8). key
 * (may be NULL) names a request whose dipoles stay resident for the next one
 * of the same key. AMP_ERR_ARG for null arrays or n_atoms < 2, AMP_ERR_STATE
 * after amp_server_destroy began. A request larger than the whole memory
 * budget is accepted and fails alone (its result has AMP_ERR_OOM). */
int amp_server_submit(amp_server* s, int n_atoms, double box, double cutoff, double beta, int grid,
                      const double* xyz, const double* q, const double* dip, const double* quad,
                      const double* alpha, const double* thole, const int* mol, const char* key,
                      long long* ticket);

/* AMP_PENDING while the request runs or waits. Once it has finished:
 * AMP_OK, its dipoles into mu [N][3] (host; may be NULL) and its record into
 * *res (may be NULL); the ticket is then released (a later poll returns
 * AMP_ERR_ARG). AMP_ERR_ARG for an unknown ticket. */
int amp_server_poll(amp_server* s, long long ticket, double* mu, amp_server_result* res);

/* amp_server_poll that waits up to timeout_s seconds (< 0: without limit);
 * AMP_PENDING if the time ran out first. */
int amp_server_wait(amp_server* s, long long ticket, double timeout_s, double* mu, amp_server_result* res);

/* Counters at the time of the call. */
int amp_server_stats(amp_server* s, amp_server_counters* out);

/* Finish the requests already queued, stop the threads, free the device
 * memory. NULL is ignored. */
void amp_server_destroy(amp_server* s);

/* Polarization energy without any allocation. The paper has no counterpart to
 * this entry point: it exists for callers that cannot allocate device memory
 * when they need the energy (a host framework that owns all device memory in
 * its own pool, or a loop that must not pay the implicit synchronisation of
 * cudaMalloc/cudaFree). Same value as amp_polarization_energy, U = -1/2 C
 * sum_i mu_i . E0_i (kcal/mol), but no context is needed and nothing is
 * allocated: the only scratch (one float64 partial per 256 atoms) is a fixed
 * 32 KiB array in device memory owned by the library, present on every GPU
 * that loads it until the process exits.
 *   n_atoms: 1 .. AMP_NOALLOC_MAX_ATOMS; larger returns AMP_ERR_TOO_LARGE and
 *            launches nothing.
 *   mu, E0:  device [N][3] float64 (caller's);  U: DEVICE pointer to one
 *            double, written on the stream (the call does not synchronise).
 *   cuda_stream: cudaStream_t as void* (NULL = legacy default stream).
 * The first call on each device resolves the array's device address once;
 * make it before any stream capture. All calls share the array: calls whose
 * kernels overlap on the GPU race and give wrong results. Each call writes
 * every partial it reads, so no clearing between calls is needed.
 * Returns AMP_OK, AMP_ERR_ARG (null pointer, n_atoms < 1), AMP_ERR_TOO_LARGE
 * or AMP_ERR_CUDA. A CUDA error already pending on the calling thread (from an
 * earlier call) is left pending and the call returns AMP_ERR_CUDA without
 * launching; a launch error of this call is cleared and returned as
 * AMP_ERR_CUDA. */
#define AMP_ERR_TOO_LARGE (-7)
#define AMP_NOALLOC_MAX_ATOMS 1048576
int amp_polarization_energy_noalloc(int n_atoms, const double* mu, const double* E0, double* U,
                                    void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* AMOEBAPOL_H */
