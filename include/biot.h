/*
 * biot.h - C ABI of the GB300 space-time Biot poroelasticity library.
 *
 * The library applies and solves the monolithic space-time slab system of the
 * fully coupled Biot equations (Köcher, "Space-Time-Parallel Poroelasticity
 * Simulation"):
 *
 *   strong form (paper §Poroelasticity): quasi-static momentum with the
 *   effective stress C:eps(u) - b p I, Darcy's law eta K^{-1} q + grad p = 0 and
 *   the storage equation b d_t div u + (1/M) d_t p + div q = f (the volumetric
 *   mean stress substituted, so K_dr cancels from the operator);
 *   space (paper §Discretisation in Space): continuous Q2 displacement,
 *   Raviart-Thomas RT1 flux, discontinuous Q1 (DGQ1) pressure on a Cartesian
 *   quad/hex mesh;
 *   time (paper §Discretisation in Time): discontinuous Galerkin dG(r),
 *   r = 0, 1, 2, on slabs I_n = (t_{n-1}, t_n), Lagrange basis on the r+1
 *   right-Radau points (the last one is t_n, so the last temporal DoF is the
 *   end state U(t_n^-));
 *   slab system (paper §Monolithic Approach):
 *     calA X = (D (x) S + tau M_t (x) A_s) X = F + (phi(0) e_r^T (x) S) X_prev
 *   with A_s = [[A, 0, -bE], [0, Mq, -B^T], [0, B, 0]],
 *        S   = [[0, 0, 0], [0, 0, 0], [b E^T, 0, (1/M) Mp]];
 *   solver (paper §Monolithic Approach, §Preconditioning technology):
 *   restarted flexible GMRES, right-preconditioned by the time-spectral
 *   decomposition of M_t^{-1} D (real block form; the +-beta S couplings of a
 *   complex eigenvalue pair are kept through one block Gauss-Seidel sweep by
 *   default, or dropped as in the paper's "diagonal blockwise L_j" with
 *   opts.pair_coupling = -1) and a block-triangular fixed-stress
 *   preconditioner per block: flux-pressure block first with the
 *   displacement coupling replaced by (b^2/K_dr) Mp, then the displacement
 *   block by a geometric-multigrid V-cycle with Chebyshev-Jacobi smoothing.
 *
 * Vector layout.  A spatial vector ("one temporal level", length n_space) is
 *   [u_0 | .. | u_{d-1} | q_0 | .. | q_{d-1} | p]
 *   u_c : Q2 nodes, (2n_x+1) x (2n_y+1) [x (2n_z+1)], x fastest;
 *   q_c : 2n_c+1 Lagrange points {0,1/2,1} per cell along direction c, times
 *         the two Gauss points (1/2 -+ sqrt(3)/6) per cell across every
 *         other direction (2n_t), x fastest;
 *   p   : the 2 x 2 [x 2] Gauss points of every cell as one (2n_x) x (2n_y)
 *         [x (2n_z)] grid, x fastest.
 * A slab vector is r+1 spatial vectors back to back (time-major).
 * Essential (constrained) DoFs are identity rows of every operator; right-hand
 * sides must carry the prescribed value there (only homogeneous data is
 * supported: 0).
 *
 * Memory.  Unless stated otherwise, vector arguments are DEVICE pointers
 * owned by the caller, 8-byte aligned (FP64) or 4-byte aligned (FP32).  The
 * library allocates its own workspace in biot_setup (and, lazily, Krylov
 * bases on the first solve) and frees it in biot_destroy.  All GPU work is
 * enqueued on the given stream (a cudaStream_t passed as void*, NULL = the
 * legacy default stream); calls that report results on the host synchronise
 * that stream.
 *
 * Errors.  Every entry point returns BIOT_OK or a BIOT_E* code; no C++
 * exception crosses the ABI.  biot_last_error(ctx) gives a message for the
 * last failing call on that context.  On BIOT_ECUDA the context is left in an
 * unspecified but destroyable state.
 */
#ifndef BIOT_H
#define BIOT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  BIOT_OK = 0,
  BIOT_EINVAL = 1,      /* invalid argument (sizes, coefficients out of range, NULL) */
  BIOT_ENOMEM = 2,      /* device allocation failed */
  BIOT_ECUDA = 3,       /* a CUDA call failed */
  BIOT_ENOCONV = 4,     /* iteration limit reached before the tolerance */
  BIOT_EBREAKDOWN = 5,  /* non-finite value met in the Krylov iteration */
  BIOT_ETIMEOUT = 6     /* a bounded device-side wait ran out */
};

/* boundary condition codes per face, faces numbered 2*dir + side (side 0 = lower) */
enum { BIOT_U_NATURAL = 0, BIOT_U_DIRICHLET = 1, BIOT_U_ROLLER = 2 }; /* traction | all comps | normal comp */
enum { BIOT_F_NATURAL = 0, BIOT_F_NOFLOW = 1 };                      /* pressure | q.n = 0 essential      */

/* arithmetic of a call; BIOT_FIXED_STRESS selects (as a solve mode, FP64) the fixed-stress
 * iterative coupling of paper §Iterative Coupling Approach instead of the monolithic FGMRES:
 * sweeps of the flow solve with fixed volumetric mean stress followed by the deformation solve
 * with fixed pressure (the block preconditioner's sub-solves), each relaxed by the
 * residual-minimising factor; max_iters bounds the sweeps */
enum { BIOT_FP64 = 0, BIOT_FP32 = 1, BIOT_MIXED = 2, BIOT_FIXED_STRESS = 3 };

typedef struct biot_ctx* biot_t;

typedef struct {
  int dim;       /* 2 or 3 */
  int n[3];      /* cells per direction */
  double lo[3];  /* box corner */
  double hi[3];  /* box corner */
  int u_bc[6];   /* BIOT_U_* per face */
  int f_bc[6];   /* BIOT_F_* per face */
} biot_mesh;

/* Coefficients (paper §Poroelasticity): Biot coefficient 0 < b < 1, 1/M >= 0,
 * drained bulk modulus K_dr > 0 (enters only the fixed-stress preconditioner,
 * beta = b^2 / K_dr), Lame coefficients lambda >= 0, mu > 0 (isotropic C),
 * fluid viscosity eta > 0, and the isotropic permeability of every cell
 * (HOST array, length n_x n_y [n_z], lexicographic, x fastest, all > 0). */
typedef struct {
  double b, invM, K_dr, lambda, mu, eta;
  const double* K_cell;
} biot_coeffs;

typedef struct {
  int gmres_restart;    /* m (default 30) */
  int cheb_degree;      /* Chebyshev degree of the elasticity smoother (default 3, at most 128) */
  int schur_degree;     /* Chebyshev degree of the flux-pressure Schur solve (at most 128; 0 (default):
                           chosen per tau from the spectral bounds, see biot_schur_bounds) */
  int mg_min_cells;     /* stop coarsening at this many cells per direction (default 2) */
  double beta_fs;       /* fixed-stress parameter; <= 0 selects b^2 / K_dr */
  int flux_mass_exact;  /* flux-pressure block: 0 (default) replaces the Darcy mass by its diagonal;
                           1 inverts it exactly by line solves */
  int pair_coupling;    /* complex eigen-pair of the time matrix (r >= 1): 0 (default) applies one block
                           Gauss-Seidel sweep with the +-beta S coupling; -1 drops the coupling (the
                           paper's diagonal-blockwise L_j preconditioner) */
  int schur_mg;         /* flux-pressure Schur solve with the lumped Darcy mass: 1 one V-cycle of a
                           cell-centred multigrid (Gauss points aggregated per cell, then 2^d cells per
                           coarse cell); -1 Chebyshev-Jacobi of degree schur_degree; 0 (default) chooses:
                           the V-cycle in 2-D when the Lanczos estimate of cond(Dinv Schur) exceeds 600,
                           Chebyshev otherwise */
} biot_opts;

typedef struct {
  double tol;           /* relative true residual ||b - calA x|| / ||b|| (default 1e-10) */
  int max_iters;        /* total Krylov iterations (inner ones for MIXED), default 2000 */
  int mode;             /* BIOT_FP64, BIOT_MIXED or BIOT_FIXED_STRESS */
  double inner_tol;     /* MIXED: relative tolerance of each FP32 inner solve (default 1e-5) */
  int transpose;        /* 1: solve calA^T x = rhs (adjoint) */
} biot_solve_opts;

typedef struct {
  int iterations;       /* Krylov iterations (all inner iterations for MIXED; sweeps for BIOT_FIXED_STRESS) */
  int refinements;      /* MIXED: outer refinement steps */
  int restarts;
  double rel_residual;  /* final true relative residual (FP64) */
  double seconds;       /* wall time of the call (host clock, synchronised) */
} biot_stats;

/* Create a context for one mesh, coefficient set and time order r (0..2).
 * Builds the 1-D reference tables, the multigrid hierarchy (dense coarse
 * inverse in FP64) and the time-spectral transform on the current CUDA
 * device.  opts may be NULL (defaults).  Errors: EINVAL for dim not in {2,3},
 * n < 1, r not in 0..2, b not in (0,1), invM < 0, K_dr <= 0, mu <= 0,
 * lambda < 0, eta <= 0, any K_cell <= 0 or non-finite; ENOMEM; ECUDA. */
int biot_setup(const biot_mesh* mesh, const biot_coeffs* coeffs, int r, const biot_opts* opts, biot_t* out);

/* Batched context: nb independent instances of the same mesh, coefficients
 * and time order that differ only in their permeability fields (coeffs->K_cell:
 * HOST array of nb * n_cells values, instance-major) and their loads.  Every
 * kernel of the apply, preconditioner and solver covers all instances in one
 * launch (the instance is part of the launch grid) and every Krylov scalar is
 * kept per instance.  Vector layout of a batched slab vector: level-major,
 * the spatial vector of temporal level k of instance b starts at
 * (k * nb + b) * n_space (biot_sizes reports per-instance sizes).
 * biot_apply_slab and biot_precondition accept batched vectors; solves run in
 * BIOT_MIXED mode through biot_march_batch.  Requires the lumped Darcy mass
 * (opts->flux_mass_exact = 0).  Errors as biot_setup, EINVAL for nb outside
 * 1..4096.  (The paper solves one problem at a time; this serves many-instance
 * studies such as permeability sweeps.) */
int biot_setup_batch(const biot_mesh* mesh, const biot_coeffs* coeffs, int r, const biot_opts* opts, int nb, biot_t* out);

/* Host-side time tables of dG(r) (paper §Discretisation in Time, §Monolithic
 * Approach), no GPU needed: the r+1 right-Radau nodes on [0,1], the diagonal of
 * the slab mass M_t (Radau weights), phi_k(0), the jump-augmented derivative matrix
 * D (row-major), and the real block form of M_t^{-1} D = V Lambda V^{-1} that the
 * preconditioner uses: V, W = V^{-1} M_t^{-1}, the real part lam of the eigenvalue
 * owning each transformed component, the first component `pair` of the complex
 * pair (-1: none) and its imaginary part pair_beta (block [[a, b], [-b, a]]).
 * Any output may be NULL.  Errors: EINVAL for r outside 0..2. */
int biot_time_tables(int r, double* nodes, double* w, double* phi0, double* D, double* V, double* W, double* lam, int* pair,
                     double* pair_beta);

/* Sizes: DoFs per temporal level and per slab, number of cells (per instance). */
int biot_sizes(biot_t ctx, int64_t* n_space, int64_t* n_slab, int64_t* n_cells);

/* Replace the cellwise permeability (HOST array, n_cells, > 0). */
int biot_set_permeability(biot_t ctx, const double* K_cell);

/* Replace the cellwise permeability by its log-parametrisation K_c = K0 exp(g_c) (paper
 * §Poroelasticity: Darcy's law with the permeability K; the log field g is the variable of
 * biot_adjoint_grad's gradient).  g: HOST array, n_cells; EINVAL for K0 <= 0 or any
 * non-finite K_c. */
int biot_set_log_permeability(biot_t ctx, const double* g, double K0);

/* y = calA x (transpose = 0) or calA^T x (transpose = 1) for one slab of
 * length tau > 0 (paper §Monolithic Approach block system, applied matrix-free
 * in Kronecker form).  prec = BIOT_FP64: x, y are double*; BIOT_FP32: float*.
 * x and y must not overlap. */
int biot_apply_slab(biot_t ctx, double tau, const void* x, void* y, int prec, int transpose, void* stream);

/* Apply the slab preconditioner P ~ calA^{-1} (or P^T ~ calA^{-T}) once:
 * z = P r.  prec as in biot_apply_slab. */
int biot_precondition(biot_t ctx, double tau, const void* r, void* z, int prec, int transpose, void* stream);

/* Solve calA x = rhs (or calA^T x = rhs) for one slab (paper §Monolithic Approach: the
 * coupled system of all r+1 temporal DoFs solved at once; §Preconditioning technology:
 * GMRES, right-preconditioned by the time-spectral block-triangular fixed-stress
 * preconditioner).  rhs, x: double*, n_slab; x holds the initial guess on entry and the
 * solution on exit.  opts/stats may be NULL.  Returns EINVAL for a non-finite right-hand
 * side, ENOCONV (x = best iterate, finite) if max_iters is reached first, EBREAKDOWN on
 * non-finite values inside the iteration. */
int biot_solve_slab(biot_t ctx, double tau, const double* rhs, double* x, const biot_solve_opts* opts, biot_stats* stats,
                    void* stream);

/* Time marching over `slabs` slabs of (0, T] (paper §Discretisation in Time:
 * the discontinuous test space gives a slab-by-slab march).  The load is
 * F(x, t) = sum_m g_m(t) f_m(x) with nterms spatial load vectors f_terms[m]
 * (each n_space, assembled right-hand sides of one temporal level; constrained
 * entries are ignored) and polynomial time profiles
 * g_m(t) = tcoef[4m] + tcoef[4m+1] t + tcoef[4m+2] t^2 + tcoef[4m+3] t^3
 * (HOST array).  U0 (n_space) is the state at t = 0 (only u and p matter);
 * U_end (n_space) receives U(T^-).  f_terms, U0 and U_end may each be HOST or
 * DEVICE pointers (detected); host data is copied inside the call.  X_all,
 * if not NULL, is a DEVICE array of slabs * n_slab doubles receiving every
 * slab solution.  iters_per_slab (HOST, may be NULL) receives the Krylov
 * iterations of each slab. */
int biot_march(biot_t ctx, double T, int slabs, int nterms, const double* const* f_terms, const double* tcoef,
               const double* U0, double* U_end, double* X_all, const biot_solve_opts* opts, int* iters_per_slab,
               biot_stats* stats, void* stream);

/* Resumable march: slabs first .. first + count - 1 of the partition of (0, T] into `slabs`
 * slabs of length tau = T / slabs (paper §Discretisation in Time: the state carried from
 * one slab to the next is U(t_n^-) alone, so a march can stop after any slab and restart
 * from that state).  U_first (n_space, HOST or DEVICE) is U(t_first^-), U_end receives
 * U(t_{first+count}^-); loads, X_all (count * n_slab) and iters_per_slab (count) as in
 * biot_march, whose result equals, bitwise, a sequence of biot_march_resume calls that
 * covers the same slabs on the same context.  Errors: EINVAL unless
 * 0 <= first < first + count <= slabs, and for batched contexts. */
int biot_march_resume(biot_t ctx, double T, int slabs, int first, int count, int nterms, const double* const* f_terms,
                      const double* tcoef, const double* U_first, double* U_end, double* X_all, const biot_solve_opts* opts,
                      int* iters_per_slab, biot_stats* stats, void* stream);

/* Marches every instance of a batched context (biot_setup_batch) over the same
 * `slabs` slabs of (0, T] (paper §Discretisation in Time), all instances in
 * lockstep: one batched right-hand side, one batched mixed-precision solve per
 * slab.  f_terms holds nb * nterms pointers (instance b's term m at
 * f_terms[b * nterms + m], n_space each, HOST or DEVICE); the time profiles
 * tcoef (4 * nterms, HOST) are shared.  U0 (nb pointers, or NULL for zero
 * initial states; entries may be NULL) and U_end (nb pointers) are per-instance
 * states of n_space entries, HOST or DEVICE.  iters, stats and status (HOST,
 * nb entries each, may be NULL) receive each instance's total Krylov
 * iterations, statistics and return code; the call returns BIOT_OK or the
 * first failing code.  Only BIOT_MIXED solves (opts->mode) are batched; a
 * context with nb = 1 marches as biot_march. */
int biot_march_batch(biot_t ctx, double T, int slabs, int nterms, const double* const* f_terms, const double* tcoef,
                     const double* const* U0, double* const* U_end, const biot_solve_opts* opts, int* iters,
                     biot_stats* stats, int* status, void* stream);

/* Adjoint gradient of J = j^T U(T^-) with respect to the cellwise
 * log-permeability g_c (K_c = K0 exp(g_c)): the dual problem marched backwards
 * over slabs with the transposed slab operator, the forward slab solutions
 * recomputed from end-state checkpoints (recompute = 1) or kept from the
 * forward pass (recompute = 0).  j_goal (DEVICE, n_space) is the goal
 * weight vector (see biot_goal_mean_pressure); the load is as in biot_march.
 * J_out (HOST) receives J; dJ_dlogK (DEVICE, n_cells) receives the gradient. */
int biot_adjoint_grad(biot_t ctx, double T, int slabs, int nterms, const double* const* f_terms, const double* tcoef,
                      const double* U0, const double* j_goal, const biot_solve_opts* opts, int recompute, double* J_out,
                      double* dJ_dlogK, void* stream);

/* Goal-oriented estimate of the time-discretisation error (paper §Abstract:
 * goal-oriented, duality-based adaptivity) of J = j^T U(T^-) for the dG(r)
 * march of `ctx` against dG(r+1) (`ctx_r1`: same mesh, boundary codes and
 * coefficients, time order r + 1).  The dG(r) slab solutions are embedded into
 * the dG(r+1) slab system (a degree-r polynomial is a degree-(r+1) one) and their
 * residuals are weighted with the dG(r+1) dual solution; eta_slab (HOST, slabs
 * entries, may be NULL) receives the slab indicators eta_n, eta_out (HOST) their
 * sum, which equals J(U_{r+1}) - J(U_r) up to the solver tolerances, and J_out
 * (HOST) J(U_r).  Loads, U0 and j_goal as in biot_adjoint_grad; opts->mode as in
 * biot_march (the dual solves use the transposed operator).  Allocates its
 * temporaries (slabs + 1 states and every dG(r) slab solution) per call.  Errors:
 * EINVAL for batched contexts, mismatched contexts or bad arguments. */
int biot_dwr_time_estimate(biot_t ctx, biot_t ctx_r1, double T, int slabs, int nterms, const double* const* f_terms,
                           const double* tcoef, const double* U0, const double* j_goal, const biot_solve_opts* opts,
                           double* eta_slab, double* eta_out, double* J_out, void* stream);

/* Batched marches: `count` independent instances, each with its own mesh,
 * coefficients (K_cell on the host), time order r, horizon T and slab count, and
 * either a built-in load (load_kind >= 0: one BIOT_LOAD_* preset of magnitude
 * load_value, constant in time) or explicit load terms as in biot_march
 * (load_kind = -1).  U0 / U_end (n_space each, host or device, may be NULL) are
 * the instance's initial and end states.  Instances that share everything but
 * the permeability and the load (mesh, boundary codes, coefficients, r, T,
 * slabs, time profiles) form a group; with sopts->mode = BIOT_MIXED every group
 * of two or more is solved as one batched context (biot_setup_batch /
 * biot_march_batch: all its instances in every launch), at most `workers`
 * instances per context (<= 0: 64).  Other instances (FP64 mode, groups of one,
 * the 2-D manufactured presets, whose load depends on the instance's
 * permeability) are marched one by one with a context cache keyed by shape.
 * status[i] and stats[i] (host arrays, may be NULL) receive each instance's
 * return code and statistics; the call returns BIOT_OK or the first failing
 * code.  (The paper solves one problem at a time; batching serves the
 * many-instance studies its space-time method targets, e.g. parameter sweeps.) */
typedef struct {
  biot_mesh mesh;
  biot_coeffs coeffs;
  int r;
  double T;
  int slabs;
  int load_kind;
  double load_value;
  int nterms;
  const double* const* f_terms;
  const double* tcoef;
  const double* U0;
  double* U_end;
} biot_batch_item;
int biot_solve_batch(const biot_batch_item* items, int count, const biot_opts* opts, const biot_solve_opts* sopts,
                     int workers, int* status, biot_stats* stats);

/* Goal weight vector of J = mean pressure over the box [lo, hi] (exact
 * integration of the DGQ1 pressure over the clipped cells), written to the
 * DEVICE array j (n_space; zero outside the pressure block). */
int biot_goal_mean_pressure(biot_t ctx, const double* lo, const double* hi, double* j, void* stream);

/* Built-in spatial load vectors (one temporal level, DEVICE output, n_space):
 *  BIOT_LOAD_TRACTION_TOP  : traction -value * n on the upper face of the last
 *                            direction (compressive load of magnitude value);
 *  BIOT_LOAD_MMS2D_CONST   : time-constant part of the 2-D manufactured load
 *                            (source b pi sin(pi(x+y)) + (1/M) cos(pi x)cos(pi y));
 *  BIOT_LOAD_MMS2D_LINEAR  : part linear in t (body force, source and the
 *                            natural-pressure boundary term) of the manufactured
 *                            solution u = (S t, S t), p = cos(pi x)cos(pi y) t. */
enum { BIOT_LOAD_TRACTION_TOP = 0, BIOT_LOAD_MMS2D_CONST = 1, BIOT_LOAD_MMS2D_LINEAR = 2 };
int biot_load_preset(biot_t ctx, int kind, double value, double* f, void* stream);

/* Diagnostics: apply one piece of the slab preconditioner to a single spatial
 * vector (n_space entries, double* for BIOT_FP64, float* for BIOT_FP32); the
 * blocks a piece does not produce are zero in `out`.
 *   BIOT_PART_FLUX_MASS_INV: out_q = (tau Mq)^{-1} in_q on free flux DoFs (exact,
 *                            by line solves), out_q = in_q on no-flow DoFs;
 *   BIOT_PART_SCHUR:        out_p = ((1/M + beta) Mp + tau B Mq^{-1} B^T) in_p, the
 *                            flux-pressure Schur complement of the dG(0)-type block
 *                            with lambda = 1 and the fixed-stress term beta Mp;
 *   BIOT_PART_VCYCLE:       out_u = one multigrid V-cycle for tau A x = in_u from x = 0;
 *   BIOT_PART_ELASTICITY:   out_u = tau A in_u (constrained rows identity);
 *   BIOT_PART_SCHUR_STEP:   out_p = in_p - diag(Shat)^{-1} Shat in_p with Shat the lumped-Darcy-mass
 *                            BIOT_PART_SCHUR operator: one step of the flux-pressure Chebyshev-Jacobi
 *                            kernel the solver runs (weights 0 and 1, zero right-hand side); EINVAL for
 *                            batched contexts and flux_mass_exact = 1. */
enum { BIOT_PART_FLUX_MASS_INV = 0, BIOT_PART_SCHUR = 1, BIOT_PART_VCYCLE = 2, BIOT_PART_ELASTICITY = 3,
       BIOT_PART_SCHUR_STEP = 4 };
int biot_apply_part(biot_t ctx, int part, double tau, const void* in, void* out, int prec, void* stream);

/* Allocation-free flux-pressure Schur apply, for callers that cannot call
 * cudaMalloc where they need it (a caching allocator that has reserved the whole
 * device, latency-critical loops that cannot afford cudaMalloc's implicit
 * device-wide synchronisation, embedded or real-time hosts that forbid device
 * allocation after start-up).  The paper has no counterpart: this is an interface
 * variant of biot_apply_part(BIOT_PART_SCHUR) with the default lumped Darcy mass,
 *   out_p = ((1/M + beta) Mp + tau B diag(Mq)^{-1} B^T) in_p,  other blocks of out = 0,
 * on spatial vectors (n_space doubles, DEVICE).  Its flux-grid scratch lives in a
 * static device array of 2^20 doubles (8 MiB, held by every GPU that loads the
 * library until the process exits); meshes with more flux DoFs are rejected with
 * BIOT_EINVAL.  The first call on a device looks up that array's device address
 * (once per device, with that device current; with CUDA's lazy module loading the
 * driver also materialises the array at that moment); make that first call before
 * any stream capture.  All calls share the array: calls that overlap on the GPU (other
 * streams or devices' threads racing on one device) race on it.  The context must
 * have been created by biot_setup (EINVAL for batched contexts of biot_setup_batch) with
 * the default lumped Darcy mass (EINVAL when opts->flux_mass_exact = 1); this call itself
 * allocates nothing. */
int biot_schur_apply_noalloc(biot_t ctx, double tau, const double* in, double* out, void* stream);

/* Tracing.  biot_profile(ctx, 1) makes every launch of the displacement-row
 * operator kernel (the elasticity apply, the dominant kernel of the solver)
 * record a pair of CUDA events on its launching stream; biot_counters returns
 * the number of kernels this process has launched through the library so far
 * (launches; a replayed CUDA graph counts its kernel nodes; setting the
 * environment variable BIOT_NO_GRAPHS=1 before biot_setup disables graphs),
 * and the number and summed device time in milliseconds of the
 * operator launches recorded since the previous call (op_launches, op_ms;
 * synchronises on those events, then forgets them).  Either output may be NULL. */
int biot_profile(biot_t ctx, int enable);
int biot_counters(biot_t ctx, int64_t* launches, int64_t* op_launches, double* op_ms);

/* Per-kernel tracing detail (after biot_profile(ctx, 1)): for kind
 * BIOT_KERNEL_ELASTICITY_FP32 (displacement-row operator in FP32: the z-marching kernel on
 * 3-D grids of 1e5 nodes or more, the 2-D kernel), BIOT_KERNEL_ELASTICITY_FP32_COARSE (the
 * FP32 3-D operator on grids below 1e5 nodes), BIOT_KERNEL_ELASTICITY_FP64 and
 * BIOT_KERNEL_SCHUR_FP32 (one Chebyshev step of the flux-pressure Schur solve),
 * the number of launches recorded since the last query, their summed device time
 * in ms (CUDA events on the launching stream) and their summed work units (Q2 node
 * x right-hand side for the elasticity operator, Gauss pressure point x
 * right-hand side for the Schur step).  Synchronises on the events, then forgets
 * them.  With profiling on, CUDA graphs are not used. */
enum {
  BIOT_KERNEL_ELASTICITY_FP32 = 0,
  BIOT_KERNEL_ELASTICITY_FP64 = 1,
  BIOT_KERNEL_SCHUR_FP32 = 2,
  BIOT_KERNEL_ELASTICITY_FP32_COARSE = 3
};
int biot_kernel_stats(biot_t ctx, int kind, int64_t* launches, double* ms, double* units);

/* Measured arithmetic peak of the CUDA cores on the current device: a kernel of
 * independent fused multiply-add chains (prec = BIOT_FP32 or BIOT_FP64) over every SM,
 * calibrated to run about 60 ms and timed with CUDA events on `stream`.  tflops
 * (HOST, may be NULL) receives the achieved TFLOP/s (2 flop per FMA), ms the duration of
 * the timed launch.  The paper has no counterpart: this is the denominator against which
 * the operator kernels' FP32 and FP64 arithmetic rates are reported.  No context needed;
 * allocates nothing.  Errors: EINVAL for another prec, ECUDA. */
int biot_fma_peak(int prec, double* tflops, double* ms, void* stream);

/* Spectral bounds of the Jacobi-scaled lumped Schur complement D^{-1} Shat of this tau, the
 * operator whose inverse the flux-pressure block of the preconditioner approximates
 * (paper §Preconditioning; Shat = cm Mp + tau B diag(Mq)^{-1} B^T, cm the storage
 * coefficient of each temporal level).  They come from 30 FP64 Lanczos steps on every
 * temporal level (cached per tau; the first call for a tau allocates the FP64
 * preconditioner workspace).  bounds (HOST, 4 doubles): the smallest and largest Ritz values
 * (over all temporal levels), then the interval [lo, hi] the Chebyshev-Jacobi solve is built
 * on.  degree (HOST, may be NULL): the Chebyshev degree the solve uses for this tau, 0 when
 * the cell-centred multigrid replaces it.  Errors: EINVAL (NULL bounds, tau <= 0), ECUDA. */
int biot_schur_bounds(biot_t ctx, double tau, double* bounds, int* degree, void* stream);

/* Launch-shape tuning table.  The first FP32 solve of a context times every run length
 * (planes per block) of the z-marching elasticity kernel on each multigrid level that uses
 * it, for each column count the solver launches, with CUDA events on the solve's stream, and
 * keeps the fastest; every candidate produces bitwise-identical results, so the choice
 * changes only the time.  Results persist in a JSON object {"key": value} in the file
 * $BIOT_TUNE_CACHE, else $XDG_CACHE_HOME/biot_gb300/tune.json, else
 * $HOME/.cache/biot_gb300/tune.json (read once per process, rewritten atomically on every
 * new entry; an unreadable or malformed file is ignored).  Environment BIOT_TUNE=0 turns the
 * measurement off (a stored value is still used; without one the kernel's heuristic applies).
 * Keys have the form "elast3_zrun|<device>_sm<SMs>|<nx>x<ny>x<nz>|cols<c>" (node counts).
 * These three calls touch only the host table and the file (no GPU, no context):
 * biot_tune_get returns the stored value of `key` or -1; biot_tune_put stores `value` under
 * `key` (EINVAL for an empty key or one with '"' or '\\'); biot_tune_cache_path writes the
 * file's path into buf (HOST, len bytes; EINVAL when it does not fit). */
int biot_tune_get(const char* key);
int biot_tune_put(const char* key, int value);
int biot_tune_cache_path(char* buf, int len);

const char* biot_last_error(biot_t ctx);
void biot_destroy(biot_t ctx);

#ifdef __cplusplus
}
#endif

#endif /* BIOT_H */
