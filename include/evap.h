/*
 * evap.h - C ABI of the GB300 matrix-free operators of the diffuse-interface evaporation model
 *          (Schreter-Fleischhacker et al., "A consistent diffuse-interface model for two-phase flow problems
 *          with rapid evaporation", arXiv 2401.07805).
 *
 * The library applies, cell by cell and without assembling matrices (Sec. 2.5: y = sum_i R_i^T A_i R_i x), the
 * finite element operators of the model on a uniform n^3 hexahedral mesh of [0, L]^3:
 *   - the linearized momentum operator for Q_p velocity (p = 2 or 3): mass/dt + Newton convection + viscous
 *     stress with the corrected rate of deformation (Eqs. modified_rate_of_deformation, modified_viscous_stress),
 *     with the reciprocal density (Eq. rhoEff) and arithmetic viscosity (Eq. muEff), plus the divergence row
 *     with the evaporation source (Eq. continuity, Eq. evaporDil; first line of Eq. weakNavierStokes);
 *   - the Q1 level-set advection (Crank-Nicolson, Eq. weakFormLevelSet) and reinitialization operators
 *     (Eq. reinitialization), driven by the transport velocity of Eqs. (transport_vel_local_continuous),
 *     (transport_vel_extension_liquid), (transport_vel_extension_gas) with the closest-point projection of App. C;
 *   - the adjoint of the momentum apply and a restarted GMRES solve with an FP32 inner operator and FP64
 *     iterative refinement.
 *
 * Conventions shared by every entry point
 *   Mesh:     n cells per axis, h = L / n.  Velocity (Q_p) nodes: M = p n + 1 per axis, N_u = M^3; pressure-space
 *             (Q1) nodes: N_p = (n + 1)^3; level-set / mass-flux (Q1) nodes on the level-set mesh (the velocity
 *             mesh subdivided n_sub times, cell size h / n_sub): N_phi = (n_sub n + 1)^3 (N_phi = N_p for n_sub = 1).
 *             Node index i + M (j + M k), i fastest (x), then y, then z.  Inside a cell the Q_p nodes sit at the
 *             Gauss-Lobatto points of [0, 1].  At a velocity quadrature point the level set is the Q1 interpolant of
 *             the level-set cell containing it (a point on a sub-cell face takes the upper sub-cell).
 *   Vectors:  component-major: v[c * N + node] for c = 0, 1, 2 (x, y, z components).
 *   Pointers: every array argument is a DEVICE pointer owned by the caller (e.g. a contiguous torch CUDA
 *             tensor).  The library keeps no reference to caller arrays after a call returns on the host:
 *             evap_set_fields copies its inputs into library-owned device memory.  Output arrays must not alias
 *             inputs.
 *   Streams:  `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  All work of a call is
 *             enqueued on that stream and the call returns without synchronizing, except where stated.
 *   Errors:   every function returns EVAP_OK (0) or a negative status; evap_status_string() names it and
 *             evap_last_error() returns the message of the most recent failure in the calling host thread.
 *             Arguments are validated before any work is enqueued; on EVAP_EINVAL nothing was enqueued.
 *   Precision: `prec` selects the arithmetic of an operator apply: 64 (x, y are double*) or 32 (float*).  The
 *             material law (Heaviside, density, viscosity, normal, dilation rate) is always evaluated in FP64
 *             (in evap_set_fields) and rounded to the apply precision.
 */
#ifndef EVAP_H
#define EVAP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct evap_mesh* evap_handle; /* opaque, owned by the library */

enum evap_status {
    EVAP_OK = 0,
    EVAP_EINVAL = -1,      /* null pointer, bad size, degree, mode or precision */
    EVAP_ECUDA = -2,       /* a CUDA call or kernel launch failed; evap_last_error() has the CUDA message */
    EVAP_ENOTCONV = -3,    /* solve hit its iteration cap; the last iterate and its residual are returned */
    EVAP_ENOFIELDS = -4,   /* an apply or solve was called before evap_set_fields */
    EVAP_ENOMEM = -5,      /* device allocation failed */
    EVAP_ENONFINITE = -6,  /* input checks on (evap_set_checks): an input array holds a NaN or an Inf; the check's
                              reduction was enqueued and synchronized, the call's own work was not */
    EVAP_ETIMEOUT = -7     /* a bounded device-side wait gave up (the grid barrier of a single-launch solver): the
                              kernel returned without finishing, the context stays usable, the output is undefined */
};

enum evap_levelset_mode {
    EVAP_ADVECT = 0,       /* y = (w, x) + theta dt (w, u_Gamma . grad x)                           Eq. weakFormLevelSet */
    EVAP_REINIT = 1,       /* y = (w, x)/dtau + eps (grad w . n, grad x . n)                     Eq. reinitialization */
    EVAP_REINIT_RHS = 2    /* y = (w, x)/dtau + (grad w, (1 - x^2)/2 n)   (explicit part, x = psi at pseudo-time 0) */
};

typedef struct {
    double rho_l, rho_g;   /* phase densities, reciprocal interpolation Eq. (rhoEff) */
    double mu_l, mu_g;     /* phase viscosities, arithmetic interpolation Eq. (muEff) */
    double eps;            /* interface thickness parameter, Eq. (initial_phi) */
    double dt;             /* time step of the level-set Crank-Nicolson operator */
    double c_mass;         /* mass coefficient of the momentum operator (1/dt; 1.5/dt is the BDF2 leading term) */
    double theta;          /* Crank-Nicolson weight (1/2) */
    double dtau;           /* reinitialization pseudo-time step, min(eps, dt) (Sec. 2.2.2) */
    int variant;           /* transport velocity: 1 local (Eq. transport_vel_local_continuous),
                              2 liquid extension (Eq. transport_vel_extension_liquid), 3 gas extension */
    int stress;            /* 0 standard Stokes (Eq. stokesLaw), 1 corrected (Eq. modified_viscous_stress) */
    int corr_zone;         /* 0: correction only in the interface zone 0 < H < 1 (Sec. 2.4.2); 1: everywhere */
    int newton;            /* 1: Newton linearization (x . grad) u0 included (App. D); 0: Picard */
    unsigned dirichlet_faces; /* velocity Dirichlet faces, bit 2a: x_a = 0, bit 2a+1: x_a = L (applies: homogeneous;
                                 data in evap_solve_saddle, evap_time_step) */
    double cpp_tol;        /* closest-point tolerance in cell units (App. C) */
    int cpp_kmax;          /* closest-point outer iteration cap (App. C) */
    double eta_n;          /* normal filter constant, Eq. (normal_vector_regularized): radius eta_n h^2 (default 2) */
    double eta_kappa;      /* curvature filter constant, Eq. (curvature_regularized) (default 2) */
    int n_sub;             /* level-set mesh: the velocity mesh subdivided n_sub times per direction (Sec. 2.5; 1 or 2,
                              0 reads as 1): the level set and the mass flux are Q1 on it, N_phi = (n_sub n + 1)^3
                              nodes; the pressure stays Q1 on the velocity mesh, N_p = (n + 1)^3 nodes */
} evap_params;

/* Create the mesh/operator object.  n_cells >= 1, degree_u in {2, 3}, L > 0, prm not NULL with rho_l, rho_g,
 * eps, dtau > 0, variant in {1,2,3}.  Allocates the library-owned device state of the current CUDA device
 * (fields, FP32 copies, quadrature-point coefficient table, transport velocity).  *out is set on success only. */
int evap_create_mesh(int n_cells, int degree_u, double L, const evap_params* prm, evap_handle* out);

/* Release all device memory of the handle (synchronizes the device). NULL is accepted and ignored. */
int evap_destroy(evap_handle h);

/* Number of Q_p velocity nodes (N_u; a velocity vector has 3 N_u entries) and of level-set nodes (N_phi). */
int evap_sizes(evap_handle h, int64_t* n_u, int64_t* n_phi);

/* Number of Q1 pressure nodes N_p (the space of the divergence row y_p, the pressure p and w_p). */
int evap_pressure_size(evap_handle h, int64_t* n_p);

/* Input checks (off by default): with on != 0 every later call first counts the NaN and Inf entries of its input
 * arrays (the fields of evap_set_fields, x / f / p / w / n / kappa / psi of the applies and solves) by one device
 * reduction, synchronizes the stream, and returns EVAP_ENONFINITE without doing its work if any is found. */
int evap_set_checks(evap_handle h, int on);

/* Deterministic accumulation (off by default).  With on != 0 the operator applies (evap_apply_momentum at both
 * precisions with its divergence row, the velocity-pressure apply, evap_apply_levelset, evap_apply_adjoint) and the
 * Jacobi diagonal of the solves add the cells' contributions in 8 passes, one per parity class of the cell
 * coordinates (cells of one class share no node), with plain loads and stores instead of atomic adds: every entry
 * is summed in a fixed order, so these results, and the iterates and iteration counts of evap_solve, are bitwise
 * reproducible from run to run.  Costs 8 launches per apply instead of one.  Section 2.5's y = sum_i R_i^T A_i R_i x
 * is the same sum in another order. */
int evap_set_deterministic(evap_handle h, int on);

/* Set the coefficient fields of the operators: phi [N_phi] (regularized level set, Eq. initial_phi; values are
 * clamped to [-1, 1]), u [3 N_u] (velocity about which the momentum operator is linearized; also the fluid
 * velocity of the transport velocity), mdot [N_phi] (evaporative mass flux, Eq. evaporDil).  Copies the fields,
 * evaluates the material law at every quadrature point of the interface cells (Eqs. heaviside, rhoEff, muEff,
 * normal_vector, delta, evaporDil) in FP64, and computes the transport velocity u_Gamma [3 N_phi] of the selected
 * variant (App. C closest-point projection for variants 2/3).  Synchronizes the stream twice (the sizes of the
 * interface-cell table and of the projection band are read back to size the work). */
int evap_set_fields(evap_handle h, const double* phi, const double* u, const double* mdot, void* stream);

/* Replace the transport velocity used by EVAP_ADVECT with caller data u_gamma [3 N_phi] (copied). */
int evap_set_transport_velocity(evap_handle h, const double* u_gamma, void* stream);

/* Copy the current transport velocity to u_gamma [3 N_phi] and the per-node closest-point flags to flags
 * [N_phi] (0 converged or not projected, 1 not converged; either pointer may be NULL).  If n_flagged is not NULL
 * the number of flagged nodes is written to it (host pointer; this synchronizes the stream). */
int evap_get_transport_velocity(evap_handle h, double* u_gamma, int32_t* flags, int64_t* n_flagged, void* stream);

/* Points whose fluid velocity the last transport-velocity pass took (evap_set_fields, evap_update_transport_velocity,
 * or the last fixed-point pass of evap_advect_levelset), y [3 N_phi] in physical coordinates, component-major: the
 * closest point on the isocontour d = 3 eps (variant 2) or d = -3 eps (variant 3) of every node of the projection
 * band (App. C; for a flagged node the last iterate), the node itself elsewhere and for variant 1.  Lets a caller
 * check each projection on its own terms.  Not meaningful after evap_set_transport_velocity. */
int evap_get_closest_points(evap_handle h, double* y, void* stream);

/* Recompute the transport velocity (variant of the parameters; App. C closest-point projection for variants 2/3)
 * from the fields of the last evap_set_fields, replacing any u_Gamma given by evap_set_transport_velocity.  The
 * same pass evap_set_fields runs; separate so that it can be rerun or timed alone.  Synchronizes the stream once. */
int evap_update_transport_velocity(evap_handle h, void* stream);

/* Statistics of the last closest-point pass, written to host pointers (any may be NULL; synchronizes the stream):
 * band_nodes = Q1 nodes that ran the projection, evaluations = point evaluations of phi_h and grad phi_h they made,
 * flagged = nodes whose iteration did not converge.  Variant 1 (no projection) reports zeros. */
int evap_transport_stats(evap_handle h, int64_t* band_nodes, int64_t* evaluations, int64_t* flagged, void* stream);

/* Momentum apply y = A x (velocity block of Eq. weakNavierStokes linearized about u, App. D):
 *   y_(i,c) = sum_q W_q [ N_i rho (c_mass x_c + (u . grad) x_c + newton (x . grad) u_c) + grad N_i . 2 mu eps_mod(x)_c ]
 * on unconstrained DoFs; on Dirichlet DoFs y = x and x does not enter other rows.  If y_p is not NULL the
 * divergence row y_p [N_p] = sum_q W_q N^1_j (div x - v_dil) is written too (same precision), with the dilation rate
 * v_dil = mdot (1/rho_g - 1/rho_l) delta (Eq. evaporDil with the sign of the paper's 1D solution, App. A
 * Eq. stefan_diffuse_velocity: evaporation, mdot > 0, expands the volume; the printed Eq. evaporDil has the bracket
 * reversed).
 * prec 64: x, y, y_p double*;  prec 32: float*.  x [3 N_u], y [3 N_u]. */
int evap_apply_momentum(evap_handle h, int prec, const void* x, void* y, void* y_p, void* stream);

/* Level-set apply y = A x on Q1 for the given mode (evap_levelset_mode); x, y [N_phi]; prec 64 or 32.
 * The normal n is grad phi / |grad phi| of the level set of evap_set_fields. */
int evap_apply_levelset(evap_handle h, int mode, int prec, const void* x, void* y, void* stream);

/* ---- level-set geometry sub-solver (steps 2 and 3 of Algorithm 2), FP64, homogeneous Neumann conditions ----
 * Each linear system is solved by conjugate gradients with the diagonal preconditioner to
 * |r| <= max(1e-12 |r_0|, 1e-20) (cap 1000 iterations; EVAP_ENOTCONV if not reached, results still written).
 * iters (total CG iterations) and relres (largest final |r|/|r_0|) are host pointers and may be NULL; these calls
 * synchronize the stream every few iterations. */

/* Projected normal n [3 N_phi] (component-major) of the level set of evap_set_fields, Eq. (normal_vector_regularized):
 * (M + eta_n h^2 K) n_c = (N_i, nbar_c), nbar = grad phi / |grad phi| at the point (Eq. normal_vector; zero where
 * |grad phi| h <= 1e-4). */
int evap_projected_normal(evap_handle h, double* n, int* iters, double* relres, void* stream);

/* Regularized curvature kappa [N_phi] of the Q1 normal field n [3 N_phi], Eqs. (curvature), (curvature_regularized):
 * (M + eta_kappa h^2 K) kappa = -(N_i, div n_h). */
int evap_curvature(evap_handle h, const double* n, double* kappa, int* iters, double* relres, void* stream);

/* Frozen normal of the reinitialization operators (EVAP_REINIT, EVAP_REINIT_RHS and evap_reinitialize): the nodal
 * field n [3 N_phi] (copied; normalized at each quadrature point, zero where |n_h| <= 1e-4), e.g. the projected
 * normal; n = NULL restores the unit normal grad phi / |grad phi| of the level set. */
int evap_set_levelset_normal(evap_handle h, const double* n, void* stream);

/* Reinitialization, Eq. (reinitialization) (Algorithm 2, step 2): psi [N_phi] holds psi^0 on entry and psi^steps on
 * return after `steps` semi-implicit pseudo-time steps (M/dtau + eps K_n) psi^(k+1) = M psi^k/dtau +
 * (grad N_i . n, (1 - (psi^k)^2)/2), n the frozen normal.  last_change (host, may be NULL) = |psi^steps -
 * psi^(steps-1)|_2. */
int evap_reinitialize(evap_handle h, double* psi, int steps, int* iters, double* last_change, void* stream);

/* Level-set advection, Eqs. (transport), (weakFormLevelSet) with Crank-Nicolson in time (Algorithm 2, step 1):
 * phi^n is the (clamped) level set of evap_set_fields; phi^(0) = phi^n and pass k computes the transport velocity of
 * clamp(phi^(k), -1, 1) (the mesh's variant, with the fields' u and mdot) and solves
 *   (M + theta dt C(u_Gamma)) phi^(k+1) = (M - (1 - theta) dt C(u_Gamma)) phi^n,  C_ij = sum_q W N_i u_Gamma . grad N_j,
 * by GMRES(30) with the diagonal preconditioner, started from phi^(k), to |r| <= max(1e-12 |b|, 1e-20) (b the
 * right-hand side: the residual of a zero start).  The fixed point
 * stops after max_iters passes or once |phi^(k+1) - phi^(k)|_2 <= tol (tol = 0: exactly max_iters passes).
 * phi [N_phi] (device) receives phi^(k) of the last pass (phi^n when max_iters = 0).  The mesh's level set stays
 * phi^n; its transport velocity (evap_get_transport_velocity, EVAP_ADVECT) is left as that of the last pass.
 * fp_iters, lin_iters (GMRES operator applications, summed) and last_change (|phi^(k) - phi^(k-1)|_2 of the last
 * pass) are host outputs and may be NULL.  Returns EVAP_ENOTCONV if a linear solve missed its tolerance (phi still
 * written), EVAP_EINVAL for max_iters < 0 or tol < 0. */
int evap_advect_levelset(evap_handle h, double* phi, int max_iters, double tol, int* fp_iters, int* lin_iters,
                         double* last_change, void* stream);

/* Surface-tension force f [3 N_u] of Eq. (surfaceTension) in the velocity test space (the right-hand side of the
 * momentum equation): f_(i,c) = sum_q W_q N_i alpha kappa_h n_c delta(phi) rho(phi) c_rho with the density-scaled
 * delta, c_rho = (rho_g - rho_l) / (rho_l rho_g ln(rho_g / rho_l)); kappa [N_phi] and n [3 N_phi] are Q1 fields (e.g.
 * from evap_curvature and evap_projected_normal; n is normalized at each point, zero where |n_h| <= 1e-4), phi is the
 * level set of evap_set_fields.  Dirichlet-constrained entries are 0.  EVAP_EINVAL if rho_l == rho_g. */
int evap_surface_tension(evap_handle h, const double* n, const double* kappa, double alpha, double* f, void* stream);

/* Adjoint of the momentum apply for L = w . A(phi, mdot, u) x + w_p . (B x - g(phi, mdot)):
 *   g_x = A^T w + B^T w_p,  g_u0 = dL/du [3 N_u],  g_phi = dL/dphi [N_phi],  g_mdot = dL/dmdot [N_phi],
 * with the quadrature-point coefficients of evap_set_fields and the chain-rule factors of the material law that
 * depend only on phi and mdot (tabulated by evap_set_fields at the points of the interface cells); x and w are
 * interpolated in the call.  w [3 N_u] and x [3 N_u] required; w_p [N_p] may be
 * NULL (no divergence row); any g_* may be NULL (not computed).  FP64 only. */
int evap_apply_adjoint(evap_handle h, const double* w, const double* w_p, const double* x, double* g_x,
                       double* g_u0, double* g_phi, double* g_mdot, void* stream);

/* Solve A x = f for the momentum operator with restarted GMRES(restart) and a right preconditioner: the
 * tensor-product mass inverse P = Sigma (Mx (x) My (x) Mz)^(-1) Sigma, Sigma = sqrt(diag(M) / diag(A)) on the free
 * DoFs (the 1D Q_p mass matrices of the uniform mesh; the identity on Dirichlet DoFs), which fits the operator's
 * dominant inertia term rho c_m M better than its diagonal alone.  mixed = 0: FP64 throughout; mixed = 1:
 * FP32 operator and Krylov basis inside FP64 iterative refinement (outer residual r = f - A x, norms and dot
 * products in FP64).  x holds the initial guess on entry and the solution on exit.  Stops when ||f - A x|| <=
 * rtol ||f|| (FP64 residual) or after max_iter operator applications.  iters_out (host, may be NULL): operator
 * applications used; relres_out (host, may be NULL): final ||f - A x|| / ||f||.  Synchronizes the stream.
 * Returns EVAP_ENOTCONV if the cap was reached. */
int evap_solve(evap_handle h, const double* f, double* x, int mixed, int restart, double rtol, int max_iter,
               int* iters_out, double* relres_out, void* stream);

/* Velocity-pressure system of Eq. (weakNavierStokes) with the Q1 pressure (Sec. 2.5, k_p = 1):
 *   y   = A x - B^T p   [3 N_u]  (the pressure term -(div v, p); Dirichlet-constrained rows: y = x)
 *   y_p = B x           [N_p]    (the divergence row without its source: the continuity equation is B x = g with
 *                                 g_j = sum_q W N1_j v_dil, Eq. continuity with the dilation rate of Eq. evaporDil)
 * A the momentum operator of evap_apply_momentum, B its divergence row (Dirichlet entries of x read as 0).
 * x [3 N_u], p [N_p], y, y_p device arrays, FP64; x and y must not alias.  Faces that are not Dirichlet
 * (dirichlet_faces) are open: the weak form's natural condition (zero traction) holds there. */
int evap_apply_saddle(evap_handle h, const double* x, const double* p, double* y, double* y_p, void* stream);

/* y = S~ x with S~ = B diag(A)^(-1) B^T, the Schur approximation of the velocity-pressure preconditioner (B the
 * divergence row, diag(A) the FP32 Jacobi diagonal of the momentum operator, the velocity DoFs of Dirichlet faces left
 * out), assembled as a symmetric 125-point stencil on the Q1 pressure lattice and applied in FP32 arithmetic.
 * x, y [N_p] device arrays, FP64.  Exposed to check the assembled operator against B diag(A)^(-1) B^T. */
int evap_apply_schur(evap_handle h, const double* x, double* y, void* stream);

/* Solve [A, -B^T; B, 0] [x; p] = [f; g] (g the continuity right-hand side of the fields) by flexible GMRES(restart)
 * with the block upper-triangular right preconditioner [A~, -B^T; 0, S~]: A~^(-1) a fixed budget of 14 FP32 GMRES
 * applications on A with the preconditioner of evap_solve, S~ = B diag(A)^(-1) B^T (an approximation of the Schur
 * complement B A^(-1) B^T that keeps the discrete B and so the pressure nodes of open faces) solved by 24 CG
 * iterations with its operator applied in FP32: the block-triangular preconditioner of Sec. 2.5 with its ILU velocity
 * block and its Cahouet-Chabard Schur approximation replaced.
 * Dirichlet data: the entries of f on the Dirichlet DoFs are the prescribed velocity there (0 for walls at rest, an
 * inflow otherwise); they are lifted, i.e. the system solved is K_D [x; p] = [f; g], whose constrained rows are x = f
 * and whose free rows keep the columns of the Dirichlet DoFs (A_ff x_f + A_fc f_c - B^T p = f_f, B_f x_f + B_c f_c = g);
 * with f = 0 there (homogeneous data) K_D is K.  The lifting costs one more velocity-pressure application and is
 * skipped when f vanishes on the Dirichlet DoFs.
 * x, p hold the initial guess on entry and the solution on exit.  Stops when ||b - K [x; p]|| <= rtol ||b|| (b the
 * lifted right-hand side, [f; g] for homogeneous data) or after max_iter operator applications; iters (host, may be
 * NULL): operator applications; relres (host, may be NULL): the final relative residual.  Synchronizes the stream.  EVAP_EINVAL if every face is Dirichlet (the pressure
 * level is then undetermined), restart outside [1, 255], rtol <= 0 or max_iter < 1; EVAP_ENOTCONV if the cap was
 * reached. */
int evap_solve_saddle(evap_handle h, const double* f, double* x, double* p, int restart, double rtol, int max_iter,
                      int* iters, double* relres, void* stream);

/* One time step of the coupled problem (the Navier-Stokes step, then Algorithm 2), for meshes with at least one open
 * face:
 *   1. the nonlinear velocity-pressure system [A(u), -B^T; B, 0] [u; p] = [f; g], A(u) the Picard operator (the
 *      momentum operator linearized about u without the Newton term), f_(i,c) = sum_q W N_i rho (c_m u*_c +
 *      gravity_c), with the Dirichlet data of u^n (the velocity on the Dirichlet faces keeps its value of u^n: walls
 *      at rest where it is 0, an inflow where it is not; lifted as in evap_solve_saddle, also in the nonlinear
 *      residual): BDF1 (u_prev NULL: c_m = 1/dt, u* = u^n) or BDF2 (u_prev = u^(n-1): c_m = 3/(2 dt),
 *      u* = (4 u^n - u^(n-1)) / 3); the mesh's c_mass is replaced by the scheme's for the step.  Nonlinear
 *      iterations from u^(0) = u^n, at most picard_iters of them, stopping before an iteration k >= 1 once the
 *      nonlinear residual R^(k) = [f; g] - K(u^(k)) [u^(k); p^(k)] has |R^(k)| <= picard_atol (the paper's
 *      Navier-Stokes nonlinear tolerance is 1e-10); each solve by evap_solve_saddle (restart 30, ns_rtol, at most 2000
 *      applications):
 *        mesh newton = 0, Picard: solve K(u^(k)) [u^(k+1); p^(k+1)] = [f; g] from the latest iterate; picard_iters = 1
 *          gives the semi-implicit step;
 *        mesh newton = 1, Newton (App. D): solve J(u^(k)) [du; dp] = R^(k) from zero with the Jacobian J, the operator
 *          with the Newton term (x . grad) u^(k), and add the correction (zero Dirichlet data);
 *      with alpha != 0 (surface tension coefficient) f also carries the force of evap_surface_tension with the
 *      projected normal and regularized curvature of phi^n;
 *   2. the advection fixed point (evap_advect_levelset, fp_iters passes, tol 0) with the transport velocity of
 *      u^(n+1), the result clamped to [-1, 1]; its projected normal; reinit_steps reinitialization steps with that
 *      normal frozen (evap_reinitialize), starting from the clamped field.
 * phi [N_phi], u [3 N_u], p [N_p]: device arrays holding the state at t^n on entry and at t^(n+1) on exit;
 * mdot [N_phi] device; gravity: host double[3] or NULL (no body force).  ns_iters / ns_relres (host, may be NULL):
 * operator applications of all velocity-pressure solves and the relative residual of the last; picard_res (host,
 * may be NULL): the last nonlinear residual evaluated (-1 if none, i.e. picard_iters = 1).  The call sets the fields
 * from its inputs first (as evap_set_fields) and leaves the mesh without fields afterwards (call evap_set_fields
 * before the next apply), with the unit-normal reinitialization operators restored.  Synchronizes the stream.
 * EVAP_EINVAL on dt <= 0, a closed box, alpha != 0 with rho_l == rho_g, picard_iters < 1, picard_atol < 0,
 * fp_iters < 1, reinit_steps < 0 or ns_rtol <= 0; EVAP_ENOTCONV if a sub-solve missed its tolerance (the step is still
 * completed). */
int evap_time_step(evap_handle h, double* phi, double* u, double* p, const double* mdot, const double* u_prev,
                   const double* gravity, double alpha, int picard_iters, double picard_atol, int fp_iters,
                   int reinit_steps, double ns_rtol, int* ns_iters, double* ns_relres, double* picard_res,
                   void* stream);

/* Diagonal of the momentum operator [3 N_u] (1 on Dirichlet DoFs; it sets the scale Sigma of evap_solve's
 * preconditioner), evaluated in FP32 arithmetic from the FP64 coefficient table and written as double. */
int evap_jacobi_diagonal(evap_handle h, double* diag, void* stream);

/* Allocation-free variant of evap_jacobi_diagonal, for callers that cannot let the library call cudaMalloc when
 * they need the diagonal: their device memory is owned by another allocator, or they must not let the library
 * synchronize the device (cudaMalloc/cudaFree may).  The paper has no counterpart.
 * Writes the same diagonal [3 N_u] (FP32 arithmetic, written as double, 1 on Dirichlet DoFs) into diag, accumulating
 * in a fixed 16 MiB array that is part of the library image on every GPU that loads it (held until exit).  Limit:
 * 3 N_u <= 4194304 (Q2 up to 55^3 cells, Q3 up to 36^3); larger meshes return EVAP_EINVAL.  The handle's device must be
 * current.  The first call on a device looks up that array's device address (cudaGetSymbolAddress); make that
 * first call before any stream capture.  The array keeps the last call's contents and is cleared at the start of
 * every call; calls that overlap on the GPU (other streams, other handles, other threads) race on it and must be
 * serialized by the caller.  Calls no cudaMalloc, cudaFree or allocating library routine. */
int evap_jacobi_diagonal_noalloc(evap_handle h, double* diag, void* stream);

/* Measured FMA throughput of the current device in TFLOP/s (prec 64: FP64, 32: FP32), *tflops a host pointer: about
 * 50 ms of independent FMA chains on every SM, timed with CUDA events after one warm-up launch (synchronizes the
 * stream).  The denominator of the roofline fractions of ALU-bound kernels.  The paper has no counterpart
 * (instrumentation). */
int evap_fma_probe(int prec, double* tflops, void* stream);

const char* evap_status_string(int status);
const char* evap_last_error(void);

/* Number of CUDA kernels this library has launched in the process so far (all handles, all threads); used to
 * count the kernels of a timed region.  The paper has no counterpart (instrumentation). */
int64_t evap_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* EVAP_H */
