/*
 * natconv.h — C ABI of the GB300 (sm_103a) library for the stabilised Darcy–Boussinesq
 * natural-convection state solve, its adjoint and the design sensitivities of
 * Pollini, Sigmund, Andreasen & Alexandersen, arXiv 1904.00182.
 *
 * Model (Sec. 2.2, Eq. goveq): Darcy velocity u = -kappa/mu (grad P + rho0 alpha g T)
 * (Eq. finaldarcy) substituted into continuity, coupled to the convection-diffusion of T.
 * Unknowns: P and T at every node of a structured grid of cubic trilinear (Q1) elements
 * (Sec. 2.2: "the number of DOFs is reduced to only 2"), discretised with the SUPG
 * Petrov–Galerkin weak form of App. A (Eq. weakstable, Eq. finalsyseq R(s) = M(s) s - f).
 * The design field gamma (one value per element, 1 = solid, 0 = fluid, Sec. 2.2) is
 * regularised by a PDE filter (Sec. 5.1) and mapped to permeability and conductivity by RAMP
 * (Sec. 5.2, Eqs. condRAMP, permRAMP). The state solve is a damped Newton method whose
 * damping minimises ||R|| (Sec. 5.4); the objective gradient comes from an adjoint solve
 * (Sec. 5.1). Linear systems: flexible GMRES (Sec. 5.4, Table 4) preconditioned by a
 * geometric multigrid V-cycle (this library's design; the paper defers the preconditioner).
 *
 * Set-up used by every problem (synthetic heated base plate):
 *   box nx*h x ny*h x nz*h, gravity along -z; the bottom `heated_layers` element layers are a
 *   solid, non-design heat source region Omega_h (Sec. 2.2) with uniform source Q; P = 0 and
 *   T = 0 on the top face z = nz*h; every other face carries zero normal flux of fluid and
 *   heat (natural conditions q_u = q_h = 0 of Eq. goveq's boundary conditions).
 *
 * Data layout (all arrays FP64, C order):
 *   node (i,j,k), 0<=i<=nx, 0<=j<=ny, 0<=k<=nz, has index n = i + (nx+1)*(j + (ny+1)*k);
 *   element (i,j,k), 0<=i<nx, ..., has index e = i + nx*(j + ny*k);
 *   a "state vector" is 2*N doubles, node-interleaved pairs (P_n, T_n), N = number of nodes;
 *   design arrays are E doubles; velocities are 3*E doubles (u_x,u_y,u_z per element).
 *
 * Pointers: every array argument may point to host memory (pageable or pinned) or to
 * device memory of the problem's device: the library copies with unified addressing.
 * Arguments are borrowed for the duration of the call only. The library owns all of its
 * device workspace (allocated in nc_create_problem, freed in nc_destroy_problem).
 *
 * Streams and threads: each problem runs its work on the CUDA stream given at creation
 * (NULL = a stream the library creates). Every call returns after its work has finished.
 * Calls on one problem must not overlap; calls on different problems may run concurrently
 * from different host threads and then overlap on the device.
 *
 * Errors: every call returns an nc_status and never aborts or traps on the device. On
 * failure, nc_last_error() returns a message for that problem. The call order
 * set_design -> solve_state -> solve_adjoint -> sensitivities is enforced (NC_ERR_STATE).
 */
#ifndef NATCONV_H
#define NATCONV_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NC_OK = 0,
  NC_ERR_ARG = 1,      /* invalid argument (sizes, NaN or out-of-range design values ...) */
  NC_ERR_OOM = 2,      /* device allocation failed */
  NC_ERR_CUDA = 3,     /* a CUDA runtime call or kernel launch failed */
  NC_ERR_DIVERGED = 4, /* Newton found no damping factor that reduces ||R||, after source ramping */
  NC_ERR_MAXIT = 5,    /* iteration limit reached before the tolerance */
  NC_ERR_NAN = 6,      /* a non-finite residual or Krylov quantity appeared */
  NC_ERR_TIMEOUT = 7,  /* the call exceeded params.timeout_s of wall-clock time */
  NC_ERR_STATE = 8     /* call order violated (e.g. solve_state before set_design) */
} nc_status;

enum { NC_PREC_MIXED = 0, NC_PREC_FP64 = 1 };
/* Arithmetic of the outer residuals on the mixed-precision path (nc_params.outer_arith). */
enum { NC_ARITH_DF64 = 0, NC_ARITH_FP64 = 1 };
/* Krylov basis storage on the mixed-precision path (nc_params.krylov_basis). */
enum { NC_BASIS_FP64 = 0, NC_BASIS_FP32 = 1 };
/* Objectives: the mean temperature over the heated region (Galerkin weights; equal to the thermal
 * compliance of Eq. objfunc when the total power is 1), or the discrete thermal compliance of
 * Eq. objdiscr, sum_e f_tQ,e^T t_e, whose SUPG-weighted source load depends on the state. */
enum { NC_OBJ_MEAN_T_HEATED = 0, NC_OBJ_SUPG_COMPLIANCE = 1 };

/* Boundary conditions (nc_params.bc). NC_BC_TOP: P = T = 0 on the top face z = nz h, every other face
 * natural (no flux, no normal Darcy flow). NC_BC_CAVITY: the quarter of a closed cavity with symmetry
 * planes x = 0 and y = 0 (Sec. 6.1): T = 0 on the outer walls x = nx h, y = ny h and the top, the
 * bottom insulated, no normal flow through any face, and P = 0 at the top outer corner. */
enum { NC_BC_TOP = 0, NC_BC_CAVITY = 1 };

/* Shape of the heated and design regions (nc_params.region_shape). NC_REGION_BOX: boxes at the corner
 * x = y = 0 (heat_nx ..., design_nx ...). NC_REGION_CYLINDER (the suspended cylinder of Sec. 7): the
 * heated region is the cylinder of radius heat_radius around the z axis through that corner, over the
 * element layers [heat_z0, heat_z0 + heated_layers); the design region is the annulus out to
 * design_radius over the same layers. An element belongs to a region when its centroid does; radii
 * are in element sizes. */
enum { NC_REGION_BOX = 0, NC_REGION_CYLINDER = 1 };

/* Operator of the multigrid's finest level on the NC_PREC_MIXED path (nc_params.mg_op0). The outer
 * FGMRES is flexible (Sec. 5.4), so its preconditioner may apply another operator than J.
 * NC_MGOP_EXACT: the exact Newton Jacobian J(s) (FP32). NC_MGOP_PICARD: the frozen-coefficient
 * operator: the continuity rows of J; energy rows sum_q w [N*_a rho0 c_p u0 . grad dT + k grad N_a .
 * grad dT] with the element's centroid velocity u0 and tau frozen at s (no derivatives of u, u0 or
 * tau, no dP coupling): about 40 % of the arithmetic of J. The Krylov operator stays exact. */
enum { NC_MGOP_EXACT = 0, NC_MGOP_PICARD = 1 };

/* Smoothers of the multigrid levels below the finest (their operators are assembled 27-point stencils of
 * 2x2 blocks). NC_SMOOTH_BLOCK_JACOBI: damped 2x2 block Jacobi, x += omega D^-1 (b - A x).
 * NC_SMOOTH_ZLINE: damped z-line block Jacobi, x += omega T^-1 (b - A x), with T the block-tridiagonal
 * part of A that couples each node column (fixed i, j) in z with itself, factored once per set-up;
 * aimed at convection along the buoyancy direction z. */
enum { NC_SMOOTH_BLOCK_JACOBI = 0, NC_SMOOTH_ZLINE = 1 };

/* Inner solver of the PDE filter's Helmholtz system (Sec. 5.2), inside FP64 iterative refinement.
 * NC_FILTER_SPECTRAL: a direct FP32 solve in the cosine basis of each axis, which diagonalises the
 * 1D Q1 stiffness and mass matrices with Neumann ends (six dense FP32 transforms through cuBLAS and
 * one scaling per solve). NC_FILTER_CHEBYSHEV: Jacobi-preconditioned FP32 Chebyshev iterations. */
enum { NC_FILTER_SPECTRAL = 0, NC_FILTER_CHEBYSHEV = 1 };

typedef struct nc_problem nc_problem;

typedef struct {
  int nx, ny, nz; /* elements per direction, each >= 1 */
  double h;       /* element edge length (> 0) */
} nc_grid;

/* Parameters; nc_default_params() fills the defaults shown in brackets. */
typedef struct {
  double alpha;         /* thermal expansion coefficient (Sec. 2.1) [1e3] */
  double kappa_f;       /* fluid permeability; <= 0: Eq. nusselt5 with dT = tune_dT, H = 1,
                           L = 0.5 and unit fluid properties (Sec. 3) [0] */
  double tune_dT;       /* dT used by Eq. nusselt5 when kappa_f <= 0 [1] */
  double kappa_ratio;   /* kappa_s / kappa_f [1e-6] */
  double k_f, k_s;      /* fluid and solid conductivity (Sec. 6.1) [1, 100] */
  double q_c, q_p;      /* RAMP penalties of Eqs. condRAMP / permRAMP (Sec. 6.2) [8.81, 8] */
  double Q;             /* heat source in Omega_h; <= 0: total power 1 [0] */
  int heated_layers;    /* element layers of Omega_h at the bottom [2] */
  double rho0, mu, cp, g; /* reference density, viscosity, heat capacity, |g| (Sec. 6.1) [1] */
  double filter_radius; /* PDE filter radius in element sizes (Sec. 6.3) [2.5] */
  double newton_rtol;   /* stop when ||R_free(s)|| <= newton_rtol * ||R_free(0)|| [1e-8] */
  int newton_maxit;     /* [50] */
  double krylov_rtol;   /* upper bound of the FGMRES relative tolerance per Newton step [1e-2] */
  int krylov_maxit;     /* FGMRES iterations per linear solve [300] */
  int restart;          /* FGMRES restart length, <= 64 [30] */
  int precision;        /* NC_PREC_MIXED (FP32 multigrid preconditioner and Krylov operator; Newton
                           residual, adjoint residual and sensitivities in outer_arith, Krylov
                           orthogonalisation in krylov_basis, coarse-grid residual, Hessenberg and
                           Newton update in FP64) or NC_PREC_FP64 (IEEE FP64 throughout) [MIXED] */
  int mg_levels;        /* 0: coarsen while every dimension is even [0] */
  int nu_pre, nu_post;  /* smoothing sweeps; the first pre-sweep starts from x = 0 [1, 2] */
  double omega;         /* damping of the block-Jacobi smoother [0.9] */
  double filter_rtol;   /* relative residual tolerance of the filter solve; on NC_PREC_MIXED with
                           filter_rtol >= 1e-13 its refinement runs in double-float (about 48
                           significant bits), otherwise in FP64 [1e-12] */
  double timeout_s;     /* wall-clock limit of one call [600] */
  double adjoint_rtol;  /* adjoint stops at ||df/ds - J^T lambda|| <= adjoint_rtol ||df/ds||;
                           <= 0: the state's newton_rtol [0] */
  int coarse_refactor;  /* when the coarsest multigrid matrix is inverted anew: 1 at every set-up; 0 at
                           the first set-up of each solve call; 2 only once per problem. Later set-ups
                           keep the inverse and the coarse solve's FP64 refinement step against the
                           current matrix corrects for the change [0] */
  double krylov_eta_min; /* lower bound of the Newton forcing term; <= 0: 1e-12 [0] */
  double adjoint_eta_first; /* FGMRES tolerance of the first adjoint refinement pass; <= 0: 1e-5 with
                               NC_PREC_MIXED, the adjoint tolerance with NC_PREC_FP64 [0] */
  int mg_tail_nodes;    /* the multigrid levels below the finest with at most this many nodes, down
                           to the coarsest, run as one fused kernel on a thread-block cluster (the
                           same arithmetic as separate launches); 0: separate launches, the faster
                           choice measured on GB300 (the fused kernel's cluster barriers between its
                           steps cost more than the launches they save) [0] */
  double mg_reuse_below; /* a Newton step whose relative residual is at most this keeps the multigrid
                            hierarchy of the previous step (lagged preconditioner); 0: rebuild at
                            every step [1e-2] */
  int outer_arith;      /* NC_PREC_MIXED only: arithmetic of the Newton residual, the adjoint
                           refinement residual J^T lambda and the sensitivities. NC_ARITH_FP64: IEEE
                           FP64; NC_ARITH_DF64: double-float (hi + lo pairs of floats, about 48
                           significant bits, on the FP32 units; inputs and outputs FP64) [FP64] */
  int krylov_basis;     /* NC_PREC_MIXED only, fixed at creation: FGMRES basis vectors and their
                           Gram-Schmidt in NC_BASIS_FP64 or NC_BASIS_FP32 (FP32 products, FP64 sums
                           across threads) [FP64] */
  double krylov_reorth; /* classical Gram-Schmidt takes a second pass when the first kept less than
                           this fraction of ||w||^2 (1/2: the DGKS test; 1: always); <= 0: the
                           default of the basis type [0] */
  int adjoint_df64_steps; /* NC_PREC_MIXED with outer_arith = NC_ARITH_FP64: an adjoint refinement
                           residual df/ds - J^T lambda that is not expected to meet the tolerance
                           (previous relative residual times the last FGMRES reduction above
                           10 x the tolerance) only steers the next correction and is computed in
                           double-float; every residual that accepts lambda is IEEE FP64 (a
                           double-float one inside the tolerance is recomputed in FP64 first).
                           0: every refinement residual in FP64 [1] */
  int bc;               /* NC_BC_TOP or NC_BC_CAVITY, fixed at creation [NC_BC_TOP] */
  int heat_nx, heat_ny; /* heated region (passive solid holding the source Q): the element box
                           [0, heat_nx) x [0, heat_ny) x [0, heated_layers); 0: the full extent [0, 0] */
  int design_nx, design_ny, design_nz; /* design region: [0, design_nx) x [0, design_ny) x
                           [heated_layers, heated_layers + design_nz); 0: the full extent. Elements
                           outside both boxes are passive fluid (filtered density 0) [0, 0, 0] */
  int region_shape;     /* NC_REGION_BOX or NC_REGION_CYLINDER [NC_REGION_BOX] */
  double heat_radius, design_radius; /* NC_REGION_CYLINDER: radii in element sizes [0, 0] */
  int heat_z0;          /* NC_REGION_CYLINDER: first element layer of both regions [0] */
  int mg_op0;           /* NC_PREC_MIXED only: NC_MGOP_EXACT or NC_MGOP_PICARD [NC_MGOP_PICARD] */
  int mg_tail_ctas;     /* CTAs (1024 threads each) of the thread-block cluster that runs the fused
                           multigrid tail, 1..16; 0: the largest cluster the device schedules [0] */
  int elem_chunk;       /* FP32 finest-level operators (Krylov operator and multigrid level 0): -1 one
                           thread per element; 1, 2, 4, 8, 16 (0: 4) elements per thread, each thread
                           walking a column of elements with the shared node plane in registers (fewer
                           loads and atomics, but more registers: measured slower on GB300) [-1] */
  int mg_nu_coarse;     /* post-smoothing sweeps on the multigrid levels from mg_nu_coarse_level down
                           to the one above the coarsest; 0: nu_post [0] */
  int mg_nu_coarse_level; /* first level that takes mg_nu_coarse sweeps (levels >= 1; 0: 1) [0] */
  int mg_smoother;      /* smoother of the multigrid levels below the finest (the finest level keeps 2x2
                           block Jacobi): NC_SMOOTH_BLOCK_JACOBI or NC_SMOOTH_ZLINE. Fixed at creation;
                           NC_SMOOTH_ZLINE needs mg_tail_nodes = 0 [NC_SMOOTH_BLOCK_JACOBI] */
  int filter_method;    /* NC_FILTER_SPECTRAL or NC_FILTER_CHEBYSHEV [NC_FILTER_SPECTRAL] */
  int mg_galerkin;      /* NC_PREC_MIXED only: the element operator whose Galerkin products form the
                           multigrid levels below the finest (and whose block diagonal smooths the
                           finest), NC_MGOP_EXACT (J(s)) or NC_MGOP_PICARD [NC_MGOP_PICARD] */
} nc_params;

/* Per-solve statistics (any pointer argument of this type may be NULL). */
typedef struct {
  int newton_its;        /* Newton steps taken */
  int krylov_its;        /* FGMRES iterations summed over the steps */
  int residual_evals;    /* FP64 residual evaluations (including damping trials) */
  int ramped;            /* 1 if the source ramp (Sec. 5.4) was needed */
  double rel_residual;   /* final ||R_free|| / ||R_free(0)|| */
  double res_hist[64];   /* relative residual after each Newton step (first 64) */
  int krylov_hist[64];   /* FGMRES iterations of each Newton step (first 64) */
  double t_setup_ms;     /* multigrid set-up time */
  double t_krylov_ms;    /* FGMRES time */
  double t_total_ms;     /* wall time of the call */
  double alg_bytes;      /* algorithmic bytes of the operator kernels launched */
  long long kernel_launches; /* library kernels launched by the call */
  int mg_setups;         /* multigrid hierarchies built by the call */
} nc_stats;

/* Fill *p with the defaults. Returns NC_ERR_ARG if p is NULL. */
nc_status nc_default_params(nc_params* p);

/* Create a problem on the current CUDA device: validates g and p, resolves kappa_f, and
 * allocates every device buffer (state, materials, Krylov basis, multigrid hierarchy).
 * stream: a cudaStream_t or NULL. On success *out owns the problem. */
nc_status nc_create_problem(const nc_grid* g, const nc_params* p, void* stream, nc_problem** out);

/* Release every device buffer of the problem. Accepts NULL. */
nc_status nc_destroy_problem(nc_problem* pb);

/* Device bytes nc_create_problem would allocate for (g, p) (for admission control). */
nc_status nc_footprint_bytes(const nc_grid* g, const nc_params* p, size_t* bytes);

/* Replace the parameters of an existing problem without reallocating (e.g. a new buoyancy factor
 * for a pooled problem). precision, mg_levels and restart must equal the creation values
 * (NC_ERR_ARG otherwise). The problem then needs a new nc_set_design. */
nc_status nc_set_params(nc_problem* pb, const nc_params* p);

/* Design pipeline, Sec. 5.1-5.2: rho (E values in [0,1], finite; NC_ERR_ARG otherwise) ->
 * gamma = 1 on Omega_h (the heated box) and 0 on passive fluid -> PDE filter -> gamma~ = 1 on Omega_h
 * and 0 on passive fluid -> RAMP kappa_e, k_e. Values of rho outside the design box are ignored.
 * Resets the state to zero unless nc_set_state is called afterwards. */
nc_status nc_set_design(nc_problem* pb, const double* rho);

/* Warm start (Sec. 5.4): P and T (N values each) become the initial Newton guess. Values on
 * the Dirichlet set of params.bc are forced to 0. Requires a design. */
nc_status nc_set_state(nc_problem* pb, const double* P, const double* T);

/* Damped Newton state solve (Sec. 5.4) to params.newton_rtol. Requires a design.
 * On NC_ERR_DIVERGED / NC_ERR_MAXIT the last iterate is kept and stats are filled. */
nc_status nc_solve_state(nc_problem* pb, nc_stats* stats);

/* Objective (Eq. objdiscr, read as the mean temperature over Omega_h with Galerkin weights)
 * of the current state. Requires a solved state. */
nc_status nc_objective(nc_problem* pb, int objective, double* f);

/* Adjoint solve J(s)^T lambda = df/ds on the free DOFs (Sec. 5.1) at the solved state;
 * writes the objective to *f_out (may be NULL). */
nc_status nc_solve_adjoint(nc_problem* pb, int objective, double* f_out, nc_stats* stats);

/* df/drho (E values) by the chain rule through RAMP and the filter transpose; 0 on passive elements.
 * Requires a solved adjoint. */
nc_status nc_sensitivities(nc_problem* pb, double* dfdrho);

/* Copy the solved fields out: P, T (N values each, either may be NULL) and the centroid
 * Darcy velocity u (3E values, Eq. finaldarcy, may be NULL). */
nc_status nc_get_fields(const nc_problem* pb, double* P, double* T, double* u);

/* Copy the adjoint solution lambda out (2N doubles, node-interleaved like a state vector; 0 on
 * the Dirichlet rows). Requires a solved adjoint. */
nc_status nc_get_adjoint(const nc_problem* pb, double* lam);

/* The resolved fluid and solid permeabilities kappa_f (Eq. nusselt5 when params.kappa_f <= 0) and
 * kappa_s = kappa_ratio * kappa_f (Eq. permRAMP). Either pointer may be NULL. */
nc_status nc_get_permeabilities(const nc_problem* pb, double* kappa_f, double* kappa_s);

/* Filtered design gamma~, kappa_e and k_e (E values each; any may be NULL). */
nc_status nc_get_design_fields(const nc_problem* pb, double* gamma_tilde, double* kappa, double* k);

/* Operator-level entry points: one step of the path on caller data, for parity checks.
 * s, v, w, out are state vectors (2N doubles). Entries of v and w on the Dirichlet set of params.bc
 * are ignored; the corresponding outputs are: R_d = s_d (residual), 0 (products). */

/* R(s) (Eq. finalsyseq) and ||R_free(s)||^2 (norm2_free may be NULL), in the arithmetic of the
 * Newton residual (FP64 on the FP64 path, outer_arith on the mixed path). Requires a design. */
nc_status nc_eval_residual(nc_problem* pb, const double* s, double* R, double* norm2_free);

/* Exact Newton Jacobian product J(s) v, including the derivatives of tau and N*, computed in
 * FP64 (precision = NC_PREC_FP64) or FP32 (NC_PREC_MIXED). Requires a design. */
nc_status nc_apply_jacobian(nc_problem* pb, const double* s, const double* v, double* out,
                            int precision);

/* Transposed product J(s)^T w (the adjoint operator) in the arithmetic of the adjoint refinement
 * residual (FP64 on the FP64 path, outer_arith on the mixed path). Requires a design. */
nc_status nc_apply_jacobian_transpose(nc_problem* pb, const double* s, const double* w,
                                      double* out);

/* The frozen-coefficient finest-level multigrid operator (NC_MGOP_PICARD) at the state s applied to v
 * (transpose = 0) or its transpose (transpose = 1), computed in FP32 from FP64 inputs: s, v, out are
 * 2N doubles (node-interleaved P, T; device or host). Fixed rows of v are ignored and those of out are
 * zero, as for nc_apply_jacobian. Requires a design. Has no counterpart in the paper (an operator of
 * this library's preconditioner); it exists so the operator can be checked on its own. */
nc_status nc_apply_picard(nc_problem* pb, const double* s, const double* v, double* out, int transpose);

/* Kernel classes timed when profiling is on (nc_set_profiling). */
enum {
  NC_PROF_RESIDUAL = 0,     /* FP64 residual element sweep */
  NC_PROF_OUTER_OP64 = 1,   /* FP64 J v / J^T w (Krylov operator, adjoint refinement residual) */
  NC_PROF_OUTER_OP32 = 2,   /* FP32 J v / J^T w of the Krylov solver */
  NC_PROF_MG_OP0 = 3,       /* multigrid finest-level operator (matrix-free Jacobian) */
  NC_PROF_MG_STENCIL = 4,   /* stencil operators of multigrid levels >= 2 (fused smoothing / residual) */
  NC_PROF_MG_SETUP = 5,     /* element Jacobians of the finest level and their Galerkin product */
  NC_PROF_SMOOTH = 6,       /* block-Jacobi updates, restriction, prolongation */
  NC_PROF_KRYLOV_VEC = 7,   /* FGMRES dot products and vector updates */
  NC_PROF_FILTER = 8,       /* PDE filter operator and vectors */
  NC_PROF_SENS = 9,         /* FP64 element sensitivities */
  NC_PROF_OTHER = 10,       /* every other library kernel (casts, copies ...) */
  NC_PROF_MG_COARSE_SETUP = 11, /* coarse-level Galerkin products, stencils, block-diagonal inverses */
  NC_PROF_COARSE_FACTOR = 12,   /* inverse of the coarsest-level matrix */
  NC_PROF_COARSE_SOLVE = 13,    /* coarsest-level solve inside the V-cycle */
  NC_PROF_MG_STENCIL_L1 = 14,   /* stencil operators of multigrid level 1 (the largest stencil level) */
  NC_PROF_MG_TAIL = 15,         /* fused V-cycle on the small coarse levels (one cluster kernel) */
  NC_PROF_ADJ_DF64 = 16,        /* double-float J^T lambda of steering adjoint refinement passes */
  NC_PROF_MG_OP0_PICARD = 17,   /* multigrid finest-level operator, frozen-coefficient (NC_MGOP_PICARD) */
  NC_PROF_NCLASSES = 18
};

/* Per-launch CUDA-event timing of kernel classes for calls on pb: bit c of class_mask times class
 * c (0: off; -1: all classes). Setting a mask resets the accumulated times. Timing adds two event
 * records per timed launch. */
nc_status nc_set_profiling(nc_problem* pb, int class_mask);

/* Accumulated device time (ms), launches, algorithmic bytes and algorithmic floating-point
 * operations of kernel class cls since profiling was turned on. Any output pointer may be NULL. */
nc_status nc_get_profile(const nc_problem* pb, int cls, double* ms, long long* launches, double* bytes,
                         double* flops);

/* Kernel launches and algorithmic bytes of every library kernel on pb since creation
 * (monotonic counters; any output pointer may be NULL). */
nc_status nc_counters(const nc_problem* pb, long long* launches, double* bytes);

/* Allocation-free squared norm of the free rows of a state vector (the norm of the Newton stopping
 * test): *out_dev = sum of a_r^2 over the rows r of s_dev that are free under the boundary conditions
 * bc (NC_BC_TOP: P and T of every node below the top face; NC_BC_CAVITY: every component outside the
 * closed cavity's fixed set, i.e. T off the outer walls and the top, P everywhere except the top outer
 * corner). For a residual of a state that meets the boundary conditions this is the norm that
 * nc_eval_residual reports; the fixed rows of such a residual hold s on the fixed set and are never
 * summed here.
 * The paper has no counterpart: this entry point serves callers that cannot allocate device memory
 * on this path (all device memory handed out from their own pre-reserved pool, a hard memory budget,
 * or no cudaMalloc/cudaFree because those calls can synchronise the device). It allocates nothing:
 * its partial sums live in a fixed 64 KiB device array owned by the library (one per device that
 * loads it, kept until exit), so grids with more than 8192 * 4096 summed entries are rejected with
 * NC_ERR_ARG. s_dev (2N doubles, node-interleaved P, T) and out_dev (1 double) are device pointers of
 * the current device. The work is queued on `stream` (a cudaStream_t, NULL = the legacy default
 * stream); *out_dev is valid once the stream has completed it. The first call on a device looks up
 * the device address of the array (cudaGetSymbolAddress), so make that first call before any stream
 * capture; the address is kept for the life of the process, so do not call this entry point on a
 * device again after a cudaDeviceReset of it. Every call shares the array and leaves its last
 * contents there; calls that overlap on the GPU race.
 * Returns NC_ERR_ARG for NULL pointers, an unknown bc or bad sizes and NC_ERR_CUDA if a launch fails. */
nc_status nc_norm2_free_noalloc(const nc_grid* g, int bc, const double* s_dev, double* out_dev, void* stream);

/* Message of the last failed call on pb (or, if pb is NULL, of the calling thread's last failed
 * call without a problem, e.g. nc_create_problem). Never NULL. */
const char* nc_last_error(const nc_problem* pb);

#ifdef __cplusplus
}
#endif
#endif /* NATCONV_H */
