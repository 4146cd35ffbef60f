/*
 * mb.h -- C-ABI of libmb: GB300-native hot path of the MULTIBAT 3-D Li-ion
 * cell model with lithium plating (arXiv:1704.04139).
 *
 * Every function returns an int status (MB_OK = 0, negative on error); the
 * message of the last error of the calling thread is returned by
 * mb_last_error().  Handles are opaque and owned by the library; every array
 * argument is owned by the caller and only borrowed for the duration of the
 * call.  Plain pointers are host pointers unless the function name ends in
 * _dev, in which case they are device pointers of the current CUDA device and
 * the work is enqueued on the given stream (a cudaStream_t passed as void*;
 * NULL = the legacy default stream) and the call returns when that stream
 * has completed it.  SI units throughout.
 *
 * State layout of a cell with N voxels and F plating faces (n = 2N + F):
 *   u = [ c (N) | phi (N) | n_pl (F) ]
 * Voxels are in [t][y][z] order with z fastest; t is the through-cell axis.
 * Plating faces are all graphite-electrolyte faces, ordered by the graphite
 * voxel's linear index, then by direction (-t, +t, -y, +y, -z, +z).
 * Residual rows have the same layout: R = [ R_c | R_phi | R_n ].
 *
 * Phase labels: 0 electrolyte (E), 1 graphite anode (G), 2 cathode (K),
 * 3 lithium foil (L), 4 negative collector (CN), 5 positive collector (CP).
 *
 * Sign convention: I_app > 0 delithiates the anode (the paper's delithiation
 * current density mu, Sec. 3.2); a charge is I_app < 0.
 */
#ifndef MB_H
#define MB_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define MB_OK        0
#define MB_EINVAL   -1   /* bad argument */
#define MB_ENOMEM   -2   /* device memory exhausted / admission refused */
#define MB_EBADGEOM -3   /* forbidden phase contact (e.g. anode touching cathode) */
#define MB_ENOCONV  -4   /* Newton did not converge after all step halvings */
#define MB_ECUTOFF  -5   /* step completed, voltage limit reached */
#define MB_ETIMEOUT -6   /* a bounded device wait gave up */
#define MB_EPENDING -7   /* serving: result not ready yet */
#define MB_ECUDA    -8   /* CUDA runtime error */

/* ---- parameter table (Sec. 2.2-2.3; values are placeholders, see params.json) ----
 * U0(x) = ocp[0] + ocp[1] x + ocp[2] exp(-ocp[3] x) + ocp[4] tanh((x - ocp[5]) / ocp[6]),
 * x = c / cmax.  n_c = Pl_layer_m / Pl_Vm_Li (mol/m^2). */
typedef struct {
    double F, R, T, clamp_rel;
    double E_c0, E_D, E_kappa, E_tplus, E_tdf;
    double G_cmax, G_D, G_sigma, G_i00, G_x0, G_ocp[7];
    double K_cmax, K_D, K_sigma, K_i00, K_x0, K_ocp[7];
    double L_sigma, L_i00;
    double CN_sigma, CP_sigma;
    double Pl_i00, Pl_layer_m, Pl_Vm_Li;
} mb_params;

/* Both paths: FP64 state and Newton residual; FP32 arithmetic in the Krylov
 * solver and the preconditioner, with float-float storage of the vectors that
 * carry near-null components.  They differ in the Krylov operator's
 * linearisation coefficients: */
#define MB_PREC_FP64  0   /* coefficients from the FP64 state in FP64 */
#define MB_PREC_MIXED 1   /* coefficients from the FP32 copy of the state in FP32 */

typedef struct {
    int    precision;      /* MB_PREC_FP64 or MB_PREC_MIXED */
    double newton_tol;     /* stop when lam*||delta||_s <= tol (scaled max-norm), or when the
                              estimated remaining error is (newton_rate_test) */
    int    newton_maxit;   /* per active-set pass */
    int    gmres_m;        /* FGMRES restart length */
    int    krylov_maxit;   /* per Newton iteration */
    double krylov_rtol;    /* relative residual reduction per linear solve */
    int    max_passes;     /* plating active-set passes per step (>= 1) */
    int    max_halvings;   /* dt halvings on Newton failure */
    int    mg_coarse_cells;/* multigrid: coarsen until at most this many cells */
    int    mg_smooth;      /* fine-level block-Jacobi sweeps before and after the coarse correction (1..8) */
    int    mg_kcycle;      /* FGMRES iterations of the level-1 K-cycle (1..16; default 5) */
    int    mg_coarse_pre;  /* damped block-Jacobi sweeps before the coarse correction on levels >= 1
                              (1..4; default 2) */
    int    mg_coarse_post; /* ... and after it (1..4; default 2) */
    int    mg_bf16;        /* 1: the fine smoother's stencil and the coarse-level operators are
                              applied from BF16 copies (FP32 arithmetic); 0: FP32 operators */
    int    mg_stream;      /* how the BF16 coarse sweeps and products fetch their operator rows
                              (same results in every mode): 0 plain loads; 1 each block first
                              prefetches into L2 the rows of the block one resident wave ahead
                              (bulk asynchronous prefetch); 2 post-smoothing sweeps of levels with
                              at least one tile of 256 cells per SM stage rows, right-hand side and
                              iterate in shared memory by bulk asynchronous copies (persistent,
                              double-buffered); 3 (default) plain loads, the level-1 post-smoothing
                              sweeps with at most 48 registers (5 blocks of 256 per SM instead of 4:
                              37.3 against 41.1 us per sweep and 1 % faster steps on a 4.2M-voxel
                              cell, the fastest mode measured) */
    int    pass_start;     /* Newton start of plating active-set passes after the first: 0 u_old
                              (the previous time level); 1 (default) the previous pass's converged
                              state.  The solution of a pass depends only on its frozen gates, not on
                              the start. */
    int    mg_kcycle_reorth; /* 1 (default): the level-1 K-cycle orthogonalises by two classical
                              Gram-Schmidt passes; 0: one pass (2 % faster on a 4.2M-voxel cell,
                              but FGMRES preconditioned with it stagnated on a small half cell) */
    int    krylov_forcing; /* 0: every linear solve to krylov_rtol; 1 (default): Eisenstat-Walker
                              forcing terms (choice 2, safeguarded) within [krylov_rtol, 0.1]:
                              26 % fewer preconditioner applications per step on a 4.2M-voxel
                              cell; the Newton tolerance, and so the converged state, is the same */
    int    mg_tail;        /* 0 (default): one launch per coarse sweep, restriction and coarsest
                              solve; 1: the V-cycle from the first level >= 2 that one wave of the
                              GPU covers (one block of 512 threads per SM) down to the coarsest
                              solve and back runs as one persistent cooperative launch with grid
                              barriers between its phases (same results); k >= 2: the same from
                              the first level >= k that one wave covers (0..16).  Per-level
                              launches measured faster on GB300 inside the preconditioner's CUDA
                              graph (2.27 against 2.43 ms per application on a 4.2M-voxel cell with
                              the tail from level 2).  Applies to BF16 operators (mg_bf16 = 1). */
    int    pc_lag;         /* 0: the preconditioner (row scales, condensation, level operators,
                              coarse inverse, fine stencil) is rebuilt at every Newton iteration;
                              1 (default): at the first iteration of each Newton solve and then only
                              when the iterate has moved by more than pc_lag_drift since the last
                              rebuild, when a linear solve took more than 1.5 x + 2 the Krylov
                              iterations of the first solve after the last rebuild, or when a solve
                              with the lagged preconditioner did not reach its tolerance (that solve
                              is repeated after the rebuild).  The Krylov operator is always the
                              current linearisation */
    double pc_lag_drift;   /* with pc_lag = 1 the preconditioner is rebuilt once the damped Newton
                              updates since its last rebuild sum to more than this in the step
                              cap's scaled max-norm (the change of the exponentials' arguments and
                              of the plated inventories relative to max(n_c, |n|)), so that a lagged
                              preconditioner only serves iterates close to the one it was built at:
                              its coarse correction of the near-null potential mode follows the
                              Butler-Volmer partials, which change fast with the state, and its row
                              scales define the norm of the Krylov tolerance.  Default 0.05; >= 0 */
    int    mg_pdl;         /* 1: the kernels of a preconditioner application are launched with
                              programmatic dependent launch: each may be scheduled while its
                              predecessor drains and waits, before its first memory access, until
                              that predecessor has completed (same results); 0 (default): plain
                              launches, measured faster on GB300 inside the captured graph (111.4
                              against 112.2 ms per step on a 4.2M-voxel cell) */
    int    newton_rate_test; /* 1 (default): a Newton solve also stops when the error left after the
                              current update, estimated from two consecutive full steps as
                              (rho / (1 - rho) + relres) |d_k| with rho = |d_k| / |d_k-1| < 0.5 and
                              relres the linear solve's relative residual (the scaled max-norm of
                              the convergence test), is below newton_tol: the iteration that would
                              only confirm a quadratically converged state is skipped; 0: only an
                              update below newton_tol stops it.  The reduced models built on this
                              cell apply the same rule to their Newton iteration (ROM tolerance
                              1e-12 in the step cap's scaled max-norm, LU or GMRES steps exact
                              enough that the linear residual term is left out) */
} mb_solver_opts;

typedef struct {
    int    newton_its;     /* summed over passes and sub-steps */
    int    krylov_its;
    int    passes;
    int    flips;          /* plating gates flipped between passes (re-solved) */
    int    unresolved_flips; /* gates that still flipped after the last allowed pass: the accepted
                              state is then not consistent with its gates on these faces (0 when
                              the active set settled) */
    int    halvings;
    double dt_used;
    double V_cell;         /* mean Phi over the t = nt-1 collector layer (s_cp) */
    double mean_c_solid;   /* mean graphite concentration (s_ac) */
    double Li_total;       /* V * sum_{E,G,K} c + A * sum n  (mol) */
    double Li_anode;       /* V * sum_G c + A * sum n (mol) */
    double Li_plated;      /* A * sum n (mol) */
    double res_norm;       /* final scaled max-norm of the FP64 residual */
} mb_step_info;

typedef struct {
    int64_t n_vox, n_faces, n_unknowns;
    int     nt, ny, nz;
    double  h;
    double  i_1c;          /* 1C current density: F V cmax_G (1-x0_G) n_G / 3600 s / (ny nz h^2) */
    int64_t count[6];      /* voxels per phase label */
    int64_t device_bytes;  /* device memory held by the cell */
    int64_t n_iface;       /* solid-electrolyte faces with kinetics (G, K, L): F plating faces first */
} mb_cell_info;

typedef struct mb_cell mb_cell;

const char* mb_last_error(void);
void mb_opts_default(mb_solver_opts* o);

/* Geometry ingest and face classification (Sec. 2.4, Table interfaceCond).
 * labels: host uint8[nt*ny*nz].  Sets the rest state (table concentrations,
 * equilibrium potentials, no plated Li).  MB_EBADGEOM on a G-K, G-CP, K-CN,
 * K-L or CN-CP contact. */
int mb_cell_create(const uint8_t* labels, int nt, int ny, int nz, double h,
                   const mb_params* p, const mb_solver_opts* o, mb_cell** out);
int mb_cell_destroy(mb_cell* cell);
int mb_cell_info_get(mb_cell* cell, mb_cell_info* info);
/* kinetic scales of the parameter study: exchange-current scale s_i0 (both
 * electrodes' Butler-Volmer prefactors) and plating rate scale k_pl. */
int mb_cell_set_scales(mb_cell* cell, double s_i0, double k_pl);
int mb_cell_set_opts(mb_cell* cell, const mb_solver_opts* o);
/* plating face list: graphite voxel, electrolyte voxel, direction 0..5 (host int32[F] each) */
int mb_plating_faces(mb_cell* cell, int32_t* g, int32_t* e, int32_t* dir);

/* State u (host double[n]) in the layout above. */
int mb_state_get(mb_cell* cell, double* u);
int mb_state_set(mb_cell* cell, const double* u);

/* One implicit Euler step of Eq. (ap4:detailed): Newton-Krylov with the
 * plating active-set passes; dt halved on failure up to max_halvings times.
 * Newton updates are capped at 0.25 in the max-norm of the voxel unknowns
 * (c, phi) scaled by (c_ref, 1 V) and of the plated-Li inventories relative
 * to max(n_c, |n|); convergence is tested on every unknown in the scales
 * (c_ref, 1 V, n_c).  Returns MB_ENOCONV when every halving failed
 * (state unchanged). */
int mb_step(mb_cell* cell, double dt, double I_app, mb_step_info* info);

/* Adaptive time step (Sec. workflow:discretization: the step size is
 * adapted; the controller is this library's).  One accepted implicit Euler
 * step of size at most dt_try: its local error is estimated from the two
 * previous states (the state before the last accepted adaptive step, the
 * current one) as e = dt/(2 dt + dt_prev) |u_new - u_pred|_s, u_pred their
 * linear extrapolation to t + dt and |.|_s the max-norm scaled by the
 * unknown scales (c_ref, 1 V, n_c); a step with e > tol is rejected and
 * retried with dt * clamp(0.9 sqrt(tol/e), 0.2, 2) (down to dt_min, at most
 * max_rejects times); the accepted step proposes dt_next by the same factor
 * within [dt_min, dt_max].  Without a history (after mb_cell_create,
 * mb_state_set, mb_step or mb_adapt_reset) the step of size dt_try is
 * accepted without an estimate.  The first call allocates two state-size
 * buffers.  info as mb_step (summed over the tried steps); MB_ENOCONV as
 * mb_step (state unchanged). */
typedef struct {
    double tol;            /* local error bound in the scaled max-norm */
    double dt_min, dt_max; /* step size bounds (s) */
    int    max_rejects;    /* rejected tries per accepted step */
} mb_adapt_opts;
typedef struct {
    double dt_used;        /* size of the accepted step (s) */
    double dt_next;        /* proposed size of the next step (s) */
    double err;            /* its local error estimate (0 without history) */
    int    rejects;        /* rejected tries before it */
} mb_adapt_info;
int mb_step_adaptive(mb_cell* cell, double dt_try, double I_app, const mb_adapt_opts* o, mb_adapt_info* ai,
                     mb_step_info* info);
int mb_adapt_reset(mb_cell* cell);

/* FP64 residual R(u; u_old, dt, I_app) of Eq. (ap4:detailed) with plating
 * gates gate (uint8[F], 1 = active; NULL = gates taken at u_old as mb_step
 * does).  u, u_old, r: double[n]. */
int mb_residual(mb_cell* cell, const double* u, const double* u_old, const uint8_t* gate,
                double dt, double I_app, double* r);
int mb_residual_dev(mb_cell* cell, const double* u, const double* u_old, const uint8_t* gate,
                    double dt, double I_app, double* r, void* stream);

/* Jacobian-vector product J(u) v of the residual above (analytic, no finite
 * differences).  J does not depend on u_old or I_app.  FP64 variant:
 * double[n] in/out; FP32 variant: float u, v, jv (the mixed-precision Krylov
 * operator). */
int mb_jvp(mb_cell* cell, const double* u, const uint8_t* gate, double dt,
           const double* v, double* jv);
int mb_jvp_dev(mb_cell* cell, const double* u, const uint8_t* gate, double dt,
               const double* v, double* jv, void* stream);
int mb_jvp_f32_dev(mb_cell* cell, const float* u, const uint8_t* gate, double dt,
                   const float* v, float* jv, void* stream);

/* Kernel timing and launch counting.  While enabled, every launch of the
 * timed kernel classes below is bracketed by CUDA events recorded on the
 * stream it is launched on; mb_prof_read returns the number of timed
 * launches and their summed device time (ms) since the last enable/reset.
 * mb_launch_count returns the number of kernels the library has launched
 * for this cell since its creation (always counted). */
#define MB_PROF_JVP      0   /* Jacobian-vector product kernel (Krylov operator) */
#define MB_PROF_RESIDUAL 1   /* FP64 residual kernel */
#define MB_PROF_PRECOND  2   /* one whole preconditioner application (many kernels) */
#define MB_PROF_SMOOTH   3   /* fine-level smoothing sweep (assembled stencil; 2 mg_smooth - 1 per
                                preconditioner application) */
#define MB_PROF_LSMOOTH  4   /* level-1 post-smoothing sweep (mg_coarse_post per V-cycle of the K-cycle) */
int mb_prof_enable(mb_cell* cell, int on);
int mb_prof_read(mb_cell* cell, int kind, int64_t* count, double* total_ms);
int mb_prof_reset(mb_cell* cell);
int mb_launch_count(mb_cell* cell, int64_t* count);
/* The CUDA stream (cudaStream_t, as void*) on which mb_step and the other
 * host-pointer calls of this cell enqueue their work. */
int mb_cell_stream(mb_cell* cell, void** stream);

/* ---- reduced-order model (Sec. workflow:MOR, Eq. ap4:fully_reduced) ----
 * The reduced model of a cell: reduced basis U (the POD spaces of c, n and phi
 * in the full state layout), the empirical-interpolation points of the
 * interface terms (Butler-Volmer, counter electrode, plating: one common
 * basis, Eqs. ise_gr, ise_li, iplel) and of the migration term with 1/c (Eq.
 * phiel), and the projected operators.  Residual of instance b at reduced
 * coefficients a (N_r):
 *   Ms (a - a_old)/dt + Alin a + mu bbnd + Pbv f_bv(a) + P1c f_1c(a)
 * f_bv(a)[m] = s_i0 (BV rows) + (CE rows) + k_pl g (plating rows) of the
 * full-order interface terms at point p_bv[m] of the reconstructed state U a,
 * f_1c(a)[m] the migration term at p_1c[m]; the plating gate g follows the
 * full-order rule on the reconstructed state.  Points index residual rows of
 * the layout [R_c | R_phi | R_n]; the face rows are weighted by A.  All arrays
 * are host, row-major, FP64, copied by mb_rom_create. */
typedef struct {
    int n_r;                 /* reduced dimension N_r */
    int n_bv, n_1c;          /* interpolation points of the interface and migration terms */
    const double* U;         /* n x n_r: basis in the full state layout (n = 2N + F) */
    const int64_t* p_bv;     /* n_bv residual rows */
    const int64_t* p_1c;     /* n_1c residual rows */
    const double* Ms;        /* n_r x n_r projected storage */
    const double* Alin;      /* n_r x n_r projected linear part */
    const double* bbnd;      /* n_r projected boundary term (per unit I_app) */
    const double* Pbv;       /* n_r x n_bv projected interpolation basis of the interface terms */
    const double* P1c;       /* n_r x n_1c projected interpolation basis of the migration term */
    const double* s_cp;      /* n_r: cell potential functional (mean phi of the last t-layer) */
    const double* s_ac;      /* n_r: mean graphite concentration functional */
    const double* a0;        /* n_r: initial coefficients */
} mb_rom_data;

typedef struct {
    double I_app;            /* applied current density (A/m^2), the paper's mu */
    double s_i0;             /* exchange-current scale */
    double k_pl;             /* plating rate scale */
} mb_rom_params;

typedef struct {
    int64_t newton_its;      /* reduced Newton iterations summed over instances and steps */
    int64_t flips;           /* plating gate flips summed over instances and steps */
    int     failed;          /* instances whose Newton iteration did not converge */
} mb_rom_info;

typedef struct mb_rom mb_rom;

/* Offline construction (Sec. workflow:MOR) from full-order solves of the
 * cell: n_steps steps of size dt at every parameter point from the cell's
 * current state (restored afterwards; it is also the reduced initial state),
 * every Newton stage a snapshot; POD of c, plated Li n and phi separately in
 * the L^2 inner product (at most n_c, n_n, n_phi modes, none below pod_tol of
 * the largest singular value of the block; the Gram-matrix route resolves
 * down to ~1e-7); EI-Greedy on the interface terms (at most m_bv points) and
 * on the migration term (at most m_1c), stopping below ei_tol of the largest
 * training entry; projections as in mb_rom_data. */
typedef struct {
    int n_params;                    /* snapshot parameter points */
    const mb_rom_params* params;     /* n_params */
    double dt;                       /* snapshot step */
    int n_steps;                     /* steps per snapshot trajectory */
    int n_c, n_n, n_phi;             /* POD dimension bounds */
    int m_bv, m_1c;                  /* EI dimension bounds */
    double pod_tol, ei_tol;          /* relative cut-offs */
} mb_rom_build_opts;
int mb_rom_build(mb_cell* cell, const mb_rom_build_opts* o, mb_rom** out);
/* The pair of Sec. workflow:MOR's certification step from one snapshot set:
 * the validation model with the bounds and tolerances of o (*rom_val), and the
 * reduced model that keeps ceil(frac x) of each of its POD blocks and of each
 * of its EI bases (*rom; the paper's 97 %: frac = 0.97).  Both are truncations
 * of the same POD and EI-Greedy, so the validation bases contain the reduced
 * ones (mb_rom_estimate_batch). */
int mb_rom_build_pair(mb_cell* cell, const mb_rom_build_opts* o, double frac, mb_rom** rom, mb_rom** rom_val);
/* Dimensions of a reduced model: N_r and the two numbers of points. */
int mb_rom_dims(mb_rom* rom, int* n_r, int* n_bv, int* n_1c);
/* Reduced modes by field: basis columns supported only on the concentration
 * rows (n_c), the plated-Li face rows (n_n) or the potential rows (n_phi). */
int mb_rom_block_dims(mb_rom* rom, int* n_c, int* n_n, int* n_phi);

/* Build the reduced model of `cell` from the arrays of d (MB_EINVAL on
 * inconsistent sizes or points outside the residual). */
int mb_rom_create(mb_cell* cell, const mb_rom_data* d, mb_rom** out);
int mb_rom_destroy(mb_rom* rom);
/* Reduced trajectories of B instances from a0 with the instance parameters
 * prm[B]: n_steps implicit Euler steps of size dt.  V_out and sac_out
 * (host double[B * (n_steps + 1)], instance-major, entry 0 the initial
 * state) receive s_cp and s_ac; a_final (host double[B * n_r]) the final
 * coefficients (may be NULL).  Newton per step and instance: step length
 * min(1, 0.25 / m), m the max-norm of U_loc delta on the stencil closure of
 * the points with the voxel unknowns (c, phi) in their scales and the plated
 * inventories relative to max(n_c, |n|) of the current reconstruction,
 * converged at lam m <= 1e-12 (the same scaled norm) or at a full step with
 * m <= 1e-10 that did not halve the previous m (the rounding floor of the
 * reconstruction), at most 30 iterations;
 * plating active-set passes as mb_step (at most 3); an instance whose step
 * fails retakes it from the state before it as 2^h steps of dt / 2^h, h = 1
 * .. max_halvings of the cell's options (as mb_step halves its step).  The state, the
 * interpolated terms and the residual are FP64 and the reconstruction at the
 * points float-float (~2^-44 relative; the converged result is the FP64 one
 * to that rounding); the Newton matrix is formed with FP32 accuracy (three TF32
 * tensor-core products per operand pair) and factorised in FP32; an instance
 * whose iteration stagnates, or that has not converged after 8 iterations,
 * takes its Newton steps for the rest of the time step by FP64 GMRES
 * preconditioned with its last FP32 LU.  Returns MB_ENOCONV if some instance
 * failed (its outputs are then NaN from that step on). */
int mb_rom_solve_batch(mb_rom* rom, int B, const mb_rom_params* prm, int n_steps, double dt, double* V_out,
                       double* sac_out, double* a_final, mb_rom_info* info);

/* As mb_rom_solve_batch, with the reduced coefficients of every step in
 * a_traj (host double[B * (n_steps + 1) * n_r], instance-major, then step;
 * entry 0 the initial coefficients): the reduced trajectories, from which
 * U a reconstructs the fields (Sec. workflow:MOR). */
int mb_rom_solve_batch_traj(mb_rom* rom, int B, const mb_rom_params* prm, int n_steps, double dt, double* V_out,
                            double* sac_out, double* a_traj, mb_rom_info* info);
/* The reduced basis U in the full state layout (host double[n * n_r],
 * row-major: row i is unknown i of [c | phi | n_pl]). */
int mb_rom_basis(mb_rom* rom, double* U);

/* Hierarchical a-posteriori error estimate (Sec. workflow:MOR, Eqs.
 * ap4:saturation and ap4:estimate): B instances with parameters prm run
 * n_steps steps of size dt in the reduced model `rom` and in a larger
 * validation model `rom_val` of the same cell; per instance, step and field,
 *   est = ||U a - U_val a_val||_W / (1 - theta),
 * the L^2 norm of the voxel grid (weight V per voxel value, A per plated-Li
 * face value) of the difference of the two reconstructions, for the fields
 * c, phi and n (the plated-Li inventory, a state the paper's estimate does
 * not have).  rom_val's basis must be W-orthonormal on each field (as the
 * POD of mb_rom_build and of the oracle gives); rom's need not lie in its
 * span.  The maps between the two bases are formed on the host at the first
 * call for a pair (O(n N_r^2) flops) and kept with rom; per step the
 * estimate costs O(N_val N_r + N_r^2) FP64 flops per instance on the
 * coefficients (no reconstruction).  est_out: host double[B * (n_steps + 1)
 * * 3], instance-major, then step, then field (c, phi, n); V_out and
 * V_val_out (may be NULL): host double[B * (n_steps + 1)], the two models'
 * cell potentials; norm_val_out (may be NULL): as est_out, the W-norms of
 * the validation model's fields (the denominators of relative errors).
 * theta in [0, 1).  MB_EINVAL for models of different
 * cells or a validation basis that is not W-orthonormal per field;
 * MB_ENOCONV (estimates NaN from then on) if an instance failed in either
 * model. */
int mb_rom_estimate_batch(mb_rom* rom, mb_rom* rom_val, double theta, int B, const mb_rom_params* prm,
                          int n_steps, double dt, double* V_out, double* V_val_out, double* est_out,
                          double* norm_val_out, mb_rom_info* info);

/* ---- serving loop (parameter-study queries; no counterpart in the paper) ----
 * Requests arrive at any time (mb_serve_submit never blocks).  Reduced-model
 * requests are admitted into the free slots of one resident batch of the
 * reduced model (mb_rom) at step boundaries and leave it when their protocol
 * is done, so requests that arrive while others run join the same batched
 * launches; each instance's arithmetic does not depend on the others in the
 * batch, so a result is the same alone and in the mix.  Full-order
 * requests (validation solves) run on worker threads with their own streams
 * and cells (created from the server's cell template on a worker's first
 * request, kept and reset to the initial state for the next ones; a worker
 * creates its cell while the device memory of the existing ones stays within
 * fom_budget_bytes); their work overlaps with the reduced batch on the
 * device. */
#define MB_REQ_ROM 0
#define MB_REQ_FOM 1
typedef struct {
    mb_rom* rom;                     /* reduced model for MB_REQ_ROM (not owned; NULL: none) */
    const uint8_t* fom_labels;       /* full-order cell template (copied; NULL: no MB_REQ_FOM) */
    int nt, ny, nz;
    double h;
    const mb_params* params;         /* template parameters (copied) */
    const mb_solver_opts* fom_opts;  /* NULL: defaults */
    int rom_slots;                   /* slots of the resident reduced batch (>= 1) */
    int64_t fom_budget_bytes;        /* device memory for concurrent full-order cells */
    int fom_workers;                 /* threads running full-order requests (>= 1) */
} mb_serve_opts;

typedef struct {
    int kind;                        /* MB_REQ_ROM or MB_REQ_FOM */
    mb_rom_params prm;               /* current density, exchange-current scale, plating rate scale */
    int n_steps;                     /* protocol length */
    double dt;                       /* step (s) */
    double v_cutoff;                 /* > 0: the protocol ends after the first step whose cell potential
                                        reaches v_cutoff (status MB_ECUTOFF, n_steps the steps done) */
} mb_request;

typedef struct {
    int status;                      /* MB_OK, MB_ECUTOFF (ended at the voltage limit), MB_ENOCONV or
                                        another error of the request */
    int n_steps;                     /* steps done */
    double t_submit, t_start, t_done;/* server clock (s since mb_serve_create) */
    double* V;                       /* caller-provided, n_steps + 1 cell potentials (may be NULL) */
    double* s_ac;                    /* caller-provided, n_steps + 1 mean graphite concentrations (may be NULL) */
} mb_result;

typedef struct mb_server mb_server;

int mb_serve_create(const mb_serve_opts* o, mb_server** out);
/* Queue a request; *ticket identifies it.  Never blocks. */
int mb_serve_submit(mb_server* srv, const mb_request* req, uint64_t* ticket);
/* MB_EPENDING while the request runs; MB_OK once done (out filled, the
 * ticket released); MB_EINVAL for an unknown ticket. */
int mb_serve_poll(mb_server* srv, uint64_t ticket, mb_result* out);
/* Stops the threads after the running work; pending requests are dropped. */
int mb_serve_destroy(mb_server* srv);

/* ---- residual without allocation (no counterpart in the paper) ----
 * Same result as mb_residual_dev with gate == NULL (gates taken at u_old),
 * for callers that may not allocate memory at call time: a serving loop whose
 * device memory is all reserved up front by another allocator, where a
 * cudaMalloc fails or stalls, or a latency-bound thread that must not wait on
 * an allocator.  The F bytes of gate scratch live in a fixed array in the
 * library's static device memory (MB_NOALLOC_MAX_FACES bytes per device)
 * instead of the cell's buffers; the success path calls cudaMalloc, cudaFree
 * or any other allocating routine nowhere.  Nothing in the scratch has to
 * start at zero: each call writes every byte it reads.
 *   u, u_old, r: device double[n] of the current device; stream as for the
 *   other _dev calls; the call returns when the stream has completed it.
 * The first call on each device resolves the scratch address
 * (cudaGetSymbolAddress, which may load the library's device code): make it
 * with that device current and before any stream capture.  All calls on one
 * device share the one scratch array, so calls that overlap in time (other
 * threads, other streams, other cells) race: order them on one stream or on
 * the host.  MB_EINVAL for a cell with more than MB_NOALLOC_MAX_FACES plating
 * faces, when the current device is not the cell's, or for an invalid
 * argument; MB_ECUDA on a CUDA error.  A failing call
 * stores its message for mb_last_error in host memory. */
#define MB_NOALLOC_MAX_FACES 4194304
int mb_residual_dev_noalloc(mb_cell* cell, const double* u, const double* u_old, double dt, double I_app,
                            double* r, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MB_H */
