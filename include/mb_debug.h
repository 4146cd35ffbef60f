/*
 * mb_debug.h -- inspection hooks of libmb's Newton-Krylov preconditioner,
 * used by the test suite to check each stage against an independent
 * reference.  Not needed by applications.  Host pointers throughout; every
 * call synchronises.
 */
#ifndef MB_DEBUG_H
#define MB_DEBUG_H

#include "mb.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Assemble the preconditioner at state u (double[n], converted to FP32) for
 * step dt with plating gates gate (uint8[F]) and apply it to r (double[n],
 * the scaled Krylov residual): z = M^-1 r. */
int mb_debug_precond(mb_cell* cell, const double* u, const uint8_t* gate, double dt, const double* r,
                     double* z);

/* Number of coarse levels and the grid of level l (1-based). */
int mb_debug_levels(mb_cell* cell, int* nlev);
int mb_debug_level_dims(mb_cell* cell, int level, int* nt, int* ny, int* nz);

/* Copy level l's operator after mb_debug_precond: aself float[cells*16]
 * (4x4 self block per coarse cell, row-major, classes: 0 electrolyte c,
 * 1 electrolyte phi, 2 anode-side phi, 3 cathode-side phi), off
 * float[cells*96] (six outgoing 4x4 blocks in direction order -t,+t,-y,+y,
 * -z,+z), mask uint8[cells] (classes present). */
int mb_debug_level_op(mb_cell* cell, int level, float* aself, float* off, uint8_t* mask);

/* Fine level after mb_debug_precond: dinv float[4N] (inverse of the scaled
 * condensed 2x2 (c, phi) diagonal block per voxel, row-major) and fc
 * float[8F] (per plating face: scaled D_n, dR_n/dphi_g, dR_n/dc_e,
 * dR_n/dphi_e, dR_phi(g)/dn, dR_c(e)/dn, dR_phi(e)/dn, unused) and rowdiag
 * float[n] (magnitude of each row's diagonal entry of the scaled Jacobian,
 * by which the Krylov rows are divided; mb_debug_precond's r and z are in
 * those row-equilibrated units on input). */
int mb_debug_fine(mb_cell* cell, float* dinv, float* fc, float* rowdiag);
/* The assembled fine smoother stencil of the last mb_debug_precond, as FP32:
 * out[(k * N + v) * 2 + col] for row block k = 2q + r (q = 0 self block of the
 * difference form, 1 + d coupling in direction d; r = 0 c row, 1 phi row),
 * col = 0 c, 1 phi; 14 x N x 2 floats. */
int mb_debug_fine_stencil(mb_cell* cell, float* out);

/* The reduced model's Newton-matrix kernel on given arrays: J[b] = P GU_b +
 * Ms dt_inv[b] + Alin for b < B (P Nr x M row-major, GU M x (B Nr) row-major
 * with column b Nr + j, Ms and Alin Nr x Nr, J B x Nr x Nr); tc = 1 the
 * tensor-core (3xTF32) kernel, 0 FP32 FMA. */
int mb_debug_rom_jac(int Nr, int M, int B, const float* P, const float* GU, const float* Ms, const float* Alin,
                     const double* dt_inv, int tc, float* J);
/* The reduced model's Newton-step LU kernel on given matrices: delta[b] =
 * -J[b]^-1 r[b] for b < B (J B x Nr x Nr row-major, r and delta B x Nr), in
 * FP64 (fp64 = 1) or FP32 arithmetic, the matrix in shared memory (in_place =
 * 0; MB_EINVAL when it does not fit) or factorised in place in device memory. */
int mb_debug_rom_lu(int Nr, int B, int fp64, int in_place, const double* J, const double* r, double* delta);
/* Escalated instances of the online solve: GMRES on FP64 products preconditioned by
 * the instance's last FP32 LU (on = 1, the default), or the FP64 Newton matrix and LU (0). */
int mb_debug_rom_refine(mb_rom* rom, int on);
/* Take each time step of the online solve as one CUDA graph launch (on = 1,
 * the default: conditional nodes run the active-set passes, the Newton
 * iterations and the escalated branch on the device) or drive the loops from
 * the host (0).  Both give the same results. */
int mb_debug_rom_graph(mb_rom* rom, int on);
/* The online solve's Newton-matrix GEMM: 2 on tcgen05 with the accumulator in
 * tensor memory (models with N_r <= 256), 1 mma.sync tensor-core kernel, 0
 * FP32 FMA; all three with FP32 accuracy (3xTF32 on the tensor cores).  By
 * default the first batch of each (N_r, M, B) times the variants the model
 * admits and keeps the fastest; this call fixes the variant instead. */
int mb_debug_rom_tensor(mb_rom* rom, int on);
/* State of slot b of the last batch: failed (0 no, 1 still iterating at the
 * iteration limit, 2 a non-finite update), the Newton iterations of its last
 * pass, the last scaled update norm and whether it had escalated to FP64. */
int mb_debug_rom_slot(mb_rom* rom, int b, int* failed, int* pass_its, float* last_norm, int* escalated);
/* The variant in use (as above) and the last autotuning's time per variant
 * in ms per launch over the whole batch (ms[3]; -1 where not timed). */
int mb_debug_rom_gemm_tuning(mb_rom* rom, int* choice, float* ms);

/* The solver's own Newton residual (interface currents evaluated once per
 * face, then the voxel rows) at u, u_old with gates gate (uint8[F]); the
 * result equals mb_residual's up to the rounding of the summation order.
 * Host double[n] in and out. */
int mb_debug_residual_split(mb_cell* cell, const double* u, const double* u_old, const uint8_t* gate,
                            double dt, double I_app, double* r);

/* Full-order cells of a server: alive now, the most alive at one time since
 * mb_serve_create, and the measured device memory of one cell (0 before the
 * first cell exists). */
int mb_debug_serve_cells(mb_server* srv, int* alive, int* peak, int64_t* cell_bytes);

/* The offline build's symmetric eigensolver (host code, no device needed):
 * A = V diag(w) V^T for a symmetric n x n matrix A (host, row-major, read
 * only), w (host double[n], unordered) and V (host double[n*n], row-major,
 * column j the unit eigenvector of w[j]).  MB_EINVAL for n < 1, a null
 * pointer, or when the QR iteration does not converge. */
int mb_debug_symeig(int n, const double* A, double* w, double* V);

#ifdef __cplusplus
}
#endif
#endif /* MB_DEBUG_H */
