// precond.cu -- preconditioner of the scaled Newton system S_r^-1 J S_u.
//
// 1. Plating rows are condensed out exactly: each face row R_n(f) depends on
//    its own n_f and on the potentials/concentration of its two voxels only,
//    so with D_n = dR_n/dn the voxel system S = J_vv - J_vn D_n^-1 J_nv has
//    the sparsity of the face couplings.  The preconditioner solves
//    S z_v = r_v - J_vn D_n^-1 r_n approximately and back-substitutes
//    z_n = D_n^-1 (r_n - J_nv z_v).
// 2. Fine level: NU_FINE damped 2x2 (c, phi) block-Jacobi sweeps of S before
//    and after the coarse correction; S z is applied as the matrix-free JVP
//    of [z_v, -D_n^-1 J_nv z_v].  Several post-sweeps are needed: with a
//    current source the correction carries a large, weakly pinned potential
//    component, and the jumps its piecewise-constant prolongation leaves at
//    aggregate boundaries otherwise dominate the residual.
// 3. Coarse levels: aggregation of 2x2x2 blocks split by class
//    (0 electrolyte c, 1 electrolyte phi, 2 anode-side phi: G, CN,
//    3 cathode-side phi: K, CP, L); Galerkin operators with piecewise-constant
//    prolongation stored per coarse cell as a 4x4 self block and six 4x4
//    outgoing blocks.  The self block is (row sums by class) - (outgoing
//    couplings), so the large intra-phase conductances never cancel.
//    Level 1 is solved by a K-cycle: FGMRES(KCYC) run entirely on the device,
//    preconditioned by a V-cycle (NU damped 4x4 block-Jacobi sweeps before and
//    after each coarse correction); the coarsest level is solved with an
//    explicit FP64 inverse.  Coarse vectors are FP64, operators FP32.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>

#include <vector>

#include "mb_internal.h"
#include "mb_reduce.cuh"

namespace mb {

constexpr int NCLS = 4;
constexpr int BLK = NCLS * NCLS;          // 16 floats per 4x4 block
constexpr int OFFW = 6 * BLK;             // 96 floats of outgoing couplings per cell
constexpr float OMEGA_FINE = 0.8f;
constexpr double OMEGA_COARSE = 0.7;
constexpr double ALPHA = 1.0;             // scaling of coarse corrections below level 1
constexpr int NU = 2;                     // smoothing sweeps per coarse level (pre and post)
constexpr int NU_FINE = 4;                // fine-level block-Jacobi sweeps (pre and post)
constexpr int KCYC = 16;                  // FGMRES iterations of the level-1 K-cycle (<= 16)
constexpr int MAX_LEVELS = 16;
constexpr int COARSE_MAX = 256;           // dense coarsest system size bound (4 x cells)
constexpr int FCW = 8;                    // floats of condensation coefficients per face

// coarse-level vectors are FP64: FP32 coarse iterates lose the weakly
// coupled (Butler-Volmer) modes to rounding, while FP32 operators are fine
struct alignas(32) D4 {
    double x, y, z, w;
};
__host__ __device__ inline D4 d4(double a, double b, double c, double d) { return D4{a, b, c, d}; }

struct Level {
    int nt = 0, ny = 0, nz = 0;
    int64_t cells = 0;
    float* off = nullptr;     // cells x 6 x 16
    float* ex = nullptr;      // cells x 16  row sums by class
    float* aself = nullptr;   // cells x 16
    float* sinv = nullptr;    // cells x 16
    uint8_t* mask = nullptr;  // cells: classes present
    D4* x = nullptr;          // cells
    D4* x2 = nullptr;         // cells
    D4* b = nullptr;          // cells
};

struct Precond {
    float* dinv = nullptr;     // 4 per voxel: inverse of the condensed scaled (c, phi) block
    float* fc = nullptr;       // FCW per plating face: condensation coefficients (scaled)
    double* rv = nullptr;      // n: condensed right-hand side
    double* t = nullptr;       // n: S z
    int nlev = 0;              // coarse levels (index 1..nlev; lv[0] unused)
    Level lv[MAX_LEVELS + 1];
    int ncoarse = 0;
    double* cdense = nullptr;
    double* cinv = nullptr;
    int* cstat = nullptr;
    // level-1 K-cycle workspace (FP64 arrays of 4 x cells)
    double* kV = nullptr;      // (KCYC+1) x m4
    double* kZ = nullptr;      // KCYC x m4
    double* kw = nullptr;      // m4
    double* kH = nullptr;      // (KCYC+1) x KCYC + scalars
    double* kred = nullptr;    // RED_BLOCKS x 8 partials
};

static const dim3 PB(32, 8, 1);
static inline dim3 pgrid(int nt, int ny, int nz) { return dim3((nz + 31) / 32, (ny + 7) / 8, nt); }
static inline unsigned nblk(int64_t n) { return (unsigned)((n + 255) / 256); }

__host__ __device__ inline int phi_class(int p) {
    return p == PE ? 1 : ((p == PG || p == PCN) ? 2 : 3);
}

// plating face f of voxel v in direction d towards w (-1 if none)
__device__ inline int64_t face_of(int lv, int lw, uint32_t code, uint32_t cw_code, int d, int& rank) {
    if (lv == PG && lw == PE) return (int64_t)vc_fbase(code) + rank++;
    if (lv == PE && lw == PG)
        return (int64_t)vc_fbase(cw_code) + __popc(vc_emask(cw_code) & ((1u << opp_dir(d)) - 1u));
    return -1;
}

// ------------------------------------------------------------ fine level
__global__ void __launch_bounds__(256)
k_bj_setup(DevParams P, Dims D, const uint32_t* __restrict__ vc, const float* __restrict__ u,
           const uint8_t* __restrict__ gate, double dt, double s_i0d, double k_pld,
           float* __restrict__ dinv, float* __restrict__ fc, float* __restrict__ rowdiag) {
    int z = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    int t = blockIdx.z;
    if (z >= D.nz || y >= D.ny) return;
    const int64_t N = D.N;
    int64_t v = (int64_t)t * D.syz + (int64_t)y * D.nz + z;
    const float* cc = u;
    const float* ph = u + N;
    const float* nn = u + 2 * N;
    const float s_i0 = float(s_i0d), k_pl = float(k_pld);
    const float dtf = float(dt), idt = float(1.0 / dt);
    const float nc = float(sqrt(sqrt(P.nc4)));
    const float A = float(P.A), c0 = float(P.cref[PE]);
    uint32_t code = vc[v];
    int lv = vc_phase(code);
    float cv = cc[v], pv = ph[v];
    float d00 = 0.f, d01 = 0.f, d10 = 0.f, d11 = 0.f;
    float dgc = 0.f, dgp = 0.f;   // uncondensed diagonal entries
    const int64_t off[6] = {-D.syz, D.syz, -(int64_t)D.nz, (int64_t)D.nz, -1, 1};
    const bool inb[6] = {t > 0, t < D.nt - 1, y > 0, y < D.ny - 1, z > 0, z < D.nz - 1};
    int rank = 0;
    for (int d = 0; d < 6; ++d) {
        if (!inb[d]) continue;
        int64_t w = v + off[d];
        uint32_t cw_code = vc[w];
        int lw = vc_phase(cw_code);
        int64_t f = face_of(lv, lw, code, cw_code, d, rank);
        float nf = 0.f;
        bool g = false;
        if (f >= 0) {
            nf = nn[f];
            g = gate[f] != 0;
        }
        FaceJac<float> J;
        face_jacobian<float>(P, lv, lw, cv, pv, cc[w], ph[w], nf, g, s_i0, k_pl, J);
        d00 += J.c[0]; d01 += J.c[1]; d10 += J.p[0]; d11 += J.p[1];
        dgc += J.c[0]; dgp += J.p[1];
        if (f >= 0) {
            float jnn = idt + J.n[4];                 // dR_n/dn (unscaled)
            if (lv == PG) {
                d11 -= J.p[4] * J.n[1] / jnn;         // Schur term on phi_g
                fc[FCW * f + 0] = dtf * jnn;          // scaled D_n
                rowdiag[2 * N + f] = fabsf(dtf * jnn);
                fc[FCW * f + 1] = J.n[1] * dtf / nc;  // dR_n/dphi_g
                fc[FCW * f + 2] = J.n[2] * c0 * dtf / nc;   // dR_n/dc_e
                fc[FCW * f + 3] = J.n[3] * dtf / nc;  // dR_n/dphi_e
                fc[FCW * f + 4] = J.p[4] * nc / A;    // dR_phi(g)/dn
            } else {
                d00 -= J.c[4] * J.n[0] / jnn;
                d01 -= J.c[4] * J.n[1] / jnn;
                d10 -= J.p[4] * J.n[0] / jnn;
                d11 -= J.p[4] * J.n[1] / jnn;
                fc[FCW * f + 5] = float(double(J.c[4]) * double(nc) * dt / (P.V * P.cref[PE]));   // dR_c(e)/dn
                fc[FCW * f + 6] = J.p[4] * nc / A;    // dR_phi(e)/dn
            }
        }
    }
    if (t == 0 && lv == PCN) { d11 += float(P.g_dir); dgp += float(P.g_dir); }
    float src, suc = float(P.cref[lv]);
    if (has_c(lv)) {
        d00 += float(P.V / dt);
        dgc += float(P.V / dt);
        src = float(P.V * P.cref[lv] / dt);
        rowdiag[v] = fmaxf(fabsf(dgc * float(dt / P.V)), 1e-30f);
    } else {
        d00 = 1.f; d01 = 0.f; src = 1.f;
        rowdiag[v] = 1.f;
    }
    rowdiag[N + v] = fmaxf(fabsf(dgp / A), 1e-30f);
    float a = d00 * suc / src, b = d01 / src, c = d10 * suc / A, e = d11 / A;
    float id = 1.f / (a * e - b * c);
    reinterpret_cast<float4*>(dinv)[v] = make_float4(e * id, -b * id, -c * id, a * id);
}

// condensed right-hand side r_v - J_vn D_n^-1 r_n (voxel rows of rv); FP64
// vectors (the preconditioned directions carry large near-null components
// whose small structure FP32 would lose), FP32 coefficients
__global__ void __launch_bounds__(256)
k_condense_rhs(Dims D, const uint32_t* __restrict__ vc, const float* __restrict__ fc, const double* __restrict__ r,
               const float* __restrict__ rowdiag, double* __restrict__ rv) {
    int z = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    int t = blockIdx.z;
    if (z >= D.nz || y >= D.ny) return;
    const int64_t N = D.N;
    int64_t v = (int64_t)t * D.syz + (int64_t)y * D.nz + z;
    uint32_t code = vc[v];
    int lv = vc_phase(code);
    // the Krylov residual is row-equilibrated: undo it first
    double rc = r[v] * (double)rowdiag[v], rp = r[N + v] * (double)rowdiag[N + v];
    if (lv == PG || lv == PE) {
        const int64_t off[6] = {-D.syz, D.syz, -(int64_t)D.nz, (int64_t)D.nz, -1, 1};
        const bool inb[6] = {t > 0, t < D.nt - 1, y > 0, y < D.ny - 1, z > 0, z < D.nz - 1};
        int rank = 0;
        for (int d = 0; d < 6; ++d) {
            if (!inb[d]) continue;
            uint32_t cw_code = vc[v + off[d]];
            int64_t f = face_of(lv, vc_phase(cw_code), code, cw_code, d, rank);
            if (f < 0) continue;
            double q = r[2 * N + f] * (double)rowdiag[2 * N + f] / (double)fc[FCW * f + 0];
            if (lv == PG) {
                rp -= (double)fc[FCW * f + 4] * q;
            } else {
                rc -= (double)fc[FCW * f + 5] * q;
                rp -= (double)fc[FCW * f + 6] * q;
            }
        }
    }
    rv[v] = rc;
    rv[N + v] = rp;
}

// z_n = (rn - J_nv z_v) / D_n  with rn = r_n (back-substitution) or 0 (elimination)
__global__ void k_face_solve(Dims D, const int32_t* __restrict__ pg, const int32_t* __restrict__ pe,
                             const float* __restrict__ fc, const double* __restrict__ r,
                             const float* __restrict__ rowdiag, double* __restrict__ z) {
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= D.F) return;
    const int64_t N = D.N;
    int64_t g = pg[f], e = pe[f];
    const float* cf = fc + FCW * f;
    double jz = (double)cf[1] * z[N + g] + (double)cf[2] * z[e] + (double)cf[3] * z[N + e];
    double rn = r ? r[2 * N + f] * (double)rowdiag[2 * N + f] : 0.0;
    z[2 * N + f] = (rn - jz) / (double)cf[0];
}

// z = omega D^-1 rv  (accumulate = false);  z += omega D^-1 (rv - t)  (accumulate = true); voxel rows
__global__ void k_bj_apply(Dims D, const float* __restrict__ dinv, const double* __restrict__ rv,
                           const double* __restrict__ t, double omega, bool accumulate, double* __restrict__ z) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t N = D.N;
    if (i >= N) return;
    double rc = rv[i], rp = rv[N + i];
    if (accumulate) { rc -= t[i]; rp -= t[N + i]; }
    float4 m = reinterpret_cast<const float4*>(dinv)[i];
    double zc = omega * ((double)m.x * rc + (double)m.y * rp), zp = omega * ((double)m.z * rc + (double)m.w * rp);
    if (accumulate) { zc += z[i]; zp += z[N + i]; }
    z[i] = zc;
    z[N + i] = zp;
}

// ------------------------------------------------------- level-1 assembly
__device__ inline void acc_blk(float* blk, int k, int kk, float v) { blk[k * NCLS + kk] += v; }

__global__ void __launch_bounds__(128)
k_assemble_l1(DevParams P, Dims D, const uint32_t* __restrict__ vc, const float* __restrict__ u,
              const uint8_t* __restrict__ gate, double dt, double s_i0d, double k_pld, Level L1) {
    int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= L1.cells) return;
    int cz = (int)(cell % L1.nz);
    int cy = (int)((cell / L1.nz) % L1.ny);
    int ct = (int)(cell / ((int64_t)L1.nz * L1.ny));
    const int64_t N = D.N;
    const float* cc = u;
    const float* ph = u + N;
    const float* nn = u + 2 * N;
    const float s_i0 = float(s_i0d), k_pl = float(k_pld);
    const float A = float(P.A);
    const float c0 = float(P.cref[PE]);
    const float idt = float(1.0 / dt);
    // scaling of rows (1/s_r) and columns (s_u) into the Krylov units
    const float sc_cc = float(dt / P.V);                 // (row c, col c)
    const float sc_cp = float(dt / (P.V * P.cref[PE]));  // (row c, col phi)
    const float sc_pc = c0 / A;                          // (row phi, col c)
    const float sc_pp = 1.f / A;                         // (row phi, col phi)
    float ex[BLK];
    float off[OFFW];
    for (int i = 0; i < BLK; ++i) ex[i] = 0.f;
    for (int i = 0; i < OFFW; ++i) off[i] = 0.f;
    uint32_t mask = 0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int e = 0; e < 2; ++e) {
                int t = 2 * ct + a, y = 2 * cy + b, z = 2 * cz + e;
                if (t >= D.nt || y >= D.ny || z >= D.nz) continue;
                int64_t v = (int64_t)t * D.syz + (int64_t)y * D.nz + z;
                uint32_t code = vc[v];
                int lv = vc_phase(code);
                int kv = phi_class(lv);
                mask |= 1u << kv;
                if (lv == PE) {
                    mask |= 1u;
                    acc_blk(ex, 0, 0, 1.f);   // storage V/dt, scaled
                }
                if (t == 0 && lv == PCN) acc_blk(ex, kv, kv, float(P.g_dir) * sc_pp);
                float cv = cc[v], pv = ph[v];
                const int64_t offs[6] = {-D.syz, D.syz, -(int64_t)D.nz, (int64_t)D.nz, -1, 1};
                const bool inb[6] = {t > 0, t < D.nt - 1, y > 0, y < D.ny - 1, z > 0, z < D.nz - 1};
                const int loc[6] = {a, a, b, b, e, e};
                int rank = 0;
                for (int d = 0; d < 6; ++d) {
                    if (!inb[d]) continue;
                    int64_t w = v + offs[d];
                    uint32_t cw_code = vc[w];
                    int lw = vc_phase(cw_code);
                    int kw = phi_class(lw);
                    // neighbour outside this coarse cell?
                    bool other = (d & 1) ? (loc[d] == 1) : (loc[d] == 0);
                    float* od = off + d * BLK;
                    int64_t f = face_of(lv, lw, code, cw_code, d, rank);
                    float nf = 0.f;
                    bool g = false;
                    if (f >= 0) {
                        nf = nn[f];
                        g = gate[f] != 0;
                    }
                    float cw = cc[w], pw = ph[w];
                    FaceJac<float> J;
                    face_jacobian<float>(P, lv, lw, cv, pv, cw, pw, nf, g, s_i0, k_pl, J);
                    if (lv == PE && lw == PE) {
                        // row sums of the face terms without cancellation:
                        // dj/dc_v + dj/dc_w = gm dc/S^2 (m_v + m_w); the conduction parts cancel exactly
                        float cmin = float(P.cmin[PE]);
                        float S = fmaxf(cv, cmin) + fmaxf(cw, cmin);
                        float exc = float(P.E_gm) * (cw - cv) / (S * S) *
                                    ((cv >= cmin ? 1.f : 0.f) + (cw >= cmin ? 1.f : 0.f));
                        acc_blk(ex, 0, 0, float(P.E_tF) * exc * sc_cc);
                        acc_blk(ex, 1, 0, exc * sc_pc);
                        if (other) {
                            acc_blk(od, 0, 0, J.c[2] * sc_cc);
                            acc_blk(od, 0, 1, J.c[3] * sc_cp);
                            acc_blk(od, 1, 0, J.p[2] * sc_pc);
                            acc_blk(od, 1, 1, J.p[3] * sc_pp);
                        }
                    } else if (lv != PE && lw != PE) {
                        // conduction between electronic conductors (solid c rows are not coarse)
                        if (kv == kw) {
                            if (other) acc_blk(od, kv, kv, J.p[3] * sc_pp);
                        } else {
                            acc_blk(ex, kv, kv, J.p[1] * sc_pp);
                            acc_blk(ex, kv, kw, J.p[3] * sc_pp);
                            if (other) acc_blk(od, kv, kw, J.p[3] * sc_pp);
                        }
                    } else if (lv != PE) {
                        // solid v, electrolyte w (interface kinetics; zero for collectors)
                        float s_pp = J.p[1], s_pc = J.p[2], s_pe = J.p[3];
                        if (f >= 0) {   // condensed plating row
                            float jnn = idt + J.n[4];
                            s_pp -= J.p[4] * J.n[1] / jnn;
                            s_pc -= J.p[4] * J.n[2] / jnn;
                            s_pe -= J.p[4] * J.n[3] / jnn;
                        }
                        acc_blk(ex, kv, kv, s_pp * sc_pp);
                        acc_blk(ex, kv, 0, s_pc * sc_pc);
                        acc_blk(ex, kv, 1, s_pe * sc_pp);
                        if (other) {
                            acc_blk(od, kv, 0, s_pc * sc_pc);
                            acc_blk(od, kv, 1, s_pe * sc_pp);
                        }
                    } else {
                        // electrolyte v, solid w
                        float cc0 = J.c[0], cc1 = J.c[1], cc3 = J.c[3];
                        float pp0 = J.p[0], pp1 = J.p[1], pp3 = J.p[3];
                        if (f >= 0) {   // condensed plating row
                            float jnn = idt + J.n[4];
                            cc0 -= J.c[4] * J.n[0] / jnn; cc1 -= J.c[4] * J.n[1] / jnn; cc3 -= J.c[4] * J.n[3] / jnn;
                            pp0 -= J.p[4] * J.n[0] / jnn; pp1 -= J.p[4] * J.n[1] / jnn; pp3 -= J.p[4] * J.n[3] / jnn;
                        }
                        acc_blk(ex, 0, 0, cc0 * sc_cc);
                        acc_blk(ex, 0, 1, cc1 * sc_cp);
                        acc_blk(ex, 0, kw, cc3 * sc_cp);
                        acc_blk(ex, 1, 0, pp0 * sc_pc);
                        acc_blk(ex, 1, 1, pp1 * sc_pp);
                        acc_blk(ex, 1, kw, pp3 * sc_pp);
                        if (other) {
                            acc_blk(od, 0, kw, cc3 * sc_cp);
                            acc_blk(od, 1, kw, pp3 * sc_pp);
                        }
                    }
                }
            }
    for (int i = 0; i < BLK; ++i) L1.ex[cell * BLK + i] = ex[i];
    for (int i = 0; i < OFFW; ++i) L1.off[cell * OFFW + i] = off[i];
    L1.mask[cell] = (uint8_t)mask;
}

// Galerkin coarsening of a coarse level: row sums add up; a child's outgoing
// couplings in direction d leave the parent when the child sits on its d side.
__global__ void k_assemble_up(Level F, Level C) {
    int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= C.cells) return;
    int cz = (int)(cell % C.nz);
    int cy = (int)((cell / C.nz) % C.ny);
    int ct = (int)(cell / ((int64_t)C.nz * C.ny));
    float ex[BLK];
    float off[OFFW];
    for (int i = 0; i < BLK; ++i) ex[i] = 0.f;
    for (int i = 0; i < OFFW; ++i) off[i] = 0.f;
    uint32_t mask = 0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int e = 0; e < 2; ++e) {
                int t = 2 * ct + a, y = 2 * cy + b, z = 2 * cz + e;
                if (t >= F.nt || y >= F.ny || z >= F.nz) continue;
                int64_t ch = ((int64_t)t * F.ny + y) * F.nz + z;
                mask |= F.mask[ch];
                for (int i = 0; i < BLK; ++i) ex[i] += F.ex[ch * BLK + i];
                const int loc[6] = {a, a, b, b, e, e};
                for (int d = 0; d < 6; ++d) {
                    bool other = (d & 1) ? (loc[d] == 1) : (loc[d] == 0);
                    if (!other) continue;
                    for (int i = 0; i < BLK; ++i) off[d * BLK + i] += F.off[ch * OFFW + d * BLK + i];
                }
            }
    for (int i = 0; i < BLK; ++i) C.ex[cell * BLK + i] = ex[i];
    for (int i = 0; i < OFFW; ++i) C.off[cell * OFFW + i] = off[i];
    C.mask[cell] = (uint8_t)mask;
}

// self block = row sums - outgoing couplings; absent classes get an identity
// row; the block inverse by Gauss-Jordan with partial pivoting (FP64).
__global__ void k_finalize(Level L) {
    int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= L.cells) return;
    double a[NCLS][2 * NCLS];
    uint32_t mask = L.mask[cell];
    for (int k = 0; k < NCLS; ++k)
        for (int kk = 0; kk < NCLS; ++kk) {
            double s = L.ex[cell * BLK + k * NCLS + kk];
            for (int d = 0; d < 6; ++d) s -= L.off[cell * OFFW + d * BLK + k * NCLS + kk];
            if (!((mask >> k) & 1u) || !((mask >> kk) & 1u)) s = (k == kk && !((mask >> k) & 1u)) ? 1.0 : 0.0;
            a[k][kk] = s;
            a[k][NCLS + kk] = (k == kk) ? 1.0 : 0.0;
            L.aself[cell * BLK + k * NCLS + kk] = (float)s;
        }
    for (int col = 0; col < NCLS; ++col) {
        int piv = col;
        for (int r = col + 1; r < NCLS; ++r)
            if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        if (piv != col)
            for (int j = 0; j < 2 * NCLS; ++j) { double tmp = a[col][j]; a[col][j] = a[piv][j]; a[piv][j] = tmp; }
        double p = a[col][col];
        double ip = p != 0.0 ? 1.0 / p : 0.0;
        for (int j = 0; j < 2 * NCLS; ++j) a[col][j] *= ip;
        for (int r = 0; r < NCLS; ++r) {
            if (r == col) continue;
            double fct = a[r][col];
            if (fct != 0.0)
                for (int j = 0; j < 2 * NCLS; ++j) a[r][j] -= fct * a[col][j];
        }
    }
    for (int k = 0; k < NCLS; ++k)
        for (int kk = 0; kk < NCLS; ++kk) L.sinv[cell * BLK + k * NCLS + kk] = (float)a[k][NCLS + kk];
}

// ----------------------------------------------------- coarsest dense solve
__global__ void k_coarse_dense(Level L, int n, double* __restrict__ Ad) {
    int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= n) return;
    int64_t cell = row / NCLS;
    int k = row % NCLS;
    for (int j = 0; j < n; ++j) Ad[(int64_t)row * n + j] = 0.0;
    int cz = (int)(cell % L.nz);
    int cy = (int)((cell / L.nz) % L.ny);
    int ct = (int)(cell / ((int64_t)L.nz * L.ny));
    for (int kk = 0; kk < NCLS; ++kk) Ad[(int64_t)row * n + cell * NCLS + kk] = L.aself[cell * BLK + k * NCLS + kk];
    const int dt_[6] = {-1, 1, 0, 0, 0, 0}, dy_[6] = {0, 0, -1, 1, 0, 0}, dz_[6] = {0, 0, 0, 0, -1, 1};
    for (int d = 0; d < 6; ++d) {
        int t = ct + dt_[d], y = cy + dy_[d], z = cz + dz_[d];
        if (t < 0 || t >= L.nt || y < 0 || y >= L.ny || z < 0 || z >= L.nz) continue;
        int64_t nb = ((int64_t)t * L.ny + y) * L.nz + z;
        for (int kk = 0; kk < NCLS; ++kk)
            Ad[(int64_t)row * n + nb * NCLS + kk] += L.off[cell * OFFW + d * BLK + k * NCLS + kk];
    }
}

// Gauss-Jordan inverse with partial pivoting, one block.
__global__ void k_coarse_invert(int n, double* __restrict__ A, double* __restrict__ Ainv, int* __restrict__ stat) {
    __shared__ int piv;
    __shared__ double pval;
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) Ainv[i] = (i / n == i % n) ? 1.0 : 0.0;
    __syncthreads();
    for (int col = 0; col < n; ++col) {
        if (threadIdx.x == 0) {
            int p = col;
            double best = fabs(A[(int64_t)col * n + col]);
            for (int r = col + 1; r < n; ++r) {
                double v = fabs(A[(int64_t)r * n + col]);
                if (v > best) { best = v; p = r; }
            }
            piv = p;
            pval = A[(int64_t)p * n + col];
            if (pval == 0.0) *stat = 1;
        }
        __syncthreads();
        if (piv != col) {
            for (int j = threadIdx.x; j < n; j += blockDim.x) {
                double t1 = A[(int64_t)col * n + j]; A[(int64_t)col * n + j] = A[(int64_t)piv * n + j]; A[(int64_t)piv * n + j] = t1;
                double t2 = Ainv[(int64_t)col * n + j]; Ainv[(int64_t)col * n + j] = Ainv[(int64_t)piv * n + j]; Ainv[(int64_t)piv * n + j] = t2;
            }
        }
        __syncthreads();
        double ip = pval != 0.0 ? 1.0 / pval : 0.0;
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            A[(int64_t)col * n + j] *= ip;
            Ainv[(int64_t)col * n + j] *= ip;
        }
        __syncthreads();
        // A[r][col] is only read here (column col of A is cleared afterwards)
        for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
            int r = idx / n, j = idx % n;
            if (r == col) continue;
            double f = A[(int64_t)r * n + col];
            if (j != col) A[(int64_t)r * n + j] -= f * A[(int64_t)col * n + j];
            Ainv[(int64_t)r * n + j] -= f * Ainv[(int64_t)col * n + j];
        }
        __syncthreads();
        for (int r = threadIdx.x; r < n; r += blockDim.x)
            if (r != col) A[(int64_t)r * n + col] = 0.0;
        __syncthreads();
    }
}

// x = Ainv b (FP64 accumulation), one block
__global__ void k_coarse_solve(int n, const double* __restrict__ Ainv, const D4* __restrict__ b,
                               D4* __restrict__ x) {
    __shared__ double sb[COARSE_MAX];
    const double* bf = reinterpret_cast<const double*>(b);
    for (int i = threadIdx.x; i < n; i += blockDim.x) sb[i] = bf[i];
    __syncthreads();
    double* xf = reinterpret_cast<double*>(x);
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        double acc = 0.0;
        for (int j = 0; j < n; ++j) acc += Ainv[(int64_t)r * n + j] * sb[j];
        xf[r] = acc;
    }
}

// --------------------------------------------------------- coarse smoothing
__device__ inline D4 mv4(const float* m, D4 x) {
    return d4((double)m[0] * x.x + (double)m[1] * x.y + (double)m[2] * x.z + (double)m[3] * x.w,
              (double)m[4] * x.x + (double)m[5] * x.y + (double)m[6] * x.z + (double)m[7] * x.w,
              (double)m[8] * x.x + (double)m[9] * x.y + (double)m[10] * x.z + (double)m[11] * x.w,
              (double)m[12] * x.x + (double)m[13] * x.y + (double)m[14] * x.z + (double)m[15] * x.w);
}
__device__ inline D4 f4sub(D4 a, D4 b) { return d4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w); }
__device__ inline D4 f4add(D4 a, D4 b) { return d4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }
__device__ inline D4 f4scale(double s, D4 a) { return d4(s * a.x, s * a.y, s * a.z, s * a.w); }

// effective iterate of a cell: x (if given) plus alpha times the prolonged coarse correction (if given)
__device__ inline D4 xeff(const D4* x, const D4* ec, double alpha, int ccny, int ccnz, int t, int y, int z,
                          int64_t cell) {
    D4 r = x ? x[cell] : d4(0.0, 0.0, 0.0, 0.0);
    if (ec) r = f4add(r, f4scale(alpha, ec[((int64_t)(t >> 1) * ccny + (y >> 1)) * ccnz + (z >> 1)]));
    return r;
}

// A x at one cell of level L
__device__ inline D4 cell_apply(const Level& L, const D4* x, const D4* ec, double alpha, int ccny, int ccnz, int t,
                                int y, int z, int64_t cell) {
    D4 acc = mv4(L.aself + cell * BLK, xeff(x, ec, alpha, ccny, ccnz, t, y, z, cell));
    const int dt_[6] = {-1, 1, 0, 0, 0, 0}, dy_[6] = {0, 0, -1, 1, 0, 0}, dz_[6] = {0, 0, 0, 0, -1, 1};
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        int tt = t + dt_[d], yy = y + dy_[d], zz = z + dz_[d];
        if (tt < 0 || tt >= L.nt || yy < 0 || yy >= L.ny || zz < 0 || zz >= L.nz) continue;
        int64_t nb = ((int64_t)tt * L.ny + yy) * L.nz + zz;
        acc = f4add(acc, mv4(L.off + cell * OFFW + d * BLK, xeff(x, ec, alpha, ccny, ccnz, tt, yy, zz, nb)));
    }
    return acc;
}

__device__ inline void cell_coords(const Level& L, int64_t cell, int& t, int& y, int& z) {
    z = (int)(cell % L.nz);
    y = (int)((cell / L.nz) % L.ny);
    t = (int)(cell / ((int64_t)L.nz * L.ny));
}

// x_out = xe + omega Sinv (b - A xe), xe = x_in (+ alpha * prolonged ec)
__global__ void k_lvl_smooth(Level L, const D4* __restrict__ x_in, const D4* __restrict__ ec, double alpha, int ccny,
                             int ccnz, double omega, D4* __restrict__ x_out) {
    int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= L.cells) return;
    int t, y, z;
    cell_coords(L, cell, t, y, z);
    D4 xe = xeff(x_in, ec, alpha, ccny, ccnz, t, y, z, cell);
    D4 r = (x_in || ec) ? f4sub(L.b[cell], cell_apply(L, x_in, ec, alpha, ccny, ccnz, t, y, z, cell)) : L.b[cell];
    x_out[cell] = f4add(xe, f4scale(omega, mv4(L.sinv + cell * BLK, r)));
}

__global__ void k_lvl_matvec(Level L, const D4* __restrict__ x, D4* __restrict__ y_out) {
    int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= L.cells) return;
    int t, y, z;
    cell_coords(L, cell, t, y, z);
    y_out[cell] = cell_apply(L, x, nullptr, 0.0, 0, 0, t, y, z, cell);
}

// bc(parent) = sum over children of (b - A x)
__global__ void k_lvl_restrict(Level L, const D4* __restrict__ x, Level C) {
    int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= C.cells) return;
    int ct, cy, cz;
    cell_coords(C, cell, ct, cy, cz);
    D4 acc = d4(0.0, 0.0, 0.0, 0.0);
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int e = 0; e < 2; ++e) {
                int t = 2 * ct + a, y = 2 * cy + b, z = 2 * cz + e;
                if (t >= L.nt || y >= L.ny || z >= L.nz) continue;
                int64_t ch = ((int64_t)t * L.ny + y) * L.nz + z;
                acc = f4add(acc, f4sub(L.b[ch], cell_apply(L, x, nullptr, 0.0, 0, 0, t, y, z, ch)));
            }
    C.b[cell] = acc;
}

// ----------------------------------------------------- fine <-> level 1
__global__ void k_restrict_fine(Dims D, const uint32_t* __restrict__ vc, const double* __restrict__ r,
                                const double* __restrict__ t, Level C) {
    int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= C.cells) return;
    int ct, cy, cz;
    cell_coords(C, cell, ct, cy, cz);
    double acc[NCLS] = {0.0, 0.0, 0.0, 0.0};
    const int64_t N = D.N;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int e = 0; e < 2; ++e) {
                int tt = 2 * ct + a, y = 2 * cy + b, z = 2 * cz + e;
                if (tt >= D.nt || y >= D.ny || z >= D.nz) continue;
                int64_t v = (int64_t)tt * D.syz + (int64_t)y * D.nz + z;
                int lv = vc_phase(vc[v]);
                acc[phi_class(lv)] += r[N + v] - t[N + v];
                if (lv == PE) acc[0] += r[v] - t[v];
            }
    C.b[cell] = d4(acc[0], acc[1], acc[2], acc[3]);
}

__global__ void k_prolong_fine(Dims D, const uint32_t* __restrict__ vc, Level C, const D4* __restrict__ e1,
                               double* __restrict__ z) {
    int zz = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    int t = blockIdx.z;
    if (zz >= D.nz || y >= D.ny) return;
    int64_t v = (int64_t)t * D.syz + (int64_t)y * D.nz + zz;
    int lv = vc_phase(vc[v]);
    D4 e = e1[((int64_t)(t >> 1) * C.ny + (y >> 1)) * C.nz + (zz >> 1)];
    double ev[NCLS] = {e.x, e.y, e.z, e.w};
    z[D.N + v] += ev[phi_class(lv)];
    if (lv == PE) z[v] += e.x;
}

// ------------------------------------------- device-side FGMRES (K-cycle)
// Small Krylov kernels whose scalars stay in device memory, so the level-1
// K-cycle needs no host round trip.
__global__ void __launch_bounds__(RED_THREADS)
k_kdot(const double* __restrict__ V, int64_t stride, int cnt, const double* __restrict__ w, int64_t n,
       double* partials) {
    double acc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double wi = w[i];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (j < cnt) acc[j] += V[j * stride + i] * wi;
    }
    block_reduce_store<8, false>(acc, partials);
}

// w += sign * sum_j h[j] V_j (h on the device)
__global__ void k_kupdate(const double* __restrict__ V, int64_t stride, int cnt, const double* __restrict__ h,
                          double sign, double* __restrict__ w, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double acc = 0.0;
    for (int j = 0; j < cnt; ++j) acc += h[j] * V[j * stride + i];
    w[i] = w[i] + sign * acc;
}

// out = a / sqrt(max(d2, tiny))
__global__ void k_knormalize(const double* __restrict__ a, const double* __restrict__ d2, double* __restrict__ out,
                             int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double nrm = sqrt(fmax(*d2, 1e-300));
    out[i] = a[i] / nrm;
}

// H layout: col-major (KCYC+1) x KCYC at H[j*(KCYC+1) + i]; s[0] = ||b||^2, s[1..] CGS scratch
// After CGS2 of column j: h = h1 + h2, H[j+1, j] = ||w||.
__global__ void k_kcol(double* H, int j, const double* h1, const double* h2, const double* wn2) {
    int i = threadIdx.x;
    if (i <= j) H[j * (KCYC + 1) + i] = h1[i] + h2[i];
    if (i == 0) H[j * (KCYC + 1) + j + 1] = sqrt(fmax(*wn2, 0.0));
}

// least squares min || beta e1 - H y || by Givens rotations (one thread)
__global__ void k_klsq(const double* H, const double* b2, int k, double* y) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double R[KCYC + 1][KCYC];
    double g[KCYC + 1];
    for (int j = 0; j < k; ++j)
        for (int i = 0; i <= k; ++i) R[i][j] = H[j * (KCYC + 1) + i];
    for (int i = 0; i <= k; ++i) g[i] = 0.0;
    g[0] = sqrt(fmax(*b2, 0.0));
    for (int j = 0; j < k; ++j) {
        double a = R[j][j], b = R[j + 1][j];
        double den = sqrt(a * a + b * b);
        double cs = den > 0 ? a / den : 1.0, sn = den > 0 ? b / den : 0.0;
        for (int l = j; l < k; ++l) {
            double r1 = R[j][l], r2 = R[j + 1][l];
            R[j][l] = cs * r1 + sn * r2;
            R[j + 1][l] = -sn * r1 + cs * r2;
        }
        double g1 = g[j], g2 = g[j + 1];
        g[j] = cs * g1 + sn * g2;
        g[j + 1] = -sn * g1 + cs * g2;
    }
    for (int i = k - 1; i >= 0; --i) {
        double acc = g[i];
        for (int l = i + 1; l < k; ++l) acc -= R[i][l] * y[l];
        y[i] = R[i][i] != 0.0 ? acc / R[i][i] : 0.0;
    }
}

// ------------------------------------------------------------ host side
int precond_create(mb_cell* c) {
    Precond* p = new Precond();
    c->pc = p;
    const Dims& D = c->D;
    p->dinv = (float*)cell_alloc(c, 16 * D.N);
    p->fc = (float*)cell_alloc(c, 4 * FCW * (D.F ? D.F : 1));
    p->rv = (double*)cell_alloc(c, 8 * c->n);
    p->t = (double*)cell_alloc(c, 8 * c->n);
    c->rowdiag = (float*)cell_alloc(c, 4 * c->n);
    if (!p->dinv || !p->fc || !p->rv || !p->t || !c->rowdiag) return MB_ENOMEM;
    int coarse_cells = c->opt.mg_coarse_cells;
    if (coarse_cells < 1) coarse_cells = 1;
    if (coarse_cells * NCLS > COARSE_MAX) coarse_cells = COARSE_MAX / NCLS;
    int nt = D.nt, ny = D.ny, nz = D.nz;
    int nlev = 0;
    while (nlev < MAX_LEVELS) {
        nt = (nt + 1) / 2; ny = (ny + 1) / 2; nz = (nz + 1) / 2;
        ++nlev;
        Level& L = p->lv[nlev];
        L.nt = nt; L.ny = ny; L.nz = nz;
        L.cells = (int64_t)nt * ny * nz;
        L.off = (float*)cell_alloc(c, 4 * (size_t)L.cells * OFFW);
        L.ex = (float*)cell_alloc(c, 4 * (size_t)L.cells * BLK);
        L.aself = (float*)cell_alloc(c, 4 * (size_t)L.cells * BLK);
        L.sinv = (float*)cell_alloc(c, 4 * (size_t)L.cells * BLK);
        L.mask = (uint8_t*)cell_alloc(c, (size_t)L.cells);
        L.x = (D4*)cell_alloc(c, 32 * (size_t)L.cells);
        L.x2 = (D4*)cell_alloc(c, 32 * (size_t)L.cells);
        L.b = (D4*)cell_alloc(c, 32 * (size_t)L.cells);
        if (!L.off || !L.ex || !L.aself || !L.sinv || !L.mask || !L.x || !L.x2 || !L.b) return MB_ENOMEM;
        if (L.cells <= coarse_cells) break;
        if (nt == 1 && ny == 1 && nz == 1) break;
    }
    p->nlev = nlev;
    p->ncoarse = (int)(p->lv[nlev].cells * NCLS);
    if (p->ncoarse > COARSE_MAX) {
        set_error("multigrid: coarsest level too large");
        return MB_EINVAL;
    }
    size_t nn = (size_t)p->ncoarse * p->ncoarse;
    p->cdense = (double*)cell_alloc(c, 8 * nn);
    p->cinv = (double*)cell_alloc(c, 8 * nn);
    p->cstat = (int*)cell_alloc(c, 16);
    int64_t m4 = 4 * p->lv[1].cells;
    p->kV = (double*)cell_alloc(c, 8 * (size_t)m4 * (KCYC + 1));
    p->kZ = (double*)cell_alloc(c, 8 * (size_t)m4 * KCYC);
    p->kw = (double*)cell_alloc(c, 8 * (size_t)m4);
    p->kH = (double*)cell_alloc(c, 8 * (size_t)((KCYC + 1) * KCYC + 64));
    p->kred = (double*)cell_alloc(c, 8 * (size_t)RED_BLOCKS * 8);
    if (!p->cdense || !p->cinv || !p->cstat || !p->kV || !p->kZ || !p->kw || !p->kH || !p->kred) return MB_ENOMEM;
    return MB_OK;
}

void precond_destroy(mb_cell* c) {
    delete c->pc;
    c->pc = nullptr;
}

int precond_setup(mb_cell* c, const float* u32, const uint8_t* gate, double dt) {
    Precond* p = c->pc;
    const Dims& D = c->D;
    cudaStream_t s = c->stream;
    k_bj_setup<<<pgrid(D.nt, D.ny, D.nz), PB, 0, s>>>(c->P, D, c->vcode, u32, gate, dt, c->s_i0, c->k_pl,
                                                       p->dinv, p->fc, c->rowdiag), ::mb::count_launch(c);
    Level& L1 = p->lv[1];
    k_assemble_l1<<<(unsigned)((L1.cells + 127) / 128), 128, 0, s>>>(c->P, D, c->vcode, u32, gate, dt, c->s_i0,
                                                                      c->k_pl, L1), ::mb::count_launch(c);
    for (int l = 2; l <= p->nlev; ++l)
        k_assemble_up<<<nblk(p->lv[l].cells), 256, 0, s>>>(p->lv[l - 1], p->lv[l]), ::mb::count_launch(c);
    for (int l = 1; l <= p->nlev; ++l) k_finalize<<<nblk(p->lv[l].cells), 256, 0, s>>>(p->lv[l]), ::mb::count_launch(c);
    int n = p->ncoarse;
    Level& Lc = p->lv[p->nlev];
    k_coarse_dense<<<(n + 127) / 128, 128, 0, s>>>(Lc, n, p->cdense), ::mb::count_launch(c);
    MB_CUDA(cudaMemsetAsync(p->cstat, 0, 4, s));
    k_coarse_invert<<<1, 256, 0, s>>>(n, p->cdense, p->cinv, p->cstat), ::mb::count_launch(c);
    MB_CUDA_LAUNCH("precond_setup");
    return MB_OK;
}

// V-cycle on levels l..nlev with right-hand side lv[l].b; result in lv[l].x
static void vcycle(mb_cell* c, int l) {
    Precond* p = c->pc;
    cudaStream_t s = c->stream;
    Level& L = p->lv[l];
    if (l == p->nlev) {
        k_coarse_solve<<<1, 256, 0, s>>>(p->ncoarse, p->cinv, L.b, L.x), ::mb::count_launch(c);
        return;
    }
    Level& C = p->lv[l + 1];
    unsigned g = nblk(L.cells);
    k_lvl_smooth<<<g, 256, 0, s>>>(L, nullptr, nullptr, 0.0, 0, 0, OMEGA_COARSE, L.x), ::mb::count_launch(c);
    for (int k = 1; k < NU; ++k) {
        k_lvl_smooth<<<g, 256, 0, s>>>(L, L.x, nullptr, 0.0, 0, 0, OMEGA_COARSE, L.x2), ::mb::count_launch(c);
        std::swap(L.x, L.x2);
    }
    k_lvl_restrict<<<nblk(C.cells), 256, 0, s>>>(L, L.x, C), ::mb::count_launch(c);
    vcycle(c, l + 1);
    // post-smoothing, the first sweep applied to x + ALPHA P e
    k_lvl_smooth<<<g, 256, 0, s>>>(L, L.x, C.x, ALPHA, C.ny, C.nz, OMEGA_COARSE, L.x2), ::mb::count_launch(c);
    std::swap(L.x, L.x2);
    for (int k = 1; k < NU; ++k) {
        k_lvl_smooth<<<g, 256, 0, s>>>(L, L.x, nullptr, 0.0, 0, 0, OMEGA_COARSE, L.x2), ::mb::count_launch(c);
        std::swap(L.x, L.x2);
    }
}

static void kdots(mb_cell* c, const double* V, int64_t stride, int cnt, const double* w, int64_t n, double* out) {
    Precond* p = c->pc;
    cudaStream_t s = c->stream;
    for (int j0 = 0; j0 < cnt; j0 += 8) {
        int k = cnt - j0 < 8 ? cnt - j0 : 8;
        k_kdot<<<RED_BLOCKS, RED_THREADS, 0, s>>>(V + j0 * stride, stride, k, w, n, p->kred), ::mb::count_launch(c);
        k_reduce_final<false><<<k, RED_THREADS, 0, s>>>(p->kred, k, out + j0), ::mb::count_launch(c);
    }
}

// Level-1 K-cycle: KCYC iterations of FGMRES on A1 x = b1 (b1 = lv[1].b),
// preconditioned by the V-cycle; result in lv[1].x.  No host synchronisation.
static void kcycle_l1(mb_cell* c) {
    Precond* p = c->pc;
    cudaStream_t s = c->stream;
    Level& L = p->lv[1];
    if (p->nlev == 1) {
        vcycle(c, 1);
        return;
    }
    const int64_t m4 = 4 * L.cells;
    const unsigned g = nblk(m4);
    double* H = p->kH;
    double* sc = p->kH + (KCYC + 1) * KCYC;   // scalars: [0] ||b||^2, [8..] h1, [24..] h2, [40] ||w||^2, [48..] y
    double* b2 = sc;
    double* h1 = sc + 8;
    double* h2 = sc + 24;
    double* wn2 = sc + 40;
    double* y = sc + 48;
    const double* b = reinterpret_cast<const double*>(L.b);
    kdots(c, b, 0, 1, b, m4, b2);
    k_knormalize<<<g, 256, 0, s>>>(b, b2, p->kV, m4), ::mb::count_launch(c);
    D4* bsave = L.b;   // the V-cycle reads lv[1].b: point it at the Krylov vector
    for (int j = 0; j < KCYC; ++j) {
        double* Vj = p->kV + j * m4;
        double* Zj = p->kZ + j * m4;
        L.b = reinterpret_cast<D4*>(Vj);
        vcycle(c, 1);
        cudaMemcpyAsync(Zj, L.x, 8 * m4, cudaMemcpyDeviceToDevice, s);
        k_lvl_matvec<<<nblk(L.cells), 256, 0, s>>>(L, reinterpret_cast<const D4*>(Zj), reinterpret_cast<D4*>(p->kw)), ::mb::count_launch(c);
        kdots(c, p->kV, m4, j + 1, p->kw, m4, h1);
        k_kupdate<<<g, 256, 0, s>>>(p->kV, m4, j + 1, h1, -1.0, p->kw, m4), ::mb::count_launch(c);
        kdots(c, p->kV, m4, j + 1, p->kw, m4, h2);
        k_kupdate<<<g, 256, 0, s>>>(p->kV, m4, j + 1, h2, -1.0, p->kw, m4), ::mb::count_launch(c);
        kdots(c, p->kw, 0, 1, p->kw, m4, wn2);
        k_kcol<<<1, 32, 0, s>>>(H, j, h1, h2, wn2), ::mb::count_launch(c);
        k_knormalize<<<g, 256, 0, s>>>(p->kw, wn2, p->kV + (j + 1) * m4, m4), ::mb::count_launch(c);
    }
    L.b = bsave;
    k_klsq<<<1, 1, 0, s>>>(H, b2, KCYC, y), ::mb::count_launch(c);
    cudaMemsetAsync(L.x, 0, 32 * L.cells, s);
    k_kupdate<<<g, 256, 0, s>>>(p->kZ, m4, KCYC, y, 1.0, reinterpret_cast<double*>(L.x), m4), ::mb::count_launch(c);
}

// ---- MB_DEBUG >= 2: 2-norms of the intermediate vectors of one application
template <class T>
__global__ void __launch_bounds__(RED_THREADS) k_sumsq(const T* __restrict__ a, int64_t n, double* partials) {
    double acc[1] = {0.0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc[0] += (double)a[i] * (double)a[i];
    block_reduce_store<1, false>(acc, partials);
}

template <class T>
static double dbg_norm(mb_cell* c, const T* a, int64_t n) {
    k_sumsq<T><<<RED_BLOCKS, RED_THREADS, 0, c->stream>>>(a, n, c->pc->kred), ::mb::count_launch(c);
    k_reduce_final<false><<<1, RED_THREADS, 0, c->stream>>>(c->pc->kred, 1, c->red_out + 63), ::mb::count_launch(c);
    double h = 0.0;
    cudaMemcpyAsync(&h, c->red_out + 63, 8, cudaMemcpyDeviceToHost, c->stream);
    cudaStreamSynchronize(c->stream);
    return sqrt(h);
}

int debug_level();

int precond_apply(mb_cell* c, const float* u32, const uint8_t* gate, double dt, const double* r, double* z) {
    if (debug_level() >= 2) {
        Precond* p = c->pc;
        int rc = 0;
        const Dims& D = c->D;
        fprintf(stderr, "[mb-pc] levels %d coarse n %d |r| %.3e |rowdiag| %.3e\n", p->nlev, p->ncoarse,
                dbg_norm(c, r, c->n), dbg_norm(c, c->rowdiag, c->n));
        (void)rc; (void)D;
    }
    Precond* p = c->pc;
    const Dims& D = c->D;
    cudaStream_t s = c->stream;
    const dim3 vg = pgrid(D.nt, D.ny, D.nz);
    const unsigned fg = nblk(D.F ? D.F : 1);
    cudaEvent_t ev_pc;
    prof_begin(c, s, &ev_pc);
    // condensed right-hand side, then NU_FINE damped block-Jacobi sweeps from zero
    k_condense_rhs<<<vg, PB, 0, s>>>(D, c->vcode, p->fc, r, c->rowdiag, p->rv), ::mb::count_launch(c);
    k_bj_apply<<<nblk(D.N), 256, 0, s>>>(D, p->dinv, p->rv, nullptr, OMEGA_FINE, false, z), ::mb::count_launch(c);
    // t = S z_v  (S applied as the JVP of [z_v, -D_n^-1 J_nv z_v])
    auto apply_S = [&]() -> int {
        if (D.F) k_face_solve<<<fg, 256, 0, s>>>(D, c->pf_g, c->pf_e, p->fc, nullptr, c->rowdiag, z), ::mb::count_launch(c);
        return launch_jvp<float, double>(c, u32, gate, dt, z, p->t, s, 1);
    };
    int rc;
    for (int k = 1; k < NU_FINE; ++k) {
        if ((rc = apply_S())) return rc;
        k_bj_apply<<<nblk(D.N), 256, 0, s>>>(D, p->dinv, p->rv, p->t, OMEGA_FINE, true, z), ::mb::count_launch(c);
    }
    if ((rc = apply_S())) return rc;
    Level& L1 = p->lv[1];
    k_restrict_fine<<<nblk(L1.cells), 256, 0, s>>>(D, c->vcode, p->rv, p->t, L1), ::mb::count_launch(c);
    if (debug_level() >= 2)
        fprintf(stderr, "[mb-pc] |rv| %.3e |z0| %.3e |Sz0| %.3e |b1| %.3e\n", dbg_norm(c, p->rv, 2 * D.N),
                dbg_norm(c, z, 2 * D.N), dbg_norm(c, p->t, 2 * D.N),
                dbg_norm(c, reinterpret_cast<const double*>(L1.b), 4 * L1.cells));
    kcycle_l1(c);
    if (debug_level() >= 2)
        fprintf(stderr, "[mb-pc] |x1| %.3e\n", dbg_norm(c, reinterpret_cast<const double*>(L1.x), 4 * L1.cells));
    k_prolong_fine<<<vg, PB, 0, s>>>(D, c->vcode, L1, L1.x, z), ::mb::count_launch(c);
    // NU_FINE post-smoothing sweeps (they remove the jumps of the piecewise-constant prolongation)
    for (int k = 0; k < NU_FINE; ++k) {
        if ((rc = apply_S())) return rc;
        k_bj_apply<<<nblk(D.N), 256, 0, s>>>(D, p->dinv, p->rv, p->t, OMEGA_FINE, true, z), ::mb::count_launch(c);
    }
    // back-substitution of the plating rows
    if (D.F) k_face_solve<<<fg, 256, 0, s>>>(D, c->pf_g, c->pf_e, p->fc, r, c->rowdiag, z), ::mb::count_launch(c);
    prof_end(c, s, PROF_PRECOND, ev_pc);
    if (debug_level() >= 2) fprintf(stderr, "[mb-pc] |z| %.3e\n", dbg_norm(c, z, c->n));
    MB_CUDA_LAUNCH("precond_apply");
    return MB_OK;
}

}  // namespace mb

// ------------------------------------------------------------ test hooks
#include "../../include/mb_debug.h"

using namespace mb;

template <class A, class B>
__global__ void k_cvt(const A* __restrict__ a, B* __restrict__ b, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (B)a[i];
}

extern "C" {

int mb_debug_precond(mb_cell* c, const double* u, const uint8_t* gate, double dt, const double* r, double* z) {
    if (!c || !u || !r || !z || !(dt > 0)) { set_error("mb_debug_precond: invalid argument"); return MB_EINVAL; }
    int64_t n = c->n, F = c->D.F;
    cudaStream_t s = c->stream;
    double *du = nullptr, *r64 = nullptr, *z64 = nullptr;
    MB_CUDA(cudaMalloc(&du, 8 * n));
    MB_CUDA(cudaMalloc(&r64, 8 * n));
    MB_CUDA(cudaMalloc(&z64, 8 * n));
    MB_CUDA(cudaMemcpyAsync(du, u, 8 * n, cudaMemcpyHostToDevice, s));
    k_cvt<double, float><<<nblk(n), 256, 0, s>>>(du, c->u32, n), ::mb::count_launch(c);
    if (F) MB_CUDA(cudaMemcpyAsync(c->gate2, gate, F, cudaMemcpyHostToDevice, s));
    MB_CUDA(cudaMemcpyAsync(r64, r, 8 * n, cudaMemcpyHostToDevice, s));
    int rc = precond_setup(c, c->u32, c->gate2, dt);
    if (!rc) rc = precond_apply(c, c->u32, c->gate2, dt, r64, z64);
    if (!rc) {
        cudaMemcpyAsync(z, z64, 8 * n, cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) rc = cuda_fail(cudaGetLastError(), "debug_precond");
    }
    cudaStreamSynchronize(s);
    cudaFree(du); cudaFree(r64); cudaFree(z64);
    return rc;
}

int mb_debug_levels(mb_cell* c, int* nlev) {
    if (!c || !nlev) return MB_EINVAL;
    *nlev = c->pc->nlev;
    return MB_OK;
}

int mb_debug_level_dims(mb_cell* c, int level, int* nt, int* ny, int* nz) {
    if (!c || level < 1 || level > c->pc->nlev) { set_error("mb_debug_level_dims: bad level"); return MB_EINVAL; }
    const Level& L = c->pc->lv[level];
    *nt = L.nt; *ny = L.ny; *nz = L.nz;
    return MB_OK;
}

int mb_debug_level_op(mb_cell* c, int level, float* aself, float* off, uint8_t* mask) {
    if (!c || level < 1 || level > c->pc->nlev) { set_error("mb_debug_level_op: bad level"); return MB_EINVAL; }
    const Level& L = c->pc->lv[level];
    if (aself) MB_CUDA(cudaMemcpy(aself, L.aself, 4 * BLK * L.cells, cudaMemcpyDeviceToHost));
    if (off) MB_CUDA(cudaMemcpy(off, L.off, 4 * OFFW * L.cells, cudaMemcpyDeviceToHost));
    if (mask) MB_CUDA(cudaMemcpy(mask, L.mask, L.cells, cudaMemcpyDeviceToHost));
    return MB_OK;
}

int mb_debug_fine(mb_cell* c, float* dinv, float* fc, float* rowdiag) {
    if (!c) return MB_EINVAL;
    if (rowdiag) MB_CUDA(cudaMemcpy(rowdiag, c->rowdiag, 4 * c->n, cudaMemcpyDeviceToHost));
    if (dinv) MB_CUDA(cudaMemcpy(dinv, c->pc->dinv, 16 * c->D.N, cudaMemcpyDeviceToHost));
    if (fc && c->D.F) MB_CUDA(cudaMemcpy(fc, c->pc->fc, 4 * FCW * c->D.F, cudaMemcpyDeviceToHost));
    return MB_OK;
}

}  // extern "C"
