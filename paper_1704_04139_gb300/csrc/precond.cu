// precond.cu -- preconditioner of the scaled Newton system S_r^-1 J S_u.
//
// 1. Plating rows are condensed out exactly: each face row R_n(f) depends on
//    its own n_f and on the potentials/concentration of its two voxels only,
//    so with D_n = dR_n/dn the voxel system S = J_vv - J_vn D_n^-1 J_nv has
//    the sparsity of the face couplings.  The preconditioner solves
//    S z_v = r_v - J_vn D_n^-1 r_n approximately and back-substitutes
//    z_n = D_n^-1 (r_n - J_nv z_v).
// 2. Fine level: nu_fine (mg_smooth) damped 2x2 (c, phi) block-Jacobi sweeps of S before
//    and after the coarse correction.  S is assembled once per linear solve
//    as a seven-point stencil of 2x2 blocks in difference form (from the same
//    interface partials as the Krylov operator, with the plating rows
//    eliminated face by face), and each sweep is one streaming kernel:
//    product, residual and block update.  Several post-sweeps are needed:
//    with a current source the correction carries a large, weakly pinned
//    potential component, and the jumps its piecewise-constant prolongation
//    leaves at aggregate boundaries otherwise dominate the residual.
// 3. Coarse levels: aggregation of 2x2x2 blocks split by class
//    (0 electrolyte c, 1 electrolyte phi, 2 anode-side phi: G, CN,
//    3 cathode-side phi: K, CP, L); Galerkin operators with piecewise-constant
//    prolongation stored per coarse cell as the block row sums by class (ex)
//    and six 4x4 outgoing blocks (off), applied in difference form
//    A x = ex x_i + sum_d off_d (x_nb - x_i), so that the large intra-phase
//    conductances never meet the iterate's large near-null components.
//    Level 1 is solved by a K-cycle: FGMRES(KCYC) run entirely on the device,
//    preconditioned by a V-cycle (mg_coarse_pre / mg_coarse_post damped 4x4
//    block-Jacobi sweeps before / after each coarse correction); the coarsest level is solved with an
//    explicit FP64 inverse.
// Precision: all arithmetic of the application is FP32; iterates and
// corrections (z, coarse x, K-cycle directions) are float-float, residuals and
// Krylov bases FP32.  Coarse operators are assembled in FP32; with mg_bf16 the
// smoothing, residual and K-cycle products read a BF16 copy (each 4x4 block
// row packed as four BF16 in 8 bytes), which halves the dominant byte stream
// of the coarse levels.  The difference form keeps their null space exact
// under this rounding: constants per class are annihilated whatever the
// couplings' values.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <vector>

#include "mb_internal.h"
#include "mb_reduce.cuh"

namespace mb {

constexpr int NCLS = 4;
constexpr int BLK = NCLS * NCLS;          // 16 floats per 4x4 block
constexpr int OFFW = 6 * BLK;             // 96 floats of outgoing couplings per cell
constexpr float OMEGA_FINE = 0.8f;
constexpr float OMEGA_COARSE = 0.7f;
constexpr int KCYC_MAX = 16;              // longest level-1 K-cycle (FGMRES iterations)
constexpr int MAX_LEVELS = 16;
constexpr int COARSE_MAX = 256;           // dense coarsest system size bound (4 x cells)
constexpr int FCW = 8;                    // floats of condensation coefficients per face
constexpr int FSTK = 14;                  // row blocks of the assembled fine stencil per voxel
constexpr int SWT = 256;                  // cells per tile of the staged coarse sweep (= its threads)

// float-float 4-vector of one coarse cell
struct alignas(32) DF4 {
    float4 h, l;
};
__device__ inline float4 df4_val(const DF4& a) {
    return make_float4(a.h.x + a.l.x, a.h.y + a.l.y, a.h.z + a.l.z, a.h.w + a.l.w);
}
__device__ inline float4 df4_diff(const DF4& a, const DF4& b) {
    return make_float4(df_diff(make_float2(a.h.x, a.l.x), make_float2(b.h.x, b.l.x)),
                       df_diff(make_float2(a.h.y, a.l.y), make_float2(b.h.y, b.l.y)),
                       df_diff(make_float2(a.h.z, a.l.z), make_float2(b.h.z, b.l.z)),
                       df_diff(make_float2(a.h.w, a.l.w), make_float2(b.h.w, b.l.w)));
}
__device__ inline DF4 df4_pack(float2 x, float2 y, float2 z, float2 w) {
    DF4 r;
    r.h = make_float4(x.x, y.x, z.x, w.x);
    r.l = make_float4(x.y, y.y, z.y, w.y);
    return r;
}
__device__ inline DF4 df4_add(const DF4& a, const DF4& b) {
    return df4_pack(df_add(make_float2(a.h.x, a.l.x), make_float2(b.h.x, b.l.x)),
                    df_add(make_float2(a.h.y, a.l.y), make_float2(b.h.y, b.l.y)),
                    df_add(make_float2(a.h.z, a.l.z), make_float2(b.h.z, b.l.z)),
                    df_add(make_float2(a.h.w, a.l.w), make_float2(b.h.w, b.l.w)));
}
__device__ inline DF4 df4_add_f(const DF4& a, float4 b) {
    return df4_pack(df_add_f(make_float2(a.h.x, a.l.x), b.x), df_add_f(make_float2(a.h.y, a.l.y), b.y),
                    df_add_f(make_float2(a.h.z, a.l.z), b.z), df_add_f(make_float2(a.h.w, a.l.w), b.w));
}
__device__ inline DF4 df4_zero() {
    DF4 r;
    r.h = make_float4(0.f, 0.f, 0.f, 0.f);
    r.l = r.h;
    return r;
}

struct Level {
    int nt = 0, ny = 0, nz = 0;
    int64_t cells = 0;
    // operators, structure of arrays: entry e of cell i at [e * cells + i]
    float* off = nullptr;     // 6 x 16 x cells  outgoing couplings (direction d, block entry k*4+kk)
    float* ex = nullptr;      // 16 x cells  row sums by class (summed up the hierarchy)
    float* exd = nullptr;     // 16 x cells  self block of the difference form (absent classes fixed up)
    float* aself = nullptr;   // 16 x cells  self block ex - sum_d off_d (absent classes fixed up)
    float* sinv = nullptr;    // 16 x cells  inverse of the self block
    uint8_t* mask = nullptr;  // cells: classes present
    uint2* pk = nullptr;      // 32 x pst  BF16 copy: rows of off_0..off_5, exd, sinv (4 BF16 per row)
    int64_t pst = 0;          // row stride of pk: cells rounded up to a whole tile of the staged sweep
    DF4* x = nullptr;         // cells
    DF4* x2 = nullptr;        // cells
    float4* b = nullptr;      // cells
};

// One captured preconditioner application for a fixed (r, z) buffer pair.
struct PcGraph {
    const float* r = nullptr;
    float2* z = nullptr;
    int kcyc = 0;
    int nu = 0;
    int reorth = 0;
    int tail = 0;
    int pdl = 0;
    cudaGraphExec_t exec = nullptr;
    int64_t nodes = 0;                 // kernels per execution
    std::vector<ProfPair> ev;          // timing events recorded by the graph (prof graphs)
};

struct Precond {
    std::vector<PcGraph> graphs;
    int pending = -1;          // graph whose last execution still has to be harvested
    bool graphs_off = false;   // capture failed once: direct launches from then on
    float* dinv = nullptr;     // 4 per voxel: inverse of the condensed scaled (c, phi) block
    float* fc = nullptr;       // FCW per plating face: condensation coefficients (scaled)
    float* rv = nullptr;       // 2N: condensed right-hand side
    float* t = nullptr;        // 2N: S z
    void* fst = nullptr;       // FSTK x N: assembled fine stencil (float2, or two BF16 per word)
    float2* zs = nullptr;      // 2N: second fine iterate (sweeps alternate between it and z)
    int nlev = 0;              // coarse levels (index 1..nlev; lv[0] unused)
    Level lv[MAX_LEVELS + 1];
    int ncoarse = 0;
    double* cdense = nullptr;
    double* cinv = nullptr;
    int* cstat = nullptr;
    int kcyc = 0;              // level-1 K-cycle length
    bool b16 = false;          // applications read the BF16 operator copies
    int nsm = 0;               // SMs of the device (grid of the persistent staged sweep)
    int pf[3] = {0, 0, 0};     // L2 prefetch distance (blocks of one resident wave) of the BF16
                               // sweep, fused first sweeps and product
    int* err = nullptr;        // device flag: a bounded wait gave up (1 staged sweep, 2 its drain, 4 the tail)
    unsigned* tbar = nullptr;  // grid barrier of the persistent coarse tail
    int tail_l0 = 0;           // first level of the persistent tail (0: none)
    int tail_blocks = 0;       // its grid (blocks of TAIL_THREADS, all co-resident)
    int nu_fine = 0;           // fine-level block-Jacobi sweeps before and after the coarse correction
    // level-1 K-cycle workspace
    float* kV = nullptr;       // (KCYC_MAX+1) x m4  FP32 basis
    DF4* kZ = nullptr;         // KCYC_MAX x cells   preconditioned directions
    float* kw = nullptr;       // m4
    double* kH = nullptr;      // (KCYC_MAX+1) x KCYC_MAX + scalars
    double* kred = nullptr;    // RED_BLOCKS x 8 partials
};

// set when a staged sweep timed out and could not drain its bulk copies: the
// plain sweep is used from then on in this process
static std::atomic<bool> g_staged_broken{false};
// set when a persistent coarse tail timed out at a grid barrier, or a graph
// containing it could not be captured: per-level launches from then on
static std::atomic<bool> g_tail_broken{false};

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

// interface face (index into the stored partials) of voxel v in direction d
// towards w, -1 for the other face types; irank counts v's own interface faces
__device__ inline int64_t iface_of(int lv, int lw, uint32_t code, uint32_t cw_code, int d, int& irank) {
    if ((lv == PG || lv == PK || lv == PL) && lw == PE) return (int64_t)vc_fbase(code) + irank++;
    if (lv == PE && (lw == PG || lw == PK || lw == PL))
        return (int64_t)vc_fbase(cw_code) + __popc(vc_emask(cw_code) & ((1u << opp_dir(d)) - 1u));
    return -1;
}

// The set-up's scalars that depend on dt, rounded to FP32 once on the host
// (evaluated per thread they would be FP64 divisions, and GB300's FP64 rate
// is a small fraction of its FP32 rate)
struct SetupScal {
    float dtf, idt;      // dt, 1/dt
    float V_dt, dt_V;    // V/dt, dt/V
    double fc5;          // n_c dt / (V c_ref,E): dR_c(e)/dn in the Krylov units (one FP64 product per face)
    float src[6];        // V c_ref,l / dt (c-row scale per phase)
    float suc[6];        // c_ref,l (c-column scale per phase)
};

static SetupScal setup_scal(const DevParamsF& P, double dt) {
    // the values the kernels formerly evaluated per thread from the FP32
    // parameter copy, with the same roundings
    SetupScal S;
    S.dtf = float(dt);
    S.idt = float(1.0 / dt);
    S.V_dt = float(double(P.V) / dt);
    S.dt_V = float(dt / double(P.V));
    S.fc5 = double(P.nc) * dt / double(P.V * P.cref[PE]);
    for (int l = 0; l < 6; ++l) {
        S.src[l] = float(double(P.V * P.cref[l]) / dt);
        S.suc[l] = P.cref[l];
    }
    return S;
}

// ------------------------------------------------------------ fine level
__global__ void __launch_bounds__(256)
k_bj_setup(ParT<float> P, Dims D, const uint32_t* __restrict__ vc, const uint16_t* __restrict__ zperm,
           const float* __restrict__ u,
           const float* __restrict__ icoef, SetupScal S, float* __restrict__ dinv, float* __restrict__ fc,
           float* __restrict__ rowdiag, float* __restrict__ rowinv) {
    __shared__ float s_src[6], s_suc[6];
    {
        const int tid = threadIdx.y * blockDim.x + threadIdx.x;
        if (tid < 6) {
            s_src[tid] = S.src[tid];
            s_suc[tid] = S.suc[tid];
        }
        __syncthreads();
    }
    int z = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    int t = blockIdx.z;
    if (z >= D.nz || y >= D.ny) return;
    z = zperm[((int64_t)t * D.ny + y) * D.nz + z];   // phase-grouped thread order within the z-line
    const int64_t N = D.N;
    int64_t v = (int64_t)t * D.syz + (int64_t)y * D.nz + z;
    const float* cc = u;
    const float dtf = S.dtf, idt = S.idt;
    const float nc = P.nc;
    const float A = float(P.A), c0 = float(P.cref[PE]);
    uint32_t code = vc[v];
    int lv = vc_phase(code);
    float cv = cc[v];
    float d00 = 0.f, d01 = 0.f, d10 = 0.f, d11 = 0.f;
    float dgc = 0.f, dgp = 0.f;   // uncondensed diagonal entries
    const int64_t off[6] = {-D.syz, D.syz, -(int64_t)D.nz, (int64_t)D.nz, -1, 1};
    const bool inb[6] = {t > 0, t < D.nt - 1, y > 0, y < D.ny - 1, z > 0, z < D.nz - 1};
    int rank = 0, irank = 0;
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        if (!inb[d]) continue;
        int64_t w = v + off[d];
        uint32_t cw_code = vc[w];
        int lw = vc_phase(cw_code);
        int64_t f = face_of(lv, lw, code, cw_code, d, rank);
        FaceJac<float> J;
        face_jacobian_lin<float>(P, lv, lw, cv, cc[w], icoef, D.NI, iface_of(lv, lw, code, cw_code, d, irank), J);
        d00 += J.c[0]; d01 += J.c[1]; d10 += J.p[0]; d11 += J.p[1];
        dgc += J.c[0]; dgp += J.p[1];
        if (f >= 0) {
            float jnn = idt + J.n[4];                 // dR_n/dn (unscaled)
            if (lv == PG) {
                d11 -= J.p[4] * J.n[1] / jnn;         // Schur term on phi_g
                fc[FCW * f + 0] = dtf * jnn;          // scaled D_n
                rowdiag[2 * N + f] = fabsf(dtf * jnn);
                rowinv[2 * N + f] = 1.f / fabsf(dtf * jnn);
                fc[FCW * f + 1] = J.n[1] * dtf / nc;  // dR_n/dphi_g
                fc[FCW * f + 2] = J.n[2] * c0 * dtf / nc;   // dR_n/dc_e
                fc[FCW * f + 3] = J.n[3] * dtf / nc;  // dR_n/dphi_e
                fc[FCW * f + 4] = J.p[4] * nc / A;    // dR_phi(g)/dn
            } else {
                d00 -= J.c[4] * J.n[0] / jnn;
                d01 -= J.c[4] * J.n[1] / jnn;
                d10 -= J.p[4] * J.n[0] / jnn;
                d11 -= J.p[4] * J.n[1] / jnn;
                fc[FCW * f + 5] = float(double(J.c[4]) * S.fc5);   // dR_c(e)/dn
                fc[FCW * f + 6] = J.p[4] * nc / A;    // dR_phi(e)/dn
            }
        }
    }
    if (t == 0 && lv == PCN) { d11 += float(P.g_dir); dgp += float(P.g_dir); }
    float src, suc = s_suc[lv];
    if (has_c(lv)) {
        d00 += S.V_dt;
        dgc += S.V_dt;
        src = s_src[lv];
        rowdiag[v] = fmaxf(fabsf(dgc * S.dt_V), 1e-30f);
        rowinv[v] = 1.f / rowdiag[v];
    } else {
        d00 = 1.f; d01 = 0.f; src = 1.f;
        rowdiag[v] = 1.f;
        rowinv[v] = 1.f;
    }
    rowdiag[N + v] = fmaxf(fabsf(dgp / A), 1e-30f);
    rowinv[N + v] = 1.f / rowdiag[N + v];
    float a = d00 * suc / src, b = d01 / src, c = d10 * suc / A, e = d11 / A;
    float id = 1.f / (a * e - b * c);
    reinterpret_cast<float4*>(dinv)[v] = make_float4(e * id, -b * id, -c * id, a * id);
}

// condensed right-hand side r_v - J_vn D_n^-1 r_n (voxel rows of rv), FP32
__global__ void __launch_bounds__(256)
k_condense_rhs(Dims D, const uint32_t* __restrict__ vc, const float* __restrict__ fc, const float* __restrict__ r,
               const float* __restrict__ rowdiag, float* __restrict__ rv) {
    pdl_entry();
    int z = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    int t = blockIdx.z;
    if (z >= D.nz || y >= D.ny) return;
    const int64_t N = D.N;
    int64_t v = (int64_t)t * D.syz + (int64_t)y * D.nz + z;
    uint32_t code = vc[v];
    int lv = vc_phase(code);
    // the Krylov residual is row-equilibrated: undo it first
    float rc = r[v] * rowdiag[v], rp = r[N + v] * rowdiag[N + v];
    if (lv == PG || lv == PE) {
        const int64_t off[6] = {-D.syz, D.syz, -(int64_t)D.nz, (int64_t)D.nz, -1, 1};
        const bool inb[6] = {t > 0, t < D.nt - 1, y > 0, y < D.ny - 1, z > 0, z < D.nz - 1};
        int rank = 0;
        for (int d = 0; d < 6; ++d) {
            if (!inb[d]) continue;
            uint32_t cw_code = vc[v + off[d]];
            int64_t f = face_of(lv, vc_phase(cw_code), code, cw_code, d, rank);
            if (f < 0) continue;
            float q = r[2 * N + f] * rowdiag[2 * N + f] / fc[FCW * f + 0];
            if (lv == PG) {
                rp -= fc[FCW * f + 4] * q;
            } else {
                rc -= fc[FCW * f + 5] * q;
                rp -= fc[FCW * f + 6] * q;
            }
        }
    }
    rv[v] = rc;
    rv[N + v] = rp;
}

// z_n = (rn - J_nv z_v) / D_n  with rn = r_n (back-substitution) or 0
// (elimination).  dR_n/dphi_e = -dR_n/dphi_g exactly, so J_nv z_v is taken in
// difference form: fc1 (z_phi_g - z_phi_e) + fc2 z_c_e.
__global__ void k_face_solve(Dims D, const int32_t* __restrict__ pg, const int32_t* __restrict__ pe,
                             const float* __restrict__ fc, const float* __restrict__ r,
                             const float* __restrict__ rowdiag, float2* __restrict__ z) {
    pdl_entry();
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= D.F) return;
    const int64_t N = D.N;
    int64_t g = pg[f], e = pe[f];
    const float* cf = fc + FCW * f;
    float jz = cf[1] * df_diff(z[N + g], z[N + e]) + cf[2] * df_val(z[e]);
    float rn = r ? r[2 * N + f] * rowdiag[2 * N + f] : 0.f;
    z[2 * N + f] = make_float2((rn - jz) / cf[0], 0.f);
}

// z = omega D^-1 rv  (accumulate = false);  z += omega D^-1 (rv - t)  (accumulate = true); voxel rows
__global__ void k_bj_apply(Dims D, const float* __restrict__ dinv, const float* __restrict__ rv,
                           const float* __restrict__ t, float omega, bool accumulate, float2* __restrict__ z) {
    pdl_entry();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t N = D.N;
    if (i >= N) return;
    float rc = rv[i], rp = rv[N + i];
    if (accumulate) { rc -= t[i]; rp -= t[N + i]; }
    float4 m = reinterpret_cast<const float4*>(dinv)[i];
    float zc = omega * (m.x * rc + m.y * rp), zp = omega * (m.z * rc + m.w * rp);
    if (accumulate) {
        z[i] = df_add_f(z[i], zc);
        z[N + i] = df_add_f(z[N + i], zp);
    } else {
        z[i] = make_float2(zc, 0.f);
        z[N + i] = make_float2(zp, 0.f);
    }
}

// ------------------------------------------------------- level-1 assembly
__device__ inline void acc_blk(float* blk, int k, int kk, float v) { blk[k * NCLS + kk] += v; }

__global__ void __launch_bounds__(128)
k_assemble_l1(ParT<float> P, Dims D, const uint32_t* __restrict__ vc, const float* __restrict__ u,
              const float* __restrict__ icoef, double dt, Level L1) {
    int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= L1.cells) return;
    int cz = (int)(cell % L1.nz);
    int cy = (int)((cell / L1.nz) % L1.ny);
    int ct = (int)(cell / ((int64_t)L1.nz * L1.ny));
    const float* cc = u;
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
                float cv = cc[v];
                const int64_t offs[6] = {-D.syz, D.syz, -(int64_t)D.nz, (int64_t)D.nz, -1, 1};
                const bool inb[6] = {t > 0, t < D.nt - 1, y > 0, y < D.ny - 1, z > 0, z < D.nz - 1};
                const int loc[6] = {a, a, b, b, e, e};
                int rank = 0, irank = 0;
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
                    float cw = cc[w];
                    FaceJac<float> J;
                    face_jacobian_lin<float>(P, lv, lw, cv, cw, icoef, D.NI, iface_of(lv, lw, code, cw_code, d, irank),
                                             J);
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
    for (int i = 0; i < BLK; ++i) L1.ex[(int64_t)i * L1.cells + cell] = ex[i];
    for (int i = 0; i < OFFW; ++i) L1.off[(int64_t)i * L1.cells + cell] = off[i];
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
                for (int i = 0; i < BLK; ++i) ex[i] += F.ex[(int64_t)i * F.cells + ch];
                const int loc[6] = {a, a, b, b, e, e};
                for (int d = 0; d < 6; ++d) {
                    bool other = (d & 1) ? (loc[d] == 1) : (loc[d] == 0);
                    if (!other) continue;
                    for (int i = 0; i < BLK; ++i) off[d * BLK + i] += F.off[(int64_t)(d * BLK + i) * F.cells + ch];
                }
            }
    for (int i = 0; i < BLK; ++i) C.ex[(int64_t)i * C.cells + cell] = ex[i];
    for (int i = 0; i < OFFW; ++i) C.off[(int64_t)i * C.cells + cell] = off[i];
    C.mask[cell] = (uint8_t)mask;
}

// self block = row sums - outgoing couplings; absent classes get an identity
// row (and zero columns); the block inverse by Gauss-Jordan with partial
// pivoting (FP32: it only serves the smoother).  exd is the self block of the difference form:
// ex for present classes, the fixed-up self block plus the outgoing sums
// elsewhere, so that exd x_i + sum_d off_d (x_nb - x_i) = aself x_i + sum_d off_d x_nb.
__global__ void k_finalize(Level L) {
    int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= L.cells) return;
    float a[NCLS][2 * NCLS];
    uint32_t mask = L.mask[cell];
#pragma unroll
    for (int k = 0; k < NCLS; ++k)
#pragma unroll
        for (int kk = 0; kk < NCLS; ++kk) {
            float so = 0.f;
            for (int d = 0; d < 6; ++d) so += L.off[(int64_t)(d * BLK + k * NCLS + kk) * L.cells + cell];
            const float ex = L.ex[(int64_t)(k * NCLS + kk) * L.cells + cell];
            float s = ex - so;
            float sd = ex;
            if (!((mask >> k) & 1u) || !((mask >> kk) & 1u)) {
                s = (k == kk && !((mask >> k) & 1u)) ? 1.f : 0.f;
                sd = s + so;
            }
            a[k][kk] = s;
            a[k][NCLS + kk] = (k == kk) ? 1.f : 0.f;
            L.aself[(int64_t)(k * NCLS + kk) * L.cells + cell] = s;
            L.exd[(int64_t)(k * NCLS + kk) * L.cells + cell] = sd;
        }
#pragma unroll
    for (int col = 0; col < NCLS; ++col) {
        int piv = col;
        float pmax = fabsf(a[col][col]);
#pragma unroll
        for (int r = col + 1; r < NCLS; ++r) {
            const float ar = fabsf(a[r][col]);
            if (ar > pmax) { pmax = ar; piv = r; }
        }
        // row swap with compile-time row indices (a runtime index would put a[][] in local memory)
#pragma unroll
        for (int r = col + 1; r < NCLS; ++r)
            if (r == piv)
#pragma unroll
                for (int j = 0; j < 2 * NCLS; ++j) { float tmp = a[col][j]; a[col][j] = a[r][j]; a[r][j] = tmp; }
        const float p = a[col][col];
        const float ip = p != 0.f ? 1.f / p : 0.f;
#pragma unroll
        for (int j = 0; j < 2 * NCLS; ++j) a[col][j] *= ip;
#pragma unroll
        for (int r = 0; r < NCLS; ++r) {
            if (r == col) continue;
            const float fct = a[r][col];
#pragma unroll
            for (int j = 0; j < 2 * NCLS; ++j) a[r][j] -= fct * a[col][j];
        }
    }
#pragma unroll
    for (int k = 0; k < NCLS; ++k)
#pragma unroll
        for (int kk = 0; kk < NCLS; ++kk) L.sinv[(int64_t)(k * NCLS + kk) * L.cells + cell] = a[k][NCLS + kk];
    // BF16 copy, block q (0..5 off_d, 6 exd, 7 sinv), row k: pk[(4q + k) * cells + cell]
    for (int q = 0; q < 8; ++q) {
        const float* src = q < 6 ? L.off + (int64_t)q * BLK * L.cells : (q == 6 ? L.exd : L.sinv);
        for (int k = 0; k < NCLS; ++k) {
            uint32_t h[NCLS];
            for (int kk = 0; kk < NCLS; ++kk)
                h[kk] = __bfloat16_as_ushort(__float2bfloat16_rn(src[(int64_t)(k * NCLS + kk) * L.cells + cell]));
            L.pk[(int64_t)(4 * q + k) * L.pst + cell] = make_uint2(h[0] | (h[1] << 16), h[2] | (h[3] << 16));
        }
    }
}

// ----------------------------------------------------- coarsest dense solve
// dense FP64 matrix of the coarsest level; the self block is formed in FP64
// from the difference-form data (exd - sum_d off_d), as the level's own
// difference-form product does, so no FP32 rounding breaks its row sums
__global__ void k_coarse_dense(Level L, int n, double* __restrict__ Ad) {
    int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= n) return;
    int64_t cell = row / NCLS;
    int k = row % NCLS;
    for (int j = 0; j < n; ++j) Ad[(int64_t)row * n + j] = 0.0;
    int cz = (int)(cell % L.nz);
    int cy = (int)((cell / L.nz) % L.ny);
    int ct = (int)(cell / ((int64_t)L.nz * L.ny));
    const int dt_[6] = {-1, 1, 0, 0, 0, 0}, dy_[6] = {0, 0, -1, 1, 0, 0}, dz_[6] = {0, 0, 0, 0, -1, 1};
    for (int kk = 0; kk < NCLS; ++kk) {
        double sd = L.exd[(int64_t)(k * NCLS + kk) * L.cells + cell];
        for (int d = 0; d < 6; ++d) {
            int t = ct + dt_[d], y = cy + dy_[d], z = cz + dz_[d];
            if (t < 0 || t >= L.nt || y < 0 || y >= L.ny || z < 0 || z >= L.nz) continue;
            sd -= L.off[(int64_t)(d * BLK + k * NCLS + kk) * L.cells + cell];
        }
        Ad[(int64_t)row * n + cell * NCLS + kk] = sd;
    }
    for (int d = 0; d < 6; ++d) {
        int t = ct + dt_[d], y = cy + dy_[d], z = cz + dz_[d];
        if (t < 0 || t >= L.nt || y < 0 || y >= L.ny || z < 0 || z >= L.nz) continue;
        int64_t nb = ((int64_t)t * L.ny + y) * L.nz + z;
        for (int kk = 0; kk < NCLS; ++kk)
            Ad[(int64_t)row * n + nb * NCLS + kk] += L.off[(int64_t)(d * BLK + k * NCLS + kk) * L.cells + cell];
    }
}

// Gauss-Jordan inverse with partial pivoting (largest magnitude, lowest row
// on ties), one block; the pivot search is a block reduction.
__global__ void k_coarse_invert(int n, double* __restrict__ A, double* __restrict__ Ainv, int* __restrict__ stat) {
    __shared__ int piv;
    __shared__ double pval;
    __shared__ double wv[32];
    __shared__ int wi[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) Ainv[i] = (i / n == i % n) ? 1.0 : 0.0;
    __syncthreads();
    for (int col = 0; col < n; ++col) {
        double best = -1.0;
        int bi = n;
        for (int r = col + threadIdx.x; r < n; r += blockDim.x) {
            const double v = fabs(A[(int64_t)r * n + col]);
            if (v > best) { best = v; bi = r; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double v2 = __shfl_down_sync(0xffffffffu, best, o);
            const int i2 = __shfl_down_sync(0xffffffffu, bi, o);
            if (v2 > best || (v2 == best && i2 < bi)) { best = v2; bi = i2; }
        }
        if (lane == 0) { wv[wid] = best; wi[wid] = bi; }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < nw; ++w)
                if (wv[w] > best || (wv[w] == best && wi[w] < bi)) { best = wv[w]; bi = wi[w]; }
            piv = bi;
            pval = A[(int64_t)bi * n + col];
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

// The same inverse with the matrix held in shared memory and inverted in
// place (Gauss-Jordan with row interchanges; the interchanges are undone as
// column swaps at the end), one block of 1024 threads, n <= CINV_SMEM_MAX.
// Per pivot column: warp 0 finds the pivot (largest magnitude, lowest row on
// ties), the rows are swapped, column k is saved and the pivot row scaled,
// then every other row is eliminated.  FP64 throughout.
constexpr int CINV_SMEM_MAX = 160;       // 160^2 doubles = 200 KB of shared memory
constexpr int CINV_THREADS = 1024;
__global__ void __launch_bounds__(CINV_THREADS)
k_coarse_invert_smem(int n, const double* __restrict__ A, double* __restrict__ Ainv, int* __restrict__ stat) {
    extern __shared__ __align__(16) double sA[];   // n x n, then colk[n]
    __shared__ int perm[CINV_SMEM_MAX];
    __shared__ int piv;
    __shared__ double pval;
    double* colk = sA + n * n;
    const int tid = threadIdx.x;
    for (int i = tid; i < n * n; i += blockDim.x) sA[i] = A[i];
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (tid < 32) {
            double best = -1.0;
            int bi = n;
            for (int r = k + tid; r < n; r += 32) {
                const double v = fabs(sA[r * n + k]);
                if (v > best) { best = v; bi = r; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double v2 = __shfl_down_sync(0xffffffffu, best, o);
                const int i2 = __shfl_down_sync(0xffffffffu, bi, o);
                if (v2 > best || (v2 == best && i2 < bi)) { best = v2; bi = i2; }
            }
            if (tid == 0) {
                piv = bi;
                pval = sA[bi * n + k];
                perm[k] = bi;
                if (pval == 0.0) *stat = 1;
            }
        }
        __syncthreads();
        const int p = piv;
        if (p != k) {
            for (int j = tid; j < n; j += blockDim.x) {
                const double t = sA[k * n + j];
                sA[k * n + j] = sA[p * n + j];
                sA[p * n + j] = t;
            }
            __syncthreads();
        }
        const double inv = pval != 0.0 ? 1.0 / pval : 0.0;
        // column k of the other rows (read before the elimination overwrites it)
        // and the scaled pivot row (its diagonal becomes 1/pivot)
        for (int i = tid; i < n; i += blockDim.x)
            if (i != k) colk[i] = sA[i * n + k];
        for (int j = tid; j < n; j += blockDim.x) sA[k * n + j] = (j == k ? 1.0 : sA[k * n + j]) * inv;
        __syncthreads();
        for (int idx = tid; idx < n * n; idx += blockDim.x) {
            const int i = idx / n, j = idx - i * n;
            if (i == k) continue;
            sA[idx] = (j == k ? 0.0 : sA[idx]) - colk[i] * sA[k * n + j];
        }
        __syncthreads();
    }
    // undo the row interchanges as column swaps, last first
    for (int k = n - 1; k >= 0; --k) {
        const int p = perm[k];
        if (p != k) {
            for (int i = tid; i < n; i += blockDim.x) {
                const double t = sA[i * n + k];
                sA[i * n + k] = sA[i * n + p];
                sA[i * n + p] = t;
            }
            __syncthreads();
        }
    }
    for (int i = tid; i < n * n; i += blockDim.x) Ainv[i] = sA[i];
}

// x = Ainv b (FP64 accumulation), one block; x stored float-float.  One warp
// per row (coalesced loads of Ainv), lane partial sums combined by shuffles.
__device__ inline void coarse_solve_block(int n, const double* __restrict__ Ainv, const float4* b, DF4* x,
                                          double* sb, double* sx) {
    const float* bf = reinterpret_cast<const float*>(b);
    for (int i = threadIdx.x; i < n; i += blockDim.x) sb[i] = (double)bf[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int r = threadIdx.x >> 5; r < n; r += nw) {
        double acc = 0.0;
        for (int j = lane; j < n; j += 32) acc += Ainv[(int64_t)r * n + j] * sb[j];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) sx[r] = acc;
    }
    __syncthreads();
    for (int cell = threadIdx.x; cell < n / NCLS; cell += blockDim.x)
        x[cell] = df4_pack(df_from_double(sx[4 * cell]), df_from_double(sx[4 * cell + 1]),
                           df_from_double(sx[4 * cell + 2]), df_from_double(sx[4 * cell + 3]));
}
// The same product spread over blocks of CS_ROWS rows (whole cells): the FP64
// dot products are bound by the SM's FP64 pipe, so one block alone took
// ~17 us for n = 128; CS_ROWS = 16 spreads them over 8 SMs.
constexpr int CS_ROWS = 16;
__global__ void __launch_bounds__(256) k_coarse_solve(int n, const double* __restrict__ Ainv,
                                                      const float4* __restrict__ b, DF4* __restrict__ x) {
    pdl_entry();
    __shared__ double sb[COARSE_MAX];
    __shared__ double sx[CS_ROWS];
    const float* bf = reinterpret_cast<const float*>(b);
    for (int i = threadIdx.x; i < n; i += blockDim.x) sb[i] = (double)bf[i];
    __syncthreads();
    const int r0 = blockIdx.x * CS_ROWS;
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int q = threadIdx.x >> 5; q < CS_ROWS; q += nw) {
        const int r = r0 + q;
        double acc = 0.0;
        if (r < n)
            for (int j = lane; j < n; j += 32) acc += Ainv[(int64_t)r * n + j] * sb[j];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) sx[q] = acc;
    }
    __syncthreads();
    const int c0 = r0 / NCLS;
    for (int k = threadIdx.x; k < CS_ROWS / NCLS; k += blockDim.x) {
        const int cell = c0 + k;
        if (cell >= n / NCLS) break;
        x[cell] = df4_pack(df_from_double(sx[4 * k]), df_from_double(sx[4 * k + 1]), df_from_double(sx[4 * k + 2]),
                           df_from_double(sx[4 * k + 3]));
    }
}

// ------------------------------------------------ assembled fine smoother
// The condensed scaled operator S (the smoother's units: rows over the
// residual scale, unknowns in Krylov units) per voxel in difference form,
//   (S z)_v = Dv z_v + sum_d O_d (z_nb - z_v),
// 2x2 blocks with rows and columns (c, phi).  Row block k = 2q + r (q = 0
// self, 1 + d direction d; r = 0 c row, 1 phi row) holds the row's two
// column entries at [k * N + v]: a float2, or two BF16 in one word.
template <bool B16>
__device__ inline float2 fst_ld(const void* fst, int k, int64_t N, int64_t v) {
    if (B16) {
        const uint32_t w = static_cast<const uint32_t*>(fst)[k * N + v];
        return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
    }
    return static_cast<const float2*>(fst)[k * N + v];
}
template <bool B16>
__device__ inline void fst_st(void* fst, int k, int64_t N, int64_t v, float a, float b) {
    if (B16) {
        const uint32_t lo = __bfloat16_as_ushort(__float2bfloat16_rn(a));
        const uint32_t hi = __bfloat16_as_ushort(__float2bfloat16_rn(b));
        static_cast<uint32_t*>(fst)[k * N + v] = lo | (hi << 16);
    } else {
        static_cast<float2*>(fst)[k * N + v] = make_float2(a, b);
    }
}

// Assembly, one thread per voxel.  Per face the coefficients of the
// linearised fluxes on (dphi_w - dphi_v, dc_w - dc_v, dc_v, dc_w, dn_f) are
// those of the Krylov operator's stencil (same interface partials icoef, same
// FP32 concentrations); a plating face's dn_f is eliminated with its own row
// (F dn/dt + i_pl linearised = 0), and the absolute c_w terms are moved into
// difference form: p dc_w = p c_ref,w ((z_c,w - z_c,v) + z_c,v).
template <bool B16>
__global__ void __launch_bounds__(256)
k_assemble_fine(ParT<float> P, Dims D, const uint32_t* __restrict__ vc, const uint16_t* __restrict__ zperm,
                const float* __restrict__ c32,
                const float* __restrict__ icoef, const float* __restrict__ scal, void* __restrict__ fst) {
    int z = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int t = blockIdx.z;
    if (z >= D.nz || y >= D.ny) return;
    z = zperm[((int64_t)t * D.ny + y) * D.nz + z];   // phase-grouped thread order within the z-line
    const int64_t N = D.N, NI = D.NI;
    const int64_t v = (int64_t)t * D.syz + (int64_t)y * D.nz + z;
    const uint32_t code = vc[v];
    const int lv = vc_phase(code);
    const float crv = P.cref[lv], crE = P.cref[PE];
    const float A = P.A, AF = P.A * P.invF;
    const float dt_inv = scal[0];
    const float Fdt = dt_inv / P.invF;   // F / dt
    const bool vkin = lv == PG || lv == PK || lv == PL;
    const int64_t off[6] = {-D.syz, D.syz, -(int64_t)D.nz, (int64_t)D.nz, -1, 1};
    const bool inb[6] = {t > 0, t < D.nt - 1, y > 0, y < D.ny - 1, z > 0, z < D.nz - 1};
    float Dcc = 0.f, Dcp = 0.f, Dpc = 0.f, Dpp = 0.f;
    float Occ[6], Ocp[6], Opc[6], Opp[6];
    int64_t ibase = (int64_t)vc_fbase(code);
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        Occ[d] = Ocp[d] = Opc[d] = Opp[d] = 0.f;
        if (!inb[d]) continue;
        const int64_t w = v + off[d];
        const uint32_t cw_code = vc[w];
        const int lw = vc_phase(cw_code);
        float p1 = 0.f, p2 = 0.f, p3 = 0.f, p4 = 0.f;   // phi row on (ddp, ddc, dcv, dcw)
        float q1 = 0.f, q2 = 0.f, q3 = 0.f, q4 = 0.f;   // c row
        float crd = 0.f, crw = 0.f;                     // c_ref of the ddc and dcw terms
        if (lv == PE && lw == PE) {
            crd = crE;
            crw = crE;
            const float cv = c32[v], cw = c32[w], cmin = P.cmin[PE];
            const float iS = __frcp_rn(fmaxf(cv, cmin) + fmaxf(cw, cmin));
            const float gr = P.E_gm * (cw - cv) * iS * iS;
            p1 = -P.E_gk;
            p2 = -P.E_gm * iS;
            p3 = cv >= cmin ? gr : 0.f;
            p4 = cw >= cmin ? gr : 0.f;
            q1 = P.E_tF * p1;
            q2 = -P.E_gD + P.E_tF * p2;
            q3 = P.E_tF * p3;
            q4 = P.E_tF * p4;
        } else if (lv == lw && (lv == PG || lv == PK)) {
            crd = crv;
            q2 = -P.gD[lv];
            p1 = -P.gsig[lv][lw];
        } else if (lv != PE && lw != PE) {
            p1 = -P.gsig[lv][lw];
        } else if (vkin && lw == PE) {
            const int64_t i = ibase++;
            const float i_eta = icoef[i], ip_eta = icoef[NI + i], i_cs = icoef[2 * NI + i];
            const float i_ce = icoef[3 * NI + i], ip_ce = icoef[4 * NI + i], ip_n = icoef[5 * NI + i];
            crw = crE;
            p1 = -A * (i_eta + ip_eta);
            p3 = A * i_cs;
            p4 = A * (i_ce + ip_ce);
            if (lv != PL) {
                q1 = -AF * i_eta;
                q3 = AF * i_cs;
                q4 = AF * i_ce;
            }
            if (lv == PG) {   // dn_f = (ip_eta ddp - ip_ce dcw) / (ip_n + F/dt)
                const float p5 = A * ip_n, k = 1.f / (ip_n + Fdt);
                p1 += p5 * k * ip_eta;
                p4 -= p5 * k * ip_ce;
            }
        } else if (lv == PE && (lw == PG || lw == PK || lw == PL)) {
            const int64_t i = (int64_t)vc_fbase(cw_code) + __popc(vc_emask(cw_code) & ((1u << opp_dir(d)) - 1u));
            const float i_eta = icoef[i], ip_eta = icoef[NI + i], i_cs = icoef[2 * NI + i];
            const float i_ce = icoef[3 * NI + i], ip_ce = icoef[4 * NI + i], ip_n = icoef[5 * NI + i];
            crw = P.cref[lw];
            p1 = -A * (i_eta + ip_eta);
            p3 = -A * (i_ce + ip_ce);
            p4 = -A * i_cs;
            q1 = -AF * (i_eta + ip_eta);
            q3 = -AF * (i_ce + ip_ce);
            q4 = -AF * i_cs;
            if (lw == PG) {   // dn_f = (-ip_eta ddp - ip_ce dcv) / (ip_n + F/dt) from this side
                const float p5 = -A * ip_n, q5 = -AF * ip_n, k = 1.f / (ip_n + Fdt);
                p1 -= p5 * k * ip_eta;
                p3 -= p5 * k * ip_ce;
                q1 -= q5 * k * ip_eta;
                q3 -= q5 * k * ip_ce;
            }
        }
        Opp[d] = p1;
        Opc[d] = p2 * crd + p4 * crw;
        Dpc += p3 * crv + p4 * crw;
        Ocp[d] = q1;
        Occ[d] = q2 * crd + q4 * crw;
        Dcc += q3 * crv + q4 * crw;
    }
    if (t == 0 && lv == PCN) Dpp += P.g_dir;
    if (has_c(lv)) {
        const float sc = scal[1 + lv];
        Dcc = (Dcc + P.V * dt_inv * crv) * sc;
        Dcp *= sc;
#pragma unroll
        for (int d = 0; d < 6; ++d) { Occ[d] *= sc; Ocp[d] *= sc; }
    } else {   // identity row of a phase without concentration
        Dcc = crv;
        Dcp = 0.f;
#pragma unroll
        for (int d = 0; d < 6; ++d) { Occ[d] = 0.f; Ocp[d] = 0.f; }
    }
    const float sp = scal[7];
    fst_st<B16>(fst, 0, N, v, Dcc, Dcp);
    fst_st<B16>(fst, 1, N, v, Dpc * sp, Dpp * sp);
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        fst_st<B16>(fst, 2 + 2 * d, N, v, Occ[d], Ocp[d]);
        fst_st<B16>(fst, 3 + 2 * d, N, v, Opc[d] * sp, Opp[d] * sp);
    }
}

// S z at one voxel from the assembled stencil, differences from the
// float-float iterate; a neighbour outside the grid is replaced by the voxel
// itself (zero difference, zero coupling)
template <bool B16>
__device__ inline float2 fine_Sz(const Dims& D, const void* __restrict__ fst, const float2* __restrict__ zin, int t,
                                 int y, int z, int64_t v, float2 zc, float2 zp) {
    const int64_t N = D.N;
    const float2 s0 = fst_ld<B16>(fst, 0, N, v), s1 = fst_ld<B16>(fst, 1, N, v);
    const float vc = df_val(zc), vp = df_val(zp);
    float yc = s0.x * vc + s0.y * vp, yp = s1.x * vc + s1.y * vp;
    const int64_t off[6] = {-D.syz, D.syz, -(int64_t)D.nz, (int64_t)D.nz, -1, 1};
    const bool inb[6] = {t > 0, t < D.nt - 1, y > 0, y < D.ny - 1, z > 0, z < D.nz - 1};
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        const int64_t nb = inb[d] ? v + off[d] : v;
        const float dc = df_diff(zin[nb], zc), dp = df_diff(zin[N + nb], zp);
        const float2 o0 = fst_ld<B16>(fst, 2 + 2 * d, N, v), o1 = fst_ld<B16>(fst, 3 + 2 * d, N, v);
        yc += o0.x * dc + o0.y * dp;
        yp += o1.x * dc + o1.y * dp;
    }
    return make_float2(yc, yp);
}

// one damped block-Jacobi sweep, zout = zin + omega Dinv (rv - S zin) (SWEEP),
// or the product tout = S zin; voxel rows only
template <bool B16, bool SWEEP>
__global__ void __launch_bounds__(256)
k_fine_stencil(Dims D, const void* __restrict__ fst, const float* __restrict__ dinv, const float* __restrict__ rv,
               const float2* __restrict__ zin, float omega, float2* __restrict__ zout, float* __restrict__ tout) {
    pdl_entry();
    const int z = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int t = blockIdx.z;
    if (z >= D.nz || y >= D.ny) return;
    const int64_t N = D.N;
    const int64_t v = (int64_t)t * D.syz + (int64_t)y * D.nz + z;
    const float2 zc = zin[v], zp = zin[N + v];
    const float2 sz = fine_Sz<B16>(D, fst, zin, t, y, z, v, zc, zp);
    if (!SWEEP) {
        tout[v] = sz.x;
        tout[N + v] = sz.y;
        return;
    }
    const float rc = rv[v] - sz.x, rp = rv[N + v] - sz.y;
    const float4 m = reinterpret_cast<const float4*>(dinv)[v];
    zout[v] = df_add_f(zc, omega * (m.x * rc + m.y * rp));
    zout[N + v] = df_add_f(zp, omega * (m.z * rc + m.w * rp));
}

// --------------------------------------------------------- coarse smoothing
// 4x4 block (row-major entries k*4+kk stored st apart: structure-of-arrays
// over the cells, so that a warp's loads of one entry are contiguous) times x
__device__ inline float4 mv4(const float* __restrict__ m, int64_t st, float4 x) {
    return make_float4(m[0] * x.x + m[st] * x.y + m[2 * st] * x.z + m[3 * st] * x.w,
                       m[4 * st] * x.x + m[5 * st] * x.y + m[6 * st] * x.z + m[7 * st] * x.w,
                       m[8 * st] * x.x + m[9 * st] * x.y + m[10 * st] * x.z + m[11 * st] * x.w,
                       m[12 * st] * x.x + m[13 * st] * x.y + m[14 * st] * x.z + m[15 * st] * x.w);
}
// the same product from the BF16 copy: row k of block q is one 8-byte word
__device__ inline float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ inline float bf_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }
__device__ inline float bf_row(uint2 w, float4 x) {
    return bf_lo(w.x) * x.x + bf_hi(w.x) * x.y + bf_lo(w.y) * x.z + bf_hi(w.y) * x.w;
}
__device__ inline float4 mv4b(const uint2* __restrict__ m, int64_t st, float4 x) {
    return make_float4(bf_row(m[0], x), bf_row(m[st], x), bf_row(m[2 * st], x), bf_row(m[3 * st], x));
}
// block q of the level operator (0..5 off_d, 6 exd, 7 sinv) times x
template <bool B16>
__device__ inline float4 lvl_mv(const Level& L, int q, int64_t cell, float4 x) {
    if (B16) return mv4b(L.pk + (int64_t)4 * q * L.pst + cell, L.pst, x);
    const float* m = q < 6 ? L.off + (int64_t)q * BLK * L.cells : (q == 6 ? L.exd : L.sinv);
    return mv4(m + cell, L.cells, x);
}
__device__ inline float4 f4add(float4 a, float4 b) { return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }
__device__ inline float4 f4sub(float4 a, float4 b) { return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w); }
__device__ inline float4 f4scale(float s, float4 a) { return make_float4(s * a.x, s * a.y, s * a.z, s * a.w); }

// effective iterate of a cell: x (if given) plus the prolonged coarse correction (if given)
__device__ inline DF4 xeff(const DF4* x, const DF4* ec, int ccny, int ccnz, int t, int y, int z, int64_t cell) {
    DF4 r = x ? x[cell] : df4_zero();
    if (ec) r = df4_add(r, ec[((int64_t)(t >> 1) * ccny + (y >> 1)) * ccnz + (z >> 1)]);
    return r;
}

// A xe at one cell of level L in difference form (xe_i given; xf(t, y, z, cell)
// gives the neighbours' iterates).  Branch-free: a neighbour outside the
// level is replaced by the cell itself, whose difference is exactly zero
// (and whose coupling is zero: no face leaves the domain), so that all loads
// of the cell can be in flight together.
template <bool B16, class XF>
__device__ inline float4 cell_apply_g(const Level& L, int t, int y, int z, int64_t cell, const DF4& xi, XF xf) {
    float4 acc = lvl_mv<B16>(L, 6, cell, df4_val(xi));
    const int64_t syz = (int64_t)L.ny * L.nz;
    const bool inb[6] = {t > 0, t < L.nt - 1, y > 0, y < L.ny - 1, z > 0, z < L.nz - 1};
    const int64_t st[6] = {-syz, syz, -(int64_t)L.nz, (int64_t)L.nz, -1, 1};
    const int dt_[6] = {-1, 1, 0, 0, 0, 0}, dy_[6] = {0, 0, -1, 1, 0, 0}, dz_[6] = {0, 0, 0, 0, -1, 1};
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        const int tt = inb[d] ? t + dt_[d] : t, yy = inb[d] ? y + dy_[d] : y, zz = inb[d] ? z + dz_[d] : z;
        const int64_t nb = inb[d] ? cell + st[d] : cell;
        acc = f4add(acc, lvl_mv<B16>(L, d, cell, df4_diff(xf(tt, yy, zz, nb), xi)));
    }
    return acc;
}
template <bool B16>
__device__ inline float4 cell_apply(const Level& L, const DF4* x, const DF4* ec, int ccny, int ccnz, int t, int y,
                                    int z, int64_t cell, const DF4& xi) {
    return cell_apply_g<B16>(L, t, y, z, cell, xi, [&](int tt, int yy, int zz, int64_t nb) {
        return xeff(x, ec, ccny, ccnz, tt, yy, zz, nb);
    });
}
// the first sweep from zero, x1 = omega Sinv b, at one cell (float-float with a zero tail)
template <bool B16>
__device__ inline DF4 first_sweep(const Level& L, int64_t cell, float omega) {
    DF4 o;
    o.h = f4scale(omega, lvl_mv<B16>(L, 7, cell, L.b[cell]));
    o.l = make_float4(0.f, 0.f, 0.f, 0.f);
    return o;
}

__device__ inline void cell_coords(const Level& L, int64_t cell, int& t, int& y, int& z) {
    z = (int)(cell % L.nz);
    y = (int)((cell / L.nz) % L.ny);
    t = (int)(cell / ((int64_t)L.nz * L.ny));
}

// --------------------------------------- bulk asynchronous copies (PTX)
constexpr int SW_OP = 32 * SWT * 8;                    // operator rows of a tile
constexpr int SW_STAGE = SW_OP + SWT * 16 + SWT * 32;   // + rhs + iterate
constexpr int SW_SMEM = 2 * SW_STAGE;
constexpr int SW_SPIN = 1 << 22;

__device__ inline uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ inline void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ inline void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    uint64_t state;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;"
                 : "=l"(state)
                 : "r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
    (void)state;
}
__device__ inline bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ inline bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    for (int i = 0; i < SW_SPIN; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16)
__device__ inline void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// L2 prefetch of a global range (16-byte aligned, size a multiple of 16)
__device__ inline void bulk_prefetch_l2(const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
// one thread: L2 prefetch of the operator rows [r0, r1) of the block of SWT
// cells `blk` (and its right-hand side and iterate when given)
__device__ inline void lvl_prefetch(const Level& L, int64_t blk, int r0, int r1, const void* x) {
    const int64_t c0 = blk * SWT;
    if (c0 >= L.cells) return;
    const int nv = (int)(L.cells - c0 < SWT ? L.cells - c0 : SWT);
    for (int r = r0; r < r1; ++r) bulk_prefetch_l2(L.pk + (int64_t)r * L.pst + c0, SWT * 8);
    if (L.b) bulk_prefetch_l2(L.b + c0, (uint32_t)nv * 16);
    if (x) bulk_prefetch_l2(static_cast<const DF4*>(x) + c0, (uint32_t)nv * 32);
}

// x_out = xe + omega Sinv (b - A xe), xe = x_in (+ prolonged ec); both absent: x_out = omega Sinv b
// pf > 0 (BF16 operators, blocks of SWT threads): the block's thread 0 first
// prefetches into L2 the operator rows, right-hand side and iterate of block
// blockIdx.x + pf, about one resident wave ahead
// one cell of a damped block-Jacobi sweep (the body of k_lvl_smooth)
template <bool B16>
// (no __restrict__ on the iterates: the persistent tail reads in one phase what
// another block wrote in an earlier phase of the same launch, so these loads
// must not take the read-only non-coherent path)
__device__ inline void smooth_cell(const Level& L, const DF4* x_in, const DF4* ec, int ccny, int ccnz, float omega,
                                   DF4* x_out, int64_t cell) {
    int t, y, z;
    cell_coords(L, cell, t, y, z);
    if (!x_in && !ec) {
        float4 c = f4scale(omega, lvl_mv<B16>(L, 7, cell, L.b[cell]));
        DF4 o;
        o.h = c;
        o.l = make_float4(0.f, 0.f, 0.f, 0.f);
        x_out[cell] = o;
        return;
    }
    DF4 xe = xeff(x_in, ec, ccny, ccnz, t, y, z, cell);
    float4 r = f4sub(L.b[cell], cell_apply<B16>(L, x_in, ec, ccny, ccnz, t, y, z, cell, xe));
    x_out[cell] = df4_add_f(xe, f4scale(omega, lvl_mv<B16>(L, 7, cell, r)));
}

template <bool B16>
__global__ void k_lvl_smooth(Level L, const DF4* __restrict__ x_in, const DF4* __restrict__ ec, int ccny,
                             int ccnz, float omega, DF4* __restrict__ x_out, int pf) {
    pdl_entry();
    if (B16 && pf > 0 && threadIdx.x == 0) lvl_prefetch(L, (int64_t)blockIdx.x + pf, 0, 32, x_in);
    int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= L.cells) return;
    smooth_cell<B16>(L, x_in, ec, ccny, ccnz, omega, x_out, cell);
}

// ---------------------------------------- staged sweep (bulk async copies)
// The same sweep as k_lvl_smooth<true> from an iterate, with the tile's
// operator rows, right-hand side and iterate moved into shared memory by
// cp.async.bulk (completion counted on an mbarrier) while the previous tile
// is computed: a persistent grid, one CTA of SWT threads per SM, two stages.
// The neighbours' iterates (and the prolonged correction) are read from
// global memory (L1/L2).  Every wait is bounded; on a timeout the CTA sets
// *err, waits (bounded) for its copies in flight and returns.
// one thread: copies of tile `tile` into stage buffer sb
__device__ inline void sw_issue(const Level& L, const DF4* x_in, int64_t tile, uint8_t* sb, uint64_t* bar) {
    const int64_t c0 = tile * SWT;
    const int nv = (int)(L.cells - c0 < SWT ? L.cells - c0 : SWT);
    mbar_expect_tx(bar, (uint32_t)(SW_OP + nv * 16 + nv * 32));
    for (int r = 0; r < 32; ++r)
        bulk_g2s(sb + (size_t)r * SWT * 8, L.pk + (int64_t)r * L.pst + c0, SWT * 8, bar);
    bulk_g2s(sb + SW_OP, L.b + c0, (uint32_t)nv * 16, bar);
    bulk_g2s(sb + SW_OP + SWT * 16, x_in + c0, (uint32_t)nv * 32, bar);
}

__global__ void __launch_bounds__(SWT, 1)
k_lvl_smooth_staged(Level L, const DF4* __restrict__ x_in, const DF4* __restrict__ ec, int ccny, int ccnz,
                    float omega, DF4* __restrict__ x_out, int* __restrict__ err) {
    extern __shared__ __align__(128) uint8_t sw_smem[];
    __shared__ __align__(8) uint64_t bar[2];
    const int tid = threadIdx.x;
    const int64_t ntiles = (L.cells + SWT - 1) / SWT;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    int64_t tile = blockIdx.x;
    if (tid == 0 && tile < ntiles) sw_issue(L, x_in, tile, sw_smem, &bar[0]);
    uint32_t parity[2] = {0u, 0u};
    bool pending[2] = {tile < ntiles, false};
    int st = 0;
    for (; tile < ntiles; tile += gridDim.x) {
        const int64_t next = tile + gridDim.x;
        if (next < ntiles) {
            // the other stage was released by the barrier at the end of the previous tile
            if (tid == 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                sw_issue(L, x_in, next, sw_smem + (st ^ 1) * SW_STAGE, &bar[st ^ 1]);
            }
            pending[st ^ 1] = true;
        }
        const bool ok = __syncthreads_and(mbar_wait_bounded(&bar[st], parity[st]));
        if (!ok) {
            if (tid == 0) {
                atomicOr(err, 1);
                // drain the copies in flight; if that wait gives up too, copies
                // may still land in this CTA's shared memory after it exits
                for (int k = 0; k < 2; ++k)
                    if (pending[k] && !mbar_wait_bounded(&bar[k], parity[k])) atomicOr(err, 2);
            }
            return;
        }
        pending[st] = false;
        parity[st] ^= 1u;
        const int64_t cell = tile * SWT + tid;
        if (cell < L.cells) {
            const uint8_t* sb = sw_smem + st * SW_STAGE;
            const uint2* op = reinterpret_cast<const uint2*>(sb);
            int t, y, z;
            cell_coords(L, cell, t, y, z);
            DF4 xe = reinterpret_cast<const DF4*>(sb + SW_OP + SWT * 16)[tid];
            if (ec) xe = df4_add(xe, ec[((int64_t)(t >> 1) * ccny + (y >> 1)) * ccnz + (z >> 1)]);
            float4 acc = mv4b(op + 24 * SWT + tid, SWT, df4_val(xe));
            const int64_t syz = (int64_t)L.ny * L.nz;
            const bool inb[6] = {t > 0, t < L.nt - 1, y > 0, y < L.ny - 1, z > 0, z < L.nz - 1};
            const int64_t stp[6] = {-syz, syz, -(int64_t)L.nz, (int64_t)L.nz, -1, 1};
            const int dt_[6] = {-1, 1, 0, 0, 0, 0}, dy_[6] = {0, 0, -1, 1, 0, 0}, dz_[6] = {0, 0, 0, 0, -1, 1};
#pragma unroll
            for (int d = 0; d < 6; ++d) {
                const int tt = inb[d] ? t + dt_[d] : t, yy = inb[d] ? y + dy_[d] : y, zz = inb[d] ? z + dz_[d] : z;
                const int64_t nb = inb[d] ? cell + stp[d] : cell;
                acc = f4add(acc, mv4b(op + 4 * d * SWT + tid, SWT,
                                      df4_diff(xeff(x_in, ec, ccny, ccnz, tt, yy, zz, nb), xe)));
            }
            const float4 b = reinterpret_cast<const float4*>(sb + SW_OP)[tid];
            const float4 r = f4sub(b, acc);
            x_out[cell] = df4_add_f(xe, f4scale(omega, mv4b(op + 28 * SWT + tid, SWT, r)));
        }
        __syncthreads();
        st ^= 1;
    }
}

// the first two sweeps from zero in one pass: x2 = x1 + omega Sinv (b - A x1)
// with x1 = omega Sinv b evaluated where it is needed (the cell and its
// neighbours), bit-identical to two k_lvl_smooth launches
template <bool B16>
__device__ inline void smooth2_cell(const Level& L, float omega, DF4* x_out, int64_t cell) {
    int t, y, z;
    cell_coords(L, cell, t, y, z);
    const DF4 x1 = first_sweep<B16>(L, cell, omega);
    float4 r = f4sub(L.b[cell], cell_apply_g<B16>(L, t, y, z, cell, x1, [&](int, int, int, int64_t nb) {
                         return first_sweep<B16>(L, nb, omega);
                     }));
    x_out[cell] = df4_add_f(x1, f4scale(omega, lvl_mv<B16>(L, 7, cell, r)));
}

template <bool B16>
__global__ void k_lvl_smooth2(Level L, float omega, DF4* __restrict__ x_out, int pf) {
    pdl_entry();
    if (B16 && pf > 0 && threadIdx.x == 0) lvl_prefetch(L, (int64_t)blockIdx.x + pf, 0, 32, nullptr);
    int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= L.cells) return;
    smooth2_cell<B16>(L, omega, x_out, cell);
}

// The level-1 BF16 sweep with at most 48 registers per thread (5 blocks of 256
// per SM instead of 4): more cells' loads in flight for a sweep bound by memory
// latency at the cost of a few spilled registers (mg_stream = 3; measured 37.7
// against 41.5 us per level-1 sweep on a 4.2M-voxel cell, but the same bounds
// on the fused first sweeps and the coarse levels made the step slower).
__global__ void __launch_bounds__(256, 5) k_lvl_smooth_o5(Level L, const DF4* __restrict__ x_in,
                                                           const DF4* __restrict__ ec, int ccny, int ccnz,
                                                           float omega, DF4* __restrict__ x_out) {
    int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= L.cells) return;
    smooth_cell<true>(L, x_in, ec, ccny, ccnz, omega, x_out, cell);
}

template <bool B16>
__global__ void k_lvl_matvec(Level L, const DF4* __restrict__ x, float4* __restrict__ y_out, int pf) {
    pdl_entry();
    if (B16 && pf > 0 && threadIdx.x == 0) lvl_prefetch(L, (int64_t)blockIdx.x + pf, 0, 28, x);
    int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= L.cells) return;
    int t, y, z;
    cell_coords(L, cell, t, y, z);
    y_out[cell] = cell_apply<B16>(L, x, nullptr, 0, 0, t, y, z, cell, x[cell]);
}

// bc(parent) = sum over children of (b - A x): one thread per child (eight
// consecutive threads per parent), summed by shuffles within the octet
// thread tid of the restriction (eight consecutive threads per parent; whole
// warps must call it together)
template <bool B16>
__device__ inline void restrict_thread(const Level& L, const DF4* x, const Level& C, int64_t tid) {
    const int64_t cell = tid >> 3;
    const int k = (int)(tid & 7);
    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
    if (cell < C.cells) {
        int ct, cy, cz;
        cell_coords(C, cell, ct, cy, cz);
        int t = 2 * ct + (k >> 2), y = 2 * cy + ((k >> 1) & 1), z = 2 * cz + (k & 1);
        if (t < L.nt && y < L.ny && z < L.nz) {
            int64_t ch = ((int64_t)t * L.ny + y) * L.nz + z;
            r = f4sub(L.b[ch], cell_apply<B16>(L, x, nullptr, 0, 0, t, y, z, ch, x[ch]));
        }
    }
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
        r.x += __shfl_xor_sync(0xffffffffu, r.x, o);
        r.y += __shfl_xor_sync(0xffffffffu, r.y, o);
        r.z += __shfl_xor_sync(0xffffffffu, r.z, o);
        r.w += __shfl_xor_sync(0xffffffffu, r.w, o);
    }
    if (k == 0 && cell < C.cells) C.b[cell] = r;
}

template <bool B16>
__global__ void k_lvl_restrict(Level L, const DF4* __restrict__ x, Level C) {
    pdl_entry();
    restrict_thread<B16>(L, x, C, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

// ------------------------------------- coarse tail in one persistent launch
// The V-cycle on levels l0..nlev (BF16 operators) as one cooperative launch:
// the phases of the per-level kernels (fused first sweeps, further
// pre-sweeps, restriction, the coarsest dense solve by block 0, post-sweeps
// with the prolonged correction) run the same per-cell code in grid-stride
// loops, separated by a grid barrier instead of kernel boundaries, so the
// results are bit-identical to the per-level launches.  Every barrier wait is
// bounded: on a timeout a block sets bit 4 of *err and returns (the kernel
// holds no asynchronous copies).  Iterates alternate between x and x2 of each
// level exactly as the host-side sequence does.
constexpr int TAIL_THREADS = 512;
constexpr int TAIL_SPIN = 1 << 20;        // polls (64 ns apart) per barrier before giving up

struct TailLv {
    int nt, ny, nz;
    int64_t cells, pst;
    const uint2* pk;
    float4* b;
    DF4* x;
    DF4* x2;
};
struct TailArgs {
    int l0, nlev, nu_pre, nu_post, ncoarse;
    const double* cinv;
    unsigned* bar;       // [0] arrivals, [1] generation: zeroed before each launch
    int* err;
    TailLv lv[MAX_LEVELS + 1];
};

__device__ inline Level tail_level(const TailLv& t) {
    Level L;
    L.nt = t.nt; L.ny = t.ny; L.nz = t.nz;
    L.cells = t.cells;
    L.pst = t.pst;
    L.pk = const_cast<uint2*>(t.pk);
    L.b = t.b;
    return L;
}

// grid barrier; false if the wait gave up
__device__ inline bool tail_barrier(unsigned* bar, unsigned& gen) {
    __syncthreads();
    int ok = 1;
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned arrived = atomicAdd(&bar[0], 1u) + 1u;
        if (arrived == gridDim.x) {
            atomicExch(&bar[0], 0u);
            __threadfence();
            atomicExch(&bar[1], gen + 1u);
        } else {
            const volatile unsigned* g = bar + 1;
            int i = 0;
            while (*g == gen) {
                if (++i > TAIL_SPIN) { ok = 0; break; }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    ++gen;
    return __syncthreads_and(ok) != 0;
}

__global__ void __launch_bounds__(TAIL_THREADS, 1) k_vtail(TailArgs a) {
    __shared__ double sb[COARSE_MAX];
    __shared__ double sx[COARSE_MAX];
    unsigned gen = 0;
    unsigned par = 0;    // bit l: level l's current iterate is x2
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gs = (int64_t)gridDim.x * blockDim.x;
    auto X = [&](int l) { return ((par >> l) & 1u) ? a.lv[l].x2 : a.lv[l].x; };
    auto Y = [&](int l) { return ((par >> l) & 1u) ? a.lv[l].x : a.lv[l].x2; };
#define TAIL_SYNC()                                        \
    do {                                                   \
        if (!tail_barrier(a.bar, gen)) {                   \
            if (threadIdx.x == 0) atomicOr(a.err, 4);      \
            return;                                        \
        }                                                  \
    } while (0)
    for (int l = a.l0; l < a.nlev; ++l) {
        const Level L = tail_level(a.lv[l]);
        DF4* x = X(l);
        for (int64_t cell = gtid; cell < L.cells; cell += gs) {
            if (a.nu_pre >= 2) smooth2_cell<true>(L, OMEGA_COARSE, x, cell);
            else smooth_cell<true>(L, nullptr, nullptr, 0, 0, OMEGA_COARSE, x, cell);
        }
        TAIL_SYNC();
        for (int k = 2; k < a.nu_pre; ++k) {
            const DF4* xi = X(l);
            DF4* xo = Y(l);
            for (int64_t cell = gtid; cell < L.cells; cell += gs)
                smooth_cell<true>(L, xi, nullptr, 0, 0, OMEGA_COARSE, xo, cell);
            par ^= 1u << l;
            TAIL_SYNC();
        }
        const Level C = tail_level(a.lv[l + 1]);
        const int64_t nthr = (8 * C.cells + 31) / 32 * 32;     // whole warps (the octet shuffles)
        for (int64_t t = gtid; t < nthr; t += gs) restrict_thread<true>(L, X(l), C, t);
        TAIL_SYNC();
    }
    if (blockIdx.x == 0) coarse_solve_block(a.ncoarse, a.cinv, a.lv[a.nlev].b, X(a.nlev), sb, sx);
    for (int l = a.nlev - 1; l >= a.l0; --l) {
        TAIL_SYNC();
        const Level L = tail_level(a.lv[l]);
        const TailLv& C = a.lv[l + 1];
        {
            const DF4* xi = X(l);
            const DF4* ec = X(l + 1);
            DF4* xo = Y(l);
            for (int64_t cell = gtid; cell < L.cells; cell += gs)
                smooth_cell<true>(L, xi, ec, C.ny, C.nz, OMEGA_COARSE, xo, cell);
            par ^= 1u << l;
        }
        for (int k = 1; k < a.nu_post; ++k) {
            TAIL_SYNC();
            const DF4* xi = X(l);
            DF4* xo = Y(l);
            for (int64_t cell = gtid; cell < L.cells; cell += gs)
                smooth_cell<true>(L, xi, nullptr, 0, 0, OMEGA_COARSE, xo, cell);
            par ^= 1u << l;
        }
    }
#undef TAIL_SYNC
}

// ----------------------------------------------------- fine <-> level 1
__global__ void k_restrict_fine(Dims D, const uint32_t* __restrict__ vc, const float* __restrict__ r,
                                const float* __restrict__ t, Level C) {
    pdl_entry();
    int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= C.cells) return;
    int ct, cy, cz;
    cell_coords(C, cell, ct, cy, cz);
    float acc[NCLS] = {0.f, 0.f, 0.f, 0.f};
    const int64_t N = D.N;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int e = 0; e < 2; ++e) {
                int tt = 2 * ct + a, y = 2 * cy + b, z = 2 * cz + e;
                if (tt >= D.nt || y >= D.ny || z >= D.nz) continue;
                int64_t v = (int64_t)tt * D.syz + (int64_t)y * D.nz + z;
                int lv = vc_phase(vc[v]);
                const int k = phi_class(lv);
                const float rp = r[N + v] - t[N + v];
#pragma unroll
                for (int q = 0; q < NCLS; ++q)   // compile-time index: acc stays in registers
                    if (q == k) acc[q] += rp;
                if (lv == PE) acc[0] += r[v] - t[v];
            }
    C.b[cell] = make_float4(acc[0], acc[1], acc[2], acc[3]);
}

__global__ void k_prolong_fine(Dims D, const uint32_t* __restrict__ vc, Level C, const DF4* __restrict__ e1,
                               float2* __restrict__ z) {
    pdl_entry();
    int zz = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    int t = blockIdx.z;
    if (zz >= D.nz || y >= D.ny) return;
    int64_t v = (int64_t)t * D.syz + (int64_t)y * D.nz + zz;
    int lv = vc_phase(vc[v]);
    const DF4 e = e1[((int64_t)(t >> 1) * C.ny + (y >> 1)) * C.nz + (zz >> 1)];
    const int k = phi_class(lv);
    const float2 ek = k == 1 ? make_float2(e.h.y, e.l.y) : (k == 2 ? make_float2(e.h.z, e.l.z) : make_float2(e.h.w, e.l.w));
    z[D.N + v] = df_add(z[D.N + v], ek);
    if (lv == PE) z[v] = df_add(z[v], make_float2(e.h.x, e.l.x));
}

// ------------------------------------------- device-side FGMRES (K-cycle)
// Small Krylov kernels whose scalars stay in device memory, so the level-1
// K-cycle needs no host round trip.  Basis vectors FP32, dot products with
// FP32 products and FP64 block sums.
__global__ void __launch_bounds__(RED_THREADS)
k_kdot(const float* __restrict__ V, int64_t stride, int cnt, const float* __restrict__ w, int64_t n,
       double* partials) {
    pdl_entry();
    float acc32[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc32[j] = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float wi = w[i];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (j < cnt) acc32[j] = fmaf(V[j * stride + i], wi, acc32[j]);
    }
    block_reduce_store_f32<8>(acc32, partials);
}

// w += sign * sum_j h[j] V_j (h on the device; converted once per block)
__global__ void k_kupdate(const float* __restrict__ V, int64_t stride, int cnt, const double* __restrict__ h,
                          float sign, float* __restrict__ w, int64_t n) {
    pdl_entry();
    __shared__ float hs[KCYC_MAX + 1];
    if (threadIdx.x < cnt) hs[threadIdx.x] = (float)h[threadIdx.x];
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float acc = 0.f;
    for (int j = 0; j < cnt; ++j) acc = fmaf(hs[j], V[j * stride + i], acc);
    w[i] = fmaf(sign, acc, w[i]);
}

// The two passes of classical Gram-Schmidt fused with the products that
// follow them: w -= sum_j h[j] V_j (as k_kupdate), then the block partials of
// the updated w against V_j, j < cnt (the second pass's coefficients) or, NORM,
// against itself.  Same grid and summation order as k_kdot, so the results
// equal the unfused sequence bit for bit.  cnt <= 8.
template <bool NORM>
__global__ void __launch_bounds__(RED_THREADS)
k_kupd_dot(const float* __restrict__ V, int64_t stride, int cnt, const double* __restrict__ h,
           float* __restrict__ w, int64_t n, double* partials) {
    pdl_entry();
    constexpr int K = NORM ? 1 : 8;
    __shared__ float hs[8];
    if (threadIdx.x < cnt) hs[threadIdx.x] = (float)h[threadIdx.x];
    __syncthreads();
    float acc32[K];
#pragma unroll
    for (int j = 0; j < K; ++j) acc32[j] = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float v[8];
        float a = 0.f;
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (j < cnt) {
                v[j] = V[j * stride + i];
                a = fmaf(hs[j], v[j], a);
            }
        const float wi = fmaf(-1.f, a, w[i]);
        w[i] = wi;
        if (NORM) {
            acc32[0] = fmaf(wi, wi, acc32[0]);
        } else {
#pragma unroll
            for (int j = 0; j < K; ++j)
                if (j < cnt) acc32[j] = fmaf(v[j], wi, acc32[j]);
        }
    }
    block_reduce_store_f32<K>(acc32, partials);
}

// out = a / sqrt(max(d2, tiny)) (the scale computed once per block)
__global__ void k_knormalize(const float* __restrict__ a, const double* __restrict__ d2, float* __restrict__ out,
                             int64_t n) {
    pdl_entry();
    __shared__ float inv;
    if (threadIdx.x == 0) inv = (float)(1.0 / sqrt(fmax(*d2, 1e-300)));
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = a[i] * inv;
}

// H layout: col-major (KCYC_MAX+1) x KCYC_MAX at H[j*(KCYC_MAX+1) + i]
// After CGS2 of column j: h = h1 + h2, H[j+1, j] = ||w||.
__global__ void k_kcol(double* H, int j, const double* h1, const double* h2, const double* wn2) {
    pdl_entry();
    int i = threadIdx.x;
    if (i <= j) H[j * (KCYC_MAX + 1) + i] = h1[i] + h2[i];
    if (i == 0) H[j * (KCYC_MAX + 1) + j + 1] = sqrt(fmax(*wn2, 0.0));
}

// least squares min || beta e1 - H y || by Givens rotations (one thread);
// y also written as float-float pairs for the combination kernel
__global__ void k_klsq(const double* H, const double* b2, int k, double* y, float2* ydf) {
    pdl_entry();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double R[KCYC_MAX + 1][KCYC_MAX];
    double g[KCYC_MAX + 1];
    for (int j = 0; j < k; ++j)
        for (int i = 0; i <= k; ++i) R[i][j] = H[j * (KCYC_MAX + 1) + i];
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
    for (int i = 0; i < k; ++i) ydf[i] = df_from_double(y[i]);
}

// x = sum_j y_j Z_j in float-float arithmetic
__global__ void k_kcombine(const DF4* __restrict__ Z, int64_t cells, int k, const float2* __restrict__ ydf,
                           DF4* __restrict__ x) {
    pdl_entry();
    int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= cells) return;
    float2 a0 = make_float2(0.f, 0.f), a1 = a0, a2 = a0, a3 = a0;
    for (int j = 0; j < k; ++j) {
        const float2 yj = ydf[j];
        const DF4 z = Z[j * cells + cell];
        a0 = df_add(a0, df_mul(make_float2(z.h.x, z.l.x), yj));
        a1 = df_add(a1, df_mul(make_float2(z.h.y, z.l.y), yj));
        a2 = df_add(a2, df_mul(make_float2(z.h.z, z.l.z), yj));
        a3 = df_add(a3, df_mul(make_float2(z.h.w, z.l.w), yj));
    }
    x[cell] = df4_pack(a0, a1, a2, a3);
}

// ------------------------------------------------------------ host side
int precond_create(mb_cell* c) {
    Precond* p = new Precond();
    c->pc = p;
    const Dims& D = c->D;
    p->dinv = (float*)cell_alloc(c, 16 * D.N);
    p->fc = (float*)cell_alloc(c, 4 * FCW * (D.F ? D.F : 1));
    p->rv = (float*)cell_alloc(c, 8 * D.N);
    p->t = (float*)cell_alloc(c, 8 * D.N);
    p->b16 = c->opt.mg_bf16 != 0;
    {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || p->nsm < 1)
            return cuda_fail(cudaGetLastError(), "multiprocessor count");
        if (cudaFuncSetAttribute(k_lvl_smooth_staged, cudaFuncAttributeMaxDynamicSharedMemorySize, SW_SMEM) !=
            cudaSuccess)
            return cuda_fail(cudaGetLastError(), "staged sweep shared memory");
        if (cudaFuncSetAttribute(k_coarse_invert_smem, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 8 * (CINV_SMEM_MAX * CINV_SMEM_MAX + CINV_SMEM_MAX)) != cudaSuccess)
            return cuda_fail(cudaGetLastError(), "coarse inverse shared memory");
        int nb[3] = {0, 0, 0};
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb[0], k_lvl_smooth<true>, 256, 0) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb[1], k_lvl_smooth2<true>, 256, 0) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb[2], k_lvl_matvec<true>, 256, 0) != cudaSuccess)
            return cuda_fail(cudaGetLastError(), "occupancy");
        for (int k = 0; k < 3; ++k) p->pf[k] = (nb[k] > 0 ? nb[k] : 1) * p->nsm;
    }
    p->err = (int*)cell_alloc(c, 16);
    if (!p->err) return MB_ENOMEM;
    MB_CUDA(cudaMemsetAsync(p->err, 0, 16, c->stream));
    p->fst = cell_alloc(c, (p->b16 ? 4 : 8) * (size_t)FSTK * D.N);
    p->zs = (float2*)cell_alloc(c, 16 * (size_t)D.N);
    if (!p->fst || !p->zs) return MB_ENOMEM;
    c->rowdiag = (float*)cell_alloc(c, 4 * c->n);
    c->rowinv = (float*)cell_alloc(c, 4 * c->n);
    if (!p->dinv || !p->fc || !p->rv || !p->t || !c->rowdiag || !c->rowinv) return MB_ENOMEM;
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
        L.exd = (float*)cell_alloc(c, 4 * (size_t)L.cells * BLK);
        L.aself = (float*)cell_alloc(c, 4 * (size_t)L.cells * BLK);
        L.sinv = (float*)cell_alloc(c, 4 * (size_t)L.cells * BLK);
        L.mask = (uint8_t*)cell_alloc(c, (size_t)L.cells);
        L.x = (DF4*)cell_alloc(c, sizeof(DF4) * (size_t)L.cells);
        L.x2 = (DF4*)cell_alloc(c, sizeof(DF4) * (size_t)L.cells);
        L.b = (float4*)cell_alloc(c, 16 * (size_t)L.cells);
        L.pst = (L.cells + SWT - 1) / SWT * SWT;
        L.pk = (uint2*)cell_alloc(c, 8 * 32 * (size_t)L.pst);
        if (!L.off || !L.ex || !L.exd || !L.aself || !L.sinv || !L.mask || !L.x || !L.x2 || !L.b || !L.pk)
            return MB_ENOMEM;
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
    p->kV = (float*)cell_alloc(c, 4 * (size_t)m4 * (KCYC_MAX + 1));
    p->kZ = (DF4*)cell_alloc(c, sizeof(DF4) * (size_t)p->lv[1].cells * KCYC_MAX);
    p->kw = (float*)cell_alloc(c, 4 * (size_t)m4);
    p->kH = (double*)cell_alloc(c, 8 * (size_t)((KCYC_MAX + 1) * KCYC_MAX + 128));
    p->kred = (double*)cell_alloc(c, 8 * (size_t)RED_BLOCKS * 8);
    if (!p->cdense || !p->cinv || !p->cstat || !p->kV || !p->kZ || !p->kw || !p->kH || !p->kred) return MB_ENOMEM;
    // persistent coarse tail: from the first level >= max(2, mg_tail) that
    // one block of TAIL_THREADS threads per SM covers; its grid is one block per
    // TAIL_THREADS cells of that level (all co-resident), so a small cell's
    // tail is a single block and does not wait for the whole GPU
    p->tbar = (unsigned*)cell_alloc(c, 16);
    if (!p->tbar) return MB_ENOMEM;
    p->tail_l0 = 0;
    if (c->opt.mg_tail && p->b16 && p->nlev >= 3) {
        int dev = 0, coop = 0, occ = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_vtail, TAIL_THREADS, 0) != cudaSuccess)
            return cuda_fail(cudaGetLastError(), "coarse tail occupancy");
        if (coop && occ >= 1) {
            const int64_t cap = (int64_t)p->nsm * TAIL_THREADS;
            for (int l = c->opt.mg_tail > 2 ? c->opt.mg_tail : 2; l < p->nlev; ++l)
                if (p->lv[l].cells <= cap) {
                    p->tail_l0 = l;
                    p->tail_blocks = (int)((p->lv[l].cells + TAIL_THREADS - 1) / TAIL_THREADS);
                    break;
                }
        }
    }
    return MB_OK;
}

static void graph_free(PcGraph& G) {
    if (G.exec) cudaGraphExecDestroy(G.exec);
    for (auto& e : G.ev) {
        cudaEventDestroy(e.e0);
        cudaEventDestroy(e.e1);
    }
    G.exec = nullptr;
    G.ev.clear();
}

void precond_destroy(mb_cell* c) {
    if (c->pc)
        for (auto& G : c->pc->graphs) graph_free(G);
    delete c->pc;
    c->pc = nullptr;
}

int precond_setup(mb_cell* c, const float* u32, const uint8_t* gate, double dt) {
    Precond* p = c->pc;
    p->kcyc = c->opt.mg_kcycle < 1 ? 1 : (c->opt.mg_kcycle > KCYC_MAX ? KCYC_MAX : c->opt.mg_kcycle);
    p->nu_fine = c->opt.mg_smooth < 1 ? 1 : (c->opt.mg_smooth > 8 ? 8 : c->opt.mg_smooth);
    const Dims& D = c->D;
    cudaStream_t s = c->stream;
    (void)gate;
    const SetupScal ss = setup_scal(c->Pf, dt);
    k_bj_setup<<<pgrid(D.nt, D.ny, D.nz), PB, 0, s>>>(c->Pf, D, c->vcode, c->zperm, u32, c->icoef, ss, p->dinv, p->fc,
                                                       c->rowdiag, c->rowinv), ::mb::count_launch(c);
    Level& L1 = p->lv[1];
    k_assemble_l1<<<(unsigned)((L1.cells + 127) / 128), 128, 0, s>>>(c->Pf, D, c->vcode, u32, c->icoef, dt, L1),
        ::mb::count_launch(c);
    for (int l = 2; l <= p->nlev; ++l)
        k_assemble_up<<<nblk(p->lv[l].cells), 256, 0, s>>>(p->lv[l - 1], p->lv[l]), ::mb::count_launch(c);
    for (int l = 1; l <= p->nlev; ++l) k_finalize<<<nblk(p->lv[l].cells), 256, 0, s>>>(p->lv[l]), ::mb::count_launch(c);
    int n = p->ncoarse;
    Level& Lc = p->lv[p->nlev];
    k_coarse_dense<<<(n + 127) / 128, 128, 0, s>>>(Lc, n, p->cdense), ::mb::count_launch(c);
    MB_CUDA(cudaMemsetAsync(p->cstat, 0, 4, s));
    if (n <= CINV_SMEM_MAX)
        k_coarse_invert_smem<<<1, CINV_THREADS, (size_t)8 * (n * n + n), s>>>(n, p->cdense, p->cinv, p->cstat);
    else
        k_coarse_invert<<<1, 256, 0, s>>>(n, p->cdense, p->cinv, p->cstat);
    ::mb::count_launch(c);
    MB_CUDA_LAUNCH("precond_setup");
    return MB_OK;
}

// launch of a kernel of the application: plain, or (mg_pdl) with programmatic
// stream serialization; every kernel launched through here starts with pdl_entry()
template <typename... KArgs, typename... Args>
static void klaunch(const mb_cell* c, void (*k)(KArgs...), dim3 g, dim3 b, size_t smem, cudaStream_t s,
                    Args... args) {
    if (!c->opt.mg_pdl) {
        k<<<g, b, smem, s>>>(args...);
        return;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = g;
    cfg.blockDim = b;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k, args...);
}

// launches of the level kernels with the operator storage chosen at set-up
static void lvl_smooth(mb_cell* c, Level& L, const DF4* xin, const DF4* ec, int ccny, int ccnz, DF4* xout,
                       bool timed = false) {
    cudaStream_t s = c->stream;
    unsigned g = nblk(L.cells);
    cudaEvent_t ev = nullptr;
    timed = timed && (xin || ec);
    if (timed) prof_begin(c, s, &ev);
    const Precond* p = c->pc;
    const int64_t ntiles = (L.cells + SWT - 1) / SWT;
    if (p->b16 && c->opt.mg_stream == 2 && xin && ntiles >= p->nsm && !g_staged_broken.load())
        k_lvl_smooth_staged<<<p->nsm, SWT, SW_SMEM, s>>>(L, xin, ec, ccny, ccnz, OMEGA_COARSE, xout, p->err);
    else if (p->b16 && c->opt.mg_stream == 3 && &L == &p->lv[1])
        // always a plain launch (the kernel has no programmatic-launch entry: it
        // starts after its predecessor completes, and a programmatically launched
        // successor waits for its completion)
        k_lvl_smooth_o5<<<g, 256, 0, s>>>(L, xin, ec, ccny, ccnz, OMEGA_COARSE, xout);
    else if (p->b16)
        klaunch(c, k_lvl_smooth<true>, g, 256, 0, s, L, xin, ec, ccny, ccnz, OMEGA_COARSE, xout,
                c->opt.mg_stream == 1 ? p->pf[0] : 0);
    else
        klaunch(c, k_lvl_smooth<false>, g, 256, 0, s, L, xin, ec, ccny, ccnz, OMEGA_COARSE, xout, 0);
    ::mb::count_launch(c);
    if (timed) prof_end(c, s, PROF_LSMOOTH, ev);
}
static void lvl_smooth2(mb_cell* c, Level& L, DF4* xout) {
    cudaStream_t s = c->stream;
    unsigned g = nblk(L.cells);
    if (c->pc->b16)
        klaunch(c, k_lvl_smooth2<true>, g, 256, 0, s, L, OMEGA_COARSE, xout, c->opt.mg_stream == 1 ? c->pc->pf[1] : 0);
    else
        klaunch(c, k_lvl_smooth2<false>, g, 256, 0, s, L, OMEGA_COARSE, xout, 0);
    ::mb::count_launch(c);
}
static void lvl_restrict(mb_cell* c, Level& L, const DF4* x, Level& C) {
    cudaStream_t s = c->stream;
    unsigned g = nblk(8 * C.cells);
    if (c->pc->b16)
        klaunch(c, k_lvl_restrict<true>, g, 256, 0, s, L, x, C);
    else
        klaunch(c, k_lvl_restrict<false>, g, 256, 0, s, L, x, C);
    ::mb::count_launch(c);
}
static void lvl_matvec(mb_cell* c, Level& L, const DF4* x, float* y) {
    cudaStream_t s = c->stream;
    unsigned g = nblk(L.cells);
    if (c->pc->b16)
        klaunch(c, k_lvl_matvec<true>, g, 256, 0, s, L, x, reinterpret_cast<float4*>(y),
                                             c->opt.mg_stream == 1 ? c->pc->pf[2] : 0);
    else
        klaunch(c, k_lvl_matvec<false>, g, 256, 0, s, L, x, reinterpret_cast<float4*>(y), 0);
    ::mb::count_launch(c);
}

// the V-cycle on levels tail_l0..nlev as one cooperative launch (k_vtail)
static void launch_tail(mb_cell* c) {
    Precond* p = c->pc;
    cudaStream_t s = c->stream;
    TailArgs a;
    memset(&a, 0, sizeof(a));
    a.l0 = p->tail_l0;
    a.nlev = p->nlev;
    a.nu_pre = c->opt.mg_coarse_pre;
    a.nu_post = c->opt.mg_coarse_post;
    a.ncoarse = p->ncoarse;
    a.cinv = p->cinv;
    a.bar = p->tbar;
    a.err = p->err;
    for (int l = a.l0; l <= p->nlev; ++l) {
        const Level& L = p->lv[l];
        a.lv[l] = TailLv{L.nt, L.ny, L.nz, L.cells, L.pst, L.pk, L.b, L.x, L.x2};
    }
    cudaMemsetAsync(p->tbar, 0, 8, s);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)p->tail_blocks);
    cfg.blockDim = dim3(TAIL_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_vtail, a);
    ::mb::count_launch(c);
    // the kernel alternates each level's iterates as the per-level sequence does
    const int swaps = (c->opt.mg_coarse_pre > 2 ? c->opt.mg_coarse_pre - 2 : 0) + c->opt.mg_coarse_post;
    if (swaps & 1)
        for (int l = a.l0; l < p->nlev; ++l) std::swap(p->lv[l].x, p->lv[l].x2);
}

// V-cycle on levels l..nlev with right-hand side lv[l].b; result in lv[l].x
static void vcycle(mb_cell* c, int l) {
    Precond* p = c->pc;
    cudaStream_t s = c->stream;
    if (p->tail_l0 && l == p->tail_l0 && !g_tail_broken.load()) {
        launch_tail(c);
        return;
    }
    Level& L = p->lv[l];
    if (l == p->nlev) {
        klaunch(c, k_coarse_solve, (unsigned)((p->ncoarse + CS_ROWS - 1) / CS_ROWS), 256, 0, s, p->ncoarse, p->cinv, L.b, L.x),
            ::mb::count_launch(c);
        return;
    }
    Level& C = p->lv[l + 1];
    const bool timed = l == 1;
    const int nu_pre = c->opt.mg_coarse_pre, nu_post = c->opt.mg_coarse_post;
    // pre-smoothing from zero; the first two sweeps fused
    if (nu_pre >= 2)
        lvl_smooth2(c, L, L.x);
    else
        lvl_smooth(c, L, nullptr, nullptr, 0, 0, L.x);
    for (int k = 2; k < nu_pre; ++k) {
        lvl_smooth(c, L, L.x, nullptr, 0, 0, L.x2);
        std::swap(L.x, L.x2);
    }
    lvl_restrict(c, L, L.x, C);
    vcycle(c, l + 1);
    // post-smoothing, the first sweep applied to x + P e
    lvl_smooth(c, L, L.x, C.x, C.ny, C.nz, L.x2, timed);
    std::swap(L.x, L.x2);
    for (int k = 1; k < nu_post; ++k) {
        lvl_smooth(c, L, L.x, nullptr, 0, 0, L.x2, timed);
        std::swap(L.x, L.x2);
    }
}

static void kdots(mb_cell* c, const float* V, int64_t stride, int cnt, const float* w, int64_t n, double* out) {
    Precond* p = c->pc;
    cudaStream_t s = c->stream;
    for (int j0 = 0; j0 < cnt; j0 += 8) {
        int k = cnt - j0 < 8 ? cnt - j0 : 8;
        klaunch(c, k_kdot, RED_BLOCKS, RED_THREADS, 0, s, V + j0 * stride, stride, k, w, n, p->kred), ::mb::count_launch(c);
        klaunch(c, k_reduce_final<false>, k, RED_THREADS, 0, s, p->kred, k, out + j0), ::mb::count_launch(c);
    }
}

// Level-1 K-cycle: kcyc iterations of FGMRES on A1 x = b1 (b1 = lv[1].b),
// preconditioned by the V-cycle; result in lv[1].x.  No host synchronisation.
static void kcycle_l1(mb_cell* c) {
    Precond* p = c->pc;
    cudaStream_t s = c->stream;
    Level& L = p->lv[1];
    if (p->nlev == 1) {
        vcycle(c, 1);
        return;
    }
    const int K = p->kcyc;
    const int64_t m4 = 4 * L.cells;
    const unsigned g = nblk(m4);
    double* H = p->kH;
    // scalars: [0] ||b||^2, [8..] h1, [24..] h2, [40] ||w||^2, [48..] y, [64..] y as float-float pairs
    double* sc = p->kH + (KCYC_MAX + 1) * KCYC_MAX;
    double* b2 = sc;
    double* h1 = sc + 8;
    double* h2 = sc + 24;
    double* wn2 = sc + 40;
    double* y = sc + 48;
    float2* ydf = reinterpret_cast<float2*>(sc + 64);
    const float* b = reinterpret_cast<const float*>(L.b);
    kdots(c, b, 0, 1, b, m4, b2);
    klaunch(c, k_knormalize, g, 256, 0, s, b, b2, p->kV, m4), ::mb::count_launch(c);
    float4* bsave = L.b;   // the V-cycle reads lv[1].b: point it at the Krylov vector
    // with an even number of iterate swaps in the V-cycle the result lands in
    // the buffer level 1's x pointed at when it began: point it at Z_j directly
    const int nswap = std::max(c->opt.mg_coarse_pre - 2, 0) + c->opt.mg_coarse_post;
    for (int j = 0; j < K; ++j) {
        float* Vj = p->kV + j * m4;
        DF4* Zj = p->kZ + j * L.cells;
        L.b = reinterpret_cast<float4*>(Vj);
        if (nswap % 2 == 0) {
            DF4* const x0 = L.x;
            L.x = Zj;
            vcycle(c, 1);
            L.x = x0;
        } else {
            vcycle(c, 1);
            cudaMemcpyAsync(Zj, L.x, sizeof(DF4) * L.cells, cudaMemcpyDeviceToDevice, s);
        }
        lvl_matvec(c, L, Zj, p->kw);
        kdots(c, p->kV, m4, j + 1, p->kw, m4, h1);
        if (!c->opt.mg_kcycle_reorth && j + 1 <= 8) {
            // one classical Gram-Schmidt pass, fused with the norm that follows it
            cudaMemsetAsync(h2, 0, 8 * (size_t)(j + 1), s);
            klaunch(c, k_kupd_dot<true>, RED_BLOCKS, RED_THREADS, 0, s, p->kV, m4, j + 1, h1, p->kw, m4, p->kred),
                ::mb::count_launch(c);
            klaunch(c, k_reduce_final<false>, 1, RED_THREADS, 0, s, p->kred, 1, wn2), ::mb::count_launch(c);
        } else if (j + 1 <= 8) {
            // CGS2 with each update fused into the products that follow it
            klaunch(c, k_kupd_dot<false>, RED_BLOCKS, RED_THREADS, 0, s, p->kV, m4, j + 1, h1, p->kw, m4, p->kred),
                ::mb::count_launch(c);
            klaunch(c, k_reduce_final<false>, j + 1, RED_THREADS, 0, s, p->kred, j + 1, h2), ::mb::count_launch(c);
            klaunch(c, k_kupd_dot<true>, RED_BLOCKS, RED_THREADS, 0, s, p->kV, m4, j + 1, h2, p->kw, m4, p->kred),
                ::mb::count_launch(c);
            klaunch(c, k_reduce_final<false>, 1, RED_THREADS, 0, s, p->kred, 1, wn2), ::mb::count_launch(c);
        } else {
            klaunch(c, k_kupdate, g, 256, 0, s, p->kV, m4, j + 1, h1, -1.f, p->kw, m4), ::mb::count_launch(c);
            kdots(c, p->kV, m4, j + 1, p->kw, m4, h2);
            klaunch(c, k_kupdate, g, 256, 0, s, p->kV, m4, j + 1, h2, -1.f, p->kw, m4), ::mb::count_launch(c);
            kdots(c, p->kw, 0, 1, p->kw, m4, wn2);
        }
        klaunch(c, k_kcol, 1, 32, 0, s, H, j, h1, h2, wn2), ::mb::count_launch(c);
        klaunch(c, k_knormalize, g, 256, 0, s, p->kw, wn2, p->kV + (j + 1) * m4, m4), ::mb::count_launch(c);
    }
    L.b = bsave;
    klaunch(c, k_klsq, 1, 1, 0, s, H, b2, K, y, ydf), ::mb::count_launch(c);
    klaunch(c, k_kcombine, nblk(L.cells), 256, 0, s, p->kZ, L.cells, K, ydf, L.x), ::mb::count_launch(c);
}

// ---- MB_DEBUG >= 2: 2-norms of the intermediate vectors of one application
template <class T>
__device__ inline double dbg_sq(T a) { return (double)a * (double)a; }
template <>
__device__ inline double dbg_sq<float2>(float2 a) { double v = df_to_double(a); return v * v; }

template <class T>
__global__ void __launch_bounds__(RED_THREADS) k_sumsq(const T* __restrict__ a, int64_t n, double* partials) {
    double acc[1] = {0.0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc[0] += dbg_sq<T>(a[i]);
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

// the kernel sequence of one application (stream-ordered, no host synchronisation
// unless MB_DEBUG >= 2)
// fine stencil launches with the storage chosen at creation
static void fine_sweep(mb_cell* c, const float2* zin, float2* zout) {
    Precond* p = c->pc;
    const Dims& D = c->D;
    cudaStream_t s = c->stream;
    const dim3 vg = pgrid(D.nt, D.ny, D.nz);
    cudaEvent_t ev;
    prof_begin(c, s, &ev);
    if (p->b16)
        klaunch(c, k_fine_stencil<true, true>, vg, PB, 0, s, D, p->fst, p->dinv, p->rv, zin, OMEGA_FINE, zout, nullptr);
    else
        klaunch(c, k_fine_stencil<false, true>, vg, PB, 0, s, D, p->fst, p->dinv, p->rv, zin, OMEGA_FINE, zout, nullptr);
    ::mb::count_launch(c);
    prof_end(c, s, PROF_SMOOTH, ev);
}
static void fine_product(mb_cell* c, const float2* zin, float* tout) {
    Precond* p = c->pc;
    const Dims& D = c->D;
    cudaStream_t s = c->stream;
    const dim3 vg = pgrid(D.nt, D.ny, D.nz);
    if (p->b16)
        klaunch(c, k_fine_stencil<true, false>, vg, PB, 0, s, D, p->fst, nullptr, nullptr, zin, 0.f, nullptr, tout);
    else
        klaunch(c, k_fine_stencil<false, false>, vg, PB, 0, s, D, p->fst, nullptr, nullptr, zin, 0.f, nullptr, tout);
    ::mb::count_launch(c);
}

int precond_check(mb_cell* c) {
    Precond* p = c->pc;
    int h = 0;
    MB_CUDA(cudaMemcpyAsync(&h, p->err, 4, cudaMemcpyDeviceToHost, c->stream));
    MB_CUDA(cudaStreamSynchronize(c->stream));
    if (h) {
        MB_CUDA(cudaMemsetAsync(p->err, 0, 4, c->stream));
        if (h & 6) {
            // a staged sweep could not drain its copies, or a persistent tail gave up
            // at a grid barrier: never launch that kernel again in this process; the
            // graphs that contain it are captured anew
            if (h & 2) g_staged_broken.store(true);
            if (h & 4) g_tail_broken.store(true);
            for (auto& G : p->graphs) graph_free(G);
            p->graphs.clear();
            p->pending = -1;
        }
        set_error("preconditioner: a bounded wait for staged operator data gave up");
        return MB_ETIMEOUT;
    }
    return MB_OK;
}

int precond_setup_fine(mb_cell* c) {
    Precond* p = c->pc;
    const Dims& D = c->D;
    cudaStream_t s = c->stream;
    const dim3 vg = pgrid(D.nt, D.ny, D.nz);
    if (p->b16)
        k_assemble_fine<true><<<vg, PB, 0, s>>>(c->Pf, D, c->vcode, c->zperm, c->u32, c->icoef, c->d_dtinv, p->fst);
    else
        k_assemble_fine<false><<<vg, PB, 0, s>>>(c->Pf, D, c->vcode, c->zperm, c->u32, c->icoef, c->d_dtinv, p->fst);
    ::mb::count_launch(c);
    MB_CUDA_LAUNCH("precond_setup_fine");
    return MB_OK;
}

static int apply_body(mb_cell* c, const float* r, float2* z) {
    Precond* p = c->pc;
    const Dims& D = c->D;
    cudaStream_t s = c->stream;
    if (debug_level() >= 2)
        fprintf(stderr, "[mb-pc] levels %d coarse n %d |r| %.3e |rowdiag| %.3e\n", p->nlev, p->ncoarse,
                dbg_norm(c, r, c->n), dbg_norm(c, c->rowdiag, c->n));
    const dim3 vg = pgrid(D.nt, D.ny, D.nz);
    const unsigned fg = nblk(D.F ? D.F : 1);
    // condensed right-hand side, then nu_fine damped block-Jacobi sweeps from
    // zero; the sweeps alternate between zs and z, and the first one (from
    // zero) writes where the last one must end up in z
    klaunch(c, k_condense_rhs, vg, PB, 0, s, D, c->vcode, p->fc, r, c->rowdiag, p->rv), ::mb::count_launch(c);
    float2* za = (p->nu_fine - 1) % 2 == 0 ? z : p->zs;
    float2* zb = za == z ? p->zs : z;
    klaunch(c, k_bj_apply, nblk(D.N), 256, 0, s, D, p->dinv, p->rv, nullptr, OMEGA_FINE, false, za), ::mb::count_launch(c);
    for (int k = 1; k < p->nu_fine; ++k) {
        fine_sweep(c, za, zb);
        std::swap(za, zb);
    }
    // t = S z for the restricted residual
    fine_product(c, z, p->t);
    Level& L1 = p->lv[1];
    klaunch(c, k_restrict_fine, nblk(L1.cells), 256, 0, s, D, c->vcode, p->rv, p->t, L1), ::mb::count_launch(c);
    if (debug_level() >= 2)
        fprintf(stderr, "[mb-pc] |rv| %.3e |z0| %.3e |Sz0| %.3e |b1| %.3e\n", dbg_norm(c, p->rv, 2 * D.N),
                dbg_norm(c, z, 2 * D.N), dbg_norm(c, p->t, 2 * D.N),
                dbg_norm(c, reinterpret_cast<const float*>(L1.b), 4 * L1.cells));
    kcycle_l1(c);
    if (debug_level() >= 2) {
        lvl_matvec(c, L1, L1.x, p->kw);
        fprintf(stderr, "[mb-pc] |x1| %.3e |A1 x1| %.3e\n",
                dbg_norm(c, reinterpret_cast<const float2*>(L1.x), 4 * L1.cells), dbg_norm(c, p->kw, 4 * L1.cells));
    }
    klaunch(c, k_prolong_fine, vg, PB, 0, s, D, c->vcode, L1, L1.x, z), ::mb::count_launch(c);
    // nu_fine post-smoothing sweeps (they remove the jumps of the piecewise-constant prolongation)
    za = z;
    zb = p->zs;
    for (int k = 0; k < p->nu_fine; ++k) {
        fine_sweep(c, za, zb);
        std::swap(za, zb);
    }
    if (za != z) MB_CUDA(cudaMemcpyAsync(z, za, 16 * (size_t)D.N, cudaMemcpyDeviceToDevice, s));
    // back-substitution of the plating rows
    if (D.F) klaunch(c, k_face_solve, fg, 256, 0, s, D, c->pf_g, c->pf_e, p->fc, r, c->rowdiag, z), ::mb::count_launch(c);
    if (debug_level() >= 2) fprintf(stderr, "[mb-pc] |z| %.3e\n", dbg_norm(c, z, c->n));
    MB_CUDA_LAUNCH("precond_apply");
    return MB_OK;
}

void precond_harvest(mb_cell* c) {
    Precond* p = c->pc;
    if (!p || p->pending < 0) return;
    PcGraph& G = p->graphs[p->pending];
    p->pending = -1;
    if (G.ev.empty()) return;
    bool ok = cudaEventSynchronize(G.ev.back().e1) == cudaSuccess;
    for (size_t k = 0; ok && k < G.ev.size(); ++k) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, G.ev[k].e0, G.ev[k].e1) == cudaSuccess) {
            c->prof.acc_ms[G.ev[k].kind] += ms;
            c->prof.acc_n[G.ev[k].kind] += 1;
        }
    }
    // a failed timing query must not surface as the error of a later launch
    cudaGetLastError();
}

// capture the application for (r, z) into a new graph; false if capture is not possible
static bool capture_graph(mb_cell* c, const float* r, float2* z, PcGraph& G) {
    Precond* p = c->pc;
    cudaStream_t s = c->stream;
    G.r = r;
    G.z = z;
    G.kcyc = p->kcyc;
    G.nu = p->nu_fine;
    G.reorth = c->opt.mg_kcycle_reorth;
    G.tail = c->opt.mg_tail;
    G.pdl = c->opt.mg_pdl;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const int64_t saved = c->launches;
    c->prof.capture = &G.ev;
    int rc = apply_body(c, r, z);
    c->prof.capture = nullptr;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &g);
    G.nodes = c->launches - saved;
    c->launches = saved;
    bool ok = rc == MB_OK && e == cudaSuccess && g;
    if (ok) ok = cudaGraphInstantiate(&G.exec, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    if (!ok) {
        cudaGetLastError();
        graph_free(G);
    }
    return ok;
}

int precond_apply(mb_cell* c, const float* u32, const uint8_t* gate, double dt, const float* r, float2* z,
                  bool graph) {
    (void)u32; (void)gate; (void)dt;
    Precond* p = c->pc;
    cudaStream_t s = c->stream;
    cudaEvent_t ev_pc;
    if (!graph || p->graphs_off || debug_level() >= 2) {
        prof_begin(c, s, &ev_pc);
        int rc = apply_body(c, r, z);
        prof_end(c, s, PROF_PRECOND, ev_pc);
        return rc;
    }
    precond_harvest(c);
    int idx = -1;
    for (size_t i = 0; i < p->graphs.size(); ++i) {
        const PcGraph& G = p->graphs[i];
        if (G.r == r && G.z == z && G.kcyc == p->kcyc && G.nu == p->nu_fine && G.reorth == c->opt.mg_kcycle_reorth &&
            G.tail == c->opt.mg_tail && G.pdl == c->opt.mg_pdl) {
            idx = (int)i;
            break;
        }
    }
    if (idx < 0) {
        PcGraph G;
        bool ok = capture_graph(c, r, z, G);
        if (!ok && p->tail_l0 && !g_tail_broken.load()) {
            // a cooperative launch that cannot be captured: per-level launches instead
            g_tail_broken.store(true);
            ok = capture_graph(c, r, z, G);
        }
        if (!ok) {
            p->graphs_off = true;
            return precond_apply(c, u32, gate, dt, r, z, false);
        }
        p->graphs.push_back(G);
        idx = (int)p->graphs.size() - 1;
    }
    PcGraph& G = p->graphs[idx];
    prof_begin(c, s, &ev_pc);
    MB_CUDA(cudaGraphLaunch(G.exec, s));
    prof_end(c, s, PROF_PRECOND, ev_pc);
    count_launch(c, (int)G.nodes);
    if (c->prof.enabled && !G.ev.empty()) p->pending = idx;
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

__global__ void k_df_to_double(const float2* __restrict__ a, double* __restrict__ b, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = df_to_double(a[i]);
}

extern "C" {

int mb_debug_precond(mb_cell* c, const double* u, const uint8_t* gate, double dt, const double* r, double* z) {
    if (!c || !u || !r || !z || !(dt > 0)) { set_error("mb_debug_precond: invalid argument"); return MB_EINVAL; }
    int64_t n = c->n, F = c->D.F;
    cudaStream_t s = c->stream;
    double *du = nullptr, *r64 = nullptr, *z64 = nullptr;
    float* r32 = nullptr;
    float2* zdf = nullptr;
    MB_CUDA(cudaMalloc(&du, 8 * n));
    MB_CUDA(cudaMalloc(&r64, 8 * n));
    MB_CUDA(cudaMalloc(&z64, 8 * n));
    MB_CUDA(cudaMalloc(&r32, 4 * n));
    MB_CUDA(cudaMalloc(&zdf, 8 * n));
    MB_CUDA(cudaMemcpyAsync(du, u, 8 * n, cudaMemcpyHostToDevice, s));
    k_cvt<double, float><<<nblk(n), 256, 0, s>>>(du, c->u32, n), ::mb::count_launch(c);
    if (F) MB_CUDA(cudaMemcpyAsync(c->gate2, gate, F, cudaMemcpyHostToDevice, s));
    MB_CUDA(cudaMemcpyAsync(r64, r, 8 * n, cudaMemcpyHostToDevice, s));
    k_cvt<double, float><<<nblk(n), 256, 0, s>>>(r64, r32, n), ::mb::count_launch(c);
    int rc = launch_lin_setup<float>(c, c->u32, c->gate2, s);
    if (!rc) rc = set_dt(c, dt, s);
    if (!rc) rc = precond_setup(c, c->u32, c->gate2, dt);
    if (!rc) rc = precond_setup_fine(c);
    if (!rc) rc = precond_apply(c, c->u32, c->gate2, dt, r32, zdf, false);
    if (!rc) {
        k_df_to_double<<<nblk(n), 256, 0, s>>>(zdf, z64, n), ::mb::count_launch(c);
        cudaMemcpyAsync(z, z64, 8 * n, cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) rc = cuda_fail(cudaGetLastError(), "debug_precond");
    }
    cudaStreamSynchronize(s);
    cudaFree(du); cudaFree(r64); cudaFree(z64); cudaFree(r32); cudaFree(zdf);
    return rc;
}

int mb_debug_residual_split(mb_cell* c, const double* u, const double* u_old, const uint8_t* gate, double dt,
                            double I_app, double* r) {
    if (!c || !u || !u_old || !r || !(dt > 0)) { set_error("mb_debug_residual_split: invalid argument"); return MB_EINVAL; }
    int64_t n = c->n, F = c->D.F;
    cudaStream_t s = c->stream;
    MB_CUDA(cudaMemcpyAsync(c->du, u, 8 * n, cudaMemcpyHostToDevice, s));
    MB_CUDA(cudaMemcpyAsync(c->u_pass, u_old, 8 * n, cudaMemcpyHostToDevice, s));
    if (F) MB_CUDA(cudaMemcpyAsync(c->gate2, gate, F, cudaMemcpyHostToDevice, s));
    int rc = launch_residual_split(c, c->du, c->u_pass, c->gate2, dt, I_app, c->r, s);
    if (rc) return rc;
    MB_CUDA(cudaMemcpyAsync(r, c->r, 8 * n, cudaMemcpyDeviceToHost, s));
    MB_CUDA(cudaStreamSynchronize(s));
    return MB_OK;
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
    // device layout is structure of arrays; the caller gets one record per cell
    std::vector<float> tmp;
    if (aself) {
        tmp.resize((size_t)BLK * L.cells);
        MB_CUDA(cudaMemcpy(tmp.data(), L.aself, 4 * BLK * L.cells, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < L.cells; ++i)
            for (int e = 0; e < BLK; ++e) aself[i * BLK + e] = tmp[(size_t)e * L.cells + i];
    }
    if (off) {
        tmp.resize((size_t)OFFW * L.cells);
        MB_CUDA(cudaMemcpy(tmp.data(), L.off, 4 * OFFW * L.cells, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < L.cells; ++i)
            for (int e = 0; e < OFFW; ++e) off[i * OFFW + e] = tmp[(size_t)e * L.cells + i];
    }
    if (mask) MB_CUDA(cudaMemcpy(mask, L.mask, L.cells, cudaMemcpyDeviceToHost));
    return MB_OK;
}

__global__ void k_fst_to_f32(const uint32_t* __restrict__ a, float2* __restrict__ b, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = make_float2(__uint_as_float(a[i] << 16), __uint_as_float(a[i] & 0xffff0000u));
}

int mb_debug_fine_stencil(mb_cell* c, float* out) {
    if (!c || !out) { set_error("mb_debug_fine_stencil: invalid argument"); return MB_EINVAL; }
    const int64_t m = (int64_t)FSTK * c->D.N;
    if (!c->pc->b16) {
        MB_CUDA(cudaMemcpy(out, c->pc->fst, 8 * m, cudaMemcpyDeviceToHost));
        return MB_OK;
    }
    float2* tmp = nullptr;
    MB_CUDA(cudaMalloc(&tmp, 8 * m));
    k_fst_to_f32<<<nblk(m), 256, 0, c->stream>>>(static_cast<const uint32_t*>(c->pc->fst), tmp, m);
    cudaError_t e = cudaMemcpyAsync(out, tmp, 8 * m, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(e, "debug_fine_stencil");
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
